// dugks_step_static: the T3S3 step without any device allocation.
//
// Who needs this: callers that are not allowed to allocate device memory
// themselves or through this library -- for example a plugin running inside
// an application that owns all device memory through its own pool and
// forbids allocations outside it, or a latency-critical loop that cannot
// afford the implicit device-wide synchronisation that cudaMalloc/cudaFree
// may cause.  They pass the input and output state; every intermediate
// (velocity tables, moments, g, f~', the accumulator, face values) lives in
// one file-scope device array of fixed size, kStaticScratchBytes.
//
// Properties a caller must know:
//   - The array is part of the library's device image: every GPU on which
//     the library's module is loaded holds these kStaticScratchBytes until
//     the process exits.
//   - Its device address is looked up once per device, on the first call
//     made with that device current (cudaGetSymbolAddress); make that first
//     call before any stream capture.
//   - Every call uploads the velocity tables from host vectors that live only
//     for the call, so a call made while its stream is capturing a CUDA graph
//     is refused (DUGKS_EINVAL): a captured copy would point at freed memory.
//   - All calls share the one array and it keeps the last call's contents.
//     Nothing in it needs to start at zero: every intermediate is fully
//     written before it is read within a step.  Calls that overlap on the GPU
//     (on different streams, or from several threads) race on the array and
//     give wrong results; serialise them.
//   - No cudaMalloc, cudaFree or allocating library routine is called.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dugks.h"
#include "dugks_internal.cuh"

using namespace dugks;

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

int sfail(int code, const std::string& m) {
  set_last_error(m);   // read back through dugks_last_error()
  return code;
}

std::mutex s_mu;
void* s_base[kMaxDevices] = {nullptr};

// Device address of g_static_scratch for the current device (set-up on the
// first call per device).
int scratch_base(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sfail(DUGKS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return sfail(DUGKS_EINVAL, "device index beyond the static table");
  std::lock_guard<std::mutex> lk(s_mu);
  if (!s_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return sfail(DUGKS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    s_base[dev] = p;
  }
  *out = s_base[dev];
  return DUGKS_OK;
}

size_t up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

extern "C" int dugks_step_static(const dugks_mesh* mesh, const dugks_velset* vel, double tau,
                                 double dt, const dugks_bc bc[4], const double* fhat_in,
                                 double* fhat_out, int nsteps, void* cuda_stream) {
  if (!mesh || !vel || !bc || !fhat_in || !fhat_out)
    return sfail(DUGKS_EINVAL, "dugks_step_static: NULL argument");
  if (nsteps < 0) return sfail(DUGKS_EINVAL, "dugks_step_static: nsteps must be >= 0");
  const int nx = mesh->nx, ny = mesh->ny, nv = vel->nv;
  if (nx < 1 || ny < 1 || nv < 1 || !vel->xi_x || !vel->xi_y || !vel->w)
    return sfail(DUGKS_EINVAL, "dugks_step_static: empty mesh or velocity set");
  if (!finite_pos(mesh->dx) || !finite_pos(mesh->dy) || !finite_pos(tau) || !finite_pos(dt) ||
      !finite_pos(vel->RT))
    return sfail(DUGKS_EINVAL, "dugks_step_static: dx, dy, tau, dt, RT must be > 0");

  // scratch layout and the size limit (checked before anything touches the GPU)
  const size_t N = (size_t)nx * ny, nvN = (size_t)nv * N;
  const size_t nfx = (size_t)nv * ny * (nx + 1), nfy = (size_t)nv * (ny + 1) * nx;
  const size_t o_vel = 0;
  const size_t o_opp = o_vel + up(7 * (size_t)nv * sizeof(double));
  const size_t o_mom = o_opp + up((size_t)nv * sizeof(int));
  const size_t o_g = o_mom + up(3 * N * sizeof(double));
  const size_t o_ftp = o_g + up(nvN * sizeof(double));
  const size_t o_acc = o_ftp + up(nvN * sizeof(double));
  const size_t o_fbx = o_acc + up(nvN * sizeof(double));
  const size_t o_fby = o_fbx + up(nfx * sizeof(double));
  const size_t need = o_fby + up(nfy * sizeof(double));
  if (N > (size_t)1 << 30 || nvN > ((size_t)1 << 40) || need > kStaticScratchBytes)
    return sfail(DUGKS_EINVAL,
                 "dugks_step_static: problem needs " + std::to_string(need) +
                     " bytes of scratch, more than the fixed " +
                     std::to_string(kStaticScratchBytes) + " (use dugks_init/dugks_step)");

  for (int s = 0; s < 4; ++s)
    if (bc[s].kind < 0 || bc[s].kind > 2 || !std::isfinite(bc[s].uw_x) || !std::isfinite(bc[s].uw_y))
      return sfail(DUGKS_EINVAL, "dugks_step_static: bad boundary");
  const bool px = bc[DUGKS_WEST].kind == DUGKS_BC_PERIODIC;
  const bool py = bc[DUGKS_SOUTH].kind == DUGKS_BC_PERIODIC;
  if (px != (bc[DUGKS_EAST].kind == DUGKS_BC_PERIODIC) ||
      py != (bc[DUGKS_NORTH].kind == DUGKS_BC_PERIODIC))
    return sfail(DUGKS_EINVAL, "dugks_step_static: periodic sides must come in pairs");
  if ((!px && nx < 3) || (!py && ny < 3))
    return sfail(DUGKS_EINVAL, "dugks_step_static: a wall direction needs >= 3 cells");

  // host tables: xi_x, xi_y, w, feq_wall[4]; opposite velocities
  std::vector<double> tab(7 * (size_t)nv, 0.0);
  std::vector<int> opp(nv, -1);
  double vmax = 0.0;
  for (int k = 0; k < nv; ++k) {
    if (!std::isfinite(vel->xi_x[k]) || !std::isfinite(vel->xi_y[k]) || !std::isfinite(vel->w[k]))
      return sfail(DUGKS_EINVAL, "dugks_step_static: non-finite velocity or weight");
    tab[k] = vel->xi_x[k];
    tab[nv + k] = vel->xi_y[k];
    tab[2 * nv + k] = vel->w[k];
    vmax = std::fmax(vmax, std::fabs(vel->xi_x[k]) + std::fabs(vel->xi_y[k]));
  }
  for (int k = 0; k < nv; ++k)
    for (int q = 0; q < nv; ++q)
      if (std::fabs(vel->xi_x[q] + vel->xi_x[k]) + std::fabs(vel->xi_y[q] + vel->xi_y[k]) <=
          1e-12 * (1.0 + vmax)) {
        opp[k] = q;
        break;
      }
  DevParams p{};
  const double invRT = 1.0 / vel->RT;
  for (int s = 0; s < 4; ++s) {
    p.bc_kind[s] = bc[s].kind;
    p.uw_x[s] = bc[s].uw_x;
    p.uw_y[s] = bc[s].uw_y;
    if (bc[s].kind == DUGKS_BC_PERIODIC) continue;
    const double nxs = (s == DUGKS_WEST) ? -1.0 : (s == DUGKS_EAST) ? 1.0 : 0.0;
    const double nys = (s == DUGKS_SOUTH) ? -1.0 : (s == DUGKS_NORTH) ? 1.0 : 0.0;
    double den = 0.0;
    for (int k = 0; k < nv; ++k) {
      const double eu = (vel->xi_x[k] * bc[s].uw_x + vel->xi_y[k] * bc[s].uw_y) * invRT;
      const double uu = (bc[s].uw_x * bc[s].uw_x + bc[s].uw_y * bc[s].uw_y) * invRT;
      const double fw = vel->w[k] * (1.0 + eu + 0.5 * eu * eu - 0.5 * uu);
      tab[(3 + s) * (size_t)nv + k] = fw;
      const double xn = vel->xi_x[k] * nxs + vel->xi_y[k] * nys;
      if (xn < 0.0) {
        den -= xn * fw;
        if (bc[s].kind == DUGKS_BC_BOUNCEBACK && opp[k] < 0)
          return sfail(DUGKS_EINVAL, "dugks_step_static: bounce-back needs -xi_k in the set");
      }
    }
    if (bc[s].kind == DUGKS_BC_DIFFUSE && !(den > 0.0))
      return sfail(DUGKS_EINVAL, "dugks_step_static: diffuse wall without leaving velocities");
    p.ds_den[s] = den;
    if (bc[s].kind == DUGKS_BC_DIFFUSE) p.has_ds = 1;
  }

  // fhat_in and fhat_out: the same array, or two arrays that do not overlap
  {
    const size_t bytes = nvN * sizeof(double);
    const char* a = reinterpret_cast<const char*>(fhat_in);
    const char* b = reinterpret_cast<const char*>(fhat_out);
    if (a != b && a < b + bytes && b < a + bytes)
      return sfail(DUGKS_EINVAL, "dugks_step_static: fhat_in and fhat_out overlap without being equal");
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(st, &cs);
    if (ce != cudaSuccess)
      return sfail(DUGKS_ECUDA, std::string("dugks_step_static: cudaStreamIsCapturing: ") +
                                    cudaGetErrorString(ce));
    if (cs != cudaStreamCaptureStatusNone)
      return sfail(DUGKS_EINVAL,
                   "dugks_step_static: the stream is capturing a graph; this call uploads "
                   "its velocity tables from call-local host memory and cannot be captured");
  }

  void* base_v = nullptr;
  int rc = scratch_base(&base_v);
  if (rc != DUGKS_OK) return rc;
  unsigned char* base = static_cast<unsigned char*>(base_v);
  double* dvel = reinterpret_cast<double*>(base + o_vel);
  int* dopp = reinterpret_cast<int*>(base + o_opp);
  double* mom = reinterpret_cast<double*>(base + o_mom);
  double* g = reinterpret_cast<double*>(base + o_g);
  double* ftp = reinterpret_cast<double*>(base + o_ftp);
  double* acc = reinterpret_cast<double*>(base + o_acc);
  double* fbx = reinterpret_cast<double*>(base + o_fbx);
  double* fby = reinterpret_cast<double*>(base + o_fby);

  cudaError_t e = cudaMemcpyAsync(dvel, tab.data(), tab.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dopp, opp.data(), opp.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && fhat_out != fhat_in)
    e = cudaMemcpyAsync(fhat_out, fhat_in, nvN * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return sfail(DUGKS_ECUDA, std::string("dugks_step_static copy: ") + cudaGetErrorString(e));

  p.nx = nx;
  p.ny = ny;
  p.nv = nv;
  p.N = (int)N;
  p.px = px;
  p.py = py;
  p.dx = mesh->dx;
  p.dy = mesh->dy;
  p.inv_dx = 1.0 / mesh->dx;
  p.inv_dy = 1.0 / mesh->dy;
  p.tau = tau;
  p.dt = dt;
  p.RT = vel->RT;
  p.inv_RT = invRT;
  p.xi_x = dvel;
  p.xi_y = dvel + nv;
  p.w = dvel + 2 * (size_t)nv;
  p.feq_wall = dvel + 3 * (size_t)nv;
  p.opp = dopp;

  // same stage coefficients as dugks_init (Sec. 2.1.3)
  StageCoef s1{}, s2{};
  s1.a = (12.0 * tau - dt) / (12.0 * tau + 3.0 * dt);
  s1.b = 4.0 * dt / (12.0 * tau + 3.0 * dt);
  s1.h = dt / 6.0;
  s2.a = (24.0 * tau - 5.0 * dt) / (24.0 * tau + 4.0 * dt);
  s2.b = 9.0 * dt / (24.0 * tau + 4.0 * dt);
  s2.h = 5.0 * dt / 12.0;
  for (StageCoef* s : {&s1, &s2}) {
    s->alpha = 2.0 * tau / (2.0 * tau + s->h);
    s->beta = s->h / (2.0 * tau + s->h);
  }
  const double c_om = -6.0 * dt / (6.0 * tau + dt);
  const int G = nv <= 32 ? 1 : 8;
  double* f = fhat_out;
  for (int n = 0; n < nsteps && e == cudaSuccess; ++n) {
    e = launch_cell(p, G, 1, f, g, mom, s1.a, s1.b, st);
    if (e == cudaSuccess) e = launch_face(p, G, 0, g, mom, fbx, s1, st);
    if (e == cudaSuccess) e = launch_face(p, G, 1, g, mom, fby, s1, st);
    if (e == cudaSuccess) e = launch_update1(p, f, g, fbx, fby, ftp, acc, st);
    if (e == cudaSuccess) e = launch_cell(p, G, 2, ftp, g, mom, s2.a, s2.b, st);
    if (e == cudaSuccess) e = launch_face(p, G, 0, g, mom, fbx, s2, st);
    if (e == cudaSuccess) e = launch_face(p, G, 1, g, mom, fby, s2, st);
    if (e == cudaSuccess) e = launch_update2(p, ftp, acc, mom, fbx, fby, f, c_om, st);
  }
  if (e != cudaSuccess) return sfail(DUGKS_ECUDA, std::string("dugks_step_static launch: ") + cudaGetErrorString(e));
  return DUGKS_OK;
}
