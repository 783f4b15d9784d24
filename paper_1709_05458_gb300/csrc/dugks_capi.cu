// C-ABI host side of the DUGKS library: validation, device state, launch
// sequencing of the T3S3 step (Sec. 2.1.3 of arXiv:1709.05458), copies and
// launch profiling.  Declarations and argument contracts: include/dugks.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "../../include/dugks.h"
#include "dugks_internal.cuh"

using namespace dugks;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(DUGKS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

const char* kNames[K_NUM] = {
    "cell_stage1", "face_x_stage1", "face_y_stage1", "update_stage1",
    "cell_stage2", "face_x_stage2", "face_y_stage2", "update_stage2",
    "moments",     "set_equilibrium", "check",
    "d2q9_prologue", "d2q9_stage1", "d2q9_stage2",
    "d2q9m_stage1", "d2q9m_stage2", "convert",
    "gdev_cell", "gdev_face_x", "gdev_face_y", "gdev_walls", "gdev_update_stage1",
    "gdev_update_stage2", "t2_cell", "t2_face_x", "t2_face_y", "t2_update",
    "d2q9dw_stage1", "d2q9dw_stage2", "gnc_sums", "gnc_cellfin", "gnc_walls", "gnc_facefin",
    "gnc_update_stage1", "gnc_update_stage2"};

struct Pending {
  int id;
  cudaEvent_t a, b;
};

}  // namespace

void dugks::set_last_error(const std::string& msg) { g_err = msg; }

struct dugks_ctx {
  DevParams p{};
  cudaStream_t stream = nullptr;
  int groups = 1;
  StageCoef s1{}, s2{};
  double c_om = 0.0;            // dt Omega(f') = c_om (f~' - feq'), eq. collisionterm
  // device buffers
  double* fhat = nullptr;       // state f^ [nv][N]
  double* ftp = nullptr;        // f~(t') [nv][N]
  double* acc = nullptr;        // f^+ + 3dt/7 L* [nv][N]
  double* g = nullptr;          // f-bar^{+,h} of the current stage [nv][N]
  double* fbx = nullptr;        // x-face f [nv][ny][nx+1]
  double* fby = nullptr;        // y-face f [nv][ny+1][nx]
  double* mom = nullptr;        // rho, ux, uy [3][N]
  double* mom_aux = nullptr;    // moments written by dugks_get_state(DUGKS_STATE_F) [3][N]
  double* vel = nullptr;        // xi_x, xi_y, w, feq_wall[4]  ([7][nv])
  int* opp = nullptr;           // [nv]
  double* part = nullptr;       // partial face moments of the large-set face kernels
  int nchx = 0, nchy = 0;       // velocity chunks of those kernels (0: not used)
  int* flag = nullptr;          // [1]
  // fused D2Q9 path: buffers fhat = f^, g = g1, ftp = g2, acc = X, mom[0..N) and
  // mom[N..2N) = rho of the two stage base states
  bool d2q9 = false;
  bool g1_valid = false;
  D2Q9Params dp{};
  D2Q9Stage ds1{}, ds2{};
  // DUGKS_F64_DW: the fused D2Q9 kernels in double-word arithmetic on the
  // same FP64 arrays, with the parameters split into FP32 pairs
  bool dwa = false;
  D2Q9ParamsDW dwp{};
  D2Q9StageDW dws1{}, dws2{};
  // deviation storage (store 1 = FP32, 2 = BF16): fhat, g, ftp, acc hold
  // typed deviations d = f - W rho0; fbx is the FP64 staging buffer
  int store = 0;
  double rho0 = 1.0;
  D2Q9StageF df1{}, df2{};
  // deviation storage on the generic path (any velocity set): launch set-up
  // and the FP32 equilibrium parameters of the last cell pass ([5][N])
  bool gdev = false;
  GDevStep gs{};
  void* eqp = nullptr;
  // the class-moment generic path (dugks_gnc.cu), which steps the generic
  // contexts with FP32 / BF16 storage: its step descriptor and the buffers
  // it adds to those above
  bool gnc = false;
  GncStep gn{};
  void* gn_eq2 = nullptr;       // equilibrium parameters at t' [5][N]
  double* gn_mom2 = nullptr;    // rho, u at t' [3][N]
  void* gn_wf = nullptr;        // wall faces' f-bar [nv][nw]
  double* gn_wrho = nullptr;    // wall densities [nw]
  double* gn_sums = nullptr;    // class sums [nsplit][ncls][10][N]
  float* gn_nu = nullptr;       // stencil moments [ncombo][18][N]
  void* gn_tab = nullptr;       // class tables, quadrature and face weights
  void* vf = nullptr;           // velocity table of that path (4-vector rows [3][nv])
  void* gpad = nullptr;         // padded stage field of that path
  void* fpar = nullptr;         // face equilibrium parameters of that path
  double* twt = nullptr;        // FP64 Taylor weight tables of that path
  // time scheme (dugks_set_scheme): 0 T3S3; 1 T2S3, 2 T2S2 on the generic
  // kernels with the T2 stage coefficients below
  int scheme = DUGKS_T3S3;
  StageCoef t2{};               // g = a f~ + b feq, h = dt/2, f = alpha f-bar + beta feq
  double t2a = 0.0, t2b = 0.0;  // f~^+ = t2a f~ + t2b feq
  int batched = 0;              // number of batches holding this context
  cudaEvent_t ev_copy = nullptr;  // end of dugks_set_state's host upload
  // adjoint (allocated on first use): forward intermediates and adjoint fields
  double *a_g1 = nullptr, *a_g2 = nullptr, *a_ftp = nullptr, *a_acc = nullptr;
  double *a_mom1 = nullptr, *a_mom2 = nullptr, *a_tbar = nullptr, *a_gbar = nullptr;
  double *a_lam = nullptr, *a_out = nullptr, *a_phix = nullptr, *a_phiy = nullptr;
  double *a_rhob = nullptr, *a_grads = nullptr;
  double* a_fbs = nullptr;      // forward f-bar of the faces of one direction [nv][nf]
  std::vector<double*> ckpt;    // checkpoint store for dugks_adjoint_run
  // profiling
  bool prof = false;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  long long launches[K_NUM] = {0};
  double ms[K_NUM] = {0.0};

  cudaEvent_t ev() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void drain() {
    for (auto& q : pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess) {
        ms[q.id] += t;
        launches[q.id] += 1;
      }
      pool.push_back(q.a);
      pool.push_back(q.b);
    }
    pending.clear();
  }
};

struct dugks_batch {
  std::vector<dugks_ctx*> ctxs;
  std::vector<dugks_ctx*> own;      // instances run by their own launches
  // the own instances in branches of the captured graph: branch streams,
  // the instances of each branch, fork and join events
  std::vector<cudaStream_t> bstreams;
  std::vector<std::vector<dugks_ctx*>> branches;
  std::vector<cudaEvent_t> bevents;
  std::vector<dugks_ctx*> fused;    // instances of the persistent D2Q9 launch
  // class-moment instances, grouped by storage and tie flag: one batched
  // launch per kernel and stage for each group, in a branch of its own
  std::vector<GncBatch> gnc;
  std::vector<cudaStream_t> gstreams;
  cudaStream_t stream = nullptr;
  D2Q9BatchItem* items = nullptr;   // device
  int* tile_start = nullptr;        // device, nitems + 1
  int* counters = nullptr;          // device, 2
  int nitems = 0, max_ty = 1, blocks = 0;
  std::map<int, cudaGraphExec_t> graphs;
};

namespace {

// Bracket one launch with profiling events when enabled.
template <typename F>
int launch(dugks_ctx* c, int id, F&& f) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (c->prof) {
    if (c->pending.size() > 200000) {  // bound host memory: fold finished ones
      cudaStreamSynchronize(c->stream);
      c->drain();
    }
    a = c->ev();
    b = c->ev();
    cudaEventRecord(a, c->stream);
  }
  cudaError_t e = f();
  if (c->prof) {
    cudaEventRecord(b, c->stream);
    c->pending.push_back({id, a, b});
  }
  if (e != cudaSuccess) return cuda_fail(e, kNames[id]);
  return DUGKS_OK;
}

#define TRY(x)                        \
  do {                                \
    int rc__ = (x);                   \
    if (rc__ != DUGKS_OK) return rc__; \
  } while (0)

int copy_in(dugks_ctx* c, double* dst, const double* src, size_t n, int on_device) {
  cudaError_t e = cudaMemcpyAsync(dst, src, n * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy to device");
  if (!on_device) {  // host buffer may be freed by the caller after return
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy to device");
  }
  return DUGKS_OK;
}

int copy_out(dugks_ctx* c, double* dst, const double* src, size_t n, int on_device) {
  cudaError_t e = cudaMemcpyAsync(dst, src, n * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy from device");
  if (!on_device) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy from device");
  }
  return DUGKS_OK;
}

void free_all(dugks_ctx* c) {
  double* bufs[] = {c->fhat, c->ftp, c->acc, c->g, c->fbx, c->fby, c->mom, c->mom_aux, c->vel, c->part,
                    c->a_g1, c->a_g2, c->a_ftp, c->a_acc, c->a_mom1, c->a_mom2, c->a_tbar,
                    c->a_gbar, c->a_lam, c->a_out, c->a_phix, c->a_phiy, c->a_rhob, c->a_grads,
                    c->a_fbs};
  for (double* b : bufs)
    if (b) cudaFree(b);
  for (double* b : c->ckpt)
    if (b) cudaFree(b);
  if (c->opp) cudaFree(c->opp);
  if (c->flag) cudaFree(c->flag);
  if (c->eqp) cudaFree(c->eqp);
  if (c->vf) cudaFree(c->vf);
  if (c->gpad) cudaFree(c->gpad);
  if (c->fpar) cudaFree(c->fpar);
  if (c->twt) cudaFree(c->twt);
  if (c->gn_eq2) cudaFree(c->gn_eq2);
  if (c->gn_mom2) cudaFree(c->gn_mom2);
  if (c->gn_wf) cudaFree(c->gn_wf);
  if (c->gn_wrho) cudaFree(c->gn_wrho);
  if (c->gn_sums) cudaFree(c->gn_sums);
  if (c->gn_nu) cudaFree(c->gn_nu);
  if (c->gn_tab) cudaFree(c->gn_tab);
  for (auto& q : c->pending) {
    cudaEventDestroy(q.a);
    cudaEventDestroy(q.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  if (c->ev_copy) cudaEventDestroy(c->ev_copy);
}

// Face-value weights about one cell centre for the foot offset (a dx, b dy):
// T[dy+1][dx+1] (eq. flux_DS as printed, central differences).
void taylor_weights(double a, double b, double T[3][3]) {
  double w[9];
  flux_ds_weights<double>(a, b, w);
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) T[r][q] = w[r * 3 + q];
}

// Interface weight tables of one stage (interface step h, flux factor fac).
void d2q9_stage_tables(D2Q9Stage& S, double c, double dx, double dy, double tau, double h,
                       double fac) {
  std::memset(&S, 0, sizeof(S));
  const double alpha = 2 * tau / (2 * tau + h);
  S.gamma = h / (2 * tau);
  for (int k = 0; k < 9; ++k) {
    const int ex = k / 3 - 1, ey = k % 3 - 1;
    const double cx = c * ex, cy = c * ey;
    double TL[3][3], TR[3][3], TB[3][3], TT[3][3];
    taylor_weights((0.5 * dx - cx * h) / dx, (-cy * h) / dy, TL);    // from cell fi-1
    taylor_weights((-0.5 * dx - cx * h) / dx, (-cy * h) / dy, TR);   // from cell fi
    taylor_weights((-cx * h) / dx, (0.5 * dy - cy * h) / dy, TB);    // from cell fj-1
    taylor_weights((-cx * h) / dx, (-0.5 * dy - cy * h) / dy, TT);   // from cell fj
    const double wl = ex > 0 ? 1.0 : (ex < 0 ? 0.0 : 0.5), wr = ex < 0 ? 1.0 : (ex > 0 ? 0.0 : 0.5);
    const double wb = ey > 0 ? 1.0 : (ey < 0 ? 0.0 : 0.5), wt = ey < 0 ? 1.0 : (ey > 0 ? 0.0 : 0.5);
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) {
        S.wx[k][r][q] += wl * TL[r][q];
        S.wx[k][r][q + 1] += wr * TR[r][q];
        S.wy[k][r][q] += wb * TB[r][q];
        S.wy[k][r + 1][q] += wt * TT[r][q];
        S.wxL[k][r][q] = TL[r][q];
        S.wxR[k][r][q] = TR[r][q];
        S.wyB[k][r][q] = TB[r][q];
        S.wyT[k][r][q] = TT[r][q];
      }
    S.kx[k] = -fac * alpha * cx / dx;
    S.ky[k] = -fac * alpha * cy / dy;
  }
}

// Is the velocity set xi_k = c (k/3 - 1, k%3 - 1)?  Returns c (> 0) or 0.
double d2q9_speed(const dugks_velset* v) {
  if (v->nv != 9) return 0.0;
  const double c = v->xi_x[6];
  if (!(c > 0.0)) return 0.0;
  for (int k = 0; k < 9; ++k)
    if (v->xi_x[k] != c * (k / 3 - 1) || v->xi_y[k] != c * (k % 3 - 1)) return 0.0;
  return c;
}

// Tile height of the fused D2Q9 kernels: the height whose tiles finish
// soonest when an SM holds b = min(occ[ty], ceil(tiles / SMs)) blocks at a
// time (a one-wave grid is spread evenly by the launch), at a cost of ty + 1
// face rows per tile scaled by the throughput gained from co-resident
// blocks, which overlap one another's barriers and loads.  FP64 and
// double-word kernels (bound by the FP64 pipe or by issue): 6 % for b >= 2
// (measured at 256^2 and 1024^2 for both arithmetics).  FP32 / BF16
// deviation kernels (latency-bound at 2-3 blocks): b^(-1/4), fitted to
// heights 4..16 at 1024^2, where 7 resident blocks of height 4 ran 17 %
// faster than 2 of height 13.  Ties go to the lower height, or with
// prefer_tall (the issue-bound double-word kernels, which gain from the
// smaller halo share of taller tiles) to the taller one.  occ[ty]: resident
// blocks per SM at height ty.
int d2q9_tile_height(int nx, int ny, int sms, int maxty, bool prefer_tall, const int* occ,
                     bool dev_kernels) {
  int best = 8;
  double bestc = 1e300;
  for (int ty = 4; ty <= maxty; ++ty) {
    const long tiles = (long)((nx + 31) / 32) * ((ny + ty - 1) / ty);
    const long b = std::max(1L, std::min<long>(std::max(1, occ[ty]), (tiles + sms - 1) / sms));
    const long waves = (tiles + sms * b - 1) / (sms * b);
    const double eff = dev_kernels ? std::pow((double)b, -0.25) : (b >= 2 ? 0.94 : 1.0);
    const double cost = (double)waves * b * (ty + 1) * eff;
    if (cost < bestc - 1e-9 || (prefer_tall && cost <= bestc + 1e-9)) {
      bestc = cost;
      best = ty;
    }
  }
  return best;
}

int one_step_d2q9(dugks_ctx* c) {
  cudaStream_t s = c->stream;
  const size_t N = c->p.N;
  if (!c->g1_valid) {
    TRY(launch(c, K_D2Q9_PROLOGUE, [&] {
      return c->dwa ? launch_d2q9dw_cell(c->dwp, c->fhat, c->g, c->mom, s)
                    : launch_d2q9_cell(c->dp, true, c->fhat, c->g, c->mom, s);
    }));
    c->g1_valid = true;
  }
  if (c->dwa) {
    c->dwp.ty = c->dp.ty;                         // the tile height may have been retuned
    TRY(launch(c, K_D2Q9DW_STAGE1, [&] {
      return launch_d2q9dw_stage(c->dwp, c->dws1, 1, c->g, c->fhat, c->mom, c->ftp, c->acc,
                                 c->mom + N, s);
    }));
    TRY(launch(c, K_D2Q9DW_STAGE2, [&] {
      return launch_d2q9dw_stage(c->dwp, c->dws2, 2, c->ftp, c->acc, c->mom + N, c->fhat, c->g,
                                 c->mom, s);
    }));
    return DUGKS_OK;
  }
  TRY(launch(c, K_D2Q9_STAGE1, [&] {
    return launch_d2q9_stage(c->dp, c->ds1, 1, c->g, c->fhat, c->mom, c->ftp, c->acc, c->mom + N, s);
  }));
  TRY(launch(c, K_D2Q9_STAGE2, [&] {
    return launch_d2q9_stage(c->dp, c->ds2, 2, c->ftp, c->acc, c->mom + N, c->fhat, c->g, c->mom, s);
  }));
  return DUGKS_OK;
}

int one_step_d2q9m(dugks_ctx* c) {
  cudaStream_t s = c->stream;
  const size_t N = c->p.N;
  if (!c->g1_valid) {
    TRY(launch(c, K_D2Q9_PROLOGUE, [&] {
      return launch_dev_cell(c->p, c->store, c->rho0, c->fhat, c->g, c->mom, c->s1.a, c->s1.b, 1, s);
    }));
    c->g1_valid = true;
  }
  TRY(launch(c, K_D2Q9M_STAGE1, [&] {
    return launch_d2q9m_stage(c->dp, c->df1, c->store, 1, c->rho0, c->g, c->fhat, c->mom, c->ftp,
                              c->acc, c->mom + N, s);
  }));
  TRY(launch(c, K_D2Q9M_STAGE2, [&] {
    return launch_d2q9m_stage(c->dp, c->df2, c->store, 2, c->rho0, c->ftp, c->acc, c->mom + N,
                              c->fhat, c->g, c->mom, s);
  }));
  return DUGKS_OK;
}

// faces of one direction and stage for the generic path: the large-set
// kernels for interior faces plus the generic kernel for wall faces, or the
// generic kernel for all faces
cudaError_t faces(dugks_ctx* c, int dir, const StageCoef& sc, double* fb) {
  const DevParams& p = c->p;
  const int nch = dir == 0 ? c->nchx : c->nchy;
  if (!nch) return launch_face(p, c->groups, dir, c->g, c->mom, fb, sc, c->stream);
  cudaError_t e = launch_nc_faces(p, dir, c->g, fb, c->part, nch, sc, c->stream);
  if (e == cudaSuccess && !(dir == 0 ? p.px : p.py))
    e = launch_face(p, c->groups, dir, c->g, c->mom, fb, sc, c->stream, 1);
  return e;
}

int one_step(dugks_ctx* c) {
  const DevParams& p = c->p;
  cudaStream_t s = c->stream;
  const int G = c->groups;
  // Step (1): moments of f^, g1 = f-bar^{+,dt/6}; faces at t*; L*; Step (2): f~(t')
  TRY(launch(c, K_CELL_STAGE1, [&] { return launch_cell(p, G, 1, c->fhat, c->g, c->mom, c->s1.a, c->s1.b, s); }));
  TRY(launch(c, K_FACE_X_STAGE1, [&] { return faces(c, 0, c->s1, c->fbx); }));
  TRY(launch(c, K_FACE_Y_STAGE1, [&] { return faces(c, 1, c->s1, c->fby); }));
  TRY(launch(c, K_UPDATE_STAGE1, [&] { return launch_update1(p, c->fhat, c->g, c->fbx, c->fby, c->ftp, c->acc, s); }));
  // Step (2) collision at t' and Step (3): g2 = f-bar^{+,5dt/12}(t'); faces at t**; Step (4)
  TRY(launch(c, K_CELL_STAGE2, [&] { return launch_cell(p, G, 2, c->ftp, c->g, c->mom, c->s2.a, c->s2.b, s); }));
  TRY(launch(c, K_FACE_X_STAGE2, [&] { return faces(c, 0, c->s2, c->fbx); }));
  TRY(launch(c, K_FACE_Y_STAGE2, [&] { return faces(c, 1, c->s2, c->fby); }));
  TRY(launch(c, K_UPDATE_STAGE2, [&] { return launch_update2(p, c->ftp, c->acc, c->mom, c->fbx, c->fby, c->fhat, c->c_om, s); }));
  return DUGKS_OK;
}

// Deviation storage on the generic path: the same eight launch groups as
// one_step, FP32/BF16 arrays, FP64 moment sums.
int one_step_gdev(dugks_ctx* c) {
  const GDevStep& g = c->gs;
  cudaStream_t s = c->stream;
  for (int stage = 1; stage <= 2; ++stage) {
    TRY(launch(c, K_GDEV_CELL, [&] { return launch_gdev_cell(g, stage, s); }));
    TRY(launch(c, K_GDEV_FACE_X, [&] { return launch_gdev_faces(g, stage, 0, s); }));
    TRY(launch(c, K_GDEV_FACE_Y, [&] { return launch_gdev_faces(g, stage, 1, s); }));
    TRY(launch(c, K_GDEV_WALLS, [&] { return launch_gdev_walls(g, stage, s); }));
    TRY(launch(c, stage == 1 ? K_GDEV_UPDATE1 : K_GDEV_UPDATE2,
               [&] { return launch_gdev_update(g, stage, s); }));
  }
  return DUGKS_OK;
}

// The class-moment generic path: per stage the class sums of the source,
// the cell and face finalisers, the wall faces and the update.
int one_step_gnc(dugks_ctx* c) {
  const GncStep& g = c->gn;
  cudaStream_t s = c->stream;
  const bool walls = !(c->p.px && c->p.py);
  for (int stage = 1; stage <= 2; ++stage) {
    TRY(launch(c, K_GNC_SUMS, [&] { return launch_gnc_sums(g, stage, s); }));
    TRY(launch(c, K_GNC_CELLFIN, [&] { return launch_gnc_cellfin(g, stage, s); }));
    TRY(launch(c, K_GNC_FACEFIN, [&] { return launch_gnc_facefin(g, stage, s); }));
    if (walls) TRY(launch(c, K_GNC_WALLS, [&] { return launch_gnc_walls(g, stage, s); }));
    TRY(launch(c, stage == 1 ? K_GNC_UPDATE1 : K_GNC_UPDATE2,
               [&] { return launch_gnc_update(g, stage, s); }));
  }
  return DUGKS_OK;
}

// rho, u of the current f^ into c->mom on the class-moment path
int gnc_moments(dugks_ctx* c) {
  TRY(launch(c, K_GNC_SUMS, [&] { return launch_gnc_sums(c->gn, 1, c->stream); }));
  TRY(launch(c, K_GNC_CELLFIN, [&] { return launch_gnc_cellfin(c->gn, 1, c->stream); }));
  return DUGKS_OK;
}

// One T2 step of size dt (Remark I, eq. feqIntD2nd_Explicit with Q7) on the
// generic kernels: g = f-bar^{+,dt/2} from f~, faces at t_n + dt/2 with the
// quadratic (T2S3) or first-order (T2S2) expansion, f~^{n+1} = f~^+ + dt L.
int one_step_t2(dugks_ctx* c) {
  const DevParams& p = c->p;
  cudaStream_t s = c->stream;
  const int G = c->groups;
  TRY(launch(c, K_T2_CELL, [&] { return launch_cell(p, G, 1, c->fhat, c->g, c->mom, c->t2.a, c->t2.b, s); }));
  TRY(launch(c, K_T2_FACE_X, [&] { return faces(c, 0, c->t2, c->fbx); }));
  TRY(launch(c, K_T2_FACE_Y, [&] { return faces(c, 1, c->t2, c->fby); }));
  TRY(launch(c, K_T2_UPDATE, [&] { return launch_update_t2(p, c->mom, c->fbx, c->fby, c->fhat, c->t2a, c->t2b, s); }));
  return DUGKS_OK;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

int advance(dugks_ctx* c) {
  if (c->scheme != DUGKS_T3S3) return one_step_t2(c);
  if (c->gnc) return one_step_gnc(c);
  if (c->gdev) return one_step_gdev(c);
  if (c->store) return one_step_d2q9m(c);
  return c->d2q9 ? one_step_d2q9(c) : one_step(c);
}

// g1 of the current state for the fused paths (run eagerly before capture)
int ensure_g1(dugks_ctx* c) {
  if (c->gnc) return DUGKS_OK;                     // every step starts from the sums
  if (!c->d2q9 || c->g1_valid) return DUGKS_OK;
  cudaStream_t s = c->stream;
  if (c->store)
    TRY(launch(c, K_D2Q9_PROLOGUE, [&] {
      return launch_dev_cell(c->p, c->store, c->rho0, c->fhat, c->g, c->mom, c->s1.a, c->s1.b, 1, s);
    }));
  else
    TRY(launch(c, K_D2Q9_PROLOGUE, [&] {
      return c->dwa ? launch_d2q9dw_cell(c->dwp, c->fhat, c->g, c->mom, s)
                    : launch_d2q9_cell(c->dp, true, c->fhat, c->g, c->mom, s);
    }));
  c->g1_valid = true;
  return DUGKS_OK;
}

int ensure_adjoint(dugks_ctx* c) {
  if (c->a_grads) return DUGKS_OK;
  const size_t nvN = (size_t)c->p.nv * c->p.N, N = c->p.N;
  const size_t nfx = (size_t)c->p.nv * c->p.ny * (c->p.nx + 1);
  const size_t nfy = (size_t)c->p.nv * (c->p.ny + 1) * c->p.nx;
  cudaError_t e = cudaSuccess;
  auto al = [&](double** p, size_t n) {
    if (e == cudaSuccess) e = cudaMalloc((void**)p, n * sizeof(double));
  };
  al(&c->a_g1, nvN); al(&c->a_g2, nvN); al(&c->a_ftp, nvN); al(&c->a_acc, nvN);
  al(&c->a_mom1, 3 * N); al(&c->a_mom2, 3 * N); al(&c->a_tbar, nvN); al(&c->a_gbar, nvN);
  al(&c->a_lam, nvN); al(&c->a_out, nvN); al(&c->a_phix, nfx); al(&c->a_phiy, nfy);
  al(&c->a_rhob, N); al(&c->a_grads, 16); al(&c->a_fbs, std::max(nfx, nfy));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? DUGKS_ENOMEM : DUGKS_ECUDA,
                std::string("adjoint buffers: ") + cudaGetErrorString(e));
  }
  return DUGKS_OK;
}

#define CK(x)                                       \
  do {                                              \
    cudaError_t e__ = (x);                          \
    if (e__ != cudaSuccess) return cuda_fail(e__, "adjoint"); \
  } while (0)

// Adjoint of one T3S3 step taken from the current state c->fhat:
// a_lam = lambda^{n+1} in, a_out = lambda^n out, a_grads[0..8] += parameter
// adjoints.  Forward intermediates are recomputed by the generic kernels.
int adjoint_core(dugks_ctx* c) {
  const DevParams& p = c->p;
  cudaStream_t s = c->stream;
  const int G = c->groups;
  const size_t nvN = (size_t)p.nv * p.N;
  const double tau = p.tau, dt = p.dt;
  // forward recomputation: g1 and the moments of f^, f~(t') (the fused
  // stage-1 kernel for D2Q9 sets, else the face and update kernels), g2 and
  // the moments of f~(t')
  CK(launch_cell(p, G, 1, c->fhat, c->a_g1, c->a_mom1, c->s1.a, c->s1.b, s));
  if (c->d2q9) {
    CK(launch_d2q9_ftp(c->dp, c->ds1, c->a_g1, c->fhat, c->a_mom1, c->a_g2, c->a_ftp,
                       c->a_mom2, s));
  } else {
    CK(launch_face(p, G, 0, c->a_g1, c->a_mom1, c->fbx, c->s1, s));
    CK(launch_face(p, G, 1, c->a_g1, c->a_mom1, c->fby, c->s1, s));
    CK(launch_update1(p, c->fhat, c->a_g1, c->fbx, c->fby, c->a_ftp, c->a_acc, s));
  }
  CK(launch_cell(p, G, 2, c->a_ftp, c->a_g2, c->a_mom2, c->s2.a, c->s2.b, s));
  // tau-derivatives of the coefficients
  const double c34 = 0.75 * c->c_om;
  const double da1 = 48.0 * dt / ((12 * tau + 3 * dt) * (12 * tau + 3 * dt));
  const double da2 = 216.0 * dt / ((24 * tau + 4 * dt) * (24 * tau + 4 * dt));
  const double dc = 27.0 * dt / ((6 * tau + dt) * (6 * tau + dt));
  const double dal1 = 2 * c->s1.h / ((2 * tau + c->s1.h) * (2 * tau + c->s1.h));
  const double dal2 = 2 * c->s2.h / ((2 * tau + c->s2.h) * (2 * tau + c->s2.h));
  const size_t N = p.N;
  // stage 2: f^^{n+1} = X + c (f~' - feq') + 4dt/7 L**
  CK(launch_axpby(nvN, c->a_lam, c34, nullptr, 0.0, c->a_tbar, s));
  CK(launch_flux_T(p, 0, c->a_lam, 4.0 * dt / 7.0, nullptr, 0.0, c->a_phix, s));
  CK(launch_flux_T(p, 1, c->a_lam, 4.0 * dt / 7.0, nullptr, 0.0, c->a_phiy, s));
  CK(cudaMemsetAsync(c->a_gbar, 0, nvN * sizeof(double), s));
  CK(cudaMemsetAsync(c->a_rhob, 0, N * sizeof(double), s));
  CK(launch_face_T(p, 0, c->a_g2, c->a_mom2, c->a_phix, c->a_gbar, c->a_rhob, c->a_grads, c->s2, dal2, c->a_fbs, s));
  CK(launch_face_T(p, 1, c->a_g2, c->a_mom2, c->a_phiy, c->a_gbar, c->a_rhob, c->a_grads, c->s2, dal2, c->a_fbs, s));
  CK(launch_cell_T(p, c->a_ftp, c->a_gbar, c->a_lam, c->a_rhob, c->a_tbar, c->s2.a, c->s2.b, c34,
                   da2, dc, c->a_grads, s));
  // stage 1: f~' = 5/4 g1 - 1/4 f^ + dt/3 L*,  X = 1/4 f^ + 3/4 g1 + 3dt/7 L*
  CK(launch_axpby(nvN, c->a_tbar, 1.25, c->a_lam, 0.75, c->a_gbar, s));
  CK(launch_axpby(nvN, c->a_tbar, -0.25, c->a_lam, 0.25, c->a_out, s));
  CK(launch_flux_T(p, 0, c->a_tbar, dt / 3.0, c->a_lam, 3.0 * dt / 7.0, c->a_phix, s));
  CK(launch_flux_T(p, 1, c->a_tbar, dt / 3.0, c->a_lam, 3.0 * dt / 7.0, c->a_phiy, s));
  CK(cudaMemsetAsync(c->a_rhob, 0, N * sizeof(double), s));
  CK(launch_face_T(p, 0, c->a_g1, c->a_mom1, c->a_phix, c->a_gbar, c->a_rhob, c->a_grads, c->s1, dal1, c->a_fbs, s));
  CK(launch_face_T(p, 1, c->a_g1, c->a_mom1, c->a_phiy, c->a_gbar, c->a_rhob, c->a_grads, c->s1, dal1, c->a_fbs, s));
  CK(launch_cell_T(p, c->fhat, c->a_gbar, nullptr, c->a_rhob, c->a_out, c->s1.a, c->s1.b, 0.0,
                   da1, 0.0, c->a_grads, s));
  return DUGKS_OK;
}

int read_grads(dugks_ctx* c, double* dJ_dtau, double* dJ_duw) {
  double h[9];
  cudaError_t e = cudaMemcpyAsync(h, c->a_grads, 9 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint gradients");
  if (dJ_dtau) *dJ_dtau += h[0];
  if (dJ_duw)
    for (int i = 0; i < 8; ++i) dJ_duw[i] += h[1 + i];
  return DUGKS_OK;
}

}  // namespace

extern "C" {

const char* dugks_last_error(void) { return g_err.c_str(); }

const char* dugks_kernel_name(int id) {
  return (id >= 0 && id < K_NUM) ? kNames[id] : "";
}

int dugks_init(const dugks_mesh* mesh, const dugks_velset* vel, double tau, double dt,
               const dugks_bc bc[4], int storage, void* cuda_stream, dugks_ctx** out) {
  return dugks_init_ex(mesh, vel, tau, dt, bc, storage, DUGKS_PATH_AUTO, cuda_stream, out);
}

int dugks_init_ex(const dugks_mesh* mesh, const dugks_velset* vel, double tau, double dt,
                  const dugks_bc bc[4], int storage, int path, void* cuda_stream, dugks_ctx** out) {
  g_err.clear();
  if (!out) return fail(DUGKS_EINVAL, "out is NULL");
  *out = nullptr;
  if (path < DUGKS_PATH_AUTO || path > DUGKS_PATH_REFERENCE) return fail(DUGKS_EINVAL, "unknown kernel path");
  if (path == DUGKS_PATH_REFERENCE && storage != DUGKS_FP64)
    return fail(DUGKS_ENOTIMPL, "the reference kernels store FP64");
  if (!mesh || !vel || !bc) return fail(DUGKS_EINVAL, "NULL mesh, velocity set or bc");
  if (storage < DUGKS_FP64 || storage > DUGKS_F64_DW) return fail(DUGKS_ENOTIMPL, "unknown storage form");
  if (mesh->nx < 1 || mesh->ny < 1) return fail(DUGKS_EINVAL, "nx, ny must be >= 1");
  if ((long long)mesh->nx * mesh->ny > (1LL << 31) - 1)
    return fail(DUGKS_EINVAL, "too many cells");
  if (!finite_pos(mesh->dx) || !finite_pos(mesh->dy)) return fail(DUGKS_EINVAL, "dx, dy must be > 0");
  if (!finite_pos(tau) || !finite_pos(dt)) return fail(DUGKS_EINVAL, "tau, dt must be > 0 and finite");
  const int nv = vel->nv;
  if (nv < 1 || !vel->xi_x || !vel->xi_y || !vel->w) return fail(DUGKS_EINVAL, "empty velocity set");
  if (!finite_pos(vel->RT)) return fail(DUGKS_EINVAL, "RT must be > 0");
  if ((long long)nv * mesh->nx * mesh->ny * 8LL > (1LL << 40))
    return fail(DUGKS_EINVAL, "state larger than 1 TiB");
  for (int k = 0; k < nv; ++k)
    if (!std::isfinite(vel->xi_x[k]) || !std::isfinite(vel->xi_y[k]) || !std::isfinite(vel->w[k]))
      return fail(DUGKS_EINVAL, "non-finite velocity or weight");
  // double-word arithmetic: FP64 arrays, taken by the fused D2Q9 kernels only
  const bool dwa = storage == DUGKS_F64_DW;
  if (dwa) {
    if (!(d2q9_speed(vel) > 0.0) || path != DUGKS_PATH_AUTO)
      return fail(DUGKS_ENOTIMPL, "double-word arithmetic runs on the fused D2Q9 kernels only");
    storage = DUGKS_FP64;
  }
  for (int s = 0; s < 4; ++s) {
    if (bc[s].kind < 0 || bc[s].kind > 2) return fail(DUGKS_EINVAL, "unknown boundary kind");
    if (!std::isfinite(bc[s].uw_x) || !std::isfinite(bc[s].uw_y))
      return fail(DUGKS_EINVAL, "non-finite wall velocity");
  }
  const bool px = bc[DUGKS_WEST].kind == DUGKS_BC_PERIODIC;
  const bool py = bc[DUGKS_SOUTH].kind == DUGKS_BC_PERIODIC;
  if (px != (bc[DUGKS_EAST].kind == DUGKS_BC_PERIODIC))
    return fail(DUGKS_EINVAL, "west and east must both be periodic or both walls");
  if (py != (bc[DUGKS_NORTH].kind == DUGKS_BC_PERIODIC))
    return fail(DUGKS_EINVAL, "south and north must both be periodic or both walls");
  if (!px && mesh->nx < 3) return fail(DUGKS_EINVAL, "walls in x need nx >= 3");
  if (!py && mesh->ny < 3) return fail(DUGKS_EINVAL, "walls in y need ny >= 3");

  // opposite velocities (bounce-back) and wall equilibria (diffuse)
  std::vector<int> opp(nv, -1);
  double vmax = 0.0;
  for (int k = 0; k < nv; ++k) vmax = std::fmax(vmax, std::fabs(vel->xi_x[k]) + std::fabs(vel->xi_y[k]));
  for (int k = 0; k < nv; ++k)
    for (int q = 0; q < nv; ++q)
      if (std::fabs(vel->xi_x[q] + vel->xi_x[k]) + std::fabs(vel->xi_y[q] + vel->xi_y[k]) <=
          1e-12 * (1.0 + vmax)) {
        opp[k] = q;
        break;
      }
  std::vector<double> host(7 * (size_t)nv, 0.0);
  for (int k = 0; k < nv; ++k) {
    host[k] = vel->xi_x[k];
    host[nv + k] = vel->xi_y[k];
    host[2 * nv + k] = vel->w[k];
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
    int nout = 0;
    for (int k = 0; k < nv; ++k) {
      const double eu = (vel->xi_x[k] * bc[s].uw_x + vel->xi_y[k] * bc[s].uw_y) * invRT;
      const double uu = (bc[s].uw_x * bc[s].uw_x + bc[s].uw_y * bc[s].uw_y) * invRT;
      const double fw = vel->w[k] * (1.0 + eu + 0.5 * eu * eu - 0.5 * uu);
      host[(3 + s) * (size_t)nv + k] = fw;
      const double xn = vel->xi_x[k] * nxs + vel->xi_y[k] * nys;
      if (xn < 0.0) {
        ++nout;
        den -= xn * fw;
        if (bc[s].kind == DUGKS_BC_BOUNCEBACK && opp[k] < 0)
          return fail(DUGKS_EINVAL, "bounce-back needs -xi_k in the velocity set");
      }
    }
    if (bc[s].kind == DUGKS_BC_DIFFUSE && (nout == 0 || !(den > 0.0)))
      return fail(DUGKS_EINVAL, "diffuse wall without velocities leaving it");
    p.ds_den[s] = den;
    if (bc[s].kind == DUGKS_BC_DIFFUSE) p.has_ds = 1;
  }

  dugks_ctx* c = new dugks_ctx();
  c->stream = (cudaStream_t)cuda_stream;
  c->groups = nv <= 32 ? 1 : 8;
  p.nx = mesh->nx;
  p.ny = mesh->ny;
  p.nv = nv;
  p.N = mesh->nx * mesh->ny;
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

  const size_t nvN = (size_t)nv * p.N;
  const size_t nfx = (size_t)nv * p.ny * (p.nx + 1), nfy = (size_t)nv * (p.ny + 1) * p.nx;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](double** ptr, size_t n) {
    if (e == cudaSuccess) e = cudaMalloc((void**)ptr, n * sizeof(double));
  };
  alloc(&c->fhat, nvN);
  alloc(&c->ftp, nvN);
  alloc(&c->acc, nvN);
  alloc(&c->g, nvN);
  alloc(&c->fbx, nfx);
  alloc(&c->fby, nfy);
  alloc(&c->mom, 3 * (size_t)p.N);
  alloc(&c->mom_aux, 3 * (size_t)p.N);
  if (c->groups > 1) {          // large velocity sets: interior-face kernels of dugks_nc.cu
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->nchx = nc_chunks(p, 0, sms);
    c->nchy = nc_chunks(p, 1, sms);
    const size_t nfmax = std::max((size_t)p.ny * (p.nx + 1), (size_t)(p.ny + 1) * p.nx);
    alloc(&c->part, (size_t)std::max(c->nchx, c->nchy) * 3 * nfmax);
  }
  alloc(&c->vel, host.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->opp, nv * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->flag, sizeof(int));
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? DUGKS_ENOMEM : DUGKS_ECUDA,
                std::string("device allocation: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpy(c->vel, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->opp, opp.data(), nv * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->fhat, 0, nvN * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    return cuda_fail(e, "dugks_init");
  }
  p.xi_x = c->vel;
  p.xi_y = c->vel + nv;
  p.w = c->vel + 2 * (size_t)nv;
  p.feq_wall = c->vel + 3 * (size_t)nv;
  p.opp = c->opp;
  c->p = p;

  // Stage coefficients (Sec. 2.1.3; readings in the oracle's header):
  //   g1 = ((12 tau - dt) f^ + 4 dt feq) / (12 tau + 3 dt)          eq. f_bar_1_6
  //   g2 = ((24 tau - 5 dt) f~' + 9 dt feq') / (24 tau + 4 dt)      eq. fbp_5_12 (derived form)
  //   f  = (2 tau f-bar + h feq) / (2 tau + h)                     eq. recover2f
  //   dt Omega' = -6 dt / (6 tau + dt) (f~' - feq')                eq. collisionterm
  const double T = tau;
  c->s1.a = (12.0 * T - dt) / (12.0 * T + 3.0 * dt);
  c->s1.b = 4.0 * dt / (12.0 * T + 3.0 * dt);
  c->s1.h = dt / 6.0;
  c->s2.a = (24.0 * T - 5.0 * dt) / (24.0 * T + 4.0 * dt);
  c->s2.b = 9.0 * dt / (24.0 * T + 4.0 * dt);
  c->s2.h = 5.0 * dt / 12.0;
  for (StageCoef* s : {&c->s1, &c->s2}) {
    s->alpha = 2.0 * T / (2.0 * T + s->h);
    s->beta = s->h / (2.0 * T + s->h);
  }
  c->c_om = -6.0 * dt / (6.0 * T + dt);
  // T2 schemes (Remark I): h = dt/2; f-bar^{+,h} from f~ = f - dt/2 Omega
  // (the same map as the oracle's t2_step), f~^+ = ((2 tau - dt) f~ +
  // 2 dt feq)/(2 tau + dt)
  c->t2.h = 0.5 * dt;
  c->t2.a = (2.0 * T - c->t2.h) / (2.0 * T + 2.0 * c->t2.h);
  c->t2.b = 3.0 * c->t2.h / (2.0 * T + 2.0 * c->t2.h);
  c->t2.alpha = 2.0 * T / (2.0 * T + c->t2.h);
  c->t2.beta = c->t2.h / (2.0 * T + c->t2.h);
  c->t2a = (2.0 * T - dt) / (2.0 * T + dt);
  c->t2b = 2.0 * dt / (2.0 * T + dt);

  // fused D2Q9 path
  const double cd = d2q9_speed(vel);
  const bool forced = path != DUGKS_PATH_AUTO;
  // The optimised generic kernels (dugks_generic_mixed.cu for FP64,
  // dugks_gnc.cu for the deviation forms) step every context that the fused
  // D2Q9 kernels do not take: any velocity set, any storage.
  // DUGKS_PATH_REFERENCE keeps an FP64 context on the reference kernels
  // (dugks_kernels.cu, dugks_nc.cu), which also run the T2 schemes, the
  // adjoint's recomputation and the allocation-free entry.
  const bool generic = !(cd > 0.0 && !forced);
  if (generic && path != DUGKS_PATH_REFERENCE) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool f64 = storage == DUGKS_FP64;
    const double rho0 = f64 ? 0.0 : c->rho0;         // FP64: the arrays hold f itself
    const size_t csz = f64 ? sizeof(double) : sizeof(float);   // compute type
    GDevStep& g = c->gs;
    g.p = c->p;
    g.store = storage;
    g.ref.rho0 = rho0;
    for (int k = 0; k < nv; ++k) {
      g.ref.W += rho0 * vel->w[k];
      g.ref.Wx += rho0 * vel->w[k] * vel->xi_x[k];
      g.ref.Wy += rho0 * vel->w[k] * vel->xi_y[k];
    }
    for (int sd = 0; sd < 4; ++sd) {     // outgoing flux of the reference state per wall
      const double nxs = sd == DUGKS_WEST ? -1.0 : sd == DUGKS_EAST ? 1.0 : 0.0;
      const double nys = sd == DUGKS_SOUTH ? -1.0 : sd == DUGKS_NORTH ? 1.0 : 0.0;
      double o = 0.0;
      for (int k = 0; k < nv; ++k) {
        const double xn = vel->xi_x[k] * nxs + vel->xi_y[k] * nys;
        if (xn > 0.0) o += xn * vel->w[k];
      }
      g.ds_out[sd] = rho0 * o;
    }
    g.s1 = c->s1;
    g.s2 = c->s2;
    g.c_om = c->c_om;
    {   // tensor velocity grid with xi_x constant over runs of n >= 16 (n % 16 == 0)
      int n = 0;
      while ((long long)(n + 1) * (n + 1) <= nv) ++n;
      bool tg = n * n == nv && n % 16 == 0;
      for (int k = 0; tg && k < nv; ++k)
        tg = vel->xi_x[k] == vel->xi_x[(k / n) * n] && vel->xi_y[k] == vel->xi_y[k % n];
      g.tgrid = tg ? 1 : 0;
    }
    // the FP64 generic kernels (dugks_generic_mixed.cu); the deviation forms
    // take the class-moment kernels (below) and share this descriptor's
    // tables and buffers
    if (f64) {
      e = gdev_prepare(storage);
      g.nchx = gdev_chunks(p, 0, sms, storage);
      g.nchy = gdev_chunks(p, 1, sms, storage);
    } else {
      g.nchx = g.nchy = 1;
    }
    g.mch = nv > 32 ? 4 : 1;
    // partial moments: this path's face and cell passes and (FP64) the
    // first generic kernels share one buffer, used at different times
    if (c->part) {
      cudaFree(c->part);
      c->part = nullptr;
    }
    const size_t nfmax = std::max((size_t)p.ny * (p.nx + 1), (size_t)(p.ny + 1) * p.nx);
    const int pch = std::max(std::max(std::max(g.nchx, g.nchy), g.mch), std::max(c->nchx, c->nchy));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->part, (size_t)pch * 3 * nfmax * sizeof(double));
    g.pitch = gdev_pitch(p.nx);
    g.plane = (size_t)(p.ny + 4) * g.pitch;
    // The deviation forms take the class-moment path (below): one streaming
    // pass per stage for the moments, and an update that forms g and the
    // face values on chip, about 24 bytes of the stored type per update and
    // bound by instruction issue.  FP64 storage is bound by the 2-lane FP64
    // pipe instead, and keeps the kernels of dugks_generic_mixed.cu, which
    // store g and the face values but need about 160 FP64 flops per update.
    const bool use_gnc = !f64;
    if (e == cudaSuccess && !use_gnc) e = cudaMalloc(&c->gpad, g.plane * nv * csz);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->eqp, 5 * (size_t)p.N * csz);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->fpar, 5 * 2 * nfmax * csz);
    // velocity table in the compute type, 4-vector rows [3][nv]:
    // (xi_x hi, lo, xi_y hi, lo), (xi_x, xi_y, W_k, 0), flux factors (below);
    // FP32: hi = xi rounded to FP32, lo = the FP32 rounding of the remainder;
    // FP64: hi = xi, lo = 0
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->vf, 12 * (size_t)nv * csz);
    if (e == cudaSuccess) {
      std::vector<double> t(12 * (size_t)nv, 0.0);
      for (int k = 0; k < nv; ++k) {
        const double x = vel->xi_x[k], y = vel->xi_y[k];
        const double xh = f64 ? x : (double)(float)x, yh = f64 ? y : (double)(float)y;
        double* r0 = t.data() + 4 * (size_t)k;
        double* r1 = t.data() + 4 * ((size_t)nv + k);
        double* r2 = t.data() + 4 * (2 * (size_t)nv + k);
        r0[0] = xh;
        r0[1] = x - xh;
        r0[2] = yh;
        r0[3] = y - yh;
        r1[0] = xh;
        r1[1] = yh;
        r1[2] = vel->w[k];
        // flux factors of the two stages: -(dt/3) alpha_1 xi/dx and
        // -(4 dt/7) alpha_2 xi/dx (x and y)
        r2[0] = -(dt / 3.0) * c->s1.alpha * x / mesh->dx;
        r2[1] = -(dt / 3.0) * c->s1.alpha * y / mesh->dy;
        r2[2] = -(4.0 * dt / 7.0) * c->s2.alpha * x / mesh->dx;
        r2[3] = -(4.0 * dt / 7.0) * c->s2.alpha * y / mesh->dy;
      }
      if (f64) {
        e = cudaMemcpy(c->vf, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice);
      } else {
        std::vector<float> tf(t.begin(), t.end());
        e = cudaMemcpy(c->vf, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice);
      }
    }
    // FP64: the face-value weights of the upwind expansions per stage,
    // direction and velocity (lower cell, upper cell), central differences
    // on the 3x3 neighbourhood, foot offset (a dx, b dy) (eq. flux_DS)
    if (e == cudaSuccess && f64) {
      std::vector<double> w(4 * (size_t)nv * 18);
      auto taylor = [](double a, double b, double* T) {
        double w[9];
        flux_ds_weights<double>(a, b, w);
        for (int q = 0; q < 9; ++q) T[q] = w[q];
      };
      for (int st = 0; st < 2; ++st) {
        const double h = st == 0 ? c->s1.h : c->s2.h;
        for (int dir = 0; dir < 2; ++dir)
          for (int k = 0; k < nv; ++k) {
            const double x = vel->xi_x[k], y = vel->xi_y[k];
            double* T = w.data() + ((size_t)(2 * st + dir) * nv + k) * 18;
            if (dir == 0) {
              taylor((0.5 * p.dx - x * h) * p.inv_dx, -y * h * p.inv_dy, T);
              taylor((-0.5 * p.dx - x * h) * p.inv_dx, -y * h * p.inv_dy, T + 9);
            } else {
              taylor(-x * h * p.inv_dx, (0.5 * p.dy - y * h) * p.inv_dy, T);
              taylor(-x * h * p.inv_dx, (-0.5 * p.dy - y * h) * p.inv_dy, T + 9);
            }
          }
      }
      e = cudaMalloc((void**)&c->twt, w.size() * sizeof(double));
      if (e == cudaSuccess)
        e = cudaMemcpy(c->twt, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      free_all(c);
      delete c;
      cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? DUGKS_ENOMEM : DUGKS_ECUDA,
                  std::string("generic path set-up: ") + cudaGetErrorString(e));
    }
    g.tw = c->twt;
    g.fhat = c->fhat;
    g.g = c->gpad;
    g.ftp = c->ftp;
    g.acc = c->acc;
    g.fbx = c->fbx;
    g.fby = c->fby;
    g.eqp = c->eqp;
    g.fpx = c->fpar;
    g.fpy = (char*)c->fpar + 5 * nfmax * csz;
    g.vq = c->vf;
    g.mom = c->mom;
    g.part = c->part;
    if (use_gnc) {
      // the class-moment path: its descriptor shares the velocity table, the
      // t_n parameters and moments and the face parameters with the above
      GncStep& n = c->gn;
      n.p = c->p;
      n.ref = g.ref;
      n.store = storage;
      n.s1 = c->s1;
      n.s2 = c->s2;
      n.c_om = c->c_om;
      n.fhat = c->fhat;
      n.ftp = c->ftp;
      n.eqn = (float*)c->eqp;
      n.mom_n = c->mom;
      n.fpx = (float*)c->fpar;
      n.fpy = (float*)((char*)c->fpar + 5 * nfmax * csz);
      n.vq = c->vf;
      for (int sd = 0; sd < 4; ++sd) n.ds_out[sd] = g.ds_out[sd];
      GncTables tb;
      if (e == cudaSuccess &&
          !gnc_tables(n, vel->xi_x, vel->xi_y, vel->w, host.data() + 3 * (size_t)nv, opp.data(), tb))
        e = cudaErrorInvalidValue;
      n.nch = gnc_chunks(n, sms);
      n.nsplit = gnc_splits(n, tb, sms);
      n.kc = (nv + n.nch - 1) / n.nch;
      n.nch = (nv + n.kc - 1) / n.kc;
      // one device block for the tables: ints, then floats (16-byte aligned)
      const size_t ni = tb.cls_off.size() + tb.cls_k.size() + tb.wsrc.size();
      const size_t ioff = 0, foff = ((ni * sizeof(int) + 15) / 16) * 16;
      const size_t nf1 = tb.cls_mono.size(), nf2 = tb.zc.size(), nf3 = tb.fwt.size();
      const size_t nf4 = tb.wbb.size();
      const size_t tab_bytes = foff + (nf1 + nf2 + nf3 + nf4) * sizeof(float);
      if (e == cudaSuccess) e = cudaMalloc(&c->gn_eq2, 5 * (size_t)p.N * csz);
      if (e == cudaSuccess) e = cudaMalloc((void**)&c->gn_mom2, 3 * (size_t)p.N * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&c->gn_wf, (size_t)nv * n.nw * csz);
      if (e == cudaSuccess) e = cudaMalloc((void**)&c->gn_wrho, (size_t)n.nw * sizeof(double));
      if (e == cudaSuccess)
        e = cudaMalloc((void**)&c->gn_sums, (size_t)n.nsplit * n.ncls * 10 * p.N * sizeof(double));
      if (e == cudaSuccess)
        e = cudaMalloc((void**)&c->gn_nu, (size_t)n.ncombo * 18 * p.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&c->gn_tab, tab_bytes);
      if (e == cudaSuccess) {
        std::vector<char> blob(tab_bytes, 0);
        std::memcpy(blob.data() + ioff, tb.cls_off.data(), tb.cls_off.size() * sizeof(int));
        std::memcpy(blob.data() + ioff + tb.cls_off.size() * sizeof(int), tb.cls_k.data(),
                    tb.cls_k.size() * sizeof(int));
        std::memcpy(blob.data() + ioff + (tb.cls_off.size() + tb.cls_k.size()) * sizeof(int),
                    tb.wsrc.data(), tb.wsrc.size() * sizeof(int));
        std::memcpy(blob.data() + foff, tb.cls_mono.data(), nf1 * sizeof(float));
        std::memcpy(blob.data() + foff + nf1 * sizeof(float), tb.zc.data(), nf2 * sizeof(float));
        std::memcpy(blob.data() + foff + (nf1 + nf2) * sizeof(float), tb.fwt.data(), nf3 * sizeof(float));
        std::memcpy(blob.data() + foff + (nf1 + nf2 + nf3) * sizeof(float), tb.wbb.data(),
                    nf4 * sizeof(float));
        e = cudaMemcpy(c->gn_tab, blob.data(), tab_bytes, cudaMemcpyHostToDevice);
      }
      if (e == cudaSuccess) e = gnc_prepare(storage);
      if (e != cudaSuccess) {
        free_all(c);
        delete c;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? DUGKS_ENOMEM : DUGKS_ECUDA,
                    std::string("class-moment path set-up: ") + cudaGetErrorString(e));
      }
      const char* tab = (const char*)c->gn_tab;
      n.cls_off = (const int*)(tab + ioff);
      n.cls_k = n.cls_off + tb.cls_off.size();
      n.wsrc = n.cls_k + tb.cls_k.size();
      n.cls_mono = (const float*)(tab + foff);
      n.zc = n.cls_mono + nf1;
      n.fwt = n.zc + nf2;
      n.wbb = (const float2*)(n.fwt + nf3);
      n.eqp = (float*)c->gn_eq2;
      n.mom_p = c->gn_mom2;
      n.wf = (float*)c->gn_wf;
      n.wrho = c->gn_wrho;
      n.sums = c->gn_sums;
      n.nu = c->gn_nu;
      c->gnc = true;
    }
    c->store = storage;
    c->gdev = true;
  }
  if (cd > 0.0 && !forced) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    D2Q9Params& q = c->dp;
    q.nx = p.nx;
    q.ny = p.ny;
    q.N = p.N;
    q.px = p.px;
    q.py = p.py;
    q.wsym = vel->w[1] == vel->w[3] && vel->w[1] == vel->w[5] && vel->w[1] == vel->w[7] &&
             vel->w[0] == vel->w[2] && vel->w[0] == vel->w[6] && vel->w[0] == vel->w[8];
    e = d2q9_prepare(0);
    const bool devk = storage == DUGKS_G_FP32 || storage == DUGKS_G_BF16;
    if (e == cudaSuccess && devk) e = d2q9m_prepare();
    {
      // resident blocks of the context's stage kernels at each height (the
      // double-word kernels keep the one-block model)
      int occ[17];
      for (int t = 0; t <= 16; ++t)
        occ[t] = e != cudaSuccess ? 1
                 : storage == DUGKS_FP64 ? d2q9_occupancy(dwa, q.wsym, t)
                 : devk ? d2q9m_occupancy(storage == DUGKS_G_FP32 ? 1 : 2, t) : 1;
      q.ty = d2q9_tile_height(p.nx, p.ny, sms, d2q9_max_ty(dwa), dwa, occ, devk);
    }
    for (int k = 0; k < 9; ++k) q.W[k] = vel->w[k];
    q.c3 = cd * cd / vel->RT;
    q.base_div = 0.5 / q.c3;
    q.half_mb = 0.5 - q.base_div;
    q.c_over_RT = cd / vel->RT;
    q.c = cd;
    q.a1 = c->s1.a;
    q.b1 = c->s1.b;
    q.a2 = c->s2.a;
    q.b2 = c->s2.b;
    q.c_om34 = 0.75 * c->c_om;
    q.r37 = 9.0 / 7.0;
    for (int s4 = 0; s4 < 4; ++s4) {
      q.bc_kind[s4] = bc[s4].kind;
      q.ds_den[s4] = p.ds_den[s4];
      for (int k = 0; k < 9; ++k) {
        q.feq_wall[s4][k] = host[(3 + s4) * (size_t)nv + k];
        q.bb[s4][k] = 2.0 * vel->w[k] *
                      (vel->xi_x[k] * bc[s4].uw_x + vel->xi_y[k] * bc[s4].uw_y) * invRT;
      }
    }
    d2q9_stage_tables(c->ds1, cd, p.dx, p.dy, T, c->s1.h, dt / 3.0);
    d2q9_stage_tables(c->ds2, cd, p.dx, p.dy, T, c->s2.h, 4.0 * dt / 7.0);
    if (dwa) {
      c->dwa = true;
      d2q9_params_to_dw(q, c->dwp);
      d2q9_stage_to_dw(c->ds1, c->dws1);
      d2q9_stage_to_dw(c->ds2, c->dws2);
    }
    if (e == cudaSuccess && storage != DUGKS_FP64) {
      c->store = storage;
      d2q9_stage_to_float(c->ds1, c->df1);
      d2q9_stage_to_float(c->ds2, c->df2);
    }
    if (e != cudaSuccess) {
      free_all(c);
      delete c;
      return cuda_fail(e, "dugks_init (fused D2Q9 set-up)");
    }
    c->d2q9 = true;
  }
  *out = c;
  if (dt / tau > 12.0)
    g_err = "warning: dt/tau > 12 exceeds the stability bound of the scheme";
  return DUGKS_OK;
}

int dugks_set_equilibrium(dugks_ctx* c, const double* rho, const double* ux, const double* uy,
                          int on_device) {
  if (!c || !rho || !ux || !uy) return fail(DUGKS_EINVAL, "NULL argument");
  const size_t N = c->p.N;
  const double *r = rho, *u = ux, *v = uy;
  if (!on_device) {  // stage through the moment buffer
    TRY(copy_in(c, c->mom, rho, N, 0));
    TRY(copy_in(c, c->mom + N, ux, N, 0));
    TRY(copy_in(c, c->mom + 2 * N, uy, N, 0));
    r = c->mom;
    u = c->mom + N;
    v = c->mom + 2 * N;
  }
  if (c->store)
    TRY(launch(c, K_SET_EQ, [&] { return launch_dev_set_eq(c->p, c->store, c->rho0, r, u, v, c->fhat, c->stream); }));
  else
    TRY(launch(c, K_SET_EQ, [&] { return launch_set_eq(c->p, r, u, v, c->fhat, c->stream); }));
  c->g1_valid = false;
  return DUGKS_OK;
}

int dugks_set_state(dugks_ctx* c, const double* fhat, int on_device) {
  if (!c || !fhat) return fail(DUGKS_EINVAL, "NULL argument");
  c->g1_valid = false;
  if (!on_device && !c->ev_copy &&
      cudaEventCreateWithFlags(&c->ev_copy, cudaEventDisableTiming) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "dugks_set_state");
  const size_t n = (size_t)c->p.nv * c->p.N;
  const double* src = fhat;
  if (!on_device || !c->store) {                  // deviation forms convert from a staging copy
    double* dst = c->store ? c->fbx : c->fhat;
    cudaError_t e = cudaMemcpyAsync(dst, fhat, n * sizeof(double),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess && !on_device) e = cudaEventRecord(c->ev_copy, c->stream);
    if (e != cudaSuccess) {
      cudaStreamSynchronize(c->stream);
      return cuda_fail(e, "copy to device");
    }
    src = dst;
  }
  // the conversion and the fused paths' g1 prologue are queued right behind
  // the copy; the call returns once the copy itself is done (the caller may
  // free or reuse a host buffer after return)
  int rc = DUGKS_OK;
  if (c->store)
    rc = launch(c, K_CONVERT, [&] { return launch_dev_from_f64(c->p, c->store, c->rho0, src, c->fhat, c->stream); });
  if (rc == DUGKS_OK && c->d2q9 && c->scheme == DUGKS_T3S3) rc = ensure_g1(c);
  if (!on_device) {
    const cudaError_t e = cudaEventSynchronize(c->ev_copy);
    if (e != cudaSuccess && rc == DUGKS_OK) return cuda_fail(e, "copy to device");
  }
  return rc;
}

int dugks_get_state(dugks_ctx* c, double* fhat, int which, int on_device) {
  if (!c || !fhat) return fail(DUGKS_EINVAL, "NULL argument");
  if (which != DUGKS_STATE_SCHEME && which != DUGKS_STATE_F)
    return fail(DUGKS_EINVAL, "which must be DUGKS_STATE_SCHEME or DUGKS_STATE_F");
  if (which == DUGKS_STATE_F) {
    // f from the scheme's variable x = f - c dt Omega(f): f = (tau x + c dt
    // feq)/(tau + c dt) with c = 1/4 (T3S3, eq. feqIntD3rdHat2) or 1/2 (T2,
    // eq. feqIntD2nd_Explicit); feq from the moments of x (the collision
    // conserves them)
    const double cdt = (c->scheme == DUGKS_T3S3 ? 0.25 : 0.5) * c->p.dt;
    const double a = c->p.tau / (c->p.tau + cdt), b = cdt / (c->p.tau + cdt);
    const double* src = c->fhat;
    if (c->store) {
      TRY(launch(c, K_CONVERT, [&] { return launch_f64_from_dev(c->p, c->store, c->rho0, c->fhat, c->fbx, c->stream); }));
      src = c->fbx;
    }
    double* dst = on_device ? fhat : c->fby;
    TRY(launch(c, K_MOMENTS, [&] {
      return launch_cell(c->p, c->groups, 1, src, dst, c->mom_aux, a, b, c->stream);
    }));
    if (on_device) return DUGKS_OK;
    return copy_out(c, fhat, c->fby, (size_t)c->p.nv * c->p.N, 0);
  }
  if (c->store) {
    double* dst = on_device ? fhat : c->fbx;
    TRY(launch(c, K_CONVERT, [&] { return launch_f64_from_dev(c->p, c->store, c->rho0, c->fhat, dst, c->stream); }));
    if (on_device) return DUGKS_OK;
    return copy_out(c, fhat, c->fbx, (size_t)c->p.nv * c->p.N, 0);
  }
  return copy_out(c, fhat, c->fhat, (size_t)c->p.nv * c->p.N, on_device);
}

int dugks_step(dugks_ctx* c, int n) {
  if (!c) return fail(DUGKS_EINVAL, "NULL context");
  if (n < 0) return fail(DUGKS_EINVAL, "n must be >= 0");
  for (int i = 0; i < n; ++i) TRY(advance(c));
  return DUGKS_OK;
}

int dugks_moments(dugks_ctx* c, double* rho, double* ux, double* uy, int on_device) {
  if (!c) return fail(DUGKS_EINVAL, "NULL context");
  // the class-moment path: the class sums of f^ and the cell finaliser of
  // stage 1 (which the next step recomputes anyway) give rho, u in c->mom
  double* mom = c->mom;
  if (c->gnc) TRY(gnc_moments(c));
  else TRY(launch(c, K_MOMENTS, [&] {
    if (c->store)
      return launch_dev_cell(c->p, c->store, c->rho0, c->fhat, nullptr, mom, 0.0, 0.0, 0, c->stream);
    if (c->d2q9) return launch_d2q9_cell(c->dp, false, c->fhat, nullptr, mom, c->stream);
    return launch_cell(c->p, c->groups, 0, c->fhat, nullptr, mom, 0.0, 0.0, c->stream);
  }));
  // the copies are queued on the stream; one synchronisation for host buffers.
  // rho, ux, uy consecutive in one buffer (the layout of mom): one copy
  const size_t N = c->p.N;
  double* dst[3] = {rho, ux, uy};
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (rho && ux == rho + N && uy == rho + 2 * N) {
    cudaError_t e = cudaMemcpyAsync(rho, mom, 3 * N * sizeof(double), kind, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy from device");
  } else {
    for (int m = 0; m < 3; ++m) {
      if (!dst[m]) continue;
      cudaError_t e = cudaMemcpyAsync(dst[m], mom + m * N, N * sizeof(double), kind, c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "copy from device");
    }
  }
  if (!on_device) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy from device");
  }
  return DUGKS_OK;
}

int dugks_check(dugks_ctx* c) {
  if (!c) return fail(DUGKS_EINVAL, "NULL context");
  cudaError_t e = cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dugks_check");
  double* mom = c->mom;
  if (c->gnc) TRY(gnc_moments(c));
  else TRY(launch(c, K_MOMENTS, [&] {
    return c->store ? launch_dev_cell(c->p, c->store, c->rho0, c->fhat, nullptr, mom, 0.0, 0.0, 0, c->stream)
                    : launch_cell(c->p, c->groups, 0, c->fhat, nullptr, mom, 0.0, 0.0, c->stream);
  }));
  TRY(launch(c, K_CHECK, [&] { return launch_check(c->p, mom, c->flag, c->stream); }));
  int h = 0;
  e = cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dugks_check");
  if (h) return fail(DUGKS_EUNSTABLE, "non-finite or non-positive density in the state");
  return DUGKS_OK;
}

int dugks_synchronize(dugks_ctx* c) {
  if (!c) return fail(DUGKS_EINVAL, "NULL context");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dugks_synchronize");
  return DUGKS_OK;
}

int dugks_profile(dugks_ctx* c, int enable) {
  if (!c) return fail(DUGKS_EINVAL, "NULL context");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dugks_profile");
  c->drain();
  for (int i = 0; i < K_NUM; ++i) {
    c->launches[i] = 0;
    c->ms[i] = 0.0;
  }
  c->prof = enable != 0;
  return DUGKS_OK;
}

int dugks_profile_read(dugks_ctx* c, long long* launches, double* ms, int n) {
  if (!c) return fail(DUGKS_EINVAL, "NULL context");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dugks_profile_read");
  c->drain();
  for (int i = 0; i < n && i < K_NUM; ++i) {
    if (launches) launches[i] = c->launches[i];
    if (ms) ms[i] = c->ms[i];
  }
  return K_NUM;
}

int dugks_adjoint_step(dugks_ctx* c, const double* lam_in, double* lam_out, double* dJ_dtau,
                       double* dJ_duw, int on_device) {
  if (!c || !lam_in || !lam_out) return fail(DUGKS_EINVAL, "NULL argument");
  if (c->store || c->dwa) return fail(DUGKS_ENOTIMPL, "the adjoint needs DUGKS_FP64 storage");
  if (c->scheme != DUGKS_T3S3) return fail(DUGKS_ENOTIMPL, "the adjoint is that of the T3S3 step");
  TRY(ensure_adjoint(c));
  const size_t nvN = (size_t)c->p.nv * c->p.N;
  CK(cudaMemsetAsync(c->a_grads, 0, 16 * sizeof(double), c->stream));
  TRY(copy_in(c, c->a_lam, lam_in, nvN, on_device));
  TRY(adjoint_core(c));
  TRY(copy_out(c, lam_out, c->a_out, nvN, on_device));
  return read_grads(c, dJ_dtau, dJ_duw);
}

int dugks_adjoint_run(dugks_ctx* c, const double* fhat0, int nsteps, int every,
                      const double* lam_final, double* lam0, double* dJ_dtau, double* dJ_duw,
                      int on_device) {
  if (!c || !fhat0 || !lam_final || !lam0) return fail(DUGKS_EINVAL, "NULL argument");
  if (nsteps < 0 || every < 1) return fail(DUGKS_EINVAL, "nsteps >= 0 and every >= 1 required");
  if (c->store || c->dwa) return fail(DUGKS_ENOTIMPL, "the adjoint needs DUGKS_FP64 storage");
  if (c->scheme != DUGKS_T3S3) return fail(DUGKS_ENOTIMPL, "the adjoint is that of the T3S3 step");
  TRY(ensure_adjoint(c));
  const size_t nvN = (size_t)c->p.nv * c->p.N;
  const int nseg = (nsteps + every - 1) / every;
  const size_t need = (size_t)nseg + (size_t)every + 1;   // checkpoints + one segment + f^N
  while (c->ckpt.size() < need) {
    double* b = nullptr;
    cudaError_t e = cudaMalloc((void**)&b, nvN * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(DUGKS_ENOMEM, "checkpoint store: " + std::string(cudaGetErrorString(e)));
    }
    c->ckpt.push_back(b);
  }
  double** cp = c->ckpt.data();               // cp[0..nseg): checkpoints
  double** seg = cp + nseg;                   // seg[0..every): states of one segment
  double* fin = cp[need - 1];                 // f^N
  auto set_dev = [&](const double* src) {
    c->g1_valid = false;
    return cudaMemcpyAsync(c->fhat, src, nvN * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  };
  // forward with checkpoints
  TRY(copy_in(c, c->fhat, fhat0, nvN, on_device));
  c->g1_valid = false;
  for (int n = 0; n < nsteps; ++n) {
    if (n % every == 0)
      CK(cudaMemcpyAsync(cp[n / every], c->fhat, nvN * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    TRY(advance(c));
  }
  CK(cudaMemcpyAsync(fin, c->fhat, nvN * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  // reverse sweep, recomputing each segment from its checkpoint
  CK(cudaMemsetAsync(c->a_grads, 0, 16 * sizeof(double), c->stream));
  TRY(copy_in(c, c->a_lam, lam_final, nvN, on_device));
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int start = sg * every, len = std::min(every, nsteps - start);
    CK(set_dev(cp[sg]));
    for (int m = 0; m < len; ++m) {
      CK(cudaMemcpyAsync(seg[m], c->fhat, nvN * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      if (m + 1 < len) TRY(advance(c));
    }
    for (int m = len - 1; m >= 0; --m) {
      CK(set_dev(seg[m]));
      TRY(adjoint_core(c));
      std::swap(c->a_lam, c->a_out);
    }
  }
  TRY(copy_out(c, lam0, c->a_lam, nvN, on_device));
  CK(set_dev(fin));
  return read_grads(c, dJ_dtau, dJ_duw);
}

int dugks_adjoint_equilibrium(dugks_ctx* c, const double* rho, const double* ux,
                              const double* uy, const double* lam, double* drho, double* dux,
                              double* duy, int on_device) {
  if (!c || !rho || !ux || !uy || !lam) return fail(DUGKS_EINVAL, "NULL argument");
  TRY(ensure_adjoint(c));
  const size_t N = c->p.N, nvN = (size_t)c->p.nv * N;
  // stage everything through adjoint buffers (a_mom1: rho, ux, uy; a_lam; a_mom2: outputs)
  TRY(copy_in(c, c->a_mom1, rho, N, on_device));
  TRY(copy_in(c, c->a_mom1 + N, ux, N, on_device));
  TRY(copy_in(c, c->a_mom1 + 2 * N, uy, N, on_device));
  TRY(copy_in(c, c->a_lam, lam, nvN, on_device));
  CK(launch_eq_T(c->p, c->a_mom1, c->a_mom1 + N, c->a_mom1 + 2 * N, c->a_lam, c->a_mom2,
                 c->a_mom2 + N, c->a_mom2 + 2 * N, c->stream));
  if (drho) TRY(copy_out(c, drho, c->a_mom2, N, on_device));
  if (dux) TRY(copy_out(c, dux, c->a_mom2 + N, N, on_device));
  if (duy) TRY(copy_out(c, duy, c->a_mom2 + 2 * N, N, on_device));
  return DUGKS_OK;
}

int dugks_autotune(dugks_ctx* c, int trials, int* ty_out) {
  if (!c) return fail(DUGKS_EINVAL, "NULL context");
  if (!c->d2q9) return fail(DUGKS_ENOTIMPL, "tile autotuning applies to the D2Q9 kernels");
  if (trials < 1) trials = 3;
  const size_t bytes = (size_t)c->p.nv * c->p.N * sizeof(double);
  cudaStream_t s = c->stream;
  const bool prof = c->prof;
  c->prof = false;
  CK(cudaMemcpyAsync(c->fbx, c->fhat, bytes, cudaMemcpyDeviceToDevice, s));   // save f^
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  int best = c->dp.ty;
  float best_ms = 1e30f;
  for (int ty = 4; ty <= d2q9_max_ty(c->dwa); ++ty) {
    c->dp.ty = ty;
    c->g1_valid = false;
    int rc = advance(c);                                  // warm-up incl. the prologue
    if (rc == DUGKS_OK) rc = cudaEventRecord(a, s) == cudaSuccess ? DUGKS_OK : DUGKS_ECUDA;
    for (int i = 0; i < trials && rc == DUGKS_OK; ++i) rc = advance(c);
    if (rc == DUGKS_OK) rc = cudaEventRecord(b, s) == cudaSuccess ? DUGKS_OK : DUGKS_ECUDA;
    float ms = 0.f;
    if (rc == DUGKS_OK && cudaEventSynchronize(b) == cudaSuccess &&
        cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = ty;
    }
    CK(cudaMemcpyAsync(c->fhat, c->fbx, bytes, cudaMemcpyDeviceToDevice, s));  // restore f^
    if (rc != DUGKS_OK) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      c->prof = prof;
      return rc;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->dp.ty = best;
  c->g1_valid = false;
  c->prof = prof;
  if (ty_out) *ty_out = best;
  return dugks_synchronize(c);
}

int dugks_set_tile_height(dugks_ctx* c, int ty) {
  if (!c) return fail(DUGKS_EINVAL, "NULL context");
  if (!c->d2q9) return fail(DUGKS_ENOTIMPL, "the tile height applies to the D2Q9 kernels");
  if (ty < 4 || ty > d2q9_max_ty(c->dwa)) return fail(DUGKS_EINVAL, "tile height out of range");
  c->dp.ty = ty;
  c->dwp.ty = ty;
  return DUGKS_OK;
}

int dugks_tile_height(dugks_ctx* c, int* ty_out) {
  if (!c || !ty_out) return fail(DUGKS_EINVAL, "NULL argument");
  if (!c->d2q9) return fail(DUGKS_ENOTIMPL, "the tile height applies to the D2Q9 kernels");
  *ty_out = c->dp.ty;
  return DUGKS_OK;
}

namespace {
// The persistent launch's work items for tile height ty: per fused instance
// its parameters and arrays and its first tile; device tables (re)written.
cudaError_t batch_items(dugks_batch* b, int ty) {
  std::vector<D2Q9BatchItem> items;
  std::vector<int> start(1, 0);
  for (dugks_ctx* c : b->fused) {
    D2Q9BatchItem it{};
    it.P = c->dp;
    it.P.ty = ty;
    it.S1 = c->ds1;
    it.S2 = c->ds2;
    it.fhat = c->fhat;
    it.g1 = c->g;
    it.g2 = c->ftp;
    it.X = c->acc;
    it.mom = c->mom;
    it.tiles_x = (c->p.nx + 31) / 32;
    start.push_back(start.back() + it.tiles_x * ((c->p.ny + ty - 1) / ty));
    items.push_back(it);
  }
  cudaError_t e = cudaSuccess;
  if (!b->items) e = cudaMalloc((void**)&b->items, items.size() * sizeof(D2Q9BatchItem));
  if (e == cudaSuccess && !b->tile_start) e = cudaMalloc((void**)&b->tile_start, start.size() * sizeof(int));
  if (e == cudaSuccess && !b->counters) e = cudaMalloc((void**)&b->counters, 2 * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->items, items.data(), items.size() * sizeof(D2Q9BatchItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->tile_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice);
  int dev = 0, sms = 152;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->nitems = (int)items.size();
  b->max_ty = ty;
  b->blocks = sms * d2q9_batch_blocks_per_sm(ty);
  return e;
}
}  // namespace

int dugks_batch_create(dugks_ctx* const* ctxs, int n, dugks_batch** out) {
  if (!out) return fail(DUGKS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1) return fail(DUGKS_EINVAL, "empty batch");
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(DUGKS_EINVAL, "NULL context in the batch");
    if (ctxs[i]->stream != ctxs[0]->stream)
      return fail(DUGKS_EINVAL, "batched contexts must share one stream");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(DUGKS_EINVAL, "a context appears twice in the batch");
  }
  if (!ctxs[0]->stream) return fail(DUGKS_EINVAL, "batching needs a non-default stream (graph capture)");
  dugks_batch* b = new dugks_batch();
  b->stream = ctxs[0]->stream;
  auto fused = [](const dugks_ctx* c) {
    return c->d2q9 && c->store == 0 && !c->dwa && c->scheme == DUGKS_T3S3;
  };
  // one tile height for all fused instances, the largest of theirs: every
  // block of the persistent launch has that many rows of threads, and a
  // shorter tile would leave some of them idle (results do not depend on it;
  // dugks_batch_autotune times the others)
  for (int i = 0; i < n; ++i)
    if (fused(ctxs[i])) b->max_ty = std::max(b->max_ty, ctxs[i]->dp.ty);
  for (int i = 0; i < n; ++i) {
    dugks_ctx* c = ctxs[i];
    b->ctxs.push_back(c);
    c->batched += 1;
    if (fused(c)) b->fused.push_back(c);
    else b->own.push_back(c);
  }
  cudaError_t e = cudaSuccess;
  // class-moment instances (T3S3) run batched: one group per (storage, ties)
  {
    std::map<std::pair<int, int>, std::vector<const GncStep*>> groups;
    std::vector<dugks_ctx*> rest;
    for (dugks_ctx* c : b->own) {
      if (c->gnc && c->scheme == DUGKS_T3S3) groups[{c->gn.store, c->gn.ties}].push_back(&c->gn);
      else rest.push_back(c);
    }
    b->own = rest;
    for (auto& kv : groups) {
      if (e != cudaSuccess) break;
      GncBatch gb;
      e = gnc_batch_init(kv.second.data(), (int)kv.second.size(), gb);
      if (e == cudaSuccess) b->gnc.push_back(gb);
      cudaStream_t gs = nullptr;
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
      if (e == cudaSuccess) b->gstreams.push_back(gs);
    }
  }
  // Own instances go into up to kBranches graph branches, largest first into
  // the branch with the least work (cells x velocities), so that their
  // kernels run concurrently with each other and with the persistent launch.
  {
    constexpr int kBranches = 8;
    const int nb = std::min<int>(kBranches, (int)b->own.size());
    std::vector<dugks_ctx*> order = b->own;
    std::stable_sort(order.begin(), order.end(), [](const dugks_ctx* x, const dugks_ctx* y) {
      return (double)x->p.N * x->p.nv > (double)y->p.N * y->p.nv;
    });
    b->branches.assign(nb, {});
    std::vector<double> load(nb, 0.0);
    for (dugks_ctx* c : order) {
      const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      b->branches[q].push_back(c);
      load[q] += (double)c->p.N * c->p.nv;
    }
    for (int q = 0; q < nb && e == cudaSuccess; ++q) {
      cudaStream_t bs = nullptr;
      e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
      if (e == cudaSuccess) b->bstreams.push_back(bs);
    }
    for (int q = 0; q < nb + (int)b->gnc.size() + 1 && e == cudaSuccess; ++q) {   // fork + joins
      cudaEvent_t ev = nullptr;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) b->bevents.push_back(ev);
    }
  }
  if (e == cudaSuccess && !b->fused.empty()) e = batch_items(b, b->max_ty);
  if (e != cudaSuccess) {
    dugks_batch_destroy(b);
    return cuda_fail(e, "dugks_batch_create");
  }
  *out = b;
  return DUGKS_OK;
}

int dugks_batch_step(dugks_batch* b, int nsteps) {
  if (!b) return fail(DUGKS_EINVAL, "NULL batch");
  if (nsteps < 0) return fail(DUGKS_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return DUGKS_OK;
  for (dugks_ctx* c : b->ctxs) TRY(ensure_g1(c));
  auto found = b->graphs.find(nsteps);
  if (found == b->graphs.end()) {
    std::vector<bool> prof;
    for (dugks_ctx* c : b->ctxs) {
      prof.push_back(c->prof);
      c->prof = false;
    }
    cudaStream_t s = b->stream;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? DUGKS_OK : cuda_fail(e, "begin capture");
    for (int i = 0; i < nsteps && rc == DUGKS_OK; ++i) {
      if (b->nitems) {
        e = cudaMemsetAsync(b->counters, 0, 2 * sizeof(int), s);
        if (e == cudaSuccess)
          e = launch_d2q9_batch(1, b->items, b->tile_start, b->nitems, b->max_ty, b->counters, b->blocks, s);
        if (e == cudaSuccess)
          e = launch_d2q9_batch(2, b->items, b->tile_start, b->nitems, b->max_ty, b->counters + 1, b->blocks, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "batched launch");
      }
    }
    // the own instances: each branch forks from the capturing stream, runs
    // its instances' steps on its stream and joins back; a class-moment
    // group is one branch that steps all its instances with batched launches
    if (rc == DUGKS_OK && (!b->branches.empty() || !b->gnc.empty())) {
      e = cudaEventRecord(b->bevents[0], s);
      if (e != cudaSuccess) rc = cuda_fail(e, "batch fork");
      for (size_t q = 0; q < b->gnc.size() && rc == DUGKS_OK; ++q) {
        cudaStream_t gs = b->gstreams[q];
        e = cudaStreamWaitEvent(gs, b->bevents[0], 0);
        for (int i = 0; i < nsteps && e == cudaSuccess; ++i)
          for (int stage = 1; stage <= 2 && e == cudaSuccess; ++stage)
            e = launch_gnc_batch_stage(b->gnc[q], stage, gs);
        cudaEvent_t ev = b->bevents[b->branches.size() + 1 + q];
        if (e == cudaSuccess) e = cudaEventRecord(ev, gs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "batched class-moment launch");
      }
      for (size_t q = 0; q < b->branches.size() && rc == DUGKS_OK; ++q) {
        cudaStream_t bs = b->bstreams[q];
        e = cudaStreamWaitEvent(bs, b->bevents[0], 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "batch fork");
        for (dugks_ctx* c : b->branches[q]) c->stream = bs;
        for (int i = 0; i < nsteps && rc == DUGKS_OK; ++i)
          for (dugks_ctx* c : b->branches[q]) {
            rc = advance(c);
            if (rc != DUGKS_OK) break;
          }
        for (dugks_ctx* c : b->branches[q]) c->stream = s;
        if (rc == DUGKS_OK) {
          e = cudaEventRecord(b->bevents[q + 1], bs);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->bevents[q + 1], 0);
          if (e != cudaSuccess) rc = cuda_fail(e, "batch join");
        }
      }
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    for (size_t k = 0; k < b->ctxs.size(); ++k) b->ctxs[k]->prof = prof[k];
    if (rc == DUGKS_OK && e != cudaSuccess) rc = cuda_fail(e, "end capture");
    cudaGraphExec_t x = nullptr;
    if (rc == DUGKS_OK) {
      e = cudaGraphInstantiate(&x, g, 0);
      if (e != cudaSuccess) rc = cuda_fail(e, "graph instantiate");
    }
    if (g) cudaGraphDestroy(g);
    if (rc != DUGKS_OK) return rc;
    found = b->graphs.emplace(nsteps, x).first;
  }
  cudaError_t e = cudaGraphLaunch(found->second, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return DUGKS_OK;
}

int dugks_batch_autotune(dugks_batch* b, int trials, int* ty_out) {
  if (!b) return fail(DUGKS_EINVAL, "NULL batch");
  if (b->fused.empty()) {
    if (ty_out) *ty_out = 0;
    return DUGKS_OK;
  }
  if (trials < 1) trials = 3;
  cudaStream_t s = b->stream;
  // save f^ of the fused instances (their face arrays are free between steps)
  for (dugks_ctx* c : b->fused)
    CK(cudaMemcpyAsync(c->fbx, c->fhat, (size_t)c->p.nv * c->p.N * sizeof(double),
                       cudaMemcpyDeviceToDevice, s));
  cudaEvent_t ea, eb;
  CK(cudaEventCreate(&ea));
  CK(cudaEventCreate(&eb));
  int best = b->max_ty;
  float best_ms = 1e30f;
  int rc = DUGKS_OK;
  for (int ty = 4; ty <= d2q9_max_ty(false) && rc == DUGKS_OK; ++ty) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = batch_items(b, ty);
    for (dugks_ctx* c : b->fused) c->g1_valid = false;
    for (dugks_ctx* c : b->fused)
      if (rc == DUGKS_OK && e == cudaSuccess) rc = ensure_g1(c);
    auto step = [&] {
      cudaError_t x = cudaMemsetAsync(b->counters, 0, 2 * sizeof(int), s);
      if (x == cudaSuccess)
        x = launch_d2q9_batch(1, b->items, b->tile_start, b->nitems, b->max_ty, b->counters, b->blocks, s);
      if (x == cudaSuccess)
        x = launch_d2q9_batch(2, b->items, b->tile_start, b->nitems, b->max_ty, b->counters + 1, b->blocks, s);
      return x;
    };
    if (e == cudaSuccess && rc == DUGKS_OK) e = step();            // warm-up
    if (e == cudaSuccess && rc == DUGKS_OK) e = cudaEventRecord(ea, s);
    for (int i = 0; i < trials && e == cudaSuccess && rc == DUGKS_OK; ++i) e = step();
    if (e == cudaSuccess && rc == DUGKS_OK) e = cudaEventRecord(eb, s);
    float ms = 0.f;
    if (e == cudaSuccess && rc == DUGKS_OK) e = cudaEventSynchronize(eb);
    if (e == cudaSuccess && rc == DUGKS_OK) e = cudaEventElapsedTime(&ms, ea, eb);
    if (e == cudaSuccess && rc == DUGKS_OK && ms < best_ms) {
      best_ms = ms;
      best = ty;
    }
    for (dugks_ctx* c : b->fused)                                  // restore f^
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->fhat, c->fbx, (size_t)c->p.nv * c->p.N * sizeof(double),
                            cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess && rc == DUGKS_OK) rc = cuda_fail(e, "dugks_batch_autotune");
  }
  cudaEventDestroy(ea);
  cudaEventDestroy(eb);
  if (rc != DUGKS_OK) return rc;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = batch_items(b, best);
  if (e != cudaSuccess) return cuda_fail(e, "dugks_batch_autotune");
  for (dugks_ctx* c : b->fused) c->g1_valid = false;
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);    // captured with the old shape
  b->graphs.clear();
  if (ty_out) *ty_out = best;
  return DUGKS_OK;
}

int dugks_batch_destroy(dugks_batch* b) {
  if (!b) return DUGKS_OK;
  cudaStreamSynchronize(b->stream);
  for (dugks_ctx* c : b->ctxs) c->batched -= 1;
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  if (b->items) cudaFree(b->items);
  if (b->tile_start) cudaFree(b->tile_start);
  if (b->counters) cudaFree(b->counters);
  for (cudaEvent_t ev : b->bevents) cudaEventDestroy(ev);
  for (cudaStream_t bs : b->bstreams) cudaStreamDestroy(bs);
  for (GncBatch& gb : b->gnc) gnc_batch_free(gb);
  for (cudaStream_t gs : b->gstreams) cudaStreamDestroy(gs);
  delete b;
  return DUGKS_OK;
}

int dugks_set_scheme(dugks_ctx* c, int scheme) {
  if (!c) return fail(DUGKS_EINVAL, "NULL context");
  if (scheme < DUGKS_T3S3 || scheme > DUGKS_T2S2) return fail(DUGKS_EINVAL, "unknown scheme");
  if (c->batched) return fail(DUGKS_EINVAL, "the context belongs to a batch");
  if (scheme != DUGKS_T3S3 && (c->store || c->dwa))
    return fail(DUGKS_ENOTIMPL, "the T2 schemes run with DUGKS_FP64 storage");
  c->scheme = scheme;
  c->p.recon = scheme == DUGKS_T2S2 ? 1 : 0;
  c->g1_valid = false;
  return DUGKS_OK;
}

int dugks_destroy(dugks_ctx* c) {
  if (!c) return DUGKS_OK;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
  return DUGKS_OK;
}

}  // extern "C"
