// Mixed-precision fused D2Q9 T3S3 kernels (deviation storage in FP32/BF16).
//
// Same two-launch structure as the FP64 kernels (dugks_d2q9.cu), with every
// per-(cell, velocity) array holding the deviation d = f - W_k rho0 from the
// reference equilibrium at rest.  Because the maps of the step are affine
// with coefficients summing to one (g = a f + b feq with a + b = 1, stencil
// weights summing to one, ghost extrapolation 3 - 3 + 1), they apply to
// deviations unchanged, and the stored values are O(Ma) W_k instead of
// O(1) W_k, which keeps FP32/BF16 rounding small relative to f.
//
// Precision split: stencil dot products, fluxes, the per-velocity assembly
// of the equilibrium deviation W_k((rho - rho0) + rho (P_k - 1)), the face
// moments and the face equilibria, and all combinations run in FP32; the
// cell moment sums (rho, rho u), which the collision conserves, are exact
// (fixed point), rounded to FP64 for the stored density and once more to
// FP32 for the cell's equilibrium parameters 1/rho, u / RT and
// |u|^2 / (2 RT), formed in FP32 like the faces' (Sec. 2.2 moments;
// Sec. 2.1.1 equilibrium).
#include <cuda_bf16.h>

#include <cmath>

#include "dugks_fp.cuh"
#include "dugks_internal.cuh"

namespace dugks {

namespace {

constexpr int TX = 32;
constexpr int HALO = 2;
constexpr int SW = TX + 2 * HALO;
constexpr int kMaxTY = 16;
constexpr int kMaxThreads = TX * (kMaxTY + 1);

template <typename T> __device__ __forceinline__ float ld(const T* p);
template <> __device__ __forceinline__ float ld<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
template <typename T> __device__ __forceinline__ void st(T* p, float v);
template <> __device__ __forceinline__ void st<float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void st<__nv_bfloat16>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}

struct MixedConst {
  double rho0;          // reference density of the deviations
  double rho0W;         // rho0 * sum_k W_k
  double sxW, syW;      // rho0 * (sum_{ex=1} W - sum_{ex=-1} W), same for y
  long long fr0W;       // rho0 sum W in 56-fraction-bit fixed point
  long long fdr0;       // rho0 (sum W - 1), fixed point
  long long fsxW, fsyW; // sxW, syW, fixed point
  double inW[4];        // rho0 * sum of W over the velocities hitting each wall
  float W[9];
  float bb[4][9];       // bounce-back: rho_w * bb + (W_opp - W_k) rho0
  float bbc[4][9];
  float r37, com, a1, b1, a2, b2;   // FP32 copies of the stage coefficients
  float c3f, base_divf;             // FP32 copies of c^2/RT and 1/(2 c^2/RT)
  float r0Wf, dr0f, sxWf, syWf;     // FP32 copies of rho0W, rho0 (sum W - 1), sxW, syW
};

template <int K> struct Vel {
  static constexpr int ex = K / 3 - 1;
  static constexpr int ey = K % 3 - 1;
};

template <int R0, int R1, int Q0, int Q1, int NCOL>
__device__ __forceinline__ float wdotf(const float* __restrict__ s, const float* w) {
  float acc = 0.0f;
#pragma unroll
  for (int r = R0; r <= R1; ++r)
#pragma unroll
    for (int q = Q0; q <= Q1; ++q) {
      const float v = s[r * SW + q];
      acc = (r == R0 && q == Q0) ? w[r * NCOL + q] * v : fmaf(w[r * NCOL + q], v, acc);
    }
  return acc;
}

template <int K>
__device__ __forceinline__ float xface_valf(const float* __restrict__ s, const D2Q9StageF& S) {
  constexpr int ex = Vel<K>::ex, ey = Vel<K>::ey;
  constexpr int q0 = ex < 0 ? 1 : 0, q1 = ex > 0 ? 2 : 3;
  constexpr int r0 = ey == 0 ? 1 : 0, r1 = ey == 0 ? 1 : 2;
  return wdotf<r0, r1, q0, q1, 4>(s, &S.wx[K][0][0]);
}

template <int K>
__device__ __forceinline__ float yface_valf(const float* __restrict__ s, const D2Q9StageF& S) {
  constexpr int ex = Vel<K>::ex, ey = Vel<K>::ey;
  constexpr int q0 = ey < 0 ? 1 : 0, q1 = ey > 0 ? 2 : 3;
  constexpr int c0 = ex == 0 ? 1 : 0, c1 = ex == 0 ? 1 : 2;
  return wdotf<q0, q1, c0, c1, 3>(s, &S.wy[K][0][0]);
}


// FP32 value -> signed fixed point with 56 fraction bits (resolution
// 1.4e-17, comparable to the FP64 rounding of O(0.1) terms).  `bad` is set
// for |x| >= 8, inf or NaN (nine such terms keep the sum below 2^7), which
// the caller turns into a NaN moment so that dugks_check reports it.
__device__ __forceinline__ long long f2fix(float x, unsigned& bad) {
  const unsigned b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xffu);
  const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = e - 94;                          // x * 2^56 = m * 2^(e - 94)
  unsigned long long v = sh >= 0 ? (m << (sh & 63)) : (m >> ((-sh) & 63));
  v = (sh < -63 || e == 0) ? 0ull : v;
  bad |= (unsigned)(e >= 130);
  return (b >> 31) ? -(long long)v : (long long)v;
}

// fixed point (56 fraction bits) -> FP64, round to nearest, integer pipe only
__device__ __forceinline__ double fix2d(long long v) {
  const unsigned long long s = v < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  const unsigned long long n = a << (lz & 63);    // leading one at bit 63
  const unsigned long long bits =
      ((unsigned long long)(1023 + 7 - lz) << 52) + ((n >> 11) & 0xfffffffffffffull) +
      ((n >> 10) & 1ull);
  return __longlong_as_double((long long)(a == 0 ? 0ull : (bits | s)));
}

// Moments of f = W rho0 + d (Sec. 2.2): the sums over the nine velocities,
// including the reference part rho0 W, are accumulated exactly in 64-bit
// fixed point on the integer pipe and rounded once to FP64 (absolute error
// <= 1.2e-16, the order of FP64 summation of O(0.1) terms).  dr = rho - rho0.
__device__ __forceinline__ void dev_sums(const float (&d)[9], const MixedConst& M, double& rho,
                                         double& dr, double& sx, double& sy) {
  unsigned bad = 0u;
  long long v[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = f2fix(d[k], bad);
  const long long a = v[0] + v[1] + v[2];
  const long long b = v[6] + v[7] + v[8];
  const long long r = a + b + (v[3] + v[4] + v[5]);
  const long long y = (v[2] + v[5] + v[8]) - (v[0] + v[3] + v[6]);
  rho = bad ? __longlong_as_double(0x7ff8000000000000ll) : fix2d(r + M.fr0W);
  dr = fix2d(r + M.fdr0);
  sx = fix2d(b - a + M.fsxW);
  sy = fix2d(y + M.fsyW);
}



// The face moments of f-bar, summed in FP32: they set only the face
// equilibrium, which is assembled in FP32 (the cell moments, which the
// collision conserves, keep the exact sums of dev_sums).
__device__ __forceinline__ void dev_sums_f(const float (&d)[9], const MixedConst& M, float& rho,
                                           float& dr, float& sx, float& sy) {
  const float a = (d[0] + d[1]) + d[2];
  const float b = (d[6] + d[7]) + d[8];
  const float r = (a + b) + ((d[3] + d[4]) + d[5]);
  const float y = ((d[2] + d[5]) + d[8]) - ((d[0] + d[3]) + d[6]);
  rho = r + M.r0Wf;
  dr = r + M.dr0f;
  sx = (b - a) + M.sxWf;
  sy = y + M.syWf;
}

// Face equilibrium deviations W_k (rho P_k - rho0) in FP32 from the FP32
// moments: 1/rho from the hardware reciprocal approximation refined by one
// Newton step (relative error ~2^-23), u/RT and the constant part in FP32.
// The per-velocity assembly is FP32 in either form; its parameters here
// carry a few units in the last place of FP32 instead of one rounding.
__device__ __forceinline__ void dev_feq_f(float rho, float dr, float sx, float sy,
                                          const MixedConst& M, float (&fe)[9]) {
  float rr;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rr) : "f"(rho));
  rr = fmaf(rr, fmaf(-rho, rr, 1.0f), rr);
  const float rc = M.c3f * rr;
  const float ux = sx * rc, uy = sy * rc;
  const float b1 = -fmaf(ux, ux, uy * uy) * M.base_divf;
  const float r = rho;
  const float sp = ux + uy, sm = ux - uy;
  float p1[9];                                                  // P_k - 1
  p1[4] = b1;
  const float bx = fmaf(0.5f * ux, ux, b1), by = fmaf(0.5f * uy, uy, b1);
  const float bs = fmaf(0.5f * sp, sp, b1), bd = fmaf(0.5f * sm, sm, b1);
  p1[7] = bx + ux; p1[1] = bx - ux;
  p1[5] = by + uy; p1[3] = by - uy;
  p1[8] = bs + sp; p1[0] = bs - sp;
  p1[6] = bd + sm; p1[2] = bd - sm;
#pragma unroll
  for (int k = 0; k < 9; ++k) fe[k] = M.W[k] * fmaf(r, p1[k], dr);
}


// A staged coordinate of a tile with its 2-cell halo: >= 0 the cell it holds
// (in the domain or its periodic image); -1 a wall ghost; -2 beyond the
// ghost band (never read by a computed face).
__device__ __forceinline__ int stage_coord(int x, int n, bool per) {
  if (x >= 0 && x < n) return x;
  if (per) return ((x % n) + n) % n;
  return (x >= -2 && x <= n + 1) ? -1 : -2;
}

// Taps of a staged coordinate for the ghost fill, as positions in the
// staged tile (t0 = tile origin, s = this position): itself when it holds a
// cell, else the three cells next to the wall with the weights of the
// quadratic extrapolation (3, -3, 1 and 6, -8, 3); a tile holding a ghost
// holds those cells too (walls need three cells across).
__device__ __forceinline__ int ghost_taps(int x, int ix, int n, int t0, int s, int (&pos)[3],
                                          float (&c)[3]) {
  if (ix >= 0) { pos[0] = s; c[0] = 1.f; return 1; }
  const int b = x < 0 ? 0 : n - 1, d = x < 0 ? 1 : -1;
  const bool near = x == -1 || x == n;
  c[0] = near ? 3.f : 6.f;
  c[1] = near ? -3.f : -8.f;
  c[2] = near ? 1.f : 3.f;
#pragma unroll
  for (int m = 0; m < 3; ++m) pos[m] = b + m * d - t0 + HALO;
  return 3;
}

// Wall face in deviation form: tangential velocities from the fluid cell only,
// leaving ones by bounce-back (eq. BB) or diffuse scattering.
template <int DIR>
__device__ __forceinline__ void wall_dev(float (&fb)[9], const float* __restrict__ s0, int stride,
                                         const D2Q9StageF& S, const D2Q9Params& P,
                                         const MixedConst& M, int side, bool hi, double rho_w) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int en = DIR == 0 ? (k / 3 - 1) : (k % 3 - 1);
    if (en != 0) continue;
    const float* sk = s0 + k * stride + (hi ? (DIR == 0 ? 1 : SW) : 0);
    const float* w = DIR == 0 ? (hi ? &S.wxR[k][0][0] : &S.wxL[k][0][0])
                              : (hi ? &S.wyT[k][0][0] : &S.wyB[k][0][0]);
    float v = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) v = fmaf(w[a * 3 + b], sk[a * SW + b], v);
    fb[k] = v;
  }
  const int nsg = hi ? -1 : 1;
  if (P.bc_kind[side] == BC_BOUNCEBACK) {
    const float rw = (float)rho_w;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int en = DIR == 0 ? (k / 3 - 1) : (k % 3 - 1);
      if (nsg * en < 0) fb[k] = fmaf(rw, M.bb[side][k], fb[8 - k] + M.bbc[side][k]);
    }
  } else {
    double num = M.inW[side];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int en = DIR == 0 ? (k / 3 - 1) : (k % 3 - 1);
      if (nsg * en > 0) num += (double)fb[k];
    }
    const double rd = num * P.c / P.ds_den[side];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int en = DIR == 0 ? (k / 3 - 1) : (k % 3 - 1);
      if (nsg * en < 0) fb[k] = (float)fma(rd, P.feq_wall[side][k], -P.W[k] * M.rho0);
    }
  }
}

// f/alpha = f-bar + gamma feq for one face of direction DIR (0: x, 1: y);
// the tangential velocities (no flux through the face) keep f-bar
template <int DIR>
__device__ __forceinline__ void face_recover_dev(float (&fb)[9], const D2Q9StageF& S,
                                                 const D2Q9Params& P, const MixedConst& M) {
  float rho, dr, sx, sy;
  dev_sums_f(fb, M, rho, dr, sx, sy);
  float fe[9];
  dev_feq_f(rho, dr, sx, sy, M, fe);
  (void)P;
#pragma unroll
  for (int k = 0; k < 9; ++k)
    if (DIR == 0 ? (k / 3 != 1) : (k % 3 != 1)) fb[k] = fmaf(S.gamma, fe[k], fb[k]);
}

template <int STAGE, typename T>
__global__ void __launch_bounds__(kMaxThreads)
k_d2q9m(D2Q9Params P, D2Q9StageF S, MixedConst M, const T* __restrict__ gin,
        const T* __restrict__ own, const double* __restrict__ rho_in, T* __restrict__ out0,
        T* __restrict__ out1, double* __restrict__ rho_out) {
  extern __shared__ float smf[];
  const int TY = P.ty;
  const int SH = TY + 2 * HALO;
  float* sg = smf;                                 // [9][SH][SW]
  float* sfx = sg + 9 * SH * SW;                   // [9][TY][TX+1]
  float* sfy = sfx + 9 * TY * (TX + 1);            // [9][TY+1][TX]
  const int nx = P.nx, ny = P.ny, N = P.N;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int stride = SH * SW;
  // launched as a programmatic dependent of the previous stage kernel when
  // the grid is one wave: wait for it (a no-op otherwise) before any read
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // staged tile: cells of the domain and their periodic images first, then
  // the wall ghosts extrapolated from them (no chain of global loads)
  for (int p = tid; p < SH * SW; p += nthr) {
    const int rr = p / SW, cc = p - rr * SW;
    const int ix = stage_coord(x0 + cc - HALO, nx, P.px);
    const int iy = stage_coord(y0 + rr - HALO, ny, P.py);
    if (ix >= 0 && iy >= 0) {
      const T* src = gin + iy * nx + ix;
#pragma unroll
      for (int k = 0; k < 9; ++k) sg[k * stride + rr * SW + cc] = ld(src + (size_t)k * N);
    } else if (ix == -2 || iy == -2) {
#pragma unroll
      for (int k = 0; k < 9; ++k) sg[k * stride + rr * SW + cc] = 0.f;
    }
  }
  // ghosts: one (ghost, velocity) pair per thread; ghost columns (every
  // row of the band, corners included), then ghost rows (columns that hold
  // a cell)
  const bool gw = !P.px && x0 == 0, gs = !P.py && y0 == 0;
  const int ce = nx - x0 + HALO, rn = ny - y0 + HALO;    // first east column, north row
  const int ngc = (gw ? 2 : 0) + (P.px ? 0 : max(0, min(2, SW - ce)));
  const int ngr = (gs ? 2 : 0) + (P.py ? 0 : max(0, min(2, SH - rn)));
  if (ngc + ngr > 0) {
    __syncthreads();
    const int ncol = ngc * SH * 9;
    for (int t = tid; t < ncol + ngr * SW * 9; t += nthr) {
      int rr, cc, k;
      if (t < ncol) {
        const int q = t / 9, ci = q / SH;
        k = t - q * 9;
        rr = q - ci * SH;
        cc = (gw && ci < 2) ? ci : ce + ci - (gw ? 2 : 0);
      } else {
        const int q = (t - ncol) / 9, ri = q / SW;
        k = (t - ncol) - q * 9;
        cc = q - ri * SW;
        rr = (gs && ri < 2) ? ri : rn + ri - (gs ? 2 : 0);
      }
      const int x = x0 + cc - HALO, y = y0 + rr - HALO;
      const int ix = stage_coord(x, nx, P.px), iy = stage_coord(y, ny, P.py);
      if (ix == -2 || iy == -2 || (t >= ncol && ix < 0)) continue;
      int pc[3], pr[3];
      float cx[3], cy[3];
      const int nxr = ghost_taps(x, ix, nx, x0, cc, pc, cx);
      const int nyr = ghost_taps(y, iy, ny, y0, rr, pr, cy);
      float v = 0.f;
      for (int a = 0; a < nyr; ++a)
        for (int b = 0; b < nxr; ++b)
          v = fmaf(cy[a] * cx[b], sg[k * stride + pr[a] * SW + pc[b]], v);
      sg[k * stride + rr * SW + cc] = v;
    }
  }
  __syncthreads();
  // the tile is staged: the next stage kernel may begin launching
  asm volatile("griddepcontrol.launch_dependents;");

  // x-faces; wall faces (fi = 0 or nx) after all the others, so that no
  // warp of interior faces diverges on one
  const int wc0 = (!P.px && x0 == 0) ? 0 : -1;
  const int wc1 = (!P.px && nx - x0 <= TX) ? nx - x0 : -1;
  const int nmain = TX + 1 - (wc0 >= 0) - (wc1 >= 0);
  for (int t = tid; t < TY * (TX + 1); t += nthr) {
    int r, fc;
    if (t < TY * nmain) {
      r = t / nmain;
      fc = t - r * nmain;
      if (wc0 >= 0) ++fc;
      if (wc1 >= 0 && fc >= wc1) ++fc;
    } else {
      const int u = t - TY * nmain, w = u / TY;
      r = u - w * TY;
      fc = (w == 0 && wc0 >= 0) ? wc0 : wc1;
    }
    const int j = y0 + r, fi = x0 + fc;
    if (j >= ny || fi > nx) continue;
    float fb[9];
    const float* s0 = sg + (r + 1) * SW + fc;
    fb[0] = xface_valf<0>(s0 + 0 * stride, S);
    fb[1] = xface_valf<1>(s0 + 1 * stride, S);
    fb[2] = xface_valf<2>(s0 + 2 * stride, S);
    fb[3] = xface_valf<3>(s0 + 3 * stride, S);
    fb[4] = xface_valf<4>(s0 + 4 * stride, S);
    fb[5] = xface_valf<5>(s0 + 5 * stride, S);
    fb[6] = xface_valf<6>(s0 + 6 * stride, S);
    fb[7] = xface_valf<7>(s0 + 7 * stride, S);
    fb[8] = xface_valf<8>(s0 + 8 * stride, S);
    if (!P.px && (fi == 0 || fi == nx)) {
      const bool hi = fi == 0;
      wall_dev<0>(fb, s0, stride, S, P, M, hi ? SIDE_W : SIDE_E, hi,
                  rho_in[j * nx + (hi ? 0 : nx - 1)]);
    }
    face_recover_dev<0>(fb, S, P, M);
#pragma unroll
    for (int k = 0; k < 9; ++k)
      if (k / 3 != 1) sfx[(k * TY + r) * (TX + 1) + fc] = fb[k];   // read back: e_x != 0 only
  }

  for (int t = tid; t < (TY + 1) * TX; t += nthr) {
    const int fr = t / TX, c = t - fr * TX;
    const int fj = y0 + fr, i = x0 + c;
    if (i >= nx || fj > ny) continue;
    float fb[9];
    const float* s0 = sg + fr * SW + (c + 1);
    fb[0] = yface_valf<0>(s0 + 0 * stride, S);
    fb[1] = yface_valf<1>(s0 + 1 * stride, S);
    fb[2] = yface_valf<2>(s0 + 2 * stride, S);
    fb[3] = yface_valf<3>(s0 + 3 * stride, S);
    fb[4] = yface_valf<4>(s0 + 4 * stride, S);
    fb[5] = yface_valf<5>(s0 + 5 * stride, S);
    fb[6] = yface_valf<6>(s0 + 6 * stride, S);
    fb[7] = yface_valf<7>(s0 + 7 * stride, S);
    fb[8] = yface_valf<8>(s0 + 8 * stride, S);
    if (!P.py && (fj == 0 || fj == ny)) {
      const bool hi = fj == 0;
      wall_dev<1>(fb, s0, stride, S, P, M, hi ? SIDE_S : SIDE_N, hi,
                  rho_in[(hi ? 0 : ny - 1) * nx + i]);
    }
    face_recover_dev<1>(fb, S, P, M);
#pragma unroll
    for (int k = 0; k < 9; ++k)
      if (k % 3 != 1) sfy[(k * (TY + 1) + fr) * TX + c] = fb[k];   // read back: e_y != 0 only
  }
  __syncthreads();

  for (int t = tid; t < TY * TX; t += nthr) {
    const int r = t / TX, c = t - r * TX;
    const int j = y0 + r, i = x0 + c;
    if (j >= ny || i >= nx) continue;
    const int cell = j * nx + i;
    float L[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int ex = k / 3 - 1, ey = k % 3 - 1;
      float v = 0.f;
      if (ex != 0)
        v = S.kx[k] * (sfx[(k * TY + r) * (TX + 1) + c + 1] - sfx[(k * TY + r) * (TX + 1) + c]);
      if (ey != 0) {
        const float d = sfy[(k * (TY + 1) + r + 1) * TX + c] - sfy[(k * (TY + 1) + r) * TX + c];
        v = (ex != 0) ? fmaf(S.ky[k], d, v) : S.ky[k] * d;
      }
      L[k] = v;
    }
    if (STAGE == 1) {
      float ft[9], X[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float g1 = sg[k * stride + (r + HALO) * SW + c + HALO];
        const float fh = ld(own + (size_t)k * N + cell);
        ft[k] = fmaf(1.25f, g1, fmaf(-0.25f, fh, L[k]));
        X[k] = fmaf(0.25f, fh, fmaf(0.75f, g1, M.r37 * L[k]));
      }
      double rho, dr, sx, sy;
      dev_sums(ft, M, rho, dr, sx, sy);
      float fe[9];
      dev_feq_f(d2f_bits(rho), d2f_bits(dr), d2f_bits(sx), d2f_bits(sy), M, fe);
      const float com = M.com, a2 = M.a2, b2 = M.b2;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        st(out0 + (size_t)k * N + cell, fmaf(b2, fe[k], a2 * ft[k]));
        st(out1 + (size_t)k * N + cell, fmaf(com, ft[k] - fe[k], X[k]));
      }
      rho_out[cell] = rho;
    } else {
      float fh[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) fh[k] = ld(own + (size_t)k * N + cell) + L[k];
      double rho, dr, sx, sy;
      dev_sums(fh, M, rho, dr, sx, sy);
      float fe[9];
      dev_feq_f(d2f_bits(rho), d2f_bits(dr), d2f_bits(sx), d2f_bits(sy), M, fe);
      const float a1 = M.a1, b1 = M.b1;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        st(out0 + (size_t)k * N + cell, fh[k]);
        st(out1 + (size_t)k * N + cell, fmaf(b1, fe[k], a1 * fh[k]));
      }
      rho_out[cell] = rho;
    }
  }
}

// ---------------------------------------------- conversions and cell passes
template <typename T>
__global__ void k_dev_from_f64(DevParams p, double rho0, const double* __restrict__ f,
                               T* __restrict__ d) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.nv * p.N) return;
  const int k = (int)(t / p.N);
  st(d + t, (float)(f[t] - __ldg(p.w + k) * rho0));
}

template <typename T>
__global__ void k_f64_from_dev(DevParams p, double rho0, const T* __restrict__ d,
                               double* __restrict__ f) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.nv * p.N) return;
  const int k = (int)(t / p.N);
  f[t] = (double)ld(d + t) + __ldg(p.w + k) * rho0;
}

// per cell: FP64 moments of f = W rho0 + d; optionally g = a f + b feq as a deviation
template <typename T>
__global__ void k_dev_cell(DevParams p, double rho0, const T* __restrict__ d, T* __restrict__ g,
                           double* __restrict__ mom, double a, double b, int write_g) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.N) return;
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int k = 0; k < p.nv; ++k) {
    const double f = (double)ld(d + (size_t)k * p.N + cell) + __ldg(p.w + k) * rho0;
    r += f;
    jx += __ldg(p.xi_x + k) * f;
    jy += __ldg(p.xi_y + k) * f;
  }
  const double ux = jx / r, uy = jy / r;
  mom[cell] = r;
  mom[p.N + cell] = ux;
  mom[2 * p.N + cell] = uy;
  if (!write_g) return;
  const double uu = (ux * ux + uy * uy) * p.inv_RT;
  for (int k = 0; k < p.nv; ++k) {
    const size_t idx = (size_t)k * p.N + cell;
    const double eu = (__ldg(p.xi_x + k) * ux + __ldg(p.xi_y + k) * uy) * p.inv_RT;
    const double w = __ldg(p.w + k);
    const double feq_dev = w * (r * (1.0 + eu + 0.5 * eu * eu - 0.5 * uu) - rho0);
    const double dv = (double)ld(d + idx);
    st(g + idx, (float)(a * dv + b * feq_dev));
  }
}

template <typename T>
__global__ void k_dev_set_eq(DevParams p, double rho0, const double* __restrict__ rho,
                             const double* __restrict__ ux, const double* __restrict__ uy,
                             T* __restrict__ d) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.nv * p.N) return;
  const int k = (int)(t / p.N);
  const int cell = (int)(t - (size_t)k * p.N);
  const double u = ux[cell], v = uy[cell];
  const double eu = (__ldg(p.xi_x + k) * u + __ldg(p.xi_y + k) * v) * p.inv_RT;
  const double uu = (u * u + v * v) * p.inv_RT;
  st(d + t, (float)(__ldg(p.w + k) * (rho[cell] * (1.0 + eu + 0.5 * eu * eu - 0.5 * uu) - rho0)));
}

unsigned nblk(size_t n) { return (unsigned)((n + 255) / 256); }

template <typename T>
MixedConst mixed_const(const D2Q9Params& P, double rho0) {
  MixedConst M{};
  M.rho0 = rho0;
  double sw = 0.0, sxp = 0.0, syp = 0.0;
  for (int k = 0; k < 9; ++k) {
    sw += P.W[k];
    sxp += (k / 3 - 1) * P.W[k];
    syp += (k % 3 - 1) * P.W[k];
    M.W[k] = (float)P.W[k];
  }
  M.rho0W = rho0 * sw;
  M.fr0W = llrint(std::ldexp(rho0 * sw, 56));
  M.fdr0 = llrint(std::ldexp(rho0 * (sw - 1.0), 56));
  M.fsxW = llrint(std::ldexp(rho0 * sxp, 56));
  M.fsyW = llrint(std::ldexp(rho0 * syp, 56));
  M.r0Wf = (float)(rho0 * sw);
  M.dr0f = (float)(rho0 * (sw - 1.0));
  M.sxWf = (float)(rho0 * sxp);
  M.syWf = (float)(rho0 * syp);
  M.c3f = (float)P.c3;
  M.base_divf = (float)P.base_div;
  M.r37 = (float)P.r37;
  M.com = (float)P.c_om34;
  M.a1 = (float)P.a1;
  M.b1 = (float)P.b1;
  M.a2 = (float)P.a2;
  M.b2 = (float)P.b2;
  M.sxW = rho0 * sxp;
  M.syW = rho0 * syp;
  for (int s = 0; s < 4; ++s) {
    const int dir = (s == SIDE_W || s == SIDE_E) ? 0 : 1;
    const int nsg = (s == SIDE_W || s == SIDE_S) ? -1 : 1;
    double in = 0.0;
    for (int k = 0; k < 9; ++k) {
      const int en = dir == 0 ? (k / 3 - 1) : (k % 3 - 1);
      if (nsg * en > 0) in += P.W[k];
      M.bb[s][k] = (float)P.bb[s][k];
      M.bbc[s][k] = (float)((P.W[8 - k] - P.W[k]) * rho0);
    }
    M.inW[s] = rho0 * in;
  }
  return M;
}

size_t smem_bytes(int ty) {
  return sizeof(float) * (9 * (ty + 2 * HALO) * SW + 9 * ty * (TX + 1) + 9 * (ty + 1) * TX);
}

}  // namespace

void d2q9_stage_to_float(const D2Q9Stage& s, D2Q9StageF& f) {
  const double* a = &s.wx[0][0][0];
  float* b = &f.wx[0][0][0];
  for (int i = 0; i < 108; ++i) b[i] = (float)a[i];
  a = &s.wy[0][0][0]; b = &f.wy[0][0][0];
  for (int i = 0; i < 108; ++i) b[i] = (float)a[i];
  a = &s.wxL[0][0][0]; b = &f.wxL[0][0][0];
  for (int i = 0; i < 81; ++i) b[i] = (float)a[i];
  a = &s.wxR[0][0][0]; b = &f.wxR[0][0][0];
  for (int i = 0; i < 81; ++i) b[i] = (float)a[i];
  a = &s.wyB[0][0][0]; b = &f.wyB[0][0][0];
  for (int i = 0; i < 81; ++i) b[i] = (float)a[i];
  a = &s.wyT[0][0][0]; b = &f.wyT[0][0][0];
  for (int i = 0; i < 81; ++i) b[i] = (float)a[i];
  f.gamma = (float)s.gamma;
  for (int k = 0; k < 9; ++k) {
    f.kx[k] = (float)s.kx[k];
    f.ky[k] = (float)s.ky[k];
  }
}

cudaError_t d2q9m_prepare() {
  const int bytes = (int)smem_bytes(kMaxTY);
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* fn) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)k_d2q9m<1, float>);
  set((const void*)k_d2q9m<2, float>);
  set((const void*)k_d2q9m<1, __nv_bfloat16>);
  set((const void*)k_d2q9m<2, __nv_bfloat16>);
  return e;
}

// Resident blocks per SM of the deviation-storage stage kernels at tile
// height ty (the smaller of the two stages'; store 1 FP32, else BF16), after
// d2q9m_prepare; 0 on error.
int d2q9m_occupancy(int store, int ty) {
  if (ty < 1 || ty > kMaxTY) return 0;
  const int threads = TX * (ty + 1);
  const size_t bytes = smem_bytes(ty);
  int a = 0, b = 0;
  cudaError_t e;
  if (store == 1) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_d2q9m<1, float>, threads, bytes);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_d2q9m<2, float>, threads, bytes);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_d2q9m<1, __nv_bfloat16>, threads, bytes);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_d2q9m<2, __nv_bfloat16>, threads, bytes);
  }
  return e == cudaSuccess ? (a < b ? a : b) : 0;
}

cudaError_t launch_d2q9m_stage(const D2Q9Params& p, const D2Q9StageF& s, int store, int stage,
                               double rho0, const void* gin, const void* own,
                               const double* rho_in, void* out0, void* out1, double* rho_out,
                               cudaStream_t st_) {
  if (p.ty < 1 || p.ty > kMaxTY) return cudaErrorInvalidValue;
  dim3 grid((p.nx + TX - 1) / TX, (p.ny + p.ty - 1) / p.ty);
  const int threads = TX * (p.ty + 1);
  const size_t bytes = smem_bytes(p.ty);
  // one-wave grids launch as programmatic dependents of the previous kernel
  // (its tail overlaps this grid's launch); multi-wave grids plainly
  // resident blocks per GPU at this form and height, queried once
  static int slots[2][kMaxTY + 1] = {};
  int& sl = slots[store == 1 ? 0 : 1][p.ty];
  if (sl == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int occ = d2q9m_occupancy(store, p.ty);
    sl = sms > 0 && occ > 0 ? sms * occ : -1;
  }
  const bool one_wave = sl > 0 && (long)grid.x * grid.y <= (long)sl;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = st_;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = one_wave ? 1 : 0;
  cudaError_t e;
  if (store == 1) {
    const MixedConst M = mixed_const<float>(p, rho0);
    auto* g = (const float*)gin; auto* o = (const float*)own;
    auto* a = (float*)out0; auto* b = (float*)out1;
    e = cudaLaunchKernelEx(&cfg, stage == 1 ? k_d2q9m<1, float> : k_d2q9m<2, float>, p, s, M, g, o,
                           rho_in, a, b, rho_out);
  } else {
    const MixedConst M = mixed_const<__nv_bfloat16>(p, rho0);
    auto* g = (const __nv_bfloat16*)gin; auto* o = (const __nv_bfloat16*)own;
    auto* a = (__nv_bfloat16*)out0; auto* b = (__nv_bfloat16*)out1;
    e = cudaLaunchKernelEx(&cfg, stage == 1 ? k_d2q9m<1, __nv_bfloat16> : k_d2q9m<2, __nv_bfloat16>,
                           p, s, M, g, o, rho_in, a, b, rho_out);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_dev_from_f64(const DevParams& p, int store, double rho0, const double* f,
                                void* d, cudaStream_t st_) {
  const size_t n = (size_t)p.nv * p.N;
  if (store == 1) k_dev_from_f64<float><<<nblk(n), 256, 0, st_>>>(p, rho0, f, (float*)d);
  else k_dev_from_f64<__nv_bfloat16><<<nblk(n), 256, 0, st_>>>(p, rho0, f, (__nv_bfloat16*)d);
  return cudaGetLastError();
}

cudaError_t launch_f64_from_dev(const DevParams& p, int store, double rho0, const void* d,
                                double* f, cudaStream_t st_) {
  const size_t n = (size_t)p.nv * p.N;
  if (store == 1) k_f64_from_dev<float><<<nblk(n), 256, 0, st_>>>(p, rho0, (const float*)d, f);
  else k_f64_from_dev<__nv_bfloat16><<<nblk(n), 256, 0, st_>>>(p, rho0, (const __nv_bfloat16*)d, f);
  return cudaGetLastError();
}

cudaError_t launch_dev_cell(const DevParams& p, int store, double rho0, const void* d, void* g,
                            double* mom, double a, double b, int write_g, cudaStream_t st_) {
  if (store == 1)
    k_dev_cell<float><<<nblk(p.N), 256, 0, st_>>>(p, rho0, (const float*)d, (float*)g, mom, a, b, write_g);
  else
    k_dev_cell<__nv_bfloat16><<<nblk(p.N), 256, 0, st_>>>(p, rho0, (const __nv_bfloat16*)d,
                                                          (__nv_bfloat16*)g, mom, a, b, write_g);
  return cudaGetLastError();
}

cudaError_t launch_dev_set_eq(const DevParams& p, int store, double rho0, const double* rho,
                              const double* ux, const double* uy, void* d, cudaStream_t st_) {
  const size_t n = (size_t)p.nv * p.N;
  if (store == 1)
    k_dev_set_eq<float><<<nblk(n), 256, 0, st_>>>(p, rho0, rho, ux, uy, (float*)d);
  else
    k_dev_set_eq<__nv_bfloat16><<<nblk(n), 256, 0, st_>>>(p, rho0, rho, ux, uy, (__nv_bfloat16*)d);
  return cudaGetLastError();
}

}  // namespace dugks
