// Fused sm_103a kernels of the T3S3 step for the D2Q9 velocity set, FP64.
//
// GB300 executes FP64 at 2 DFMA per SM per clock, so this path is bound by
// the FP64 pipe, not by HBM: the design minimises FP64 instructions per
// (cell, velocity) update and keeps every intermediate that is not needed by
// a neighbouring tile out of global memory.
//
// One time step = two launches over 32 x ty cell tiles (one thread block per
// tile; ty chosen so the number of tiles fills the 152 SMs):
//   stage 1 kernel: g1 tile (+2-cell halo) -> smem; interface values at
//     t* = t_n + dt/6 for every x- and y-face of the tile (eqs. interfaceEvof,
//     flux_DS; walls of Sec. 2.3; eq. recover2f) -> smem; per cell: L*,
//     f~(t') (eqs. f_tilde_1_3, feqIntD2nd_Explicit), its moments, feq',
//     dt Omega' (eq. collisionterm) and g2 = f-bar^{+,5dt/12}(t'); writes g2
//     and X = f^+ + 3dt/7 L* + 3/4 dt Omega' (eqs. fhp, feqIntD3rdHat2_DS).
//   stage 2 kernel: g2 tile -> interfaces at t** = t_n + 3dt/4 -> per cell
//     f^^{n+1} = X + 4dt/7 L**, then the cell part of the next step's stage 1
//     (moments of f^^{n+1}, feq, g1 = f-bar^{+,dt/6}, eq. f_bar_1_6); writes
//     f^ and g1.
// Interface values are linear in the 3x3 neighbourhood of the upwind cell
// (quadratic Taylor expansion, central differences), so each is a dot
// product with per-(stage, velocity) weights computed on the host; the zero
// pattern of those weights is fixed at compile time per velocity.  The face
// value is kept as f/alpha = f-bar + gamma feq (alpha is folded into the
// flux scale), and equilibria use P = B +- e with B = base + e^2/2.
#include <type_traits>

#include "dugks_fp.cuh"
#include "dugks_internal.cuh"

namespace dugks {

namespace {

constexpr int TX = 32;
constexpr int HALO = 2;
constexpr int SW = TX + 2 * HALO;        // smem tile width
constexpr int kMaxTY = 16;
constexpr int kMaxThreads = TX * (kMaxTY + 1);

// ---------------------------------------------------------------- helpers
template <int K> struct Vel {
  static constexpr int ex = K / 3 - 1;
  static constexpr int ey = K % 3 - 1;
};

// dot product of a weight block with the smem stencil, compile-time extents
template <int R0, int R1, int Q0, int Q1, int NCOL>
__device__ __forceinline__ double wdot(const double* __restrict__ s, const double* w) {
  double acc = 0.0;
#pragma unroll
  for (int r = R0; r <= R1; ++r)
#pragma unroll
    for (int q = Q0; q <= Q1; ++q) {
      const double v = s[r * SW + q];
      acc = (r == R0 && q == Q0) ? w[r * NCOL + q] * v : fma(w[r * NCOL + q], v, acc);
    }
  return acc;
}

// interior x-face value of velocity K; s -> smem (row j-1, col fi-2)
template <int K>
__device__ __forceinline__ double xface_val(const double* __restrict__ s, const D2Q9Stage& S) {
  constexpr int ex = Vel<K>::ex, ey = Vel<K>::ey;
  constexpr int q0 = ex < 0 ? 1 : 0, q1 = ex > 0 ? 2 : 3;
  constexpr int r0 = ey == 0 ? 1 : 0, r1 = ey == 0 ? 1 : 2;
  return wdot<r0, r1, q0, q1, 4>(s, &S.wx[K][0][0]);
}

// interior y-face value of velocity K; s -> smem (row j-2, col i-1); the
// weight block is [row q][col] so rows and columns swap roles
template <int K>
__device__ __forceinline__ double yface_val(const double* __restrict__ s, const D2Q9Stage& S) {
  constexpr int ex = Vel<K>::ex, ey = Vel<K>::ey;
  constexpr int q0 = ey < 0 ? 1 : 0, q1 = ey > 0 ? 2 : 3;
  constexpr int c0 = ex == 0 ? 1 : 0, c1 = ex == 0 ? 1 : 2;
  return wdot<q0, q1, c0, c1, 3>(s, &S.wy[K][0][0]);
}

// Equilibrium polynomials P_k = 1 + e + e^2/2 - |ut|^2 base_div for the nine
// velocities, e = ex ut_x + ey ut_y, in the pair form P(+-e) = B +- e with
// the B of the four velocity pairs from uu = |ut|^2, xx = ut_x^2 and
// p = ut_x ut_y:  B_x = base + xx/2, B_y = base + (uu - xx)/2,
// B_(+-1,+-1) = base + uu/2 + p, B_(+-1,-+1) = base + uu/2 - p.
__device__ __forceinline__ void d2q9_poly(double utx, double uty, const D2Q9Params& Q,
                                          double (&P)[9]) {
  const double xx = utx * utx;
  const double uu = fma(uty, uty, xx);
  const double base = fma(uu, -Q.base_div, 1.0);
  const double bh = fma(uu, Q.half_mb, 1.0);            // base + uu/2
  const double pxy = utx * uty;
  const double bx = fma(0.5, xx, base);
  const double by = fma(-0.5, xx, bh);
  const double bs = bh + pxy, bd = bh - pxy;
  const double sp = utx + uty, sm = utx - uty;
  P[4] = base;
  P[7] = bx + utx;  P[1] = bx - utx;          // (+-1, 0)
  P[5] = by + uty;  P[3] = by - uty;          // (0, +-1)
  P[8] = bs + sp;   P[0] = bs - sp;           // (+1,+1), (-1,-1)
  P[6] = bd + sm;   P[2] = bd - sm;           // (+1,-1), (-1,+1)
}

// s W_k of velocity K.  WS: the weights depend only on |e_k|^2 (rest,
// axis, diagonal), and ws = (s W_rest, s W_axis, s W_diagonal) precomputed;
// otherwise one product per velocity.
template <bool WS, int K>
__device__ __forceinline__ double wk(const D2Q9Params& P, double s, const double (&ws)[3]) {
  if constexpr (WS) return K == 4 ? ws[0] : ((K & 1) ? ws[1] : ws[2]);
  else return s * P.W[K];
}
template <bool WS>
__device__ __forceinline__ void wclasses(const D2Q9Params& P, double s, double (&ws)[3]) {
  if constexpr (WS) {
    ws[0] = s * P.W[4];
    ws[1] = s * P.W[1];
    ws[2] = s * P.W[0];
  } else {
    ws[0] = ws[1] = ws[2] = 0.0;
  }
}

// unrolled loop over the nine velocities with a compile-time index
template <int K = 0, typename F>
__device__ __forceinline__ void for9(F&& f) {
  if constexpr (K < 9) {
    f(std::integral_constant<int, K>{});
    for9<K + 1>(f);
  }
}

// ut = c u / RT from the sums: (c^2/RT) (sx, sy) / rho
__device__ __forceinline__ void d2q9_ut(double rho, double sx, double sy, const D2Q9Params& P,
                                        double& utx, double& uty) {
  const double rc = P.c3 * rcp_fast(rho);
  utx = sx * rc;
  uty = sy * rc;
}

// rho, sx = sum_{ex=1} f - sum_{ex=-1} f, sy likewise
__device__ __forceinline__ void d2q9_sums(const double (&f)[9], double& rho, double& sx, double& sy) {
  const double a = f[0] + f[1] + f[2];     // ex = -1
  const double b = f[6] + f[7] + f[8];     // ex = +1
  rho = (a + b) + (f[3] + f[4] + f[5]);
  sx = b - a;
  sy = (f[2] + f[5] + f[8]) - (f[0] + f[3] + f[6]);
}

// f/alpha = f-bar + gamma feq(moments of f-bar) for one face, in place
template <bool WS>
__device__ __forceinline__ void face_recover(double (&fb)[9], const D2Q9Stage& S,
                                             const D2Q9Params& P) {
  double rho, sx, sy;
  d2q9_sums(fb, rho, sx, sy);
  double utx, uty;
  d2q9_ut(rho, sx, sy, P, utx, uty);
  double Pk[9], ws[3];
  d2q9_poly(utx, uty, P, Pk);
  const double gr = S.gamma * rho;
  wclasses<WS>(P, gr, ws);
  for9([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    fb[k] = fma(wk<WS, k>(P, gr, ws), Pk[k], fb[k]);
  });
}

// Resolve a (possibly ghost) cell to a combination of interior cells:
// periodic wrap, or the quadratic extrapolation along the wall normal
// (g_-1 = 3g_0 - 3g_1 + g_2, g_-2 = 6g_0 - 8g_1 + 3g_2), x then y.
__device__ __forceinline__ int resolve1(int x, int n, bool per, int (&i)[3], double (&c)[3]) {
  if (x >= 0 && x < n) { i[0] = x; c[0] = 1.0; return 1; }
  if (per) { i[0] = ((x % n) + n) % n; c[0] = 1.0; return 1; }
  if (x == -1 || x == n) {
    const int b = x < 0 ? 0 : n - 1, s = x < 0 ? 1 : -1;
    i[0] = b; i[1] = b + s; i[2] = b + 2 * s; c[0] = 3.0; c[1] = -3.0; c[2] = 1.0; return 3;
  }
  if (x == -2 || x == n + 1) {
    const int b = x < 0 ? 0 : n - 1, s = x < 0 ? 1 : -1;
    i[0] = b; i[1] = b + s; i[2] = b + 2 * s; c[0] = 6.0; c[1] = -8.0; c[2] = 3.0; return 3;
  }
  return 0;   // beyond the ghost band: never read by a computed face
}

// ---------------------------------------------------------------- kernel
// One 32 x P.ty tile of one stage (all phases); every thread of the block
// takes part (blockDim.x >= 32 (P.ty + 1)).
template <int STAGE, bool WS>
__device__ __forceinline__ void d2q9_tile(const D2Q9Params& P, const D2Q9Stage& S,
                                          const double* __restrict__ gin,
                                          const double* __restrict__ own,
                                          const double* __restrict__ rho_in,
                                          double* __restrict__ out0, double* __restrict__ out1,
                                          double* __restrict__ rho_out, int x0, int y0,
                                          double* __restrict__ smem) {
  const int TY = P.ty;
  const int SH = TY + 2 * HALO;
  double* sg = smem;                               // [9][SH][SW]
  double* sfx = sg + 9 * SH * SW;                  // [9][TY][TX+1]
  double* sfy = sfx + 9 * TY * (TX + 1);           // [9][TY+1][TX]
  const int nx = P.nx, ny = P.ny, N = P.N;
  const int tid = threadIdx.x, nthr = blockDim.x;

  // phase 0: g tile with a 2-cell halo (wrap or wall ghosts)
  for (int p = tid; p < SH * SW; p += nthr) {
    const int rr = p / SW, cc = p - rr * SW;
    int ix[3], iy[3];
    double cx[3], cy[3];
    const int nxr = resolve1(x0 + cc - HALO, nx, P.px, ix, cx);
    const int nyr = resolve1(y0 + rr - HALO, ny, P.py, iy, cy);
    if (nxr == 1 && nyr == 1) {
      const double* src = gin + iy[0] * nx + ix[0];
#pragma unroll
      for (int k = 0; k < 9; ++k) sg[(k * SH + rr) * SW + cc] = __ldg(src + (size_t)k * N);
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        double v = 0.0;
        for (int a = 0; a < nyr; ++a)
          for (int b = 0; b < nxr; ++b)
            v = fma(cy[a] * cx[b], __ldg(gin + (size_t)k * N + iy[a] * nx + ix[b]), v);
        sg[(k * SH + rr) * SW + cc] = v;
      }
    }
  }
  __syncthreads();

  // phase 1: x-faces fi = x0 + fc, fc = 0..TX, rows r < TY
  for (int t = tid; t < TY * (TX + 1); t += nthr) {
    const int r = t / (TX + 1), fc = t - r * (TX + 1);
    const int j = y0 + r, fi = x0 + fc;
    if (j >= ny || fi > nx) continue;
    double fb[9];
    const double* s0 = sg + (r + 1) * SW + fc;   // row j-1, col fi-2
    const int stride = SH * SW;
    fb[0] = xface_val<0>(s0 + 0 * stride, S);
    fb[1] = xface_val<1>(s0 + 1 * stride, S);
    fb[2] = xface_val<2>(s0 + 2 * stride, S);
    fb[3] = xface_val<3>(s0 + 3 * stride, S);
    fb[4] = xface_val<4>(s0 + 4 * stride, S);
    fb[5] = xface_val<5>(s0 + 5 * stride, S);
    fb[6] = xface_val<6>(s0 + 6 * stride, S);
    fb[7] = xface_val<7>(s0 + 7 * stride, S);
    fb[8] = xface_val<8>(s0 + 8 * stride, S);
    if (!P.px && (fi == 0 || fi == nx)) {
      const bool hi = fi == 0;                    // fluid cell on the +x side (west wall)
      const int side = hi ? SIDE_W : SIDE_E;
      const double rw = rho_in[j * nx + (hi ? 0 : nx - 1)];
      // per-velocity tangential rows need the velocity-k slice
      double fw[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) fw[k] = fb[k];
      // tangential (ex = 0) velocities are k = 3, 4, 5: recompute one-sided
#pragma unroll
      for (int k = 3; k <= 5; ++k) {
        const double(&w)[3][3] = hi ? S.wxR[k] : S.wxL[k];
        const double* sk = s0 + k * stride + (hi ? 1 : 0);
        double v = 0.0;
#pragma unroll
        for (int rr2 = 0; rr2 < 3; ++rr2)
#pragma unroll
          for (int q = 0; q < 3; ++q) v = fma(w[rr2][q], sk[rr2 * SW + q], v);
        fw[k] = v;
      }
      const double nsg = hi ? -1.0 : 1.0;
      if (P.bc_kind[side] == BC_BOUNCEBACK) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k / 3 - 1) < 0) fw[k] = fma(rw, P.bb[side][k], fw[8 - k]);
      } else {
        double num = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k / 3 - 1) > 0) num += fw[k];
        const double rd = num * P.c / P.ds_den[side];
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k / 3 - 1) < 0) fw[k] = rd * P.feq_wall[side][k];
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) fb[k] = fw[k];
    }
    face_recover<WS>(fb, S, P);
#pragma unroll
    for (int k = 0; k < 9; ++k) sfx[(k * TY + r) * (TX + 1) + fc] = fb[k];
  }

  // phase 2: y-faces fj = y0 + fr, fr = 0..TY, cols c < TX
  for (int t = tid; t < (TY + 1) * TX; t += nthr) {
    const int fr = t / TX, c = t - fr * TX;
    const int fj = y0 + fr, i = x0 + c;
    if (i >= nx || fj > ny) continue;
    double fb[9];
    const double* s0 = sg + fr * SW + (c + 1);   // row fj-2, col i-1
    const int stride = SH * SW;
    fb[0] = yface_val<0>(s0 + 0 * stride, S);
    fb[1] = yface_val<1>(s0 + 1 * stride, S);
    fb[2] = yface_val<2>(s0 + 2 * stride, S);
    fb[3] = yface_val<3>(s0 + 3 * stride, S);
    fb[4] = yface_val<4>(s0 + 4 * stride, S);
    fb[5] = yface_val<5>(s0 + 5 * stride, S);
    fb[6] = yface_val<6>(s0 + 6 * stride, S);
    fb[7] = yface_val<7>(s0 + 7 * stride, S);
    fb[8] = yface_val<8>(s0 + 8 * stride, S);
    if (!P.py && (fj == 0 || fj == ny)) {
      const bool hi = fj == 0;                    // fluid cell above (south wall)
      const int side = hi ? SIDE_S : SIDE_N;
      const double rw = rho_in[(hi ? 0 : ny - 1) * nx + i];
      double fw[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) fw[k] = fb[k];
      // tangential (ey = 0) velocities are k = 1, 4, 7
#pragma unroll
      for (int k = 1; k <= 7; k += 3) {
        const double(&w)[3][3] = hi ? S.wyT[k] : S.wyB[k];
        const double* sk = s0 + k * stride + (hi ? SW : 0);
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) v = fma(w[q][cc], sk[q * SW + cc], v);
        fw[k] = v;
      }
      const double nsg = hi ? -1.0 : 1.0;
      if (P.bc_kind[side] == BC_BOUNCEBACK) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k % 3 - 1) < 0) fw[k] = fma(rw, P.bb[side][k], fw[8 - k]);
      } else {
        double num = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k % 3 - 1) > 0) num += fw[k];
        const double rd = num * P.c / P.ds_den[side];
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k % 3 - 1) < 0) fw[k] = rd * P.feq_wall[side][k];
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) fb[k] = fw[k];
    }
    face_recover<WS>(fb, S, P);
#pragma unroll
    for (int k = 0; k < 9; ++k) sfy[(k * (TY + 1) + fr) * TX + c] = fb[k];
  }
  __syncthreads();

  // phase 3: cells
  for (int t = tid; t < TY * TX; t += nthr) {
    const int r = t / TX, c = t - r * TX;
    const int j = y0 + r, i = x0 + c;
    if (j >= ny || i >= nx) continue;
    const int cell = j * nx + i;
    double L[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int ex = k / 3 - 1, ey = k % 3 - 1;
      double v = 0.0;
      if (ex != 0)
        v = S.kx[k] * (sfx[(k * TY + r) * (TX + 1) + c + 1] - sfx[(k * TY + r) * (TX + 1) + c]);
      if (ey != 0) {
        const double d = sfy[(k * (TY + 1) + r + 1) * TX + c] - sfy[(k * (TY + 1) + r) * TX + c];
        v = (ex != 0) ? fma(S.ky[k], d, v) : S.ky[k] * d;
      }
      L[k] = v;
    }
    if (STAGE == 1) {
      // L[k] = dt/3 L*.  f~' = 5/4 g1 - 1/4 f^ + dt/3 L*;  X0 = 1/4 f^ + 3/4 g1 + 3dt/7 L*
      // X0 = f^+ + 3dt/7 L* with L* written through f~' (dt/3 L* = f~' -
      // 5/4 g1 + 1/4 f^):  X0 = r37 f~' + Xg,  Xg = (3/4 - 5/4 r37) g1 +
      // (1/4 + 1/4 r37) f^;  the r37 f~' part joins the c_om34 f~' term below
      const double cg = 0.75 - 1.25 * P.r37, cf = 0.25 + 0.25 * P.r37;
      const double cft = P.c_om34 + P.r37;
      double ft[9], X[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const double g1 = sg[(k * SH + r + HALO) * SW + c + HALO];
        const double fh = __ldg(own + (size_t)k * N + cell);
        ft[k] = fma(1.25, g1, fma(-0.25, fh, L[k]));
        X[k] = fma(cf, fh, cg * g1);
      }
      double rho, sx, sy;
      d2q9_sums(ft, rho, sx, sy);
      double utx, uty;
      d2q9_ut(rho, sx, sy, P, utx, uty);
      double Pk[9], rcw[3], rbw[3];
      d2q9_poly(utx, uty, P, Pk);
      // X += 3/4 dt Omega' = c_om34 (f~' - feq');  g2 = a2 f~' + b2 feq'
      const double rc = -P.c_om34 * rho, rb = P.b2 * rho;
      wclasses<WS>(P, rc, rcw);
      wclasses<WS>(P, rb, rbw);
      for9([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const double xk = fma(cft, ft[k], fma(wk<WS, k>(P, rc, rcw), Pk[k], X[k]));
        const double g2 = fma(wk<WS, k>(P, rb, rbw), Pk[k], P.a2 * ft[k]);
        out0[(size_t)k * N + cell] = g2;
        out1[(size_t)k * N + cell] = xk;
      });
      rho_out[cell] = rho;
    } else {
      // L[k] = 4dt/7 L**.  f^^{n+1} = X + 4dt/7 L**; then g1 of the next step
      double fh[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) fh[k] = __ldg(own + (size_t)k * N + cell) + L[k];
      double rho, sx, sy;
      d2q9_sums(fh, rho, sx, sy);
      double utx, uty;
      d2q9_ut(rho, sx, sy, P, utx, uty);
      double Pk[9], rbw[3];
      d2q9_poly(utx, uty, P, Pk);
      const double rb = P.b1 * rho;
      wclasses<WS>(P, rb, rbw);
      for9([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const double g1 = fma(wk<WS, k>(P, rb, rbw), Pk[k], P.a1 * fh[k]);
        out0[(size_t)k * N + cell] = fh[k];
        out1[(size_t)k * N + cell] = g1;
      });
      rho_out[cell] = rho;
    }
  }
}

template <int STAGE, bool WS>
__global__ void __launch_bounds__(kMaxThreads)
k_d2q9(D2Q9Params P, D2Q9Stage S, const double* __restrict__ gin,
       const double* __restrict__ own, const double* __restrict__ rho_in,
       double* __restrict__ out0, double* __restrict__ out1, double* __restrict__ rho_out) {
  extern __shared__ double smem[];
  d2q9_tile<STAGE, WS>(P, S, gin, own, rho_in, out0, out1, rho_out, blockIdx.x * TX,
                       blockIdx.y * P.ty, smem);
}

// Persistent batched stage kernel: blocks take (instance, tile) work items
// from an atomic counter until all tiles of all instances are done (no
// waiting on other blocks).  Instance parameters and stage tables are read
// through the read-only cache.
template <int STAGE>
__global__ void __launch_bounds__(kMaxThreads, 1)
k_d2q9_batch(const D2Q9BatchItem* __restrict__ items, const int* __restrict__ tile_start,
             int nitems, int* __restrict__ counter) {
  extern __shared__ double smem[];
  __shared__ int s_tile, s_item;
  const int total = tile_start[nitems];
  for (int guard = 0; guard < (1 << 30); ++guard) {
    if (threadIdx.x == 0) {
      const int t = atomicAdd(counter, 1);
      int lo = 0, hi = nitems - 1;
      while (lo < hi) {                 // last item with tile_start <= t
        const int mid = (lo + hi + 1) >> 1;
        if (tile_start[mid] <= t) lo = mid; else hi = mid - 1;
      }
      s_tile = t;
      s_item = lo;
    }
    __syncthreads();
    const int t = s_tile, it = s_item;
    __syncthreads();
    if (t >= total) break;
    const D2Q9BatchItem& I = items[it];
    const int local = t - tile_start[it];
    const int bx = local % I.tiles_x, by = local / I.tiles_x;
    if constexpr (STAGE == 1)
      d2q9_tile<1, false>(I.P, I.S1, I.g1, I.fhat, I.mom, I.g2, I.X, I.mom + I.P.N, bx * TX,
                          by * I.P.ty, smem);
    else
      d2q9_tile<2, false>(I.P, I.S2, I.g2, I.X, I.mom + I.P.N, I.fhat, I.g1, I.mom, bx * TX,
                          by * I.P.ty, smem);
    __syncthreads();
  }
}

}  // namespace

size_t d2q9_smem_bytes(int ty) {
  return sizeof(double) * (9 * (ty + 2 * HALO) * SW + 9 * ty * (TX + 1) + 9 * (ty + 1) * TX);
}

cudaError_t d2q9_prepare(int ty) {
  // the attribute is per function: always allow the largest tile so that
  // contexts with different tile heights can coexist
  (void)ty;
  const int bytes = (int)d2q9_smem_bytes(kMaxTY);
  cudaError_t e = cudaFuncSetAttribute(k_d2q9<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_d2q9<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_d2q9<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_d2q9<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_d2q9_batch<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_d2q9_batch<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

cudaError_t launch_d2q9_batch(int stage, const D2Q9BatchItem* items, const int* tile_start,
                              int nitems, int max_ty, int* counter, int blocks, cudaStream_t st) {
  const int threads = TX * (max_ty + 1);
  const size_t bytes = d2q9_smem_bytes(max_ty);
  if (stage == 1) k_d2q9_batch<1><<<blocks, threads, bytes, st>>>(items, tile_start, nitems, counter);
  else k_d2q9_batch<2><<<blocks, threads, bytes, st>>>(items, tile_start, nitems, counter);
  return cudaGetLastError();
}

int d2q9_batch_blocks_per_sm(int max_ty) {
  int n = 0;
  const int threads = TX * (max_ty + 1);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_d2q9_batch<1>, threads, d2q9_smem_bytes(max_ty));
  return n < 1 ? 1 : n;
}

cudaError_t launch_d2q9_stage(const D2Q9Params& p, const D2Q9Stage& s, int stage,
                              const double* gin, const double* own, const double* rho_in,
                              double* out0, double* out1, double* rho_out, cudaStream_t st) {
  if (p.ty < 1 || p.ty > kMaxTY) return cudaErrorInvalidValue;
  dim3 grid((p.nx + TX - 1) / TX, (p.ny + p.ty - 1) / p.ty);
  const int threads = TX * (p.ty + 1);
  const size_t bytes = d2q9_smem_bytes(p.ty);
  if (p.wsym) {
    if (stage == 1)
      k_d2q9<1, true><<<grid, threads, bytes, st>>>(p, s, gin, own, rho_in, out0, out1, rho_out);
    else
      k_d2q9<2, true><<<grid, threads, bytes, st>>>(p, s, gin, own, rho_in, out0, out1, rho_out);
  } else {
    if (stage == 1)
      k_d2q9<1, false><<<grid, threads, bytes, st>>>(p, s, gin, own, rho_in, out0, out1, rho_out);
    else
      k_d2q9<2, false><<<grid, threads, bytes, st>>>(p, s, gin, own, rho_in, out0, out1, rho_out);
  }
  return cudaGetLastError();
}

}  // namespace dugks
