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
//
// The tile code is written once over its arithmetic type A: double (the
// FP64 kernels) or dw, double-word FP32 pairs (dugks_dw.cuh), which keep FP64
// arrays but run every operation on the FP32 pipes -- GB300 issues those at
// 64 times its FP64 rate -- with a unit roundoff of 2^-48 instead of 2^-53.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "dugks_dw.cuh"
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

// Arithmetic of the tile code.  Par / Stg: the parameter structs in that
// arithmetic; load / store: FP64 memory <-> A; cst: an FP32-exact constant;
// rcp: 1/x; diffuse: the diffuse wall density factor num c / ds_den.
template <typename A> struct Arith;
template <> struct Arith<double> {
  // tiles up to 32 x 16, one block per SM (no minimum given to the compiler)
  static constexpr int kMaxTY = 16, kThreads = TX * (kMaxTY + 1), kMinBlocks = 0;
  using Par = D2Q9Params;
  using Stg = D2Q9Stage;
  using Acc = double;
  static __device__ __forceinline__ double load(const double* p) { return __ldg(p); }
  static __device__ __forceinline__ double store(double x) { return x; }
  static __device__ __forceinline__ double cst(float x) { return (double)x; }
  // ghost extrapolation coefficients (small integers, exact in FP32),
  // converted on the integer pipe
  static __device__ __forceinline__ double coef(float x) { return f2d_bits(x); }
  static __device__ __forceinline__ double rcp(double x) { return rcp_fast(x); }
  static __device__ __forceinline__ double diffuse(double num, const Par& P, int side) {
    return num * P.c / P.ds_den[side];
  }
  static __device__ __forceinline__ void dot_first(double& a, double w, double v) { a = w * v; }
  static __device__ __forceinline__ void dot_add(double& a, double w, double v) { a = fma(w, v, a); }
  static __device__ __forceinline__ double dot_value(double a) { return a; }
};
template <> struct Arith<dw> {
  // tiles up to 32 x 12 so that two blocks share an SM (2 x 100 KB of
  // shared memory, <= 72 registers per thread): one block's phase barriers
  // and instruction fetches overlap the other's arithmetic
  static constexpr int kMaxTY = 12, kThreads = TX * (kMaxTY + 1), kMinBlocks = 2;
  using Par = D2Q9ParamsDW;
  using Stg = D2Q9StageDW;
  using Acc = dw_acc;
  static __device__ __forceinline__ dw load(const double* p) { return dw_from_d(__ldg(p)); }
  static __device__ __forceinline__ double store(dw x) { return dw_to_d(x); }
  static __device__ __forceinline__ dw cst(float x) { return dw{x, 0.0f}; }
  // ghost extrapolation coefficients (small integers, exact in FP32)
  static __device__ __forceinline__ dw coef(float x) { return dw{x, 0.0f}; }
  static __device__ __forceinline__ dw rcp(dw x) { return dw_rcp(x); }
  static __device__ __forceinline__ dw diffuse(dw num, const Par& P, int side) {
    return num * P.c_ds[side];
  }
  static __device__ __forceinline__ void dot_first(dw_acc& a, dw w, dw v) { dw_acc_first(a, w, v); }
  static __device__ __forceinline__ void dot_add(dw_acc& a, dw w, dw v) { dw_acc_add(a, w, v); }
  static __device__ __forceinline__ dw dot_value(const dw_acc& a) { return dw_acc_value(a); }
};

// dot product of a weight block with the smem stencil, compile-time extents.
// The double-word form keeps the rows after the first in a loop: its
// stage code is bound by instruction fetch, and a rolled row is a third of
// the code for a few loop instructions.
template <typename A, int R0, int R1, int Q0, int Q1, int NCOL>
__device__ __forceinline__ A wdot(const A* __restrict__ s, const A* w) {
  typename Arith<A>::Acc acc;
  if constexpr (std::is_same<A, dw>::value) {
#pragma unroll
    for (int q = Q0; q <= Q1; ++q) {
      if (q == Q0) Arith<A>::dot_first(acc, w[R0 * NCOL + q], s[R0 * SW + q]);
      else Arith<A>::dot_add(acc, w[R0 * NCOL + q], s[R0 * SW + q]);
    }
#pragma unroll 1
    for (int r = R0 + 1; r <= R1; ++r)
#pragma unroll
      for (int q = Q0; q <= Q1; ++q) Arith<A>::dot_add(acc, w[r * NCOL + q], s[r * SW + q]);
  } else {
#pragma unroll
    for (int r = R0; r <= R1; ++r)
#pragma unroll
      for (int q = Q0; q <= Q1; ++q) {
        const A v = s[r * SW + q];
        if (r == R0 && q == Q0) Arith<A>::dot_first(acc, w[r * NCOL + q], v);
        else Arith<A>::dot_add(acc, w[r * NCOL + q], v);
      }
  }
  return Arith<A>::dot_value(acc);
}

// interior x-face value of velocity K; s -> smem (row j-1, col fi-2)
template <typename A, int K>
__device__ __forceinline__ A xface_val(const A* __restrict__ s, const typename Arith<A>::Stg& S) {
  constexpr int ex = Vel<K>::ex, ey = Vel<K>::ey;
  constexpr int q0 = ex < 0 ? 1 : 0, q1 = ex > 0 ? 2 : 3;
  constexpr int r0 = ey == 0 ? 1 : 0, r1 = ey == 0 ? 1 : 2;
  return wdot<A, r0, r1, q0, q1, 4>(s, &S.wx[K][0][0]);
}

// interior y-face value of velocity K; s -> smem (row j-2, col i-1); the
// weight block is [row q][col] so rows and columns swap roles
template <typename A, int K>
__device__ __forceinline__ A yface_val(const A* __restrict__ s, const typename Arith<A>::Stg& S) {
  constexpr int ex = Vel<K>::ex, ey = Vel<K>::ey;
  constexpr int q0 = ey < 0 ? 1 : 0, q1 = ey > 0 ? 2 : 3;
  constexpr int c0 = ex == 0 ? 1 : 0, c1 = ex == 0 ? 1 : 2;
  return wdot<A, q0, q1, c0, c1, 3>(s, &S.wy[K][0][0]);
}

// Equilibrium polynomials P_k = 1 + e + e^2/2 - |ut|^2 base_div for the nine
// velocities, e = ex ut_x + ey ut_y, in the pair form P(+-e) = B +- e with
// the B of the four velocity pairs from uu = |ut|^2, xx = ut_x^2 and
// p = ut_x ut_y:  B_x = base + xx/2, B_y = base + (uu - xx)/2,
// B_(+-1,+-1) = base + uu/2 + p, B_(+-1,-+1) = base + uu/2 - p.
template <typename A>
__device__ __forceinline__ void d2q9_poly(A utx, A uty, const typename Arith<A>::Par& Q,
                                          A (&P)[9]) {
  using R = Arith<A>;
  const A xx = utx * utx;
  const A uu = fma(uty, uty, xx);
  const A base = fma(uu, -Q.base_div, R::cst(1.0f));
  const A bh = fma(uu, Q.half_mb, R::cst(1.0f));        // base + uu/2
  const A pxy = utx * uty;
  const A bx = fma(R::cst(0.5f), xx, base);
  const A by = fma(R::cst(-0.5f), xx, bh);
  const A bs = bh + pxy, bd = bh - pxy;
  const A sp = utx + uty, sm = utx - uty;
  P[4] = base;
  P[7] = bx + utx;  P[1] = bx - utx;          // (+-1, 0)
  P[5] = by + uty;  P[3] = by - uty;          // (0, +-1)
  P[8] = bs + sp;   P[0] = bs - sp;           // (+1,+1), (-1,-1)
  P[6] = bd + sm;   P[2] = bd - sm;           // (+1,-1), (-1,+1)
}

// s W_k of velocity K.  WS: the weights depend only on |e_k|^2 (rest,
// axis, diagonal), and ws = (s W_rest, s W_axis, s W_diagonal) precomputed;
// otherwise one product per velocity.
template <bool WS, int K, typename A>
__device__ __forceinline__ A wk(const typename Arith<A>::Par& P, A s, const A (&ws)[3]) {
  if constexpr (WS) return K == 4 ? ws[0] : ((K & 1) ? ws[1] : ws[2]);
  else return s * P.W[K];
}
template <bool WS, typename A>
__device__ __forceinline__ void wclasses(const typename Arith<A>::Par& P, A s, A (&ws)[3]) {
  if constexpr (WS) {
    ws[0] = s * P.W[4];
    ws[1] = s * P.W[1];
    ws[2] = s * P.W[0];
  } else {
    ws[0] = ws[1] = ws[2] = Arith<A>::cst(0.0f);
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

// velocity K crosses a face of direction DIR (0: x, 1: y)
template <int DIR, int K>
__device__ __forceinline__ constexpr bool crosses() {
  return DIR == 0 ? (K / 3 != 1) : (K % 3 != 1);
}

// ut = c u / RT from the sums: (c^2/RT) (sx, sy) / rho
template <typename A>
__device__ __forceinline__ void d2q9_ut(A rho, A sx, A sy, const typename Arith<A>::Par& P,
                                        A& utx, A& uty) {
  const A rc = P.c3 * Arith<A>::rcp(rho);
  utx = sx * rc;
  uty = sy * rc;
}

// rho, sx = sum_{ex=1} f - sum_{ex=-1} f, sy likewise
template <typename A>
__device__ __forceinline__ void d2q9_sums(const A (&f)[9], A& rho, A& sx, A& sy) {
  const A a = f[0] + f[1] + f[2];          // ex = -1
  const A b = f[6] + f[7] + f[8];          // ex = +1
  rho = (a + b) + (f[3] + f[4] + f[5]);
  sx = b - a;
  sy = (f[2] + f[5] + f[8]) - (f[0] + f[3] + f[6]);
}

// f/alpha = f-bar + gamma feq(moments of f-bar) for one face of direction
// DIR (0: x-face, 1: y-face), in place.  The moments take all nine f-bar;
// the flux through the face only the velocities that cross it, so the
// tangential ones (e_x = 0 at an x-face, e_y = 0 at a y-face) keep f-bar.
template <bool WS, int DIR, typename A>
__device__ __forceinline__ void face_recover(A (&fb)[9], const typename Arith<A>::Stg& S,
                                             const typename Arith<A>::Par& P) {
  A rho, sx, sy;
  d2q9_sums(fb, rho, sx, sy);
  A utx, uty;
  d2q9_ut(rho, sx, sy, P, utx, uty);
  A Pk[9], ws[3];
  d2q9_poly(utx, uty, P, Pk);
  const A gr = S.gamma * rho;
  wclasses<WS>(P, gr, ws);
  for9([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (crosses<DIR, k>()) fb[k] = fma(wk<WS, k>(P, gr, ws), Pk[k], fb[k]);
  });
}

// A staged coordinate x of a tile with its 2-cell halo: >= 0 the cell it
// holds (in the domain, or its periodic image); -1 a wall ghost; -2 beyond
// the ghost band (never read by a computed face).
__device__ __forceinline__ int stage_coord(int x, int n, bool per) {
  if (x >= 0 && x < n) return x;
  if (per) return ((x % n) + n) % n;
  return (x >= -2 && x <= n + 1) ? -1 : -2;
}

// Taps of a staged coordinate for the ghost fill, as positions in the
// staged tile (t0 = tile origin, s = this position): itself with weight 1
// when it holds a cell, else the three cells next to the wall with the
// weights of the quadratic extrapolation along the wall normal
// (g_-1 = 3g_0 - 3g_1 + g_2, g_-2 = 6g_0 - 8g_1 + 3g_2).  Walls need three
// cells across, and a tile holding a ghost holds those three cells too.
// The weights and their products are exact in FP32.
__device__ __forceinline__ int ghost_taps(int x, int ix, int n, int t0, int s, int (&pos)[3],
                                          float (&c)[3]) {
  if (ix >= 0) { pos[0] = s; c[0] = 1.0f; return 1; }
  const int b = x < 0 ? 0 : n - 1, d = x < 0 ? 1 : -1;
  const bool near = x == -1 || x == n;
  c[0] = near ? 3.0f : 6.0f;
  c[1] = near ? -3.0f : -8.0f;
  c[2] = near ? 1.0f : 3.0f;
#pragma unroll
  for (int m = 0; m < 3; ++m) pos[m] = b + m * d - t0 + HALO;
  return 3;
}

// Cell part of a stage in double-word arithmetic.  The maps are written so
// that a uniform equilibrium passes every one of them exactly whatever the
// rounding of the coefficients: g = f + b (feq - f) instead of a f + b feq
// (a + b = 1 holds in FP64 to 2^-53 but only to 2^-49 for coefficients
// split into FP32 pairs, a bias that would accumulate step after step), and
// X = f^/4 + 3 g1/4 + r37 (dt/3 L*) + c_om34 (f~' - feq') with the 3dt/7 L*
// term taken from the flux itself (eq. fhp; 3dt/7 = r37 dt/3).
template <int STAGE, bool WS>
__device__ __forceinline__ void d2q9_cell_dw(const D2Q9ParamsDW& P, const dw (&L)[9],
                                             const dw* __restrict__ sg,
                                             const double* __restrict__ own,
                                             double* __restrict__ out0, double* __restrict__ out1,
                                             double* __restrict__ rho_out, int cell, int N,
                                             int SH, int r, int c) {
  using R = Arith<dw>;
  dw f[9], X[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const dw fh = R::load(own + (size_t)k * N + cell);
    if (STAGE == 1) {
      // L[k] = dt/3 L*: f~' = 5/4 g1 - 1/4 f^ + dt/3 L*
      const dw g1 = sg[(k * SH + r + HALO) * SW + c + HALO];
      f[k] = fma(R::cst(1.25f), g1, fma(R::cst(-0.25f), fh, L[k]));
      X[k] = fma(P.r37, L[k], fma(R::cst(0.25f), fh, R::cst(0.75f) * g1));
    } else {
      // L[k] = 4dt/7 L**: f^^{n+1} = X + 4dt/7 L**
      f[k] = fh + L[k];
    }
  }
  dw rho, sx, sy;
  d2q9_sums(f, rho, sx, sy);
  dw utx, uty;
  d2q9_ut(rho, sx, sy, P, utx, uty);
  dw Pk[9], rw[3];
  d2q9_poly(utx, uty, P, Pk);
  wclasses<WS>(P, rho, rw);
  const dw b = STAGE == 1 ? P.b2 : P.b1;
  for9([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const dw d = wk<WS, k>(P, rho, rw) * Pk[k] - f[k];      // feq - f
    const dw g = fma(b, d, f[k]);                           // g2 (stage 1) or g1
    if (STAGE == 1) {
      out0[(size_t)k * N + cell] = R::store(g);
      out1[(size_t)k * N + cell] = R::store(fma(-P.c_om34, d, X[k]));
    } else {
      out0[(size_t)k * N + cell] = R::store(f[k]);
      out1[(size_t)k * N + cell] = R::store(g);
    }
  });
  rho_out[cell] = R::store(rho);
}

// ---------------------------------------------------------------- kernel
// One 32 x P.ty tile of one stage (all phases); every thread of the block
// takes part (blockDim.x >= 32 (P.ty + 1)).
// FT (stage 1, FP64): out1 receives f~(t') itself instead of X (the
// adjoint's recomputation of the forward intermediates).
template <int STAGE, bool WS, typename A, bool FT = false>
__device__ __forceinline__ void d2q9_tile(const typename Arith<A>::Par& P,
                                          const typename Arith<A>::Stg& S,
                                          const double* __restrict__ gin,
                                          const double* __restrict__ own,
                                          const double* __restrict__ rho_in,
                                          double* __restrict__ out0, double* __restrict__ out1,
                                          double* __restrict__ rho_out, int x0, int y0,
                                          A* __restrict__ smem) {
  using R = Arith<A>;
  const int TY = P.ty;
  const int SH = TY + 2 * HALO;
  A* sg = smem;                                    // [9][SH][SW]
  A* sfx = sg + 9 * SH * SW;                       // [9][TY][TX+1]
  A* sfy = sfx + 9 * TY * (TX + 1);                // [9][TY+1][TX]
  const int nx = P.nx, ny = P.ny, N = P.N;
  const int tid = threadIdx.x, nthr = blockDim.x;

  // launched as a programmatic dependent of the previous stage kernel: wait
  // for it to complete (no-op otherwise) before reading its outputs
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // phase 0: g tile with a 2-cell halo.  (a) Cells of the domain and their
  // periodic images from global memory (beyond the ghost band: zero);
  // (b) wall ghosts, extrapolated from the cells staged in (a), so that no
  // ghost waits on a chain of global loads (a wall tile otherwise spent
  // 10 us of a 66 us stage here at 256^2, and the stage waits for it).
  for (int p = tid; p < SH * SW; p += nthr) {
    const int rr = p / SW, cc = p - rr * SW;
    const int ix = stage_coord(x0 + cc - HALO, nx, P.px);
    const int iy = stage_coord(y0 + rr - HALO, ny, P.py);
    if (ix >= 0 && iy >= 0) {
      const double* src = gin + iy * nx + ix;
#pragma unroll
      for (int k = 0; k < 9; ++k) sg[(k * SH + rr) * SW + cc] = R::load(src + (size_t)k * N);
    } else if (ix == -2 || iy == -2) {
#pragma unroll
      for (int k = 0; k < 9; ++k) sg[(k * SH + rr) * SW + cc] = R::cst(0.0f);
    }
  }
  // (b) one (ghost, velocity) pair per thread, so that the FP64 work fills
  // whole warps: ghost columns (x beyond a wall; every row of the band,
  // corners included), then ghost rows (y beyond a wall; columns that hold
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
      A v = R::cst(0.0f);
      for (int a = 0; a < nyr; ++a)
        for (int b = 0; b < nxr; ++b)
          v = fma(R::coef(cy[a] * cx[b]), sg[(k * SH + pr[a]) * SW + pc[b]], v);
      sg[(k * SH + rr) * SW + cc] = v;
    }
  }
  __syncthreads();
  // this block's inputs are in shared memory: the next stage kernel may
  // begin launching (it waits for this grid's completion before reading)
  asm volatile("griddepcontrol.launch_dependents;");

  // phase 1: x-faces fi = x0 + fc, fc = 0..TX, rows r < TY.  Wall faces
  // (fi = 0 or nx; more work) are taken by threads after all the others, so
  // that with one wall column every other warp takes one row of 32
  // interior faces and none diverges on a wall face.
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
    A fb[9];
    const A* s0 = sg + (r + 1) * SW + fc;   // row j-1, col fi-2
    const int stride = SH * SW;
    if (P.px || (fi != 0 && fi != nx)) {
      fb[0] = xface_val<A, 0>(s0 + 0 * stride, S);
      fb[1] = xface_val<A, 1>(s0 + 1 * stride, S);
      fb[2] = xface_val<A, 2>(s0 + 2 * stride, S);
      fb[3] = xface_val<A, 3>(s0 + 3 * stride, S);
      fb[4] = xface_val<A, 4>(s0 + 4 * stride, S);
      fb[5] = xface_val<A, 5>(s0 + 5 * stride, S);
      fb[6] = xface_val<A, 6>(s0 + 6 * stride, S);
      fb[7] = xface_val<A, 7>(s0 + 7 * stride, S);
      fb[8] = xface_val<A, 8>(s0 + 8 * stride, S);
    } else {
      // wall face: only the velocities that leave the fluid toward the wall
      // take the interior stencil; the tangential ones (e_x = 0, k = 3..5)
      // take the one-sided one on the fluid side, and the ones entering the
      // fluid come from the wall condition (eq. BB or diffuse scattering)
      const bool hi = fi == 0;                    // fluid cell on the +x side (west wall)
      const int side = hi ? SIDE_W : SIDE_E;
      const A rw = R::load(rho_in + j * nx + (hi ? 0 : nx - 1));
      if (hi) {
        fb[0] = xface_val<A, 0>(s0 + 0 * stride, S);
        fb[1] = xface_val<A, 1>(s0 + 1 * stride, S);
        fb[2] = xface_val<A, 2>(s0 + 2 * stride, S);
      } else {
        fb[6] = xface_val<A, 6>(s0 + 6 * stride, S);
        fb[7] = xface_val<A, 7>(s0 + 7 * stride, S);
        fb[8] = xface_val<A, 8>(s0 + 8 * stride, S);
      }
#pragma unroll
      for (int k = 3; k <= 5; ++k) {
        const A(&w)[3][3] = hi ? S.wxR[k] : S.wxL[k];
        const A* sk = s0 + k * stride + (hi ? 1 : 0);
        A v = R::cst(0.0f);
#pragma unroll
        for (int rr2 = 0; rr2 < 3; ++rr2)
#pragma unroll
          for (int q = 0; q < 3; ++q) v = fma(w[rr2][q], sk[rr2 * SW + q], v);
        fb[k] = v;
      }
      const int nsg = hi ? -1 : 1;
      if (P.bc_kind[side] == BC_BOUNCEBACK) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k / 3 - 1) < 0) fb[k] = fma(rw, P.bb[side][k], fb[8 - k]);
      } else {
        A num = R::cst(0.0f);
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k / 3 - 1) > 0) num = num + fb[k];
        const A rd = R::diffuse(num, P, side);
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k / 3 - 1) < 0) fb[k] = rd * P.feq_wall[side][k];
      }
    }
    face_recover<WS, 0>(fb, S, P);
    // only the velocities that cross the face are read back (cell phase)
    for9([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (crosses<0, k>()) sfx[(k * TY + r) * (TX + 1) + fc] = fb[k];
    });
  }

  // phase 2: y-faces fj = y0 + fr, fr = 0..TY, cols c < TX
  for (int t = tid; t < (TY + 1) * TX; t += nthr) {
    const int fr = t / TX, c = t - fr * TX;
    const int fj = y0 + fr, i = x0 + c;
    if (i >= nx || fj > ny) continue;
    A fb[9];
    const A* s0 = sg + fr * SW + (c + 1);   // row fj-2, col i-1
    const int stride = SH * SW;
    if (P.py || (fj != 0 && fj != ny)) {
      fb[0] = yface_val<A, 0>(s0 + 0 * stride, S);
      fb[1] = yface_val<A, 1>(s0 + 1 * stride, S);
      fb[2] = yface_val<A, 2>(s0 + 2 * stride, S);
      fb[3] = yface_val<A, 3>(s0 + 3 * stride, S);
      fb[4] = yface_val<A, 4>(s0 + 4 * stride, S);
      fb[5] = yface_val<A, 5>(s0 + 5 * stride, S);
      fb[6] = yface_val<A, 6>(s0 + 6 * stride, S);
      fb[7] = yface_val<A, 7>(s0 + 7 * stride, S);
      fb[8] = yface_val<A, 8>(s0 + 8 * stride, S);
    } else {
      // wall face (a whole warp: one row of faces): leaving velocities from
      // the interior stencil, tangential ones (e_y = 0, k = 1, 4, 7)
      // one-sided, entering ones from the wall condition
      const bool hi = fj == 0;                    // fluid cell above (south wall)
      const int side = hi ? SIDE_S : SIDE_N;
      const A rw = R::load(rho_in + (hi ? 0 : ny - 1) * nx + i);
      if (hi) {
        fb[0] = yface_val<A, 0>(s0 + 0 * stride, S);
        fb[3] = yface_val<A, 3>(s0 + 3 * stride, S);
        fb[6] = yface_val<A, 6>(s0 + 6 * stride, S);
      } else {
        fb[2] = yface_val<A, 2>(s0 + 2 * stride, S);
        fb[5] = yface_val<A, 5>(s0 + 5 * stride, S);
        fb[8] = yface_val<A, 8>(s0 + 8 * stride, S);
      }
#pragma unroll
      for (int k = 1; k <= 7; k += 3) {
        const A(&w)[3][3] = hi ? S.wyT[k] : S.wyB[k];
        const A* sk = s0 + k * stride + (hi ? SW : 0);
        A v = R::cst(0.0f);
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) v = fma(w[q][cc], sk[q * SW + cc], v);
        fb[k] = v;
      }
      const int nsg = hi ? -1 : 1;
      if (P.bc_kind[side] == BC_BOUNCEBACK) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k % 3 - 1) < 0) fb[k] = fma(rw, P.bb[side][k], fb[8 - k]);
      } else {
        A num = R::cst(0.0f);
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k % 3 - 1) > 0) num = num + fb[k];
        const A rd = R::diffuse(num, P, side);
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (nsg * (k % 3 - 1) < 0) fb[k] = rd * P.feq_wall[side][k];
      }
    }
    face_recover<WS, 1>(fb, S, P);
    for9([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (crosses<1, k>()) sfy[(k * (TY + 1) + fr) * TX + c] = fb[k];
    });
  }
  __syncthreads();

  // phase 3: cells
  for (int t = tid; t < TY * TX; t += nthr) {
    const int r = t / TX, c = t - r * TX;
    const int j = y0 + r, i = x0 + c;
    if (j >= ny || i >= nx) continue;
    const int cell = j * nx + i;
    A L[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int ex = k / 3 - 1, ey = k % 3 - 1;
      A v = R::cst(0.0f);
      if (ex != 0)
        v = S.kx[k] * (sfx[(k * TY + r) * (TX + 1) + c + 1] - sfx[(k * TY + r) * (TX + 1) + c]);
      if (ey != 0) {
        const A d = sfy[(k * (TY + 1) + r + 1) * TX + c] - sfy[(k * (TY + 1) + r) * TX + c];
        v = (ex != 0) ? fma(S.ky[k], d, v) : S.ky[k] * d;
      }
      L[k] = v;
    }
    if constexpr (std::is_same<A, dw>::value) {
      d2q9_cell_dw<STAGE, WS>(P, L, sg, own, out0, out1, rho_out, cell, N, SH, r, c);
    } else if (STAGE == 1) {
      // L[k] = dt/3 L*.  f~' = 5/4 g1 - 1/4 f^ + dt/3 L*;  X0 = 1/4 f^ + 3/4 g1 + 3dt/7 L*
      // X0 = f^+ + 3dt/7 L* with L* written through f~' (dt/3 L* = f~' -
      // 5/4 g1 + 1/4 f^):  X0 = r37 f~' + Xg,  Xg = (3/4 - 5/4 r37) g1 +
      // (1/4 + 1/4 r37) f^;  the r37 f~' part joins the c_om34 f~' term below
      const A cg = R::cst(0.75f) - R::cst(1.25f) * P.r37, cf = R::cst(0.25f) + R::cst(0.25f) * P.r37;
      const A cft = P.c_om34 + P.r37;
      A ft[9], X[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const A g1 = sg[(k * SH + r + HALO) * SW + c + HALO];
        const A fh = R::load(own + (size_t)k * N + cell);
        ft[k] = fma(R::cst(1.25f), g1, fma(R::cst(-0.25f), fh, L[k]));
        X[k] = fma(cf, fh, cg * g1);
      }
      A rho, sx, sy;
      d2q9_sums(ft, rho, sx, sy);
      A utx, uty;
      d2q9_ut(rho, sx, sy, P, utx, uty);
      A Pk[9], rcw[3], rbw[3];
      d2q9_poly(utx, uty, P, Pk);
      // X += 3/4 dt Omega' = c_om34 (f~' - feq');  g2 = a2 f~' + b2 feq'
      const A rc = -P.c_om34 * rho, rb = P.b2 * rho;
      wclasses<WS>(P, rc, rcw);
      wclasses<WS>(P, rb, rbw);
      for9([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const A xk = fma(cft, ft[k], fma(wk<WS, k>(P, rc, rcw), Pk[k], X[k]));
        const A g2 = fma(wk<WS, k>(P, rb, rbw), Pk[k], P.a2 * ft[k]);
        out0[(size_t)k * N + cell] = R::store(g2);
        out1[(size_t)k * N + cell] = R::store(FT ? ft[k] : xk);
      });
      rho_out[cell] = R::store(rho);
    } else {
      // L[k] = 4dt/7 L**.  f^^{n+1} = X + 4dt/7 L**; then g1 of the next step
      A fh[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) fh[k] = R::load(own + (size_t)k * N + cell) + L[k];
      A rho, sx, sy;
      d2q9_sums(fh, rho, sx, sy);
      A utx, uty;
      d2q9_ut(rho, sx, sy, P, utx, uty);
      A Pk[9], rbw[3];
      d2q9_poly(utx, uty, P, Pk);
      const A rb = P.b1 * rho;
      wclasses<WS>(P, rb, rbw);
      for9([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const A g1 = fma(wk<WS, k>(P, rb, rbw), Pk[k], P.a1 * fh[k]);
        out0[(size_t)k * N + cell] = R::store(fh[k]);
        out1[(size_t)k * N + cell] = R::store(g1);
      });
      rho_out[cell] = R::store(rho);
    }
  }
}

// the stage tables stay in parameter space when the double-word stencil
// indexes its rows at run time
template <int STAGE, bool WS, typename A>
__global__ void __launch_bounds__(Arith<A>::kThreads, Arith<A>::kMinBlocks)
k_d2q9(typename Arith<A>::Par P, const __grid_constant__ typename Arith<A>::Stg S,
       const double* __restrict__ gin,
       const double* __restrict__ own, const double* __restrict__ rho_in,
       double* __restrict__ out0, double* __restrict__ out1, double* __restrict__ rho_out) {
  extern __shared__ double smem[];
  static_assert(sizeof(A) == sizeof(double), "tile buffers are sized for 8-byte values");
  d2q9_tile<STAGE, WS, A>(P, S, gin, own, rho_in, out0, out1, rho_out, blockIdx.x * TX,
                          blockIdx.y * P.ty, reinterpret_cast<A*>(smem));
}

// The g1 prologue of the double-word form, in the arithmetic and order of
// its stage-2 tail (d2q9_cell_dw), so that a run restarted from its state
// continues as it would have: g1 = f + b1 (feq - f), and the moments.
template <bool WS>
__global__ void __launch_bounds__(256)
k_d2q9dw_cell(D2Q9ParamsDW P, const double* __restrict__ fhat, double* __restrict__ g1,
              double* __restrict__ mom) {
  using R = Arith<dw>;
  const int N = P.N;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= N) return;
  dw f[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) f[k] = R::load(fhat + (size_t)k * N + cell);
  dw rho, sx, sy;
  d2q9_sums(f, rho, sx, sy);
  dw utx, uty;
  d2q9_ut(rho, sx, sy, P, utx, uty);
  dw Pk[9], rw[3];
  d2q9_poly(utx, uty, P, Pk);
  wclasses<WS>(P, rho, rw);
  for9([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const dw d = wk<WS, k>(P, rho, rw) * Pk[k] - f[k];
    g1[(size_t)k * N + cell] = R::store(fma(P.b1, d, f[k]));
  });
  const dw cr = P.c * R::rcp(rho);
  mom[cell] = R::store(rho);
  mom[N + cell] = R::store(sx * cr);
  mom[2 * N + cell] = R::store(sy * cr);
}

// Stage 1 with f~(t') as the second output (see d2q9_tile's FT).
template <bool WS>
__global__ void __launch_bounds__(kMaxThreads)
k_d2q9_ftp(D2Q9Params P, D2Q9Stage S, const double* __restrict__ gin,
           const double* __restrict__ own, const double* __restrict__ rho_in,
           double* __restrict__ out0, double* __restrict__ out1, double* __restrict__ rho_out) {
  extern __shared__ double smem[];
  d2q9_tile<1, WS, double, true>(P, S, gin, own, rho_in, out0, out1, rho_out, blockIdx.x * TX,
                                 blockIdx.y * P.ty, smem);
}

// Cell pass of the fused path outside a step, one thread per cell: the
// moments of f^ (rho, ux, uy; Sec. 2.2) into mom[3][N] and, with G, g1 =
// f-bar^{+,dt/6} of eq. f_bar_1_6 in the stage-2 kernel's own arithmetic
// (the prologue after a new state).
template <bool G, bool WS>
__global__ void __launch_bounds__(256)
k_d2q9_cell(D2Q9Params P, const double* __restrict__ fhat, double* __restrict__ g1,
            double* __restrict__ mom) {
  const int N = P.N;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= N) return;
  double f[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) f[k] = __ldg(fhat + (size_t)k * N + cell);
  double rho, sx, sy;
  d2q9_sums(f, rho, sx, sy);
  const double cr = P.c / rho;
  mom[cell] = rho;
  mom[N + cell] = sx * cr;
  mom[2 * N + cell] = sy * cr;
  if constexpr (G) {
    double utx, uty;
    d2q9_ut(rho, sx, sy, P, utx, uty);
    double Pk[9], rbw[3];
    d2q9_poly(utx, uty, P, Pk);
    const double rb = P.b1 * rho;
    wclasses<WS>(P, rb, rbw);
    for9([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      g1[(size_t)k * N + cell] = fma(wk<WS, k>(P, rb, rbw), Pk[k], P.a1 * f[k]);
    });
  }
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
      d2q9_tile<1, false, double>(I.P, I.S1, I.g1, I.fhat, I.mom, I.g2, I.X, I.mom + I.P.N,
                                  bx * TX, by * I.P.ty, smem);
    else
      d2q9_tile<2, false, double>(I.P, I.S2, I.g2, I.X, I.mom + I.P.N, I.fhat, I.g1, I.mom,
                                  bx * TX, by * I.P.ty, smem);
    __syncthreads();
  }
}

}  // namespace

size_t d2q9_smem_bytes(int ty) {
  return sizeof(double) * (9 * (ty + 2 * HALO) * SW + 9 * ty * (TX + 1) + 9 * (ty + 1) * TX);
}

template <typename A>
cudaError_t allow_smem(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_d2q9<1, true, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_d2q9<2, true, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_d2q9<1, false, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_d2q9<2, false, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

// Shared memory per SM, the part reserved per block and the opt-in maximum
// per block of the current device.
struct SmemLimits {
  int per_sm = 0, reserved = 0, optin = 0, sms = 0;
};
SmemLimits smem_limits() {
  SmemLimits l;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l.per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l.reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SmemLimits{};
  return l;
}

cudaError_t d2q9_prepare(int ty) {
  // the attribute is per function: allow the largest tile so that contexts
  // with different tile heights can coexist, and for the stage kernels the
  // device maximum, which the one-wave padding of stage_smem may use
  (void)ty;
  const int bytes = (int)d2q9_smem_bytes(kMaxTY);
  const SmemLimits l = smem_limits();
  cudaError_t e = allow_smem<double>(std::max(bytes, l.optin));
  if (e == cudaSuccess) e = allow_smem<dw>(std::max((int)d2q9_smem_bytes(Arith<dw>::kMaxTY), l.optin));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_d2q9_ftp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_d2q9_ftp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
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

namespace {
// Per-device cache of the stage kernels' occupancy (blocks per SM at each
// tile height, unpadded) and of the one-wave padding of stage_smem.
template <typename A>
struct StageCache {
  struct Entry {
    int occ = -1, cap = -1;
    size_t bytes = 0;
  };
  std::mutex mu;
  Entry e[2][2][kMaxTY + 1];
  SmemLimits lim;
  int dev = -1;
};

template <typename A>
StageCache<A>& stage_cache() {
  static StageCache<A> c;
  return c;
}

template <typename A>
auto stage_kernel(int stage, bool wsym) {
  return wsym ? (stage == 1 ? k_d2q9<1, true, A> : k_d2q9<2, true, A>)
              : (stage == 1 ? k_d2q9<1, false, A> : k_d2q9<2, false, A>);
}

// the cache entry of (stage, wsym, ty) with its occupancy filled in, or
// nullptr; the caller holds c.mu
template <typename A>
typename StageCache<A>::Entry* stage_entry(StageCache<A>& c, int stage, bool wsym, int ty) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if (dev != c.dev) {                         // (re)read the limits of this device
    c.lim = smem_limits();
    c.dev = dev;
    for (auto& a : c.e)
      for (auto& b : a)
        for (auto& x : b) x = typename StageCache<A>::Entry{};
  }
  if (c.lim.sms <= 0 || ty < 1 || ty > kMaxTY) return nullptr;
  auto& en = c.e[stage - 1][wsym ? 1 : 0][ty];
  if (en.occ < 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        &en.occ, stage_kernel<A>(stage, wsym), TX * (ty + 1),
                        d2q9_smem_bytes(ty)) != cudaSuccess) {
    en.occ = 0;
    cudaGetLastError();
  }
  return &en;
}

// Dynamic shared memory of a stage launch.  A grid of at most one wave
// (tiles <= SMs x resident blocks per SM) is not spread evenly by the block
// scheduler: some SMs receive as many tiles as fit (three 32 x 7 tiles of the
// double-word kernels at 256^2) while others receive one, and the wave lasts
// as long as the fullest SM.  Padding the request so that no more than
// ceil(tiles / SMs) blocks fit on an SM spreads the tiles evenly (measured
// at 256^2: double-word 103.2 -> 97.2 us per step at ty = 7; FP64 at its
// chosen height, one block per SM, unchanged).
template <typename A>
size_t stage_smem(int stage, bool wsym, int ty, long tiles) {
  const size_t need = d2q9_smem_bytes(ty);
  StageCache<A>& c = stage_cache<A>();
  std::lock_guard<std::mutex> lock(c.mu);
  auto* en = stage_entry(c, stage, wsym, ty);
  if (!en) return need;
  const long cap = (tiles + c.lim.sms - 1) / c.lim.sms;
  if (en->occ <= 0 || cap >= en->occ) return need;
  if (en->cap != cap) {
    // (cap + 1) (bytes + reserved) > per_sm >= cap (bytes + reserved)
    size_t pad = (size_t)(c.lim.per_sm / (cap + 1) - c.lim.reserved + 16);
    pad = std::max(need, (pad + 15) & ~(size_t)15);
    int got = 0;
    if (pad > (size_t)c.lim.optin ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&got, stage_kernel<A>(stage, wsym),
                                                      TX * (ty + 1), pad) != cudaSuccess ||
        got != cap) {
      cudaGetLastError();
      pad = need;
    }
    en->cap = (int)cap;
    en->bytes = pad;
  }
  return en->bytes;
}

template <typename A>
int stage_occupancy(bool wsym, int ty) {
  StageCache<A>& c = stage_cache<A>();
  std::lock_guard<std::mutex> lock(c.mu);
  int occ = 1 << 30;
  for (int stage = 1; stage <= 2; ++stage) {
    auto* en = stage_entry(c, stage, wsym, ty);
    occ = std::min(occ, en ? en->occ : 0);
  }
  return occ;
}

template <typename A>
cudaError_t launch_stage(const typename Arith<A>::Par& p, const typename Arith<A>::Stg& s,
                         int stage, const double* gin, const double* own, const double* rho_in,
                         double* out0, double* out1, double* rho_out, cudaStream_t st) {
  if (p.ty < 1 || p.ty > Arith<A>::kMaxTY) return cudaErrorInvalidValue;
  dim3 grid((p.nx + TX - 1) / TX, (p.ny + p.ty - 1) / p.ty);
  const int threads = TX * (p.ty + 1);
  const size_t bytes = stage_smem<A>(stage, p.wsym, p.ty, (long)grid.x * grid.y);
  // programmatic dependent launch: this grid may be scheduled while the
  // previous kernel on the stream finishes; the tile code waits for that
  // kernel's completion before its first global read
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const auto kern = p.wsym ? (stage == 1 ? k_d2q9<1, true, A> : k_d2q9<2, true, A>)
                           : (stage == 1 ? k_d2q9<1, false, A> : k_d2q9<2, false, A>);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, p, s, gin, own, rho_in, out0, out1, rho_out);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// x = h + l with h = x rounded to FP32 and l the FP32 rounding of x - h
dw split(double x) {
  const float h = (float)x;
  return dw{h, (float)(x - (double)h)};
}
template <size_t N>
void split_all(const double (&x)[N], dw (&d)[N]) {
  for (size_t i = 0; i < N; ++i) d[i] = split(x[i]);
}
template <size_t N, size_t M>
void split_all(const double (&x)[N][M], dw (&d)[N][M]) {
  for (size_t i = 0; i < N; ++i) split_all(x[i], d[i]);
}
template <size_t N, size_t M, size_t L>
void split_all(const double (&x)[N][M][L], dw (&d)[N][M][L]) {
  for (size_t i = 0; i < N; ++i) split_all(x[i], d[i]);
}
}  // namespace

cudaError_t launch_d2q9_ftp(const D2Q9Params& p, const D2Q9Stage& s, const double* g1,
                            const double* fhat, const double* rho_fhat, double* g2, double* ftp,
                            double* rho_ftp, cudaStream_t st) {
  if (p.ty < 1 || p.ty > kMaxTY) return cudaErrorInvalidValue;
  const dim3 grid((p.nx + TX - 1) / TX, (p.ny + p.ty - 1) / p.ty);
  const int threads = TX * (p.ty + 1);
  const size_t bytes = d2q9_smem_bytes(p.ty);
  if (p.wsym)
    k_d2q9_ftp<true><<<grid, threads, bytes, st>>>(p, s, g1, fhat, rho_fhat, g2, ftp, rho_ftp);
  else
    k_d2q9_ftp<false><<<grid, threads, bytes, st>>>(p, s, g1, fhat, rho_fhat, g2, ftp, rho_ftp);
  return cudaGetLastError();
}

cudaError_t launch_d2q9dw_cell(const D2Q9ParamsDW& p, const double* fhat, double* g1,
                               double* mom, cudaStream_t st) {
  const int blocks = (p.N + 255) / 256;
  if (p.wsym) k_d2q9dw_cell<true><<<blocks, 256, 0, st>>>(p, fhat, g1, mom);
  else k_d2q9dw_cell<false><<<blocks, 256, 0, st>>>(p, fhat, g1, mom);
  return cudaGetLastError();
}

cudaError_t launch_d2q9_cell(const D2Q9Params& p, bool write_g, const double* fhat, double* g1,
                             double* mom, cudaStream_t st) {
  const int blocks = (p.N + 255) / 256;
  if (write_g) {
    if (p.wsym) k_d2q9_cell<true, true><<<blocks, 256, 0, st>>>(p, fhat, g1, mom);
    else k_d2q9_cell<true, false><<<blocks, 256, 0, st>>>(p, fhat, g1, mom);
  } else {
    k_d2q9_cell<false, false><<<blocks, 256, 0, st>>>(p, fhat, g1, mom);
  }
  return cudaGetLastError();
}

int d2q9_max_ty(bool dwa) { return dwa ? Arith<dw>::kMaxTY : Arith<double>::kMaxTY; }
int d2q9_occupancy(bool dwa, bool wsym, int ty) {
  if (ty < 1 || ty > d2q9_max_ty(dwa)) return 0;
  return dwa ? stage_occupancy<dw>(wsym, ty) : stage_occupancy<double>(wsym, ty);
}

cudaError_t launch_d2q9_stage(const D2Q9Params& p, const D2Q9Stage& s, int stage,
                              const double* gin, const double* own, const double* rho_in,
                              double* out0, double* out1, double* rho_out, cudaStream_t st) {
  return launch_stage<double>(p, s, stage, gin, own, rho_in, out0, out1, rho_out, st);
}

cudaError_t launch_d2q9dw_stage(const D2Q9ParamsDW& p, const D2Q9StageDW& s, int stage,
                                const double* gin, const double* own, const double* rho_in,
                                double* out0, double* out1, double* rho_out, cudaStream_t st) {
  return launch_stage<dw>(p, s, stage, gin, own, rho_in, out0, out1, rho_out, st);
}

void d2q9_params_to_dw(const D2Q9Params& p, D2Q9ParamsDW& d) {
  d.nx = p.nx;
  d.ny = p.ny;
  d.N = p.N;
  d.px = p.px;
  d.py = p.py;
  d.ty = p.ty;
  split_all(p.W, d.W);
  d.c3 = split(p.c3);
  d.base_div = split(p.base_div);
  d.half_mb = split(p.half_mb);
  d.wsym = p.wsym;
  d.c = split(p.c);
  d.a1 = split(p.a1);
  d.b1 = split(p.b1);
  d.a2 = split(p.a2);
  d.b2 = split(p.b2);
  d.c_om34 = split(p.c_om34);
  d.r37 = split(p.r37);
  for (int s4 = 0; s4 < 4; ++s4) {
    d.bc_kind[s4] = p.bc_kind[s4];
    d.c_ds[s4] = split(p.ds_den[s4] > 0.0 ? p.c / p.ds_den[s4] : 0.0);
  }
  split_all(p.feq_wall, d.feq_wall);
  split_all(p.bb, d.bb);
}

void d2q9_stage_to_dw(const D2Q9Stage& s, D2Q9StageDW& d) {
  split_all(s.wx, d.wx);
  split_all(s.wy, d.wy);
  split_all(s.wxL, d.wxL);
  split_all(s.wxR, d.wxR);
  split_all(s.wyB, d.wyB);
  split_all(s.wyT, d.wyT);
  d.gamma = split(s.gamma);
  split_all(s.kx, d.kx);
  split_all(s.ky, d.ky);
}

}  // namespace dugks
