// Staged-tile kernels of the T3S3 step for any velocity set (Newton-Cotes
// grids in particular), periodic / bounce-back / diffuse walls, for the
// deviation storage forms of the generic path (FP32 / BF16 deviations
// d = f - W_k rho0, FP32 arithmetic, compensated moment sums; see
// dugks_gcommon.cuh).  The kernels are written for any compute type, but
// FP64 storage keeps the generic kernels of dugks_generic_mixed.cu: it is
// bound by the FP64 pipe, and recomputing g and the face values costs more
// FP64 operations than storing them.
//
// One stage (Sec. 2.1.3, Steps (1)-(4)) reads its source array -- f^ in
// stage 1, f~(t') in stage 2 -- twice and writes one array:
//
//   faces   per (32 x 16 cell tile, velocity chunk): every velocity plane of
//           the tile plus a two-cell halo is staged in shared memory as the
//           stage field g = a src + b feq (eqs. f_bar_1_6, fbp_5_12 derived),
//           wall ghosts extrapolated there (reading Q16); the interface
//           values f-bar of the tile's interior faces follow from the
//           upwind 3 x 3 stencils (eqs. interfaceEvof, flux_DS as printed)
//           and only their moments over the chunk leave the chip
//           (partial sums, FP64);
//   walls   per wall face: the wall rules of Sec. 2.3 on f-bar (bounce-back
//           with a moving wall, diffuse scattering), the face's moments and
//           equilibrium parameters; the wall faces' f-bar is stored (a few
//           MB);
//   facefin interior faces: chunk sums -> the face equilibrium's parameters;
//   update  per (tile, chunk): the same staging; the four face values of
//           every cell recomputed from the staged g (or read at walls),
//           f = alpha f-bar + beta feq (eq. recover2f) and the micro-flux
//           (eq. microflux) enter
//             stage 1: f~(t') = 5/4 g1 - 1/4 f^ + dt/3 L*
//             stage 2: f^^{n+1} = X + 3/4 dt Omega' + 4dt/7 L**,
//                      X = f^+ + 3dt/7 L* = 4/7 f^ - 6/7 g1 + 9/7 f~(t')
//           (eqs. f_tilde_1_3, fhp, collisionterm, feqIntD3rdHat2_DS; X is
//           recovered from f^ and f~(t') instead of being stored); the
//           output's cell moments over the chunk are written as partial
//           sums;
//   cellfin cell moments -> rho, u (FP64) and the next stage's equilibrium
//           parameters.
//
// Every equilibrium that enters an update is W_k P(xi_k) with P quadratic;
// with the flux factors they combine into W_k S(xi_k), S a cubic per cell
// (Cubic in dugks_gcommon.cuh).  Per (cell, velocity) and step the path
// moves four reads and two writes of the stored type plus the halo
// re-reads, which the 126 MB L2 mostly serves.
#include <algorithm>

#include "dugks_gcommon.cuh"

namespace dugks {

namespace {

constexpr int TXT = 32;                 // tile columns (one lane each)
constexpr int TYT = 16;                 // tile rows
constexpr int NWP = 8;                  // warps per block; warp w takes rows 2w, 2w + 1
constexpr int HXT = TXT + 4;            // staged columns i0 - 2 .. i0 + 33
constexpr int HYT = TYT + 4;            // staged rows    j0 - 2 .. j0 + 17
constexpr int NST = HXT * HYT;          // 720 staged cells
constexpr int NTH = 32 * NWP;           // 256 threads
constexpr int EPT = (NST + NTH - 1) / NTH;   // staged cells per thread (3)

template <typename C>
__device__ __forceinline__ C dot9(const C (&T)[9], C s00, C s01, C s02, C s10, C s11, C s12,
                                  C s20, C s21, C s22) {
  C v = T[0] * s00;
  v = fmx(T[1], s01, v);
  v = fmx(T[2], s02, v);
  v = fmx(T[3], s10, v);
  v = fmx(T[4], s11, v);
  v = fmx(T[5], s12, v);
  v = fmx(T[6], s20, v);
  v = fmx(T[7], s21, v);
  return fmx(T[8], s22, v);
}

// the 3 x 3 stencil of window W centred at (x, y): rows y-1..y+1 (south to
// north), columns x-1..x+1
#define STEN(W, x, y)                                                                   \
  W[(y) - 1][(x) - 1], W[(y) - 1][(x)], W[(y) - 1][(x) + 1], W[(y)][(x) - 1], W[(y)][(x)], \
      W[(y)][(x) + 1], W[(y) + 1][(x) - 1], W[(y) + 1][(x)], W[(y) + 1][(x) + 1]

// Per-velocity face-value weights (eq. flux_DS as printed), formed on the
// host per stage and velocity (gnc_weight_table) and read by every block for
// its chunk into shared memory: x-faces about the lower (left) and upper
// (right) cell, y-faces about the lower (below) and upper cell, each nine
// weights padded to twelve for 16-byte reads.  The sign of xi.n picks one
// set; a tie averages both (Q4).
constexpr int KCMAX = 128;            // velocities per chunk at most
constexpr int WPV = 48;               // weights per velocity in the table
struct FaceW {
  float x[9], y[9];                   // the set each direction's sign picks
  const float* row;                   // the velocity's row of the table (ties)
  int sx, sy;                         // sign of xi_x, xi_y
};
__device__ __forceinline__ void read9(const float* __restrict__ w, float (&T)[9]) {
  const float4 a = *reinterpret_cast<const float4*>(w);
  const float4 b = *reinterpret_cast<const float4*>(w + 4);
  T[0] = a.x; T[1] = a.y; T[2] = a.z; T[3] = a.w;
  T[4] = b.x; T[5] = b.y; T[6] = b.z; T[7] = b.w;
  T[8] = w[8];
}
__device__ __forceinline__ void face_weights(FaceW& w, const float* __restrict__ row, float cx,
                                             float cy) {
  w.row = row;
  w.sx = cx > 0.f ? 1 : (cx < 0.f ? -1 : 0);
  w.sy = cy > 0.f ? 1 : (cy < 0.f ? -1 : 0);
  read9(row + (w.sx >= 0 ? 0 : 12), w.x);
  read9(row + (w.sy >= 0 ? 24 : 36), w.y);
}

// x-face value between the cells centred at window columns xl and xl + 1
// (row y); y-face value between window rows yl and yl + 1 (column x); a tie
// averages the expansions from both cells (Q4)
template <int NR, int NC>
__device__ __forceinline__ float xface(const FaceW& w, const float (&W)[NR][NC], int xl, int y) {
  if (w.sx > 0) return dot9(w.x, STEN(W, xl, y));
  if (w.sx < 0) return dot9(w.x, STEN(W, xl + 1, y));
  float u[9];
  read9(w.row + 12, u);
  return 0.5f * (dot9(w.x, STEN(W, xl, y)) + dot9(u, STEN(W, xl + 1, y)));
}
template <int NR, int NC>
__device__ __forceinline__ float yface(const FaceW& w, const float (&W)[NR][NC], int x, int yl) {
  if (w.sy > 0) return dot9(w.y, STEN(W, x, yl));
  if (w.sy < 0) return dot9(w.y, STEN(W, x, yl + 1));
  float u[9];
  read9(w.row + 36, u);
  return 0.5f * (dot9(w.y, STEN(W, x, yl)) + dot9(u, STEN(W, x, yl + 1)));
}
// the same from the staged plane directly: x-face left of staged column cx
// (staged row cy), y-face below staged row cy (staged column cx)
__device__ __forceinline__ float stencil_at(const float* __restrict__ g, const float (&T)[9], int cx,
                                            int cy) {
  const float* b = g + (cy - 1) * HXT + cx - 1;
  float v = T[0] * b[0];
  v = fmaf(T[1], b[1], v);
  v = fmaf(T[2], b[2], v);
  v = fmaf(T[3], b[HXT], v);
  v = fmaf(T[4], b[HXT + 1], v);
  v = fmaf(T[5], b[HXT + 2], v);
  v = fmaf(T[6], b[2 * HXT], v);
  v = fmaf(T[7], b[2 * HXT + 1], v);
  return fmaf(T[8], b[2 * HXT + 2], v);
}
__device__ __forceinline__ float xface_at(const FaceW& w, const float* __restrict__ g, int cx,
                                          int cy) {
  if (w.sx > 0) return stencil_at(g, w.x, cx - 1, cy);
  if (w.sx < 0) return stencil_at(g, w.x, cx, cy);
  float u[9];
  read9(w.row + 12, u);
  return 0.5f * (stencil_at(g, w.x, cx - 1, cy) + stencil_at(g, u, cx, cy));
}
__device__ __forceinline__ float yface_at(const FaceW& w, const float* __restrict__ g, int cx,
                                          int cy) {
  if (w.sy > 0) return stencil_at(g, w.y, cx, cy - 1);
  if (w.sy < 0) return stencil_at(g, w.y, cx, cy);
  float u[9];
  read9(w.row + 36, u);
  return 0.5f * (stencil_at(g, w.y, cx, cy - 1) + stencil_at(g, u, cx, cy));
}

// the chunk's rows of the weight table into shared memory (the caller syncs
// before the first use)
__device__ __forceinline__ void load_weights(float* __restrict__ wts, const GncStep& s, int stage,
                                             int k0, int k1) {
  const float* src = s.fwt + ((size_t)(stage - 1) * s.p.nv + k0) * WPV;
  const int n = (k1 - k0) * WPV;
  for (int t = threadIdx.x; t < n; t += NTH) wts[t] = __ldg(src + t);
}

// a compute-type value as the storage type holds it
template <typename T> __device__ __forceinline__ float stored_value(float v) { return v; }
template <> __device__ __forceinline__ float stored_value<__nv_bfloat16>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

// Staging of one velocity plane of a tile.  The staged cells of a thread are
// fixed for the whole chunk: their source offsets (periodic wrap; clamped
// across a wall, where the ghost replaces the value) and the equilibrium
// parameters of their cells stay in registers.
constexpr int PD = 3;                 // velocity planes loaded ahead

template <typename T>
struct Stager {
  using C = typename Prec<T>::C;
  int off[EPT];
  EqF<C> q[EPT];
  T raw[PD][EPT];
  __device__ void init(const GncStep& s, const C* __restrict__ eq, int i0, int j0) {
    const DevParams& p = s.p;
#pragma unroll
    for (int m = 0; m < EPT; ++m) {
      const int e = threadIdx.x + NTH * m;
      const int ee = e < NST ? e : NST - 1;
      const int ex = ee % HXT, ey = ee / HXT;
      int gi = i0 - 2 + ex, gj = j0 - 2 + ey;
      if (p.px) gi = ((gi % p.nx) + p.nx) % p.nx;
      else gi = min(max(gi, 0), p.nx - 1);
      if (p.py) gj = ((gj % p.ny) + p.ny) % p.ny;
      else gj = min(max(gj, 0), p.ny - 1);
      off[m] = gj * p.nx + gi;
      q[m].vx = eq[off[m]];
      q[m].vy = eq[p.N + off[m]];
      q[m].bm1 = eq[2 * p.N + off[m]];
      q[m].r = eq[3 * p.N + off[m]];
      q[m].dr = eq[4 * p.N + off[m]];
    }
  }
  // slot u must be a compile-time constant after unrolling (registers)
  __device__ __forceinline__ void load(int u, const T* __restrict__ src, int k, int N) {
#pragma unroll
    for (int m = 0; m < EPT; ++m)
      if (threadIdx.x + NTH * m < NST) raw[u][m] = ldr(src + (size_t)k * N + off[m]);
  }
  // g = a src + b feq = src + b (feq - src) (a + b = 1; this form keeps a
  // uniform equilibrium exact whatever the rounding of b) into the buffer
  __device__ __forceinline__ void store(int u, C* __restrict__ buf, C b, C cx, C cy, C w) {
#pragma unroll
    for (int m = 0; m < EPT; ++m) {
      const int e = threadIdx.x + NTH * m;
      if (e < NST) {
        const C r = tof(raw[u][m]);
        buf[e] = fmx(b, feq_dev<C>(q[m], cx, cy, w) - r, r);
      }
    }
  }
};

// Wall ghosts of a staged plane (reading Q16): first across x-walls on the
// rows inside the mesh, then across y-walls on every staged column, so a
// corner ghost is the y-extrapolation of x-ghosts (as in the oracle).
// Uniform per block: every thread calls it, syncs included.
template <typename C>
__device__ __forceinline__ void stage_ghosts(const DevParams& p, C* __restrict__ buf, int i0,
                                             int j0, bool wx, bool wy) {
  if (wx) {
    const int xw = 1 - i0;                 // column of the west ghost (gi = -1)
    const int xe = p.nx - i0 + 2;          // column of the east ghost (gi = nx)
    for (int t = threadIdx.x; t < 2 * HYT; t += NTH) {
      const int ey = t % HYT;
      const int gj = j0 - 2 + ey;
      if (!p.py && (gj < 0 || gj >= p.ny)) continue;
      C* r = buf + ey * HXT;
      if (t < HYT) {
        if (xw >= 0 && xw + 3 < HXT) r[xw] = C(3) * r[xw + 1] - C(3) * r[xw + 2] + r[xw + 3];
      } else if (xe >= 3 && xe < HXT) {
        r[xe] = C(3) * r[xe - 1] - C(3) * r[xe - 2] + r[xe - 3];
      }
    }
    __syncthreads();
  }
  if (wy) {
    const int ys = 1 - j0, yn = p.ny - j0 + 2;
    for (int t = threadIdx.x; t < 2 * HXT; t += NTH) {
      const int ex = t % HXT;
      C* c = buf + ex;
      if (t < HXT) {
        if (ys >= 0 && ys + 3 < HYT)
          c[ys * HXT] = C(3) * c[(ys + 1) * HXT] - C(3) * c[(ys + 2) * HXT] + c[(ys + 3) * HXT];
      } else if (yn >= 3 && yn < HYT) {
        c[yn * HXT] = C(3) * c[(yn - 1) * HXT] - C(3) * c[(yn - 2) * HXT] + c[(yn - 3) * HXT];
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ bool tile_touches_walls_x(const DevParams& p, int i0) {
  return !p.px && (i0 == 0 || i0 + TXT + 2 >= p.nx);
}
__device__ __forceinline__ bool tile_touches_walls_y(const DevParams& p, int j0) {
  return !p.py && (j0 == 0 || j0 + TYT + 2 >= p.ny);
}

// ------------------------------------------------------------------ faces
// Face pass of a stage: partial moments over the chunk of the x-face at the
// left and the y-face below every cell of the tile (interior faces only).
// Velocity planes are loaded PD velocities ahead into registers; one block
// barrier per velocity (two more on tiles with wall ghosts).
template <typename T>
__global__ void __launch_bounds__(NTH, 2)
k_gnc_faces(GncStep s, int stage) {
  using C = float;
  using V4 = float4;
  __shared__ C gs[2][NST];
  __shared__ __align__(16) float wts[KCMAX * WPV];
  const DevParams& p = s.p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tiles = s.tiles_x * s.tiles_y;
  const int tile = blockIdx.x % tiles, chunk = blockIdx.x / tiles;
  const int i0 = (tile % s.tiles_x) * TXT, j0 = (tile / s.tiles_x) * TYT;
  const int k0 = chunk * s.kc, k1 = min(p.nv, k0 + s.kc);
  const StageCoef& sc = stage == 1 ? s.s1 : s.s2;
  const T* __restrict__ src = (const T*)(stage == 1 ? s.fhat : s.ftp);
  const C* __restrict__ eq = (const C*)(stage == 1 ? s.eqn : s.eqp);
  const C b = (C)sc.b;
  const V4* vq = (const V4*)s.vq;
  const bool wx = tile_touches_walls_x(p, i0), wy = tile_touches_walls_y(p, j0);

  // the thread's cells (column i, rows j, j + 1) and which of their faces count
  const int i = i0 + lane;
  bool fx[2], fy[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int j = j0 + 2 * warp + q;
    const bool cell = i < p.nx && j < p.ny;
    fx[q] = cell && (p.px || i >= 1);
    fy[q] = cell && (p.py || j >= 1);
  }
  Kah ax[2][3] = {}, ay[2][3] = {};

  load_weights(wts, s, stage, k0, k1);
  Stager<T> st;
  st.init(s, eq, i0, j0);
#pragma unroll
  for (int u = 0; u < PD; ++u)
    if (k0 + u < k1) st.load(u, src, k0 + u, p.N);
  int buf = 0;
  for (int kb = k0; kb < k1; kb += PD) {
#pragma unroll
    for (int u = 0; u < PD; ++u) {
      const int k = kb + u;
      if (k >= k1) break;                            // uniform over the block
      const V4 e4 = ld4(vq + p.nv + k);
      st.store(u, gs[buf], b, e4.x, e4.y, e4.z);
      if (k + PD < k1) st.load(u, src, k + PD, p.N);
      __syncthreads();
      stage_ghosts<C>(p, gs[buf], i0, j0, wx, wy);
      FaceW fw;
      face_weights(fw, wts + (k - k0) * WPV, e4.x, e4.y);
      // window: staged rows 2w .. 2w + 4, columns lane .. lane + 3
      C Wn[5][4];
      const C* g0 = gs[buf] + (2 * warp) * HXT + lane;
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) Wn[r][c] = g0[r * HXT + c];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        // cell q sits at window (2, 2 + q)
        if (fx[q]) {
          const C v = xface(fw, Wn, 1, 2 + q);
          kah_add(ax[q][0], v);
          kah_add(ax[q][1], e4.x * v);
          kah_add(ax[q][2], e4.y * v);
        }
        if (fy[q]) {
          const C v = yface(fw, Wn, 2, 1 + q);
          kah_add(ay[q][0], v);
          kah_add(ay[q][1], e4.x * v);
          kah_add(ay[q][2], e4.y * v);
        }
      }
      buf ^= 1;
    }
  }
  const int nfx = p.ny * (p.nx + 1), nfy = (p.ny + 1) * p.nx;
  double* px = s.pfx + (size_t)chunk * 3 * nfx;
  double* py = s.pfy + (size_t)chunk * 3 * nfy;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int j = j0 + 2 * warp + q;
    if (fx[q]) {
      const int f = j * (p.nx + 1) + i;
#pragma unroll
      for (int m = 0; m < 3; ++m) px[(size_t)m * nfx + f] = kah_value(ax[q][m]);
    }
    if (fy[q]) {
      const int f = j * p.nx + i;
#pragma unroll
      for (int m = 0; m < 3; ++m) py[(size_t)m * nfy + f] = kah_value(ay[q][m]);
    }
  }
}

// --------------------------------------------------------------- facefin
// Interior faces of both directions: chunk sums (in chunk order) -> the face
// equilibrium's assembly parameters.
template <typename C>
__global__ void __launch_bounds__(256)
k_gnc_facefin(GncStep s) {
  const DevParams& p = s.p;
  const int nfx = p.ny * (p.nx + 1), nfy = (p.ny + 1) * p.nx;
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nfx + nfy) return;
  const bool xdir = f < nfx;
  const int nf = xdir ? nfx : nfy;
  if (!xdir) f -= nfx;
  if (xdir) {
    const int fi = f % (p.nx + 1);
    if ((!p.px && (fi == 0 || fi == p.nx)) || (p.px && fi == p.nx)) return;
  } else {
    const int fj = f / p.nx;
    if ((!p.py && (fj == 0 || fj == p.ny)) || (p.py && fj == p.ny)) return;
  }
  const double* part = xdir ? s.pfx : s.pfy;
  double r = s.ref.W, jx = s.ref.Wx, jy = s.ref.Wy;
  for (int c = 0; c < s.nch; ++c) {
    const double* pc = part + (size_t)c * 3 * nf;
    r += pc[f];
    jx += pc[nf + f];
    jy += pc[2 * nf + f];
  }
  C* fp = (C*)(xdir ? s.fpx : s.fpy);
  const EqF<C> q = eq_params_j<C>(r, jx, jy, p.inv_RT, s.ref.rho0);
  store_par(fp, nf, f, q);
  // a periodic direction's face n is face 0
  if (xdir && p.px && f % (p.nx + 1) == 0) store_par(fp, nf, f + p.nx, q);
  if (!xdir && p.py && f / p.nx == 0) store_par(fp, nf, f + p.ny * p.nx, q);
}

// --------------------------------------------------------------- cellfin
// Cell moments from the chunk partials: rho, u (FP64) and the equilibrium
// parameters of the stage that reads them (which 0: f^ at t_n, 1: f~(t')).
template <typename C>
__global__ void __launch_bounds__(256)
k_gnc_cellfin(GncStep s, int which) {
  const DevParams& p = s.p;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.N) return;
  double r = s.ref.W, jx = s.ref.Wx, jy = s.ref.Wy;
  for (int c = 0; c < s.nch; ++c) {
    const double* pc = s.pc + (size_t)c * 3 * p.N;
    r += pc[cell];
    jx += pc[p.N + cell];
    jy += pc[2 * p.N + cell];
  }
  const double rinv = 1.0 / r;
  const double ux = jx * rinv, uy = jy * rinv;
  double* mom = which == 0 ? s.mom_n : s.mom_p;
  mom[cell] = r;
  mom[p.N + cell] = ux;
  mom[2 * p.N + cell] = uy;
  store_par((C*)(which == 0 ? s.eqn : s.eqp), p.N, cell,
            eq_params_u<C>(r, ux, uy, p.inv_RT, s.ref.rho0));
}

// Cell moments of the stored state over the chunks (the state's first
// step, or after it was set): one thread per cell.
template <typename T>
__global__ void __launch_bounds__(256)
k_gnc_moments(GncStep s) {
  using C = typename Prec<T>::C;
  using V4 = typename Prec<T>::V4;
  const DevParams& p = s.p;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.N) return;
  const V4* vq = (const V4*)s.vq;
  const int chunk = blockIdx.y;
  const int k0 = chunk * s.kc, k1 = min(p.nv, k0 + s.kc);
  Acc<C> a0{}, a1{}, a2{};
  const T* src = (const T*)s.fhat;
  for (int k = k0; k < k1; ++k) {
    const C d = ldv(src + (size_t)k * p.N + cell);
    const V4 xq = ld4(vq + k);
    acc_add(a0, d);
    acc_addprod(a1, xq.x, xq.y, d);
    acc_addprod(a2, xq.z, xq.w, d);
  }
  double* pc = s.pc + (size_t)chunk * 3 * p.N;
  pc[cell] = acc_value(a0);
  pc[p.N + cell] = acc_value(a1);
  pc[2 * p.N + cell] = acc_value(a2);
}

// ----------------------------------------------------------------- walls
// g of velocity k at cell (ci, cj) inside the mesh, from the stage source
template <typename T>
__device__ __forceinline__ typename Prec<T>::C g_cell(const GncStep& s, const T* __restrict__ src,
                                                      const typename Prec<T>::C* __restrict__ eq,
                                                      int k, int ci, int cj,
                                                      typename Prec<T>::C a,
                                                      typename Prec<T>::C b) {
  using C = typename Prec<T>::C;
  using V4 = typename Prec<T>::V4;
  const DevParams& p = s.p;
  const int c = cj * p.nx + ci;
  EqF<C> q;
  q.vx = eq[c];
  q.vy = eq[p.N + c];
  q.bm1 = eq[2 * p.N + c];
  q.r = eq[3 * p.N + c];
  q.dr = eq[4 * p.N + c];
  const V4 e4 = ld4((const V4*)s.vq + p.nv + k);
  const C r = ldv(src + (size_t)k * p.N + c);
  (void)a;
  return fmx(b, feq_dev<C>(q, e4.x, e4.y, e4.z) - r, r);     // src + b (feq - src)
}
// g within one ghost layer: periodic wrap, or the quadratic extrapolation
// across a wall -- along x on rows inside the mesh, then along y (Q16)
template <typename T>
__device__ typename Prec<T>::C g_ghost(const GncStep& s, const T* __restrict__ src,
                                       const typename Prec<T>::C* __restrict__ eq, int k,
                                       int ci, int cj, typename Prec<T>::C a,
                                       typename Prec<T>::C b) {
  using C = typename Prec<T>::C;
  const DevParams& p = s.p;
  if (cj < 0 || cj >= p.ny) {
    if (p.py) {
      cj = (cj < 0) ? cj + p.ny : cj - p.ny;
    } else {
      const int j0 = cj < 0 ? 0 : p.ny - 1, sg = cj < 0 ? 1 : -1;
      C v[3];
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        int ii = ci;
        if (ii < 0 || ii >= p.nx) {
          if (p.px) {
            ii = ii < 0 ? ii + p.nx : ii - p.nx;
            v[t] = g_cell<T>(s, src, eq, k, ii, j0 + t * sg, a, b);
          } else {
            const int i1 = ii < 0 ? 0 : p.nx - 1, sx = ii < 0 ? 1 : -1;
            v[t] = C(3) * g_cell<T>(s, src, eq, k, i1, j0 + t * sg, a, b) -
                   C(3) * g_cell<T>(s, src, eq, k, i1 + sx, j0 + t * sg, a, b) +
                   g_cell<T>(s, src, eq, k, i1 + 2 * sx, j0 + t * sg, a, b);
          }
        } else {
          v[t] = g_cell<T>(s, src, eq, k, ii, j0 + t * sg, a, b);
        }
      }
      return C(3) * v[0] - C(3) * v[1] + v[2];
    }
  }
  if (ci < 0 || ci >= p.nx) {
    if (p.px) {
      ci = ci < 0 ? ci + p.nx : ci - p.nx;
    } else {
      const int i1 = ci < 0 ? 0 : p.nx - 1, sx = ci < 0 ? 1 : -1;
      return C(3) * g_cell<T>(s, src, eq, k, i1, cj, a, b) -
             C(3) * g_cell<T>(s, src, eq, k, i1 + sx, cj, a, b) +
             g_cell<T>(s, src, eq, k, i1 + 2 * sx, cj, a, b);
    }
  }
  return g_cell<T>(s, src, eq, k, ci, cj, a, b);
}
// f-bar of velocity k at a wall face from the fluid cell (ci, cj): eq.
// flux_DS about that cell, foot offset (X, Y) from its centre
template <typename T>
__device__ typename Prec<T>::C wall_recon(const GncStep& s, const T* __restrict__ src,
                                          const typename Prec<T>::C* __restrict__ eq, int k,
                                          int ci, int cj, typename Prec<T>::C X,
                                          typename Prec<T>::C Y, typename Prec<T>::C a,
                                          typename Prec<T>::C b) {
  using C = typename Prec<T>::C;
  C w[9];
  flux_ds_weights<C>(X * (C)s.p.inv_dx, Y * (C)s.p.inv_dy, w);
  C v = C(0);
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx)
      v = fmx(w[(dy + 1) * 3 + dx + 1], g_ghost<T>(s, src, eq, k, ci + dx, cj + dy, a, b), v);
  return v;
}

// One wall face per block (both directions in one launch), threads over the
// velocities: fluid-side f-bar for velocities hitting or running along the
// wall, the wall rule for those leaving it, the face's moments and
// equilibrium parameters; f-bar into the wall arrays.  Face id per
// direction = 2 line + (0: W/S, 1: E/N).
template <typename T, int DIR>
__device__ __forceinline__ void gnc_wall_face(const GncStep& s, int stage, int id, double* sm) {
  using C = typename Prec<T>::C;
  using V4 = typename Prec<T>::V4;
  const DevParams& p = s.p;
  const GDevRef& ref = s.ref;
  const V4* vq = (const V4*)s.vq;
  const StageCoef& sc = stage == 1 ? s.s1 : s.s2;
  const T* __restrict__ src = (const T*)(stage == 1 ? s.fhat : s.ftp);
  const C* __restrict__ eq = (const C*)(stage == 1 ? s.eqn : s.eqp);
  const double* mom = stage == 1 ? s.mom_n : s.mom_p;
  const C a = (C)sc.a, b = (C)sc.b, h = (C)sc.h;
  const int nx = p.nx, ny = p.ny, nv = p.nv;
  const int nf = DIR == 0 ? ny * (nx + 1) : (ny + 1) * nx;
  const int nl = DIR == 0 ? ny : nx;
  const bool upper_wall = id & 1;
  const int line = id >> 1;
  const int face = DIR == 0 ? line * (nx + 1) + (upper_wall ? nx : 0)
                            : (upper_wall ? ny : 0) * nx + line;
  const int side = DIR == 0 ? (upper_wall ? SIDE_E : SIDE_W) : (upper_wall ? SIDE_N : SIDE_S);
  const bool fluid_hi = !upper_wall;
  const C nsg = fluid_hi ? C(-1) : C(1);
  const int ci = DIR == 0 ? (fluid_hi ? 0 : nx - 1) : line;
  const int cj = DIR == 0 ? line : (fluid_hi ? 0 : ny - 1);
  const int kind = p.bc_kind[side];
  const C half = C(0.5) * (C)(DIR == 0 ? p.dx : p.dy);
  const C off = fluid_hi ? -half : half;
  const C rho_w = (C)mom[cj * nx + ci];
  const C uwx = (C)p.uw_x[side], uwy = (C)p.uw_y[side];
  const C irt = (C)p.inv_RT;
  C* wf = (C*)(DIR == 0 ? s.wfx : s.wfy);
  const size_t wstride = 2 * (size_t)nl;
  const int wslot = (upper_wall ? 1 : 0) * nl + line;
  auto recon = [&](int k) {
    const V4 e4 = ld4(vq + nv + k);
    const C X = DIR == 0 ? off - e4.x * h : -e4.x * h;
    const C Y = DIR == 0 ? -e4.y * h : off - e4.y * h;
    return wall_recon<T>(s, src, eq, k, ci, cj, X, Y, a, b);
  };
  Acc<C> a0{}, a1{}, a2{}, a3{};
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    const V4 xq = ld4(vq + k);
    const C cx = xq.x, cy = xq.z;
    const C xn = nsg * (DIR == 0 ? cx : cy);
    C fbar;
    if (xn >= C(0)) {
      fbar = recon(k);
      if (xn > C(0))
        acc_addprod(a3, DIR == 0 ? nsg * xq.x : nsg * xq.z, DIR == 0 ? nsg * xq.y : nsg * xq.w,
                    fbar);
    } else if (kind == BC_BOUNCEBACK) {            // eq. BB on f-bar
      const int kk = __ldg(p.opp + k);
      const C wk = ld4(vq + nv + k).z;
      const C bbk = C(2) * wk * fmx(cx, uwx, cy * uwy) * irt;
      const C shift = (ld4(vq + nv + kk).z - wk) * (C)ref.rho0;
      fbar = fmx(rho_w, bbk, recon(kk) + shift);
    } else {
      continue;                                    // diffuse: after the reduction
    }
    wf[(size_t)k * wstride + wslot] = fbar;
    acc_add(a0, fbar);
    acc_addprod(a1, xq.x, xq.y, fbar);
    acc_addprod(a2, xq.z, xq.w, fbar);
  }
  double v[4] = {acc_value(a0), acc_value(a1), acc_value(a2), acc_value(a3)};
  block_sum<4>(v, sm);
  if (kind == BC_DIFFUSE) {                        // uniform over the block
    // rho_w balances the outgoing flux of f = W rho0 + d (Sec. 2.3, Q15)
    const double rho_ds = (s.ds_out[side] + v[3]) / p.ds_den[side];
    Acc<C> b0{}, b1{}, b2{};
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
      const V4 xq = ld4(vq + k);
      const C xn = nsg * (DIR == 0 ? xq.x : xq.z);
      if (xn < C(0)) {
        const C fbar =
            to_c<C>(fma(rho_ds, __ldg(p.feq_wall + side * nv + k), -__ldg(p.w + k) * ref.rho0));
        wf[(size_t)k * wstride + wslot] = fbar;
        acc_add(b0, fbar);
        acc_addprod(b1, xq.x, xq.y, fbar);
        acc_addprod(b2, xq.z, xq.w, fbar);
      }
    }
    double w2[3] = {acc_value(b0), acc_value(b1), acc_value(b2)};
    block_sum<3>(w2, sm);
    v[0] += w2[0];
    v[1] += w2[1];
    v[2] += w2[2];
  }
  if (threadIdx.x == 0)
    store_par((C*)(DIR == 0 ? s.fpx : s.fpy), nf, face,
              eq_params_j<C>(ref.W + v[0], ref.Wx + v[1], ref.Wy + v[2], p.inv_RT, ref.rho0));
}

// blocks [0, nwx): x-direction walls (W/E), then y-direction walls (S/N)
template <typename T>
__global__ void __launch_bounds__(256)
k_gnc_walls(GncStep s, int stage, int nwx) {
  __shared__ double sm[32 * 4];
  if ((int)blockIdx.x < nwx) gnc_wall_face<T, 0>(s, stage, blockIdx.x, sm);
  else gnc_wall_face<T, 1>(s, stage, blockIdx.x - nwx, sm);
}

// ---------------------------------------------------------------- update
// F(xi) = (x/dx)(P_E - P_W) + (y/dy)(P_N - P_S) over the faces of cell
// (i, j), scaled by sc (the face equilibria's part of the micro-flux)
template <typename C>
__device__ __forceinline__ Cubic<C> gnc_flux_cubic(const GncStep& s, int i, int j, C sc) {
  const int nx = s.p.nx, ny = s.p.ny;
  const int nfx = ny * (nx + 1), nfy = (ny + 1) * nx;
  const int fx = j * (nx + 1) + i, fy = j * nx + i;
  const C* fpx = (const C*)s.fpx;
  const C* fpy = (const C*)s.fpy;
  const Quad<C> w = quad(fpx, nfx, fx), e = quad(fpx, nfx, fx + 1);
  const Quad<C> so = quad(fpy, nfy, fy), no = quad(fpy, nfy, fy + nx);
  const C ax = sc * (C)s.p.inv_dx, ay = sc * (C)s.p.inv_dy;
  Cubic<C> F;
  F.c[0] = C(0);
  F.c[1] = ax * (e.c0 - w.c0);
  F.c[2] = ay * (no.c0 - so.c0);
  F.c[3] = ax * (e.cx - w.cx);
  F.c[4] = fmx(ax, e.cy - w.cy, ay * (no.cx - so.cx));
  F.c[5] = ay * (no.cy - so.cy);
  F.c[6] = ax * (e.cxx - w.cxx);
  F.c[7] = fmx(ax, e.cxy - w.cxy, ay * (no.cxx - so.cxx));
  F.c[8] = fmx(ax, e.cyy - w.cyy, ay * (no.cxy - so.cxy));
  F.c[9] = ay * (no.cyy - so.cyy);
  return F;
}
template <typename C>
__device__ __forceinline__ void add_quad(Cubic<C>& S, const Quad<C>& q, C sc) {
  S.c[0] = fmx(sc, q.c0, S.c[0]);
  S.c[1] = fmx(sc, q.cx, S.c[1]);
  S.c[2] = fmx(sc, q.cy, S.c[2]);
  S.c[3] = fmx(sc, q.cxx, S.c[3]);
  S.c[4] = fmx(sc, q.cxy, S.c[4]);
  S.c[5] = fmx(sc, q.cyy, S.c[5]);
}

// Update pass.  With Df = kx (fbar_E - fbar_W) + ky (fbar_N - fbar_S),
// k = -(flux scale) alpha xi / dx (velocity table row 2), P_n and P' the
// cell equilibria at t_n and t', F the faces' equilibria in the flux:
//   stage 1: f~' = 5/4 g1 - 1/4 f^ + dt/3 L*
//                = f^ + W S(xi) - sP f^ + Df,
//            S = sP P_n + sF F, sP = 5/4 b1, sF = -(dt/3) beta1;
//   stage 2: f^^{n+1} = 4/7 f^ - 6/7 g1 + 9/7 f~' + c34 (f~' - feq') + 4dt/7 L**
//                = f~' + cA (f^ - f~') + W S(xi) - (sP + sQ) f~' + Df,
//            S = sP P_n + sQ P' + sF F, cA = 4/7 - 6/7 a1, sP = -6/7 b1,
//            sQ = -c34, sF = -(4dt/7) beta2.
// Written around f^ (stage 1) or f~' (stage 2) with the same rounded
// coefficient on both sides of each difference, the maps keep a uniform
// equilibrium exact whatever the rounding of the coefficients (their exact
// sum is one; written as a plain sum of terms an FP32 step would scale the
// deviations by 1 + O(2^-24) every step).  The output's chunk moments go to
// pc.
template <typename T, int STAGE>
__global__ void __launch_bounds__(NTH, 2)
k_gnc_update(GncStep s, float cA, float cB, float sP, float sQ, float sF) {
  using C = float;
  using V4 = float4;
  __shared__ C gs[2][NST];
  __shared__ C fxs[TYT][TXT + 1];       // x-faces fi = i0 .. i0 + 32 of the tile's rows
  __shared__ C fys[TYT + 1][TXT];       // y-faces fj = j0 .. j0 + 16 of its columns
  __shared__ __align__(16) float wts[KCMAX * WPV];
  const DevParams& p = s.p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tiles = s.tiles_x * s.tiles_y;
  const int tile = blockIdx.x % tiles, chunk = blockIdx.x / tiles;
  const int i0 = (tile % s.tiles_x) * TXT, j0 = (tile / s.tiles_x) * TYT;
  const int k0 = chunk * s.kc, k1 = min(p.nv, k0 + s.kc);
  const StageCoef& sc = STAGE == 1 ? s.s1 : s.s2;
  const T* __restrict__ src = (const T*)(STAGE == 1 ? s.fhat : s.ftp);
  const C* __restrict__ eq = (const C*)(STAGE == 1 ? s.eqn : s.eqp);
  // stage 2 reads f^ of its own cells and overwrites them: no restrict, and
  // the read is a plain load issued before the store
  T* dst = (T*)(STAGE == 1 ? s.ftp : s.fhat);
  const T* fh = (const T*)s.fhat;
  const C b = (C)sc.b;
  const V4* vq = (const V4*)s.vq;
  const C* wfx = (const C*)s.wfx;
  const C* wfy = (const C*)s.wfy;
  const bool wx = tile_touches_walls_x(p, i0), wy = tile_touches_walls_y(p, j0);

  const int i = i0 + lane;
  bool ok[2];
  int cell[2];
  Cubic<C> S[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int j = j0 + 2 * warp + q;
    ok[q] = i < p.nx && j < p.ny;
    cell[q] = ok[q] ? j * p.nx + i : 0;
    if (ok[q]) {
      S[q] = gnc_flux_cubic<C>(s, i, j, sF);
      add_quad(S[q], quad((const C*)s.eqn, p.N, cell[q]), sP);
      if (STAGE == 2) add_quad(S[q], quad((const C*)s.eqp, p.N, cell[q]), sQ);
    }
  }
  // faces this thread computes: the x-face left of and the y-face below
  // each of its two cells; wall faces come from the wall pass's arrays.  The
  // tile's last x-face column (i0 + 32) and y-face row (j0 + 16) are taken
  // by warps 0 and 1 (extra index e < 48).
  const int ex_id = warp * 32 + lane;
  const bool extra = ex_id < 48;
  Kah am[2][3] = {};

  load_weights(wts, s, STAGE, k0, k1);
  Stager<T> st;
  st.init(s, eq, i0, j0);
#pragma unroll
  for (int u = 0; u < PD; ++u)
    if (k0 + u < k1) st.load(u, src, k0 + u, p.N);
  int buf = 0;
  for (int kb = k0; kb < k1; kb += PD) {
#pragma unroll
    for (int u = 0; u < PD; ++u) {
      const int k = kb + u;
      if (k >= k1) break;                            // uniform over the block
      const V4 e4 = ld4(vq + p.nv + k);
      st.store(u, gs[buf], b, e4.x, e4.y, e4.z);
      if (k + PD < k1) st.load(u, src, k + PD, p.N);
      // the cells' own values (L1 / L2 hits: the plane is being staged)
      C own[2], fown[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        own[q] = ok[q] ? ldv(src + (size_t)k * p.N + cell[q]) : C(0);
        fown[q] = (STAGE == 2 && ok[q]) ? lds(fh + (size_t)k * p.N + cell[q]) : C(0);
      }
      __syncthreads();
      stage_ghosts<C>(p, gs[buf], i0, j0, wx, wy);
      FaceW fw;
      face_weights(fw, wts + (k - k0) * WPV, e4.x, e4.y);
      {
        // window: staged rows 2w .. 2w + 4, columns lane .. lane + 3
        C Wn[5][4];
        const C* g0 = gs[buf] + (2 * warp) * HXT + lane;
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) Wn[r][c] = g0[r * HXT + c];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int r = 2 * warp + q, j = j0 + r;
          // cell (lane, r) sits at window (2, 2 + q)
          C vx = xface(fw, Wn, 1, 2 + q);
          if (!p.px && i == 0 && j < p.ny) vx = wfx[(size_t)k * 2 * p.ny + j];
          if (!p.px && i == p.nx && j < p.ny) vx = wfx[(size_t)k * 2 * p.ny + p.ny + j];
          fxs[r][lane] = vx;
          C vy = yface(fw, Wn, 2, 1 + q);
          if (!p.py && j == 0 && i < p.nx) vy = wfy[(size_t)k * 2 * p.nx + i];
          if (!p.py && j == p.ny && i < p.nx) vy = wfy[(size_t)k * 2 * p.nx + p.nx + i];
          fys[r][lane] = vy;
        }
      }
      if (extra) {
        const C* g = gs[buf];
        if (ex_id < TYT) {                           // x-face i0 + 32 of row ex_id
          const int r = ex_id, ii = i0 + TXT, j = j0 + r;
          C v = xface_at(fw, g, TXT + 2, r + 2);
          if (!p.px && ii == p.nx && j < p.ny) v = wfx[(size_t)k * 2 * p.ny + p.ny + j];
          fxs[r][TXT] = v;
        } else {                                     // y-face j0 + 16 of column ex_id - 16
          const int c = ex_id - TYT, ii = i0 + c, j = j0 + TYT;
          C v = yface_at(fw, g, c + 2, TYT + 2);
          if (!p.py && j == p.ny && ii < p.nx) v = wfy[(size_t)k * 2 * p.nx + p.nx + ii];
          fys[TYT][c] = v;
        }
      }
      __syncthreads();
      const V4 k4 = ld4(vq + 2 * p.nv + k);
      const C kx = STAGE == 1 ? k4.x : k4.z, ky = STAGE == 1 ? k4.y : k4.w;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!ok[q]) continue;
        const int r = 2 * warp + q;
        const C fW = fxs[r][lane], fE = fxs[r][lane + 1];
        const C fS = fys[r][lane], fN = fys[r + 1][lane];
        const C df = fmx(kx, fE - fW, ky * (fN - fS));
        const C ws = fmx(e4.z, cubic<C>(S[q], e4.x, e4.y), df);
        C out;
        if (STAGE == 1) {
          out = fmx(-cB, own[q], own[q] + ws);                 // cB = sP
        } else {
          out = fmx(cA, fown[q] - own[q], fmx(-cB, own[q], own[q] + ws));   // cB = sP + sQ
        }
        const C ov = stored_value<T>(out);    // the moments are those of the stored value
        stv(dst + (size_t)k * p.N + cell[q], ov);
        kah_add(am[q][0], ov);
        kah_add(am[q][1], e4.x * ov);
        kah_add(am[q][2], e4.y * ov);
      }
      buf ^= 1;
    }
  }
  double* pc = s.pc + (size_t)chunk * 3 * p.N;
#pragma unroll
  for (int q = 0; q < 2; ++q)
    if (ok[q])
#pragma unroll
      for (int m = 0; m < 3; ++m) pc[(size_t)m * p.N + cell[q]] = kah_value(am[q][m]);
}

template <typename T>
cudaError_t allow_gnc() {
  cudaError_t e = cudaFuncSetAttribute(k_gnc_faces<T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gnc_update<T, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gnc_update<T, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

int items(const GncStep& s) { return s.tiles_x * s.tiles_y * s.nch; }

}  // namespace

void gnc_weight_table(const DevParams& p, const double* xi_x, const double* xi_y,
                      const StageCoef& s1, const StageCoef& s2, float* out) {
  for (int st = 0; st < 2; ++st) {
    const double h = st == 0 ? s1.h : s2.h;
    for (int k = 0; k < p.nv; ++k) {
      const double ax = -xi_x[k] * h * p.inv_dx, by = -xi_y[k] * h * p.inv_dy;
      const double ab[4][2] = {{0.5 + ax, by}, {-0.5 + ax, by}, {ax, 0.5 + by}, {ax, -0.5 + by}};
      float* row = out + ((size_t)st * p.nv + k) * WPV;
      for (int set = 0; set < 4; ++set) {
        double w[9];
        flux_ds_weights<double>(ab[set][0], ab[set][1], w);
        for (int q = 0; q < 12; ++q) row[set * 12 + q] = q < 9 ? (float)w[q] : 0.0f;
      }
    }
  }
}

int gnc_chunks(const DevParams& p, int sms) {
  const int tiles = ((p.nx + TXT - 1) / TXT) * ((p.ny + TYT - 1) / TYT);
  const int want = (4 * 2 * sms + tiles - 1) / tiles;        // about four waves of two blocks per SM
  const int cap = (p.nv + KCMAX - 1) / KCMAX;                 // at most KCMAX velocities per chunk
  return std::max(1, std::min(p.nv, std::max(want, cap)));
}

cudaError_t gnc_prepare(int store) {
  if (store == 1) return allow_gnc<float>();
  if (store == 2) return allow_gnc<__nv_bfloat16>();
  return cudaErrorInvalidValue;
}

cudaError_t launch_gnc_moments(const GncStep& s, cudaStream_t st) {
  const dim3 grid((s.p.N + 255) / 256, s.nch);
  if (s.store == 1) k_gnc_moments<float><<<grid, 256, 0, st>>>(s);
  else k_gnc_moments<__nv_bfloat16><<<grid, 256, 0, st>>>(s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gnc_cellfin<float><<<(s.p.N + 255) / 256, 256, 0, st>>>(s, 0);
  return cudaGetLastError();
}

cudaError_t launch_gnc_faces(const GncStep& s, int stage, cudaStream_t st) {
  if (s.store == 1) k_gnc_faces<float><<<items(s), NTH, 0, st>>>(s, stage);
  else k_gnc_faces<__nv_bfloat16><<<items(s), NTH, 0, st>>>(s, stage);
  return cudaGetLastError();
}

cudaError_t launch_gnc_walls(const GncStep& s, int stage, cudaStream_t st) {
  const int nwx = s.p.px ? 0 : 2 * s.p.ny, nwy = s.p.py ? 0 : 2 * s.p.nx;
  if (nwx + nwy == 0) return cudaSuccess;
  if (s.store == 1) k_gnc_walls<float><<<nwx + nwy, 256, 0, st>>>(s, stage, nwx);
  else k_gnc_walls<__nv_bfloat16><<<nwx + nwy, 256, 0, st>>>(s, stage, nwx);
  return cudaGetLastError();
}

cudaError_t launch_gnc_facefin(const GncStep& s, cudaStream_t st) {
  const int nf = s.p.ny * (s.p.nx + 1) + (s.p.ny + 1) * s.p.nx;
  k_gnc_facefin<float><<<(nf + 255) / 256, 256, 0, st>>>(s);
  return cudaGetLastError();
}

// the update of a stage followed by the cell moments of its output
cudaError_t launch_gnc_update(const GncStep& s, int stage, cudaStream_t st) {
  const double a1 = s.s1.a, b1 = s.s1.b, dt = s.p.dt;
  const double c34 = 0.75 * s.c_om;
  // cB: the coefficient subtracted from the base (sP, or sP + sQ), formed
  // from the values the kernel puts into S, in the compute type
  double cA = 0.0, cB, sP, sQ = 0.0, sF;
  auto rc = [](double x) { return (double)(float)x; };
  if (stage == 1) {
    sP = rc(1.25 * b1);
    sF = -(dt / 3.0) * s.s1.beta;
    cB = sP;
  } else {
    cA = 4.0 / 7.0 - 6.0 / 7.0 * a1;
    sP = rc(-6.0 / 7.0 * b1);
    sQ = rc(-c34);
    sF = -(4.0 * dt / 7.0) * s.s2.beta;
    cB = (double)((float)sP + (float)sQ);
  }
  const int n = items(s);
  if (s.store == 1) {
    if (stage == 1) k_gnc_update<float, 1><<<n, NTH, 0, st>>>(s, (float)cA, (float)cB, (float)sP, (float)sQ, (float)sF);
    else k_gnc_update<float, 2><<<n, NTH, 0, st>>>(s, (float)cA, (float)cB, (float)sP, (float)sQ, (float)sF);
  } else {
    if (stage == 1) k_gnc_update<__nv_bfloat16, 1><<<n, NTH, 0, st>>>(s, (float)cA, (float)cB, (float)sP, (float)sQ, (float)sF);
    else k_gnc_update<__nv_bfloat16, 2><<<n, NTH, 0, st>>>(s, (float)cA, (float)cB, (float)sP, (float)sQ, (float)sF);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int which = stage == 1 ? 1 : 0;
  k_gnc_cellfin<float><<<(s.p.N + 255) / 256, 256, 0, st>>>(s, which);
  return cudaGetLastError();
}

}  // namespace dugks
