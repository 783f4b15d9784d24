// Optimised generic path of the T3S3 step for any velocity set (Newton-Cotes
// grids in particular), periodic / bounce-back / diffuse walls, FP64
// storage (the FP32 / BF16 deviation forms run on the class-moment kernels
// of dugks_gnc.cu).  Per stage:
//   cell pass -> ghosts -> interior faces x, y (stencils + face moments)
//   -> face parameters -> wall faces -> update.
//
// The kernels are templated on the storage type T and compute type C (the
// deviation forms ran on them until the class-moment kernels replaced them
// and are no longer instantiated): T = double computes in FP64 (plain FP64
// sums; reference density rho0 = 0, so the arrays hold f itself).  T =
// float / bf16 hold the deviation d = f - W_k rho0 and compute stencils,
// face values, stage transforms and the per-velocity equilibrium assembly
// W_k((rho - rho0) + rho (P_k - 1)) in FP32; their moment sums (Sec. 2.2)
// are carried per thread as unevaluated FP32 pairs (hi + lo) updated by
// error-free transformations -- TwoSum for each term, and the exact FMA
// residual of xi_hi d plus xi_lo d for the momentum, xi = xi_hi + xi_lo -- so
// a partial keeps ~48 significant bits; partials are combined across
// threads, warps and velocity chunks in FP64, and rho, u/RT and |u|^2/(2RT)
// are FP64 before they are rounded for the assembly (Sec. 2.1.1
// equilibrium).  No FP64 arithmetic or conversion sits in an inner loop of
// the FP32 forms: GB300 runs both on its 2-lane-per-clock FP64 pipe.  The
// maps of the step (eqs. f_bar_1_6, fbp_5_12, recover2f, f_tilde_1_3, fhp,
// feqIntD3rdHat2_DS) are affine with coefficients summing to one and the
// flux divergence of a uniform field vanishes, so they act on deviations
// unchanged.
//
// The stage field g = f-bar^{+,h} lives in a padded layout
// g[k][ny + 4][pitch], cell (i, j) at row j + 2, column i + 2, with two
// ghost layers: periodic copies, or the quadratic extrapolation across a
// wall (g_-1 = 3 g_0 - 3 g_1 + g_2; the second layer repeats the first and
// feeds no face).  The pitch is a multiple of 8 elements with room for a
// 16-byte chunk past column nx + 1, so the face kernels stage their slabs
// with aligned 16-byte asynchronous copies and no boundary logic.
#include "dugks_gcommon.cuh"

namespace dugks {

namespace {

constexpr int kThreads = 256;
constexpr int NW = 8, R = 8, LANES = 32;

// padded offset of cell (i, j) (ghosts: -2 <= i <= nx + 1, -2 <= j <= ny + 1)
__device__ __forceinline__ size_t gp_at(const GDevStep& s, int k, int i, int j) {
  return (size_t)k * s.plane + (size_t)(j + 2) * s.pitch + (i + 2);
}

// ---------------------------------------------------------------- cell
// The cell pass of a stage: moments of src (f^ or f~') -> rho, u (FP64, into
// mom) and the assembly parameters (eqp [5][N]); g = a src + b feq, into the
// padded layout.
//
// Small velocity sets: one thread per cell does both sweeps.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gcell1(GDevStep s, const T* __restrict__ src, typename Prec<T>::C a, typename Prec<T>::C b) {
  using C = typename Prec<T>::C;
  using V4 = typename Prec<T>::V4;
  const DevParams& p = s.p;
  const V4* vq = (const V4*)s.vq;
  T* __restrict__ g = (T*)s.g;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.N) return;
  const int nv = p.nv;
  Acc<C> s0{}, s1{}, s2{};
  for (int k = 0; k < nv; ++k) {
    const C d = ldv(src + (size_t)k * p.N + cell);
    const V4 xq = ld4(vq + k);
    acc_add(s0, d);
    acc_addprod(s1, xq.x, xq.y, d);
    acc_addprod(s2, xq.z, xq.w, d);
  }
  const GDevRef& ref = s.ref;
  const double rho = ref.W + acc_value(s0);
  const double rinv = 1.0 / rho;
  const double ux = (ref.Wx + acc_value(s1)) * rinv, uy = (ref.Wy + acc_value(s2)) * rinv;
  const EqF<C> q = eq_params_u<C>(rho, ux, uy, p.inv_RT, ref.rho0);
  s.mom[cell] = rho;
  s.mom[p.N + cell] = ux;
  s.mom[2 * p.N + cell] = uy;
  store_par((C*)s.eqp, p.N, cell, q);
  const int j = cell / p.nx, i = cell - j * p.nx;
  for (int k = 0; k < nv; ++k) {
    const V4 e4 = ld4(vq + nv + k);
    const C fe = feq_dev<C>(q, e4.x, e4.y, e4.z);
    stv(g + gp_at(s, k, i, j), fmx(b, fe, a * ldv(src + (size_t)k * p.N + cell)));
  }
}

// Large velocity sets, three kernels.  (1) Partial moments: 32 cells per
// block, 8 warps over a velocity chunk (eight loads in flight per thread),
// per-thread partials combined in FP64, into part[chunk][3][N].
// TG (tensor grid, chunks of whole rows of n velocities sharing xi_x): per
// row a compensated sum S of the terms and their xi_y-weighted sum, then
// rho += S and rho u_x += xi_x S once per row.
template <typename T, bool TG>
__global__ void __launch_bounds__(kThreads)
k_gmom(GDevStep s, const T* __restrict__ src, int kchunk, int n) {
  using C = typename Prec<T>::C;
  using V4 = typename Prec<T>::V4;
  constexpr int TX = 32, G = kThreads / TX, U = 8;
  __shared__ double red[3][G][TX];
  const DevParams& p = s.p;
  const V4* vq = (const V4*)s.vq;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int cell = blockIdx.x * TX + tx;
  const bool valid = cell < p.N;
  const int k0 = blockIdx.y * kchunk, k1 = min(p.nv, k0 + kchunk);
  Acc<C> s0{}, s1{}, s2{};
  if (valid && TG) {
    for (int row = k0; row < k1; row += n) {
      Acc<C> sr{};
      for (int k = row + ty; k < row + n; k += U * G) {
        T d[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k + u * G < row + n) d[u] = ldr(src + (size_t)(k + u * G) * p.N + cell);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (k + u * G < row + n) {
            const V4 xq = ld4(vq + k + u * G);
            const C du = tof(d[u]);
            acc_add(sr, du);
            acc_addprod(s2, xq.z, xq.w, du);
          }
        }
      }
      const V4 xr = ld4(vq + row);                   // the row's xi_x (hi, lo)
      acc_add_acc(s0, sr);
      acc_addprod_acc(s1, xr.x, xr.y, sr);
    }
  } else if (valid) {
    int k = k0 + ty;
    for (; k + (U - 1) * G < k1; k += U * G) {
      T d[U];
#pragma unroll
      for (int u = 0; u < U; ++u) d[u] = ldr(src + (size_t)(k + u * G) * p.N + cell);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const V4 xq = ld4(vq + k + u * G);
        const C du = tof(d[u]);
        acc_add(s0, du);
        acc_addprod(s1, xq.x, xq.y, du);
        acc_addprod(s2, xq.z, xq.w, du);
      }
    }
    for (; k < k1; k += G) {
      const C du = ldv(src + (size_t)k * p.N + cell);
      const V4 xq = ld4(vq + k);
      acc_add(s0, du);
      acc_addprod(s1, xq.x, xq.y, du);
      acc_addprod(s2, xq.z, xq.w, du);
    }
  }
  red[0][ty][tx] = acc_value(s0);
  red[1][ty][tx] = acc_value(s1);
  red[2][ty][tx] = acc_value(s2);
  __syncthreads();
  if (ty < 3 && valid) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < G; ++q) t += red[ty][q][tx];
    s.part[((size_t)blockIdx.y * 3 + ty) * p.N + cell] = t;
  }
}

// (2) Per cell: the chunks' partials in order -> rho, u, mom, eqp.
template <typename C>
__global__ void __launch_bounds__(kThreads)
k_gmomfin(GDevStep s, int nchunk) {
  const DevParams& p = s.p;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.N) return;
  double v0 = s.ref.W, v1 = s.ref.Wx, v2 = s.ref.Wy;
  for (int c = 0; c < nchunk; ++c) {
    const double* pc = s.part + (size_t)c * 3 * p.N;
    v0 += pc[cell];
    v1 += pc[p.N + cell];
    v2 += pc[2 * p.N + cell];
  }
  const double rinv = 1.0 / v0;
  const double ux = v1 * rinv, uy = v2 * rinv;
  const EqF<C> q = eq_params_u<C>(v0, ux, uy, p.inv_RT, s.ref.rho0);
  s.mom[cell] = v0;
  s.mom[p.N + cell] = ux;
  s.mom[2 * p.N + cell] = uy;
  store_par((C*)s.eqp, p.N, cell, q);
}

// (3) g = a src + b W_k P(xi_k): one thread per cell and 16 consecutive
// velocities (two batches of eight loads in flight), P the cell's
// equilibrium quadratic in xi.
template <typename T, bool TG>
__global__ void __launch_bounds__(kThreads)
k_gcellg(GDevStep s, const T* __restrict__ src, typename Prec<T>::C a, typename Prec<T>::C b) {
  using C = typename Prec<T>::C;
  using V4 = typename Prec<T>::V4;
  constexpr int CB = 16, CH = 8;
  const DevParams& p = s.p;
  const V4* vq = (const V4*)s.vq;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.N) return;
  const int nv = p.nv;
  const int j = cell / p.nx, i = cell - j * p.nx;
  const Quad<C> P = quad((const C*)s.eqp, p.N, cell);   // W_k P: W_k (rho P_k - rho0)
  // TG (tensor grid): the 16 velocities share xi_x, P(x, y) = a + y (b + y c)
  const C x0 = TG ? ld4(vq + nv + blockIdx.y * CB).x : C(0);
  const C pa = fmx(x0, fmx(x0, P.cxx, P.cx), P.c0), pb = fmx(x0, P.cxy, P.cy);
  T* __restrict__ g = (T*)s.g;
  for (int h = 0; h < CB; h += CH) {
    const int kb = blockIdx.y * CB + h;
    T d[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (kb + u < nv) d[u] = ldr(src + (size_t)(kb + u) * p.N + cell);
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int k = kb + u;
      if (k < nv) {
        const V4 e4 = ld4(vq + nv + k);
        const C x = e4.x, y = e4.y;
        const C pk = TG ? fmx(y, fmx(y, P.cyy, pb), pa)
                        : fmx(x, fmx(x, P.cxx, fmx(y, P.cxy, P.cx)), fmx(y, fmx(y, P.cyy, P.cy), P.c0));
        stv(g + gp_at(s, k, i, j), fmx(b * e4.z, pk, a * tof(d[u])));
      }
    }
  }
}

// ---------------------------------------------------------------- ghosts
// The two ghost layers of every velocity plane of g.  Positions are
// periodic copies, or one layer of quadratic extrapolation across a wall
// (along x of the y-extrapolated columns at corners); the second layer
// beyond a wall repeats the first.  Reads interior cells only.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gghost(GDevStep s) {
  using C = typename Prec<T>::C;
  const DevParams& p = s.p;
  const int nx = p.nx, ny = p.ny;
  const int W = nx + 4;
  const int per = 4 * W + 4 * ny;                 // rows -2,-1,ny,ny+1 (all columns) + 4 columns
  const int k = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per) return;
  int x, y;
  if (t < 4 * W) {
    const int rsel = t / W;
    x = t - rsel * W - 2;
    y = rsel < 2 ? rsel - 2 : ny + rsel - 2;
  } else {
    const int u = t - 4 * W;
    const int csel = u / ny;
    y = u - csel * ny;
    x = csel < 2 ? csel - 2 : nx + csel - 2;
  }
  T* __restrict__ g = (T*)s.g;
  const T* gk = g + (size_t)k * s.plane;
  int xx = x, yy = y;
  if (p.px) xx = (xx + nx) % nx;
  else xx = xx < -1 ? -1 : (xx > nx ? nx : xx);
  if (p.py) yy = (yy + ny) % ny;
  else yy = yy < -1 ? -1 : (yy > ny ? ny : yy);
  auto at = [&](int i, int j) -> C { return ldv(gk + (size_t)(j + 2) * s.pitch + (i + 2)); };
  auto col = [&](int i, int j) -> C {
    if (j < 0 || j >= ny) {
      const int b = j < 0 ? 0 : ny - 1, sg = j < 0 ? 1 : -1;
      return C(3) * at(i, b) - C(3) * at(i, b + sg) + at(i, b + 2 * sg);
    }
    return at(i, j);
  };
  C v;
  if (xx < 0 || xx >= nx) {
    const int b = xx < 0 ? 0 : nx - 1, sg = xx < 0 ? 1 : -1;
    v = C(3) * col(b, yy) - C(3) * col(b + sg, yy) + col(b + 2 * sg, yy);
  } else {
    v = col(xx, yy);
  }
  stv(g + gp_at(s, k, x, y), v);
}

// face-value weights about a cell for the foot offset (a dx, b dy) (eq.
// flux_DS as printed, central differences on the 3x3 neighbourhood):
// T[(dy+1)*3 + dx+1]
template <typename C>
__device__ __forceinline__ void taylor9(C a, C b, C (&T)[9]) {
  flux_ds_weights<C>(a, b, T);
}

// ---------------------------------------------------------- interior faces
// Pass 1: lanes over 32 faces, warps over velocities, R face rows per block.
// Each warp stages the slab of g its velocity needs (SR rows x SW columns,
// from padded column c0) in shared memory with 16-byte asynchronous copies,
// double-buffered so the next velocity's slab loads while the current one
// is used; stencils in C, per-thread partial face moments, combined in FP64
// per velocity chunk into part[chunk][3][nf].
// Face-pass grid: face columns 0 .. nx of the x faces (0 .. nx - 1 with
// walls in x: faces 0 and nx are the wall kernel's), all nx columns of the
// y faces; rows likewise.
inline int face_blocks_x(const DevParams& p, int dir) {
  return (p.nx + (dir == 0 && p.px ? 1 : 0) + LANES - 1) / LANES;
}
inline int face_blocks_y(const DevParams& p, int dir) {
  return (p.ny + (dir == 1 && p.py ? 1 : 0) + R - 1) / R;
}

template <typename T, int DIR>
struct Slab {
  static constexpr int SR = DIR == 0 ? R + 2 : R + 3;          // rows
  static constexpr int SW = sizeof(T) == 2 ? 40 : 36;          // columns (x 16-byte chunks)
  static constexpr int EPC = 16 / (int)sizeof(T);              // elements per chunk
  static constexpr int CPR = SW / EPC;                         // chunks per row
  static constexpr int NCH = SR * CPR;
  static constexpr int ELEMS = SR * SW;
  // dynamic shared memory: the warps' double-buffered slabs, later reused
  // for the cross-warp reduction of the face moments
  static constexpr size_t SLAB_BYTES = (size_t)NW * 2 * ELEMS * sizeof(T);
  static constexpr size_t RED_BYTES = (size_t)NW * R * LANES * 3 * sizeof(double);
  static constexpr size_t BYTES = SLAB_BYTES > RED_BYTES ? SLAB_BYTES : RED_BYTES;
};

template <typename T, int DIR>
__global__ void __launch_bounds__(LANES * NW, 2)
k_gfaces1(GDevStep s, typename Prec<T>::C* __restrict__ fb, typename Prec<T>::C h, int kchunk,
          const double* __restrict__ tws) {
  using C = typename Prec<T>::C;
  using V4 = typename Prec<T>::V4;
  using S = Slab<T, DIR>;
  constexpr int SW = S::SW;
  // the stencil reads rows r .. r + 2 (+1 for y faces) and columns
  // lane .. lane + 3 of the slab
  static_assert(S::SR >= R + (DIR == 0 ? 2 : 3) && SW >= LANES + 3, "slab too small");
  extern __shared__ __align__(16) double smem[];
  auto red = [&](int w, int r, int l, int m) -> double& {
    return smem[((w * R + r) * LANES + l) * 3 + m];
  };
  const DevParams& p = s.p;
  const V4* vq = (const V4*)s.vq;
  const T* __restrict__ g = (const T*)s.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nx = p.nx, ny = p.ny, nv = p.nv;
  const int nf = DIR == 0 ? ny * (nx + 1) : (ny + 1) * nx;
  const int c0 = blockIdx.x * LANES, r0 = blockIdx.y * R;
  const int k0 = blockIdx.z * kchunk, k1 = min(nv, k0 + kchunk);
  // slab origin in padded coordinates: column c0 (cell c0 - 2); first row
  // cell r0 - 1 (x faces) or r0 - 2 (y faces)
  const int prow0 = DIR == 0 ? r0 + 1 : r0;
  const int prows = ny + 4;
  const C dx = (C)p.dx, dy = (C)p.dy;
  const C idx_ = (C)p.inv_dx, idy = (C)p.inv_dy;
  Acc<C> acc[R][3];
  bool ok[R];
  const int col = c0 + lane;
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int m = 0; m < 3; ++m) acc[r][m] = Acc<C>{};
    if (DIR == 0) {
      const int j = r0 + r;
      ok[r] = j < ny && col <= nx && (p.px || (col >= 1 && col <= nx - 1));
    } else {
      const int fj = r0 + r;
      ok[r] = col < nx && fj <= ny && (p.py || (fj >= 1 && fj <= ny - 1));
    }
  }
  T* slab = reinterpret_cast<T*>(smem) + warp * 2 * S::ELEMS;
  // issue the copies of velocity k's slab into buffer b (chunks beyond the
  // padded plane feed no face and are skipped)
  auto issue = [&](int k, int b) {
    const T* gk = g + (size_t)k * s.plane;
    T* dst = slab + b * S::ELEMS;
    for (int e = lane; e < S::NCH; e += LANES) {
      const int rr = e / S::CPR, cc = (e - rr * S::CPR) * S::EPC;
      const int pr = prow0 + rr, pc = c0 + cc;
      if (pr < prows && pc + S::EPC <= s.pitch)
        cp16(dst + rr * SW + cc, gk + (size_t)pr * s.pitch + pc);
    }
  };
  int b = 0;
  if (k0 + warp < k1) issue(k0 + warp, 0);
  cp_commit();
  for (int k = k0 + warp; k < k1; k += NW) {
    if (k + NW < k1) issue(k + NW, b ^ 1);
    cp_commit();
    const V4 xq = ld4(vq + k);                     // xi_x hi, lo, xi_y hi, lo
    const C cx = xq.x, cxl = xq.y, cy = xq.z, cyl = xq.w;
    const C cn = DIR == 0 ? cx : cy;
    // the upwind cell is the lower one (slab offset 0) for xi.n > 0 and the
    // upper one (one column / row on) for xi.n < 0; xi.n = 0 averages both
    // (uniform across the warp)
    const bool up = cn < C(0), tie = cn == C(0);
    C Tw[9];
    if constexpr (sizeof(C) == 8) {
      // FP64: the stage's weights from the table [k][lower 9, upper 9]
      const double* w = tws + (size_t)k * 18 + (up ? 9 : 0);
#pragma unroll
      for (int q = 0; q < 9; ++q) Tw[q] = __ldg(w + q);
    } else {
      const C sh = up ? C(-0.5) : C(0.5);
      if (DIR == 0) taylor9<C>((sh * dx - cx * h) * idx_, -cy * h * idy, Tw);
      else taylor9<C>(-cx * h * idx_, (sh * dy - cy * h) * idy, Tw);
    }
    cp_wait1();                                    // this velocity's slab has landed
    __syncwarp();
    // x faces: rows r..r+2 (cells j-1..j+1), columns lane+q (cells fi-2+q);
    // y faces: rows r+q (cells fj-2+q), columns lane+1+q (cells i-1+q)
    const T* sl = slab + b * S::ELEMS + lane + (DIR == 0 ? 0 : 1);
    const int uoff = DIR == 0 ? 1 : SW;            // lower -> upper cell
    C* fbk = fb + (size_t)k * nf;
    if (!tie) {
      const T* sb = sl + (up ? uoff : 0);
      // FP32 arithmetic (issue-bound): a sliding window of three stencil
      // rows reads each slab row once; FP64 (FP64-pipe-bound, at its
      // register limit) reads the nine values per face
      constexpr bool WIN = sizeof(C) == 4;
      C wr[3][3];
      if constexpr (WIN) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int q = 0; q < 3; ++q) wr[a + 1][q] = lds(sb + a * SW + q);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            if constexpr (WIN) {
              if (a < 2) wr[a][q] = wr[a + 1][q];
              else wr[2][q] = lds(sb + (r + 2) * SW + q);
            } else {
              wr[a][q] = lds(sb + (r + a) * SW + q);
            }
          }
        C v = C(0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int q = 0; q < 3; ++q) v = fmx(Tw[a * 3 + q], wr[a][q], v);
        const int face = DIR == 0 ? (r0 + r) * (nx + 1) + col : (r0 + r) * nx + col;
        if (ok[r]) fbk[face] = v;
        acc_add(acc[r][0], v);                     // rows without a face are never stored
        acc_addprod(acc[r][1], cx, cxl, v);
        acc_addprod(acc[r][2], cy, cyl, v);
      }
    } else {
      C Tu[9];
      if constexpr (sizeof(C) == 8) {
#pragma unroll
        for (int q = 0; q < 9; ++q) Tu[q] = __ldg(tws + (size_t)k * 18 + 9 + q);
      } else {
        if (DIR == 0) taylor9<C>((C(-0.5) * dx - cx * h) * idx_, -cy * h * idy, Tu);
        else taylor9<C>(-cx * h * idx_, (C(-0.5) * dy - cy * h) * idy, Tu);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const T* s0 = sl + r * SW;
        C vl = C(0), vu = C(0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            vl = fmx(Tw[a * 3 + q], lds(s0 + a * SW + q), vl);
            vu = fmx(Tu[a * 3 + q], lds(s0 + uoff + a * SW + q), vu);
          }
        const C v = C(0.5) * (vl + vu);
        const int face = DIR == 0 ? (r0 + r) * (nx + 1) + col : (r0 + r) * nx + col;
        if (ok[r]) fbk[face] = v;
        acc_add(acc[r][0], v);
        acc_addprod(acc[r][1], cx, cxl, v);
        acc_addprod(acc[r][2], cy, cyl, v);
      }
    }
    __syncwarp();                                  // buffer b is refilled two velocities on
    b ^= 1;
  }
  cp_wait_all();
  __syncthreads();                                 // all slabs done: reuse the memory
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int m = 0; m < 3; ++m) red(warp, r, lane, m) = acc_value(acc[r][m]);
  __syncthreads();
  for (int e = threadIdx.x; e < R * LANES; e += LANES * NW) {
    const int r = e / LANES, l = e - r * LANES;
    const int cc = c0 + l;
    bool okf;
    int face;
    if (DIR == 0) {
      okf = (r0 + r) < ny && cc <= nx && (p.px || (cc >= 1 && cc <= nx - 1));
      face = (r0 + r) * (nx + 1) + cc;
    } else {
      okf = cc < nx && (r0 + r) <= ny && (p.py || ((r0 + r) >= 1 && (r0 + r) <= ny - 1));
      face = (r0 + r) * nx + cc;
    }
    if (!okf) continue;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      s0 += red(w, r, l, 0);
      s1 += red(w, r, l, 1);
      s2 += red(w, r, l, 2);
    }
    double* pc = s.part + (size_t)blockIdx.z * 3 * nf;
    pc[face] = s0;
    pc[nf + face] = s1;
    pc[2 * nf + face] = s2;
  }
}

// Face parameters of the interior faces: the face moments (FP64, velocity
// chunks summed in order) and the assembly parameters of the face
// equilibrium, fpar[5][nf] (eq. recover2f is applied where the update reads
// the face values: f = alpha f-bar + beta feq).  Wall faces are skipped.
template <typename C, int DIR>
__global__ void __launch_bounds__(256)
k_gfacepar(GDevStep s, C* __restrict__ fpar, int nchunk) {
  const DevParams& p = s.p;
  const int nx = p.nx, ny = p.ny;
  const int nf = DIR == 0 ? ny * (nx + 1) : (ny + 1) * nx;
  const int face = blockIdx.x * blockDim.x + threadIdx.x;
  if (face >= nf) return;
  if (DIR == 0) {
    const int fi = face % (nx + 1);
    if (!p.px && (fi == 0 || fi == nx)) return;
  } else {
    const int fj = face / nx;
    if (!p.py && (fj == 0 || fj == ny)) return;
  }
  double r = s.ref.W, jx = s.ref.Wx, jy = s.ref.Wy;
  for (int c = 0; c < nchunk; ++c) {
    const double* pc = s.part + (size_t)c * 3 * nf;
    r += pc[face];
    jx += pc[nf + face];
    jy += pc[2 * nf + face];
  }
  store_par(fpar, nf, face, eq_params_j<C>(r, jx, jy, p.inv_RT, s.ref.rho0));
}

// -------------------------------------------------------------- wall faces
// One wall face per block (both directions in one launch), the threads over
// the velocity set: fluid-side reconstruction (velocities leaving the fluid
// or along the wall), the wall rule of Sec. 2.3 for velocities entering the
// fluid (bounce-back with the moving-wall term, or diffuse scattering with
// the density that balances the outgoing flux), f-bar into fb, the face
// moments (per-thread partials, FP64 across the block) and the face's
// assembly parameters into fpar.  Per direction, face
// id = 2 line + (0: W/S wall, 1: E/N).
template <typename T, typename C>
__device__ __forceinline__ C taylor_at(const GDevStep& s, const T* __restrict__ g, int k, int ci,
                                       int cj, C X, C Y) {
  C Tw[9];
  taylor9<C>(X * (C)s.p.inv_dx, Y * (C)s.p.inv_dy, Tw);
  C v = C(0);
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx)
      v = fmx(Tw[(dy + 1) * 3 + dx + 1], ldv(g + gp_at(s, k, ci + dx, cj + dy)), v);
  return v;
}

template <typename T, int DIR>
__device__ __forceinline__ void wall_face(const GDevStep& s, int id, typename Prec<T>::C h,
                                          double* sm) {
  using C = typename Prec<T>::C;
  using V4 = typename Prec<T>::V4;
  const DevParams& p = s.p;
  const GDevRef& ref = s.ref;
  const V4* vq = (const V4*)s.vq;
  const T* __restrict__ g = (const T*)s.g;
  C* __restrict__ fb = (C*)(DIR == 0 ? s.fbx : s.fby);
  C* __restrict__ fpar = (C*)(DIR == 0 ? s.fpx : s.fpy);
  const int nx = p.nx, ny = p.ny, nv = p.nv;
  const int nf = DIR == 0 ? ny * (nx + 1) : (ny + 1) * nx;
  const bool upper_wall = id & 1;                 // east / north
  const int line = id >> 1;
  const int face = DIR == 0 ? line * (nx + 1) + (upper_wall ? nx : 0)
                            : (upper_wall ? ny : 0) * nx + line;
  const int side = DIR == 0 ? (upper_wall ? SIDE_E : SIDE_W) : (upper_wall ? SIDE_N : SIDE_S);
  // the fluid cell lies on the +normal side of W/S walls; xi.n with n the
  // fluid's outward normal is -xi_n there and +xi_n at E/N walls
  const bool fluid_hi = !upper_wall;
  const C nsg = fluid_hi ? C(-1) : C(1);
  const int ci = DIR == 0 ? (fluid_hi ? 0 : nx - 1) : line;
  const int cj = DIR == 0 ? line : (fluid_hi ? 0 : ny - 1);
  const int kind = p.bc_kind[side];
  const C half = C(0.5) * (C)(DIR == 0 ? p.dx : p.dy);
  const C off = fluid_hi ? -half : half;          // face centre from the fluid cell centre
  const C rho_w = (C)s.mom[cj * nx + ci];
  const C uwx = (C)p.uw_x[side], uwy = (C)p.uw_y[side];
  const C irt = (C)p.inv_RT;
  auto recon = [&](int k) {
    const V4 e4 = ld4(vq + nv + k);
    const C X = DIR == 0 ? off - e4.x * h : -e4.x * h;
    const C Y = DIR == 0 ? -e4.y * h : off - e4.y * h;
    return taylor_at<T, C>(s, g, k, ci, cj, X, Y);
  };
  // moments of f-bar and the outgoing flux sum(xi.n f-bar)
  Acc<C> a0{}, a1{}, a2{}, a3{};
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    const V4 xq = ld4(vq + k);
    const C cx = xq.x, cy = xq.z;
    const C xn = nsg * (DIR == 0 ? cx : cy);
    C fbar;
    if (xn >= C(0)) {                              // hits the wall or runs along it
      fbar = recon(k);
      if (xn > C(0))
        acc_addprod(a3, DIR == 0 ? nsg * xq.x : nsg * xq.z, DIR == 0 ? nsg * xq.y : nsg * xq.w,
                    fbar);
    } else if (kind == BC_BOUNCEBACK) {
      const int kk = __ldg(p.opp + k);
      const C wk = ld4(vq + nv + k).z;
      const C bbk = C(2) * wk * fmx(cx, uwx, cy * uwy) * irt;
      const C shift = (ld4(vq + nv + kk).z - wk) * (C)ref.rho0;
      fbar = fmx(rho_w, bbk, recon(kk) + shift);
    } else {
      continue;                                    // diffuse: after the reduction
    }
    fb[(size_t)k * nf + face] = fbar;
    acc_add(a0, fbar);
    acc_addprod(a1, xq.x, xq.y, fbar);
    acc_addprod(a2, xq.z, xq.w, fbar);
  }
  double v[4] = {acc_value(a0), acc_value(a1), acc_value(a2), acc_value(a3)};
  block_sum<4>(v, sm);
  if (kind == BC_DIFFUSE) {                        // uniform over the block
    // rho_ds: the outgoing flux of f = W rho0 + d over the wall's flux
    // normaliser (Sec. 2.3 diffuse scattering)
    const double rho_ds = (s.ds_out[side] + v[3]) / p.ds_den[side];
    Acc<C> b0{}, b1{}, b2{};
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
      const V4 xq = ld4(vq + k);
      const C xn = nsg * (DIR == 0 ? xq.x : xq.z);
      if (xn < C(0)) {
        const C fbar =
            to_c<C>(fma(rho_ds, __ldg(p.feq_wall + side * nv + k), -__ldg(p.w + k) * ref.rho0));
        fb[(size_t)k * nf + face] = fbar;
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
    store_par(fpar, nf, face,
              eq_params_j<C>(ref.W + v[0], ref.Wx + v[1], ref.Wy + v[2], p.inv_RT, ref.rho0));
}

// blocks [0, nwx): x-direction walls (W/E), then y-direction walls (S/N)
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gwalls(GDevStep s, typename Prec<T>::C h, int nwx) {
  __shared__ double sm[32 * 4];
  if ((int)blockIdx.x < nwx) wall_face<T, 0>(s, blockIdx.x, h, sm);
  else wall_face<T, 1>(s, blockIdx.x - nwx, h, sm);
}

// ---------------------------------------------------------------- updates
// One thread per cell and KB consecutive velocities (batches of KH loads in
// flight).  Face values are f = alpha f-bar + beta feq (eq. recover2f) and
// L = -(xi_x (f_e - f_w)/dx + xi_y (f_n - f_s)/dy) (eq. microflux).  Every
// equilibrium entering the update -- the four faces' in L, and the cell's
// in the collision term -- is W_k P(xi_k) with P quadratic in xi (Quad).
// Their combination is W_k S(xi_k) with S a cubic in (xi_x, xi_y), whose ten
// coefficients each thread forms once for its cell.
constexpr int KB = 16;

// F(xi) = (x/dx)(P_E - P_W) + (y/dy)(P_N - P_S) for the faces of cell (i, j),
// scaled by sc
template <typename C>
__device__ __forceinline__ Cubic<C> flux_cubic(const GDevStep& s, int i, int j, C sc) {
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


// f~(t') = 5/4 g1 - 1/4 f^ + dt/3 L*,  acc = 1/4 f^ + 3/4 g1 + 3dt/7 L*,
// with dt/3 L* = k1 . (face differences of f-bar) + W S(xi), S = -(dt/3)
// beta F and k1 = -(dt/3) alpha xi/dx (table row 2, x and y)
template <typename T, bool TG>
__global__ void __launch_bounds__(kThreads)
k_gupdate1(GDevStep s, typename Prec<T>::C beta, typename Prec<T>::C dt3,
           typename Prec<T>::C r37) {
  using C = typename Prec<T>::C;
  using V4 = typename Prec<T>::V4;
  constexpr int KH = Prec<T>::KH;
  const DevParams& p = s.p;
  const V4* vq = (const V4*)s.vq;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.N) return;
  const int nx = p.nx, ny = p.ny, nv = p.nv;
  const int j = cell / nx, i = cell - j * nx;
  const Cubic<C> S = flux_cubic<C>(s, i, j, -beta * dt3);
  const size_t nfx = (size_t)ny * (nx + 1), nfy = (size_t)(ny + 1) * nx;
  const C* fbx = (const C*)s.fbx + (size_t)j * (nx + 1) + i;
  const C* fby = (const C*)s.fby + (size_t)j * nx + i;
  // TG (tensor grid): the 16 velocities of this thread share xi_x
  const CubicY<C> SY = cubic_at_x<C>(S, TG ? ld4(vq + nv + blockIdx.y * KB).x : C(0));
  for (int hb = 0; hb < KB; hb += KH) {
    const int kb = blockIdx.y * KB + hb;
    T fh[KH], gg[KH];
    C fv[KH][4];
#pragma unroll
    for (int u = 0; u < KH; ++u) {
      const int k = kb + u;
      if (k < nv) {
        fh[u] = ldr((const T*)s.fhat + (size_t)k * p.N + cell);
        gg[u] = ldr((const T*)s.g + gp_at(s, k, i, j));
        fv[u][0] = __ldg(fbx + k * nfx);
        fv[u][1] = __ldg(fbx + k * nfx + 1);
        fv[u][2] = __ldg(fby + k * nfy);
        fv[u][3] = __ldg(fby + k * nfy + nx);
      }
    }
#pragma unroll
    for (int u = 0; u < KH; ++u) {
      const int k = kb + u;
      if (k < nv) {
        const V4 e4 = ld4(vq + nv + k);
        const V4 k4 = ld4(vq + 2 * nv + k);
        // Ls = dt/3 L*
        const C sk = TG ? cubic_y<C>(SY, e4.y) : cubic<C>(S, e4.x, e4.y);
        const C Ls = fmx(k4.x, fv[u][1] - fv[u][0], fmx(k4.y, fv[u][3] - fv[u][2], e4.z * sk));
        const size_t t = (size_t)k * p.N + cell;
        const C f0 = tof(fh[u]), g0 = tof(gg[u]);
        stv((T*)s.ftp + t, fmx(C(1.25), g0, fmx(C(-0.25), f0, Ls)));
        stv((T*)s.acc + t, fmx(C(0.25), f0, fmx(C(0.75), g0, r37 * Ls)));
      }
    }
  }
}

// f^^{n+1} = acc + 3/4 dt Omega' + 4dt/7 L**,  dt Omega' = c_om (f~' - feq');
// = acc + c34 f~' + k2 . (face differences of f-bar) + W S(xi),
// S = -c34 P_cell - (4dt/7) beta F  (P_cell with -rho0 for the deviations),
// k2 = -(4dt/7) alpha xi/dx (table row 2, z and w)
template <typename T, bool TG>
__global__ void __launch_bounds__(kThreads)
k_gupdate2(GDevStep s, typename Prec<T>::C beta, typename Prec<T>::C c_om34,
           typename Prec<T>::C dt47) {
  using C = typename Prec<T>::C;
  using V4 = typename Prec<T>::V4;
  constexpr int KH = Prec<T>::KH;
  const DevParams& p = s.p;
  const V4* vq = (const V4*)s.vq;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.N) return;
  const int nx = p.nx, ny = p.ny, nv = p.nv;
  const int j = cell / nx, i = cell - j * nx;
  Cubic<C> S = flux_cubic<C>(s, i, j, -dt47 * beta);
  {
    const Quad<C> c = quad((const C*)s.eqp, p.N, cell);
    S.c[0] = fmx(-c_om34, c.c0, S.c[0]);
    S.c[1] = fmx(-c_om34, c.cx, S.c[1]);
    S.c[2] = fmx(-c_om34, c.cy, S.c[2]);
    S.c[3] = fmx(-c_om34, c.cxx, S.c[3]);
    S.c[4] = fmx(-c_om34, c.cxy, S.c[4]);
    S.c[5] = fmx(-c_om34, c.cyy, S.c[5]);
  }
  const size_t nfx = (size_t)ny * (nx + 1), nfy = (size_t)(ny + 1) * nx;
  const C* fbx = (const C*)s.fbx + (size_t)j * (nx + 1) + i;
  const C* fby = (const C*)s.fby + (size_t)j * nx + i;
  const CubicY<C> SY = cubic_at_x<C>(S, TG ? ld4(vq + nv + blockIdx.y * KB).x : C(0));
  for (int hb = 0; hb < KB; hb += KH) {
    const int kb = blockIdx.y * KB + hb;
    T ft[KH], ac[KH];
    C fv[KH][4];
#pragma unroll
    for (int u = 0; u < KH; ++u) {
      const int k = kb + u;
      if (k < nv) {
        const size_t t = (size_t)k * p.N + cell;
        ft[u] = ldr((const T*)s.ftp + t);
        ac[u] = ldr((const T*)s.acc + t);
        fv[u][0] = __ldg(fbx + k * nfx);
        fv[u][1] = __ldg(fbx + k * nfx + 1);
        fv[u][2] = __ldg(fby + k * nfy);
        fv[u][3] = __ldg(fby + k * nfy + nx);
      }
    }
#pragma unroll
    for (int u = 0; u < KH; ++u) {
      const int k = kb + u;
      if (k < nv) {
        const V4 e4 = ld4(vq + nv + k);
        const V4 k4 = ld4(vq + 2 * nv + k);
        const C sk = TG ? cubic_y<C>(SY, e4.y) : cubic<C>(S, e4.x, e4.y);
        const C src = fmx(k4.z, fv[u][1] - fv[u][0], fmx(k4.w, fv[u][3] - fv[u][2], e4.z * sk));
        stv((T*)s.fhat + (size_t)k * p.N + cell, fmx(c_om34, tof(ft[u]), tof(ac[u]) + src));
      }
    }
  }
}

template <typename T>
cudaError_t cell_t(const GDevStep& s, const void* src, const StageCoef& c, cudaStream_t st) {
  using C = typename Prec<T>::C;
  const DevParams& p = s.p;
  if (s.mch <= 1) {
    k_gcell1<T><<<(p.N + kThreads - 1) / kThreads, kThreads, 0, st>>>(s, (const T*)src, (C)c.a,
                                                                    (C)c.b);
  } else {
    const int kchunk = (p.nv + s.mch - 1) / s.mch;
    const dim3 mgrid((p.N + 31) / 32, s.mch);
    // tensor grid with chunks of whole rows (n = sqrt(nv), a multiple of 16),
    // FP64 storage, rows of 64 velocities or more: one FP64 operation per
    // cell-velocity fewer on the FP64 pipe that bounds it (measured: 64 x 64
    // sets gain 1.3 %, the 16 x 16 - 32 x 32 sets of the batched workload
    // lose 3 %; the FP32 / BF16 forms no gain, BF16 a loss)
    int n = 0;
    while ((long)(n + 1) * (n + 1) <= p.nv) ++n;
    if (sizeof(T) == 8 && s.tgrid && n >= 64 && kchunk % n == 0)
      k_gmom<T, true><<<mgrid, kThreads, 0, st>>>(s, (const T*)src, kchunk, n);
    else
      k_gmom<T, false><<<mgrid, kThreads, 0, st>>>(s, (const T*)src, kchunk, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gmomfin<C><<<(p.N + kThreads - 1) / kThreads, kThreads, 0, st>>>(s, s.mch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 grid((p.N + kThreads - 1) / kThreads, (p.nv + 15) / 16);
    if (s.tgrid)
      k_gcellg<T, true><<<grid, kThreads, 0, st>>>(s, (const T*)src, (C)c.a, (C)c.b);
    else
      k_gcellg<T, false><<<grid, kThreads, 0, st>>>(s, (const T*)src, (C)c.a, (C)c.b);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int per = 4 * (p.nx + 4) + 4 * p.ny;
  k_gghost<T><<<dim3((per + kThreads - 1) / kThreads, p.nv), kThreads, 0, st>>>(s);
  return cudaGetLastError();
}

template <typename T, int DIR>
cudaError_t faces_t(const GDevStep& s, int stage, cudaStream_t st) {
  const StageCoef& c = stage == 1 ? s.s1 : s.s2;
  using C = typename Prec<T>::C;
  const DevParams& p = s.p;
  C* fb = (C*)(DIR == 0 ? s.fbx : s.fby);
  C* fpar = (C*)(DIR == 0 ? s.fpx : s.fpy);
  const int nch = DIR == 0 ? s.nchx : s.nchy;
  const int kchunk = (p.nv + nch - 1) / nch;
  const int nf = DIR == 0 ? p.ny * (p.nx + 1) : (p.ny + 1) * p.nx;
  const dim3 grid(face_blocks_x(p, DIR), face_blocks_y(p, DIR), nch);
  const double* tws = s.tw ? s.tw + ((size_t)(stage == 1 ? 0 : 2) + DIR) * p.nv * 18 : nullptr;
  k_gfaces1<T, DIR><<<grid, LANES * NW, Slab<T, DIR>::BYTES, st>>>(s, fb, (C)c.h, kchunk, tws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gfacepar<C, DIR><<<(nf + 255) / 256, 256, 0, st>>>(s, fpar, nch);
  return cudaGetLastError();
}

template <typename T>
cudaError_t walls_t(const GDevStep& s, int stage, cudaStream_t st) {
  using C = typename Prec<T>::C;
  const DevParams& p = s.p;
  const int nwx = p.px ? 0 : 2 * p.ny, nwy = p.py ? 0 : 2 * p.nx;
  if (nwx + nwy == 0) return cudaSuccess;
  const C h = (C)(stage == 1 ? s.s1.h : s.s2.h);
  const int threads = p.nv >= kThreads ? kThreads : ((p.nv + 31) / 32) * 32;
  k_gwalls<T><<<nwx + nwy, threads, 0, st>>>(s, h, nwx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t update_t(const GDevStep& s, int stage, cudaStream_t st) {
  using C = typename Prec<T>::C;
  const DevParams& p = s.p;
  const dim3 grid((p.N + kThreads - 1) / kThreads, (p.nv + KB - 1) / KB);
  const StageCoef& c = stage == 1 ? s.s1 : s.s2;
  const C be = (C)c.beta;
  if (stage == 1) {
    const C dt3 = (C)(p.dt / 3.0), r37 = (C)(9.0 / 7.0);
    if (s.tgrid) k_gupdate1<T, true><<<grid, kThreads, 0, st>>>(s, be, dt3, r37);
    else k_gupdate1<T, false><<<grid, kThreads, 0, st>>>(s, be, dt3, r37);
  } else {
    const C c34 = (C)(0.75 * s.c_om), dt47 = (C)(4.0 * p.dt / 7.0);
    if (s.tgrid) k_gupdate2<T, true><<<grid, kThreads, 0, st>>>(s, be, c34, dt47);
    else k_gupdate2<T, false><<<grid, kThreads, 0, st>>>(s, be, c34, dt47);
  }
  return cudaGetLastError();
}

template <typename T, int DIR>
int occupancy() {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gfaces1<T, DIR>, LANES * NW,
                                                    Slab<T, DIR>::BYTES) != cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  return occ;
}

template <typename T>
cudaError_t allow_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_gfaces1<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Slab<T, 0>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gfaces1<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Slab<T, 1>::BYTES);
  return e;
}

}  // namespace

// Padded g layout: the row pitch leaves a whole 16-byte chunk (8 BF16 /
// 4 FP32 / 2 FP64 elements) past the last ghost column nx + 1 and is a
// multiple of 8 elements, so every chunk the face kernels copy is aligned
// and in bounds.
int gdev_pitch(int nx) { return ((nx + 10 + 7) / 8) * 8; }

// Shared-memory limits of the face kernels (the FP64 slabs exceed the
// default 48 KiB).
cudaError_t gdev_prepare(int store) {
  if (store != 0) return cudaErrorInvalidValue;
  return allow_smem<double>();
}

// Velocity chunks of the interior-face pass 1: the grid of (face columns x
// face rows x chunks) blocks is sized to fill whole waves of resident blocks
// (time ~ waves / chunks), with a small charge per chunk for the partial
// moments that pass 2 reads back.
int gdev_chunks(const DevParams& p, int dir, int sms, int store) {
  (void)store;
  const int occ = dir == 0 ? occupancy<double, 0>() : occupancy<double, 1>();
  const long slots = (long)occ * (sms > 0 ? sms : 1);
  const long base = (long)face_blocks_x(p, dir) * face_blocks_y(p, dir);
  const int maxc = p.nv < 64 ? p.nv : 64;
  int best = 1;
  double bestc = 1e300;
  for (int c = 1; c <= maxc; ++c) {
    const long waves = (base * c + slots - 1) / slots;
    const double cost = (double)waves / c + 0.002 * c;
    if (cost < bestc - 1e-12) {
      bestc = cost;
      best = c;
    }
  }
  return best;
}

cudaError_t launch_gdev_cell(const GDevStep& s, int stage, cudaStream_t st) {
  const void* src = stage == 1 ? s.fhat : s.ftp;
  const StageCoef& c = stage == 1 ? s.s1 : s.s2;
  if (s.store != 0) return cudaErrorInvalidValue;
  return cell_t<double>(s, src, c, st);
}

cudaError_t launch_gdev_faces(const GDevStep& s, int stage, int dir, cudaStream_t st) {
  if (s.store != 0) return cudaErrorInvalidValue;
  return dir == 0 ? faces_t<double, 0>(s, stage, st) : faces_t<double, 1>(s, stage, st);
}

cudaError_t launch_gdev_walls(const GDevStep& s, int stage, cudaStream_t st) {
  if (s.store != 0) return cudaErrorInvalidValue;
  return walls_t<double>(s, stage, st);
}

cudaError_t launch_gdev_update(const GDevStep& s, int stage, cudaStream_t st) {
  if (s.store != 0) return cudaErrorInvalidValue;
  return update_t<double>(s, stage, st);
}

}  // namespace dugks
