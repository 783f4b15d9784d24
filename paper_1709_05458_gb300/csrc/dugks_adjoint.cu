// Adjoint (reverse-mode derivative) kernels of the T3S3 step, FP64, any
// velocity set, periodic / bounce-back / diffuse walls.
//
// Forward step (Sec. 2.1.3; generic form of dugks_kernels.cu):
//   stage s in {1, 2}, input x (x = f^ for s = 1, x = f~' for s = 2):
//     rho = sum x, J = sum xi x, feq(rho, J), g = a x + b feq
//     face b: fbar = T(g) (upwind reconstruction of eq. flux_DS, walls), face
//             moments -> feq_b, f_b = alpha fbar + beta feq_b
//     L_k(cell) = -(xi_x (f_E - f_W)/dx + xi_y (f_N - f_S)/dy)
//   f~' = 5/4 g1 - 1/4 f^ + dt/3 L*,  X = 1/4 f^ + 3/4 g1 + 3dt/7 L*
//   f^^{n+1} = X + c (f~' - feq') + 4dt/7 L**,  c = -(3/4) 6dt/(6tau+dt)
// The adjoint applies the transpose of each map in reverse order.  For the
// equilibrium feq_k = W_k [rho + xi.J/RT + (xi.J)^2/(2 rho RT^2) - |J|^2/(2 rho RT)]
// the Jacobian is
//   d feq_k / d rho = W_k (1 - e_k^2/2 + uu/2),
//   d feq_k / d J   = W_k (xi_k (1 + e_k) - u) / RT,   e_k = xi_k.u/RT, uu = |u|^2/RT,
// so with mu_k the adjoint of feq_k:  rho_bar = sum mu_k W_k (1 - e^2/2 + uu/2),
// J_bar = sum mu_k W_k (xi_k (1 + e_k) - u)/RT, and x_bar_k += rho_bar + xi_k.J_bar.
// Interface reconstruction weights of cell offset (dx, dy) for the foot
// offset (a dx, b dy): centre 1 - 2a^2 - 2b^2, E/W a^2 +- a/2, N/S
// b^2 +- b/2, NE = SW = ab/2, NW = SE = -ab/2 (eq. flux_DS as printed, central
// differences); their transpose scatters with atomicAdd (stencil ghosts
// beyond walls scatter through the extrapolation 3, -3, 1).
// Parameter derivatives: tau enters a, b, alpha, beta and c; the wall
// velocity enters the bounce-back term and the diffuse-wall Maxwellian.
#include "dugks_internal.cuh"

namespace dugks {

namespace {

constexpr int kT = 128;

// Adds the block's sum of v[0..M) to dst[0..M): warp shuffles, then the
// warps' partials in shared memory, one atomic per non-zero value (the
// parameter gradients would otherwise see one same-address atomic per
// thread).  Every thread of the block must call it.
template <int M>
__device__ __forceinline__ void block_add(double (&v)[M], double* __restrict__ dst) {
  __shared__ double sm[kT / 32][M];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[m] += __shfl_xor_sync(0xffffffffu, v[m], o);
  if (lane == 0)
#pragma unroll
    for (int m = 0; m < M; ++m) sm[warp][m] = v[m];
  __syncthreads();
  if (threadIdx.x < M) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w][threadIdx.x];
    if (t != 0.0) atomicAdd(dst + threadIdx.x, t);
  }
}

__device__ __forceinline__ void eq_terms(double cx, double cy, double ux, double uy,
                                         const DevParams& p, double& P, double& e) {
  e = (cx * ux + cy * uy) * p.inv_RT;
  const double uu = (ux * ux + uy * uy) * p.inv_RT;
  P = 1.0 + e + 0.5 * e * e - 0.5 * uu;
}

// add v * weight to g_bar at cell (i, j) of one velocity, mapping ghosts
__device__ __forceinline__ void add_cell(double* __restrict__ gb, const DevParams& p, int i, int j, double v) {
  // resolve x
  int ix[3] = {0, 0, 0};
  double cx[3] = {0.0, 0.0, 0.0};
  int nxr;
  if (i >= 0 && i < p.nx) { ix[0] = i; cx[0] = 1.0; nxr = 1; }
  else if (p.px) { ix[0] = (i < 0) ? i + p.nx : i - p.nx; cx[0] = 1.0; nxr = 1; }
  else {
    const int b = (i < 0) ? 0 : p.nx - 1, s = (i < 0) ? 1 : -1;
    ix[0] = b; ix[1] = b + s; ix[2] = b + 2 * s; cx[0] = 3.0; cx[1] = -3.0; cx[2] = 1.0; nxr = 3;
  }
  int iy[3] = {0, 0, 0};
  double cy[3] = {0.0, 0.0, 0.0};
  int nyr;
  if (j >= 0 && j < p.ny) { iy[0] = j; cy[0] = 1.0; nyr = 1; }
  else if (p.py) { iy[0] = (j < 0) ? j + p.ny : j - p.ny; cy[0] = 1.0; nyr = 1; }
  else {
    const int b = (j < 0) ? 0 : p.ny - 1, s = (j < 0) ? 1 : -1;
    iy[0] = b; iy[1] = b + s; iy[2] = b + 2 * s; cy[0] = 3.0; cy[1] = -3.0; cy[2] = 1.0; nyr = 3;
  }
  // fixed trip counts keep the index arrays in registers
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      if (a < nyr && b < nxr) atomicAdd(gb + iy[a] * p.nx + ix[b], v * cy[a] * cx[b]);
}

// transpose of the Taylor expansion about cell (ci, cj) at offset (dX, dY)
__device__ __forceinline__ void scatter_taylor(double* __restrict__ gb, const DevParams& p, int ci, int cj,
                               double dX, double dY, double v) {
  double T[9];
  flux_ds_weights<double>(dX * p.inv_dx, dY * p.inv_dy, T);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) add_cell(gb, p, ci + q - 1, cj + r - 1, v * T[r * 3 + q]);
}

// g at any cell within one ghost layer (forward reconstruction, as in the
// forward generic kernels): a wall ghost along x is the extrapolation
// 3 g_0 - 3 g_1 + g_2 of the y-resolved values of its row's interior cells,
// along y the same of the interior cells of its column
__device__ __forceinline__ double g_col(const double* __restrict__ gk, const DevParams& p, int i,
                                        int j) {
  if (j < 0 || j >= p.ny) {
    if (p.py) j = (j < 0) ? j + p.ny : j - p.ny;
    else {
      const int b = (j < 0) ? 0 : p.ny - 1, s = (j < 0) ? 1 : -1;
      return 3.0 * gk[b * p.nx + i] - 3.0 * gk[(b + s) * p.nx + i] + gk[(b + 2 * s) * p.nx + i];
    }
  }
  return gk[j * p.nx + i];
}
__device__ __forceinline__ double g_at(const double* __restrict__ gk, const DevParams& p, int i,
                                       int j) {
  if (i < 0 || i >= p.nx) {
    if (p.px) i = (i < 0) ? i + p.nx : i - p.nx;
    else {
      const int b = (i < 0) ? 0 : p.nx - 1, s = (i < 0) ? 1 : -1;
      return 3.0 * g_col(gk, p, b, j) - 3.0 * g_col(gk, p, b + s, j) + g_col(gk, p, b + 2 * s, j);
    }
  }
  return g_col(gk, p, i, j);
}

__device__ __forceinline__ double taylor(const double* __restrict__ gk, const DevParams& p, int ci, int cj,
                         double dX, double dY) {
  const double C = g_at(gk, p, ci, cj);
  const double E = g_at(gk, p, ci + 1, cj), W = g_at(gk, p, ci - 1, cj);
  const double N = g_at(gk, p, ci, cj + 1), S = g_at(gk, p, ci, cj - 1);
  const double NE = g_at(gk, p, ci + 1, cj + 1), NW = g_at(gk, p, ci - 1, cj + 1);
  const double SE = g_at(gk, p, ci + 1, cj - 1), SW = g_at(gk, p, ci - 1, cj - 1);
  const double gx = (E - W) * (0.5 * p.inv_dx), gy = (N - S) * (0.5 * p.inv_dy);
  const double gxx = (E - 2.0 * C + W) * (p.inv_dx * p.inv_dx);
  const double gyy = (N - 2.0 * C + S) * (p.inv_dy * p.inv_dy);
  const double gxy = (NE - NW - SE + SW) * (0.25 * p.inv_dx * p.inv_dy);
  return C + dX * gx + dY * gy + (dX * dX * gxx + 2.0 * dX * dY * gxy + dY * dY * gyy);
}

struct FaceGeo {
  int li, lj, ui, uj, side;   // lower/upper cell, wall side or -1
  bool fluid_upper;
  double nsgn;                // xi.n = nsgn * xi_normal for the outward fluid normal
};

template <int DIR>
__device__ __forceinline__ FaceGeo face_geo(const DevParams& p, int face) {
  FaceGeo f{};
  f.side = -1;
  if (DIR == 0) {
    const int j = face / (p.nx + 1), fi = face - j * (p.nx + 1);
    f.li = fi - 1; f.ui = fi; f.lj = f.uj = j;
    if (p.px) { if (f.li < 0) f.li += p.nx; if (f.ui >= p.nx) f.ui -= p.nx; }
    else if (fi == 0) f.side = SIDE_W;
    else if (fi == p.nx) f.side = SIDE_E;
  } else {
    const int fj = face / p.nx, i = face - fj * p.nx;
    f.lj = fj - 1; f.uj = fj; f.li = f.ui = i;
    if (p.py) { if (f.lj < 0) f.lj += p.ny; if (f.uj >= p.ny) f.uj -= p.ny; }
    else if (fj == 0) f.side = SIDE_S;
    else if (fj == p.ny) f.side = SIDE_N;
  }
  f.fluid_upper = (f.side == SIDE_W || f.side == SIDE_S);
  f.nsgn = f.fluid_upper ? -1.0 : 1.0;
  return f;
}

// forward f-bar of velocity k at a face (the fluid side or upwind rule),
// without the outgoing wall rules
template <int DIR>
__device__ __forceinline__ double fbar_recon(const double* __restrict__ g, const DevParams& p, const FaceGeo& f,
                             int k, double h) {
  const double cx = __ldg(p.xi_x + k), cy = __ldg(p.xi_y + k);
  const double cn = DIR == 0 ? cx : cy;
  const double half = 0.5 * (DIR == 0 ? p.dx : p.dy);
  const double* gk = g + (size_t)k * p.N;
  const double lX = DIR == 0 ? half - cx * h : -cx * h, lY = DIR == 0 ? -cy * h : half - cy * h;
  const double uX = DIR == 0 ? -half - cx * h : -cx * h, uY = DIR == 0 ? -cy * h : -half - cy * h;
  if (f.side >= 0)
    return f.fluid_upper ? taylor(gk, p, f.ui, f.uj, uX, uY) : taylor(gk, p, f.li, f.lj, lX, lY);
  if (cn > 0.0) return taylor(gk, p, f.li, f.lj, lX, lY);
  if (cn < 0.0) return taylor(gk, p, f.ui, f.uj, uX, uY);
  return 0.5 * (taylor(gk, p, f.li, f.lj, lX, lY) + taylor(gk, p, f.ui, f.uj, uX, uY));
}

template <int DIR>
__device__ __forceinline__ void fbar_scatter(double* __restrict__ gbar, const DevParams& p, const FaceGeo& f,
                             int k, double h, double v) {
  const double cx = __ldg(p.xi_x + k), cy = __ldg(p.xi_y + k);
  const double cn = DIR == 0 ? cx : cy;
  const double half = 0.5 * (DIR == 0 ? p.dx : p.dy);
  double* gk = gbar + (size_t)k * p.N;
  const double lX = DIR == 0 ? half - cx * h : -cx * h, lY = DIR == 0 ? -cy * h : half - cy * h;
  const double uX = DIR == 0 ? -half - cx * h : -cx * h, uY = DIR == 0 ? -cy * h : -half - cy * h;
  if (f.side >= 0) {
    if (f.fluid_upper) scatter_taylor(gk, p, f.ui, f.uj, uX, uY, v);
    else scatter_taylor(gk, p, f.li, f.lj, lX, lY, v);
    return;
  }
  if (cn > 0.0) scatter_taylor(gk, p, f.li, f.lj, lX, lY, v);
  else if (cn < 0.0) scatter_taylor(gk, p, f.ui, f.uj, uX, uY, v);
  else {
    scatter_taylor(gk, p, f.li, f.lj, lX, lY, 0.5 * v);
    scatter_taylor(gk, p, f.ui, f.uj, uX, uY, 0.5 * v);
  }
}

// phi (adjoint of the stored face value f) from the adjoint of L.  Stored
// x-face fi is the west face of cell fi (if fi < nx) and the east face of
// cell fi-1 (if fi > 0) -- with periodic sides faces 0 and nx are stored
// separately and each belongs to one cell only -- so
//   phi(fi) = xi_x/dx * (Lbar(cell fi) [fi < nx] - Lbar(cell fi-1) [fi > 0]).
// Lbar = sa * A + sb * B (two cell arrays, either may be NULL).
template <int DIR>
__global__ void __launch_bounds__(kT)
k_flux_T(DevParams p, const double* __restrict__ A, double sa, const double* __restrict__ B,
         double sb, double* __restrict__ phi) {
  const int nf = DIR == 0 ? p.ny * (p.nx + 1) : (p.ny + 1) * p.nx;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.nv * nf) return;
  const int k = (int)(t / nf), face = (int)(t - (size_t)k * nf);
  auto lb = [&](int cell) {
    const size_t idx = (size_t)k * p.N + cell;
    double v = 0.0;
    if (A) v += sa * A[idx];
    if (B) v += sb * B[idx];
    return v;
  };
  double v = 0.0;
  if (DIR == 0) {
    const int j = face / (p.nx + 1), fi = face - j * (p.nx + 1);
    if (fi < p.nx) v += lb(j * p.nx + fi);
    if (fi > 0) v -= lb(j * p.nx + fi - 1);
    v *= __ldg(p.xi_x + k) * p.inv_dx;
  } else {
    const int fj = face / p.nx, i = face - fj * p.nx;
    if (fj < p.ny) v += lb(fj * p.nx + i);
    if (fj > 0) v -= lb((fj - 1) * p.nx + i);
    v *= __ldg(p.xi_y + k) * p.inv_dy;
  }
  phi[t] = v;
}

// Forward f-bar of every (face, velocity) of a stage, one thread each: the
// upwind reconstruction, or at a bounce-back wall the reflected value
// (eq. BB); the leaving velocities of a diffuse wall need the face's flux
// sum and are formed by k_face_T (0 here).  fbs[k][face].
template <int DIR>
__global__ void __launch_bounds__(kT)
k_fbar_T(const __grid_constant__ DevParams p, const double* __restrict__ g,
         const double* __restrict__ mom, double* __restrict__ fbs, double h) {
  const int nf = DIR == 0 ? p.ny * (p.nx + 1) : (p.ny + 1) * p.nx;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.nv * nf) return;
  const int k = (int)(t / nf), face = (int)(t - (size_t)k * nf);
  const FaceGeo f = face_geo<DIR>(p, face);
  const int kind = f.side >= 0 ? p.bc_kind[f.side] : -1;
  const double xn = f.nsgn * (DIR == 0 ? __ldg(p.xi_x + k) : __ldg(p.xi_y + k));
  double v = 0.0;
  if (kind < 0 || xn >= 0.0) {
    v = fbar_recon<DIR>(g, p, f, k, h);
  } else if (kind == BC_BOUNCEBACK) {
    const int wcell = f.fluid_upper ? f.uj * p.nx + f.ui : f.lj * p.nx + f.li;
    const int kk = __ldg(p.opp + k);
    v = fbar_recon<DIR>(g, p, f, kk, h) +
        2.0 * mom[wcell] * __ldg(p.w + k) *
            (__ldg(p.xi_x + k) * p.uw_x[f.side] + __ldg(p.xi_y + k) * p.uw_y[f.side]) * p.inv_RT;
  }
  fbs[t] = v;
}

// Face adjoint: phi (adjoint of f_b, overwritten with the adjoint of
// f-bar), rho_bar of wall-adjacent cells (bounce-back rho_w), and this
// face's contributions to d/d tau (gr[0]) and d/d u_w (gr[1 + 2 side],
// gr[2 + 2 side]).  One thread per face, looping over all velocities; the
// forward f-bar comes from k_fbar_T, the transposed reconstruction is
// k_scatter_T's.
template <int DIR>
__device__ __forceinline__ void face_T(const DevParams& p, int face, int nf,
                                       const double* __restrict__ fbs,
                                       const double* __restrict__ mom, double* __restrict__ phi,
                                       double* __restrict__ rhobar, double alpha, double beta,
                                       double dalpha, double (&gr)[9]) {
  const FaceGeo f = face_geo<DIR>(p, face);
  const int nv = p.nv;
  const int kind = f.side >= 0 ? p.bc_kind[f.side] : -1;
  const double uwx = f.side >= 0 ? p.uw_x[f.side] : 0.0, uwy = f.side >= 0 ? p.uw_y[f.side] : 0.0;
  const int wcell = f.side < 0 ? -1 : (f.fluid_upper ? f.uj * p.nx + f.ui : f.lj * p.nx + f.li);
  const double rho_w = wcell >= 0 ? mom[wcell] : 0.0;
  auto xn_of = [&](int k) {
    return f.nsgn * (DIR == 0 ? __ldg(p.xi_x + k) : __ldg(p.xi_y + k));
  };
  auto fbar = [&](int k, double rds) {   // forward f-bar of velocity k
    if (kind == BC_DIFFUSE && xn_of(k) < 0.0) return rds * p.feq_wall[f.side * nv + k];
    return fbs[(size_t)k * nf + face];
  };
  // diffuse rho_w
  double num = 0.0, rds = 0.0;
  if (kind == BC_DIFFUSE) {
    for (int k = 0; k < nv; ++k) {
      const double xn = xn_of(k);
      if (xn > 0.0) num += xn * fbs[(size_t)k * nf + face];
    }
    rds = num / p.ds_den[f.side];
  }
  // face moments
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int k = 0; k < nv; ++k) {
    const double v = fbar(k, rds);
    r += v;
    jx += __ldg(p.xi_x + k) * v;
    jy += __ldg(p.xi_y + k) * v;
  }
  const double ux = jx / r, uy = jy / r;
  const double uu = (ux * ux + uy * uy) * p.inv_RT;
  // adjoint of the face equilibrium and d/d tau
  double rb = 0.0, jbx = 0.0, jby = 0.0, tau_bar = 0.0;
  for (int k = 0; k < nv; ++k) {
    const double cx = __ldg(p.xi_x + k), cy = __ldg(p.xi_y + k), w = __ldg(p.w + k);
    double P, e;
    eq_terms(cx, cy, ux, uy, p, P, e);
    const double ph = phi[(size_t)k * nf + face];
    const double mu = beta * ph;
    rb += mu * w * (1.0 - 0.5 * e * e + 0.5 * uu);
    jbx += mu * w * (cx * (1.0 + e) - ux) * p.inv_RT;
    jby += mu * w * (cy * (1.0 + e) - uy) * p.inv_RT;
    // f_b = alpha fbar + (1 - alpha) feq_b (alpha + beta = 1)
    tau_bar += ph * dalpha * (fbar(k, rds) - w * r * P);
  }
  // psi = adjoint of fbar, stored into phi
  for (int k = 0; k < nv; ++k) {
    const size_t idx = (size_t)k * nf + face;
    phi[idx] = alpha * phi[idx] + rb + __ldg(p.xi_x + k) * jbx + __ldg(p.xi_y + k) * jby;
  }
  double uwb_x = 0.0, uwb_y = 0.0, rwb = 0.0;
  if (kind == BC_BOUNCEBACK) {
    for (int k = 0; k < nv; ++k) {
      if (xn_of(k) >= 0.0) continue;
      const size_t idx = (size_t)k * nf + face;
      const double ps = phi[idx];
      const int kk = __ldg(p.opp + k);
      phi[(size_t)kk * nf + face] += ps;
      const double cx = __ldg(p.xi_x + k), cy = __ldg(p.xi_y + k), w = __ldg(p.w + k);
      rwb += ps * 2.0 * w * (cx * uwx + cy * uwy) * p.inv_RT;
      uwb_x += ps * 2.0 * rho_w * w * cx * p.inv_RT;
      uwb_y += ps * 2.0 * rho_w * w * cy * p.inv_RT;
      phi[idx] = 0.0;
    }
    if (wcell >= 0) atomicAdd(rhobar + wcell, rwb);
  } else if (kind == BC_DIFFUSE) {
    // f-bar_out = rds * fw_k(u_w), rds = num / den(u_w), den = -sum_out xn fw
    double rds_bar = 0.0, dden_x = 0.0, dden_y = 0.0;
    for (int k = 0; k < nv; ++k) {
      const double xn = xn_of(k);
      if (xn >= 0.0) continue;
      const size_t idx = (size_t)k * nf + face;
      const double ps = phi[idx];
      const double cx = __ldg(p.xi_x + k), cy = __ldg(p.xi_y + k), w = __ldg(p.w + k);
      double P, e;
      eq_terms(cx, cy, uwx, uwy, p, P, e);
      const double dfx = w * (cx * (1.0 + e) - uwx) * p.inv_RT;   // d fw_k / d u_w
      const double dfy = w * (cy * (1.0 + e) - uwy) * p.inv_RT;
      rds_bar += ps * p.feq_wall[f.side * nv + k];
      uwb_x += ps * rds * dfx;
      uwb_y += ps * rds * dfy;
      dden_x -= xn * dfx;
      dden_y -= xn * dfy;
      phi[idx] = 0.0;
    }
    const double den = p.ds_den[f.side];
    const double num_bar = rds_bar / den;
    const double den_bar = -rds_bar * num / (den * den);
    uwb_x += den_bar * dden_x;
    uwb_y += den_bar * dden_y;
    for (int k = 0; k < nv; ++k) {
      const double xn = xn_of(k);
      if (xn > 0.0) phi[(size_t)k * nf + face] += num_bar * xn;
    }
  }
  if (f.side >= 0 && kind >= 0) {
#pragma unroll
    for (int sd = 0; sd < 4; ++sd) {             // constant indices keep gr in registers
      gr[1 + 2 * sd] += sd == f.side ? uwb_x : 0.0;
      gr[2 + 2 * sd] += sd == f.side ? uwb_y : 0.0;
    }
  }
  gr[0] += tau_bar;
}

// the parameter block stays in parameter space under the wall-side indexing
template <int DIR>
__global__ void __launch_bounds__(kT)
k_face_T(const __grid_constant__ DevParams p, const double* __restrict__ fbs,
         const double* __restrict__ mom, double* __restrict__ phi, double* __restrict__ rhobar,
         double* __restrict__ grads, double alpha, double beta, double dalpha) {
  const int nf = DIR == 0 ? p.ny * (p.nx + 1) : (p.ny + 1) * p.nx;
  const int face = blockIdx.x * blockDim.x + threadIdx.x;
  double gr[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (face < nf) face_T<DIR>(p, face, nf, fbs, mom, phi, rhobar, alpha, beta, dalpha, gr);
  block_add<9>(gr, grads);
}

// Transpose of the reconstruction: phi (the adjoint of f-bar) of every
// (face, velocity) scattered onto g_bar, one thread each.
template <int DIR>
__global__ void __launch_bounds__(kT)
k_scatter_T(const __grid_constant__ DevParams p, const double* __restrict__ phi,
            double* __restrict__ gbar, double h) {
  const int nf = DIR == 0 ? p.ny * (p.nx + 1) : (p.ny + 1) * p.nx;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.nv * nf) return;
  const double ps = phi[t];
  if (ps == 0.0) return;
  const int k = (int)(t / nf), face = (int)(t - (size_t)k * nf);
  fbar_scatter<DIR>(gbar, p, face_geo<DIR>(p, face), k, h, ps);
}

// Cell adjoint of g = a x + b feq(x) and of an extra equilibrium use
// c_extra * feq(x) weighted by `lam` (stage 2: f^^{n+1} contains c (f~' - feq')):
//   xbar_k += a gbar_k + (extra direct c_direct lam_k) + rho_bar + xi_k.J_bar
// with mu_k = b gbar_k - c_extra lam_k, rho_bar including wall uses.
// d/d tau += sum gbar (a' x + b' feq) + c' sum lam (x - feq).
__device__ __forceinline__ double cell_T(const DevParams& p, int cell, const double* __restrict__ x,
                                         const double* __restrict__ gbar,
                                         const double* __restrict__ lam,
                                         const double* __restrict__ rhobar_extra,
                                         double* __restrict__ xbar, double a, double b,
                                         double c_extra, double da, double dc) {
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int k = 0; k < p.nv; ++k) {
    const double v = x[(size_t)k * p.N + cell];
    r += v;
    jx += __ldg(p.xi_x + k) * v;
    jy += __ldg(p.xi_y + k) * v;
  }
  const double ux = jx / r, uy = jy / r;
  const double uu = (ux * ux + uy * uy) * p.inv_RT;
  double rb = rhobar_extra ? rhobar_extra[cell] : 0.0, jbx = 0.0, jby = 0.0, tb = 0.0;
  for (int k = 0; k < p.nv; ++k) {
    const size_t idx = (size_t)k * p.N + cell;
    const double cx = __ldg(p.xi_x + k), cy = __ldg(p.xi_y + k), w = __ldg(p.w + k);
    double P, e;
    eq_terms(cx, cy, ux, uy, p, P, e);
    const double feq = w * r * P;
    const double gb = gbar[idx];
    const double lm = lam ? lam[idx] : 0.0;
    const double mu = b * gb - c_extra * lm;
    rb += mu * w * (1.0 - 0.5 * e * e + 0.5 * uu);
    jbx += mu * w * (cx * (1.0 + e) - ux) * p.inv_RT;
    jby += mu * w * (cy * (1.0 + e) - uy) * p.inv_RT;
    tb += gb * da * (x[idx] - feq) + dc * lm * (x[idx] - feq);   // b' = -a'
  }
  for (int k = 0; k < p.nv; ++k) {
    const size_t idx = (size_t)k * p.N + cell;
    xbar[idx] += a * gbar[idx] + rb + __ldg(p.xi_x + k) * jbx + __ldg(p.xi_y + k) * jby;
  }
  return tb;
}

__global__ void __launch_bounds__(kT)
k_cell_T(DevParams p, const double* __restrict__ x, const double* __restrict__ gbar,
         const double* __restrict__ lam, const double* __restrict__ rhobar_extra,
         double* __restrict__ xbar, double a, double b, double c_extra, double da,
         double dc, double* __restrict__ grads) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (cell < p.N) v[0] = cell_T(p, cell, x, gbar, lam, rhobar_extra, xbar, a, b, c_extra, da, dc);
  block_add<1>(v, grads);
}

// out = sa * A + sb * B (elementwise over nv * N), either may be NULL
__global__ void __launch_bounds__(kT)
k_axpby(size_t n, const double* __restrict__ A, double sa, const double* __restrict__ B,
        double sb, double* __restrict__ out) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double v = 0.0;
  if (A) v += sa * A[t];
  if (B) v += sb * B[t];
  out[t] = v;
}

// adjoint of f^ = feq(rho, u) (equilibrium initialisation)
__global__ void __launch_bounds__(kT)
k_eq_T(DevParams p, const double* __restrict__ rho, const double* __restrict__ ux,
       const double* __restrict__ uy, const double* __restrict__ lam, double* __restrict__ drho,
       double* __restrict__ dux, double* __restrict__ duy) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.N) return;
  const double r = rho[cell], u = ux[cell], v = uy[cell];
  double sr = 0.0, su = 0.0, sv = 0.0;
  for (int k = 0; k < p.nv; ++k) {
    const double cx = __ldg(p.xi_x + k), cy = __ldg(p.xi_y + k), w = __ldg(p.w + k);
    double P, e;
    eq_terms(cx, cy, u, v, p, P, e);
    const double l = lam[(size_t)k * p.N + cell];
    sr += l * w * P;
    su += l * w * r * (cx * (1.0 + e) - u) * p.inv_RT;
    sv += l * w * r * (cy * (1.0 + e) - v) * p.inv_RT;
  }
  if (drho) drho[cell] = sr;
  if (dux) dux[cell] = su;
  if (duy) duy[cell] = sv;
}

unsigned nb(size_t n) { return (unsigned)((n + kT - 1) / kT); }

}  // namespace

cudaError_t launch_flux_T(const DevParams& p, int dir, const double* A, double sa,
                          const double* B, double sb, double* phi, cudaStream_t s) {
  const size_t nf = dir == 0 ? (size_t)p.ny * (p.nx + 1) : (size_t)(p.ny + 1) * p.nx;
  if (dir == 0) k_flux_T<0><<<nb(nf * p.nv), kT, 0, s>>>(p, A, sa, B, sb, phi);
  else k_flux_T<1><<<nb(nf * p.nv), kT, 0, s>>>(p, A, sa, B, sb, phi);
  return cudaGetLastError();
}

cudaError_t launch_face_T(const DevParams& p, int dir, const double* g, const double* mom,
                          double* phi, double* gbar, double* rhobar, double* grads,
                          const StageCoef& c, double dalpha, double* fbs, cudaStream_t s) {
  const size_t nf = dir == 0 ? (size_t)p.ny * (p.nx + 1) : (size_t)(p.ny + 1) * p.nx;
  const size_t nk = nf * p.nv;
  if (dir == 0) {
    k_fbar_T<0><<<nb(nk), kT, 0, s>>>(p, g, mom, fbs, c.h);
    k_face_T<0><<<nb(nf), kT, 0, s>>>(p, fbs, mom, phi, rhobar, grads, c.alpha, c.beta, dalpha);
    k_scatter_T<0><<<nb(nk), kT, 0, s>>>(p, phi, gbar, c.h);
  } else {
    k_fbar_T<1><<<nb(nk), kT, 0, s>>>(p, g, mom, fbs, c.h);
    k_face_T<1><<<nb(nf), kT, 0, s>>>(p, fbs, mom, phi, rhobar, grads, c.alpha, c.beta, dalpha);
    k_scatter_T<1><<<nb(nk), kT, 0, s>>>(p, phi, gbar, c.h);
  }
  return cudaGetLastError();
}

cudaError_t launch_cell_T(const DevParams& p, const double* x, const double* gbar,
                          const double* lam, const double* rhobar, double* xbar, double a,
                          double b, double c_extra, double da, double dc, double* grads,
                          cudaStream_t s) {
  k_cell_T<<<nb(p.N), kT, 0, s>>>(p, x, gbar, lam, rhobar, xbar, a, b, c_extra, da, dc, grads);
  return cudaGetLastError();
}

cudaError_t launch_axpby(size_t n, const double* A, double sa, const double* B, double sb,
                         double* out, cudaStream_t s) {
  k_axpby<<<nb(n), kT, 0, s>>>(n, A, sa, B, sb, out);
  return cudaGetLastError();
}

cudaError_t launch_eq_T(const DevParams& p, const double* rho, const double* ux,
                        const double* uy, const double* lam, double* drho, double* dux,
                        double* duy, cudaStream_t s) {
  k_eq_T<<<nb(p.N), kT, 0, s>>>(p, rho, ux, uy, lam, drho, dux, duy);
  return cudaGetLastError();
}

}  // namespace dugks
