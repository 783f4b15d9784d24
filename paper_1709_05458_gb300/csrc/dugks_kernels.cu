// Generic sm_103a kernels of the third-order DUGKS step (any velocity set,
// periodic / bounce-back / diffuse walls), FP64 throughout.
//
// One T3S3 step (arXiv:1709.05458, Sec. 2.1.3) is eight launches:
//   stage 1: cell(f^)   -> rho,u and g1 = f-bar^{+,dt/6}      (eq. f_bar_1_6)
//            face x, y  -> f(x_b, t*) via eqs. interfaceEvof, flux_DS,
//                          wall rules of Sec. 2.3, eq. recover2f
//            update1    -> L* (eq. microflux), f~(t') (eqs. f_tilde_1_3 and
//                          feqIntD2nd_Explicit with step dt/3) and
//                          acc = f^+ + 3dt/7 L* (eq. fhp)
//   stage 2: cell(f~')  -> rho',u' and g2 = f-bar^{+,5dt/12}(t')
//            face x, y  -> f(x_b, t**)
//            update2    -> f^^{n+1} = acc + 3/4 dt Omega' + 4dt/7 L**
//                          (eqs. collisionterm, feqIntD3rdHat2_DS)
//
// Layout: f[k][j][i] (x fastest); x-faces fbx[k][j][fi], fi = 0..nx (face fi
// between cells fi-1 and fi); y-faces fby[k][fj][i], fj = 0..ny.
// Velocity groups: a block is TX = 256/G cells (or faces) along x times G
// velocity groups; each thread loops over velocities k = ty, ty+G, ... and
// the per-cell (per-face) reductions over velocity combine the G partial
// sums in shared memory.
#include "dugks_internal.cuh"

namespace dugks {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double feq_poly(double cx, double cy, double ux, double uy,
                                           double inv_RT) {
  // 1 + xi.u/RT + (xi.u)^2/(2 RT^2) - |u|^2/(2 RT)   (Sec. 2.1.1)
  const double eu = (cx * ux + cy * uy) * inv_RT;
  const double uu = (ux * ux + uy * uy) * inv_RT;
  return 1.0 + eu + 0.5 * eu * eu - 0.5 * uu;
}

// g at cell (i, j) where i is inside [0, nx) and j may be one cell outside:
// periodic wrap or quadratic extrapolation along y (g_-1 = 3g_0 - 3g_1 + g_2).
__device__ __forceinline__ double g_col(const double* __restrict__ gk, const DevParams& p,
                                        int i, int j) {
  if (j < 0 || j >= p.ny) {
    if (p.py) {
      j = (j < 0) ? j + p.ny : j - p.ny;
    } else {
      const int j0 = (j < 0) ? 0 : p.ny - 1;
      const int s = (j < 0) ? 1 : -1;
      return 3.0 * gk[j0 * p.nx + i] - 3.0 * gk[(j0 + s) * p.nx + i] +
             gk[(j0 + 2 * s) * p.nx + i];
    }
  }
  return gk[j * p.nx + i];
}

// g at any cell within one ghost layer of the mesh.
__device__ __forceinline__ double g_at(const double* __restrict__ gk, const DevParams& p,
                                       int i, int j) {
  if (i < 0 || i >= p.nx) {
    if (p.px) {
      i = (i < 0) ? i + p.nx : i - p.nx;
    } else {
      const int i0 = (i < 0) ? 0 : p.nx - 1;
      const int s = (i < 0) ? 1 : -1;
      return 3.0 * g_col(gk, p, i0, j) - 3.0 * g_col(gk, p, i0 + s, j) +
             g_col(gk, p, i0 + 2 * s, j);
    }
  }
  return g_col(gk, p, i, j);
}

// eq. flux_DS as printed: the expansion of g about the centre of cell
// (ci, cj), evaluated at offset d = (dX, dY): value + d.grad + d^T H d (no
// factor 1/2 on the second-order term, reading Q2p), derivatives by central
// differences on the 3x3 neighbourhood.
__device__ __forceinline__ double taylor(const double* __restrict__ gk, const DevParams& p,
                                         int ci, int cj, double dX, double dY) {
  double C, E, W, N, S, NE, NW, SE, SW;
  if (ci >= 1 && ci < p.nx - 1 && cj >= 1 && cj < p.ny - 1) {
    const double* r0 = gk + (cj - 1) * p.nx + ci;
    const double* r1 = r0 + p.nx;
    const double* r2 = r1 + p.nx;
    SW = __ldg(r0 - 1); S = __ldg(r0); SE = __ldg(r0 + 1);
    W = __ldg(r1 - 1);  C = __ldg(r1); E = __ldg(r1 + 1);
    NW = __ldg(r2 - 1); N = __ldg(r2); NE = __ldg(r2 + 1);
  } else {
    C = g_at(gk, p, ci, cj);
    E = g_at(gk, p, ci + 1, cj);      W = g_at(gk, p, ci - 1, cj);
    N = g_at(gk, p, ci, cj + 1);      S = g_at(gk, p, ci, cj - 1);
    NE = g_at(gk, p, ci + 1, cj + 1); NW = g_at(gk, p, ci - 1, cj + 1);
    SE = g_at(gk, p, ci + 1, cj - 1); SW = g_at(gk, p, ci - 1, cj - 1);
  }
  const double gx = (E - W) * (0.5 * p.inv_dx);
  const double gy = (N - S) * (0.5 * p.inv_dy);
  const double gxx = (E - 2.0 * C + W) * (p.inv_dx * p.inv_dx);
  const double gyy = (N - 2.0 * C + S) * (p.inv_dy * p.inv_dy);
  const double gxy = (NE - NW - SE + SW) * (0.25 * p.inv_dx * p.inv_dy);
  return C + dX * gx + dY * gy + (dX * dX * gxx + 2.0 * dX * dY * gxy + dY * dY * gyy);
}

// The original DUGKS reconstruction (T2S2, p.recon = 1): f-bar^+(x_b - xi h)
// = f-bar^+(x_b) - xi h . grad f-bar^+(x_b), the face value and gradient by
// linear interpolation between the two cells of the face (lo = left / below,
// up = right / above; a cell beyond a wall is the ghost of g_at): value
// (g_lo + g_up)/2, normal derivative (g_up - g_lo)/d, tangential derivative
// the mean of the two cells' central differences.
template <int DIR>
__device__ __forceinline__ double central_face(const double* __restrict__ gk, const DevParams& p,
                                               int li, int lj, int ui, int uj, double cxh,
                                               double cyh) {
  const double lo = g_at(gk, p, li, lj), up = g_at(gk, p, ui, uj);
  double tn;
  if (DIR == 0) {
    tn = (g_at(gk, p, li, lj + 1) - g_at(gk, p, li, lj - 1) + g_at(gk, p, ui, uj + 1) -
          g_at(gk, p, ui, uj - 1)) * (0.25 * p.inv_dy);
    return 0.5 * (lo + up) - cxh * (up - lo) * p.inv_dx - cyh * tn;
  }
  tn = (g_at(gk, p, li + 1, lj) - g_at(gk, p, li - 1, lj) + g_at(gk, p, ui + 1, uj) -
        g_at(gk, p, ui - 1, uj)) * (0.25 * p.inv_dx);
  return 0.5 * (lo + up) - cyh * (up - lo) * p.inv_dy - cxh * tn;
}

// Combine M per-thread partial sums across the G velocity groups of a block;
// on return every thread holds the block-column totals.
template <int G, int TX, int M>
__device__ __forceinline__ void group_sum(double (&v)[M], double* red /* [M][G][TX] */) {
  if constexpr (G > 1) {
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int m = 0; m < M; ++m) red[(m * G + ty) * TX + tx] = v[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < M; ++m) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < G; ++q) s += red[(m * G + q) * TX + tx];
      v[m] = s;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- cell
// STAGE 0: moments only.  STAGE 1/2: moments, then g = a * src + b * feq.
template <int G, int STAGE>
__global__ void __launch_bounds__(kThreads)
k_cell(DevParams p, const double* __restrict__ src, double* __restrict__ g,
       double* __restrict__ mom, double a, double b) {
  constexpr int TX = kThreads / G;
  __shared__ double red[3 * G * TX];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int cell = blockIdx.x * TX + tx;
  const bool valid = cell < p.N;
  double v[3] = {0.0, 0.0, 0.0};
  if (valid) {
    for (int k = ty; k < p.nv; k += G) {
      const double f = src[(size_t)k * p.N + cell];
      v[0] += f;
      v[1] += __ldg(p.xi_x + k) * f;
      v[2] += __ldg(p.xi_y + k) * f;
    }
  }
  group_sum<G, TX, 3>(v, red);
  if (!valid) return;
  const double rho = v[0], ux = v[1] / rho, uy = v[2] / rho;
  if (ty == 0) {
    mom[cell] = rho;
    mom[p.N + cell] = ux;
    mom[2 * p.N + cell] = uy;
  }
  if constexpr (STAGE > 0) {
    // feq_k = W_k rho (base + e (1 + e/2)), e = xi_k.u/RT, base = 1 - |u|^2/(2RT)
    const double vx = ux * p.inv_RT, vy = uy * p.inv_RT;
    const double base = 1.0 - 0.5 * fma(ux, vx, uy * vy);
    const double br = b * rho;
    for (int k = ty; k < p.nv; k += G) {
      const size_t idx = (size_t)k * p.N + cell;
      const double e = fma(__ldg(p.xi_x + k), vx, __ldg(p.xi_y + k) * vy);
      const double P = fma(e, fma(0.5, e, 1.0), base);
      g[idx] = fma(br * __ldg(p.w + k), P, a * src[idx]);
    }
  }
}

// ---------------------------------------------------------------- faces
// DIR 0: x-faces, DIR 1: y-faces.  "lower" cell = the one with the smaller
// index along the face normal (left / below), "upper" = right / above.
// walls_only: the launch covers only the wall faces (2 per row or column),
// indexed compactly: DIR 0 id -> row id/2, face 0 or nx; DIR 1 likewise.
template <int G, int DIR>
__global__ void __launch_bounds__(kThreads)
k_face(DevParams p, const double* __restrict__ g, const double* __restrict__ mom,
       double* __restrict__ fb, StageCoef c, int walls_only) {
  constexpr int TX = kThreads / G;
  __shared__ double red[4 * G * TX];
  const int nx = p.nx, ny = p.ny, N = p.N;
  const int nf = (DIR == 0) ? ny * (nx + 1) : (ny + 1) * nx;
  const int tx = threadIdx.x, ty = threadIdx.y;
  int face = blockIdx.x * TX + tx;
  bool valid = face < nf;
  if (walls_only) {
    const int id = face;
    valid = id < 2 * (DIR == 0 ? ny : nx);
    face = (DIR == 0) ? (id >> 1) * (nx + 1) + ((id & 1) ? nx : 0)
                      : ((id & 1) ? ny : 0) * nx + (id >> 1);
  }

  int li = 0, lj = 0, ui = 0, uj = 0, side = -1;
  if (valid) {
    if (DIR == 0) {
      const int j = face / (nx + 1);
      const int fi = face - j * (nx + 1);
      li = fi - 1; ui = fi; lj = uj = j;
      if (p.px) {
        if (li < 0) li += nx;
        if (ui >= nx) ui -= nx;
      } else if (fi == 0) {
        side = SIDE_W;
      } else if (fi == nx) {
        side = SIDE_E;
      }
    } else {
      const int fj = face / nx;
      const int i = face - fj * nx;
      lj = fj - 1; uj = fj; li = ui = i;
      if (p.py) {
        if (lj < 0) lj += ny;
        if (uj >= ny) uj -= ny;
      } else if (fj == 0) {
        side = SIDE_S;
      } else if (fj == ny) {
        side = SIDE_N;
      }
    }
  }
  // At a wall the fluid cell is the upper one for W/S and the lower for E/N;
  // xi.n with n the outward normal of the fluid is -xi_n (W/S) or +xi_n (E/N).
  const bool wall = side >= 0;
  const bool fluid_upper = (side == SIDE_W || side == SIDE_S);
  const double nsgn = fluid_upper ? -1.0 : 1.0;
  const int kind = wall ? p.bc_kind[side] : -1;
  double rho_w = 0.0, uwx = 0.0, uwy = 0.0;
  if (wall) {
    rho_w = fluid_upper ? mom[uj * nx + ui] : mom[lj * nx + li];
    uwx = p.uw_x[side];
    uwy = p.uw_y[side];
  }
  const double half = 0.5 * ((DIR == 0) ? p.dx : p.dy);
  const double h = c.h;

  double v[4] = {0.0, 0.0, 0.0, 0.0};   // rho, jx, jy, diffuse-wall numerator
  if (valid) {
    for (int k = ty; k < p.nv; k += G) {
      const double cx = __ldg(p.xi_x + k), cy = __ldg(p.xi_y + k);
      const double cn = (DIR == 0) ? cx : cy;
      const double* gk = g + (size_t)k * N;
      // offsets of the foot x_b - xi h from the lower / upper cell centre
      const double lX = (DIR == 0) ? (half - cx * h) : (-cx * h);
      const double lY = (DIR == 0) ? (-cy * h) : (half - cy * h);
      const double uX = (DIR == 0) ? (-half - cx * h) : (-cx * h);
      const double uY = (DIR == 0) ? (-cy * h) : (-half - cy * h);
      double fbar;
      if (p.recon == 1) {                      // T2S2: both cells of the face
        const int kk = (wall && nsgn * cn < 0.0 && kind == BC_BOUNCEBACK) ? __ldg(p.opp + k) : k;
        const double* gq = g + (size_t)kk * N;
        const double qx = __ldg(p.xi_x + kk), qy = __ldg(p.xi_y + kk);
        const double cf = central_face<DIR>(gq, p, li, lj, ui, uj, qx * h, qy * h);
        if (!wall) {
          fbar = cf;
        } else {
          const double xn = nsgn * cn;
          if (xn >= 0.0) {
            fbar = cf;
            if (xn > 0.0) v[3] += xn * fbar;
          } else if (kind == BC_BOUNCEBACK) {
            fbar = cf + 2.0 * rho_w * __ldg(p.w + k) * (cx * uwx + cy * uwy) * p.inv_RT;
          } else {
            continue;                          // diffuse: after the reduction
          }
        }
      } else if (!wall) {
        if (cn > 0.0) {
          fbar = taylor(gk, p, li, lj, lX, lY);
        } else if (cn < 0.0) {
          fbar = taylor(gk, p, ui, uj, uX, uY);
        } else {
          fbar = 0.5 * (taylor(gk, p, li, lj, lX, lY) + taylor(gk, p, ui, uj, uX, uY));
        }
      } else {
        const double xn = nsgn * cn;
        if (xn >= 0.0) {                       // hits the wall or runs along it
          fbar = fluid_upper ? taylor(gk, p, ui, uj, uX, uY) : taylor(gk, p, li, lj, lX, lY);
          if (xn > 0.0) v[3] += xn * fbar;
        } else if (kind == BC_BOUNCEBACK) {    // eq. BB on f-bar
          const int kk = __ldg(p.opp + k);
          const double ox = __ldg(p.xi_x + kk), oy = __ldg(p.xi_y + kk);
          const double* gkk = g + (size_t)kk * N;
          const double fin = fluid_upper
              ? taylor(gkk, p, ui, uj, (DIR == 0) ? (-half - ox * h) : (-ox * h),
                       (DIR == 0) ? (-oy * h) : (-half - oy * h))
              : taylor(gkk, p, li, lj, (DIR == 0) ? (half - ox * h) : (-ox * h),
                       (DIR == 0) ? (-oy * h) : (half - oy * h));
          fbar = fin + 2.0 * rho_w * __ldg(p.w + k) * (cx * uwx + cy * uwy) * p.inv_RT;
        } else {
          continue;                            // diffuse: after the reduction
        }
      }
      fb[(size_t)k * nf + face] = fbar;
      v[0] += fbar;
      v[1] += cx * fbar;
      v[2] += cy * fbar;
    }
  }
  group_sum<G, TX, 4>(v, red);

  if (p.has_ds) {   // uniform over the launch
    double w2[3] = {0.0, 0.0, 0.0};
    if (valid && wall && kind == BC_DIFFUSE) {
      const double rho_ds = v[3] / p.ds_den[side];
      const double* fw = p.feq_wall + side * p.nv;
      for (int k = ty; k < p.nv; k += G) {
        const double cn = (DIR == 0) ? __ldg(p.xi_x + k) : __ldg(p.xi_y + k);
        if (nsgn * cn < 0.0) {
          const double fbar = rho_ds * __ldg(fw + k);
          fb[(size_t)k * nf + face] = fbar;
          w2[0] += fbar;
          w2[1] += __ldg(p.xi_x + k) * fbar;
          w2[2] += __ldg(p.xi_y + k) * fbar;
        }
      }
    }
    group_sum<G, TX, 3>(w2, red);
    v[0] += w2[0];
    v[1] += w2[1];
    v[2] += w2[2];
  }
  if (!valid) return;

  // face equilibrium from the moments of f-bar, then f = alpha f-bar + beta feq
  const double rho = v[0], ux = v[1] / rho, uy = v[2] / rho;
  for (int k = ty; k < p.nv; k += G) {
    const size_t idx = (size_t)k * nf + face;
    const double feq = __ldg(p.w + k) * rho *
                       feq_poly(__ldg(p.xi_x + k), __ldg(p.xi_y + k), ux, uy, p.inv_RT);
    fb[idx] = c.alpha * fb[idx] + c.beta * feq;
  }
}

// ---------------------------------------------------------------- updates
__device__ __forceinline__ double microflux(const DevParams& p, const double* __restrict__ fbx,
                                            const double* __restrict__ fby, int k, int i, int j) {
  const int nx = p.nx, ny = p.ny;
  const size_t bx = (size_t)k * ny * (nx + 1) + (size_t)j * (nx + 1) + i;
  const size_t by = (size_t)k * (ny + 1) * nx + (size_t)j * nx + i;
  const double fxw = fbx[bx], fxe = fbx[bx + 1];
  const double fys = fby[by], fyn = fby[by + nx];
  return -(__ldg(p.xi_x + k) * (fxe - fxw) * p.inv_dx + __ldg(p.xi_y + k) * (fyn - fys) * p.inv_dy);
}

__global__ void __launch_bounds__(kThreads)
k_update1(DevParams p, const double* __restrict__ fhat, const double* __restrict__ g1,
          const double* __restrict__ fbx, const double* __restrict__ fby,
          double* __restrict__ ftp, double* __restrict__ acc, double dt3, double dt37) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)p.nv * p.N;
  if (t >= total) return;
  const int k = (int)(t / p.N);
  const int cell = (int)(t - (size_t)k * p.N);
  const int j = cell / p.nx, i = cell - j * p.nx;
  const double L = microflux(p, fbx, fby, k, i, j);
  const double fh = fhat[t], g = g1[t];
  ftp[t] = 1.25 * g - 0.25 * fh + dt3 * L;        // f~+(t_n) + dt/3 L*
  acc[t] = 0.25 * fh + 0.75 * g + dt37 * L;       // f^+(t_n) + 3dt/7 L*
}

__global__ void __launch_bounds__(kThreads)
k_update2(DevParams p, const double* __restrict__ ftp, const double* __restrict__ acc,
          const double* __restrict__ mom, const double* __restrict__ fbx,
          const double* __restrict__ fby, double* __restrict__ fhat, double c_om34,
          double dt47) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)p.nv * p.N;
  if (t >= total) return;
  const int k = (int)(t / p.N);
  const int cell = (int)(t - (size_t)k * p.N);
  const int j = cell / p.nx, i = cell - j * p.nx;
  const double L = microflux(p, fbx, fby, k, i, j);
  const double rho = mom[cell], ux = mom[p.N + cell], uy = mom[2 * p.N + cell];
  const double vx = ux * p.inv_RT, vy = uy * p.inv_RT;
  const double e = fma(__ldg(p.xi_x + k), vx, __ldg(p.xi_y + k) * vy);
  const double P = fma(e, fma(0.5, e, 1.0), 1.0 - 0.5 * fma(ux, vx, uy * vy));
  const double feq = __ldg(p.w + k) * rho * P;
  fhat[t] = fma(dt47, L, fma(c_om34, ftp[t] - feq, acc[t]));
}

// T2 step (Remark I, eq. feqIntD2nd_Explicit):
// f~^{n+1} = ((2 tau - dt) f~ + 2 dt feq) / (2 tau + dt) + dt L(t_n + dt/2)
__global__ void __launch_bounds__(kThreads)
k_update_t2(DevParams p, const double* __restrict__ mom, const double* __restrict__ fbx,
            const double* __restrict__ fby, double* __restrict__ ft, double a, double b) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)p.nv * p.N;
  if (t >= total) return;
  const int k = (int)(t / p.N);
  const int cell = (int)(t - (size_t)k * p.N);
  const int j = cell / p.nx, i = cell - j * p.nx;
  const double L = microflux(p, fbx, fby, k, i, j);
  const double rho = mom[cell], ux = mom[p.N + cell], uy = mom[2 * p.N + cell];
  const double vx = ux * p.inv_RT, vy = uy * p.inv_RT;
  const double e = fma(__ldg(p.xi_x + k), vx, __ldg(p.xi_y + k) * vy);
  const double P = fma(e, fma(0.5, e, 1.0), 1.0 - 0.5 * fma(ux, vx, uy * vy));
  const double feq = __ldg(p.w + k) * rho * P;
  ft[t] = fma(p.dt, L, fma(a, ft[t], b * feq));
}

__global__ void __launch_bounds__(kThreads)
k_set_eq(DevParams p, const double* __restrict__ rho, const double* __restrict__ ux,
         const double* __restrict__ uy, double* __restrict__ fhat) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)p.nv * p.N;
  if (t >= total) return;
  const int k = (int)(t / p.N);
  const int cell = (int)(t - (size_t)k * p.N);
  fhat[t] = __ldg(p.w + k) * rho[cell] *
            feq_poly(__ldg(p.xi_x + k), __ldg(p.xi_y + k), ux[cell], uy[cell], p.inv_RT);
}

__global__ void __launch_bounds__(kThreads)
k_check(DevParams p, const double* __restrict__ mom, int* __restrict__ flag) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.N) return;
  const double r = mom[cell], u = mom[p.N + cell], v = mom[2 * p.N + cell];
  if (!(r > 0.0) || !isfinite(r) || !isfinite(u) || !isfinite(v)) atomicOr(flag, 1);
}

template <int G>
cudaError_t cell_launch_g(const DevParams& p, int stage, const double* src, double* g,
                          double* mom, double a, double b, cudaStream_t s) {
  constexpr int TX = kThreads / G;
  dim3 block(TX, G), grid((p.N + TX - 1) / TX);
  if (stage == 0) k_cell<G, 0><<<grid, block, 0, s>>>(p, src, g, mom, a, b);
  else if (stage == 1) k_cell<G, 1><<<grid, block, 0, s>>>(p, src, g, mom, a, b);
  else k_cell<G, 2><<<grid, block, 0, s>>>(p, src, g, mom, a, b);
  return cudaGetLastError();
}

template <int G>
cudaError_t face_launch_g(const DevParams& p, int dir, const double* g, const double* mom,
                          double* fb, const StageCoef& c, int walls_only, cudaStream_t s) {
  constexpr int TX = kThreads / G;
  const int nf = walls_only ? 2 * (dir == 0 ? p.ny : p.nx)
                            : (dir == 0 ? p.ny * (p.nx + 1) : (p.ny + 1) * p.nx);
  dim3 block(TX, G), grid((nf + TX - 1) / TX);
  if (dir == 0) k_face<G, 0><<<grid, block, 0, s>>>(p, g, mom, fb, c, walls_only);
  else k_face<G, 1><<<grid, block, 0, s>>>(p, g, mom, fb, c, walls_only);
  return cudaGetLastError();
}

unsigned blocks_for(size_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_cell(const DevParams& p, int groups, int stage, const double* src,
                        double* g, double* mom, double a, double b, cudaStream_t s) {
  return groups == 1 ? cell_launch_g<1>(p, stage, src, g, mom, a, b, s)
                     : cell_launch_g<8>(p, stage, src, g, mom, a, b, s);
}

cudaError_t launch_face(const DevParams& p, int groups, int dir, const double* g,
                        const double* mom, double* fb, const StageCoef& c, cudaStream_t s,
                        int walls_only) {
  if (groups == 1) return face_launch_g<1>(p, dir, g, mom, fb, c, walls_only, s);
  // the few wall faces of a large velocity set: 32 velocity groups per face
  if (walls_only && p.nv > 256) return face_launch_g<32>(p, dir, g, mom, fb, c, walls_only, s);
  return face_launch_g<8>(p, dir, g, mom, fb, c, walls_only, s);
}

cudaError_t launch_update1(const DevParams& p, const double* fhat, const double* g1,
                           const double* fbx, const double* fby, double* ftp, double* acc,
                           cudaStream_t s) {
  const size_t n = (size_t)p.nv * p.N;
  k_update1<<<blocks_for(n), kThreads, 0, s>>>(p, fhat, g1, fbx, fby, ftp, acc, p.dt / 3.0,
                                               3.0 * p.dt / 7.0);
  return cudaGetLastError();
}

cudaError_t launch_update_t2(const DevParams& p, const double* mom, const double* fbx,
                            const double* fby, double* ft, double a, double b, cudaStream_t s) {
  const size_t n = (size_t)p.nv * p.N;
  k_update_t2<<<blocks_for(n), kThreads, 0, s>>>(p, mom, fbx, fby, ft, a, b);
  return cudaGetLastError();
}

cudaError_t launch_update2(const DevParams& p, const double* ftp, const double* acc,
                           const double* mom, const double* fbx, const double* fby,
                           double* fhat, double c_om, cudaStream_t s) {
  const size_t n = (size_t)p.nv * p.N;
  k_update2<<<blocks_for(n), kThreads, 0, s>>>(p, ftp, acc, mom, fbx, fby, fhat, 0.75 * c_om,
                                               4.0 * p.dt / 7.0);
  return cudaGetLastError();
}

cudaError_t launch_set_eq(const DevParams& p, const double* rho, const double* ux,
                          const double* uy, double* fhat, cudaStream_t s) {
  const size_t n = (size_t)p.nv * p.N;
  k_set_eq<<<blocks_for(n), kThreads, 0, s>>>(p, rho, ux, uy, fhat);
  return cudaGetLastError();
}

cudaError_t launch_check(const DevParams& p, const double* mom, int* flag, cudaStream_t s) {
  k_check<<<blocks_for(p.N), kThreads, 0, s>>>(p, mom, flag);
  return cudaGetLastError();
}

}  // namespace dugks
