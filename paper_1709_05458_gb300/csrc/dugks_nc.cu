// Interior-face kernels of the generic (any velocity set) path for large
// velocity sets such as Newton-Cotes grids, FP64.
//
// The interface value of velocity k at face b is the quadratic Taylor
// expansion of g about the upwind cell at the characteristic foot (eqs.
// interfaceEvof, flux_DS, central differences): a 3x3 (ties xi.n = 0: 3x4)
// stencil dot product whose weights depend only on (xi_k, h, dx, dy).  Here
// lanes run over 32 consecutive faces, warps over velocities: a warp computes
// the weights of its velocity once in registers and stages a slab of g
// (rows x 36 columns) in shared memory that serves R face rows, so a face
// value costs 9 (12) FMAs and ~1.5 loads.  Face moments are accumulated per
// thread, reduced across the warps of the block and written per velocity
// chunk; the second pass sums the chunks in a fixed order (deterministic),
// forms the face equilibrium (eq. recover2f) and turns f-bar into f.  Wall
// faces are left to the generic kernel (they need the whole velocity set at
// once for bounce-back partners and the diffuse-wall density).
#include "dugks_internal.cuh"

namespace dugks {

namespace {

constexpr int NW = 8;          // warps (velocity groups) per block
constexpr int R = 8;           // face rows per block
constexpr int LANES = 32;

// g at (gx, gy) for slab staging: interior, periodic wrap, one ghost layer
// of quadratic extrapolation (g_-1 = 3 g_0 - 3 g_1 + g_2); positions further
// out are clamped (their values feed no interior face).
__device__ __forceinline__ double slab_fetch(const double* __restrict__ gk, const DevParams& p,
                                             int gx, int gy) {
  if (gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny) return __ldg(gk + gy * p.nx + gx);
  if (p.px) gx = ((gx % p.nx) + p.nx) % p.nx;
  else gx = gx < -1 ? -1 : (gx > p.nx ? p.nx : gx);
  if (p.py) gy = ((gy % p.ny) + p.ny) % p.ny;
  else gy = gy < -1 ? -1 : (gy > p.ny ? p.ny : gy);
  auto col = [&](int x, int y) {            // x in range, y may be a ghost
    if (y < 0 || y >= p.ny) {
      const int b = y < 0 ? 0 : p.ny - 1, s = y < 0 ? 1 : -1;
      return 3.0 * __ldg(gk + b * p.nx + x) - 3.0 * __ldg(gk + (b + s) * p.nx + x) +
             __ldg(gk + (b + 2 * s) * p.nx + x);
    }
    return __ldg(gk + y * p.nx + x);
  };
  if (gx < 0 || gx >= p.nx) {
    const int b = gx < 0 ? 0 : p.nx - 1, s = gx < 0 ? 1 : -1;
    return 3.0 * col(b, gy) - 3.0 * col(b + s, gy) + col(b + 2 * s, gy);
  }
  return col(gx, gy);
}

// Taylor weights about one cell for the foot offset (a dx, b dy):
// T[(dy+1)*3 + dx+1]
__device__ __forceinline__ void taylor9(double a, double b, double (&T)[9]) {
  flux_ds_weights<double>(a, b, T);
}

// the face-value weights about the lower (left / below) or upper cell of
// the face, foot offset (a dx, b dy): eq. flux_DS as printed (p.recon = 0);
// p.recon = 1, the original DUGKS reconstruction (T2S2): face value and
// gradient interpolated linearly between the two cells of the face, written
// on the 3x3 neighbourhood of either of them (the same value from both)
__device__ __forceinline__ void weights9(const DevParams& p, int dir, bool upper, double a,
                                         double b, double (&T)[9]) {
  if (p.recon == 1) {
#pragma unroll
    for (int i = 0; i < 9; ++i) T[i] = 0.0;
    if (dir == 0) {        // normal x: a = +-1/2 - xi_x h/dx, tangential b = -xi_y h/dy
      const double q = 0.25 * b;
      if (!upper) {        // cells C (lower) and E (upper)
        T[4] = 1.0 - a; T[5] = a;
        T[7] = q; T[1] = -q; T[8] = q; T[2] = -q;
      } else {             // cells W (lower) and C (upper)
        T[3] = -a; T[4] = 1.0 + a;
        T[7] = q; T[1] = -q; T[6] = q; T[0] = -q;
      }
    } else {               // normal y: b = +-1/2 - xi_y h/dy, tangential a = -xi_x h/dx
      const double q = 0.25 * a;
      if (!upper) {        // cells C (lower) and N (upper)
        T[4] = 1.0 - b; T[7] = b;
        T[5] = q; T[3] = -q; T[8] = q; T[6] = -q;
      } else {             // cells S (lower) and C (upper)
        T[1] = -b; T[4] = 1.0 + b;
        T[5] = q; T[3] = -q; T[2] = q; T[0] = -q;
      }
    }
  } else {
    taylor9(a, b, T);
  }
}

// Pass 1.  DIR 0: x-faces (lanes over fi, rows j); DIR 1: y-faces (lanes
// over i, rows fj).  part[chunk][3][nf]: partial face moments of the chunk.
template <int DIR>
__global__ void __launch_bounds__(LANES * NW)
k_nc_faces1(DevParams p, const double* __restrict__ g, double* __restrict__ fb,
            double* __restrict__ part, double h, int kchunk) {
  constexpr int SR = DIR == 0 ? R + 2 : R + 3;      // slab rows
  constexpr int SC = DIR == 0 ? 36 : 34;            // slab columns
  // dynamic shared memory: the warps' slabs, later reused for the reduction
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto red = [&](int w, int r, int l, int m) -> double& {
    return smem[((w * R + r) * LANES + l) * 3 + m];
  };
  const int nx = p.nx, ny = p.ny;
  const int nf = DIR == 0 ? ny * (nx + 1) : (ny + 1) * nx;
  const int c0 = blockIdx.x * LANES;                // first face column (x) / cell column (y)
  const int r0 = blockIdx.y * R;                    // first face row (x: cell row j; y: face row fj)
  const int k0 = blockIdx.z * kchunk, k1 = min(p.nv, k0 + kchunk);
  // origin of the slab in cell coordinates
  const int ox = DIR == 0 ? c0 - 2 : c0 - 1;
  const int oy = DIR == 0 ? r0 - 1 : r0 - 2;
  double acc[R][3];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r][0] = acc[r][1] = acc[r][2] = 0.0;
  // which faces of this thread are interior and exist
  bool ok[R];
  const int col = c0 + lane;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (DIR == 0) {
      const int j = r0 + r, fi = col;
      ok[r] = j < ny && fi <= nx && (p.px || (fi >= 1 && fi <= nx - 1));
    } else {
      const int fj = r0 + r, i = col;
      ok[r] = i < nx && fj <= ny && (p.py || (fj >= 1 && fj <= ny - 1));
    }
  }
  double* sl = smem + warp * SR * SC;
  for (int k = k0 + warp; k < k1; k += NW) {
    const double cx = __ldg(p.xi_x + k), cy = __ldg(p.xi_y + k);
    const double cn = DIR == 0 ? cx : cy;
    // weights of the upwind expansion only (both for xi.n = 0)
    double TL[9], TU[9];
    const bool lo = cn >= 0.0, hi = cn <= 0.0;     // uniform across the warp
    if (DIR == 0) {
      const double b = -cy * h * p.inv_dy;
      if (lo) weights9(p, 0, false, (0.5 * p.dx - cx * h) * p.inv_dx, b, TL);
      if (hi) weights9(p, 0, true, (-0.5 * p.dx - cx * h) * p.inv_dx, b, TU);
    } else {
      const double a = -cx * h * p.inv_dx;
      if (lo) weights9(p, 1, false, a, (0.5 * p.dy - cy * h) * p.inv_dy, TL);
      if (hi) weights9(p, 1, true, a, (-0.5 * p.dy - cy * h) * p.inv_dy, TU);
    }
    const double* gk = g + (size_t)k * p.N;
    __syncwarp();
    for (int e = lane; e < SR * SC; e += LANES) {
      const int rr = e / SC, cc = e - rr * SC;
      sl[e] = slab_fetch(gk, p, ox + cc, oy + rr);
    }
    __syncwarp();
    double* fbk = fb + (size_t)k * nf;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!ok[r]) continue;
      double v;
      if (DIR == 0) {
        // rows r..r+2 (cells j-1..j+1), columns lane+q (cells fi-2+q)
        const double* s0 = sl + r * SC + lane;
        if (cn > 0.0) {
          v = 0.0;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int q = 0; q < 3; ++q) v = fma(TL[a * 3 + q], s0[a * SC + q], v);
        } else if (cn < 0.0) {
          v = 0.0;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int q = 0; q < 3; ++q) v = fma(TU[a * 3 + q], s0[a * SC + q + 1], v);
        } else {
          double vl = 0.0, vu = 0.0;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              vl = fma(TL[a * 3 + q], s0[a * SC + q], vl);
              vu = fma(TU[a * 3 + q], s0[a * SC + q + 1], vu);
            }
          v = 0.5 * (vl + vu);
        }
      } else {
        // rows r+q (cells fj-2+q), columns lane..lane+2 (cells i-1..i+1)
        const double* s0 = sl + r * SC + lane;
        if (cn > 0.0) {
          v = 0.0;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int q = 0; q < 3; ++q) v = fma(TL[a * 3 + q], s0[a * SC + q], v);
        } else if (cn < 0.0) {
          v = 0.0;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int q = 0; q < 3; ++q) v = fma(TU[a * 3 + q], s0[(a + 1) * SC + q], v);
        } else {
          double vl = 0.0, vu = 0.0;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              vl = fma(TL[a * 3 + q], s0[a * SC + q], vl);
              vu = fma(TU[a * 3 + q], s0[(a + 1) * SC + q], vu);
            }
          v = 0.5 * (vl + vu);
        }
      }
      const int face = DIR == 0 ? (r0 + r) * (nx + 1) + col : (r0 + r) * nx + col;
      fbk[face] = v;
      acc[r][0] += v;
      acc[r][1] = fma(cx, v, acc[r][1]);
      acc[r][2] = fma(cy, v, acc[r][2]);
    }
  }
  // reduce the warps' partial moments in a fixed order and store the chunk's part
  __syncthreads();                                  // all slabs done: reuse the memory
#pragma unroll
  for (int r = 0; r < R; ++r) {
    red(warp, r, lane, 0) = acc[r][0];
    red(warp, r, lane, 1) = acc[r][1];
    red(warp, r, lane, 2) = acc[r][2];
  }
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
    double* pc = part + (size_t)blockIdx.z * 3 * nf;
    pc[face] = s0;
    pc[nf + face] = s1;
    pc[2 * nf + face] = s2;
  }
}

// Pass 2: per (face, velocity) of the interior faces: moments summed over the
// chunks in order, f = alpha f-bar + beta feq_b.
template <int DIR>
__global__ void __launch_bounds__(256)
k_nc_faces2(DevParams p, double* __restrict__ fb, const double* __restrict__ part, int nchunk,
            double alpha, double beta) {
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
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    const double* pc = part + (size_t)c * 3 * nf;
    r += pc[face];
    jx += pc[nf + face];
    jy += pc[2 * nf + face];
  }
  const double ux = jx / r * p.inv_RT, uy = jy / r * p.inv_RT;   // u / RT
  const double base = 1.0 - 0.5 * (jx * ux + jy * uy) / r;       // 1 - |u|^2/(2RT)
  const double br = beta * r;
  for (int k = blockIdx.y; k < p.nv; k += gridDim.y) {
    const size_t idx = (size_t)k * nf + face;
    const double e = fma(__ldg(p.xi_x + k), ux, __ldg(p.xi_y + k) * uy);
    const double P = fma(e, fma(0.5, e, 1.0), base);
    fb[idx] = fma(alpha, fb[idx], br * __ldg(p.w + k) * P);
  }
}

}  // namespace

// dynamic shared memory of pass 1: max(slabs, reduction) = 48 KiB
constexpr size_t kNcSmem = sizeof(double) * NW * R * LANES * 3;
static_assert(kNcSmem >= sizeof(double) * NW * (R + 3) * 36, "slab larger than reduction");
static_assert(kNcSmem <= 48 * 1024, "within the default dynamic shared memory limit");

int nc_chunks(const DevParams& p, int dir, int sms) {
  const int tiles = (dir == 0 ? (p.nx + 1 + LANES - 1) / LANES : (p.nx + LANES - 1) / LANES) *
                    (dir == 0 ? (p.ny + R - 1) / R : (p.ny + 1 + R - 1) / R);
  int ch = (3 * sms + tiles - 1) / tiles;           // about three blocks per SM
  const int maxch = (p.nv + NW - 1) / NW;
  if (ch > maxch) ch = maxch;
  if (ch > 64) ch = 64;
  return ch < 1 ? 1 : ch;
}

cudaError_t launch_nc_faces(const DevParams& p, int dir, const double* g, double* fb,
                            double* part, int nchunk, const StageCoef& c, cudaStream_t s) {
  const int kchunk = (p.nv + nchunk - 1) / nchunk;
  const int nf = dir == 0 ? p.ny * (p.nx + 1) : (p.ny + 1) * p.nx;
  if (dir == 0) {
    dim3 grid((p.nx + 1 + LANES - 1) / LANES, (p.ny + R - 1) / R, nchunk);
    k_nc_faces1<0><<<grid, LANES * NW, kNcSmem, s>>>(p, g, fb, part, c.h, kchunk);
  } else {
    dim3 grid((p.nx + LANES - 1) / LANES, (p.ny + 1 + R - 1) / R, nchunk);
    k_nc_faces1<1><<<grid, LANES * NW, kNcSmem, s>>>(p, g, fb, part, c.h, kchunk);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 g2((nf + 255) / 256, p.nv < 64 ? p.nv : 64);
  if (dir == 0) k_nc_faces2<0><<<g2, 256, 0, s>>>(p, fb, part, nchunk, c.alpha, c.beta);
  else k_nc_faces2<1><<<g2, 256, 0, s>>>(p, fb, part, nchunk, c.alpha, c.beta);
  return cudaGetLastError();
}

}  // namespace dugks
