// Class-moment kernels of the T3S3 step for any velocity set (Newton-Cotes
// grids in particular), periodic / bounce-back / diffuse walls, for the
// deviation storage forms of the generic path (FP32 / BF16 deviations
// d = f - W_k rho0, FP32 arithmetic; helpers in dugks_gcommon.cuh).  FP64
// storage keeps the kernels of dugks_generic_mixed.cu, which are bound by the
// FP64 pipe rather than by bytes.
//
// The face equilibria of a stage (eqs. recover2f, feqIntD3rdHat2_DS) need
// only the moments (1, xi_x, xi_y) of the interface values f-bar over the
// velocities.  An interface value is a 3 x 3 stencil of the stage field
// g = a src + b feq around the upwind cell with weights T(a, b) (eq. flux_DS
// as printed) that are quadratic in the foot offset (a, b) = (a0, b0) -
// (xi_x h/dx, xi_y h/dy); so xi^m T(a, b) is a cubic polynomial in xi and
// every face moment is a fixed combination, over the stencil's nine cells,
// of the cell moments of g up to third degree taken over the velocities with
// one sign of xi_x (x-faces) or xi_y (y-faces).  A stage is then
//
//   sums    a streaming pass over the stage's source array: per cell and
//           sign class (sign xi_x, sign xi_y) the ten moments of degree <= 3
//           (the cell's rho and j among them) -- one read of the state;
//   cellfin per cell: rho, u and the equilibrium's parameters; the class
//           moments of g (the equilibrium's part by exact quadrature); the
//           18 stencil moments nu_{m,u} = sum xi^m u(a, b) g of every
//           class combination the faces use (u = 1, a, b, a^2, ab, b^2);
//   facefin per face: M_m = sum over the stencil cells and u of t_u(s)
//           nu_{m,u}, T = sum_u t_u u(a, b), wall ghosts by the quadratic
//           extrapolation of Q16 (linear, so it applies to nu), and at a wall
//           the leaving velocities by the wall rule: bounce-back mirrors the
//           incoming moments (eq. BB), diffuse scattering adds rho_w times
//           the wall equilibrium's moments with rho_w from the incoming
//           flux (Sec. 2.3, Q13-Q15);
//   walls   per wall face and velocity: f-bar (fluid side, or the wall rule);
//   update  per (32 x 16 cell tile, velocity chunk): each velocity plane of
//           the tile plus a two-cell halo is staged in shared memory as g
//           (wall ghosts extrapolated there), the x- and y-face values of
//           the tile follow from the upwind stencils (wall faces from the
//           walls pass), and f = alpha f-bar + beta feq (eq. recover2f)
//           enters
//             stage 1: f~(t') = 5/4 g1 - 1/4 f^ + dt/3 L*
//             stage 2: f^^{n+1} = X + 3/4 dt Omega' + 4dt/7 L**,
//                      X = f^+ + 3dt/7 L* = 4/7 f^ - 6/7 g1 + 9/7 f~(t')
//           (eqs. f_tilde_1_3, fhp, collisionterm, feqIntD3rdHat2_DS; X is
//           recovered from f^ and f~(t') instead of being stored).
//
// Per (cell, velocity) and step the path reads the stored type four times
// (sums and update of each stage, stage 2 also f^) and writes it twice: 24
// bytes in FP32, 12 in BF16, plus the halo re-reads of the updates, which
// the L2 serves.  The finalisers touch O(cells) data.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dugks_gcommon.cuh"

namespace dugks {

namespace {

constexpr int TXT = 32;                 // tile columns (one lane each)
constexpr int TYT = 16;                 // tile rows
constexpr int UNW = 4;                  // warps per update block
constexpr int RPW = TYT / UNW;          // rows per warp: warp w takes rows 4w .. 4w + 3
constexpr int UNT = 32 * UNW;           // 128 threads
constexpr int HXT = TXT + 4;            // staged columns i0 - 2 .. i0 + 33
constexpr int HYT = TYT + 4;            // staged rows    j0 - 2 .. j0 + 17
constexpr int NST = HXT * HYT;          // 720 staged cells
constexpr int NHALO = NST - TXT * TYT;  // 208 of them outside the tile
constexpr int HPT = (NHALO + UNT - 1) / UNT;   // halo cells per thread (2)
constexpr int EPT = RPW + HPT;          // staged cells per thread: 4 own + 2 halo
constexpr int WPV = 72;                 // face weights per velocity in the table
constexpr int NMONO = 10;               // monomials of degree <= 3
constexpr int NNU = 18;                 // stencil moments nu_{m,u}: 3 m x 6 u

// index of the monomial x^i y^j among 1, x, y, xx, xy, yy, xxx, xxy, xyy, yyy
__host__ __device__ constexpr int mono_ix(int i, int j) { return (i + j) * (i + j + 1) / 2 + j; }

// packed FP32 pairs (lo, hi) in one 64-bit register, for fma.rn.f32x2
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// the Kahan-compensated sums of two accumulators at once (kah_add lane by
// lane: each operation rounded to nearest in FP32); s and c packed as pairs
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
struct Kah2 {
  unsigned long long s, c;
};
__device__ __forceinline__ void kah_add2(Kah2& a, unsigned long long x) {
  const unsigned long long y = sub2(x, a.c);
  const unsigned long long t = add2(a.s, y);
  a.c = sub2(sub2(t, a.s), y);
  a.s = t;
}

// ------------------------------------------------------------------ sums
// Per cell and sign class: the moments sum_k pi_p(xi_k) src_k of the
// class's velocities for the ten monomials pi_p (pi_0 .. pi_9 in the table
// row of a velocity).  A block takes SCB consecutive cells (one per thread)
// and one split of one class's velocities, whose indices and monomials it
// first copies to shared memory; each thread then reads its cell's values
// SBLK velocities at a time (the next block's loads issued before the
// current block is summed), adds each block in plain FP32 and folds it into
// a Kahan-compensated sum (the cell's rho and j among them, which the
// collision must conserve: the blocked sum keeps their error at the level
// of the FP32 storage itself).
constexpr int SCB = 256;                 // cells per block
constexpr int SBLK = 16;                 // velocities per plain FP32 block
constexpr int SMAXE = 512;               // velocities per split at most
constexpr int SRING = 3;                 // streamed form: blocks of SBLK planes in the ring
// streamed form (BF16): dynamic shared memory holding the split's
// monomials and velocity indices, then the ring of its planes' values
constexpr size_t SUMS_TAB = (size_t)SMAXE * 3 * sizeof(float4) + SMAXE * sizeof(int);
template <typename T> constexpr bool sums_streamed() { return sizeof(T) == 2; }
template <typename T> constexpr size_t sums_smem() {
  return sums_streamed<T>() ? SUMS_TAB + (size_t)SRING * SBLK * SCB * sizeof(T) : 0;
}
static_assert(SUMS_TAB % 16 == 0, "the ring must start 16-byte aligned");

// velocity split z of class cls: table entries [ea, eb)
__device__ __forceinline__ void split_range(const GncStep& s, int cls, int z, int& ea, int& eb) {
  const int c0 = __ldg(s.cls_off + cls), c1 = __ldg(s.cls_off + cls + 1);
  ea = c0 + (int)((long long)(c1 - c0) * z / s.nsplit);
  eb = c0 + (int)((long long)(c1 - c0) * (z + 1) / s.nsplit);
}

template <typename T>
__device__ __forceinline__ void gnc_sums_body(const GncStep& s, int stage, int bx, int by, int bz) {
  // FP32: static tables; BF16: the tables and the ring in dynamic memory
  __shared__ float4 mono_s[sums_streamed<T>() ? 1 : SMAXE][3];
  __shared__ int kof_s[sums_streamed<T>() ? 1 : SMAXE];
  extern __shared__ __align__(16) unsigned char sdyn[];
  float4 (*mono)[3] = sums_streamed<T>() ? reinterpret_cast<float4 (*)[3]>(sdyn) : mono_s;
  int* kof = sums_streamed<T>() ? reinterpret_cast<int*>(sdyn + (size_t)SMAXE * 3 * sizeof(float4)) : kof_s;
  T* ring = reinterpret_cast<T*>(sdyn + SUMS_TAB);          // [SRING][SBLK][SCB]
  const DevParams& p = s.p;
  const int cls = by;
  int ea, eb;
  split_range(s, cls, bz, ea, eb);
  const int cnt = min(eb - ea, SMAXE);
  // the split padded to whole blocks of SBLK: padding entries read velocity
  // 0 and carry zero monomials (pi_0 = 1 included), so they add nothing
  const int cntp = (cnt + SBLK - 1) / SBLK * SBLK;
  const float4* mt = reinterpret_cast<const float4*>(s.cls_mono);
  for (int t = threadIdx.x; t < 3 * cntp; t += SCB)
    mono[t / 3][t % 3] = t < 3 * cnt ? __ldg(mt + 3 * (size_t)ea + t) : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int t = threadIdx.x; t < cntp; t += SCB) kof[t] = t < cnt ? __ldg(s.cls_k + ea + t) : 0;
  __syncthreads();
  const int c = bx * SCB + threadIdx.x;
  Kah2 acc[NMONO / 2] = {};                      // monomials (2t, 2t + 1)
  // block n of the split, summed in FP32 and folded into the Kahan sums.
  // The ten products of a value go as five packed pairs (one fma.rn.f32x2
  // is two FP32 fused multiply-adds, each rounded as fmaf): monomials
  // (pi_0, pi_1) .. (pi_8, pi_9) against (x, x)
  auto add_block = [&](const float (&x)[SBLK], int n) {
    unsigned long long part[NMONO / 2] = {};
#pragma unroll
    for (int u = 0; u < SBLK; ++u) {
      const ulonglong2 m0 = *reinterpret_cast<const ulonglong2*>(&mono[n + u][0]);
      const ulonglong2 m1 = *reinterpret_cast<const ulonglong2*>(&mono[n + u][1]);
      const unsigned long long m2 = *reinterpret_cast<const unsigned long long*>(&mono[n + u][2]);
      unsigned long long xx;
      asm("mov.b64 %0, {%1, %1};" : "=l"(xx) : "f"(x[u]));
      asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(part[0]) : "l"(m0.x), "l"(xx));
      asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(part[1]) : "l"(m0.y), "l"(xx));
      asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(part[2]) : "l"(m1.x), "l"(xx));
      asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(part[3]) : "l"(m1.y), "l"(xx));
      asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(part[4]) : "l"(m2), "l"(xx));
    }
#pragma unroll
    for (int t = 0; t < NMONO / 2; ++t) kah_add2(acc[t], part[t]);
  };
  constexpr int VPC = 16 / (int)sizeof(T);       // values per 16-byte copy
  if (sums_streamed<T>() && p.N % VPC == 0) {
    // streamed (BF16, the cell count a multiple of 8): the planes of the
    // block's cells arrive by 16-byte asynchronous copies into a ring of
    // SRING blocks of SBLK planes, two blocks ahead of the one being summed;
    // one barrier per block.  FP32 keeps the loads through registers, which
    // measured faster there (77 against 80 us at 128^2 x 4096; BF16 76
    // against 80)
    constexpr int CPP = SCB / VPC;               // copies per plane
    const int c0 = bx * SCB, ncell = min(SCB, p.N - c0);   // a multiple of VPC
    const T* __restrict__ base = (const T*)(stage == 1 ? s.fhat : s.ftp) + c0;
    const int nblk = cntp / SBLK;
    auto issue = [&](int b) {
      if (b < nblk) {
        T* dst = ring + (size_t)(b % SRING) * SBLK * SCB;
        for (int q = threadIdx.x; q < SBLK * CPP; q += SCB) {
          const int u = q / CPP, ch = q % CPP;
          if (ch * VPC < ncell)
            cp16(dst + u * SCB + ch * VPC, base + (size_t)kof[b * SBLK + u] * p.N + ch * VPC);
        }
      }
      cp_commit();
    };
    issue(0);
    issue(1);
    for (int b = 0; b < nblk; ++b) {
      cp_wait<1>();                              // this thread's copies of block b
      __syncthreads();                           // everyone's; block b - 1 read by all
      issue(b + 2);                              // into block b - 1's slot
      const T* src = ring + (size_t)(b % SRING) * SBLK * SCB + threadIdx.x;
      float x[SBLK];
#pragma unroll
      for (int u = 0; u < SBLK; ++u) x[u] = tof(src[u * SCB]);
      add_block(x, b * SBLK);
    }
  } else {
    // each thread's loads through registers, the next block's in flight
    // while the current one is summed
    if (c >= p.N) return;                        // no barrier follows
    const T* __restrict__ col = (const T*)(stage == 1 ? s.fhat : s.ftp) + c;
    auto load_block = [&](float (&x)[SBLK], int n) {
#pragma unroll
      for (int u = 0; u < SBLK; ++u) x[u] = ldv(col + (size_t)kof[n + u] * p.N);
    };
    float v[SBLK], w[SBLK];
    if (cntp > 0) load_block(v, 0);
    for (int n = 0; n < cntp; n += 2 * SBLK) {
      if (n + SBLK < cntp) load_block(w, n + SBLK);
      add_block(v, n);
      if (n + SBLK >= cntp) break;
      if (n + 2 * SBLK < cntp) load_block(v, n + 2 * SBLK);
      add_block(w, n + SBLK);
    }
  }
  if (c >= p.N) return;
  double* out = s.sums + ((size_t)bz * s.ncls + cls) * NMONO * p.N + c;
#pragma unroll
  for (int t = 0; t < NMONO / 2; ++t) {
    Kah lo, hi;
    unpack2(acc[t].s, lo.s, hi.s);
    unpack2(acc[t].c, lo.c, hi.c);
    out[(size_t)(2 * t) * p.N] = kah_value(lo);
    out[(size_t)(2 * t + 1) * p.N] = kah_value(hi);
  }
}

template <typename T>
__global__ void __launch_bounds__(SCB, 3)
k_gnc_sums(GncStep s, int stage) {
  gnc_sums_body<T>(s, stage, blockIdx.x, blockIdx.y, blockIdx.z);
}


// --------------------------------------------------------------- cellfin
// nu_{m,u} = sum xi^m u(a, b) g over a class combination, from its moments
// mu of g, with a = a0 - hx xi_x, b = b0 - hy xi_y
__device__ __forceinline__ void stencil_moments(const float (&mu)[NMONO], float a0, float b0,
                                                float hx, float hy, float (&nu)[NNU]) {
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int mi = m == 1 ? 1 : 0, mj = m == 2 ? 1 : 0;
    const float M00 = mu[mono_ix(mi, mj)];
    const float M10 = mu[mono_ix(mi + 1, mj)], M01 = mu[mono_ix(mi, mj + 1)];
    const float M20 = mu[mono_ix(mi + 2, mj)], M11 = mu[mono_ix(mi + 1, mj + 1)];
    const float M02 = mu[mono_ix(mi, mj + 2)];
    nu[6 * m + 0] = M00;
    nu[6 * m + 1] = fmaf(a0, M00, -hx * M10);
    nu[6 * m + 2] = fmaf(b0, M00, -hy * M01);
    nu[6 * m + 3] = fmaf(a0 * a0, M00, fmaf(-2.f * a0 * hx, M10, hx * hx * M20));
    nu[6 * m + 4] = fmaf(a0 * b0, M00, fmaf(-a0 * hy, M01, fmaf(-b0 * hx, M10, hx * hy * M11)));
    nu[6 * m + 5] = fmaf(b0 * b0, M00, fmaf(-2.f * b0 * hy, M01, hy * hy * M02));
  }
}

// A block takes CFC cells with CFC threads per class combination (thread
// t: cell t % CFC, combination t / CFC).  The cells' FP64 work is done once:
// the first CFC threads form rho, u from the class sums (FP64), write them
// into mom and the equilibrium's assembly parameters into eq (FP32), and
// the equilibrium polynomial's coefficients into shared memory; all threads
// round the class sums (added over the velocity splits in FP64) to FP32 in
// shared memory.  Then each (cell, combination) forms nu in FP32.
constexpr int CFC = 64;                  // cells per cellfin block
constexpr int NCLS_MAX = 9;              // sign classes: (sign xi_x, sign xi_y)
constexpr int NCMB_MAX = 12;             // class combinations at most
__device__ __forceinline__ void gnc_cellfin_body(const GncStep& s, int stage, int bx) {
  __shared__ float cs[NCLS_MAX * NMONO][CFC];   // class sums, FP32
  __shared__ float qds[6][CFC];                 // equilibrium polynomial
  const DevParams& p = s.p;
  const size_t N = p.N;
  const int cl = threadIdx.x % CFC, cb = threadIdx.x / CFC;
  const int cell = bx * CFC + cl;
  const bool in = cell < p.N;
#pragma unroll 4
  for (int t = threadIdx.x; t < s.ncls * NMONO * CFC; t += blockDim.x) {
    const int cm = t / CFC, q = t % CFC, ce = bx * CFC + q;
    double v = 0.0;
    if (ce < p.N)
#pragma unroll 1
      for (int z = 0; z < s.nsplit; ++z) v += s.sums[((size_t)z * s.ncls * NMONO + cm) * N + ce];
    cs[cm][q] = (float)v;
  }
  if (cb == 0 && in) {
    double r = s.ref.W, jx = s.ref.Wx, jy = s.ref.Wy;
#pragma unroll 1
    for (int z = 0; z < s.nsplit; ++z)
#pragma unroll 3
      for (int c = 0; c < s.ncls; ++c) {
        const double* sc = s.sums + ((size_t)z * s.ncls + c) * NMONO * N + cell;
        r += sc[0];
        jx += sc[N];
        jy += sc[2 * N];
      }
    const double ux = jx / r, uy = jy / r;
    double* mom = stage == 1 ? s.mom_n : s.mom_p;
    mom[cell] = r;
    mom[N + cell] = ux;
    mom[2 * N + cell] = uy;
    store_par(stage == 1 ? s.eqn : s.eqp, p.N, cell, eq_params_u<float>(r, ux, uy, p.inv_RT, s.ref.rho0));
    // W_k (rho P(xi_k) - rho0) = W_k sum_q qd_q pi_q(xi_k), q over 1, x, y, xx, xy, yy
    const double vx = ux * p.inv_RT, vy = uy * p.inv_RT;
    qds[0][cl] = (float)((r - s.ref.rho0) - 0.5 * r * (ux * vx + uy * vy));
    qds[1][cl] = (float)(r * vx);
    qds[2][cl] = (float)(r * vy);
    qds[3][cl] = (float)(0.5 * r * vx * vx);
    qds[4][cl] = (float)(r * vx * vy);
    qds[5][cl] = (float)(0.5 * r * vy * vy);
  }
  __syncthreads();
  if (!in || cb >= s.ncombo) return;
  const StageCoef& sc = stage == 1 ? s.s1 : s.s2;
  const float b = (float)sc.b, omb = (float)(1.0 - sc.b);
  const float hx = (float)(sc.h * p.inv_dx), hy = (float)(sc.h * p.inv_dy);
  const GncCombo& C = s.cmb[cb];
  float mu[NMONO];
#pragma unroll
  for (int t = 0; t < NMONO; ++t) mu[t] = 0.f;
  for (int c = 0; c < s.ncls; ++c) {
    const float lam = C.lam[c];
    if (lam == 0.f) continue;
#pragma unroll
    for (int t = 0; t < NMONO; ++t) mu[t] = fmaf(lam, cs[c * NMONO + t][cl], mu[t]);
  }
  // g = (1 - b) src + b feq: the equilibrium's part by the combination's
  // quadrature table zc[p][q] = sum lam W_k pi_p pi_q
  const float* z = s.zc + (size_t)cb * NMONO * 6;
  float qd[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) qd[q] = qds[q][cl];
#pragma unroll
  for (int t = 0; t < NMONO; ++t) {
    float e = 0.f;
#pragma unroll
    for (int q = 0; q < 6; ++q) e = fmaf(__ldg(z + 6 * t + q), qd[q], e);
    mu[t] = fmaf(omb, mu[t], b * e);
  }
  float nu[NNU];
  stencil_moments(mu, C.a0, C.b0, hx, hy, nu);
  float* o = s.nu + (size_t)cb * NNU * N + cell;
#pragma unroll
  for (int t = 0; t < NNU; ++t) o[(size_t)t * N] = nu[t];
}

__global__ void __launch_bounds__(CFC * NCMB_MAX)
k_gnc_cellfin(GncStep s, int stage) {
  gnc_cellfin_body(s, stage, blockIdx.x);
}


// ---------------------------------------------------------------- ghosts
// A cell (ci, cj) at most one layer outside the mesh as a combination of
// cells inside it: periodic wrap, or the quadratic extrapolation across a
// wall (Q16) -- along x on rows inside the mesh, then along y, so a corner
// is the y-extrapolation of x-ghosts (as in the oracle).  Writes up to nine
// (cell index, coefficient) pairs and returns their number.
__device__ __forceinline__ int ghost_terms_x(const DevParams& p, int ci, int cj, float cf,
                                             int* idx, float* co) {
  if (ci < 0 || ci >= p.nx) {
    if (p.px) {
      ci = ci < 0 ? ci + p.nx : ci - p.nx;
    } else {
      const int i1 = ci < 0 ? 0 : p.nx - 1, sx = ci < 0 ? 1 : -1;
      idx[0] = cj * p.nx + i1;
      idx[1] = cj * p.nx + i1 + sx;
      idx[2] = cj * p.nx + i1 + 2 * sx;
      co[0] = 3.f * cf;
      co[1] = -3.f * cf;
      co[2] = cf;
      return 3;
    }
  }
  idx[0] = cj * p.nx + ci;
  co[0] = cf;
  return 1;
}
__device__ __forceinline__ int ghost_terms(const DevParams& p, int ci, int cj, int (&idx)[9],
                                           float (&co)[9]) {
  if (cj < 0 || cj >= p.ny) {
    if (p.py) {
      cj = cj < 0 ? cj + p.ny : cj - p.ny;
    } else {
      const int j1 = cj < 0 ? 0 : p.ny - 1, sy = cj < 0 ? 1 : -1;
      int n = ghost_terms_x(p, ci, j1, 3.f, idx, co);
      n += ghost_terms_x(p, ci, j1 + sy, -3.f, idx + n, co + n);
      n += ghost_terms_x(p, ci, j1 + 2 * sy, 1.f, idx + n, co + n);
      return n;
    }
  }
  return ghost_terms_x(p, ci, cj, 1.f, idx, co);
}

// --------------------------------------------------------------- facefin
// Face moments of combination cb for the stencil about cell (ci, cj):
// M_m = sum over the nonzero t_u(s) of t_u(s) nu_{m,u}(cell + s) (the
// list tl of GncStep); cells outside the mesh by their ghost terms, the
// stencil of a cell away from the walls directly
__device__ void face_moments(const GncStep& s, int cb, int ci, int cj, float (&M)[3]) {
  const DevParams& p = s.p;
  const float* base = s.nu + (size_t)cb * NNU * p.N;
  M[0] = M[1] = M[2] = 0.f;
  const bool inside = ci >= 1 && ci + 1 < p.nx && cj >= 1 && cj + 1 < p.ny;
  const size_t plane = (size_t)6 * p.N;            // from nu_{m,u} to nu_{m+1,u}
  if (inside) {
    // five terms' loads in flight at a time
#pragma unroll 5
    for (int q = 0; q < s.ntl; ++q) {
      const int t = s.tl_s[q], u = s.tl_u[q];
      const float w = s.tl_w[q];
      const float* b = base + (size_t)u * p.N;
      const int c = (cj + t / 3 - 1) * p.nx + ci + t % 3 - 1;
      M[0] = fmaf(w, __ldg(b + c), M[0]);
      M[1] = fmaf(w, __ldg(b + plane + c), M[1]);
      M[2] = fmaf(w, __ldg(b + 2 * plane + c), M[2]);
    }
    return;
  }
#pragma unroll 1
  for (int q = 0; q < s.ntl; ++q) {
    const int t = s.tl_s[q], u = s.tl_u[q];
    const float w = s.tl_w[q];
    const float* b = base + (size_t)u * p.N;
    {
      int idx[9];
      float co[9];
      const int n = ghost_terms(p, ci + t % 3 - 1, cj + t / 3 - 1, idx, co);
      float v0 = 0.f, v1 = 0.f, v2 = 0.f;
      for (int r = 0; r < n; ++r) {
        v0 = fmaf(co[r], __ldg(b + idx[r]), v0);
        v1 = fmaf(co[r], __ldg(b + plane + idx[r]), v1);
        v2 = fmaf(co[r], __ldg(b + 2 * plane + idx[r]), v2);
      }
      M[0] = fmaf(w, v0, M[0]);
      M[1] = fmaf(w, v1, M[1]);
      M[2] = fmaf(w, v2, M[2]);
    }
  }
}

// Every face of both directions: the face moments -> the face equilibrium's
// assembly parameters; at a wall, the leaving velocities by the wall rule
// and the wall density (bounce-back: the fluid cell's rho; diffuse: from the
// incoming flux, Q15) into wrho for the walls pass.
__device__ __forceinline__ void gnc_facefin_body(const GncStep& s, int stage, int bx) {
  const DevParams& p = s.p;
  const int nfx = p.ny * (p.nx + 1), nfy = (p.ny + 1) * p.nx;
  int f = bx * 64 + threadIdx.x;
  if (f >= nfx + nfy) return;
  const bool xdir = f < nfx;
  if (!xdir) f -= nfx;
  const int nf = xdir ? nfx : nfy;
  // face position: x-face fi between cells (fi - 1, j) and (fi, j); y-face
  // fj between (i, fj - 1) and (i, fj)
  const int a = xdir ? f % (p.nx + 1) : f / p.nx;      // fi or fj
  const int l = xdir ? f / (p.nx + 1) : f % p.nx;      // j or i
  const int n = xdir ? p.nx : p.ny;
  const bool per = xdir ? p.px : p.py;
  if (per && a == n) return;                           // face n is face 0
  float M[3];
  int side = -1;
  if (!per && (a == 0 || a == n)) {
    side = xdir ? (a == 0 ? SIDE_W : SIDE_E) : (a == 0 ? SIDE_S : SIDE_N);
    const int ci = xdir ? (a == 0 ? 0 : p.nx - 1) : l;
    const int cj = xdir ? l : (a == 0 ? 0 : p.ny - 1);
    face_moments(s, s.c_wf[side], ci, cj, M);
    double d[3] = {M[0], M[1], M[2]};
    const double* mom = stage == 1 ? s.mom_n : s.mom_p;
    double rw;
    if (p.bc_kind[side] == BC_BOUNCEBACK) {
      float Mi[3] = {M[0], M[1], M[2]};
      if (s.c_win[side] != s.c_wf[side]) face_moments(s, s.c_win[side], ci, cj, Mi);
      rw = mom[cj * p.nx + ci];
      d[0] += (double)Mi[0] + rw * s.wB[side][0] + s.wH[side][0];
      d[1] += -(double)Mi[1] + rw * s.wB[side][1] + s.wH[side][1];
      d[2] += -(double)Mi[2] + rw * s.wB[side][2] + s.wH[side][2];
    } else {
      // incoming normal flux sum_{xi.n > 0} (xi.n) f-bar, n the fluid's
      // outward normal
      const double qn = (a == 0 ? -1.0 : 1.0) * (xdir ? d[1] : d[2]);
      rw = (s.ds_out[side] + qn) / p.ds_den[side];
      for (int m = 0; m < 3; ++m) d[m] += rw * s.wMo[side][m] - s.wWo[side][m];
    }
    const int slot = side == SIDE_W ? l : side == SIDE_E ? p.ny + l
                   : side == SIDE_S ? 2 * p.ny + l : 2 * p.ny + p.nx + l;
    s.wrho[slot] = rw;
    store_par(xdir ? s.fpx : s.fpy, nf, f,
              eq_params_j<float>(s.ref.W + d[0], s.ref.Wx + d[1], s.ref.Wy + d[2], p.inv_RT, s.ref.rho0));
    return;
  }
  // interior: the class with xi.n > 0 about the lower cell, xi.n < 0 about
  // the upper cell (a tie enters both combinations with weight 1/2, Q4)
  float Ml[3], Mu[3];
  if (xdir) {
    face_moments(s, s.c_lo[0], a - 1, l, Ml);
    face_moments(s, s.c_up[0], a, l, Mu);
  } else {
    face_moments(s, s.c_lo[1], l, a - 1, Ml);
    face_moments(s, s.c_up[1], l, a, Mu);
  }
  const EqF<float> q = eq_params_j<float>(s.ref.W + ((double)Ml[0] + Mu[0]),
                                          s.ref.Wx + ((double)Ml[1] + Mu[1]),
                                          s.ref.Wy + ((double)Ml[2] + Mu[2]), p.inv_RT, s.ref.rho0);
  float* fp = xdir ? s.fpx : s.fpy;
  store_par(fp, nf, f, q);
  if (per && a == 0) store_par(fp, nf, xdir ? f + p.nx : f + p.ny * p.nx, q);
}

__global__ void __launch_bounds__(64)
k_gnc_facefin(GncStep s, int stage) {
  gnc_facefin_body(s, stage, blockIdx.x);
}


// ----------------------------------------------------------------- walls

// Wall faces: f-bar per velocity.  Block: one wall side, WSEG consecutive
// wall faces, WCH velocities.  Per velocity the strip of cells at distance
// 0-2 from the wall along the segment (plus three cells on either end) is
// staged as g in shared memory, the ghosts are extrapolated there (Q16: the
// x-direction first, on rows inside the mesh, then the y-direction), and
// each thread forms one face's upwind stencil about the fluid cell.  Written
// are the fluid-side values of the velocities hitting or running along the
// wall, and diffuse scattering's f-bar_k = rho_w W_k P(xi_k; u_w) - W_k rho0
// for the leaving ones; bounce-back's leaving values (eq. BB) are formed by
// the update from the mirrored velocity's entry.
constexpr int WSEG = 128;                // wall faces per block
constexpr int WCH = 8;                   // velocities per block (their loads issued at once)
constexpr int WTW = WSEG + 6;            // strip positions along the wall
constexpr int WEPT = (3 * WTW + 127) / 128;   // staged cells per thread

__device__ __forceinline__ int wall_segments(int n) { return (n + WSEG - 1) / WSEG; }

template <typename T>
__device__ __forceinline__ void gnc_walls_body(const GncStep& s, int stage, int bx, int by) {
  __shared__ float st[2][4 * WTW];       // [depth 0 (ghost) .. 3][position]
  const DevParams& p = s.p;
  // block -> wall side and segment (walled sides only, in the order W, E, S, N)
  int id = bx, side = -1, seg = 0;
  for (int sd = 0; sd < 4 && side < 0; ++sd) {
    const bool xw = sd <= SIDE_E;
    if (xw ? p.px : p.py) continue;
    const int ns = wall_segments(xw ? p.ny : p.nx);
    if (id < ns) side = sd, seg = id;
    else id -= ns;
  }
  if (side < 0) return;
  const bool xw = side <= SIDE_E;
  const int nt = xw ? p.ny : p.nx;       // faces along the wall
  const bool tper = xw ? p.py : p.px;    // the direction along the wall is periodic
  const int t0 = seg * WSEG, t1 = min(nt, t0 + WSEG);
  const int k0 = by * WCH, k1 = min(p.nv, k0 + WCH);
  const T* __restrict__ src = (const T*)(stage == 1 ? s.fhat : s.ftp);
  const float* __restrict__ eq = stage == 1 ? s.eqn : s.eqp;
  const float b = (float)(stage == 1 ? s.s1.b : s.s2.b);
  const float4* vq = (const float4*)s.vq;
  // cell (depth d = 1..3 from the wall, position tt) of the strip
  auto cell_of = [&](int d, int tt) {
    const int i = side == SIDE_W ? d - 1 : side == SIDE_E ? p.nx - d : tt;
    const int j = side == SIDE_S ? d - 1 : side == SIDE_N ? p.ny - d : tt;
    return j * p.nx + i;
  };
  int sidx[WEPT], soff[WEPT];
  bool sin_[WEPT];
  EqF<float> sq[WEPT];
#pragma unroll
  for (int m = 0; m < WEPT; ++m) {
    const int e = threadIdx.x + 128 * m;
    const int d = 1 + e / WTW, x = e % WTW;
    int tt = t0 - 3 + x;
    bool in = e < 3 * WTW;
    if (tper) tt = ((tt % nt) + nt) % nt;
    else in = in && tt >= 0 && tt < nt;
    sin_[m] = in;
    sidx[m] = e < 3 * WTW ? d * WTW + x : -1;
    soff[m] = in ? cell_of(d, tt) : 0;
    if (in) {
      sq[m].vx = __ldg(eq + soff[m]);
      sq[m].vy = __ldg(eq + p.N + soff[m]);
      sq[m].bm1 = __ldg(eq + 2 * p.N + soff[m]);
      sq[m].r = __ldg(eq + 3 * p.N + soff[m]);
      sq[m].dr = __ldg(eq + 4 * p.N + soff[m]);
    }
  }
  const int set = side == SIDE_W ? 1 : side == SIDE_E ? 0 : side == SIDE_S ? 3 : 2;
  const int tt = t0 + threadIdx.x;       // this thread's face
  const int slot = (side == SIDE_W ? 0 : side == SIDE_E ? p.ny : side == SIDE_S ? 2 * p.ny
                                                                 : 2 * p.ny + p.nx) + tt;
  const double rw = tt < t1 ? s.wrho[slot] : 0.0;
  // the block's velocities: their face weights for this side, and for
  // diffuse scattering W_k and the wall Maxwellian's deviation from it,
  // f_wall,k - W_k (FP64 difference, rounded once)
  __shared__ float wts[WCH][9], wdev[WCH], wwk[WCH];
  for (int t = threadIdx.x; t < WCH * 9; t += 128) {
    const int q = t / 9, k = min(k0 + q, p.nv - 1);
    wts[q][t % 9] = __ldg(s.fwt + ((size_t)(stage - 1) * p.nv + k) * WPV + 12 * set + t % 9);
  }
  if (threadIdx.x < WCH) {
    const int k = min(k0 + (int)threadIdx.x, p.nv - 1);
    const double wk = __ldg(p.w + k);
    wdev[threadIdx.x] = (float)(__ldg(p.feq_wall + (size_t)side * p.nv + k) - wk);
    wwk[threadIdx.x] = (float)wk;
  }
  // diffuse leaving values rho_w f_wall,k - W_k rho0 = W_k (rho_w - rho0) +
  // rho_w (f_wall,k - W_k): FP32 terms of the result's own size
  const float rwf = (float)rw, drw = (float)(rw - s.ref.rho0);
  T raw[WCH][WEPT];
#pragma unroll
  for (int q = 0; q < WCH; ++q)
#pragma unroll
    for (int m = 0; m < WEPT; ++m)
      if (sin_[m] && k0 + q < k1) raw[q][m] = ldr(src + (size_t)(k0 + q) * p.N + soff[m]);
#pragma unroll
  for (int kq = 0; kq < WCH; ++kq) {
    const int k = k0 + kq;
    if (k >= k1) break;                  // uniform per block
    float* g = st[kq & 1];
    const float4 e4 = ld4(vq + p.nv + k);
#pragma unroll
    for (int m = 0; m < WEPT; ++m)
      if (sidx[m] >= 0) {
        float v = 0.f;
        if (sin_[m]) {
          const float r = tof(raw[kq][m]);
          v = fmaf(b, feq_dev<float>(sq[m], e4.x, e4.y, e4.z) - r, r);
        }
        g[sidx[m]] = v;
      }
    __syncthreads();
    // ghosts (reading Q16: across x on the mesh rows, then across y) in one
    // pass, each from mesh cells only: depth 0 across the wall at the mesh
    // positions; where the direction along the wall has walls, depths 1-3
    // along it beyond the strip's ends, and depth 0 there (the corner) as
    // the nine-cell product of the two extrapolations
    for (int q = threadIdx.x; q < WTW + 8; q += 128) {
      int at = -1;
      float v = 0.f;
      if (q < WTW) {
        const int t = t0 - 3 + q;
        if (tper || (t >= 0 && t < nt)) {
          at = q;
          v = 3.f * g[WTW + q] - 3.f * g[2 * WTW + q] + g[3 * WTW + q];
        }
      } else if (!tper) {
        const int u = q - WTW, d = u & 3, lowend = u < 4;
        const int xg = (lowend ? -1 : nt) - (t0 - 3);        // ghost position
        const int s1 = lowend ? 1 : -1;
        if (xg >= 0 && xg < WTW && xg + 3 * s1 >= 0 && xg + 3 * s1 < WTW) {
          auto along = [&](int dd) {
            const float* r = g + dd * WTW;
            return 3.f * r[xg + s1] - 3.f * r[xg + 2 * s1] + r[xg + 3 * s1];
          };
          at = d * WTW + xg;
          v = d > 0 ? along(d) : 3.f * along(1) - 3.f * along(2) + along(3);
        }
      }
      if (at >= 0) g[at] = v;
    }
    __syncthreads();
    if (tt < t1) {
      const float* w = wts[kq];
      float v = 0.f;
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const int dy = t / 3 - 1, dx = t % 3 - 1;
        const int d = side == SIDE_W ? dx + 1 : side == SIDE_E ? 1 - dx : side == SIDE_S ? dy + 1 : 1 - dy;
        const int q = xw ? dy : dx;
        v = fmaf(w[t], g[d * WTW + (tt + q - t0 + 3)], v);
      }
      const float xn = side == SIDE_W ? -e4.x : side == SIDE_E ? e4.x : side == SIDE_S ? -e4.y : e4.y;
      if (xn < 0.f && p.bc_kind[side] == BC_DIFFUSE) v = fmaf(rwf, wdev[kq], drw * wwk[kq]);
      s.wf[(size_t)k * s.nw + slot] = v;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(128)
k_gnc_walls(GncStep s, int stage) {
  gnc_walls_body<T>(s, stage, blockIdx.x, blockIdx.y);
}


// ---------------------------------------------------------------- update
// F(xi) = (x/dx)(P_E - P_W) + (y/dy)(P_N - P_S) over the faces of cell
// (i, j), scaled by sc (the face equilibria's part of the micro-flux)
__device__ __forceinline__ Cubic<float> gnc_flux_cubic(const GncStep& s, int i, int j, float sc) {
  const int nx = s.p.nx, ny = s.p.ny;
  const int nfx = ny * (nx + 1), nfy = (ny + 1) * nx;
  const int fx = j * (nx + 1) + i, fy = j * nx + i;
  const Quad<float> w = quad(s.fpx, nfx, fx), e = quad(s.fpx, nfx, fx + 1);
  const Quad<float> so = quad(s.fpy, nfy, fy), no = quad(s.fpy, nfy, fy + nx);
  const float ax = sc * (float)s.p.inv_dx, ay = sc * (float)s.p.inv_dy;
  Cubic<float> F;
  F.c[0] = 0.f;
  F.c[1] = ax * (e.c0 - w.c0);
  F.c[2] = ay * (no.c0 - so.c0);
  F.c[3] = ax * (e.cx - w.cx);
  F.c[4] = fmaf(ax, e.cy - w.cy, ay * (no.cx - so.cx));
  F.c[5] = ay * (no.cy - so.cy);
  F.c[6] = ax * (e.cxx - w.cxx);
  F.c[7] = fmaf(ax, e.cxy - w.cxy, ay * (no.cxx - so.cxx));
  F.c[8] = fmaf(ax, e.cyy - w.cyy, ay * (no.cxy - so.cxy));
  F.c[9] = ay * (no.cyy - so.cyy);
  return F;
}
__device__ __forceinline__ void add_quad(Cubic<float>& S, const Quad<float>& q, float sc) {
  S.c[0] = fmaf(sc, q.c0, S.c[0]);
  S.c[1] = fmaf(sc, q.cx, S.c[1]);
  S.c[2] = fmaf(sc, q.cy, S.c[2]);
  S.c[3] = fmaf(sc, q.cxx, S.c[3]);
  S.c[4] = fmaf(sc, q.cxy, S.c[4]);
  S.c[5] = fmaf(sc, q.cyy, S.c[5]);
}

// the 3 x 3 window of W with lower-left corner (row r, column c): rows
// south to north, columns west to east (the order of eq. flux_DS's weights)
#define WIN3(W, r, c)                                                                      \
  W[r][c], W[r][(c) + 1], W[r][(c) + 2], W[(r) + 1][c], W[(r) + 1][(c) + 1],                 \
      W[(r) + 1][(c) + 2], W[(r) + 2][c], W[(r) + 2][(c) + 1], W[(r) + 2][(c) + 2]

// g at the x-wall ghost in staged column sx, row sy, extrapolated from the
// three cells inwards (dx = +1 west, -1 east) by the quadratic of Q16
__device__ __forceinline__ float ghost_x(const float* __restrict__ g, int sx, int sy, int dx) {
  const float* r = g + sy * HXT + sx;
  return 3.f * r[dx] - 3.f * r[2 * dx] + r[3 * dx];
}

// Wall ghosts of a staged plane (reading Q16: across x on the mesh rows,
// then across y on every column) in one pass: a corner is the
// y-extrapolation of three x-extrapolated values, i.e. nine mesh cells, so
// no ghost reads another; the caller's barrier ends the pass (one for
// several planes).
__device__ __forceinline__ void stage_ghosts(const DevParams& p, float* __restrict__ g, int i0,
                                             int j0, bool wx, bool wy) {
  if (!wx && !wy) return;
  const int t = threadIdx.x;
  const int xw = i0 == 0 ? 1 : -64;                   // staged column of gi = -1
  const int xe = p.nx - i0 + 2 < HXT ? p.nx - i0 + 2 : -64;    // of gi = nx
  int idx = -1;
  float v = 0.f;
  if (t < 2 * HYT) {
    const int sy = t % HYT, gj = j0 - 2 + sy;
    const int sx = t < HYT ? xw : xe, d = t < HYT ? 1 : -1;
    if (wx && sx >= 0 && (p.py || (gj >= 0 && gj < p.ny))) {
      idx = sy * HXT + sx;
      v = ghost_x(g, sx, sy, d);
    }
  } else if (t < 2 * HYT + 2 * HXT) {
    const int u = t - 2 * HYT, sx = u % HXT, gi = i0 - 2 + sx;
    const int ys = j0 == 0 ? 1 : -64, yn = p.ny - j0 + 2 < HYT ? p.ny - j0 + 2 : -64;
    const int sy = u < HXT ? ys : yn, d = u < HXT ? 1 : -1;
    if (wy && sy >= 0) {
      const float* c = g + sy * HXT + sx;
      if (p.px || (gi >= 0 && gi < p.nx)) {
        idx = sy * HXT + sx;
        v = 3.f * c[d * HXT] - 3.f * c[2 * d * HXT] + c[3 * d * HXT];
      } else if ((gi == -1 || gi == p.nx) && sx + 3 * (gi < 0 ? 1 : -1) >= 0 &&
                 sx + 3 * (gi < 0 ? 1 : -1) < HXT) {
        const int dx = gi < 0 ? 1 : -1;
        idx = sy * HXT + sx;
        v = 3.f * ghost_x(g, sx, sy + d, dx) - 3.f * ghost_x(g, sx, sy + 2 * d, dx) +
            ghost_x(g, sx, sy + 3 * d, dx);
      }
    }
  }
  if (idx >= 0) g[idx] = v;
}

// staged position (column, row) of halo cell h of a tile: rows 0-1, rows
// 18-19, then columns 0, 1, 34, 35 of rows 2-17
__device__ __forceinline__ void halo_pos(int h, int& sx, int& sy) {
  if (h < 2 * HXT) {
    sy = h / HXT;
    sx = h % HXT;
  } else if (h < 4 * HXT) {
    sy = TYT + 2 + (h - 2 * HXT) / HXT;
    sx = (h - 2 * HXT) % HXT;
  } else {
    const int t = h - 4 * HXT;
    sy = 2 + t / 4;
    const int c = t % 4;
    sx = c < 2 ? c : TXT + c;
  }
}

// Ring of per-velocity inputs of the update, NRING planes deep, filled by
// asynchronous copies ahead of use (FP32: the next pair of planes while a
// pair is formed; BF16: three planes ahead): the staged plane (FP32
// storage; BF16 arrives through registers), the face weights, the velocity's
// table rows, its bounce-back coefficients, f^ of the tile's cells (stage 2,
// FP32) and the tile's wall-face values.  Offsets in floats, 16-byte aligned.
constexpr int NRING = 4;                          // a power of two
constexpr int NWALL = 2 * TYT + 2 * TXT;          // W rows, E rows, S columns, N columns
constexpr int RG = 0;                             // g (source values until converted)
constexpr int RW = RG + NST;                      // face weights (WPV)
constexpr int RV = RW + WPV;                      // (xi_x, xi_y, W, 0), flux factors
constexpr int RC = RV + 8;                        // bounce-back (c_k, shift_k) per side
constexpr int RF = RC + 8;                        // f^ of the tile's cells
constexpr int RB = RF + TXT * TYT;                // wall-face f-bar
constexpr int RPL = RB + NWALL;
static_assert(RW % 4 == 0 && RV % 4 == 0 && RC % 4 == 0 && RF % 4 == 0 && RPL % 4 == 0,
              "ring regions must be 16-byte aligned");

// cubic() of two cells at once (the same operations, lane by lane)
__device__ __forceinline__ unsigned long long cubic2(const unsigned long long (&S)[10],
                                                     unsigned long long x, unsigned long long y) {
  const unsigned long long t1 = fma2(x, S[6], fma2(y, S[7], S[3]));
  const unsigned long long t2 = fma2(y, S[8], S[4]);
  const unsigned long long t3 = fma2(y, S[9], S[5]);
  const unsigned long long X = fma2(x, t1, fma2(y, t2, S[1]));
  const unsigned long long Y = fma2(y, t3, S[2]);
  return fma2(x, X, fma2(y, Y, S[0]));
}

// two partial chains: the dependent-FMA depth of a 3 x 3 stencil halves
__device__ __forceinline__ float dot9s(const float* __restrict__ T, float s00, float s01, float s02,
                                       float s10, float s11, float s12, float s20, float s21,
                                       float s22) {
  float u = T[0] * s00;
  float v = T[1] * s01;
  u = fmaf(T[2], s02, u);
  v = fmaf(T[3], s10, v);
  u = fmaf(T[4], s11, u);
  v = fmaf(T[5], s12, v);
  u = fmaf(T[6], s20, u);
  v = fmaf(T[7], s21, v);
  u = fmaf(T[8], s22, u);
  return u + v;
}

// The x- and y-face values of a lane's cells from its stencil windows
// (window row 0, column 0 at g0): x-faces read rows 1..RPW+2, columns
// OX..OX+2, y-faces rows OY..OY+RPW+2, columns 1..3.  The x-faces' entries
// in columns 1..3 are the y-faces', so each is read once: 21 shared loads
// (27 with OX = 0) instead of 39.
template <int OX, int OY>
__device__ __forceinline__ void window_faces(const float* __restrict__ g0, const float* Tx,
                                             const float* Ty, float (&fx)[RPW],
                                             float (&fy)[RPW + 1]) {
  float Y[RPW + 3][3], X0[RPW + 2];
#pragma unroll
  for (int q = 0; q < RPW + 3; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) Y[q][c] = g0[(q + OY) * HXT + 1 + c];
  if (!OX) {
#pragma unroll
    for (int q = 0; q < RPW + 2; ++q) X0[q] = g0[(q + 1) * HXT];
  }
  // entry (q, c) of the x-face window
#define XW(q, c) (OX ? Y[(q) + 1 - OY][c] : ((c) == 0 ? X0[q] : Y[(q) + 1 - OY][(c) - 1]))
#pragma unroll
  for (int m = 0; m < RPW; ++m)
    fx[m] = dot9s(Tx, XW(m, 0), XW(m, 1), XW(m, 2), XW(m + 1, 0), XW(m + 1, 1), XW(m + 1, 2),
                  XW(m + 2, 0), XW(m + 2, 1), XW(m + 2, 2));
#undef XW
#pragma unroll
  for (int m = 0; m <= RPW; ++m) fy[m] = dot9s(Ty, WIN3(Y, m, 0));
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
// deviations by 1 + O(2^-24) every step).
//
// Warp w takes rows 4w .. 4w + 3 of the tile, lane l column i0 + l.  Each
// lane forms the x-face west of each of its cells and the y-faces south of
// them and north of the last; the east face comes from the next lane, and
// lanes 0-3 form the east faces of the tile's last column (for lane 31).
// Without tie velocities the upwind side is a uniform offset of the window
// loads; with them (TIES) every face is a 12-point stencil whose weights
// carry both sides.  FP32: one barrier per two velocities (both planes
// converted before it, both planes' faces after it); BF16: one per velocity;
// one more on tiles whose halo reaches a wall (the ghost pass).  At a wall face the value comes from the walls pass, for
// a velocity leaving a bounce-back wall as the mirrored velocity's entry
// plus rho_w c_k + shift_k (eq. BB in deviations).
template <typename T, int STAGE, bool TIES>
__device__ __forceinline__ void gnc_update_body(const GncStep& s, float cA, float cB, float sP,
                                                float sQ, float sF, int bx) {
  constexpr bool ASYNC = sizeof(T) == 4;       // FP32: the plane arrives by copies
  __shared__ __align__(16) float ring[NRING][RPL];
  __shared__ float rwb[NWALL];                 // wall densities of the tile's wall faces
  // equilibrium of the staged cells as W (c0 + E + h E^2), E = xi . (A, B):
  // (c0, A, B, h) = (rho - rho0 - rho |u|^2/2RT, rho u_x/RT, rho u_y/RT,
  // 1/(2 rho)), the assembly of feq_dev regrouped around E = rho xi.u/RT
  __shared__ float4 prm4[NST];
  const DevParams& p = s.p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tiles = s.tiles_x * s.tiles_y;
  const int tile = bx % tiles, chunk = bx / tiles;
  const int i0 = (tile % s.tiles_x) * TXT, j0 = (tile / s.tiles_x) * TYT;
  const int k0 = chunk * s.kc, k1 = min(p.nv, k0 + s.kc);
  if (k0 >= k1) return;                                     // uniform per block
  const StageCoef& sc = STAGE == 1 ? s.s1 : s.s2;
  const T* __restrict__ src = (const T*)(STAGE == 1 ? s.fhat : s.ftp);
  const float* __restrict__ eq = STAGE == 1 ? s.eqn : s.eqp;
  // stage 2 reads f^ of its own cells and overwrites them: no restrict
  T* dst = (T*)(STAGE == 1 ? s.ftp : s.fhat);
  const T* fh = (const T*)s.fhat;
  const float b = (float)sc.b;
  const float4* vq = (const float4*)s.vq;
  const float* __restrict__ fwt = s.fwt + (size_t)(STAGE - 1) * p.nv * WPV;
  const bool wx = !p.px && (i0 == 0 || i0 + TXT + 2 >= p.nx);
  const bool wy = !p.py && (j0 == 0 || j0 + TYT + 2 >= p.ny);
  const bool wall_tile = (!p.px && (i0 == 0 || i0 + TXT >= p.nx)) ||
                         (!p.py && (j0 == 0 || j0 + TYT >= p.ny));
  const int N = p.N;

  const int i = i0 + lane;
  const int jr = j0 + RPW * warp;                           // the warp's first row
  bool ok[RPW];
  int cell[RPW];
  Cubic<float> S[RPW] = {};
#pragma unroll
  for (int m = 0; m < RPW; ++m) {
    const int j = jr + m;
    ok[m] = i < p.nx && j < p.ny;
    cell[m] = ok[m] ? j * p.nx + i : 0;
    if (ok[m]) {
      S[m] = gnc_flux_cubic(s, i, j, sF);
      add_quad(S[m], quad(s.eqn, N, cell[m]), sP);
      if (STAGE == 2) add_quad(S[m], quad(s.eqp, N, cell[m]), sQ);
    }
  }
  // the cubics of cells (2q, 2q + 1) as packed FP32 pairs: both are
  // evaluated at the same xi, two per fma.rn.f32x2 (each lane rounded as
  // fmaf, so the values are those of cubic())
  unsigned long long SP[RPW / 2][10];
#pragma unroll
  for (int q = 0; q < RPW / 2; ++q)
#pragma unroll
    for (int t = 0; t < 10; ++t) SP[q][t] = pack2(S[2 * q].c[t], S[2 * q + 1].c[t]);
  // the tile's wall faces, the same for every velocity, packed in one word:
  // bits 0-3 the rows m whose x-face west of this lane's cell is on the W or
  // E wall, 4-8 the rows m (0..RPW) whose south face is on a y-wall, 9-13
  // those on the north wall, 14 the tile's last east face (lanes < RPW) on
  // the E wall, 15 a bounce-back wall, 16-23 the RB index of the lane's
  // first x-wall row; kept in shared memory, read once per velocity on wall
  // tiles only
  __shared__ unsigned wbits_s[UNT];
  unsigned wb0 = 0u;
  if (!p.px && (i == 0 || i == p.nx)) {
    wb0 |= (unsigned)((i == 0 ? 0 : TYT) + RPW * warp) << 16;
#pragma unroll
    for (int m = 0; m < RPW; ++m)
      if (jr + m < p.ny) wb0 |= 1u << m;
  }
  if (!p.px && lane < RPW && i0 + TXT == p.nx && jr + lane < p.ny) wb0 |= 1u << 14;
  if (!p.py && i < p.nx) {
#pragma unroll
    for (int m = 0; m <= RPW; ++m) {
      if (jr + m == 0) wb0 |= 1u << (4 + m);
      else if (jr + m == p.ny) wb0 |= (1u << (4 + m)) | (1u << (9 + m));
    }
  }
  if ((!p.px && (p.bc_kind[SIDE_W] == BC_BOUNCEBACK || p.bc_kind[SIDE_E] == BC_BOUNCEBACK)) ||
      (!p.py && (p.bc_kind[SIDE_S] == BC_BOUNCEBACK || p.bc_kind[SIDE_N] == BC_BOUNCEBACK)))
    wb0 |= 1u << 15;
  wbits_s[threadIdx.x] = wb0;
  // this thread's wall face in the ring's wall region (thread t < NWALL):
  // W row t, E row t - 16, S column t - 32, N column t - 64 of the tile
  int wside = -1, wslot = -1;
  if (threadIdx.x < NWALL) {
    const int t = threadIdx.x;
    if (t < 2 * TYT) {
      const int j = j0 + t % TYT;
      wside = t < TYT ? SIDE_W : SIDE_E;
      const bool here = !p.px && j < p.ny && (t < TYT ? i0 == 0 : i0 + TXT >= p.nx);
      if (here) wslot = (t < TYT ? 0 : p.ny) + j;
    } else {
      const int c = (t - 2 * TYT) % TXT, ii = i0 + c;
      const bool south = t < 2 * TYT + TXT;
      wside = south ? SIDE_S : SIDE_N;
      const bool here = !p.py && ii < p.nx && (south ? j0 == 0 : j0 + TYT >= p.ny);
      if (here) wslot = (south ? 2 * p.ny : 2 * p.ny + p.nx) + ii;
    }
    rwb[t] = wslot >= 0 ? (float)s.wrho[wslot] : 0.f;
  }

  // staging: cells (sx, sy) of the 36 x 20 plane, own cells first
  int soff[EPT], sidx[EPT];
  bool sact[EPT];
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    int sx, sy;
    if (m < RPW) {
      sx = lane + 2;
      sy = RPW * warp + m + 2;
      sact[m] = true;
    } else {
      const int h = threadIdx.x + UNT * (m - RPW);
      sact[m] = h < NHALO;
      halo_pos(sact[m] ? h : 0, sx, sy);
    }
    sidx[m] = sy * HXT + sx;
    int gi = i0 - 2 + sx, gj = j0 - 2 + sy;
    if (p.px) gi = ((gi % p.nx) + p.nx) % p.nx;
    else gi = min(max(gi, 0), p.nx - 1);
    if (p.py) gj = ((gj % p.ny) + p.ny) % p.ny;
    else gj = min(max(gj, 0), p.ny - 1);
    soff[m] = gj * p.nx + gi;
    // each thread reads back only the entries it writes: no barrier
    if (sact[m]) {
      const float vx = __ldg(eq + soff[m]), vy = __ldg(eq + N + soff[m]);
      const float bm1 = __ldg(eq + 2 * (size_t)N + soff[m]), r = __ldg(eq + 3 * (size_t)N + soff[m]);
      const float dr = __ldg(eq + 4 * (size_t)N + soff[m]);
      prm4[sidx[m]] = make_float4(fmaf(r, bm1, dr), r * vx, r * vy, 0.5f / r);
    }
  }

  // copies of velocity kq's inputs into ring buffer q; one commit group per
  // plane, also when empty, so the group count stays uniform.  FP32: the
  // planes go in pairs, one barrier for two (AHEAD = 2 planes in flight);
  // BF16 (values through registers): one plane per barrier, three ahead.
  constexpr int PAIR = ASYNC ? 2 : 1;
  constexpr int AHEAD = NRING - PAIR;
  auto issue = [&](int kq, int q, int ks) {
    if (kq < k1) {
      float* R = ring[q];
      if constexpr (ASYNC) {
#pragma unroll
        for (int m = 0; m < EPT; ++m)
          if (sact[m]) cp4(&R[RG + sidx[m]], src + (size_t)kq * N + soff[m]);
        if (STAGE == 2) {
#pragma unroll
          for (int m = 0; m < RPW; ++m)
            if (ok[m]) cp4(&R[RF + (RPW * warp + m) * TXT + lane], fh + (size_t)kq * N + cell[m]);
        }
      }
      const int t = threadIdx.x;
      if (t < WPV / 4) cp16(&R[RW + 4 * t], fwt + (size_t)kq * WPV + 4 * t);
      else if (t == WPV / 4) cp16(&R[RV], vq + p.nv + kq);
      else if (t == WPV / 4 + 1) cp16(&R[RV + 4], vq + 2 * p.nv + kq);
      else if (t < WPV / 4 + 4) cp16(&R[RC + 4 * (t - WPV / 4 - 2)], s.wbb + 4 * (size_t)kq + 2 * (t - WPV / 4 - 2));
      if (wslot >= 0) cp4(&R[RB + t], s.wf + (size_t)ks * s.nw + wslot);
    }
    cp_commit();
  };
  auto wall_src = [&](int kq) {                   // wall value's source velocity
    return wslot >= 0 && kq < k1 ? __ldg(s.wsrc + (size_t)wside * p.nv + kq) : 0;
  };
  int ksrc[PAIR];                                 // for the next iteration's issues
#pragma unroll
  for (int h = 0; h < PAIR; ++h) ksrc[h] = wall_src(k0 + AHEAD + h);
#pragma unroll
  for (int q = 0; q < AHEAD; ++q) issue(k0 + q, q, wall_src(k0 + q));
  T raw[EPT];
  if constexpr (!ASYNC) {
#pragma unroll
    for (int m = 0; m < EPT; ++m)
      if (sact[m]) raw[m] = ldr(src + (size_t)k0 * N + soff[m]);
  }

  // the faces of velocity k's plane (staged as g in ring slot R) and the
  // update of the tile's cells from their source (own) and f^ (fown) values
  auto plane_out = [&](int k, const float* R, const float4 e4, const float (&ownv)[RPW],
                       const float (&fownv)[RPW]) {
    const float* g = R + RG;
    const float* wk = R + RW;
    const int sgx = e4.x > 0.f ? 1 : (e4.x < 0.f ? -1 : 0);
    const int sgy = e4.y > 0.f ? 1 : (e4.y < 0.f ? -1 : 0);
    const float* g0 = g + (RPW * warp) * HXT + lane;       // window row 0, column 0 (cell i - 2)
    float fx[RPW], fy[RPW + 1], ext = 0.f;
    if constexpr (!TIES) {
      // x-faces: about cell i - 1 (window columns 0-2) or i (1-3); y-faces:
      // about the cell below (window rows m .. m + 2) or the cell (m + 1 ..)
      const int ox = sgx > 0 ? 0 : 1, oy = sgy > 0 ? 0 : 1;
      const float* Tx = wk + (sgx > 0 ? 0 : 12);
      const float* Ty = wk + (sgy > 0 ? 24 : 36);
      float X[RPW + 2][3], Y[RPW + 3][3];
#pragma unroll
      for (int q = 0; q < RPW + 2; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) X[q][c] = g0[(q + 1) * HXT + ox + c];
#pragma unroll
      for (int q = 0; q < RPW + 3; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) Y[q][c] = g0[(q + oy) * HXT + 1 + c];
#pragma unroll
      for (int m = 0; m < RPW; ++m) fx[m] = dot9s(Tx, WIN3(X, m, 0));
#pragma unroll
      for (int m = 0; m <= RPW; ++m) fy[m] = dot9s(Ty, WIN3(Y, m, 0));
      if (lane < RPW) {
        const float* ge = g + (RPW * warp + lane + 1) * HXT + TXT + ox;
        ext = dot9s(Tx, ge[0], ge[1], ge[2], ge[HXT], ge[HXT + 1], ge[HXT + 2], ge[2 * HXT],
                    ge[2 * HXT + 1], ge[2 * HXT + 2]);
      }
    } else {
      // 12-point stencils: x 3 rows x 4 columns, y 4 rows x 3 columns
      const float* Cx = wk + 48;
      const float* Cy = wk + 60;
      float Wn[2 * RPW][4];
#pragma unroll
      for (int q = 0; q < 2 * RPW; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) Wn[q][c] = g0[q * HXT + c];
#pragma unroll
      for (int m = 0; m < RPW; ++m) {
        float v = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) v = fmaf(Cx[4 * r + c], Wn[m + 1 + r][c], v);
        fx[m] = v;
      }
#pragma unroll
      for (int m = 0; m <= RPW; ++m) {
        float v = 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) v = fmaf(Cy[3 * r + c], Wn[m + r][1 + c], v);
        fy[m] = v;
      }
      if (lane < RPW) {
        const float* ge = g + (RPW * warp + lane + 1) * HXT + TXT;
        float v = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) v = fmaf(Cx[4 * r + c], ge[r * HXT + c], v);
        ext = v;
      }
    }
    const unsigned wbits = wall_tile ? wbits_s[threadIdx.x] : 0u;
    if (wall_tile && !((wbits >> 15) & 1u)) {
      // the walls pass's values (fluid side, or diffuse scattering)
      const float* rb = R + RB;
#pragma unroll
      for (int m = 0; m < RPW; ++m)
        if ((wbits >> m) & 1u) fx[m] = rb[(wbits >> 16) + m];
      if ((wbits >> 14) & 1u) ext = rb[TYT + RPW * warp + lane];
#pragma unroll
      for (int m = 0; m <= RPW; ++m)
        if ((wbits >> (4 + m)) & 1u) fy[m] = rb[2 * TYT + ((wbits >> (9 + m)) & 1u ? TXT : 0) + lane];
    } else if (wall_tile) {
      // the walls pass's values; bounce-back mirrors for leaving velocities
      const float* rc = R + RC;                             // (c_k, shift_k) per side
      auto wv = [&](int t, int side, bool leaving) {
        float v = R[RB + t];
        if (leaving && p.bc_kind[side] == BC_BOUNCEBACK) v = fmaf(rwb[t], rc[2 * side], v + rc[2 * side + 1]);
        return v;
      };
#pragma unroll
      for (int m = 0; m < RPW; ++m) {
        const int j = jr + m;
        if (!p.px && j < p.ny) {
          if (i == 0) fx[m] = wv(RPW * warp + m, SIDE_W, sgx > 0);
          else if (i == p.nx) fx[m] = wv(TYT + RPW * warp + m, SIDE_E, sgx < 0);
        }
      }
      if (!p.px && lane < RPW && i0 + TXT == p.nx && jr + lane < p.ny)
        ext = wv(TYT + RPW * warp + lane, SIDE_E, sgx < 0);
#pragma unroll
      for (int m = 0; m <= RPW; ++m) {
        const int j = jr + m;
        if (!p.py && i < p.nx) {
          if (j == 0) fy[m] = wv(2 * TYT + lane, SIDE_S, sgy > 0);
          else if (j == p.ny) fy[m] = wv(2 * TYT + TXT + lane, SIDE_N, sgy < 0);
        }
      }
    }

    const float4 k4 = *reinterpret_cast<const float4*>(R + RV + 4);
    const float kx = STAGE == 1 ? k4.x : k4.z, ky = STAGE == 1 ? k4.y : k4.w;
    float cw[RPW];                                          // the cells' cubics at xi
    {
      const unsigned long long xx = pack2(e4.x, e4.x), yy = pack2(e4.y, e4.y);
#pragma unroll
      for (int q = 0; q < RPW / 2; ++q) unpack2(cubic2(SP[q], xx, yy), cw[2 * q], cw[2 * q + 1]);
    }
#pragma unroll
    for (int m = 0; m < RPW; ++m) {
      float fE = __shfl_down_sync(0xffffffffu, fx[m], 1);
      const float fEx = __shfl_sync(0xffffffffu, ext, m);
      if (lane == 31) fE = fEx;
      if (!ok[m]) continue;
      const float df = fmaf(kx, fE - fx[m], ky * (fy[m + 1] - fy[m]));
      const float ws = fmaf(e4.z, cw[m], df);
      float out;
      const float o = ownv[m];
      if (STAGE == 1) out = fmaf(-cB, o, o + ws);                                    // cB = sP
      else out = fmaf(cA, fownv[m] - o, fmaf(-cB, o, o + ws));                     // cB = sP + sQ
      stv(dst + (size_t)k * N + cell[m], out);
    }
  };

  if constexpr (ASYNC) {
    for (int kp = k0; kp < k1; kp += PAIR) {
      const int np = min(PAIR, k1 - kp);
      cp_wait<AHEAD - PAIR>();                                // this thread's copies of the pair
      float own[PAIR][RPW], fown[PAIR][RPW];
#pragma unroll
      for (int h = 0; h < PAIR; ++h) {
        if (h >= np) break;
        const int k = kp + h;
        float* g = ring[(k - k0) & (NRING - 1)] + RG;
        // the velocity row is another thread's copy: read after the barrier,
        // except xi and W for the conversion, which come from the table
        const float4 e4 = ld4(vq + p.nv + k);
#pragma unroll
        for (int m = 0; m < EPT; ++m)
          if (sact[m]) {
            const float r = g[sidx[m]];
            if (m < RPW) own[h][m] = r;
            const float4 q4 = prm4[sidx[m]];
            const float E = fmaf(e4.x, q4.y, e4.y * q4.z);
            const float fe = e4.z * (fmaf(q4.w * E, E, E) + q4.x);
            g[sidx[m]] = fmaf(b, fe - r, r);
          }
      }
      __syncthreads();
      // the ring buffers of the previous pair are free once every thread is here
#pragma unroll
      for (int h = 0; h < PAIR; ++h) {
        const int kq = kp + AHEAD + h;
        const int ks = ksrc[h];
        ksrc[h] = wall_src(kq + PAIR);
        issue(kq, (kq - k0) & (NRING - 1), ks);
      }
      if (wx || wy) {
#pragma unroll
        for (int h = 0; h < PAIR; ++h)
          if (h < np) stage_ghosts(p, ring[(kp + h - k0) & (NRING - 1)] + RG, i0, j0, wx, wy);
        __syncthreads();
      }
#pragma unroll
      for (int h = 0; h < PAIR; ++h) {
        if (h >= np) break;
        const int k = kp + h;
        const float* R = ring[(k - k0) & (NRING - 1)];
#pragma unroll
        for (int m = 0; m < RPW; ++m) fown[h][m] = STAGE == 2 ? R[RF + (RPW * warp + m) * TXT + lane] : 0.f;
        plane_out(k, R, ld4(vq + p.nv + k), own[h], fown[h]);
      }
    }
  } else {
    for (int k = k0; k < k1; ++k) {
      float* R = ring[(k - k0) & (NRING - 1)];
      float* g = R + RG;
      cp_wait<NRING - 2>();                                   // this thread's copies of velocity k
      // the velocity row is another thread's copy: read after the barrier,
      // except xi and W for the conversion, which come from the table
      const float4 e4 = ld4(vq + p.nv + k);
      float own[RPW], fown[RPW];
#pragma unroll
      for (int m = 0; m < EPT; ++m)
        if (sact[m]) {
          const float r = tof(raw[m]);
          if (m < RPW) own[m] = r;
          const float4 q4 = prm4[sidx[m]];
          const float E = fmaf(e4.x, q4.y, e4.y * q4.z);
          const float fe = e4.z * (fmaf(q4.w * E, E, E) + q4.x);
          g[sidx[m]] = fmaf(b, fe - r, r);
        }
#pragma unroll
      for (int m = 0; m < RPW; ++m) fown[m] = (STAGE == 2 && ok[m]) ? lds(fh + (size_t)k * N + cell[m]) : 0.f;
      if (k + 1 < k1) {
#pragma unroll
        for (int m = 0; m < EPT; ++m)
          if (sact[m]) raw[m] = ldr(src + (size_t)(k + 1) * N + soff[m]);
      }
      __syncthreads();
      // the ring buffer of velocity k - 1 is free once every thread is here
      {
        const int kq = k + AHEAD;
        const int ks = ksrc[0];
        ksrc[0] = wall_src(kq + 1);
        issue(kq, (kq - k0) & (NRING - 1), ks);
      }
      if (wx || wy) {
        stage_ghosts(p, g, i0, j0, wx, wy);
        __syncthreads();
      }
      plane_out(k, R, e4, own, fown);
    }
  }
}

template <typename T, int STAGE, bool TIES>
__global__ void __launch_bounds__(UNT, 4)
k_gnc_update(GncStep s, float cA, float cB, float sP, float sQ, float sF) {
  gnc_update_body<T, STAGE, TIES>(s, cA, cB, sP, sQ, sF, blockIdx.x);
}


// ------------------------------------------------------------ batched
// The same kernels over many instances in one launch: the instances'
// descriptors in device memory, and per kernel the prefix sum of their
// blocks; a block finds its instance, copies the descriptor into shared
// memory and runs the instance's block of the same body, so each instance
// computes exactly what its own launch would.
__device__ __forceinline__ int batch_item(const int* __restrict__ start, int n, int b) {
  int lo = 0, hi = n;                      // start[lo] <= b < start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int batch_enter(GncStep& ss, const GncStep* __restrict__ steps,
                                           const int* __restrict__ start, int n) {
  const int i = batch_item(start, n, blockIdx.x);
  const int* a = reinterpret_cast<const int*>(steps + i);
  int* d = reinterpret_cast<int*>(&ss);
  for (int t = threadIdx.x; t < (int)(sizeof(GncStep) / 4); t += blockDim.x) d[t] = __ldg(a + t);
  __syncthreads();
  return blockIdx.x - __ldg(start + i);
}

template <typename T>
__global__ void __launch_bounds__(SCB, 3)
k_gnc_sums_b(const GncStep* steps, const int* start, int n, int stage) {
  __shared__ GncStep ss;
  const int l = batch_enter(ss, steps, start, n);
  const int gx = (ss.p.N + SCB - 1) / SCB, gy = ss.ncls;
  gnc_sums_body<T>(ss, stage, l % gx, (l / gx) % gy, l / (gx * gy));
}
__global__ void __launch_bounds__(CFC * NCMB_MAX)
k_gnc_cellfin_b(const GncStep* steps, const int* start, int n, int stage) {
  __shared__ GncStep ss;
  const int l = batch_enter(ss, steps, start, n);
  gnc_cellfin_body(ss, stage, l);
}
__global__ void __launch_bounds__(64)
k_gnc_facefin_b(const GncStep* steps, const int* start, int n, int stage) {
  __shared__ GncStep ss;
  const int l = batch_enter(ss, steps, start, n);
  gnc_facefin_body(ss, stage, l);
}
template <typename T>
__global__ void __launch_bounds__(128)
k_gnc_walls_b(const GncStep* steps, const int* start, int n, int stage) {
  __shared__ GncStep ss;
  const int l = batch_enter(ss, steps, start, n);
  int nseg = 0;
  if (!ss.p.px) nseg += 2 * wall_segments(ss.p.ny);
  if (!ss.p.py) nseg += 2 * wall_segments(ss.p.nx);
  gnc_walls_body<T>(ss, stage, l % nseg, l / nseg);
}
template <typename T, int STAGE, bool TIES>
__global__ void __launch_bounds__(UNT, 4)
k_gnc_update_b(const GncStep* steps, const int* start, int n, const float* coef) {
  __shared__ GncStep ss;
  const int l = batch_enter(ss, steps, start, n);
  const float* c = coef + (batch_item(start, n, blockIdx.x) * 2 + (STAGE - 1)) * 5;
  gnc_update_body<T, STAGE, TIES>(ss, __ldg(c), __ldg(c + 1), __ldg(c + 2), __ldg(c + 3), __ldg(c + 4), l);
}

template <typename T>
cudaError_t allow_gnc() {
  cudaError_t e = cudaSuccess;
  // the update: the smallest shared-memory carveout that keeps four blocks
  // per SM, so the rest of the unified memory serves as L1 for its copies
  // and loads (at 128^2 x 4096 the stage updates ran 2-5 % faster than with
  // all of it shared)
  int dev = 0, smem_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  for (void* f : {(void*)k_gnc_update<T, 1, false>, (void*)k_gnc_update<T, 2, false>,
                  (void*)k_gnc_update<T, 1, true>, (void*)k_gnc_update<T, 2, true>,
                  (void*)k_gnc_update_b<T, 1, false>, (void*)k_gnc_update_b<T, 2, false>,
                  (void*)k_gnc_update_b<T, 1, true>, (void*)k_gnc_update_b<T, 2, true>}) {
    cudaFuncAttributes a{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, f);
    if (e != cudaSuccess) break;
    const long need = 4L * ((long)a.sharedSizeBytes + 1024);
    const int carve = smem_sm > 0 ? (int)std::min(100L, (need * 100 + smem_sm - 1) / smem_sm) : 100;
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
  }
  // the streamed sums (BF16) hold their ring in shared memory; the FP32
  // sums keep the default split, whose L1 takes their loads in flight (a
  // full shared-memory carveout slowed them from 77 to 87 us)
  if (sums_streamed<T>())
    for (void* f : {(void*)k_gnc_sums<T>, (void*)k_gnc_sums_b<T>}) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sums_smem<T>());
      cudaFuncAttributes a{};
      if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, f);
      if (e != cudaSuccess) break;
      const long need = 3L * ((long)a.sharedSizeBytes + (long)sums_smem<T>() + 1024);   // three blocks
      const int carve = smem_sm > 0 ? (int)std::min(100L, (need * 100 + smem_sm - 1) / smem_sm) : 100;
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
    }
  return e;
}

int items(const GncStep& s) { return s.tiles_x * s.tiles_y * s.nch; }

// polynomial in (x, y) of degree <= 3 as coefficients of the ten monomials
struct Poly {
  double c[NMONO] = {};
};

}  // namespace

bool gnc_tables(GncStep& g, const double* xi_x, const double* xi_y, const double* w,
                const double* feq_wall, const int* opp, GncTables& t) {
  const DevParams& p = g.p;
  const int nv = p.nv;
  const double rho0 = g.ref.rho0;
  auto sgn = [](double v) { return v > 0.0 ? 1 : (v < 0.0 ? -1 : 0); };
  auto mono = [&](int k, int idx) {
    static const int ex[NMONO][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1},
                                     {0, 2}, {3, 0}, {2, 1}, {1, 2}, {0, 3}};
    double v = 1.0;
    for (int q = 0; q < ex[idx][0]; ++q) v *= xi_x[k];
    for (int q = 0; q < ex[idx][1]; ++q) v *= xi_y[k];
    return v;
  };
  // sign classes, in the order (sx, sy) = (-1,-1), (-1,0), ... (1,1)
  g.ncls = 0;
  t.cls_off.assign(1, 0);
  t.cls_k.clear();
  t.cls_mono.clear();
  int cls_sx[9], cls_sy[9];
  for (int sx = -1; sx <= 1; ++sx)
    for (int sy = -1; sy <= 1; ++sy) {
      int n = 0;
      for (int k = 0; k < nv; ++k)
        if (sgn(xi_x[k]) == sx && sgn(xi_y[k]) == sy) {
          t.cls_k.push_back(k);
          for (int q = 0; q < 12; ++q) t.cls_mono.push_back(q < NMONO ? (float)mono(k, q) : 0.f);
          ++n;
        }
      if (n) {
        cls_sx[g.ncls] = sx;
        cls_sy[g.ncls] = sy;
        ++g.ncls;
        t.cls_off.push_back((int)t.cls_k.size());
      }
    }
  // class combinations: interior faces (ties with weight 1/2, Q4), and per
  // wall the fluid side (ties with weight 1) and the strictly incoming
  // velocities (for the bounce-back mirror)
  g.ncombo = 0;
  auto combo = [&](double a0, double b0, auto lam_of) {
    GncCombo C{};
    C.a0 = (float)a0;
    C.b0 = (float)b0;
    for (int c = 0; c < 9; ++c) C.lam[c] = c < g.ncls ? (float)lam_of(cls_sx[c], cls_sy[c]) : 0.f;
    for (int q = 0; q < g.ncombo; ++q) {
      const GncCombo& D = g.cmb[q];
      bool same = D.a0 == C.a0 && D.b0 == C.b0;
      for (int c = 0; c < 9 && same; ++c) same = D.lam[c] == C.lam[c];
      if (same) return q;
    }
    g.cmb[g.ncombo] = C;
    return g.ncombo++;
  };
  auto half = [](int s, int want) { return s == want ? 1.0 : (s == 0 ? 0.5 : 0.0); };
  g.c_lo[0] = combo(0.5, 0.0, [&](int sx, int) { return half(sx, 1); });
  g.c_up[0] = combo(-0.5, 0.0, [&](int sx, int) { return half(sx, -1); });
  g.c_lo[1] = combo(0.0, 0.5, [&](int, int sy) { return half(sy, 1); });
  g.c_up[1] = combo(0.0, -0.5, [&](int, int sy) { return half(sy, -1); });
  for (int sd = 0; sd < 4; ++sd) g.c_wf[sd] = g.c_win[sd] = 0;
  if (!p.px) {
    g.c_wf[SIDE_W] = combo(-0.5, 0.0, [](int sx, int) { return sx <= 0 ? 1.0 : 0.0; });
    g.c_win[SIDE_W] = combo(-0.5, 0.0, [](int sx, int) { return sx < 0 ? 1.0 : 0.0; });
    g.c_wf[SIDE_E] = combo(0.5, 0.0, [](int sx, int) { return sx >= 0 ? 1.0 : 0.0; });
    g.c_win[SIDE_E] = combo(0.5, 0.0, [](int sx, int) { return sx > 0 ? 1.0 : 0.0; });
  }
  if (!p.py) {
    g.c_wf[SIDE_S] = combo(0.0, -0.5, [](int, int sy) { return sy <= 0 ? 1.0 : 0.0; });
    g.c_win[SIDE_S] = combo(0.0, -0.5, [](int, int sy) { return sy < 0 ? 1.0 : 0.0; });
    g.c_wf[SIDE_N] = combo(0.0, 0.5, [](int, int sy) { return sy >= 0 ? 1.0 : 0.0; });
    g.c_win[SIDE_N] = combo(0.0, 0.5, [](int, int sy) { return sy > 0 ? 1.0 : 0.0; });
  }
  // equilibrium quadrature per combination: zc[p][q] = sum lam W_k pi_p pi_q
  t.zc.assign((size_t)g.ncombo * NMONO * 6, 0.f);
  for (int cb = 0; cb < g.ncombo; ++cb)
    for (int pp = 0; pp < NMONO; ++pp)
      for (int q = 0; q < 6; ++q) {
        double z = 0.0;
        for (int c = 0; c < g.ncls; ++c) {
          const double lam = g.cmb[cb].lam[c];
          if (lam == 0.0) continue;
          for (int e = t.cls_off[c]; e < t.cls_off[c + 1]; ++e) {
            const int k = t.cls_k[e];
            z += lam * w[k] * mono(k, pp) * mono(k, q);
          }
        }
        t.zc[((size_t)cb * NMONO + pp) * 6 + q] = (float)z;
      }
  // T(a, b) = sum_u t_u u(a, b), u = 1, a, b, a^2, ab, b^2 (T is quadratic
  // in (a, b)): the coefficients from six evaluations, checked at a seventh
  double T00[9], Tp0[9], Tm0[9], T0p[9], T0m[9], Tpp[9], Tx[9];
  flux_ds_weights<double>(0.0, 0.0, T00);
  flux_ds_weights<double>(1.0, 0.0, Tp0);
  flux_ds_weights<double>(-1.0, 0.0, Tm0);
  flux_ds_weights<double>(0.0, 1.0, T0p);
  flux_ds_weights<double>(0.0, -1.0, T0m);
  flux_ds_weights<double>(1.0, 1.0, Tpp);
  flux_ds_weights<double>(0.3, -0.7, Tx);
  for (int q = 0; q < 9; ++q) {
    const double t1 = T00[q], ta = 0.5 * (Tp0[q] - Tm0[q]), taa = 0.5 * (Tp0[q] + Tm0[q]) - T00[q];
    const double tb = 0.5 * (T0p[q] - T0m[q]), tbb = 0.5 * (T0p[q] + T0m[q]) - T00[q];
    const double tab = Tpp[q] - t1 - ta - tb - taa - tbb;
    const double a = 0.3, bb = -0.7;
    const double chk = t1 + ta * a + tb * bb + taa * a * a + tab * a * bb + tbb * bb * bb;
    if (std::fabs(chk - Tx[q]) > 1e-12) return false;
    g.tu[0][q] = (float)t1;
    g.tu[1][q] = (float)ta;
    g.tu[2][q] = (float)tb;
    g.tu[3][q] = (float)taa;
    g.tu[4][q] = (float)tab;
    g.tu[5][q] = (float)tbb;
  }
  g.ntl = 0;
  for (int q = 0; q < 9; ++q)
    for (int u = 0; u < 6; ++u)
      if (g.tu[u][q] != 0.f) {
        g.tl_s[g.ntl] = (unsigned char)q;
        g.tl_u[g.ntl] = (unsigned char)u;
        g.tl_w[g.ntl] = g.tu[u][q];
        ++g.ntl;
      }
  // wall tables: sums over the leaving velocities (xi.n < 0, n the fluid's
  // outward normal) of pi_m times the bounce-back coefficient, the
  // deviation shift, the wall equilibrium and the reference state
  for (int sd = 0; sd < 4; ++sd) {
    for (int m = 0; m < 3; ++m) g.wB[sd][m] = g.wH[sd][m] = g.wMo[sd][m] = g.wWo[sd][m] = 0.0;
    if (p.bc_kind[sd] == BC_PERIODIC) continue;
    const double nxs = sd == SIDE_W ? -1.0 : sd == SIDE_E ? 1.0 : 0.0;
    const double nys = sd == SIDE_S ? -1.0 : sd == SIDE_N ? 1.0 : 0.0;
    for (int k = 0; k < nv; ++k) {
      const double xn = xi_x[k] * nxs + xi_y[k] * nys;
      if (!(xn < 0.0)) continue;
      const double pm[3] = {1.0, xi_x[k], xi_y[k]};
      const double ck = 2.0 * w[k] * (xi_x[k] * p.uw_x[sd] + xi_y[k] * p.uw_y[sd]) * p.inv_RT;
      const double sh = opp[k] >= 0 ? (w[opp[k]] - w[k]) * rho0 : 0.0;
      for (int m = 0; m < 3; ++m) {
        g.wB[sd][m] += pm[m] * ck;
        g.wH[sd][m] += pm[m] * sh;
        g.wMo[sd][m] += pm[m] * feq_wall[(size_t)sd * nv + k];
        g.wWo[sd][m] += pm[m] * w[k] * rho0;
      }
    }
  }
  // per velocity and side: bounce-back's c_k = 2 W_k xi_k.u_w / RT and
  // shift_k = (W_opp(k) - W_k) rho0 ([nv][4] pairs, FP32), and the velocity
  // whose wall-face entry the update reads (the mirror for a velocity
  // leaving a bounce-back wall)
  t.wbb.assign((size_t)nv * 8, 0.f);
  t.wsrc.assign(4 * (size_t)nv, 0);
  for (int sd = 0; sd < 4; ++sd) {
    const double nxs = sd == SIDE_W ? -1.0 : sd == SIDE_E ? 1.0 : 0.0;
    const double nys = sd == SIDE_S ? -1.0 : sd == SIDE_N ? 1.0 : 0.0;
    for (int k = 0; k < nv; ++k) {
      const bool leaving = xi_x[k] * nxs + xi_y[k] * nys < 0.0;
      const bool bb = p.bc_kind[sd] == BC_BOUNCEBACK;
      t.wsrc[(size_t)sd * nv + k] = (bb && leaving && opp[k] >= 0) ? opp[k] : k;
      if (!bb) continue;
      const double ck = 2.0 * w[k] * (xi_x[k] * p.uw_x[sd] + xi_y[k] * p.uw_y[sd]) * p.inv_RT;
      const double sh = opp[k] >= 0 ? (w[opp[k]] - w[k]) * rho0 : 0.0;
      t.wbb[8 * (size_t)k + 2 * sd] = (float)ck;
      t.wbb[8 * (size_t)k + 2 * sd + 1] = (float)sh;
    }
  }
  g.nw = 2 * (p.nx + p.ny);
  // face weights of eq. flux_DS per stage and velocity: four sets of 12 (x
  // about the lower / upper cell, y likewise; nine used), then the
  // 12-point x- and y-stencils with the upwind choice built in (a tie
  // velocity, Q4: half of each side)
  g.ties = 0;
  for (int k = 0; k < nv; ++k)
    if (xi_x[k] == 0.0 || xi_y[k] == 0.0) g.ties = 1;
  t.fwt.assign(2 * (size_t)nv * WPV, 0.f);
  for (int st = 0; st < 2; ++st) {
    const double h = st == 0 ? g.s1.h : g.s2.h;
    for (int k = 0; k < nv; ++k) {
      const double ax = -xi_x[k] * h * p.inv_dx, by = -xi_y[k] * h * p.inv_dy;
      const double ab[4][2] = {{0.5 + ax, by}, {-0.5 + ax, by}, {ax, 0.5 + by}, {ax, -0.5 + by}};
      double wv[4][9];
      float* row = t.fwt.data() + ((size_t)st * nv + k) * WPV;
      for (int set = 0; set < 4; ++set) {
        flux_ds_weights<double>(ab[set][0], ab[set][1], wv[set]);
        for (int q = 0; q < 9; ++q) row[set * 12 + q] = (float)wv[set][q];
      }
      const double lx = xi_x[k] > 0.0 ? 1.0 : xi_x[k] < 0.0 ? 0.0 : 0.5;   // weight of the lower side
      const double ly = xi_y[k] > 0.0 ? 1.0 : xi_y[k] < 0.0 ? 0.0 : 0.5;
      double cx[3][4] = {}, cy[4][3] = {};
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          cx[r][c] += lx * wv[0][3 * r + c];
          cx[r][c + 1] += (1.0 - lx) * wv[1][3 * r + c];
          cy[r][c] += ly * wv[2][3 * r + c];
          cy[r + 1][c] += (1.0 - ly) * wv[3][3 * r + c];
        }
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) row[48 + 4 * r + c] = (float)cx[r][c];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 3; ++c) row[60 + 3 * r + c] = (float)cy[r][c];
    }
  }
  g.tiles_x = (p.nx + TXT - 1) / TXT;
  g.tiles_y = (p.ny + TYT - 1) / TYT;
  return true;
}

// velocity splits of the class sums: at most SMAXE velocities per split,
// and about four blocks per SM where the classes have 64 velocities per
// split to spare
int gnc_splits(const GncStep& g, const GncTables& t, int sms) {
  int smallest = g.p.nv, largest = 1;
  for (int c = 0; c < g.ncls; ++c) {
    const int n = t.cls_off[c + 1] - t.cls_off[c];
    smallest = std::min(smallest, n);
    largest = std::max(largest, n);
  }
  const int need = (largest + SMAXE - 1) / SMAXE;
  const int blocks = ((g.p.N + SCB - 1) / SCB) * g.ncls;
  const int want = std::min((4 * sms + blocks - 1) / blocks, std::max(1, smallest / 64));
  return std::max(need, want);
}

// velocity chunks per tile: about one wave of update blocks
int gnc_chunks(const GncStep& g, int sms) {
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_gnc_update<float, 2, false>, UNT, 0) != cudaSuccess ||
      bps < 1) {
    cudaGetLastError();
    bps = 3;
  }
  const int tiles = g.tiles_x * g.tiles_y;
  const int want = std::max(1, (bps * sms) / tiles);
  return std::max(1, std::min(g.p.nv, want));
}

cudaError_t gnc_prepare(int store) {
  if (store == 1) return allow_gnc<float>();
  if (store == 2) return allow_gnc<__nv_bfloat16>();
  return cudaErrorInvalidValue;
}

// class sums of the stage's source, then the cell finaliser
cudaError_t launch_gnc_sums(const GncStep& s, int stage, cudaStream_t st) {
  const dim3 grid((s.p.N + SCB - 1) / SCB, s.ncls, s.nsplit);
  if (s.store == 1) k_gnc_sums<float><<<grid, SCB, sums_smem<float>(), st>>>(s, stage);
  else k_gnc_sums<__nv_bfloat16><<<grid, SCB, sums_smem<__nv_bfloat16>(), st>>>(s, stage);
  return cudaGetLastError();
}

cudaError_t launch_gnc_cellfin(const GncStep& s, int stage, cudaStream_t st) {
  k_gnc_cellfin<<<(s.p.N + CFC - 1) / CFC, CFC * s.ncombo, 0, st>>>(s, stage);
  return cudaGetLastError();
}

cudaError_t launch_gnc_facefin(const GncStep& s, int stage, cudaStream_t st) {
  const int nf = s.p.ny * (s.p.nx + 1) + (s.p.ny + 1) * s.p.nx;
  k_gnc_facefin<<<(nf + 63) / 64, 64, 0, st>>>(s, stage);
  return cudaGetLastError();
}

cudaError_t launch_gnc_walls(const GncStep& s, int stage, cudaStream_t st) {
  const int nseg = (s.p.px ? 0 : 2 * ((s.p.ny + WSEG - 1) / WSEG)) +
                   (s.p.py ? 0 : 2 * ((s.p.nx + WSEG - 1) / WSEG));
  if (nseg == 0) return cudaSuccess;
  const dim3 grid(nseg, (s.p.nv + WCH - 1) / WCH);
  if (s.store == 1) k_gnc_walls<float><<<grid, 128, 0, st>>>(s, stage);
  else k_gnc_walls<__nv_bfloat16><<<grid, 128, 0, st>>>(s, stage);
  return cudaGetLastError();
}

// the update's coefficients of stage `stage`: cA, cB, sP, sQ, sF (see the
// update's comment; cB, the coefficient subtracted from the base, sP or
// sP + sQ, is formed from the values the kernel puts into S, in FP32)
void update_coefs(const GncStep& s, int stage, float (&o)[5]) {
  const double a1 = s.s1.a, b1 = s.s1.b, dt = s.p.dt;
  const double c34 = 0.75 * s.c_om;
  float cA = 0.f, cB, sP, sQ = 0.f, sF;
  if (stage == 1) {
    sP = (float)(1.25 * b1);
    sF = (float)(-(dt / 3.0) * s.s1.beta);
    cB = sP;
  } else {
    cA = (float)(4.0 / 7.0 - 6.0 / 7.0 * a1);
    sP = (float)(-6.0 / 7.0 * b1);
    sQ = (float)(-c34);
    sF = (float)(-(4.0 * dt / 7.0) * s.s2.beta);
    cB = sP + sQ;
  }
  o[0] = cA;
  o[1] = cB;
  o[2] = sP;
  o[3] = sQ;
  o[4] = sF;
}

cudaError_t launch_gnc_update(const GncStep& s, int stage, cudaStream_t st) {
  float cf[5];
  update_coefs(s, stage, cf);
  const float cA = cf[0], cB = cf[1], sP = cf[2], sQ = cf[3], sF = cf[4];
  const int n = items(s);
#define GNC_UPD(T, ST, TI) k_gnc_update<T, ST, TI><<<n, UNT, 0, st>>>(s, cA, cB, sP, sQ, sF)
  if (s.store == 1) {
    if (s.ties) { if (stage == 1) GNC_UPD(float, 1, true); else GNC_UPD(float, 2, true); }
    else { if (stage == 1) GNC_UPD(float, 1, false); else GNC_UPD(float, 2, false); }
  } else {
    if (s.ties) { if (stage == 1) GNC_UPD(__nv_bfloat16, 1, true); else GNC_UPD(__nv_bfloat16, 2, true); }
    else { if (stage == 1) GNC_UPD(__nv_bfloat16, 1, false); else GNC_UPD(__nv_bfloat16, 2, false); }
  }
#undef GNC_UPD
  return cudaGetLastError();
}


// ------------------------------------------------------------ batched
namespace {
// blocks of each kernel for one instance: sums, cellfin, facefin, walls, update
void batch_blocks(const GncStep& s, int (&nb)[5]) {
  const DevParams& p = s.p;
  nb[0] = ((p.N + SCB - 1) / SCB) * s.ncls * s.nsplit;
  nb[1] = (p.N + CFC - 1) / CFC;
  nb[2] = (p.ny * (p.nx + 1) + (p.ny + 1) * p.nx + 63) / 64;
  const int nseg = (p.px ? 0 : 2 * ((p.ny + WSEG - 1) / WSEG)) + (p.py ? 0 : 2 * ((p.nx + WSEG - 1) / WSEG));
  nb[3] = nseg * ((p.nv + WCH - 1) / WCH);
  nb[4] = items(s);
}
}  // namespace

cudaError_t gnc_batch_init(const GncStep* const* steps, int n, GncBatch& b) {
  gnc_batch_free(b);
  if (n < 1) return cudaErrorInvalidValue;
  b.n = n;
  b.ncombo_max = 1;
  b.store = steps[0]->store;
  b.ties = steps[0]->ties;
  std::vector<GncStep> host(n);
  std::vector<int> start(5 * (size_t)(n + 1), 0);
  std::vector<float> coef(10 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    if (steps[i]->store != b.store || steps[i]->ties != b.ties) return cudaErrorInvalidValue;
    host[i] = *steps[i];
    b.ncombo_max = std::max(b.ncombo_max, host[i].ncombo);
    int nb[5];
    batch_blocks(host[i], nb);
    for (int k = 0; k < 5; ++k) start[k * (size_t)(n + 1) + i + 1] = start[k * (size_t)(n + 1) + i] + nb[k];
    for (int st = 1; st <= 2; ++st) {
      float cf[5];
      update_coefs(host[i], st, cf);
      for (int q = 0; q < 5; ++q) coef[(size_t)(2 * i + st - 1) * 5 + q] = cf[q];
    }
  }
  for (int k = 0; k < 5; ++k) b.total[k] = start[k * (size_t)(n + 1) + n];
  cudaError_t e = cudaMalloc((void**)&b.steps, host.size() * sizeof(GncStep));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b.start, start.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b.coef, coef.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(b.steps, host.data(), host.size() * sizeof(GncStep), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b.start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b.coef, coef.data(), coef.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) gnc_batch_free(b);
  return e;
}

void gnc_batch_free(GncBatch& b) {
  if (b.steps) cudaFree(b.steps);
  if (b.start) cudaFree(b.start);
  if (b.coef) cudaFree(b.coef);
  b.steps = nullptr;
  b.start = nullptr;
  b.coef = nullptr;
  b.n = 0;
}

// One stage of every instance: five launches, each over all instances.
cudaError_t launch_gnc_batch_stage(const GncBatch& b, int stage, cudaStream_t st) {
  const int n = b.n;
  const int* s0 = b.start;
  auto at = [&](int k) { return s0 + (size_t)k * (n + 1); };
  cudaError_t e = cudaSuccess;
  const bool f32 = b.store == 1;
  if (b.total[0]) {
    if (f32) k_gnc_sums_b<float><<<b.total[0], SCB, sums_smem<float>(), st>>>(b.steps, at(0), n, stage);
    else k_gnc_sums_b<__nv_bfloat16><<<b.total[0], SCB, sums_smem<__nv_bfloat16>(), st>>>(b.steps, at(0), n, stage);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && b.total[1]) {
    k_gnc_cellfin_b<<<b.total[1], CFC * b.ncombo_max, 0, st>>>(b.steps, at(1), n, stage);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && b.total[2]) {
    k_gnc_facefin_b<<<b.total[2], 64, 0, st>>>(b.steps, at(2), n, stage);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && b.total[3]) {
    if (f32) k_gnc_walls_b<float><<<b.total[3], 128, 0, st>>>(b.steps, at(3), n, stage);
    else k_gnc_walls_b<__nv_bfloat16><<<b.total[3], 128, 0, st>>>(b.steps, at(3), n, stage);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && b.total[4]) {
#define GNC_UPB(T, ST, TI) k_gnc_update_b<T, ST, TI><<<b.total[4], UNT, 0, st>>>(b.steps, at(4), n, b.coef)
    if (f32) {
      if (b.ties) { if (stage == 1) GNC_UPB(float, 1, true); else GNC_UPB(float, 2, true); }
      else { if (stage == 1) GNC_UPB(float, 1, false); else GNC_UPB(float, 2, false); }
    } else {
      if (b.ties) { if (stage == 1) GNC_UPB(__nv_bfloat16, 1, true); else GNC_UPB(__nv_bfloat16, 2, true); }
      else { if (stage == 1) GNC_UPB(__nv_bfloat16, 1, false); else GNC_UPB(__nv_bfloat16, 2, false); }
    }
#undef GNC_UPB
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace dugks
