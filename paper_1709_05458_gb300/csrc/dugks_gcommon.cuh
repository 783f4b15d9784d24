// Shared device helpers of the generic (any velocity set) kernels: storage
// and compute types of the three storage forms, loads and stores,
// compensated FP32 moment accumulators, the equilibrium's assembly
// parameters and its polynomial forms, block sums.  Included by
// dugks_generic_mixed.cu and dugks_gnc.cu (each translation unit keeps its
// own copy; everything here is inline device code).
#pragma once
#include <cuda_bf16.h>

#include "dugks_fp.cuh"
#include "dugks_internal.cuh"

namespace dugks {
namespace {

// ------------------------------------------------------------ precision
struct __align__(16) D4 {
  double x, y, z, w;
};
template <typename T> struct Prec {            // FP32 and BF16 storage
  using C = float;
  using V4 = float4;
  static constexpr int KH = 8;                  // loads in flight per batch in the updates
};
template <> struct Prec<double> {
  using C = double;
  using V4 = D4;
  static constexpr int KH = 4;
};

__device__ __forceinline__ float4 ld4(const float4* p) { return __ldg(p); }
__device__ __forceinline__ D4 ld4(const D4* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return D4{a.x, a.y, b.x, b.y};
}

// raw loads (no conversion), so a batch of loads is issued before the
// first value is used; tof converts afterwards
template <typename T> __device__ __forceinline__ T ldr(const T* p) { return __ldg(p); }
__device__ __forceinline__ float tof(float v) { return v; }
__device__ __forceinline__ float tof(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double tof(double v) { return v; }
template <typename T> __device__ __forceinline__ auto ldv(const T* p) { return tof(__ldg(p)); }
template <typename T> __device__ __forceinline__ auto lds(const T* p) { return tof(*p); }
__device__ __forceinline__ void stv(float* p, float v) { *p = v; }
__device__ __forceinline__ void stv(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void stv(double* p, double v) { *p = v; }

__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }

// FP64 -> C (FP32 on the integer pipe) and C -> FP64
template <typename C> __device__ __forceinline__ C to_c(double x);
template <> __device__ __forceinline__ float to_c<float>(double x) { return d2f_bits(x); }
template <> __device__ __forceinline__ double to_c<double>(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return f2d_bits(x); }

// asynchronous 16-byte global -> shared copy (bypassing L1) and its groups
__device__ __forceinline__ void cp16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
// asynchronous 4-byte global -> shared copy (through L1)
__device__ __forceinline__ void cp4(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
// wait until at most N of this thread's most recent copy groups are pending
template <int N> __device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- moment accumulators ----
// FP32: compensated pair s = hi + lo (error-free transformations).  add:
// TwoSum(hi, x), the rounding error goes to lo; addprod: x (ah + al) with
// ah x split exactly into p + pe by an FMA.  The _rn intrinsics keep the
// compiler from contracting or reassociating.  FP64: a plain sum (al = 0).
template <typename C> struct Acc;
template <> struct Acc<float> {
  float hi, lo;
};
template <> struct Acc<double> {
  double s;
};
__device__ __forceinline__ void acc_add(Acc<float>& a, float x) {
  const float s = __fadd_rn(a.hi, x);
  const float bp = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, e);
}
__device__ __forceinline__ void acc_addprod(Acc<float>& a, float ah, float al, float x) {
  const float p = __fmul_rn(ah, x);
  const float pe = __fmaf_rn(ah, x, -p);
  const float s = __fadd_rn(a.hi, p);
  const float bp = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, __fadd_rn(e, __fmaf_rn(al, x, pe)));
}
__device__ __forceinline__ double acc_value(const Acc<float>& a) {
  return to_d(a.hi) + to_d(a.lo);
}
// a += b and a += (xh + xl) b for an accumulated pair b
__device__ __forceinline__ void acc_add_acc(Acc<float>& a, const Acc<float>& b) {
  acc_add(a, b.hi);
  a.lo = __fadd_rn(a.lo, b.lo);
}
__device__ __forceinline__ void acc_addprod_acc(Acc<float>& a, float xh, float xl,
                                                const Acc<float>& b) {
  acc_addprod(a, xh, xl, b.hi);
  a.lo = __fmaf_rn(xh, b.lo, a.lo);
}
__device__ __forceinline__ void acc_add(Acc<double>& a, double x) { a.s += x; }
__device__ __forceinline__ void acc_addprod(Acc<double>& a, double ah, double, double x) {
  a.s = fma(ah, x, a.s);
}
__device__ __forceinline__ double acc_value(const Acc<double>& a) { return a.s; }
__device__ __forceinline__ void acc_add_acc(Acc<double>& a, const Acc<double>& b) { a.s += b.s; }
__device__ __forceinline__ void acc_addprod_acc(Acc<double>& a, double xh, double,
                                                const Acc<double>& b) {
  a.s = fma(xh, b.s, a.s);
}

// Kahan-compensated FP32 sum (Kahan 1965): s is the running sum, c the
// negated low-order part lost by the last addition.  Four operations per
// term; a product x xi is rounded once before it is added (relative 2^-24,
// the level of the FP32 values it weighs).  The value is s - c in FP64.
struct Kah {
  float s, c;
};
__device__ __forceinline__ void kah_add(Kah& a, float x) {
  const float y = __fsub_rn(x, a.c);
  const float t = __fadd_rn(a.s, y);
  a.c = __fsub_rn(__fsub_rn(t, a.s), y);
  a.s = t;
}
__device__ __forceinline__ double kah_value(const Kah& a) { return to_d(a.s) - to_d(a.c); }

// ---- equilibrium ----
// assembly parameters of one cell or face
template <typename C> struct EqF {
  C vx, vy, bm1, r, dr;          // u/RT, -|u|^2/(2RT), rho, rho - rho0
};
template <typename C>
__device__ __forceinline__ EqF<C> eq_params_u(double rho, double ux, double uy, double inv_RT,
                                              double rho0) {
  const double vx = ux * inv_RT, vy = uy * inv_RT;
  EqF<C> q;
  q.vx = to_c<C>(vx);
  q.vy = to_c<C>(vy);
  q.bm1 = to_c<C>(-0.5 * fma(ux, vx, uy * vy));
  q.r = to_c<C>(rho);
  q.dr = to_c<C>(rho - rho0);
  return q;
}
// from the sums (rho, jx, jy): one FP64 reciprocal
template <typename C>
__device__ __forceinline__ EqF<C> eq_params_j(double rho, double jx, double jy, double inv_RT,
                                              double rho0) {
  const double rinv = 1.0 / rho;
  return eq_params_u<C>(rho, jx * rinv, jy * rinv, inv_RT, rho0);
}
// W_k (rho P_k - rho0) = W_k ((rho - rho0) + rho (P_k - 1)),
// P_k - 1 = e (1 + e/2) - |u|^2/(2RT), e = xi_k.u/RT
template <typename C>
__device__ __forceinline__ C feq_dev(const EqF<C>& q, C cx, C cy, C w) {
  const C e = fmx(cx, q.vx, cy * q.vy);
  const C p1 = fmx(e, fmx(C(0.5), e, C(1)), q.bm1);
  return w * fmx(q.r, p1, q.dr);
}
template <typename C>
__device__ __forceinline__ void store_par(C* __restrict__ fp, int n, int i, const EqF<C>& q) {
  fp[i] = q.vx;
  fp[n + i] = q.vy;
  fp[2 * n + i] = q.bm1;
  fp[3 * n + i] = q.r;
  fp[4 * n + i] = q.dr;
}

// Equilibrium of a cell or face as a quadratic in xi from its assembly
// parameters: W_k P(xi_k) = W_k (rho P_k - rho0) (the equilibrium itself
// when rho0 = 0), P(xi) = c0 + cx x + cy y + cxx x^2 + cxy x y + cyy y^2.
template <typename C> struct Quad {
  C c0, cx, cy, cxx, cxy, cyy;
};
template <typename C>
__device__ __forceinline__ Quad<C> quad(const C* __restrict__ fp, int n, int i) {
  const C vx = __ldg(fp + i), vy = __ldg(fp + n + i), bm1 = __ldg(fp + 2 * n + i);
  const C r = __ldg(fp + 3 * n + i), dr = __ldg(fp + 4 * n + i);
  Quad<C> o;
  o.c0 = fmx(r, bm1, dr);
  o.cx = r * vx;
  o.cy = r * vy;
  o.cxx = C(0.5) * o.cx * vx;
  o.cxy = o.cx * vy;
  o.cyy = C(0.5) * o.cy * vy;
  return o;
}

// Sum M values over the threads of a block (warp shuffles, then the warps'
// totals in a fixed order); every thread gets the totals.  sm: [32][M].
template <int M>
__device__ __forceinline__ void block_sum(double (&v)[M], double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[m] += __shfl_xor_sync(0xffffffffu, v[m], o);
  if (lane == 0)
#pragma unroll
    for (int m = 0; m < M; ++m) sm[warp * M + m] = v[m];
  __syncthreads();
#pragma unroll
  for (int m = 0; m < M; ++m) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sm[w * M + m];
    v[m] = s;
  }
  __syncthreads();
}


// ---- cubic polynomials in xi ----
// Every equilibrium entering an update is W_k P(xi_k) with P quadratic; their
// combination with the flux factors is W_k S(xi_k) with S a cubic in
// (xi_x, xi_y): coefficients of 1, x, y, xx, xy, yy, xxx, xxy, xyy, yyy.
template <typename C> struct Cubic {           // 1, x, y, xx, xy, yy, xxx, xxy, xyy, yyy
  C c[10];
};
template <typename C>
__device__ __forceinline__ C cubic(const Cubic<C>& S, C x, C y) {
  const C t1 = fmx(x, S.c[6], fmx(y, S.c[7], S.c[3]));
  const C t2 = fmx(y, S.c[8], S.c[4]);
  const C t3 = fmx(y, S.c[9], S.c[5]);
  const C X = fmx(x, t1, fmx(y, t2, S.c[1]));
  const C Y = fmx(y, t3, S.c[2]);
  return fmx(x, X, fmx(y, Y, S.c[0]));
}
// On a tensor velocity grid whose 16 consecutive velocities share xi_x
// (GDevStep::tgrid): the cubic at fixed x as a cubic in y, b0 + y (b1 +
// y (b2 + y b3)), formed once per thread.
template <typename C> struct CubicY {
  C b0, b1, b2, b3;
};
template <typename C>
__device__ __forceinline__ CubicY<C> cubic_at_x(const Cubic<C>& S, C x) {
  CubicY<C> o;
  o.b0 = fmx(x, fmx(x, fmx(x, S.c[6], S.c[3]), S.c[1]), S.c[0]);
  o.b1 = fmx(x, fmx(x, S.c[7], S.c[4]), S.c[2]);
  o.b2 = fmx(x, S.c[8], S.c[5]);
  o.b3 = S.c[9];
  return o;
}
template <typename C>
__device__ __forceinline__ C cubic_y(const CubicY<C>& B, C y) {
  return fmx(y, fmx(y, fmx(y, B.b3, B.b2), B.b1), B.b0);
}

}  // namespace
}  // namespace dugks
