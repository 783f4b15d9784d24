// Double-word arithmetic: a value is the unevaluated sum h + l of two FP32
// numbers with |l| <= ulp(h)/2 (a 48-bit significand, unit roundoff
// u^2 = 2^-48 with u = 2^-24).  GB300 issues FP32 work at 64 times its FP64
// rate, so a double-word operation of 8-15 FP32 instructions outruns one
// FP64 instruction several times over.
//
// The operations are built from the error-free transformations
//   2Sum(a, b):     s = fl(a + b), t = (a + b) - s exactly (Knuth);
//   Fast2Sum(a, b): the same for |a| >= |b| (Dekker), three operations;
//   2Prod(a, b):    p = fl(a b), e = fma(a, b, -p) = a b - p exactly;
// in the forms analysed by Joldes, Muller and Popescu (ACM TOMS 44, 2017).
// Addition is the "sloppy" form: its error is at most a few u^2 (|x| + |y|)
// (a normwise bound, the same kind FP64 summation of the step's terms has),
// not relative to |x + y| under cancellation.  Products carry a relative
// error of a few u^2.
#pragma once

#include <cuda_runtime.h>

#include "dugks_fp.cuh"
#include "dugks_internal.cuh"   // struct dw

namespace dugks {

// the double / float overloads stay visible next to fma(dw, dw, dw)
using ::fma;

__device__ __forceinline__ dw dw_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float ap = __fsub_rn(s, b);
  const float bp = __fsub_rn(s, ap);
  return dw{s, __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp))};
}
__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dw{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dw operator-(dw x) { return dw{-x.h, -x.l}; }
__device__ __forceinline__ dw operator+(dw x, dw y) {
  const dw s = dw_two_sum(x.h, y.h);
  return dw_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }
__device__ __forceinline__ dw operator*(dw x, dw y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, e));
  return dw_fast_two_sum(p, e);
}
// x y + z with one normalisation
__device__ __forceinline__ dw fma(dw x, dw y, dw z) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, e));
  const dw s = dw_two_sum(p, z.h);
  return dw_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(z.l, e)));
}

// 1/x: the correctly rounded FP32 reciprocal r0 and one Newton step,
// r = r0 + r0 (1 - x r0); x r0 is formed exactly enough that the residual
// is within u^2 and the result within a few u^2 of 1/x.
__device__ __forceinline__ dw dw_rcp(dw x) {
  const float r0 = __frcp_rn(x.h);
  const float p = __fmul_rn(x.h, r0);
  const float pe = __fmaf_rn(x.h, r0, -p);                 // x.h r0 = p + pe
  // e = 1 - x r0 = (1 - p) - pe - x.l r0; 1 - p is exact (p within 2^-23 of 1)
  const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), pe), __fmul_rn(x.l, r0));
  return dw_fast_two_sum(r0, __fmul_rn(r0, e));
}

// double -> double-word: h = x rounded to FP32 on the integer pipe, l = the
// FP32 rounding of the exact residual x - h (one FP64 subtraction, exact by
// Sterbenz's lemma).  NaN / inf / out-of-range x give a NaN h (dugks_check
// then reports the state).
__device__ __forceinline__ dw dw_from_d(double x) {
  const float h = d2f_bits(x);
  return dw{h, d2f_bits(x - f2d_bits(h))};
}
// double-word -> double: h + l rounded once in FP64
__device__ __forceinline__ double dw_to_d(dw x) { return f2d_bits(x.h) + f2d_bits(x.l); }

// Dot-product accumulator: the sum of the exact products' high parts is
// carried as a 2Sum pair, the rounding residues and cross terms in one FP32
// word; one normalisation at the end.
struct dw_acc {
  float s, c;
};
__device__ __forceinline__ void dw_acc_first(dw_acc& a, dw w, dw v) {
  const float p = __fmul_rn(w.h, v.h);
  a.s = p;
  a.c = __fmaf_rn(w.h, v.l, __fmaf_rn(w.l, v.h, __fmaf_rn(w.h, v.h, -p)));
}
__device__ __forceinline__ void dw_acc_add(dw_acc& a, dw w, dw v) {
  const float p = __fmul_rn(w.h, v.h);
  const float e = __fmaf_rn(w.h, v.l, __fmaf_rn(w.l, v.h, __fmaf_rn(w.h, v.h, -p)));
  const dw s = dw_two_sum(a.s, p);
  a.s = s.h;
  a.c = __fadd_rn(a.c, __fadd_rn(s.l, e));
}
__device__ __forceinline__ dw dw_acc_value(const dw_acc& a) { return dw_fast_two_sum(a.s, a.c); }

}  // namespace dugks
