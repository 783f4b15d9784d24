// Floating-point helpers shared by the kernel files.
//
// GB300 runs FP64 arithmetic and every FP64 <-> FP32 conversion instruction
// on its FP64 pipe, 2 lanes per SM per clock.  The conversions below use
// integer operations instead, and the reciprocal replaces the FP64 division
// sequence by an FP32 seed and one FP64 correction step.
#pragma once

#include <cuda_runtime.h>

namespace dugks {

// Exact FP32 -> FP64.  Zero and FP32 denormals map to 0, inf / NaN stay
// inf / NaN.
__device__ __forceinline__ double f2d_bits(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned em = b & 0x7fffffffu;
  unsigned hi = (em >> 3) + 0x38000000u;          // exponent rebias 127 -> 1023
  unsigned lo = em << 29;
  hi = (em >= 0x7f800000u) ? (0x7ff00000u | ((em & 0x7fffffu) >> 3)) : hi;
  const bool tiny = em < 0x00800000u;
  hi = tiny ? 0u : hi;
  lo = tiny ? 0u : lo;
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)lo);
}

// FP64 -> FP32, rounding half away from zero on the magnitude, for values in
// the FP32 normal range; values below it map to 0, NaN, inf and values
// beyond the FP32 range to NaN (so that a broken state stays visible).
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int E = (int)((hi >> 20) & 0x7ffu) - 896;
  unsigned mag = ((unsigned)E << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  mag += (lo >> 28) & 1u;
  mag = (E <= 0) ? 0u : mag;
  mag = (E >= 255) ? 0x7fc00000u : mag;
  return __uint_as_float(mag | (hi & 0x80000000u));
}

// 1/x for x in the FP32 normal range: FP32 seed (rcp.approx, integer-pipe
// conversions) and two FP64 Newton steps, error ~2^-92 before rounding.
__device__ __forceinline__ double rcp64(double x) {
  float sf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(sf) : "f"(d2f_bits(x)));
  double r = f2d_bits(sf);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// 1/x with three FP64 instructions for |x| in [2^-100, 2^100]: the FP32 seed
// r (relative error e0 <= 2^-22) corrected once by r (1 + e + e^2),
// e = 1 - x r, whose error is e0^3 <= 2^-66 before the final rounding, so the
// result is within one unit in the last place of 1/x.  Other magnitudes
// (never met by a stable state) take the FP64 division.
__device__ __forceinline__ double rcp_fast(double x) {
  const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
  if (ex < 1023u - 100u || ex > 1023u + 100u) return 1.0 / x;
  float sf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(sf) : "f"(d2f_bits(x)));
  const double r = f2d_bits(sf);
  const double e = fma(-x, r, 1.0);
  return fma(fma(e, e, e), r, r);
}

}  // namespace dugks
