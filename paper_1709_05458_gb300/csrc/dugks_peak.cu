// Arithmetic-throughput microbenchmark: the denominator of the ALU roofline
// that the FP64 form of the step is bound by.  The paper has no counterpart;
// this is measurement support (declared in include/dugks.h).
//
// Each thread runs kChains independent fused multiply-add chains
// x <- x * m + c (m slightly below one, so the chains converge to c / (1 - m)
// and never overflow or reach subnormals) for `iters` rounds of an unrolled
// inner loop.  Enough chains and resident warps hide the pipe latency, so the
// launch time is set by the pipe's issue rate.  The final values are stored,
// which keeps the compiler from removing the work.
#include <cuda_runtime.h>

#include <string>

#include "../../include/dugks.h"
#include "dugks_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_peak_f64(double* out, int iters, double m, double c) {
  double x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_f32(double* out, int iters, float m, float c) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 1.0f + 1e-3f * (threadIdx.x + j);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// packed pairs: one fma.rn.f32x2 performs two FP32 fused multiply-adds
__global__ void __launch_bounds__(kThreads) k_peak_f32x2(double* out, int iters, float m, float c) {
  unsigned long long x[kChains];
  unsigned long long mm, cc;
  {
    float2 t = make_float2(m, m);
    mm = *reinterpret_cast<unsigned long long*>(&t);
    t = make_float2(c, c);
    cc = *reinterpret_cast<unsigned long long*>(&t);
  }
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    float2 t = make_float2(1.0f + 1e-3f * (threadIdx.x + j), 1.0f - 1e-3f * (threadIdx.x + j));
    x[j] = *reinterpret_cast<unsigned long long*>(&t);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j)
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(mm), "l"(cc));
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    float2 t = *reinterpret_cast<float2*>(&x[j]);
    s += t.x + t.y;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int dugks_alu_peak(int kind, int iters, int blocks_per_sm, double* out,
                              long long out_len, double* flops, float* ms, void* cuda_stream) {
  if (kind < 0 || kind > 2 || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 32 || !out ||
      !flops || !ms) {
    dugks::set_last_error("dugks_alu_peak: bad argument");
    return DUGKS_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    dugks::set_last_error(std::string("dugks_alu_peak: ") + cudaGetErrorString(e));
    return DUGKS_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int blocks = sms * blocks_per_sm;
  if (out_len < (long long)blocks * kThreads) {
    dugks::set_last_error("dugks_alu_peak: out needs SMs x blocks_per_sm x 256 doubles");
    return DUGKS_EINVAL;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  if (e == cudaSuccess) {
    if (kind == 0)
      k_peak_f64<<<blocks, kThreads, 0, st>>>(out, iters, 0.999999, 1e-6);
    else if (kind == 1)
      k_peak_f32<<<blocks, kThreads, 0, st>>>(out, iters, 0.9999f, 1e-4f);
    else
      k_peak_f32x2<<<blocks, kThreads, 0, st>>>(out, iters, 0.9999f, 1e-4f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) {
    dugks::set_last_error(std::string("dugks_alu_peak: ") + cudaGetErrorString(e));
    return DUGKS_ECUDA;
  }
  const double per_thread = 2.0 * kChains * kUnroll * (double)iters * (kind == 2 ? 2.0 : 1.0);
  *flops = per_thread * kThreads * (double)blocks;
  *ms = t;
  return DUGKS_OK;
}
