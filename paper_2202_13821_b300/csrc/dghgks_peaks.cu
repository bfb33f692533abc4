// dghgks_pipe_rates: measured throughput of the arithmetic the flux kernels
// issue, for the roofline of an ALU-bound residual.
//
// The residual kernels are bound by instruction issue, not by HBM: their
// roofline is the FP32 (or FP64) fused multiply-add rate of the GPU, and the
// divisions, reciprocal square roots, exponentials and erfc of the flux take
// pipe time of their own.  Each loop below runs, on every SM, enough warps
// to fill the pipes, with eight independent dependency chains per thread,
// and is timed with CUDA events:
//   FFMA, DFMA: a = a * b + c on 8 accumulators (2 FLOP per operation);
//   the FP32 flux functions fdiv, frsqrt, fexp (the approximate PTX
//   instructions the FP32 flux uses) and erfcf, each fed by its own previous
//   result through one FP32 add (x <- f(x + c), kept in a bounded range).
// The rates are operations per second over the whole GPU; the caller samples
// the SM clock meanwhile.  This is measurement infrastructure: the paper has
// no counterpart.
#include <cuda_runtime.h>

#include "dghgks.h"
#include "gks_point.cuh"

using namespace dghgks;

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) k_ffma(int iters, float b, float c, float* sink) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
  float s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 1234.5f) sink[blockIdx.x] = s;  // never true for the inputs used; keeps the loop alive
}

__global__ void __launch_bounds__(kThreads) k_dfma(int iters, double b, double c, double* sink) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (double)(threadIdx.x + j);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  double s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 1234.5) sink[blockIdx.x] = s;
}

// OP: 0 fdiv(1, x + c), 1 frsqrt(x + c), 2 fexp(-(x + c)), 3 erfcf(x + c); x stays in (0, 1.2]
template <int OP>
__device__ __forceinline__ float op_step(float x, float c) {
  const float y = x + c;
  if constexpr (OP == 0) return fdiv(1.0f, y);
  else if constexpr (OP == 1) return frsqrt(y);
  else if constexpr (OP == 2) return fexp(-y);
  else return erfcf(y);
}

template <int OP>
__global__ void __launch_bounds__(kThreads) k_sfu(int iters, float c, float* sink) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 0.1f * (float)((threadIdx.x + j) % 8);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = op_step<OP>(a[j], c);
  float s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 1234.5f) sink[blockIdx.x] = s;
}

// milliseconds of `launch` (best of three after one warm-up)
template <class F>
cudaError_t time_ms(F launch, float* best) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  *best = 1e30f;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < *best) *best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" int dghgks_pipe_rates(double* out, int n_out) {
  if (!out || n_out < DGHGKS_NRATES) return DGHGKS_EARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DGHGKS_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return DGHGKS_ECUDA;
  void* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * 64 * 1024) != cudaSuccess) return DGHGKS_ENOMEM;
  const int blocks = sms * 8;  // 8 CTAs of 8 warps per SM: 64 warps, every pipe saturated
  const double threads = (double)blocks * kThreads;
  float ms = 0;
  cudaError_t e = cudaSuccess;
  const int it_fma = 16384, it_dfma = 256, it_sfu = 1024;  // ~10-20 ms per timed launch on a B300
  e = time_ms([&] { k_ffma<<<blocks, kThreads>>>(it_fma, 0.999f, 1e-3f, static_cast<float*>(sink)); }, &ms);
  if (e == cudaSuccess) out[0] = 2.0 * threads * it_fma * 16 * kChains / (ms * 1e-3);
  if (e == cudaSuccess)
    e = time_ms([&] { k_dfma<<<blocks, kThreads>>>(it_dfma, 0.999, 1e-3, static_cast<double*>(sink)); }, &ms);
  if (e == cudaSuccess) out[1] = 2.0 * threads * it_dfma * 16 * kChains / (ms * 1e-3);
  const double sfu_ops = threads * it_sfu * 4 * kChains;
  if (e == cudaSuccess) e = time_ms([&] { k_sfu<0><<<blocks, kThreads>>>(it_sfu, 0.2f, static_cast<float*>(sink)); }, &ms);
  if (e == cudaSuccess) out[2] = sfu_ops / (ms * 1e-3);
  if (e == cudaSuccess) e = time_ms([&] { k_sfu<1><<<blocks, kThreads>>>(it_sfu, 0.2f, static_cast<float*>(sink)); }, &ms);
  if (e == cudaSuccess) out[3] = sfu_ops / (ms * 1e-3);
  if (e == cudaSuccess) e = time_ms([&] { k_sfu<2><<<blocks, kThreads>>>(it_sfu, 0.2f, static_cast<float*>(sink)); }, &ms);
  if (e == cudaSuccess) out[4] = sfu_ops / (ms * 1e-3);
  if (e == cudaSuccess) e = time_ms([&] { k_sfu<3><<<blocks, kThreads>>>(it_sfu, 0.2f, static_cast<float*>(sink)); }, &ms);
  if (e == cudaSuccess) out[5] = sfu_ops / (ms * 1e-3);
  out[6] = (double)sms;
  cudaFree(sink);
  return e == cudaSuccess ? DGHGKS_OK : DGHGKS_ECUDA;
}
