// FP64 fused multiply-add throughput of the current device: the denominator
// of the roofline of the plain FP64 step, whose stage kernels are bound by the
// double-precision ALUs rather than by HBM. A microbenchmark of the hardware,
// not a step of the method.
//
// Every thread runs 8 independent FMA chains (enough independent work to keep
// the FP64 pipes busy at any latency), the grid covers every SM several times,
// and the result is folded into a store that never happens for these inputs
// (it keeps the chains live without touching memory in the timed loop).
#include <cuda_runtime.h>

#include "../../include/wslda_td.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fp64_fma_chains(double* sink, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * double(threadIdx.x + c);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  double t = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) t += x[c];
  if (t == -1.0) sink[blockIdx.x] = t;  // never true for a in (0, 1), b > 0
}

// The same with additions: the FP64 butterflies of the transforms are mostly
// unfused additions and multiplications, each one operation per instruction.
__global__ void __launch_bounds__(256) fp64_add_chains(double* sink, int iters, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * double(threadIdx.x + c);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = x[c] + b;
    }
  }
  double t = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) t += x[c];
  if (t == -1.0) sink[blockIdx.x] = t;  // never true for b > 0
}

// Best time over `reps` launches (after one warm-up) of the chain kernel.
template <class K>
wslda_status time_chains(int reps, K launch, float* best_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  wslda_status st = WSLDA_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = WSLDA_ECUDA;
  float best = 1e30f;
  for (int r = 0; r <= reps && st == WSLDA_OK; ++r) {
    cudaEventRecord(e0, 0);
    launch();
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = WSLDA_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;
  }
  if (cudaGetLastError() != cudaSuccess) st = WSLDA_ECUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *best_ms = best;
  return st;
}

}  // namespace

extern "C" wslda_status wslda_measure_fp64_add_rate(int reps, double* tops) {
  if (!tops || reps < 1) return WSLDA_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return WSLDA_ECUDA;
  const int blocks = sms * 8, threads = 256, iters = 1024;
  double* sink = nullptr;
  if (cudaMalloc(&sink, size_t(blocks) * sizeof(double)) != cudaSuccess) return WSLDA_ENOMEM;
  float best = 0.f;
  const wslda_status st =
      time_chains(reps, [&] { fp64_add_chains<<<blocks, threads>>>(sink, iters, 1e-7); }, &best);
  cudaFree(sink);
  if (st != WSLDA_OK) return st;
  const double adds = double(blocks) * threads * double(iters) * 16.0 * kChains;
  *tops = adds / (double(best) * 1e-3) / 1e12;
  return WSLDA_OK;
}

extern "C" wslda_status wslda_measure_fp64_rate(int reps, double* tflops) {
  if (!tflops || reps < 1) return WSLDA_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return WSLDA_ECUDA;
  const int blocks = sms * 8, threads = 256, iters = 1024;
  double* sink = nullptr;  // never written (see the kernel); a valid pointer all the same
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  wslda_status st = WSLDA_OK;
  if (cudaMalloc(&sink, size_t(blocks) * sizeof(double)) != cudaSuccess) return WSLDA_ENOMEM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = WSLDA_ECUDA;
  float best = 1e30f;
  for (int r = 0; r <= reps && st == WSLDA_OK; ++r) {  // launch 0 warms up
    cudaEventRecord(e0, 0);
    fp64_fma_chains<<<blocks, threads>>>(sink, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = WSLDA_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;
  }
  if (cudaGetLastError() != cudaSuccess) st = WSLDA_ECUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (st != WSLDA_OK) return st;
  const double fmas = double(blocks) * threads * double(iters) * 16.0 * kChains;
  *tflops = 2.0 * fmas / (double(best) * 1e-3) / 1e12;
  return WSLDA_OK;
}
