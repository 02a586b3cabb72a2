// Density reduction for callers that cannot allocate device memory.
//
// wslda_densities_noalloc computes rho and nu of device-resident states like
// the context-based path does, but its only scratch (the per-chunk partial
// sums) lives in a fixed file-scope device array, so the call itself never
// allocates. Callers that own all device memory through their own pool
// allocator, or that run on a latency-critical path where cudaMalloc (which
// can synchronise the device and can fail) is not acceptable, can use it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/wslda_td.h"
#include "fft.cuh"

namespace {

// Capacity of the scratch array: 2^21 doubles (16 MiB), held by every GPU that
// loads the library until the process exits. One call needs 3 * M doubles per
// chunk of states, so M may be at most 699050 lattice sites.
constexpr int64_t kScratchDoubles = int64_t(1) << 21;
constexpr int kMaxChunks = 32;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Device address of the scratch array, resolved once per device. In host
// code the symbol name only stands in for the array; the kernel must be given
// this address. The cached address belongs to the device's primary context:
// after cudaDeviceReset (which ends that context and unloads the module) it is
// stale, so the entry point must not be used across a device reset.
constexpr int kMaxDevices = 64;
double* g_scratch_dev[kMaxDevices] = {};
std::mutex g_scratch_mutex;

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

// Partial sums over a chunk of states, one thread per site, in double:
// rho += w- |v|^2 + w+ |u|^2, nu += (w- - w+) u v^*. Every entry
// part[c][0..2][s] the reduction reads is written here, so the scratch left by
// an earlier call never needs clearing.
template <typename C>
__global__ void noalloc_partial(const C* __restrict__ phi, const double* __restrict__ wm,
                                const double* __restrict__ wp, int64_t n, int M, int64_t chunk, double* part) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  const int64_t n0 = int64_t(blockIdx.y) * chunk, n1 = n0 + chunk < n ? n0 + chunk : n;
  const int64_t stride = 2 * int64_t(M);
  double r = 0.0, nr = 0.0, ni = 0.0;
  for (int64_t k = n0; k < n1; ++k) {
    const C u = phi[k * stride + s], v = phi[k * stride + M + s];
    const double a = wm ? wm[k] : 1.0, b = wp ? wp[k] : 0.0, d = a - b;
    const double ux = u.x, uy = u.y, vx = v.x, vy = v.y;
    r += a * (vx * vx + vy * vy) + b * (ux * ux + uy * uy);
    nr += d * (ux * vx + uy * vy);
    ni += d * (uy * vx - ux * vy);
  }
  double* p = part + int64_t(blockIdx.y) * 3 * M;
  p[s] = r;
  p[M + s] = nr;
  p[2 * M + s] = ni;
}

__global__ void noalloc_reduce(const double* part, int nchunk, int M, double* rho, double* nu) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  double r = 0.0, nr = 0.0, ni = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    const double* p = part + int64_t(c) * 3 * M;
    r += p[s];
    nr += p[M + s];
    ni += p[2 * M + s];
  }
  rho[s] = r;
  nu[2 * s] = nr;
  nu[2 * s + 1] = ni;
}

}  // namespace

extern "C" wslda_status wslda_densities_noalloc(int precision, const void* uv, const double* w_minus,
                                                const double* w_plus, int64_t nstates, int nx, int ny, int nz,
                                                double* rho, double* nu, void* stream) {
  if ((precision != WSLDA_FP64 && precision != WSLDA_MIXED) || !rho || !nu || nstates < 0 || nx <= 0 || ny <= 0 ||
      nz <= 0 || (!uv && nstates > 0))
    return WSLDA_EINVAL;
  const int64_t M = int64_t(nx) * ny * nz;
  if (3 * M > kScratchDoubles) return WSLDA_ENOMEM;  // beyond the fixed scratch capacity
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return WSLDA_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int nchunk = int(kScratchDoubles / (3 * M));
  if (nchunk > kMaxChunks) nchunk = kMaxChunks;
  if (nchunk > nstates) nchunk = nstates > 0 ? int(nstates) : 1;
  const int64_t chunk = nstates > 0 ? (nstates + nchunk - 1) / nchunk : 1;
  const dim3 grid(unsigned((M + 255) / 256), unsigned(nchunk));
  if (nstates == 0) {
    cudaError_t e = cudaMemsetAsync(scratch, 0, size_t(3) * M * sizeof(double), s);
    if (e != cudaSuccess) return WSLDA_ECUDA;
    nchunk = 1;
  } else if (precision == WSLDA_MIXED) {
    noalloc_partial<float2><<<grid, 256, 0, s>>>(static_cast<const float2*>(uv), w_minus, w_plus, nstates, int(M),
                                                 chunk, scratch);
  } else {
    noalloc_partial<double2><<<grid, 256, 0, s>>>(static_cast<const double2*>(uv), w_minus, w_plus, nstates, int(M),
                                                  chunk, scratch);
  }
  noalloc_reduce<<<unsigned((M + 255) / 256), 256, 0, s>>>(scratch, nchunk, int(M), rho, nu);
  return cudaGetLastError() == cudaSuccess ? WSLDA_OK : WSLDA_ECUDA;
}
