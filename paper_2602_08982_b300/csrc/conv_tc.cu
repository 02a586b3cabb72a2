// Periodic 3x3x3 convolution of the learned starting-field network as an
// implicit GEMM on the fifth-generation tensor cores (tcgen05, kind::f16).
//
// One CTA of 128 threads computes a tile of 128 consecutive lattice sites of
// one sample and every output channel:
//   D[r][co] = sum_{d < 27} sum_ci A_d[r][ci] B_d[co][ci],
//   A_d[r][ci] = bf16(x[b][ci][r + off(d)])   (periodic neighbour, gathered),
//   B_d[co][ci] = bf16 weights of offset d,
// with r the GEMM row (M = 128), co the column (N = channels rounded up to 16)
// and (d, ci) the reduction (K = 27 x channels rounded up to 16, 16 per MMA).
// Operands are bfloat16 in shared memory in the canonical K-major layout
// without swizzle: 8-row x 16-byte core matrices, 128 bytes each; along K the
// core matrices of one operand tile are LBO bytes apart, along M/N SBO bytes.
// The accumulator is float32 in tensor memory (lane = row, column = channel),
// read back with tcgen05.ld for the epilogue (bias and tanh, or the factor
// 1 - a^2 of the backward pass through tanh).
//
// The same kernel gives the gradient with respect to a layer's input: with
// W'[ci][co][d] = W[co][ci][26 - d] (offsets mirrored, channels transposed)
// gx[ci][r] = sum_d sum_co W'[ci][co][d] g[co][r + off(d)].
//
// Flow per CTA: nine chunks of three offsets (one (dx, dy) pair each): the
// 128 threads stage the chunk's weights and gather and round
// their row of each A tile, one thread issues the chunk's MMAs and commits
// them to an mbarrier, and the next chunk waits on it before reusing the A
// and B buffers. Every wait is bounded; on a timeout bit 3 of the error word is set
// and the kernel still waits (bounded) for its MMAs, frees its tensor memory
// and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "conv_tc.cuh"

namespace wslda {
namespace {

constexpr int kRows = 128;          // GEMM rows (sites) per CTA
constexpr int kThreads = 256;       // forward kernel: two threads gather each row
constexpr int kChunk = 3;           // offsets per A buffer fill (one dx, dy pair: dz = -1, 0, 1)
constexpr unsigned kCore = 128;     // bytes per 8 x 16-byte core matrix
constexpr unsigned kTmemCols = 32;  // accumulator columns (N <= 32)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of a K-major tile without swizzle:
// start address, leading (K-direction) and stride (M/N-direction) byte
// offsets between core matrices, each encoded in 16-byte units; bit 46 is the
// descriptor version of this architecture; base offset, offset mode and
// swizzle mode are zero.
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  uint64_t d = uint64_t((addr >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

// Instruction descriptor of kind::f16: float32 accumulator (bits 4-5 = 1),
// A and B bfloat16 (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0),
// N / 8 at bits 17-22, M / 16 at bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(int n, int m) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init1(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes to shared memory become visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         int accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive float32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
  const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
  return a | (b << 16);
}

}  // namespace

namespace {

// Bounded wait (about two seconds of SM clock) for completion `parity` of the
// MMA barrier; false on a timeout.
__device__ __forceinline__ bool mma_wait(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > (4LL << 30)) return false;
  return true;
}

template <int CINP, int NP>
__global__ void __launch_bounds__(kThreads) conv_tc_kernel(const ConvTcArgs a) {
  constexpr int KG = CINP / 8;                          // 16-byte channel groups (core matrices along K)
  constexpr unsigned B_D = unsigned(KG) * (NP / 8) * kCore;      // bytes of one offset's weight tile
  constexpr unsigned B_KG = unsigned(NP / 8) * kCore;            // K-direction core stride in B
  constexpr unsigned A_KG = unsigned(kRows / 8) * kCore;         // K-direction core stride in A (2048)
  constexpr unsigned A_D = unsigned(KG) * A_KG;                  // bytes of one offset's A tile
  constexpr unsigned B_BYTES = kChunk * B_D, A_BYTES = kChunk * A_D;
  constexpr uint32_t IDESC = instr_desc(NP, kRows);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* Bs = smem;
  unsigned char* As = smem + B_BYTES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(As + A_BYTES);
  uint64_t* barp = reinterpret_cast<uint64_t*>(As + A_BYTES + 8);
  const unsigned bar = smem_u32(barp);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid % kRows, part = tid / kRows;  // row of the tile and which half of its gathers
  const int M = a.nx * a.ny * a.nz;
  const int b = blockIdx.y;
  const int s = blockIdx.x * kRows + row;  // this thread's row (site)

  if (tid == 0) {
    mbar_init1(bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  int ix = 0, iy = 0, iz = 0;
  if (s < M) {
    iz = s % a.nz;
    iy = (s / a.nz) % a.ny;
    ix = s / (a.ny * a.nz);
  }
  const float* xb = a.x + size_t(b) * a.cin * M;
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const unsigned tmem = *tslot;
  bool ok = true;
  constexpr int NCH = 27 / kChunk;
  for (int c = 0; c < NCH; ++c) {
    if (c > 0) {  // the previous chunk's MMAs have read the A buffer
      ok = mma_wait(bar, unsigned(c - 1) & 1u) && ok;
      fence_after_sync();
    }
    // the chunk's weights: 16-byte rows of 8 channels, zero past cin / cout
    for (int q = tid; q < kChunk * KG * NP; q += kThreads) {
      const int dl = q / (KG * NP), rem = q % (KG * NP), g = rem / NP, n = rem % NP;
      const int d = c * kChunk + dl;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = 8 * g + j;
        float w = 0.f;
        if (n < a.cout && k < a.cin)
          w = a.transposed ? a.w[(size_t(k) * a.cout + n) * 27 + (26 - d)] : a.w[(size_t(n) * a.cin + k) * 27 + d];
        v[j] = w;
      }
      uint4 pk = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                            pack_bf16(v[6], v[7]));
      *reinterpret_cast<uint4*>(Bs + dl * B_D + g * B_KG + (n >> 3) * kCore + (n & 7) * 16) = pk;
    }
    // this thread's half of its row of the A tiles of offsets d = 3c + dl:
    // dx = c / 3 - 1, dy = c % 3 - 1, dz = dl - 1; (offset, channel group)
    // pairs alternate between the row's two threads
#pragma unroll
    for (int dl = 0; dl < kChunk; ++dl) {
      const int q = s < M ? (wrapi(ix + c / 3 - 1, a.nx) * a.ny + wrapi(iy + c % 3 - 1, a.ny)) * a.nz +
                                wrapi(iz + dl - 1, a.nz)
                          : 0;
#pragma unroll
      for (int g = 0; g < KG; ++g) {
        if (((dl * KG + g) & 1) != part) continue;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = 8 * g + j;
          v[j] = (s < M && k < a.cin) ? xb[size_t(k) * M + q] : 0.f;
        }
        uint4 pk = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                              pack_bf16(v[6], v[7]));
        *reinterpret_cast<uint4*>(As + dl * A_D + g * A_KG + (row >> 3) * kCore + (row & 7) * 16) = pk;
      }
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const unsigned a0 = smem_u32(As), b0 = smem_u32(Bs);
      for (int dl = 0; dl < kChunk; ++dl) {
#pragma unroll
        for (int kb = 0; kb < CINP / 16; ++kb) {
          const uint64_t ad = smem_desc(a0 + dl * A_D + 2 * kb * A_KG, A_KG, kCore);
          const uint64_t bd = smem_desc(b0 + dl * B_D + 2 * kb * B_KG, B_KG, kCore);
          mma_bf16(tmem, ad, bd, IDESC, (c | dl | kb) != 0);
        }
      }
      mma_commit(bar);
    }
  }
  ok = mma_wait(bar, unsigned(NCH - 1) & 1u) && ok;  // the last chunk's completion
  if (!ok) {
    if (a.err) atomicOr(a.err, 8);
    mma_wait(bar, unsigned(NCH - 1) & 1u);
  }
  fence_after_sync();
  // epilogue (warps 0-3): lane = row of this warp's quarter of the accumulator
  if (warp < kRows / 32) {
  float v[NP];
  const unsigned taddr = tmem + (unsigned(32 * warp) << 16);
  tmem_ld16(taddr, v);
  if constexpr (NP == 32) tmem_ld16(taddr + 16, v + 16);
  (void)lane;
  if (s < M) {
    float* yb = a.y + size_t(b) * a.cout * M;
    const float* xa = a.aux ? a.aux + size_t(b) * a.cout * M : nullptr;
#pragma unroll
    for (int n = 0; n < NP; ++n) {
      if (n < a.cout) {
        float r = v[n] + (a.bias ? a.bias[n] : 0.f);
        if (a.epi == 1) r = tanhf(r);
        else if (a.epi == 2) {
          const float t = xa[size_t(n) * M + s];
          r *= 1.f - t * t;
        }
        yb[size_t(n) * M + s] = r;
      }
    }
  }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

template <int CINP, int NP>
cudaError_t launch_tc(const ConvTcArgs& a, int batch, cudaStream_t s) {
  // operands, tensor-memory slot and barrier, alignment slack
  constexpr size_t bytes = kChunk * size_t(CINP / 8) * (NP / 8) * kCore + kChunk * size_t(CINP / 8) * (kRows / 8) * kCore +
                           16 + 1024;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<CINP, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(bytes));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int M = a.nx * a.ny * a.nz;
  dim3 grid(unsigned((M + kRows - 1) / kRows), unsigned(batch));
  conv_tc_kernel<CINP, NP><<<grid, kThreads, bytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

namespace {

constexpr int kKc = 64;  // reduction (site) chunk of the weight-gradient GEMM

// Weight gradient as a split-K implicit GEMM on the tensor cores:
//   D[(d, ci)][co] = sum over sites k of bf16(x[ci][k + off(d)]) bf16(g[co][k]),
// rows (d, ci) in 128-row tiles (blockIdx.x), the batch's sites split into
// `nsplit` ranges (blockIdx.y), 64 sites per MMA round. Each CTA writes its
// float32 partial tile to part[split][row][co]; wgrad_reduce sums the splits
// in a fixed order.
template <int CINP, int NP>
__global__ void __launch_bounds__(kRows) wgrad_tc_kernel(const WgradTcArgs a) {
  constexpr unsigned A_KG = unsigned(kRows / 8) * kCore;   // K-direction core stride in A (2048)
  constexpr unsigned B_KG = unsigned(NP / 8) * kCore;      // K-direction core stride in B
  constexpr unsigned A_BYTES = (kKc / 8) * A_KG, B_BYTES = (kKc / 8) * B_KG;
  constexpr uint32_t IDESC = instr_desc(NP, kRows);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* As = smem;
  unsigned char* Bs = smem + A_BYTES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(Bs + B_BYTES);
  const unsigned bar = smem_u32(Bs + B_BYTES + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int M = a.nx * a.ny * a.nz;
  const int64_t K = int64_t(a.batch) * M;
  const int64_t k_lo = int64_t(blockIdx.y) * a.ksplit;
  const int64_t k_hi = k_lo + a.ksplit < K ? k_lo + a.ksplit : K;
  if (tid == 0) {
    mbar_init1(bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const unsigned tmem = *tslot;
  // thread -> (site of the chunk, half of the rows)
  const int kk = tid & (kKc - 1), half = tid / kKc;
  bool ok = true;
  int round = 0;
  for (int64_t k0 = k_lo; k0 < k_hi; k0 += kKc, ++round) {
    if (round > 0) {
      ok = mma_wait(bar, unsigned(round - 1) & 1u) && ok;
      fence_after_sync();
    }
    const int64_t k = k0 + kk;
    const bool live = k < k_hi;
    int b = 0, r = 0, ix = 0, iy = 0, iz = 0;
    if (live) {
      b = int(k / M);
      r = int(k % M);
      iz = r % a.nz;
      iy = (r / a.nz) % a.ny;
      ix = r / (a.ny * a.nz);
    }
    const unsigned koff = unsigned(kk & 7) * 2;  // byte of this site within its 16-byte core row
    // A: rows (d, ci) of this tile, this thread's site, 64 of the 128 rows
    for (int m = half * 64; m < half * 64 + 64; ++m) {
      const int row = blockIdx.x * kRows + m, d = row / CINP, ci = row % CINP;
      float v = 0.f;
      if (live && d < 27 && ci < a.cin) {
        const int q = (wrapi(ix + d / 9 - 1, a.nx) * a.ny + wrapi(iy + (d / 3) % 3 - 1, a.ny)) * a.nz +
                      wrapi(iz + d % 3 - 1, a.nz);
        v = a.x[(size_t(b) * a.cin + ci) * M + q];
      }
      *reinterpret_cast<__nv_bfloat16*>(As + (kk >> 3) * A_KG + (m >> 3) * kCore + (m & 7) * 16 + koff) =
          __float2bfloat16_rn(v);
    }
    // B: the output-gradient rows co, this thread's site
    for (int n = half; n < NP; n += 2) {
      float v = 0.f;
      if (live && n < a.cout) v = a.g[(size_t(b) * a.cout + n) * M + r];
      *reinterpret_cast<__nv_bfloat16*>(Bs + (kk >> 3) * B_KG + (n >> 3) * kCore + (n & 7) * 16 + koff) =
          __float2bfloat16_rn(v);
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const unsigned a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
      for (int kb = 0; kb < kKc / 16; ++kb)
        mma_bf16(tmem, smem_desc(a0 + 2 * kb * A_KG, A_KG, kCore), smem_desc(b0 + 2 * kb * B_KG, B_KG, kCore), IDESC,
                 (round | kb) != 0);
      mma_commit(bar);
    }
  }
  if (round > 0) {
    ok = mma_wait(bar, unsigned(round - 1) & 1u) && ok;
    if (!ok) {
      if (a.err && tid == 0) atomicOr(a.err, 8);
      mma_wait(bar, unsigned(round - 1) & 1u);
    }
  }
  fence_after_sync();
  float v[NP];
  const unsigned taddr = tmem + (unsigned(32 * warp) << 16);
  tmem_ld16(taddr, v);
  if constexpr (NP == 32) tmem_ld16(taddr + 16, v + 16);
  const int row = blockIdx.x * kRows + tid;
  float* dst = a.part + (size_t(blockIdx.y) * a.rows + row) * NP;
#pragma unroll
  for (int n = 0; n < NP; ++n) dst[n] = round > 0 ? v[n] : 0.f;
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// gW[co][ci][d] = sum over splits (ascending) of part[split][d * CINP + ci][co]
__global__ void wgrad_reduce(const float* __restrict__ part, int nsplit, int rows, int np, int cinp, int cin, int cout,
                             float* __restrict__ gW) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cout * cin * 27) return;
  const int co = i / (cin * 27), ci = (i / 27) % cin, d = i % 27;
  const int row = d * cinp + ci;
  float acc = 0.f;
  for (int sp = 0; sp < nsplit; ++sp) acc += part[(size_t(sp) * rows + row) * np + co];
  gW[i] = acc;
}

template <int CINP, int NP>
cudaError_t launch_wgrad(WgradTcArgs a, cudaStream_t s) {
  constexpr size_t bytes = (kKc / 8) * size_t(kRows / 8) * kCore + (kKc / 8) * size_t(NP / 8) * kCore + 16 + 1024;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel<CINP, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(bytes));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int tiles = (27 * CINP + kRows - 1) / kRows;
  a.rows = tiles * kRows;
  const int64_t K = int64_t(a.batch) * a.nx * a.ny * a.nz;
  // splits so that the grid covers about two CTAs per SM, each a whole number of 64-site chunks
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int nsplit = (2 * sms + tiles - 1) / tiles;
  if (nsplit > a.max_split) nsplit = a.max_split;
  int64_t ks = (K + nsplit - 1) / nsplit;
  ks = (ks + kKc - 1) / kKc * kKc;
  nsplit = int((K + ks - 1) / ks);
  a.ksplit = ks;
  wgrad_tc_kernel<CINP, NP><<<dim3(unsigned(tiles), unsigned(nsplit)), kRows, bytes, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n = a.cout * a.cin * 27;
  wgrad_reduce<<<unsigned((n + 255) / 256), 256, 0, s>>>(a.part, nsplit, a.rows, NP, CINP, a.cin, a.cout, a.gW);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_conv_wgrad_tc(const WgradTcArgs& a, cudaStream_t s) {
  if (a.cin < 1 || a.cin > 32 || a.cout < 1 || a.cout > 32 || a.batch < 1 || a.max_split < 1)
    return cudaErrorInvalidValue;
  const bool k32 = a.cin > 16, n32 = a.cout > 16;
  if (k32 && n32) return launch_wgrad<32, 32>(a, s);
  if (k32) return launch_wgrad<32, 16>(a, s);
  if (n32) return launch_wgrad<16, 32>(a, s);
  return launch_wgrad<16, 16>(a, s);
}

cudaError_t launch_conv_tc(const ConvTcArgs& a, int batch, cudaStream_t s) {
  if (a.cin < 1 || a.cin > 32 || a.cout < 1 || a.cout > 32 || batch < 1) return cudaErrorInvalidValue;
  const bool k32 = a.cin > 16, n32 = a.cout > 16;
  if (k32 && n32) return launch_tc<32, 32>(a, batch, s);
  if (k32) return launch_tc<32, 16>(a, batch, s);
  if (n32) return launch_tc<16, 32>(a, batch, s);
  return launch_tc<16, 16>(a, batch, s);
}

}  // namespace wslda
