// Tensor-core (tcgen05) periodic 3x3x3 convolution of the learned
// starting-field network; see conv_tc.cu.
#pragma once
#include <cuda_runtime.h>

namespace wslda {

struct ConvTcArgs {
  int nx, ny, nz;    // periodic lattice, site index (ix * ny + iy) * nz + iz
  int cin, cout;     // channels of this convolution (1..32 each)
  const float* x;    // [batch][cin][M] input, rounded to bfloat16 as it is staged
  const float* w;    // weights (float copies of bfloat16 values), layout below
  int transposed;    // 0: w[co][ci][27], offset d; 1: w[ci][co][27] read at 26 - d (input gradient)
  const float* bias; // [cout] or NULL
  int epi;           // 0: none, 1: tanh, 2: times (1 - aux^2)
  const float* aux;  // [batch][cout][M] for epi 2
  float* y;          // [batch][cout][M]
  int* err;          // bit 3 set if an MMA completion wait timed out (may be NULL)
};

// y[b][co][r] = bias[co] + sum_d sum_ci W_d[co][ci] bf16(x[b][ci][r + off(d)]),
// off(d) = (d / 9 - 1, (d / 3) % 3 - 1, d % 3 - 1), float32 accumulation.
cudaError_t launch_conv_tc(const ConvTcArgs& a, int batch, cudaStream_t s);

struct WgradTcArgs {
  int nx, ny, nz;
  int cin, cout, batch;  // layer channels (1..32 each) and samples
  const float* x;        // [batch][cin][M] layer input, rounded to bfloat16 as it is staged
  const float* g;        // [batch][cout][M] gradient of the layer output (pre-activation), rounded likewise
  float* part;           // scratch: max_split x 896 x 32 floats
  int max_split;         // largest number of site ranges (split-K) the scratch holds
  int rows, ksplit;      // set by the launcher
  float* gW;             // [cout][cin][27] result
  int* err;              // bit 3 set if an MMA completion wait timed out (may be NULL)
};

// gW[co][ci][d] = sum_b sum_r bf16(g[b][co][r]) bf16(x[b][ci][r + off(d)]),
// float32 accumulation: split-K tensor-core GEMM, then a fixed-order sum of
// the splits.
cudaError_t launch_conv_wgrad_tc(const WgradTcArgs& a, cudaStream_t s);

}  // namespace wslda
