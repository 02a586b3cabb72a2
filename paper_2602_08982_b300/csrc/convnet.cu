// Learned starting fields for the static self-consistent solver: a stack of
// four 3x3x3 convolutions with periodic wrap-around (the lattice of Sec. 3.1
// is periodic), channels 2 -> H -> H -> H -> 2, tanh between layers, trained
// on the mean squared error with Adam (Kingma and Ba, arXiv:1412.6980).
// Inputs per site: V_ext / eF and the coupling; outputs: U / eF, Delta / eF,
// which start the iteration of Alg. 1 (Sec. 3.2).
//
// Weights are kept as a float32 master copy and used in bfloat16 (rounded to
// nearest even before every forward pass); activations, accumulation,
// gradients and the optimiser are float32. Layout: activations [B][C][M]
// (M = nx ny nz, z fastest); parameters flattened per layer as
// W[co][ci][27] (offset (dx, dy, dz) in {-1,0,1}^3 at (dx+1)*9 + (dy+1)*3 +
// (dz+1)) followed by bias[co]. A layer computes
//   y[b][co][r] = bias[co] + sum_ci sum_d W[co][ci][d] x[b][ci][r + d].
//
// Kernels: quantize (bfloat16 weight copy); the convolutions themselves run on
// the tensor cores (conv_tc.cu: implicit GEMM with bfloat16 operands and
// float32 accumulation; layer inputs are rounded to bfloat16 as they are
// staged), forward with bias and tanh fused, and the input gradient as the
// same convolution with transposed, mirrored weights times 1 - a^2 through
// tanh, and the weight gradient as a split-K GEMM over the sites with a
// fixed-order sum of the splits (layer input and output gradient rounded to
// bfloat16 likewise); bias_grad, mse
// (gradient of the loss and per-block partial sums), adam, mirror_avg
// (projection onto reflection-symmetric fields).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/wslda_td.h"
#include "conv_tc.cuh"

namespace {

constexpr int kLayers = 4;
constexpr int kIO = 2;  // input and output channels

struct Lat {
  int nx, ny, nz;
};

__global__ void quantize(const float* __restrict__ theta, float* __restrict__ wq, int64_t n, const int64_t* wb,
                         const int64_t* we) {
  // weight entries [wb[l], we[l]) of each layer are rounded; biases are copied
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool w = false;
  for (int l = 0; l < kLayers; ++l) w = w || (i >= wb[l] && i < we[l]);
  wq[i] = w ? __bfloat162float(__float2bfloat16_rn(theta[i])) : theta[i];
}

// Bias gradient: CTA per output channel.
__global__ void __launch_bounds__(256) bias_grad(int M, int cout, int batch, const float* __restrict__ g,
                                                 float* __restrict__ gb) {
  __shared__ float red[8];
  const int co = blockIdx.x;
  float acc = 0.f;
  const int64_t total = int64_t(batch) * M;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    const int b = int(t / M), s = int(t % M);
    acc += g[(int64_t(b) * cout + co) * M + s];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) v += red[i];
    gb[co] = v;
  }
}

// dL/dy = 2 (y - t) / n and per-block partial sums of (y - t)^2.
__global__ void __launch_bounds__(256) mse(const float* __restrict__ y, const float* __restrict__ t, int64_t n,
                                           float* __restrict__ g, double* __restrict__ part) {
  __shared__ double red[8];
  double acc = 0.0;
  const float scale = float(2.0 / double(n));
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float d = y[i] - t[i];
    g[i] = scale * d;
    acc += double(d) * double(d);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) v += red[i];
    part[blockIdx.x] = v;
  }
}

__global__ void adam(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                     float* __restrict__ v, int64_t n, float lr, float b1, float b2, float c1, float c2, float eps) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void mirror_avg(Lat L, int64_t nfields, const float* __restrict__ y, float* __restrict__ out) {
  const int M = L.nx * L.ny * L.nz;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= nfields * M) return;
  const int64_t f = i / M;
  const int s = int(i % M);
  const int iz = s % L.nz, iy = (s / L.nz) % L.ny, ix = s / (L.ny * L.nz);
  const float* yf = y + f * M;
  // the 8 images summed in ascending site order, so every site of an orbit
  // gets the bit-identical average
  int idx[8];
  for (int k = 0; k < 8; ++k) {
    const int jx = (k & 4) ? (L.nx - ix) % L.nx : ix;
    const int jy = (k & 2) ? (L.ny - iy) % L.ny : iy;
    const int jz = (k & 1) ? (L.nz - iz) % L.nz : iz;
    int q = (jx * L.ny + jy) * L.nz + jz, k2 = k;
    while (k2 > 0 && idx[k2 - 1] > q) {
      idx[k2] = idx[k2 - 1];
      --k2;
    }
    idx[k2] = q;
  }
  float acc = 0.f;
  for (int k = 0; k < 8; ++k) acc += yf[idx[k]];
  out[i] = 0.125f * acc;
}

}  // namespace

struct wslda_net {
  Lat L{};
  int M = 0, hidden = 0, max_batch = 0;
  int cin[kLayers] = {}, cout[kLayers] = {};
  int64_t woff[kLayers] = {}, boff[kLayers] = {}, P = 0;
  float *theta = nullptr, *wq = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  float* act[kLayers + 1] = {};  // act[0] is the caller's input (not owned)
  float *g0 = nullptr, *g1 = nullptr;
  double* part = nullptr;
  int* err_d = nullptr;  // device error word (bit 3: a tensor-core completion wait timed out)
  float* wpart = nullptr;  // split-K partial sums of the weight gradient
  int64_t *wb = nullptr, *we = nullptr;
  int64_t step = 0;
  std::vector<void*> owned;
  std::string err;
};

namespace {
constexpr int kMseBlocks = 148;
constexpr int kMaxSplit = 64;  // site ranges of the weight-gradient GEMM

wslda_status net_fail(wslda_net* n, wslda_status s, const std::string& msg) {
  if (n) n->err = msg;
  return s;
}

// Layer l forward on the tensor cores: bias, tanh except after the last layer.
cudaError_t launch_fwd(const wslda_net* n, int l, const float* x, float* y, int batch, cudaStream_t s) {
  wslda::ConvTcArgs a{};
  a.nx = n->L.nx; a.ny = n->L.ny; a.nz = n->L.nz;
  a.cin = n->cin[l]; a.cout = n->cout[l];
  a.x = x; a.w = n->wq + n->woff[l]; a.transposed = 0; a.bias = n->wq + n->boff[l];
  a.epi = l < kLayers - 1 ? 1 : 0; a.aux = nullptr; a.y = y; a.err = n->err_d;
  return wslda::launch_conv_tc(a, batch, s);
}

// Gradient with respect to the input of layer l > 0 (a tanh output): the
// convolution of g with the transposed, mirrored weights, times 1 - a^2.
cudaError_t launch_bwd_data(const wslda_net* n, int l, const float* g, float* gx, int batch, cudaStream_t s) {
  wslda::ConvTcArgs a{};
  a.nx = n->L.nx; a.ny = n->L.ny; a.nz = n->L.nz;
  a.cin = n->cout[l]; a.cout = n->cin[l];
  a.x = g; a.w = n->wq + n->woff[l]; a.transposed = 1; a.bias = nullptr;
  a.epi = 2; a.aux = n->act[l]; a.y = gx; a.err = n->err_d;
  return wslda::launch_conv_tc(a, batch, s);
}

cudaError_t forward(wslda_net* n, const float* x, int batch, float* y, cudaStream_t s) {
  cudaError_t e;
  const int64_t P = n->P;
  quantize<<<unsigned((P + 255) / 256), 256, 0, s>>>(n->theta, n->wq, P, n->wb, n->we);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  n->act[0] = const_cast<float*>(x);
  for (int l = 0; l < kLayers; ++l) {
    float* out = (l == kLayers - 1 && y) ? y : n->act[l + 1];
    if ((e = launch_fwd(n, l, n->act[l], out, batch, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}
}  // namespace

extern "C" {

wslda_status wslda_net_create(int nx, int ny, int nz, int hidden, int max_batch, wslda_net** out) {
  if (!out || nx < 3 || ny < 3 || nz < 3 || (hidden != 8 && hidden != 32) || max_batch < 1) return WSLDA_EINVAL;
  *out = nullptr;
  wslda_net* n = new wslda_net();
  n->L = {nx, ny, nz};
  n->M = nx * ny * nz;
  n->hidden = hidden;
  n->max_batch = max_batch;
  const int ch[kLayers + 1] = {kIO, hidden, hidden, hidden, kIO};
  int64_t k = 0;
  for (int l = 0; l < kLayers; ++l) {
    n->cin[l] = ch[l];
    n->cout[l] = ch[l + 1];
    n->woff[l] = k;
    k += int64_t(ch[l + 1]) * ch[l] * 27;
    n->boff[l] = k;
    k += ch[l + 1];
  }
  n->P = k;
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
    n->owned.push_back(*p);
    return true;
  };
  const size_t amax = size_t(max_batch) * hidden * n->M * sizeof(float);
  bool ok = alloc((void**)&n->theta, n->P * 4) && alloc((void**)&n->wq, n->P * 4) &&
            alloc((void**)&n->grad, n->P * 4) && alloc((void**)&n->m, n->P * 4) && alloc((void**)&n->v, n->P * 4) &&
            alloc((void**)&n->g0, amax) && alloc((void**)&n->g1, amax) &&
            alloc((void**)&n->part, kMseBlocks * sizeof(double)) && alloc((void**)&n->err_d, sizeof(int)) &&
            alloc((void**)&n->wpart, size_t(kMaxSplit) * 896 * 32 * sizeof(float)) &&
            alloc((void**)&n->wb, kLayers * 8) &&
            alloc((void**)&n->we, kLayers * 8);
  for (int l = 1; l <= kLayers && ok; ++l)
    ok = alloc((void**)&n->act[l], size_t(max_batch) * ch[l] * n->M * sizeof(float));
  if (ok) {
    int64_t wb[kLayers], we[kLayers];
    for (int l = 0; l < kLayers; ++l) {
      wb[l] = n->woff[l];
      we[l] = n->boff[l];
    }
    ok = cudaMemcpy(n->wb, wb, sizeof(wb), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(n->we, we, sizeof(we), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(n->theta, 0, n->P * 4) == cudaSuccess && cudaMemset(n->m, 0, n->P * 4) == cudaSuccess &&
         cudaMemset(n->err_d, 0, sizeof(int)) == cudaSuccess &&
         cudaMemset(n->v, 0, n->P * 4) == cudaSuccess;
  }
  if (!ok) {
    for (void* p : n->owned) cudaFree(p);
    delete n;
    return WSLDA_ENOMEM;
  }
  *out = n;
  return WSLDA_OK;
}

void wslda_net_destroy(wslda_net* n) {
  if (!n) return;
  for (void* p : n->owned) cudaFree(p);
  delete n;
}

const char* wslda_net_last_error(const wslda_net* n) { return n ? n->err.c_str() : "null network"; }

int64_t wslda_net_param_count(const wslda_net* n) { return n ? n->P : -1; }

wslda_status wslda_net_set_params(wslda_net* n, const float* theta) {
  if (!n || !theta) return WSLDA_EINVAL;
  for (int64_t i = 0; i < n->P; ++i)
    if (!std::isfinite(theta[i])) return net_fail(n, WSLDA_ENAN, "non-finite parameter");
  if (cudaMemcpy(n->theta, theta, n->P * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(n->m, 0, n->P * 4) != cudaSuccess || cudaMemset(n->v, 0, n->P * 4) != cudaSuccess)
    return net_fail(n, WSLDA_ECUDA, "set_params copy failed");
  n->step = 0;
  return WSLDA_OK;
}

wslda_status wslda_net_get_params(wslda_net* n, float* theta) {
  if (!n || !theta) return WSLDA_EINVAL;
  if (cudaMemcpy(theta, n->theta, n->P * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return net_fail(n, WSLDA_ECUDA, "get_params copy failed");
  return WSLDA_OK;
}

wslda_status wslda_net_forward(wslda_net* n, const float* x, int batch, float* y, void* stream) {
  if (!n || !x || !y || batch < 1 || batch > n->max_batch) return WSLDA_EINVAL;
  cudaError_t e = forward(n, x, batch, y, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return net_fail(n, WSLDA_ECUDA, std::string("forward: ") + cudaGetErrorString(e));
  return WSLDA_OK;
}

wslda_status wslda_net_loss_grad(wslda_net* n, const float* x, const float* t, int batch, double* loss,
                                 float* grad_host, void* stream) {
  if (!n || !x || !t || !loss || batch < 1 || batch > n->max_batch) return WSLDA_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = forward(n, x, batch, nullptr, s);
  const int64_t nout = int64_t(batch) * kIO * n->M;
  float* g = n->g0;
  float* gnext = n->g1;
  if (e == cudaSuccess) {
    mse<<<kMseBlocks, 256, 0, s>>>(n->act[kLayers], t, nout, g, n->part);
    e = cudaGetLastError();
  }
  for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
    {
      wslda::WgradTcArgs w{};
      w.nx = n->L.nx; w.ny = n->L.ny; w.nz = n->L.nz;
      w.cin = n->cin[l]; w.cout = n->cout[l]; w.batch = batch;
      w.x = n->act[l]; w.g = g; w.part = n->wpart; w.max_split = kMaxSplit;
      w.gW = n->grad + n->woff[l]; w.err = n->err_d;
      if ((e = wslda::launch_conv_wgrad_tc(w, s)) != cudaSuccess) break;
    }
    bias_grad<<<unsigned(n->cout[l]), 256, 0, s>>>(n->M, n->cout[l], batch, g, n->grad + n->boff[l]);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if (l > 0) {
      e = launch_bwd_data(n, l, g, gnext, batch, s);
      std::swap(g, gnext);
    }
  }
  std::vector<double> part(kMseBlocks);
  int errw = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(part.data(), n->part, kMseBlocks * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&errw, n->err_d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && grad_host) e = cudaMemcpyAsync(grad_host, n->grad, n->P * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return net_fail(n, WSLDA_ECUDA, std::string("loss_grad: ") + cudaGetErrorString(e));
  if (errw) return net_fail(n, WSLDA_ETIMEOUT, "a tensor-core completion wait timed out");
  double acc = 0.0;
  for (double p : part) acc += p;
  *loss = acc / double(nout);
  return std::isfinite(*loss) ? WSLDA_OK : net_fail(n, WSLDA_ENAN, "non-finite loss");
}

wslda_status wslda_net_adam(wslda_net* n, double lr, void* stream) {
  if (!n || !(lr > 0.0)) return WSLDA_EINVAL;
  const double b1 = 0.9, b2 = 0.999;
  n->step += 1;
  const double c1 = 1.0 - std::pow(b1, double(n->step)), c2 = 1.0 - std::pow(b2, double(n->step));
  adam<<<unsigned((n->P + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n->theta, n->grad, n->m, n->v, n->P, float(lr), float(b1), float(b2), float(c1), float(c2), 1e-8f);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WSLDA_OK : net_fail(n, WSLDA_ECUDA, std::string("adam: ") + cudaGetErrorString(e));
}

wslda_status wslda_net_get_activation(wslda_net* n, int layer, int batch, float* out, void* stream) {
  if (!n || !out || layer < 0 || layer > kLayers - 2 || batch < 1 || batch > n->max_batch) return WSLDA_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = size_t(batch) * n->cout[layer] * n->M * sizeof(float);
  cudaError_t e = cudaMemcpyAsync(out, n->act[layer + 1], bytes, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return net_fail(n, WSLDA_ECUDA, std::string("get_activation: ") + cudaGetErrorString(e));
  return WSLDA_OK;
}

wslda_status wslda_net_symmetrize(const float* y, int64_t nfields, int nx, int ny, int nz, float* out,
                                  void* stream) {
  if (!y || !out || y == out || nfields < 0 || nx < 1 || ny < 1 || nz < 1) return WSLDA_EINVAL;
  const int64_t total = nfields * int64_t(nx) * ny * nz;
  if (total == 0) return WSLDA_OK;
  mirror_avg<<<unsigned((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(Lat{nx, ny, nz}, nfields,
                                                                                          y, out);
  return cudaGetLastError() == cudaSuccess ? WSLDA_OK : WSLDA_ECUDA;
}

}  // extern "C"
