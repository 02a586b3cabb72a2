// Site-major kernels: density reduction over states (spin-symmetric, frozen
// weights: Eqs. nab3D.., Sec. 2.5), potentials from the SLDA / BdG functional
// with the regularised coupling (Sec. 2.4, Eq. Creg), energy terms (Sec. 3.2),
// and precision conversions at the ABI boundary.
#include <cuda_runtime.h>

#include <algorithm>

#include "functional.cuh"
#include "internal.cuh"

namespace wslda {

// ---------------------------------------------------------------------------
// Density partial sums. Thread = lattice site, grid.y = chunk of states.
// rho += w- |v|^2 + w+ |u|^2 ;  nu += (w- - w+) u v^*.
// Float states: products in float, Kahan-compensated float sums over groups
// of kGroup states, each group folded into double accumulators.
// Double states: plain double sums.
// ---------------------------------------------------------------------------
constexpr int kGroup = 32;
constexpr int kBatch = 8;

__device__ __forceinline__ void kahan(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

template <typename R>
__global__ void __launch_bounds__(256) density_partial_kernel(const cx<R>* __restrict__ phi, const double* __restrict__ sc,
                                                              const R* __restrict__ wm, const R* __restrict__ wp,
                                                              int64_t nstates, int M, int64_t chunk,
                                                              double* __restrict__ part) {
  // no early exit: the float path broadcasts per-state factors with shuffles
  const int s_raw = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = s_raw < M;
  const int s = live ? s_raw : M - 1;
  const int lane = threadIdx.x & 31;
  const int64_t n0 = int64_t(blockIdx.y) * chunk;
  const int64_t n1 = min(n0 + chunk, nstates);
  const int64_t stride = 2 * int64_t(M);
  double ar = 0.0, anr = 0.0, ani = 0.0;
  if constexpr (sizeof(R) == 4) {
    for (int64_t g = n0; g < n1; g += kGroup) {
      // lane l converts the factor of state g + l once (one double op per 32 states)
      const int64_t nl = g + lane;
      const float s2l = nl < n1 ? float(sc[nl] * sc[nl]) : 0.f;
      float sr = 0.f, cr = 0.f, snr = 0.f, cnr = 0.f, sni = 0.f, cni = 0.f;
      const int ge = int(min(int64_t(kGroup), n1 - g));
      // batches of kBatch states: all their loads are issued before the sums
      for (int k0 = 0; k0 < ge; k0 += kBatch) {
        float2 ub[kBatch], vb[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
          const int64_t n = g + k0 + j;
          if (k0 + j < ge) {
            ub[j] = phi[n * stride + s];
            vb[j] = phi[n * stride + M + s];
          }
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
          const float s2 = __shfl_sync(0xffffffffu, s2l, (k0 + j) & 31);  // deferred normalisation
          if (k0 + j < ge) {
            const int64_t n = g + k0 + j;
            const float2 u = ub[j], v = vb[j];
            const float a = wm[n] * s2, b = wp[n] * s2, d = a - b;
            kahan(sr, cr, a * (v.x * v.x + v.y * v.y) + b * (u.x * u.x + u.y * u.y));
            kahan(snr, cnr, d * (u.x * v.x + u.y * v.y));
            kahan(sni, cni, d * (u.y * v.x - u.x * v.y));
          }
        }
      }
      ar += double(sr) - double(cr);
      anr += double(snr) - double(cnr);
      ani += double(sni) - double(cni);
    }
  } else {
#pragma unroll 4
    for (int64_t n = n0; n < n1; ++n) {
      const double2 u = phi[n * stride + s];
      const double2 v = phi[n * stride + M + s];
      const double s2 = sc[n] * sc[n];
      const double a = wm[n] * s2, b = wp[n] * s2, d = a - b;
      ar += a * (v.x * v.x + v.y * v.y) + b * (u.x * u.x + u.y * u.y);
      anr += d * (u.x * v.x + u.y * v.y);
      ani += d * (u.y * v.x - u.x * v.y);
    }
  }
  if (!live) return;
  double* p = part + int64_t(blockIdx.y) * 3 * M;
  p[s] = ar;
  p[M + s] = anr;
  p[2 * M + s] = ani;
}

template <typename R>
cudaError_t launch_density_partial(const cx<R>* phi, const double* sc, const R* wm, const R* wp, int64_t nstates,
                                   int M, int nchunk, int64_t chunk, double* part, cudaStream_t s) {
  dim3 grid((M + 255) / 256, nchunk);
  density_partial_kernel<R><<<grid, 256, 0, s>>>(phi, sc, wm, wp, nstates, M, chunk, part);
  return cudaGetLastError();
}
// Chunks of states for the density reduction: the grid (site blocks x chunks)
// should fill whole waves of resident blocks, so that no partial last wave
// idles most of the GPU. Among chunk counts with at least 16 states per chunk
// (at most 256 chunks), take the best wave fill, then the fewest chunks.
int density_chunks(int M, int64_t nstates, int is_float) {
  int dev = 0, sms = 148, per_sm = 8;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (is_float)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, density_partial_kernel<float>, 256, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, density_partial_kernel<double>, 256, 0);
  }
  const int64_t resident = int64_t(std::max(1, sms)) * std::max(1, per_sm);
  const int64_t sb = (M + 255) / 256;
  const int64_t hi = std::max<int64_t>(1, std::min<int64_t>(256, nstates / 16));
  int best = 1;
  double best_fill = -1.0;
  for (int64_t nc = 1; nc <= hi; ++nc) {
    const int64_t blocks = sb * nc;
    if (blocks < resident && nc < hi) continue;  // at least one full wave when possible
    const int64_t waves = (blocks + resident - 1) / resident;
    const double fill = double(blocks) / double(waves * resident);
    if (fill > best_fill + 1e-9) {
      best_fill = fill;
      best = int(nc);
    }
  }
  return best;
}

template cudaError_t launch_density_partial<float>(const float2*, const double*, const float*, const float*, int64_t,
                                                   int, int, int64_t, double*, cudaStream_t);
template cudaError_t launch_density_partial<double>(const double2*, const double*, const double*, const double*,
                                                    int64_t, int, int, int64_t, double*, cudaStream_t);

constexpr int kRegulatorIters = 60;  // fixed-point iterations for the t = 0 regulator

template <typename R>
__global__ void potentials_kernel(const double* __restrict__ part, int nchunk, int M, FunctionalDev fn,
                                  const double* __restrict__ vext, const double* __restrict__ dext, double* lam,
                                  int init_lam, const double* __restrict__ j, double* rho, double* nu, double* Uo,
                                  double* delta, fx4<R>* WD) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  double r = 0.0, nr = 0.0, ni = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    const double* p = part + int64_t(c) * 3 * M;
    r += p[s];
    nr += p[M + s];
    ni += p[2 * M + s];
  }
  const double ve = vext[s];
  // current part of U (A != 1): d/d rho_s [(1 - A) j^2 / (2 rho_s)] = (A - 1) j^2 / (2 rho_s^2)
  double ucur = 0.0;
  if (j) {
    const double rs = fmax(r, fn.rho_floor);
    const double jx = j[s], jy = j[M + s], jz = j[2 * M + s];
    ucur = (fn.A - 1.0) * (jx * jx + jy * jy + jz * jz) / (2.0 * rs * rs);
  }
  double l;
  if (init_lam) {
    // Regulator frozen at its t = 0 value: fixed point of U -> Lambda_c -> U.
    double U = 0.0, dr, di;
    for (int it = 0; it < kRegulatorIters; ++it) {
      l = regulator(fn.mu - U - ve, fn.ec, fn.A);
      site_potentials(fn, r, nr, ni, l, U, dr, di);
      U += ucur;
    }
    l = regulator(fn.mu - U - ve, fn.ec, fn.A);
    lam[s] = l;
  } else {
    l = lam[s];
  }
  double U, dr, di;
  site_potentials(fn, r, nr, ni, l, U, dr, di);
  U += ucur;
  rho[s] = r;
  nu[2 * s] = nr;
  nu[2 * s + 1] = ni;
  Uo[s] = U;
  delta[2 * s] = dr;
  delta[2 * s + 1] = di;
  fx4<R> f;
  f.x = R(U + ve - fn.mu);
  f.y = R(dr + dext[2 * s]);
  f.z = R(di + dext[2 * s + 1]);
  f.w = R(0);
  WD[s] = f;
}

template <typename R>
cudaError_t launch_potentials(const double* part, int nchunk, int M, FunctionalDev fn, const double* vext,
                              const double* dext, double* lam, int init_lam, const double* j, double* rho, double* nu,
                              double* U, double* delta, fx4<R>* WD, cudaStream_t s) {
  potentials_kernel<R><<<(M + 127) / 128, 128, 0, s>>>(part, nchunk, M, fn, vext, dext, lam, init_lam, j, rho, nu,
                                                       U, delta, WD);
  return cudaGetLastError();
}
template cudaError_t launch_potentials<float>(const double*, int, int, FunctionalDev, const double*, const double*,
                                              double*, int, const double*, double*, double*, double*, double*,
                                              float4*, cudaStream_t);
template cudaError_t launch_potentials<double>(const double*, int, int, FunctionalDev, const double*, const double*,
                                               double*, int, const double*, double*, double*, double*, double*,
                                               double4*, cudaStream_t);

// ---------------------------------------------------------------------------
// Current potential (A != 1): A_d = (1 - A) j_d / rho_s at each site and its
// divergence by the periodic first-derivative matrices of Eq. d_dxA, applied
// as direct sums along the three axes (d1 holds the first column of each
// circulant matrix, axis by axis). Output {A_x, A_y, A_z, div A / 2}.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void current_fields_kernel(int nx, int ny, int nz, double one_minus_A, double rho_floor,
                                      const double* __restrict__ rho, const double* __restrict__ j,
                                      const double* __restrict__ d1, fx4<R>* __restrict__ AV) {
  const int M = nx * ny * nz;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  const int x = s / (ny * nz), y = (s / nz) % ny, z = s % nz;
  auto comp = [&](int d, int site) { return one_minus_A * j[d * M + site] / fmax(rho[site], rho_floor); };
  double div = 0.0;
  for (int l = 0; l < nx; ++l) div += d1[(x - l + nx) % nx] * comp(0, (l * ny + y) * nz + z);
  for (int l = 0; l < ny; ++l) div += d1[nx + (y - l + ny) % ny] * comp(1, (x * ny + l) * nz + z);
  for (int l = 0; l < nz; ++l) div += d1[nx + ny + (z - l + nz) % nz] * comp(2, (x * ny + y) * nz + l);
  fx4<R> f;
  f.x = R(comp(0, s));
  f.y = R(comp(1, s));
  f.z = R(comp(2, s));
  f.w = R(0.5 * div);
  AV[s] = f;
}
template <typename R>
cudaError_t launch_current_fields(int nx, int ny, int nz, double A, double rho_floor, const double* rho,
                                  const double* j, const double* d1, fx4<R>* AV, cudaStream_t s) {
  const int M = nx * ny * nz;
  current_fields_kernel<R><<<(M + 127) / 128, 128, 0, s>>>(nx, ny, nz, 1.0 - A, rho_floor, rho, j, d1, AV);
  return cudaGetLastError();
}
template cudaError_t launch_current_fields<float>(int, int, int, double, double, const double*, const double*,
                                                  const double*, float4*, cudaStream_t);
template cudaError_t launch_current_fields<double>(int, int, int, double, double, const double*, const double*,
                                                   const double*, double4*, cudaStream_t);

// ---------------------------------------------------------------------------
// tau and j: sums over states of the per-state contributions (read-out only).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void sum_tauj_partial(const cx<R>* __restrict__ c, int64_t nstates, int M, int64_t chunk, double* part) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  const int64_t n0 = int64_t(blockIdx.y) * chunk, n1 = min(n0 + chunk, nstates);
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for (int64_t n = n0; n < n1; ++n) {
    const cx<R> p = c[n * 2 * M + s], q = c[n * 2 * M + M + s];
    a0 += p.x;
    a1 += p.y;
    a2 += q.x;
    a3 += q.y;
  }
  double* o = part + int64_t(blockIdx.y) * 4 * M;
  o[s] = a0;
  o[M + s] = a1;
  o[2 * M + s] = a2;
  o[3 * M + s] = a3;
}
__global__ void sum_tauj_final(const double* part, int nchunk, int M, double* tau, double* j) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  double a[4] = {0, 0, 0, 0};
  for (int cidx = 0; cidx < nchunk; ++cidx)
    for (int k = 0; k < 4; ++k) a[k] += part[int64_t(cidx) * 4 * M + int64_t(k) * M + s];
  tau[s] = a[0];
  j[s] = a[1];
  j[M + s] = a[2];
  j[2 * M + s] = a[3];
}
template <typename R>
cudaError_t launch_sum_tauj(const cx<R>* contrib, int64_t nstates, int M, int nchunk, int64_t chunk, double* part,
                            double* tau, double* j, cudaStream_t s) {
  sum_tauj_partial<R><<<dim3((M + 255) / 256, nchunk), 256, 0, s>>>(contrib, nstates, M, chunk, part);
  sum_tauj_final<<<(M + 255) / 256, 256, 0, s>>>(part, nchunk, M, tau, j);
  return cudaGetLastError();
}
template cudaError_t launch_sum_tauj<float>(const float2*, int64_t, int, int, int64_t, double*, double*, double*,
                                            cudaStream_t);
template cudaError_t launch_sum_tauj<double>(const double2*, int64_t, int, int, int64_t, double*, double*, double*,
                                             cudaStream_t);

// ---------------------------------------------------------------------------
// Deferred normalisation: per-state factor 1/sqrt(dV sum of the CTA partials).
// ---------------------------------------------------------------------------
__global__ void finalize_norm_kernel(const double* npart, int cs, int64_t n, double dV, double* sc, int* err) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = 0.0;
  for (int r = 0; r < cs; ++r) t += npart[i * 16 + r];
  const double nrm = t * dV;
  if (!(nrm > 0.0) || !isfinite(nrm)) atomicOr(err, 1);
  sc[i] = 1.0 / sqrt(nrm);
}
cudaError_t launch_finalize_norm(const double* npart, int cs, int64_t n, double dV, double* sc, int* err,
                                 cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  finalize_norm_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(npart, cs, n, dV, sc, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Quantum friction (Sec. 5.2.4) on the H fields. bp3 holds the sums of the
// per-state friction contributions as [3][M]: [1] = Re B', [2] = Im B'.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(1024) apply_friction_kernel(int M, double dV, double alpha, double beta,
                                                              double gamma, double rho0, double n_req,
                                                              const double* rho, const double* nu,
                                                              const double* delta, const double* divj,
                                                              const double* bp3, fx4<R>* WD) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int s = threadIdx.x; s < M; s += blockDim.x) acc += 2.0 * rho[s];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  double N = 0.0;
  for (int i = 0; i < int(blockDim.x >> 5); ++i) N += red[i];
  N *= dV;
  const double gt = gamma * (N - n_req) / n_req;
  for (int s = threadIdx.x; s < M; s += blockDim.x) {
    const double dU = -(alpha / rho0) * divj[s];
    const double th = atan2(nu[2 * s + 1], nu[2 * s]) - atan2(bp3[2 * M + s], bp3[M + s]);
    const double f = beta * sin(th);
    const double dr = delta[2 * s], di = delta[2 * s + 1];
    fx4<R> w = WD[s];
    w.x = R(double(w.x) + dU);
    w.y = R(double(w.y) + (f * dr - gt * di));  // Delta (f + i gt)
    w.z = R(double(w.z) + (f * di + gt * dr));
    WD[s] = w;
  }
}

template <typename R>
cudaError_t launch_apply_friction(int M, double dV, double alpha, double beta, double gamma, double rho0,
                                  double n_req, const double* rho, const double* nu, const double* delta,
                                  const double* divj, const double* bp3, fx4<R>* WD, cudaStream_t s) {
  apply_friction_kernel<R><<<1, 1024, 0, s>>>(M, dV, alpha, beta, gamma, rho0, n_req, rho, nu, delta, divj, bp3, WD);
  return cudaGetLastError();
}
template cudaError_t launch_apply_friction<float>(int, double, double, double, double, double, double, const double*,
                                                  const double*, const double*, const double*, const double*,
                                                  float4*, cudaStream_t);
template cudaError_t launch_apply_friction<double>(int, double, double, double, double, double, double,
                                                   const double*, const double*, const double*, const double*,
                                                   const double*, double4*, cudaStream_t);

// ---------------------------------------------------------------------------
// Energy (Sec. 3.2, A = 1): one block, fixed-order tree sums in double.
// out8 = e_kin, e_pot, e_pair, e_ext, e_pair_ext, e_total, n_part.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) energy_kernel(int M, int64_t nstates, FunctionalDev fn,
                                                      const double* rho_s, const double* nu, const double* delta,
                                                      const double* vext, const double* dext, const double* ekin2,
                                                      const double* wm, const double* wp, const double* j, double dV,
                                                      double* out8) {
  __shared__ double sh[7][32];
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t n = threadIdx.x; n < nstates; n += blockDim.x)
    acc[0] += 2.0 * (wm[n] * ekin2[2 * n + 1] + wp[n] * ekin2[2 * n]);  // <v|-lap|v> = 2 <v|T|v>
  for (int s = threadIdx.x; s < M; s += blockDim.x) {
    const double rho = 2.0 * rho_s[s];
    if (fn.kind == 0) acc[1] += 0.6 * fn.B * rho * fermi_energy(rho) * dV;
    acc[2] += -(delta[2 * s] * nu[2 * s] + delta[2 * s + 1] * nu[2 * s + 1]) * dV;
    acc[3] += vext[s] * rho * dV;
    acc[4] += -2.0 * (dext[2 * s] * nu[2 * s] + dext[2 * s + 1] * nu[2 * s + 1]) * dV;
    acc[5] += rho * dV;
    if (j) {  // current terms (A != 1): sum_s (1 - A) j_s^2 / (2 rho_s)
      const double rs = fmax(rho_s[s], fn.rho_floor);
      const double jx = j[s], jy = j[M + s], jz = j[2 * M + s];
      acc[6] += (1.0 - fn.A) * (jx * jx + jy * jy + jz * jz) / rs * dV;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < 7; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[7];
    for (int k = 0; k < 7; ++k) {
      t[k] = 0.0;
      for (int i = 0; i < int(blockDim.x >> 5); ++i) t[k] += sh[k][i];
    }
    out8[0] = t[0];
    out8[1] = t[1];
    out8[2] = t[2];
    out8[3] = t[3];
    out8[4] = t[4];
    out8[5] = t[0] + t[1] + t[2] + t[3] + t[4] + t[6];
    out8[6] = t[5];
    out8[7] = t[6];
  }
}

cudaError_t launch_energy(int M, int64_t nstates, FunctionalDev fn, const double* rho, const double* nu,
                          const double* delta, const double* vext, const double* dext, const double* ekin2,
                          const double* wm, const double* wp, const double* j, double dV, double* out8,
                          cudaStream_t s) {
  energy_kernel<<<1, 1024, 0, s>>>(M, nstates, fn, rho, nu, delta, vext, dext, ekin2, wm, wp, j, dV, out8);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conversions at the boundary (complex double <-> working precision).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void narrow_kernel(const double* __restrict__ src, cx<R>* __restrict__ dst, int64_t n, int* err) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = src[2 * i], b = src[2 * i + 1];
  if (!isfinite(a) || !isfinite(b)) atomicOr(err, 2);
  cx<R> c;
  c.x = R(a);
  c.y = R(b);
  dst[i] = c;
}
// dst = sc[state] * src, the state of element i being (first + i) / per_state
template <typename R>
__global__ void widen_kernel(const cx<R>* __restrict__ src, double* __restrict__ dst, int64_t n, const double* sc,
                             int64_t first, int64_t per_state) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cx<R> c = src[i];
  const double f = sc ? sc[(first + i) / per_state] : 1.0;
  dst[2 * i] = f * double(c.x);
  dst[2 * i + 1] = f * double(c.y);
}
// dst = sc[state] * src between complex float / double arrays (sc NULL: 1);
// non-finite source values set bit 1 of the error word.
template <typename S, typename D>
__global__ void rescale_kernel(const S* src, D* dst, int64_t n, const double* sc,
                               int64_t first, int64_t per_state, int* err) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const S c = src[i];
  if (err && (!isfinite(double(c.x)) || !isfinite(double(c.y)))) atomicOr(err, 2);
  const double f = sc ? sc[(first + i) / per_state] : 1.0;
  D d;
  d.x = decltype(d.x)(f * double(c.x));
  d.y = decltype(d.y)(f * double(c.y));
  dst[i] = d;
}
// Component `comp` of every state times a site-dependent complex factor:
// dst[n][comp][r] *= phase[r] (phase interleaved doubles, product in double).
template <typename R>
__global__ void imprint_kernel(cx<R>* __restrict__ states, int64_t nstates, int M, int comp,
                               const double* __restrict__ phase) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= nstates * M) return;
  const int64_t n = i / M;
  const int r = int(i % M);
  cx<R>& z = states[(2 * n + comp) * M + r];
  const double a = double(z.x), b = double(z.y), c = phase[2 * r], d = phase[2 * r + 1];
  z.x = R(a * c - b * d);
  z.y = R(a * d + b * c);
}
__global__ void fill_kernel(double* p, double v, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
template <typename R>
__global__ void to_real_kernel(const double* __restrict__ src, R* __restrict__ dst, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = R(src[i]);
}

template <typename R>
cudaError_t launch_narrow(const double* src, cx<R>* dst, int64_t n, int* err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  narrow_kernel<R><<<unsigned((n + 255) / 256), 256, 0, s>>>(src, dst, n, err);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_widen(const cx<R>* src, double* dst, int64_t n, const double* sc, int64_t first, int64_t per_state,
                         cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  widen_kernel<R><<<unsigned((n + 255) / 256), 256, 0, s>>>(src, dst, n, sc, first, per_state);
  return cudaGetLastError();
}
template <typename S, typename D>
cudaError_t launch_rescale(const S* src, D* dst, int64_t n, const double* sc, int64_t first, int64_t per_state,
                           int* err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  rescale_kernel<S, D><<<unsigned((n + 255) / 256), 256, 0, s>>>(src, dst, n, sc, first, per_state, err);
  return cudaGetLastError();
}
template cudaError_t launch_rescale<float2, float2>(const float2*, float2*, int64_t, const double*, int64_t, int64_t,
                                                    int*, cudaStream_t);
template cudaError_t launch_rescale<float2, double2>(const float2*, double2*, int64_t, const double*, int64_t,
                                                     int64_t, int*, cudaStream_t);
template cudaError_t launch_rescale<double2, float2>(const double2*, float2*, int64_t, const double*, int64_t,
                                                     int64_t, int*, cudaStream_t);

template <typename R>
cudaError_t launch_imprint(cx<R>* states, int64_t nstates, int M, int comp, const double* phase, cudaStream_t s) {
  const int64_t total = nstates * M;
  if (total == 0) return cudaSuccess;
  imprint_kernel<R><<<unsigned((total + 255) / 256), 256, 0, s>>>(states, nstates, M, comp, phase);
  return cudaGetLastError();
}
template cudaError_t launch_imprint<float>(float2*, int64_t, int, int, const double*, cudaStream_t);
template cudaError_t launch_imprint<double>(double2*, int64_t, int, int, const double*, cudaStream_t);

cudaError_t launch_fill(double* p, double v, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  fill_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_to_real(const double* src, R* dst, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  to_real_kernel<R><<<unsigned((n + 255) / 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}
template cudaError_t launch_narrow<float>(const double*, float2*, int64_t, int*, cudaStream_t);
template cudaError_t launch_narrow<double>(const double*, double2*, int64_t, int*, cudaStream_t);
template cudaError_t launch_widen<float>(const float2*, double*, int64_t, const double*, int64_t, int64_t,
                                        cudaStream_t);
template cudaError_t launch_widen<double>(const double2*, double*, int64_t, const double*, int64_t, int64_t,
                                         cudaStream_t);
template cudaError_t launch_to_real<float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_to_real<double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace wslda
