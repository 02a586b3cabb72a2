// Static self-consistent solver (Alg. 1, Sec. 3.2) for trapped, spin-symmetric
// T = 0 systems with real potentials that are symmetric under the reflections
// i -> N - i (mod N) of each axis (a trap centred on site N/2).
//
// The Laplacian of Eq. D2 depends on i - j only and is even in it, so it
// commutes with the reflections; so do the diagonal fields. In the basis of
// even and odd combinations per axis,
//   even: e_0 = d_0, e_{N/2} = d_{N/2}, e_a = (d_a + d_{N-a})/sqrt2  (N/2+1)
//   odd : o_a = (d_a - d_{N-a})/sqrt2, 0 < a < N/2                  (N/2-1)
// the 2M x 2M matrix of Eq. HpsiEpsi splits into 8 real symmetric blocks
// [[h, D], [D, -h]] of size 2 m_b (m_b = product of the per-axis sizes), with
// h = -L_b/2 + W: the block Laplacian is the Kronecker sum of the per-axis
// parity blocks of Eq. D2, and W, D are the field values at the block's
// representative sites. The (u, v) -> (-v, u) symmetry maps E to -E inside
// each block, so each block holds m_b positive eigenvalues, and the 8 blocks
// together hold the M positive-energy states.
//
// One iteration (map K of Alg. 1, then linear mixing) on the device:
//   build_block   block matrix from (U_in, Delta_in, V_ext, mu)
//   cusolverDnDsyevd (library eigensolver, double precision)
//   block_density rho_sigma, nu at the representative sites (fundamental domain)
//   block_kinetic <u|T|u>, <v|T|v> of each positive-energy state
//   scf_fields    densities on the whole lattice, regulator at the input mean
//                 field, output potentials K[p]
//   energy terms  (the energy kernel of the time-dependent path)
//   scf_mix       p <- m K[p] + (1 - m) p, or the modified Broyden update
//                 (broyden_* kernels, multi_dot, a k x k solve on the host)
// and at the end unfold_states writes the eigenstates into the box.
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "functional.cuh"
#include "internal.cuh"

namespace wslda {
namespace {

struct BlockGeom {
  int m;                    // sites in the block
  int mx, my, mz;           // per-axis block sizes
  int px, py, pz;           // per-axis parity, 0 even, 1 odd
  int nx, ny, nz;           // lattice
  const double *Dx, *Dy, *Dz;  // per-axis parity blocks of Eq. D2, row-major
};

// Lattice coordinate of block index a along an axis: even blocks start at
// site 0, odd blocks at site 1.
__device__ __forceinline__ int lattice_site(const BlockGeom& g, int a, int b, int c) {
  return ((a + g.px) * g.ny + (b + g.py)) * g.nz + (c + g.pz);
}

__device__ __forceinline__ void decode(const BlockGeom& g, int r, int& a, int& b, int& c) {
  c = r % g.mz;
  const int t = r / g.mz;
  b = t % g.my;
  a = t / g.my;
}

template <typename T>
__global__ void build_block(BlockGeom g, const double* __restrict__ U, const double* __restrict__ D,
                            const double* __restrict__ vext, double mu, T* __restrict__ H) {
  const int64_t n2 = 2 * int64_t(g.m);
  const int64_t total = n2 * n2;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int col = int(idx / n2), row = int(idx - int64_t(col) * n2);  // column-major
    const int ru = row >= g.m, cu = col >= g.m;
    const int r = row - ru * g.m, c = col - cu * g.m;
    double v = 0.0;
    if (ru == cu) {
      int a, b, cc, a2, b2, c2;
      decode(g, r, a, b, cc);
      decode(g, c, a2, b2, c2);
      double L = 0.0;
      if (b == b2 && cc == c2) L += g.Dx[a * g.mx + a2];
      if (a == a2 && cc == c2) L += g.Dy[b * g.my + b2];
      if (a == a2 && b == b2) L += g.Dz[cc * g.mz + c2];
      double h = -0.5 * L;
      if (r == c) {
        const int s = lattice_site(g, a, b, cc);
        h += U[s] + vext[s] - mu;
      }
      v = ru ? -h : h;
    } else if (r == c) {
      int a, b, cc;
      decode(g, r, a, b, cc);
      v = D[lattice_site(g, a, b, cc)];
    }
    H[idx] = T(v);
  }
}

// Weight of a representative site in the density: 1/2 per axis whose
// coordinate is not a fixed point of the reflection (the basis vector is
// spread over two sites there).
__device__ __forceinline__ double orbit_weight(int i, int n) { return (i == 0 || 2 * i == n) ? 1.0 : 0.5; }

// Thread = block row r; sums over the m positive-energy columns.
template <typename T>
__global__ void block_density(BlockGeom g, const T* __restrict__ Z, double inv_dV, double* __restrict__ frho,
                              double* __restrict__ fnu) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.m) return;
  const int64_t n2 = 2 * int64_t(g.m);
  double sr = 0.0, sn = 0.0;
  for (int j = g.m; j < 2 * g.m; ++j) {
    const T* col = Z + int64_t(j) * n2;
    const double cu = col[r], cv = col[g.m + r];
    sr += cv * cv;
    sn += cu * cv;
  }
  int a, b, c;
  decode(g, r, a, b, c);
  const int ix = a + g.px, iy = b + g.py, iz = c + g.pz;
  const int hy = g.ny / 2 + 1, hz = g.nz / 2 + 1;
  const double w = orbit_weight(ix, g.nx) * orbit_weight(iy, g.ny) * orbit_weight(iz, g.nz) * inv_dV;
  const int f = (ix * hy + iy) * hz + iz;
  frho[f] += w * sr;
  fnu[f] += w * sn;
}

// CTA = one positive-energy state (column m + blockIdx.x). The column is
// staged in shared memory, L_b is applied through its Kronecker structure,
// and <u|-L/2|u>, <v|-L/2|v> are written as ekin2[2 j], ekin2[2 j + 1].
template <typename T>
__global__ void __launch_bounds__(256) block_kinetic(BlockGeom g, const T* __restrict__ Z,
                                                     double* __restrict__ ekin2) {
  extern __shared__ __align__(16) unsigned char col_raw[];
  T* col = reinterpret_cast<T*>(col_raw);
  __shared__ double red[2][8];
  const int j = blockIdx.x;
  const int64_t n2 = 2 * int64_t(g.m);
  const T* src = Z + (int64_t(g.m) + j) * n2;
  for (int i = threadIdx.x; i < 2 * g.m; i += blockDim.x) col[i] = src[i];
  __syncthreads();
  double tu = 0.0, tv = 0.0;
  for (int r = threadIdx.x; r < g.m; r += blockDim.x) {
    int a, b, c;
    decode(g, r, a, b, c);
    double lu = 0.0, lv = 0.0;
    for (int k = 0; k < g.mx; ++k) {
      const double d = g.Dx[a * g.mx + k];
      const int q = (k * g.my + b) * g.mz + c;
      lu += d * col[q];
      lv += d * col[g.m + q];
    }
    for (int k = 0; k < g.my; ++k) {
      const double d = g.Dy[b * g.my + k];
      const int q = (a * g.my + k) * g.mz + c;
      lu += d * col[q];
      lv += d * col[g.m + q];
    }
    for (int k = 0; k < g.mz; ++k) {
      const double d = g.Dz[c * g.mz + k];
      const int q = (a * g.my + b) * g.mz + k;
      lu += d * col[q];
      lv += d * col[g.m + q];
    }
    tu += col[r] * lu;
    tv += col[g.m + r] * lv;
  }
  for (int o = 16; o > 0; o >>= 1) {
    tu += __shfl_xor_sync(0xffffffffu, tu, o);
    tv += __shfl_xor_sync(0xffffffffu, tv, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = tu;
    red[1][w] = tv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double su = 0.0, sv = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) {
      su += red[0][i];
      sv += red[1][i];
    }
    ekin2[2 * j] = -0.5 * su;
    ekin2[2 * j + 1] = -0.5 * sv;
  }
}

__device__ __forceinline__ int fold(int i, int n) { return i <= n / 2 ? i : n - i; }

// Densities on the whole lattice from the fundamental domain, regulator at
// the input mean field, output potentials K[p].
__global__ void scf_fields(int nx, int ny, int nz, const double* __restrict__ frho, const double* __restrict__ fnu,
                           const double* __restrict__ Uin, const double* __restrict__ vext, FunctionalDev fn,
                           double* __restrict__ rho, double* __restrict__ nu, double* __restrict__ Uout,
                           double* __restrict__ delta) {
  const int M = nx * ny * nz;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  const int iz = s % nz, iy = (s / nz) % ny, ix = s / (ny * nz);
  const int f = (fold(ix, nx) * (ny / 2 + 1) + fold(iy, ny)) * (nz / 2 + 1) + fold(iz, nz);
  const double r = frho[f], n = fnu[f];
  const double lam = regulator(fn.mu - Uin[s] - vext[s], fn.ec);
  double U, dr, di;
  site_potentials(fn, r, n, 0.0, lam, U, dr, di);
  rho[s] = r;
  nu[2 * s] = n;
  nu[2 * s + 1] = 0.0;
  Uout[s] = U;
  delta[2 * s] = dr;
  delta[2 * s + 1] = di;
}

__global__ void scf_mix(int M, double m, const double* __restrict__ Uout, const double* __restrict__ delta_out,
                        double* __restrict__ Uin, double* __restrict__ Din) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  Uin[s] = m * Uout[s] + (1.0 - m) * Uin[s];
  Din[s] = m * delta_out[2 * s] + (1.0 - m) * Din[s];
}

// Modified Broyden mixing on the vector x = (U, Re Delta, mu) of length 2M + 1.
// Residual F = K[x] - x; the mu component comes from the host.
__global__ void broyden_residual(int M, const double* __restrict__ Uout, const double* __restrict__ delta_out,
                                 double mu, double mu_out, double* __restrict__ x, double* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) F[i] = Uout[i] - x[i];
  else if (i < 2 * M) F[i] = delta_out[2 * (i - M)] - x[i];
  else if (i == 2 * M) {
    x[i] = mu;
    F[i] = mu_out - mu;
  }
}

// dF <- F - F_prev, u <- x - x_prev
__global__ void broyden_diff(int n, const double* __restrict__ F, const double* __restrict__ Fp,
                             const double* __restrict__ x, const double* __restrict__ xp, double* __restrict__ dF,
                             double* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dF[i] = F[i] - Fp[i];
  u[i] = x[i] - xp[i];
}

// dF <- dF / |dF|, u <- alpha dF / |dF| + u / |dF|
__global__ void broyden_scale(int n, double inv_norm, double alpha, double* __restrict__ dF, double* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = dF[i] * inv_norm;
  dF[i] = d;
  u[i] = alpha * d + u[i] * inv_norm;
}

constexpr int kMaxDots = 17;
constexpr int kDotBlocks = 64;
struct DotList {
  const double* a[kMaxDots];
  const double* b[kMaxDots];
  int count;
};

// partial[d][block] = sum over the block's elements of a_d . b_d; the host adds
// the partials in block order.
__global__ void __launch_bounds__(256) multi_dot(DotList L, int n, double* __restrict__ partial) {
  __shared__ double red[8];
  for (int d = 0; d < L.count; ++d) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += L.a[d][i] * L.b[d][i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
      partial[d * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// x <- x + alpha F - sum_j gamma_j u_j (j in chronological order)
struct GammaList {
  const double* u[8];
  double g[8];
  int count;
};
__global__ void broyden_update(int n, double alpha, const double* __restrict__ F, GammaList G, double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double corr = 0.0;
  for (int j = 0; j < G.count; ++j) corr += G.g[j] * G.u[j][i];
  x[i] = x[i] + alpha * F[i] - corr;
}

// Block index and basis-vector value of lattice coordinate i along an axis of
// parity p; false where the odd basis vanishes (the two fixed points).
__device__ __forceinline__ bool axis_basis(int i, int n, int p, int& a, double& f) {
  const int j = fold(i, n);
  const bool fixed = (j == 0 || 2 * j == n);
  if (p == 0) {
    a = j;
    f = fixed ? 1.0 : M_SQRT1_2;
    return true;
  }
  if (fixed) return false;
  a = j - 1;
  f = i > n / 2 ? -M_SQRT1_2 : M_SQRT1_2;
  return true;
}

// Thread = (state j, lattice site s): the block eigenvector expanded on the
// lattice, scaled to sum_r dV (|u|^2 + |v|^2) = 1.
template <typename T, typename C>
__global__ void unfold_states(BlockGeom g, const T* __restrict__ Z, double inv_sqrt_dV, C* __restrict__ out) {
  const int64_t M = int64_t(g.nx) * g.ny * g.nz;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(g.m) * M) return;
  const int j = int(idx / M);
  const int s = int(idx - int64_t(j) * M);
  const int iz = s % g.nz, iy = (s / g.nz) % g.ny, ix = s / (g.ny * g.nz);
  int a, b, c;
  double fx, fy, fz;
  double u = 0.0, v = 0.0;
  if (axis_basis(ix, g.nx, g.px, a, fx) && axis_basis(iy, g.ny, g.py, b, fy) && axis_basis(iz, g.nz, g.pz, c, fz)) {
    const T* col = Z + (int64_t(g.m) + j) * 2 * g.m;
    const int r = (a * g.my + b) * g.mz + c;
    const double f = fx * fy * fz * inv_sqrt_dV;
    u = col[r] * f;
    v = col[g.m + r] * f;
  }
  C cu, cv;
  cu.x = u;
  cu.y = 0;
  cv.x = v;
  cv.y = 0;
  out[(2 * int64_t(j)) * M + s] = cu;
  out[(2 * int64_t(j) + 1) * M + s] = cv;
}

// Eq. D2 of one axis as the spectral second derivative: D_ij = (1/N) sum_l
// (-k_l^2) cos(k_l (i - j) d), the Nyquist mode kept, then its even and odd
// parity blocks B^T D B (even block first, both row-major).
std::vector<double> parity_blocks(int n, double d) {
  std::vector<double> D(size_t(n) * n);
  const double L = n * d;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int l = 0; l < n; ++l) {
        const int q = l < n / 2 ? l : l - n;
        const double k = 2.0 * M_PI * q / L;
        const long ph = (long(l) * long(((i - j) % n + n) % n)) % n;  // exact phase reduction
        s += -k * k * std::cos(2.0 * M_PI * double(ph) / n);
      }
      D[size_t(i) * n + j] = s / n;
    }
  const int ne = n / 2 + 1, no = n / 2 - 1;
  // basis vectors as (site, coefficient) pairs
  auto even = [&](int a, int& s0, int& s1, double& c) {
    s0 = a;
    s1 = (n - a) % n;
    c = (a == 0 || 2 * a == n) ? 1.0 : M_SQRT1_2;
  };
  std::vector<double> out(size_t(ne) * ne + size_t(no) * no);
  for (int a = 0; a < ne; ++a)
    for (int b = 0; b < ne; ++b) {
      int a0, a1, b0, b1;
      double ca, cb;
      even(a, a0, a1, ca);
      even(b, b0, b1, cb);
      double v = 0.0;
      // <e_a| D |e_b>, each basis vector touching one site (fixed points) or two
      const int na = (a0 == a1) ? 1 : 2, nb = (b0 == b1) ? 1 : 2;
      for (int x = 0; x < na; ++x)
        for (int y = 0; y < nb; ++y) v += ca * cb * D[size_t(x ? a1 : a0) * n + (y ? b1 : b0)];
      out[size_t(a) * ne + b] = v;
    }
  double* odd = out.data() + size_t(ne) * ne;
  for (int a = 0; a < no; ++a)
    for (int b = 0; b < no; ++b) {
      const int i0 = a + 1, i1 = n - a - 1, j0 = b + 1, j1 = n - b - 1;
      const double v = 0.5 * (D[size_t(i0) * n + j0] - D[size_t(i0) * n + j1] - D[size_t(i1) * n + j0] +
                              D[size_t(i1) * n + j1]);
      odd[size_t(a) * no + b] = v;
    }
  return out;
}

struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t get(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return e;
  }
};

struct SolverHandle {
  cusolverDnHandle_t h = nullptr;
  ~SolverHandle() {
    if (h) cusolverDnDestroy(h);
  }
};

}  // namespace

wslda_status static_solve(const ScfBox& b, const double* U0, const double* D0, const wslda_scf_params& p,
                          double* qpE, wslda_scf_result* res, std::string& err) {
  const int nx = b.lat.nx, ny = b.lat.ny, nz = b.lat.nz;
  const int M = b.M;
  const double dV = b.lat.dx * b.lat.dy * b.lat.dz;
  cudaStream_t s = b.s;
#define SCF_CUDA(call)                                        \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) {                                  \
      err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return WSLDA_ECUDA;                                     \
    }                                                         \
  } while (0)

  // per-axis parity blocks of Eq. D2
  const int ns[3] = {nx, ny, nz};
  const double ds[3] = {b.lat.dx, b.lat.dy, b.lat.dz};
  std::vector<double> tab;
  size_t off[3][2];
  int sz[3][2];
  for (int ax = 0; ax < 3; ++ax) {
    std::vector<double> t = parity_blocks(ns[ax], ds[ax]);
    sz[ax][0] = ns[ax] / 2 + 1;
    sz[ax][1] = ns[ax] / 2 - 1;
    off[ax][0] = tab.size();
    off[ax][1] = tab.size() + size_t(sz[ax][0]) * sz[ax][0];
    tab.insert(tab.end(), t.begin(), t.end());
  }
  Scratch sc;
  double* dtab;
  SCF_CUDA(sc.get(&dtab, tab.size()));
  SCF_CUDA(cudaMemcpyAsync(dtab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, s));

  // the 8 parity blocks, each with its own matrix / eigenvector buffer
  struct Blk {
    BlockGeom g;
    double *Z, *W;
    int64_t first;  // index of its first state
  };
  std::vector<Blk> blks;
  int64_t first = 0;
  for (int px = 0; px < 2; ++px)
    for (int py = 0; py < 2; ++py)
      for (int pz = 0; pz < 2; ++pz) {
        BlockGeom g{};
        g.mx = sz[0][px];
        g.my = sz[1][py];
        g.mz = sz[2][pz];
        g.m = g.mx * g.my * g.mz;
        if (g.m == 0) continue;
        g.px = px;
        g.py = py;
        g.pz = pz;
        g.nx = nx;
        g.ny = ny;
        g.nz = nz;
        g.Dx = dtab + off[0][px];
        g.Dy = dtab + off[1][py];
        g.Dz = dtab + off[2][pz];
        Blk k{g, nullptr, nullptr, first};
        SCF_CUDA(sc.get(&k.Z, size_t(2 * g.m) * size_t(2 * g.m)));
        SCF_CUDA(sc.get(&k.W, size_t(2 * g.m)));
        blks.push_back(k);
        first += g.m;
      }
  if (first != M) {
    err = "parity blocks do not cover the lattice";
    return WSLDA_EINVAL;
  }

  SolverHandle sh;
  if (cusolverDnCreate(&sh.h) != CUSOLVER_STATUS_SUCCESS) {
    err = "cusolverDnCreate failed";
    return WSLDA_ECUDA;
  }
  cusolverDnSetStream(sh.h, s);
  // the leading p.fp32_iters iterations diagonalise in single precision in
  // the same buffers (a float matrix takes half of a double one)
  int lwork = 0, lwork_s = 0;
  for (const Blk& k : blks) {
    int lw = 0;
    if (cusolverDnDsyevd_bufferSize(sh.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, 2 * k.g.m, k.Z,
                                    2 * k.g.m, k.W, &lw) != CUSOLVER_STATUS_SUCCESS) {
      err = "cusolverDnDsyevd_bufferSize failed";
      return WSLDA_ECUDA;
    }
    lwork = std::max(lwork, lw);
    if (p.fp32_iters > 0) {
      if (cusolverDnSsyevd_bufferSize(sh.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, 2 * k.g.m,
                                      reinterpret_cast<float*>(k.Z), 2 * k.g.m, reinterpret_cast<float*>(k.W),
                                      &lw) != CUSOLVER_STATUS_SUCCESS) {
        err = "cusolverDnSsyevd_bufferSize failed";
        return WSLDA_ECUDA;
      }
      lwork_s = std::max(lwork_s, lw);
    }
  }
  double *work, *Uin, *Din, *Uout, *frho, *fnu;
  int* info;
  const int nf = (nx / 2 + 1) * (ny / 2 + 1) * (nz / 2 + 1);
  SCF_CUDA(sc.get(&work, std::max<size_t>(size_t(lwork), (size_t(lwork_s) + 1) / 2)));
  SCF_CUDA(sc.get(&info, blks.size()));
  // x = (U_in, Delta_in, mu): the mixed vector; mu lives on the host between iterations
  const int nvec = 2 * M + 1;
  double* xvec;
  SCF_CUDA(sc.get(&xvec, size_t(nvec)));
  Uin = xvec;
  Din = xvec + M;
  SCF_CUDA(sc.get(&Uout, M));
  SCF_CUDA(sc.get(&frho, nf));
  SCF_CUDA(sc.get(&fnu, nf));
  SCF_CUDA(cudaMemcpyAsync(Uin, U0, size_t(M) * 8, cudaMemcpyHostToDevice, s));
  SCF_CUDA(cudaMemcpyAsync(Din, D0, size_t(M) * 8, cudaMemcpyHostToDevice, s));
  {
    std::vector<double> ones(M, 1.0), zeros(M, 0.0);
    SCF_CUDA(cudaMemcpyAsync(b.wm, ones.data(), size_t(M) * 8, cudaMemcpyHostToDevice, s));
    SCF_CUDA(cudaMemcpyAsync(b.wp, zeros.data(), size_t(M) * 8, cudaMemcpyHostToDevice, s));
    SCF_CUDA(cudaStreamSynchronize(s));
  }
  int max_smem = 0;
  for (const Blk& k : blks) max_smem = std::max(max_smem, int(2 * k.g.m * sizeof(double)));
  SCF_CUDA(cudaFuncSetAttribute(block_kinetic<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));

  // modified Broyden state: ring of (dF, u) pairs, previous x and F, dot partials
  const bool broyden = p.method == 1;
  const int mem = p.broyden_memory > 0 ? std::min(p.broyden_memory, 8) : 7;
  const double w0 = p.broyden_w0 > 0 ? p.broyden_w0 : 0.01;
  double *bF = nullptr, *bxp = nullptr, *bFp = nullptr, *bdF = nullptr, *bu = nullptr, *bpart = nullptr;
  if (broyden) {
    SCF_CUDA(sc.get(&bF, size_t(nvec)));
    SCF_CUDA(sc.get(&bxp, size_t(nvec)));
    SCF_CUDA(sc.get(&bFp, size_t(nvec)));
    SCF_CUDA(sc.get(&bdF, size_t(mem) * nvec));
    SCF_CUDA(sc.get(&bu, size_t(mem) * nvec));
    SCF_CUDA(sc.get(&bpart, size_t(kMaxDots) * kDotBlocks));
  }
  int bcount = 0, bhead = 0;       // stored pairs, next ring slot
  bool bprev = false;              // previous (x, F) present
  std::vector<std::vector<double>> A(mem, std::vector<double>(mem, 0.0));  // dF_i . dF_j by ring slot
  auto dots = [&](const DotList& L, std::vector<double>& outv) -> cudaError_t {
    multi_dot<<<kDotBlocks, 256, 0, s>>>(L, nvec, bpart);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::vector<double> h(size_t(L.count) * kDotBlocks);
    e = cudaMemcpyAsync(h.data(), bpart, h.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    outv.assign(L.count, 0.0);
    for (int d = 0; d < L.count; ++d)
      for (int k = 0; k < kDotBlocks; ++k) outv[d] += h[size_t(d) * kDotBlocks + k];
    return e;
  };
  const unsigned vgrid = unsigned((nvec + 255) / 256);

  FunctionalDev fn = b.fn;
  const double e_ref = p.e_ref > 0 ? p.e_ref : 0.5;
  const bool fixed_n = p.n_target > 0;
  double prev[6] = {0, 0, 0, 0, 0, 0};
  double cur[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double change = 0.0;
  int it = 0;
  bool converged = false;
  std::vector<std::vector<double>> evals(blks.size());
  std::vector<float> evals_s;
  bool single = false, prev_double = false;
  SCF_CUDA(cudaFuncSetAttribute(block_kinetic<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem / 2));
  for (it = 1; it <= p.max_iters; ++it) {
    single = it <= p.fp32_iters;
    if (!single && it == p.fp32_iters + 1 && p.fp32_iters > 0) {
      bcount = 0;  // the Broyden history of the single-precision phase is dropped
      bhead = 0;
      bprev = false;
    }
    SCF_CUDA(cudaMemsetAsync(frho, 0, size_t(nf) * 8, s));
    SCF_CUDA(cudaMemsetAsync(fnu, 0, size_t(nf) * 8, s));
    for (size_t bi = 0; bi < blks.size(); ++bi) {
      const Blk& k = blks[bi];
      const int n2 = 2 * k.g.m;
      const int64_t tot = int64_t(n2) * n2;
      const unsigned grid = unsigned(std::min<int64_t>((tot + 255) / 256, 148 * 16));
      if (single) {
        float* Zs = reinterpret_cast<float*>(k.Z);
        build_block<float><<<grid, 256, 0, s>>>(k.g, Uin, Din, b.vext, fn.mu, Zs);
        SCF_CUDA(cudaGetLastError());
        if (cusolverDnSsyevd(sh.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n2, Zs, n2,
                             reinterpret_cast<float*>(k.W), reinterpret_cast<float*>(work), lwork_s,
                             info + bi) != CUSOLVER_STATUS_SUCCESS) {
          err = "cusolverDnSsyevd failed";
          return WSLDA_ECUDA;
        }
        block_density<float><<<(k.g.m + 127) / 128, 128, 0, s>>>(k.g, Zs, 1.0 / dV, frho, fnu);
        block_kinetic<float><<<k.g.m, 256, 2 * k.g.m * sizeof(float), s>>>(k.g, Zs, b.ekin2 + 2 * k.first);
      } else {
        build_block<double><<<grid, 256, 0, s>>>(k.g, Uin, Din, b.vext, fn.mu, k.Z);
        SCF_CUDA(cudaGetLastError());
        if (cusolverDnDsyevd(sh.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n2, k.Z, n2, k.W, work, lwork,
                             info + bi) != CUSOLVER_STATUS_SUCCESS) {
          err = "cusolverDnDsyevd failed";
          return WSLDA_ECUDA;
        }
        block_density<double><<<(k.g.m + 127) / 128, 128, 0, s>>>(k.g, k.Z, 1.0 / dV, frho, fnu);
        block_kinetic<double><<<k.g.m, 256, 2 * k.g.m * sizeof(double), s>>>(k.g, k.Z, b.ekin2 + 2 * k.first);
      }
      SCF_CUDA(cudaGetLastError());
    }
    scf_fields<<<(M + 127) / 128, 128, 0, s>>>(nx, ny, nz, frho, fnu, Uin, b.vext, fn, b.rho, b.nu, Uout, b.delta);
    SCF_CUDA(cudaGetLastError());
    SCF_CUDA(launch_energy(M, M, fn, b.rho, b.nu, b.delta, b.vext, b.dext, b.ekin2, b.wm, b.wp, nullptr, dV, b.out8, s));
    std::vector<int> hinfo(blks.size());
    SCF_CUDA(cudaMemcpyAsync(cur, b.out8, 7 * 8, cudaMemcpyDeviceToHost, s));
    SCF_CUDA(cudaMemcpyAsync(hinfo.data(), info, blks.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    for (size_t bi = 0; bi < blks.size(); ++bi) {
      evals[bi].resize(2 * size_t(blks[bi].g.m));
      if (!single)
        SCF_CUDA(cudaMemcpyAsync(evals[bi].data(), blks[bi].W, evals[bi].size() * 8, cudaMemcpyDeviceToHost, s));
    }
    if (single) {
      SCF_CUDA(cudaStreamSynchronize(s));
      for (size_t bi = 0; bi < blks.size(); ++bi) {
        evals_s.resize(evals[bi].size());
        SCF_CUDA(cudaMemcpy(evals_s.data(), blks[bi].W, evals_s.size() * 4, cudaMemcpyDeviceToHost));
        for (size_t j = 0; j < evals_s.size(); ++j) evals[bi][j] = evals_s[j];
      }
    }
    SCF_CUDA(cudaStreamSynchronize(s));
    for (size_t bi = 0; bi < blks.size(); ++bi) {
      if (hinfo[bi] != 0) {
        err = "cusolverDnDsyevd did not converge (info " + std::to_string(hinfo[bi]) + ")";
        return WSLDA_ECUDA;
      }
      const int m = blks[bi].g.m;
      if (!(evals[bi][m - 1] < 0.0 && evals[bi][m] > 0.0)) {
        err = "a parity block has a zero quasiparticle energy (its spectrum does not split into m + m)";
        return WSLDA_EUNSUPPORTED;
      }
    }
    for (int k = 0; k < 7; ++k)
      if (!std::isfinite(cur[k])) {
        err = "non-finite energy in the static iteration";
        return WSLDA_ENAN;
      }
    const double n_sigma = 0.5 * cur[6];
    const bool n_ok = !fixed_n || std::fabs(p.n_target - n_sigma) < p.eps_npart;
    if (it >= 2) {
      change = 0.0;
      for (int k = 0; k < 6; ++k) change = std::max(change, std::fabs(cur[k] - prev[k]) / e_ref);
      // convergence is judged only between two double-precision iterations
      if (change < p.eps_energy && n_ok && !single && prev_double) {
        converged = true;
        break;
      }
    }
    for (int k = 0; k < 6; ++k) prev[k] = cur[k];
    prev_double = !single;
    if (it == p.max_iters) break;
    // Eq. update-mu is a step of the map; mu_out is mixed with the potentials
    const double mu_out = fixed_n ? fn.mu + (p.a_mu / p.n_target) * (p.n_target - n_sigma) : fn.mu;
    if (!broyden) {
      scf_mix<<<(M + 127) / 128, 128, 0, s>>>(M, p.mixing, Uout, b.delta, Uin, Din);
      SCF_CUDA(cudaGetLastError());
      fn.mu = p.mixing * mu_out + (1.0 - p.mixing) * fn.mu;
      continue;
    }
    broyden_residual<<<vgrid, 256, 0, s>>>(M, Uout, b.delta, fn.mu, mu_out, xvec, bF);
    SCF_CUDA(cudaGetLastError());
    if (bprev) {
      const int slot = bhead;
      double* dF = bdF + size_t(slot) * nvec;
      double* u = bu + size_t(slot) * nvec;
      broyden_diff<<<vgrid, 256, 0, s>>>(nvec, bF, bFp, xvec, bxp, dF, u);
      SCF_CUDA(cudaGetLastError());
      DotList L{};
      L.a[0] = dF;
      L.b[0] = dF;
      L.count = 1;
      std::vector<double> nn;
      SCF_CUDA(dots(L, nn));
      if (!(nn[0] > 0.0)) {
        err = "Broyden mixing: two consecutive residuals are equal";
        return WSLDA_ENAN;
      }
      const double inv = 1.0 / std::sqrt(nn[0]);
      broyden_scale<<<vgrid, 256, 0, s>>>(nvec, inv, p.mixing, dF, u);
      SCF_CUDA(cudaGetLastError());
      bhead = (bhead + 1) % mem;
      bcount = std::min(bcount + 1, mem);
    }
    // chronological ring slots of the stored pairs
    std::vector<int> order(bcount);
    for (int j = 0; j < bcount; ++j) order[j] = ((bhead - bcount + j) % mem + mem) % mem;
    GammaList G{};
    G.count = bcount;
    if (bcount > 0) {
      const int newest = order[bcount - 1];
      DotList L{};
      for (int j = 0; j < bcount; ++j) {  // new row of A, then c_j = dF_j . F
        L.a[j] = bdF + size_t(newest) * nvec;
        L.b[j] = bdF + size_t(order[j]) * nvec;
        L.a[bcount + j] = bdF + size_t(order[j]) * nvec;
        L.b[bcount + j] = bF;
      }
      L.count = 2 * bcount;
      std::vector<double> dv;
      SCF_CUDA(dots(L, dv));
      for (int j = 0; j < bcount; ++j) A[newest][order[j]] = A[order[j]][newest] = dv[j];
      // gamma = (w0^2 I + A)^{-1} c, by Gaussian elimination with partial pivoting
      const int k = bcount;
      std::vector<double> m(size_t(k) * (k + 1));
      for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j) m[size_t(i) * (k + 1) + j] = A[order[i]][order[j]] + (i == j ? w0 * w0 : 0.0);
        m[size_t(i) * (k + 1) + k] = dv[k + i];
      }
      for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int r = c + 1; r < k; ++r)
          if (std::fabs(m[size_t(r) * (k + 1) + c]) > std::fabs(m[size_t(piv) * (k + 1) + c])) piv = r;
        if (piv != c)
          for (int j = 0; j <= k; ++j) std::swap(m[size_t(c) * (k + 1) + j], m[size_t(piv) * (k + 1) + j]);
        for (int r = c + 1; r < k; ++r) {
          const double f = m[size_t(r) * (k + 1) + c] / m[size_t(c) * (k + 1) + c];
          for (int j = c; j <= k; ++j) m[size_t(r) * (k + 1) + j] -= f * m[size_t(c) * (k + 1) + j];
        }
      }
      for (int r = k - 1; r >= 0; --r) {
        double v = m[size_t(r) * (k + 1) + k];
        for (int j = r + 1; j < k; ++j) v -= m[size_t(r) * (k + 1) + j] * G.g[j];
        G.g[r] = v / m[size_t(r) * (k + 1) + r];
      }
      for (int j = 0; j < k; ++j) G.u[j] = bu + size_t(order[j]) * nvec;
    }
    SCF_CUDA(cudaMemcpyAsync(bxp, xvec, size_t(nvec) * 8, cudaMemcpyDeviceToDevice, s));
    SCF_CUDA(cudaMemcpyAsync(bFp, bF, size_t(nvec) * 8, cudaMemcpyDeviceToDevice, s));
    bprev = true;
    broyden_update<<<vgrid, 256, 0, s>>>(nvec, p.mixing, bF, G, xvec);
    SCF_CUDA(cudaGetLastError());
    SCF_CUDA(cudaMemcpyAsync(&fn.mu, xvec + 2 * M, 8, cudaMemcpyDeviceToHost, s));
    SCF_CUDA(cudaStreamSynchronize(s));
  }
  if (it > p.max_iters) it = p.max_iters;

  // the eigenstates of the last matrix become the box's states
  const double isq = 1.0 / std::sqrt(dV);
  for (const Blk& k : blks) {
    const int64_t tot = int64_t(k.g.m) * M;
    const unsigned grid = unsigned((tot + 255) / 256);
    const float* Zs = reinterpret_cast<const float*>(k.Z);
    if (b.prec == WSLDA_MIXED && single)
      unfold_states<float, float2><<<grid, 256, 0, s>>>(k.g, Zs, isq, static_cast<float2*>(b.states) + 2 * k.first * M);
    else if (b.prec == WSLDA_MIXED)
      unfold_states<double, float2><<<grid, 256, 0, s>>>(k.g, k.Z, isq,
                                                         static_cast<float2*>(b.states) + 2 * k.first * M);
    else if (single)
      unfold_states<float, double2><<<grid, 256, 0, s>>>(k.g, Zs, isq,
                                                         static_cast<double2*>(b.states) + 2 * k.first * M);
    else
      unfold_states<double, double2><<<grid, 256, 0, s>>>(k.g, k.Z, isq,
                                                          static_cast<double2*>(b.states) + 2 * k.first * M);
    SCF_CUDA(cudaGetLastError());
  }
  SCF_CUDA(launch_fill(b.sc, 1.0, M, s));
  SCF_CUDA(cudaStreamSynchronize(s));
  if (qpE)
    for (size_t bi = 0; bi < blks.size(); ++bi)
      for (int j = 0; j < blks[bi].g.m; ++j) qpE[blks[bi].first + j] = evals[bi][blks[bi].g.m + j];
  res->iters = it;
  res->converged = converged ? 1 : 0;
  res->mu = fn.mu;
  res->max_rel_change = change;
  res->n_sigma = 0.5 * cur[6];
  res->energy = {cur[0], cur[1], cur[2], cur[3], cur[4], cur[5], cur[6]};
#undef SCF_CUDA
  return WSLDA_OK;
}

}  // namespace wslda
