// Spin-imbalanced ASLDA (Sec. 2.3-2.4): per-site potentials, the fields of H
// that need neighbouring sites, and the energy.
//
// The states are those of the reduced problem of Eq. HpsiEpsi without the
// time-reversal reduction: phi_n = (u_{n,a}, v_{n,b}) over the whole spectrum,
// with frozen weights f(E_n) (w_plus) and f(-E_n) (w_minus). The densities of
// Eqs. na3D..jb3D are
//   rho_a = sum f(E) |u|^2,   rho_b = sum f(-E) |v|^2,   nu = 1/2 sum (f(-E) - f(E)) u v^*,
//   tau_a = sum f(E) |grad u|^2,  tau_b = sum f(-E) |grad v|^2,
//   j_a = -sum f(E) Im(u grad u^*),  j_b = sum f(-E) Im(v grad v^*);
// the host gets them from the spin-symmetric reductions with one weight set
// to zero (the u part alone, then the v part alone).
//
// Functional (Eqs. sldae-functional-generic..sldae-functional with the
// printed ASLDA parametrisation, p = (rho_a - rho_b) / (rho_a + rho_b)):
//   E = sum_s [A_s/2 (tau_s - j_s^2/rho_s) + j_s^2/(2 rho_s)] + 3/5 B(p) rho eF(rho) + g_eff |nu|^2,
//   A_a(p) = A_b(-p) = 1.094 + 0.156 p (1 - 2p^2/3 + p^4/5) - 0.532 p^2 (1 - p^2 + p^4/3),
//   B(p) = 2^(2/3) [0.357 + 0.642 p^2 - A_a(p) ((1+p)/2)^(5/3) - A_b(p) ((1-p)/2)^(5/3)],
//   1/g_eff = rho^(1/3)/C - Lambda_c (reading R1), Delta = -g_eff nu.
// Potentials (Sec. 2.2 list: V_s = dE/d rho_s, alpha_s = 2 dE/d tau_s,
// A_s = dE/d j_s) with Lambda_c held fixed; the p-derivatives of A and B add
// [1/2 (K_a A_a' + K_b A_b') + 3/5 rho eF B'] dp/d rho_s to V_s, K_s = tau_s - j_s^2/rho_s.
// Densities are floored at rho_floor inside these terms (readings R4, A3).
// The regulator follows reading R2 with the spin averages of Sec. 2.6:
// Lambda_c(mu_+ - V_+ - V_ext, E_c, A_+), A_+ = (A_a + A_b)/2, frozen at t = 0
// from the fixed point of V_+ -> Lambda_c -> V_+ reached from V_+ = 0.
#include <cuda_runtime.h>

#include "functional.cuh"
#include "internal.cuh"

namespace wslda {

namespace {

constexpr double kTwo23 = 1.5874010519681994748;  // 2^(2/3)
constexpr int kAsldaRegIters = 60;                 // the same count as the spin-symmetric regulator

__device__ __forceinline__ double aslda_A(double p) {
  const double p2 = p * p;
  return 1.094 + 0.156 * p * (1.0 - 2.0 * p2 / 3.0 + p2 * p2 / 5.0) - 0.532 * p2 * (1.0 - p2 + p2 * p2 / 3.0);
}
// dA_a/dp of the polynomial above: (1 - p^2)^2 (0.156 - 1.064 p)
__device__ __forceinline__ double aslda_dA(double p) {
  const double q = 1.0 - p * p;
  return q * q * (0.156 - 1.064 * p);
}
__device__ __forceinline__ double pow53(double x) { const double c = cbrt(x); return x * c * c; }
__device__ __forceinline__ double pow23(double x) { const double c = cbrt(x); return c * c; }
__device__ __forceinline__ double aslda_B(double p) {
  const double x = 0.5 * (1.0 + p), y = 0.5 * (1.0 - p);
  return kTwo23 * (0.357 + 0.642 * p * p - aslda_A(p) * pow53(x) - aslda_A(-p) * pow53(y));
}
__device__ __forceinline__ double aslda_dB(double p) {
  const double x = 0.5 * (1.0 + p), y = 0.5 * (1.0 - p);
  return kTwo23 * (1.284 * p - aslda_dA(p) * pow53(x) - aslda_A(p) * (5.0 / 6.0) * pow23(x) +
                   aslda_dA(-p) * pow53(y) + aslda_A(-p) * (5.0 / 6.0) * pow23(y));
}

struct SiteIn {
  double ra, rb, ta, tb, nr, ni;
  double ja[3], jb[3];
};
struct SiteOut {
  double Va, Vb, Aa, Ab, dr, di, g;
};

__device__ inline void site_aslda(const SiteIn& d, double lam, double C, double floor_, SiteOut& o) {
  const double ra = fmax(d.ra, floor_), rb = fmax(d.rb, floor_), rt = fmax(d.ra + d.rb, floor_);
  const double p = (d.ra - d.rb) / rt;
  const double ja2 = d.ja[0] * d.ja[0] + d.ja[1] * d.ja[1] + d.ja[2] * d.ja[2];
  const double jb2 = d.jb[0] * d.jb[0] + d.jb[1] * d.jb[1] + d.jb[2] * d.jb[2];
  const double Aa = aslda_A(p), Ab = aslda_A(-p);
  const double dAa = aslda_dA(p), dAb = -aslda_dA(-p);  // d/dp of A_a(p) and of A_b(p) = A_a(-p)
  const double dp_da = 2.0 * rb / (rt * rt), dp_db = -2.0 * ra / (rt * rt);
  const double Ka = d.ta - ja2 / ra, Kb = d.tb - jb2 / rb;
  const double r13 = cbrt(rt);
  const double g = 1.0 / (r13 / C - lam);
  o.dr = -g * d.nr;
  o.di = -g * d.ni;
  const double eF = fermi_energy(rt);
  const double common = aslda_B(p) * eF - (o.dr * o.dr + o.di * o.di) / (3.0 * C * r13 * r13);
  const double shape = 0.5 * (Ka * dAa + Kb * dAb) + 0.6 * rt * eF * aslda_dB(p);
  o.Va = common + shape * dp_da + (Aa - 1.0) * ja2 / (2.0 * ra * ra);
  o.Vb = common + shape * dp_db + (Ab - 1.0) * jb2 / (2.0 * rb * rb);
  o.Aa = Aa;
  o.Ab = Ab;
  o.g = g;
}

// Per-site potentials. part_a / part_b: density partials of the u part
// (weights 0, f(E)) and of the v part (weights f(-E), 0) as [nchunk][3][M];
// tj_a / tj_b: {tau, j_x, j_y, j_z} as [4][M]. Writes rho_a, rho_b, nu
// (interleaved), V_a, V_b, Delta (interleaved) and the per-site scratch
// af[8][M] = alpha_a, alpha_b, A_a (3), A_b (3) for the fields kernel.
__global__ void aslda_potentials_kernel(const double* __restrict__ part_a, const double* __restrict__ part_b,
                                        int nchunk, int M, const double* __restrict__ tj_a,
                                        const double* __restrict__ tj_b, const double* __restrict__ vext,
                                        double mu_a, double mu_b, double C, double ec, double floor_, double* lam,
                                        int init_lam, double* rho_a, double* rho_b, double* nu, double* Va,
                                        double* Vb, double* delta, double* af) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  SiteIn d;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    const double* pa = part_a + int64_t(c) * 3 * M;
    const double* pb = part_b + int64_t(c) * 3 * M;
    a0 += pa[s];
    a1 += pa[M + s];
    a2 += pa[2 * M + s];
    b0 += pb[s];
    b1 += pb[M + s];
    b2 += pb[2 * M + s];
  }
  // u part: rho = sum f(E)|u|^2, nu-sum = -sum f(E) u v^*; v part: rho = sum f(-E)|v|^2, nu-sum = sum f(-E) u v^*
  d.ra = a0;
  d.rb = b0;
  d.nr = 0.5 * (a1 + b1);
  d.ni = 0.5 * (a2 + b2);
  d.ta = tj_a[s];
  d.tb = tj_b[s];
  for (int k = 0; k < 3; ++k) {
    d.ja[k] = tj_a[(1 + k) * M + s];
    d.jb[k] = tj_b[(1 + k) * M + s];
  }
  SiteOut o;
  double l;
  if (init_lam) {
    const double mup = 0.5 * (mu_a + mu_b), ve = vext[s];
    site_aslda(d, 0.0, C, floor_, o);
    const double Ap = 0.5 * (o.Aa + o.Ab);  // A_+ depends on p only, not on the regulator
    double V = 0.0;
    for (int it = 0; it < kAsldaRegIters; ++it) {
      l = regulator(mup - V - ve, ec, Ap);
      site_aslda(d, l, C, floor_, o);
      V = 0.5 * (o.Va + o.Vb);
    }
    l = regulator(mup - V - ve, ec, Ap);
    lam[s] = l;
  } else {
    l = lam[s];
  }
  site_aslda(d, l, C, floor_, o);
  rho_a[s] = d.ra;
  rho_b[s] = d.rb;
  nu[2 * s] = d.nr;
  nu[2 * s + 1] = d.ni;
  Va[s] = o.Va;
  Vb[s] = o.Vb;
  delta[2 * s] = o.dr;
  delta[2 * s + 1] = o.di;
  const double ra = fmax(d.ra, floor_), rb = fmax(d.rb, floor_);
  af[s] = o.Aa;
  af[M + s] = o.Ab;
  for (int k = 0; k < 3; ++k) {
    af[(2 + k) * M + s] = (1.0 - o.Aa) * d.ja[k] / ra;
    af[(5 + k) * M + s] = (1.0 - o.Ab) * d.jb[k] / rb;
  }
}

// Fields of H that need neighbouring sites: lap alpha_s by the circulant
// columns of the Eq. D2 matrices (d2, Nyquist kept, the Laplacian of H) and
// div A_s by those of the first-derivative matrices (d1, Nyquist zeroed),
// as direct sums along each axis. Writes
//   WD  = {V_a + V_ext - mu_a + lap(alpha_a)/4, Re Delta, Im Delta + Delta_ext, V_b + V_ext - mu_b + lap(alpha_b)/4}
//   alf = {alpha_a / 2, alpha_b / 2},  av_a = {A_a, div A_a / 2},  av_b = {A_b, div A_b / 2}.
template <typename R>
__global__ void aslda_fields_kernel(int nx, int ny, int nz, const double* __restrict__ af,
                                    const double* __restrict__ Va, const double* __restrict__ Vb,
                                    const double* __restrict__ delta, const double* __restrict__ vext,
                                    const double* __restrict__ dext, double mu_a, double mu_b,
                                    const double* __restrict__ d1, const double* __restrict__ d2, fx4<R>* WD,
                                    cx<R>* alf, fx4<R>* av_a, fx4<R>* av_b) {
  const int M = nx * ny * nz;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  const int x = s / (ny * nz), y = (s / nz) % ny, z = s % nz;
  const int n3[3] = {nx, ny, nz};
  const int off[3] = {0, nx, nx + ny};
  double lapa = 0.0, lapb = 0.0, diva = 0.0, divb = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    const int N = n3[ax];
    const int pos = ax == 0 ? x : (ax == 1 ? y : z);
    for (int l = 0; l < N; ++l) {
      const int site = ax == 0 ? (l * ny + y) * nz + z : (ax == 1 ? (x * ny + l) * nz + z : (x * ny + y) * nz + l);
      const int k = (pos - l + N) % N;
      lapa += d2[off[ax] + k] * af[site];
      lapb += d2[off[ax] + k] * af[M + site];
      diva += d1[off[ax] + k] * af[(2 + ax) * M + site];
      divb += d1[off[ax] + k] * af[(5 + ax) * M + site];
    }
  }
  const double ve = vext[s];
  fx4<R> w;
  w.x = R(Va[s] + ve - mu_a + 0.25 * lapa);
  w.y = R(delta[2 * s] + dext[2 * s]);
  w.z = R(delta[2 * s + 1] + dext[2 * s + 1]);
  w.w = R(Vb[s] + ve - mu_b + 0.25 * lapb);
  WD[s] = w;
  cx<R> al;
  al.x = R(0.5 * af[s]);
  al.y = R(0.5 * af[M + s]);
  alf[s] = al;
  fx4<R> pa, pb;
  pa.x = R(af[2 * M + s]);
  pa.y = R(af[3 * M + s]);
  pa.z = R(af[4 * M + s]);
  pa.w = R(0.5 * diva);
  pb.x = R(af[5 * M + s]);
  pb.y = R(af[6 * M + s]);
  pb.z = R(af[7 * M + s]);
  pb.w = R(0.5 * divb);
  av_a[s] = pa;
  av_b[s] = pb;
}

// Energy terms (one block, fixed-order sums in double):
// out8 = e_kin (sum_s A_s tau_s / 2), e_pot (3/5 B rho eF), e_pair (g |nu|^2),
// e_ext (V_ext (rho_a + rho_b)), e_pair_ext (-2 Re(Delta_ext nu^*), as for the
// spin-symmetric functional), e_total, n_part (N_a + N_b), e_cur
// (sum_s (1 - A_s) j_s^2 / (2 rho_s)); then N_a, N_b; every term integrated with dV.
__global__ void __launch_bounds__(1024) aslda_energy_kernel(int M, const double* __restrict__ rho_a,
                                                            const double* __restrict__ rho_b,
                                                            const double* __restrict__ nu,
                                                            const double* __restrict__ tj_a,
                                                            const double* __restrict__ tj_b,
                                                            const double* __restrict__ lam,
                                                            const double* __restrict__ vext,
                                                            const double* __restrict__ dext, double C,
                                                            double floor_, double dV, double* out8) {
  __shared__ double sh[9][32];
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int s = threadIdx.x; s < M; s += blockDim.x) {
    SiteIn d;
    d.ra = rho_a[s];
    d.rb = rho_b[s];
    d.nr = nu[2 * s];
    d.ni = nu[2 * s + 1];
    d.ta = tj_a[s];
    d.tb = tj_b[s];
    for (int k = 0; k < 3; ++k) {
      d.ja[k] = tj_a[(1 + k) * M + s];
      d.jb[k] = tj_b[(1 + k) * M + s];
    }
    SiteOut o;
    site_aslda(d, lam[s], C, floor_, o);
    const double ra = fmax(d.ra, floor_), rb = fmax(d.rb, floor_), rt = fmax(d.ra + d.rb, floor_);
    const double p = (d.ra - d.rb) / rt;
    const double ja2 = d.ja[0] * d.ja[0] + d.ja[1] * d.ja[1] + d.ja[2] * d.ja[2];
    const double jb2 = d.jb[0] * d.jb[0] + d.jb[1] * d.jb[1] + d.jb[2] * d.jb[2];
    acc[0] += 0.5 * (o.Aa * d.ta + o.Ab * d.tb) * dV;
    acc[1] += 0.6 * aslda_B(p) * rt * fermi_energy(rt) * dV;
    acc[2] += o.g * (d.nr * d.nr + d.ni * d.ni) * dV;
    acc[3] += vext[s] * (d.ra + d.rb) * dV;
    acc[4] += -2.0 * (dext[2 * s] * d.nr + dext[2 * s + 1] * d.ni) * dV;
    acc[5] += (d.ra + d.rb) * dV;
    acc[6] += (0.5 * (1.0 - o.Aa) * ja2 / ra + 0.5 * (1.0 - o.Ab) * jb2 / rb) * dV;
    acc[7] += d.ra * dV;
    acc[8] += d.rb * dV;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < 9; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[9];
    for (int k = 0; k < 9; ++k) {
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
    out8[8] = t[7];
    out8[9] = t[8];
  }
}

}  // namespace

cudaError_t launch_aslda_potentials(const double* part_a, const double* part_b, int nchunk, int M, const double* tj_a,
                                    const double* tj_b, const double* vext, double mu_a, double mu_b, double C,
                                    double ec, double rho_floor, double* lam, int init_lam, double* rho_a,
                                    double* rho_b, double* nu, double* Va, double* Vb, double* delta, double* af,
                                    cudaStream_t s) {
  aslda_potentials_kernel<<<(M + 127) / 128, 128, 0, s>>>(part_a, part_b, nchunk, M, tj_a, tj_b, vext, mu_a, mu_b, C,
                                                          ec, rho_floor, lam, init_lam, rho_a, rho_b, nu, Va, Vb,
                                                          delta, af);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_aslda_fields(int nx, int ny, int nz, const double* af, const double* Va, const double* Vb,
                                const double* delta, const double* vext, const double* dext, double mu_a, double mu_b,
                                const double* d1, const double* d2, fx4<R>* WD, cx<R>* alf, fx4<R>* av_a,
                                fx4<R>* av_b, cudaStream_t s) {
  const int M = nx * ny * nz;
  aslda_fields_kernel<R><<<(M + 127) / 128, 128, 0, s>>>(nx, ny, nz, af, Va, Vb, delta, vext, dext, mu_a, mu_b, d1,
                                                         d2, WD, alf, av_a, av_b);
  return cudaGetLastError();
}
template cudaError_t launch_aslda_fields<float>(int, int, int, const double*, const double*, const double*,
                                                const double*, const double*, const double*, double, double,
                                                const double*, const double*, float4*, float2*, float4*, float4*,
                                                cudaStream_t);
template cudaError_t launch_aslda_fields<double>(int, int, int, const double*, const double*, const double*,
                                                 const double*, const double*, const double*, double, double,
                                                 const double*, const double*, double4*, double2*, double4*,
                                                 double4*, cudaStream_t);

cudaError_t launch_aslda_energy(int M, const double* rho_a, const double* rho_b, const double* nu, const double* tj_a,
                                const double* tj_b, const double* lam, const double* vext, const double* dext, double C,
                                double rho_floor, double dV, double* out8, cudaStream_t s) {
  aslda_energy_kernel<<<1, 1024, 0, s>>>(M, rho_a, rho_b, nu, tj_a, tj_b, lam, vext, dext, C, rho_floor, dV, out8);
  return cudaGetLastError();
}

}  // namespace wslda
