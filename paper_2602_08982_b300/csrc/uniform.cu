// Uniform BCS solution on the lattice k-set (Sec. 5.2.1, "inittype 0": the
// default initial state of the toolkit) and the device kernel that writes its
// plane-wave quasiparticle states.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "../../include/wslda_td.h"

namespace {

// Lambda_c of Eq. Creg (A = 1) as a principal-value integral; for mu < V the
// integral has no pole (arctan form); zero when k_c^2 <= 0.
double regulator_host(double mu_minus_V, double ec) {
  const double k0sq = 2.0 * mu_minus_V, kcsq = 2.0 * (ec + mu_minus_V);
  if (!(kcsq > 0.0)) return 0.0;
  const double kc = std::sqrt(kcsq), pref = kc / (2.0 * M_PI * M_PI);
  if (k0sq > 0.0) {
    const double k0 = std::sqrt(k0sq);
    return pref * (1.0 - (k0 / (2.0 * kc)) * std::log((kc + k0) / (kc - k0)));
  }
  if (k0sq < 0.0) {
    const double kap = std::sqrt(-k0sq);
    return pref * (1.0 - (kap / kc) * std::atan2(kc, kap));
  }
  return pref;
}

double kaxis(int l, int n, double d) {
  const double L = n * d;
  return l < n / 2 ? 2.0 * M_PI * l / L : 2.0 * M_PI * (l - n) / L;
}

std::vector<double> half_k2(const wslda_lattice& lat) {
  std::vector<double> out;
  out.reserve(size_t(lat.nx) * lat.ny * lat.nz);
  for (int a = 0; a < lat.nx; ++a)
    for (int b = 0; b < lat.ny; ++b)
      for (int c = 0; c < lat.nz; ++c) {
        const double kx = kaxis(a, lat.nx, lat.dx), ky = kaxis(b, lat.ny, lat.dy), kz = kaxis(c, lat.nz, lat.dz);
        out.push_back(0.5 * (kx * kx + ky * ky + kz * kz));
      }
  return out;
}

// (1/V) sum_k V_k^2 and (1/V) sum_k 1/(2 E_k)
void sums(const std::vector<double>& e, double me, double d, double vol, double& dens, double& inv2e) {
  double s1 = 0.0, s2 = 0.0;
  for (double ek : e) {
    const double xi = ek - me, E = std::sqrt(xi * xi + d * d);
    s1 += 0.5 * (1.0 - xi / E);
    s2 += 1.0 / (2.0 * E);
  }
  dens = s1 / vol;
  inv2e = s2 / vol;
}

// mu_eff from the number equation by bisection (density grows with mu_eff).
double solve_mu_eff(const std::vector<double>& e, double d, double vol, double rho_s) {
  double emax = 0.0;
  for (double x : e) emax = std::max(emax, x);
  double lo = -50.0, hi = emax + 50.0;
  for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    double dens, ie;
    sums(e, mid, d, vol, dens, ie);
    (dens < rho_s ? lo : hi) = mid;
  }
  return 0.5 * (lo + hi);
}

// partners = 0: n states (U_k, V_k) e^{ik.r}/sqrt(V). partners = 1: states
// n/2 .. n-1 are the negative-energy partners [v^*, -u^*] of states 0 .. n/2-1
// (the whole spectrum of the spin-imbalanced problem, Eq. HpsiEpsi).
__global__ void fill_plane_waves(double2* out_d, float2* out_f, int nx, int ny, int nz, double dx, double dy,
                                 double dz, double mu_eff, double delta, const int64_t* kidx, int64_t n,
                                 int partners) {
  const int64_t M = int64_t(nx) * ny * nz;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= n * M) return;
  const int64_t st = idx / M, r = idx % M;
  const int64_t half = partners ? n / 2 : n;
  const bool partner = partners && st >= half;
  const int64_t sk = partner ? st - half : st;
  const int64_t k = kidx ? kidx[sk] : sk;
  const int lx = int(k / (int64_t(ny) * nz)), ly = int((k / nz) % ny), lz = int(k % nz);
  const int ix = int(r / (int64_t(ny) * nz)), iy = int((r / nz) % ny), iz = int(r % nz);
  auto kv = [](int l, int nn, double d) {
    const double L = nn * d;
    return l < nn / 2 ? 2.0 * M_PI * l / L : 2.0 * M_PI * (l - nn) / L;
  };
  const double kx = kv(lx, nx, dx), ky = kv(ly, ny, dy), kz = kv(lz, nz, dz);
  const double xi = 0.5 * (kx * kx + ky * ky + kz * kz) - mu_eff;
  const double E = sqrt(xi * xi + delta * delta);
  const double vol = double(M) * dx * dy * dz;
  const double Uk = sqrt(0.5 * (1.0 + xi / E)) / sqrt(vol);
  const double Vk = sqrt(0.5 * (1.0 - xi / E)) / sqrt(vol);
  // phase k.r = 2 pi (lx ix / nx + ly iy / ny + lz iz / nz), reduced exactly
  const double frac = double((int64_t(lx) * ix) % nx) / nx + double((int64_t(ly) * iy) % ny) / ny +
                      double((int64_t(lz) * iz) % nz) / nz;
  double s, c;
  sincospi(2.0 * frac, &s, &c);
  const int64_t base = st * 2 * M + r;
  // partner: u = conj(V_k e^{ik.r}) = V_k e^{-ik.r}, v = -conj(U_k e^{ik.r}) = -U_k e^{-ik.r}
  const double ur = partner ? Vk * c : Uk * c, ui = partner ? -Vk * s : Uk * s;
  const double vr = partner ? -Uk * c : Vk * c, vi = partner ? Uk * s : Vk * s;
  if (out_d) {
    out_d[base] = make_double2(ur, ui);
    out_d[base + M] = make_double2(vr, vi);
  } else {
    out_f[base] = make_float2(float(ur), float(ui));
    out_f[base + M] = make_float2(float(vr), float(vi));
  }
}

}  // namespace

namespace wslda {
cudaError_t launch_fill_plane_waves(void* dst, int is_float, const wslda_lattice& lat, double mu_eff, double delta,
                                    const int64_t* kidx_dev, int64_t n, int partners, cudaStream_t s) {
  const int64_t M = int64_t(lat.nx) * lat.ny * lat.nz;
  const int64_t total = n * M;
  if (total == 0) return cudaSuccess;
  fill_plane_waves<<<unsigned((total + 255) / 256), 256, 0, s>>>(
      is_float ? nullptr : static_cast<double2*>(dst), is_float ? static_cast<float2*>(dst) : nullptr, lat.nx,
      lat.ny, lat.nz, lat.dx, lat.dy, lat.dz, mu_eff, delta, kidx_dev, n, partners);
  return cudaGetLastError();
}
}  // namespace wslda

extern "C" wslda_status wslda_uniform_solve(const wslda_lattice* lat, const wslda_functional* fn, double rho_sigma,
                                            double delta0, wslda_uniform* out) {
  if (!lat || !fn || !out || !(rho_sigma > 0.0)) return WSLDA_EINVAL;
  if (lat->nx <= 0 || lat->ny <= 0 || lat->nz <= 0 || !(lat->dx > 0 && lat->dy > 0 && lat->dz > 0))
    return WSLDA_EINVAL;
  const std::vector<double> e = half_k2(*lat);
  const double vol = double(e.size()) * lat->dx * lat->dy * lat->dz;
  const double ec = fn->ec > 0 ? fn->ec
                               : 0.5 * M_PI * M_PI *
                                     (1.0 / (lat->dx * lat->dx) + 1.0 / (lat->dy * lat->dy) + 1.0 / (lat->dz * lat->dz));
  const double rho = 2.0 * rho_sigma;
  if (fn->kind == WSLDA_FUNC_SLDA_A1) {
    if (!(delta0 > 0.0)) return WSLDA_EINVAL;
    const double me = solve_mu_eff(e, delta0, vol, rho_sigma);
    double dens, ie;
    sums(e, me, delta0, vol, dens, ie);
    const double inv_g = -ie, lam = regulator_host(me, ec);
    const double C = std::cbrt(rho) / (inv_g + lam);
    const double ef = 0.5 * std::pow(std::cbrt(3.0 * M_PI * M_PI * rho), 2.0);
    const double U = fn->B * ef - delta0 * delta0 / (3.0 * C * std::cbrt(rho) * std::cbrt(rho));
    *out = {me, delta0, U + me, U, C, lam, inv_g};
    return WSLDA_OK;
  }
  if (fn->kind != WSLDA_FUNC_BDG) return WSLDA_EINVAL;
  auto residual = [&](double d, double& me_out) {
    const double me = solve_mu_eff(e, d, vol, rho_sigma);
    double dens, ie;
    sums(e, me, d, vol, dens, ie);
    me_out = me;
    return fn->inv_4pi_a - regulator_host(me, ec) + ie;
  };
  const int ng = 80;
  double prev_d = 1e-6, me;
  double prev_r = residual(prev_d, me);
  for (int i = 1; i < ng; ++i) {
    const double d = 1e-6 * std::pow(8.0 / 1e-6, double(i) / (ng - 1));
    const double r = residual(d, me);
    if (prev_r > 0.0 && r <= 0.0) {
      double lo = prev_d, hi = d;
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        (residual(mid, me) > 0.0 ? lo : hi) = mid;
      }
      const double dd = 0.5 * (lo + hi);
      residual(dd, me);
      double dens, ie;
      sums(e, me, dd, vol, dens, ie);
      *out = {me, dd, me, 0.0, NAN, regulator_host(me, ec), -ie};
      return WSLDA_OK;
    }
    prev_d = d;
    prev_r = r;
  }
  return WSLDA_EINVAL;  // no superfluid root on this lattice
}
