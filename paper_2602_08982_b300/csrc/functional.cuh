// Pointwise functional (Sec. 2.4) and regulator (Sec. 2.6, Eq. Creg) at one
// lattice site, shared by the time-dependent potentials and the static solver.
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"

namespace wslda {

// ---------------------------------------------------------------------------
// Functional (Sec. 2.4) and regulator (Sec. 2.6) at one site.
// ---------------------------------------------------------------------------
__device__ inline double regulator(double mu_minus_V, double ec, double A = 1.0) {
  // Lambda_c = (1/2 pi^2) PV int_0^kc k^2 dk / (A k^2 - A k0^2):
  // A k0^2 / 2 = mu - V, A kc^2 / 2 = E_c + mu - V (A_+ = A, spin-symmetric).
  const double k0sq = 2.0 * mu_minus_V / A;
  const double kcsq = 2.0 * (ec + mu_minus_V) / A;
  if (!(kcsq > 0.0)) return 0.0;
  const double kc = sqrt(kcsq);
  const double pref = kc / (2.0 * M_PI * M_PI * A);
  if (k0sq > 0.0) {
    const double k0 = sqrt(k0sq);
    return pref * (1.0 - (k0 / (2.0 * kc)) * log((kc + k0) / (kc - k0)));
  }
  if (k0sq < 0.0) {
    const double kap = sqrt(-k0sq);
    return pref * (1.0 - (kap / kc) * atan2(kc, kap));
  }
  return pref;
}

__device__ __forceinline__ double fermi_energy(double rho_total) {
  const double c = cbrt(3.0 * M_PI * M_PI * rho_total);
  return 0.5 * c * c;
}

// (U, Delta) at one site from rho_sigma, nu and the regulator value lam.
__device__ inline void site_potentials(const FunctionalDev& fn, double rho_s, double nr, double ni, double lam, double& U,
                                double& dr, double& di) {
  double inv_g;
  double rho = 2.0 * rho_s;
  if (fn.kind == 0) {
    rho = fmax(rho, fn.rho_floor);
    inv_g = cbrt(rho) / fn.C - lam;
  } else {
    inv_g = fn.inv_4pi_a - lam;
  }
  const double g = 1.0 / inv_g;
  dr = -g * nr;
  di = -g * ni;
  if (fn.kind == 0) {
    const double r13 = cbrt(rho);
    U = fn.B * fermi_energy(rho) - (dr * dr + di * di) / (3.0 * fn.C * r13 * r13);
  } else {
    U = 0.0;
  }
}

}  // namespace wslda
