"""Plain FP64 CPU oracle of the static self-consistent solver (Alg. 1, Sec. 3.2).

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import or run anything in this package; the
product path never does, and this module never imports the product.

The static problem (Eq. HpsiEpsi) is solved as the fixed point K[p] = p of the
map of Alg. 1 over the potentials p = (U, Delta) (the potential-based
formulation the toolkit uses by default), iterated with linear mixing
p <- m K[p] + (1 - m) p and stopped by the energy criterion of Eq. E-conv.
One application of K, with no blocking, symmetry reduction or reordering:

  1. build the 2M x 2M matrix of Eq. HpsiEpsi from the input potentials
     (W = U + V_ext - mu, D = Delta + Delta_ext; Laplacian of Eq. D2);
  2. diagonalise it (numpy.linalg.eigh, one library step) and keep the M
     eigenpairs with E_n > 0, normalised as sum_r dV (|u|^2 + |v|^2) = 1;
  3. densities rho_sigma, nu of those states (T = 0 weights);
  4. potentials (U, Delta) from the densities, the regulator Lambda_c
     recomputed from the input mean field (reading K1).

Readings (the same on the CUDA side):
  K1  Lambda_c of Eq. Creg is evaluated every iteration at V = U_in + V_ext
      with the input mean field of that iteration (it is frozen only during
      time evolution, reading R2 of the TD oracle).
  K2  The energy scale of Eq. E-conv is the Fermi energy of the reference
      uniform system (1/2 for k_F = 1); every energy term listed in Sec. 3.2
      that the functional has (kinetic, potential, pairing, external
      potential, external pairing) and their total must change by less than
      eps_energy times that scale between two consecutive iterations.
  K3  With a particle-number target, Eq. update-mu is one more step of the
      map (as Sec. 3.2 puts it), so mu_out joins the mixed vector: linear
      mixing gives mu <- m mu_out + (1 - m) mu, and Broyden mixing carries mu
      as one more component. N counts one spin species, N_sigma = int rho_sigma.
  K4  The first iteration has no predecessor, so convergence is tested from
      the second iteration on; the returned states are the eigenstates of
      the last matrix diagonalised, and the returned potentials are its input.
  K5  The Broyden option (Sec. 3.2 lists it beside linear mixing) is the
      modified Broyden mixing of D. D. Johnson, Phys. Rev. B 38, 12807 (1988),
      in the form used for nuclear DFT by A. Baran et al., Phys. Rev. C 78,
      014318 (2008): all weights 1, w_0 = 0.01, the last 7 iterations kept, on
      the vector p = (U, Re Delta) (real problems). The first iteration mixes
      linearly.

Pins (tests/test_oracle_scf.py): uniform BdG and SLDA fixed points equal the
lattice seeds solved from the number and gap equations alone, the BdG
spectrum is +/- symmetric, a converged trapped solution is a fixed point of K
and is stationary under the TD right-hand side, the mixing parameter does not
move the fixed point, and the mu update reaches the requested N.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from . import tdslda as o

ENERGY_TERMS = ("e_kin", "e_pot", "e_pair", "e_ext", "e_pair_ext", "e_total")


@dataclass
class MapOutput:
    phi: np.ndarray       # [M, 2, M] eigenstates with E_n > 0, ascending E
    E: np.ndarray         # [M] their quasiparticle energies
    evals: np.ndarray     # [2M] full spectrum of the matrix
    rho: np.ndarray       # rho_sigma
    nu: np.ndarray
    U: np.ndarray         # output potentials K[p]
    delta: np.ndarray
    lam: np.ndarray       # regulator used (reading K1)
    energy: dict


def map_K(lat: o.Lattice, fn: o.Functional, vext, U_in, delta_in, dext=None) -> MapOutput:
    """One application of the map K of Alg. 1 (steps 1-5)."""
    # step 1: the matrix of Eq. HpsiEpsi at the input potentials
    D = delta_in if dext is None else delta_in + dext
    H = o.dense_bdg(o.Fields(W=U_in + vext - fn.mu, D=D), lat)
    # step 2: diagonalise, keep E > 0 (M of the 2M eigenvalues for this problem)
    evals, vecs = np.linalg.eigh(H)
    M = lat.M
    keep = np.argsort(evals)[M:]
    E = evals[keep]
    phi = vecs[:, keep].T.reshape(M, 2, M) / np.sqrt(lat.dV)
    # step 3: densities (T = 0)
    wm, wp = np.ones(M), np.zeros(M)
    rho, nu = o.densities(phi, wm, wp)
    # step 4: potentials, regulator at the input mean field (reading K1)
    lam = o.lambda_c(fn.mu - U_in - vext, fn.cutoff(lat))
    U_out, delta_out, _ = o.potentials(rho, nu, lam, fn)
    sysm = o.TDSystem(lat, fn, vext=vext, dext=dext, lam=lam)
    energy = sysm.energy(phi)
    return MapOutput(phi=phi, E=E, evals=evals, rho=rho, nu=nu, U=U_out, delta=delta_out, lam=lam, energy=energy)


@dataclass
class SCFResult:
    phi: np.ndarray
    E: np.ndarray
    U: np.ndarray          # input potentials of the last map application
    delta: np.ndarray
    mu: float
    iters: int
    converged: bool
    last: MapOutput
    history: list = field(default_factory=list)    # energy dict per iteration


class Broyden:
    """Modified Broyden mixing (reading K5). With p_n the input and
    F_n = K[p_n] - p_n the residual of iteration n, each step stores
    dF = (F_n - F_{n-1}) / |F_n - F_{n-1}|, u = alpha dF + (p_n - p_{n-1}) / |F_n - F_{n-1}|
    and proposes p_{n+1} = p_n + alpha F_n - sum_j gamma_j u_j with
    gamma = c (w0^2 I + A)^{-1}, A_ij = dF_i . dF_j, c_i = dF_i . F_n."""

    def __init__(self, alpha: float, memory: int = 7, w0: float = 0.01):
        self.alpha, self.memory, self.w0 = alpha, memory, w0
        self.dF, self.u = [], []
        self.prev = None

    def next(self, p, F):
        if self.prev is not None:
            p0, F0 = self.prev
            d = F - F0
            nrm = np.sqrt(d @ d)
            self.dF.append(d / nrm)
            self.u.append(self.alpha * d / nrm + (p - p0) / nrm)
            self.dF, self.u = self.dF[-self.memory:], self.u[-self.memory:]
        self.prev = (p.copy(), F.copy())
        step = p + self.alpha * F
        if self.dF:
            k = len(self.dF)
            A = np.array([[self.dF[i] @ self.dF[j] for j in range(k)] for i in range(k)])
            beta = np.linalg.inv(self.w0 ** 2 * np.eye(k) + A)
            c = np.array([self.dF[i] @ F for i in range(k)])
            gamma = c @ beta
            step = step - sum(gamma[j] * self.u[j] for j in range(k))
        return step


def static_solve(lat: o.Lattice, fn: o.Functional, vext, U0, delta0, mixing: float = 0.5,
                 eps_energy: float = 1e-6, e_ref: float = 0.5, max_iters: int = 200,
                 n_target: float | None = None, a_mu: float = 0.0, eps_npart: float = 1e-6,
                 dext=None, method: str = "linear", broyden_memory: int = 7,
                 broyden_w0: float = 0.01) -> SCFResult:
    """Linear mixing (Sec. 3.2, 'Linear mixing') or modified Broyden mixing
    (reading K5) of the potentials until the energy criterion of Eq. E-conv
    holds (and Eq. N-conv with a target N). The Broyden option requires real
    potentials."""
    U = np.array(U0, dtype=np.float64)
    delta = np.array(delta0, dtype=np.complex128)
    mu = fn.mu
    mixer = Broyden(mixing, broyden_memory, broyden_w0) if method == "broyden" else None
    hist = []
    out = None
    converged = False
    it = 0
    for it in range(1, max_iters + 1):
        out = map_K(lat, replace(fn, mu=mu), vext, U, delta, dext)
        hist.append(out.energy)
        n_sigma = lat.dV * np.sum(out.rho)
        n_ok = n_target is None or abs(n_target - n_sigma) < eps_npart
        if it >= 2:
            prev = hist[-2]
            change = max(abs(out.energy[k] - prev[k]) / e_ref for k in ENERGY_TERMS)
            if change < eps_energy and n_ok:
                converged = True
                break
        if it == max_iters:
            break
        # Eq. update-mu is a step of the map: mu_out joins the mixed vector (reading K3)
        mu_out = mu + (a_mu / n_target) * (n_target - n_sigma) if n_target is not None else mu
        if mixer is None:
            U = mixing * out.U + (1.0 - mixing) * U
            delta = mixing * out.delta + (1.0 - mixing) * delta
            mu = mixing * mu_out + (1.0 - mixing) * mu
        else:
            p = np.concatenate([U, delta.real, [mu]])
            F = np.concatenate([out.U, out.delta.real, [mu_out]]) - p
            p = mixer.next(p, F)
            U, delta, mu = p[:lat.M], p[lat.M:2 * lat.M] + 0j, float(p[-1])
    return SCFResult(phi=out.phi, E=out.E, U=U, delta=delta, mu=mu, iters=it, converged=converged,
                     last=out, history=hist)
