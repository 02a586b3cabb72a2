"""Plain FP64 CPU oracle of the spin-imbalanced ASLDA time-dependent step.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import or run anything in this package; the
product path never does, and this module never imports the product.

What it computes (the paper's general SLDA-type formulation, Secs. 2.2-2.4):
  * states of the reduced problem of Eq. HpsiEpsi, phi[n, 0] = u_{n,a},
    phi[n, 1] = v_{n,b}, with the whole spectrum (both signs of E_n, no
    time-reversal reduction) and frozen weights fp[n] = f(E_n), fm[n] = f(-E_n);
  * densities of Eqs. na3D..jb3D (rho_a, rho_b, tau_a, tau_b, nu, j_a, j_b);
  * the ASLDA functional (Eqs. sldae-functional-generic..sldae-functional with
    the printed A_a(p) = A_b(-p), B(p), C(p) = -11.11, p = (rho_a - rho_b) /
    (rho_a + rho_b)) and its potentials V_sigma = dE/d rho_sigma, alpha_sigma =
    2 dE/d tau_sigma, A_sigma = dE/d j_sigma, Delta = -dE/d nu^* (Sec. 2.2 list);
  * h_sigma of Eq. h_sigma with the kinetic operator of Eq. kinop-alpha (the
    alpha_sigma vary in space through p) and the current term -(i/2){A, grad};
  * f = -i [H - <H>_n] phi with H of Eq. HpsiEpsi (mu_a and mu_b on the
    diagonal), for the ABM integrators of tdslda.py.

Readings (shared with tdslda.py where they overlap): R1 coupling, R2 frozen
regulator (here with A_+ = (A_a + A_b)/2, V_+ and mu_+ of Sec. 2.6), R4 floors,
A2 anticommutator form. B1: tau_sigma in the energy uses the Nyquist-free
spectral gradient (Eqs. na3D..jb3D as printed); no external pairing field.

Pins (tests/test_oracle_aslda.py): the potentials equal central finite
differences of the pointwise energy density; the printed A(p), B(p) give the
normal-state energies of the unpolarised (xi_N = 2^(2/3) 0.357) and fully
polarised (0.357 + 0.642) uniform gas; Eq. kinop-alpha equals
-1/2 sum_d d_d (alpha d_d f) for band-limited alpha and f; at p = 0 the
imbalanced formulation with each state's time-reversed partner reproduces the
spin-symmetric A = 1.094 oracle (densities, potentials, f, and AB4AM5
evolution); and the energy of a Galilean boost changes by q.P + N q^2 / 2
with p != 0.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import tdslda as t

C_ASLDA = t.C_ASLDA
TWO23 = 2.0 ** (2.0 / 3.0)


# ----------------------------------------------------------------------------
# Functional parameters (Sec. 2.4, ASLDA) and their p-derivatives
# ----------------------------------------------------------------------------
def A_a(p):
    return t.aslda_A(p)


def dA_a(p):
    """d A_a / dp; the printed polynomial differentiates to (1 - p^2)^2 (0.156 - 1.064 p)."""
    return (1.0 - p * p) ** 2 * (0.156 - 1.064 * p)


def B(p):
    return t.aslda_B(p)


def dB(p):
    """d B / dp of B(p) = 2^(2/3) [0.357 + 0.642 p^2 - A_a(p) x^(5/3) - A_a(-p) y^(5/3)],
    x = (1 + p)/2, y = (1 - p)/2."""
    x, y = 0.5 * (1.0 + p), 0.5 * (1.0 - p)
    return TWO23 * (1.284 * p - dA_a(p) * x ** (5.0 / 3.0) - A_a(p) * (5.0 / 6.0) * x ** (2.0 / 3.0)
                    + dA_a(-p) * y ** (5.0 / 3.0) + A_a(-p) * (5.0 / 6.0) * y ** (2.0 / 3.0))


@dataclass
class ASLDA:
    """Chemical potentials of the two species and the regularised coupling."""
    mu_a: float
    mu_b: float
    C: float = C_ASLDA
    ec: float = -1.0          # <= 0: zone-corner cutoff (reading R5)
    rho_floor: float = 1e-12  # reading R4 / A3

    def cutoff(self, lat: t.Lattice) -> float:
        return self.ec if self.ec > 0 else t.lattice_cutoff(lat)


# ----------------------------------------------------------------------------
# Densities (Eqs. na3D..jb3D)
# ----------------------------------------------------------------------------
@dataclass
class Densities:
    rho_a: np.ndarray
    rho_b: np.ndarray
    tau_a: np.ndarray
    tau_b: np.ndarray
    nu: np.ndarray
    j_a: np.ndarray   # [3][M]
    j_b: np.ndarray


def densities(phi, fp, fm, lat: t.Lattice) -> Densities:
    u, v = phi[:, 0, :], phi[:, 1, :]
    gu, gv = t.gradient(u, lat), t.gradient(v, lat)
    rho_a = np.einsum("n,nr->r", fp, np.abs(u) ** 2)
    rho_b = np.einsum("n,nr->r", fm, np.abs(v) ** 2)
    tau_a = sum(np.einsum("n,nr->r", fp, np.abs(gu[d]) ** 2) for d in range(3))
    tau_b = sum(np.einsum("n,nr->r", fm, np.abs(gv[d]) ** 2) for d in range(3))
    nu = 0.5 * np.einsum("n,nr->r", fm - fp, u * np.conj(v))
    j_a = np.stack([-np.einsum("n,nr->r", fp, np.imag(u * np.conj(gu[d]))) for d in range(3)])
    j_b = np.stack([np.einsum("n,nr->r", fm, np.imag(v * np.conj(gv[d]))) for d in range(3)])
    return Densities(rho_a, rho_b, tau_a, tau_b, nu, j_a, j_b)


# ----------------------------------------------------------------------------
# Energy density and potentials (pointwise)
# ----------------------------------------------------------------------------
def _floored(d: Densities, fn: ASLDA):
    ra = np.maximum(d.rho_a, fn.rho_floor)
    rb = np.maximum(d.rho_b, fn.rho_floor)
    rt = np.maximum(d.rho_a + d.rho_b, fn.rho_floor)
    p = (d.rho_a - d.rho_b) / rt
    return ra, rb, rt, p


def coupling(d: Densities, lam, fn: ASLDA):
    """g_eff with 1/g_eff = rho_+^(1/3) / C - Lambda_c (reading R1)."""
    _, _, rt, _ = _floored(d, fn)
    return 1.0 / (np.cbrt(rt) / fn.C - lam)


def energy_density(d: Densities, lam, fn: ASLDA):
    """sum_s [A_s/2 (tau_s - j_s^2/rho_s) + j_s^2/(2 rho_s)] + 3/5 B rho eF(rho) + g_eff |nu|^2."""
    ra, rb, rt, p = _floored(d, fn)
    ja2, jb2 = np.sum(d.j_a ** 2, axis=0), np.sum(d.j_b ** 2, axis=0)
    e = 0.5 * A_a(p) * (d.tau_a - ja2 / ra) + 0.5 * A_a(-p) * (d.tau_b - jb2 / rb)
    e = e + 0.5 * ja2 / ra + 0.5 * jb2 / rb
    e = e + 0.6 * B(p) * rt * t.fermi_energy(rt)
    return e + coupling(d, lam, fn) * np.abs(d.nu) ** 2


@dataclass
class Potentials:
    V_a: np.ndarray
    V_b: np.ndarray
    alpha_a: np.ndarray
    alpha_b: np.ndarray
    Avec_a: np.ndarray
    Avec_b: np.ndarray
    Delta: np.ndarray
    g: np.ndarray


def potentials(d: Densities, lam, fn: ASLDA) -> Potentials:
    """Functional derivatives of energy_density with Lambda_c held fixed."""
    ra, rb, rt, p = _floored(d, fn)
    ja2, jb2 = np.sum(d.j_a ** 2, axis=0), np.sum(d.j_b ** 2, axis=0)
    Aa, Ab = A_a(p), A_a(-p)
    dAa, dAb = dA_a(p), -dA_a(-p)              # d/dp of A_a(p) and of A_b(p) = A_a(-p)
    dp_da, dp_db = 2.0 * rb / rt ** 2, -2.0 * ra / rt ** 2
    Ka, Kb = d.tau_a - ja2 / ra, d.tau_b - jb2 / rb   # Galilean-invariant combinations
    g = coupling(d, lam, fn)
    Delta = -g * d.nu
    eF = t.fermi_energy(rt)
    common = B(p) * eF - np.abs(Delta) ** 2 / (3.0 * fn.C * np.cbrt(rt) ** 2)
    shape = 0.5 * (Ka * dAa + Kb * dAb) + 0.6 * rt * eF * dB(p)   # times dp/d rho_s
    V_a = common + shape * dp_da + (Aa - 1.0) * ja2 / (2.0 * ra * ra)
    V_b = common + shape * dp_db + (Ab - 1.0) * jb2 / (2.0 * rb * rb)
    return Potentials(V_a=V_a, V_b=V_b, alpha_a=Aa, alpha_b=Ab,
                      Avec_a=(1.0 - Aa) * d.j_a / ra, Avec_b=(1.0 - Ab) * d.j_b / rb, Delta=Delta, g=g)


def regulator(d: Densities, vext_a, vext_b, fn: ASLDA, lat: t.Lattice, iters: int = t.REGULATOR_ITERS):
    """Reading R2 with the spin averages of Sec. 2.6: Lambda_c(mu_+ - V_+, E_c, A_+)
    at the fixed point of V -> Lambda_c -> V, started from V = 0."""
    ec = fn.cutoff(lat)
    mu_p = 0.5 * (fn.mu_a + fn.mu_b)
    ve = 0.5 * (vext_a + vext_b)
    _, _, _, p = _floored(d, fn)
    A_p = 0.5 * (A_a(p) + A_a(-p))
    V = np.zeros(lat.M)
    for _ in range(iters):
        lam = t.lambda_c(mu_p - V - ve, ec, A_p)
        P = potentials(d, lam, fn)
        V = 0.5 * (P.V_a + P.V_b)
    return t.lambda_c(mu_p - V - ve, ec, A_p)


# ----------------------------------------------------------------------------
# Single-particle operators and H (Eqs. h_sigma, kinop-alpha, HpsiEpsi)
# ----------------------------------------------------------------------------
def kinetic(alpha, f, lat: t.Lattice):
    """-1/2 grad.alpha grad f by Eq. kinop-alpha summed over the axes:
    -1/4 [lap(alpha f) + alpha lap f - (lap alpha) f] (the Laplacians of H)."""
    return -0.25 * (t.laplacian(alpha * f, lat) + alpha * t.laplacian(f, lat) - t.laplacian(alpha, lat).real * f)


def current(Avec, f, lat: t.Lattice):
    """-(i/2){A, grad} f as -i (A.grad f + (div A / 2) f) (reading A2)."""
    g = t.gradient(f, lat)
    divA = sum(np.real(t.gradient(Avec[d], lat)[d]) for d in range(3))
    return -1j * (sum(Avec[d] * g[d] for d in range(3)) + 0.5 * divA * f)


@dataclass
class Fields:
    W_a: np.ndarray       # V_a + V_ext,a - mu_a
    W_b: np.ndarray       # V_b + V_ext,b - mu_b
    D: np.ndarray
    alpha_a: np.ndarray
    alpha_b: np.ndarray
    Avec_a: np.ndarray
    Avec_b: np.ndarray


def apply_H(phi, F: Fields, lat: t.Lattice):
    """(H phi)_u = (h_a - mu_a) u + Delta v,  (H phi)_v = Delta^* u + (-h_b^* + mu_b) v.
    h_b^* has the current term with the opposite sign, so -h_b^* v carries
    +1/2 grad.alpha_b grad v - W_b v - (i/2){A_b, grad} v."""
    u, v = phi[:, 0, :], phi[:, 1, :]
    Hu = kinetic(F.alpha_a, u, lat) + F.W_a * u + current(F.Avec_a, u, lat) + F.D * v
    Hv = np.conj(F.D) * u - kinetic(F.alpha_b, v, lat) - F.W_b * v + current(F.Avec_b, v, lat)
    return np.stack([Hu, Hv], axis=1)


@dataclass
class ImbalancedSystem:
    lat: t.Lattice
    fn: ASLDA
    vext_a: np.ndarray
    vext_b: np.ndarray
    fp: np.ndarray        # f(E_n)
    fm: np.ndarray        # f(-E_n)
    lam: np.ndarray | None = None

    def init_regulator(self, phi):
        self.lam = regulator(densities(phi, self.fp, self.fm, self.lat), self.vext_a, self.vext_b, self.fn,
                             self.lat)

    def fields(self, phi) -> Fields:
        d = densities(phi, self.fp, self.fm, self.lat)
        P = potentials(d, self.lam, self.fn)
        return Fields(W_a=P.V_a + self.vext_a - self.fn.mu_a, W_b=P.V_b + self.vext_b - self.fn.mu_b, D=P.Delta,
                      alpha_a=P.alpha_a, alpha_b=P.alpha_b, Avec_a=P.Avec_a, Avec_b=P.Avec_b)

    def f(self, phi):
        F = self.fields(phi)
        Hphi = apply_H(phi, F, self.lat)
        En = t.expectation(phi, Hphi, self.lat)
        return -1j * (Hphi - En[:, None, None] * phi)

    def energy(self, phi) -> dict:
        d = densities(phi, self.fp, self.fm, self.lat)
        dV = self.lat.dV
        e_int = dV * np.sum(energy_density(d, self.lam, self.fn))
        e_ext = dV * np.sum(self.vext_a * d.rho_a + self.vext_b * d.rho_b)
        return dict(e_total=e_int + e_ext, n_a=dV * np.sum(d.rho_a), n_b=dV * np.sum(d.rho_b),
                    P=dV * np.sum(d.j_a + d.j_b, axis=1))


def start_stationary(sys: ImbalancedSystem, phi0) -> t.ABMHistory:
    """Stationary start (reading S1) for the ABM schemes of tdslda.py."""
    phi = t.normalize(phi0, sys.lat)
    if sys.lam is None:
        sys.init_regulator(phi)
    z = np.zeros_like(phi)
    return t.ABMHistory(phi=phi, f=[sys.f(phi), z, z.copy(), z.copy()])


def taylor_series(phi0, F: Fields, shift, h: float, r: int, lat: t.Lattice):
    """sum_{k=0}^{r} (-i h)^k / k! [H - shift]^k phi0 (Eq. Taylor-exp), term by term."""
    out = phi0.copy()
    term = phi0
    for k in range(1, r + 1):
        term = apply_H(term, F, lat) - shift[:, None, None] * term
        term = (-1j * h / k) * term
        out = out + term
    return out


def taylor_step(sys: ImbalancedSystem, phi, dt: float, r: int = 5):
    """The predictor-corrector Taylor step of Sec. 3.3 with readings T1, T2:
    H at t, the midpoint state, H at the midpoint, the state at t + dt."""
    lat = sys.lat
    F0 = sys.fields(phi)
    s0 = t.expectation(phi, apply_H(phi, F0, lat), lat)
    mid = t.normalize(taylor_series(phi, F0, s0, 0.5 * dt, r, lat), lat)
    Fm = sys.fields(mid)
    s1 = t.expectation(phi, apply_H(phi, Fm, lat), lat)
    return t.normalize(taylor_series(phi, Fm, s1, dt, r, lat), lat)


def start(sys: ImbalancedSystem, phi0, dt: float, stationary: bool, scheme: str = "AB4AM5", r: int = 5):
    """Start-up for an ABpAMq scheme: stationary (reading S1) or p - 1 Taylor
    steps (readings T2, T3), with the history ordered newest first."""
    if stationary:
        return start_stationary(sys, phi0)
    p = len(t.SCHEMES[scheme][0])
    phi = t.normalize(phi0, sys.lat)
    if sys.lam is None:
        sys.init_regulator(phi)
    hist = [sys.f(phi)]
    for _ in range(p - 1):
        phi = taylor_step(sys, phi, dt, r)
        hist.insert(0, sys.f(phi))
    return t.ABMHistory(phi=phi, f=hist, t=(p - 1) * dt, steps=p - 1)


def evolve(sys: ImbalancedSystem, st: t.ABMHistory, dt: float, nsteps: int, scheme: str = "AB4AM5"):
    for _ in range(nsteps):
        st = t.abm_step(sys, st, dt, scheme)
    return st
