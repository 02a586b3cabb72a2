"""Plain FP64 CPU oracle of the time-dependent SLDA (TDSLDA) step.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import or run anything in this package. The
product path (the CUDA library and its Python binding) never does, and this
package never imports the product.

Everything here is double precision, written for a reader who checks it against
the paper (W-SLDA Toolkit, arXiv 2602.08982) by eye: no blocking, no fusion.
Library primitives used as single steps: scipy.fft (the discrete Fourier
transform), numpy reductions, scipy root finders and quadrature.

Conventions (units m = hbar = k_B = 1, Sec. 2.1):
  * a quasiparticle state is the pair (u_n, v_n) of the reduced problem
    (Eq. HpsiEpsi), stored as phi[n, 0, :] = u_n, phi[n, 1, :] = v_n over the
    flattened lattice index (ix * NY + iy) * NZ + iz (x slowest, z fastest);
  * states are normalised as sum_r dV (|u|^2 + |v|^2) = 1;
  * spin-symmetric system, only E_n > 0 states are stored (Sec. 2.3).

Readings of points where the paper is silent or ambiguous are marked
"Reading <ID>" and are the same as the CUDA path's.

Parity pins: every function here is pinned by a test in tests/test_oracle_pins.py
against closed forms, printed numbers, textbook limits, invariants or brute
force. Partial pin: the SLDA constants used with A forced to 1 (Sec. 2.4,
"A_sigma = 1" option) have no printed number; the functional form they enter
is pinned through the A = 1.094 uniform solution instead. The current terms of
A != 1 (kinetic factor A, current potential, current part of U, anticommutator
and energy) are pinned together by the Galilean covariance of the functional
(tests/test_oracle_current.py).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft

WORKERS = max(1, os.cpu_count() or 1)
_AXES = (-3, -2, -1)


# ----------------------------------------------------------------------------
# Lattice (Sec. 3.1)
# ----------------------------------------------------------------------------
@dataclass
class Lattice:
    nx: int
    ny: int
    nz: int
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0

    @property
    def shape(self):
        return (self.nx, self.ny, self.nz)

    @property
    def M(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dV(self) -> float:
        return self.dx * self.dy * self.dz

    @property
    def volume(self) -> float:
        return self.M * self.dV

    def kaxis(self, axis: int) -> np.ndarray:
        """Fourier grid k_l = 2 pi l / L for l < N/2, 2 pi (l - N) / L otherwise
        (Sec. 3.1, Fourier components; N even)."""
        n = self.shape[axis]
        d = (self.dx, self.dy, self.dz)[axis]
        L = n * d
        l = np.arange(n)
        return np.where(l < n // 2, 2 * np.pi * l / L, 2 * np.pi * (l - n) / L)

    def k2(self) -> np.ndarray:
        """|k|^2 on the 3D grid, the Nyquist mode kept (k = -pi/dx at l = N/2)."""
        kx, ky, kz = (self.kaxis(a) for a in range(3))
        return kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2


def fft3(a):
    return sfft.fftn(a, axes=_AXES, workers=WORKERS)


def ifft3(a):
    return sfft.ifftn(a, axes=_AXES, workers=WORKERS)


def laplacian(f: np.ndarray, lat: Lattice) -> np.ndarray:
    """Spectral second derivative summed over axes (Eq. derivative-spectral, r = 2).

    `f` has trailing shape [M] (flattened) and any leading batch shape."""
    lead = f.shape[:-1]
    g = f.reshape(lead + lat.shape)
    out = ifft3(-lat.k2() * fft3(g))
    return out.reshape(lead + (lat.M,))


def gradient(f: np.ndarray, lat: Lattice):
    """Spectral first derivatives (Eq. derivative-spectral, r = 1) with the
    Nyquist contribution set to zero, as the paper prescribes for odd r."""
    lead = f.shape[:-1]
    fk = fft3(f.reshape(lead + lat.shape))
    out = []
    for ax in range(3):
        k = lat.kaxis(ax).copy()
        k[lat.shape[ax] // 2] = 0.0
        s = [1, 1, 1]
        s[ax] = -1
        out.append(ifft3(1j * k.reshape(s) * fk).reshape(lead + (lat.M,)))
    return out


def derivative_matrix_1d(n: int, d: float, order: int) -> np.ndarray:
    """Closed-form derivative matrices D^(1), D^(2) of Eqs. D1 and D2 (one axis)."""
    L = n * d
    l = np.arange(n)
    diff = l[:, None] - l[None, :]
    off = diff != 0
    D = np.zeros((n, n))
    sgn = np.where(diff % 2 == 0, 1.0, -1.0)
    if order == 1:
        D[off] = (np.pi / L) * sgn[off] / np.tan(np.pi * diff[off] / n)
    elif order == 2:
        D[off] = (2 * np.pi ** 2 / L ** 2) * (-sgn[off]) / np.sin(np.pi * diff[off] / n) ** 2
        D[~off] = -(np.pi ** 2 / (3 * d ** 2)) * (1 + 2.0 / n ** 2)
    else:
        raise ValueError(order)
    return D


def dense_laplacian(lat: Lattice) -> np.ndarray:
    """M x M Laplacian assembled from Eq. D2 along each axis (Sec. 3.2, matrix form)."""
    Dx = derivative_matrix_1d(lat.nx, lat.dx, 2)
    Dy = derivative_matrix_1d(lat.ny, lat.dy, 2)
    Dz = derivative_matrix_1d(lat.nz, lat.dz, 2)
    Ix, Iy, Iz = np.eye(lat.nx), np.eye(lat.ny), np.eye(lat.nz)
    return (np.kron(np.kron(Dx, Iy), Iz) + np.kron(np.kron(Ix, Dy), Iz)
            + np.kron(np.kron(Ix, Iy), Dz))


# ----------------------------------------------------------------------------
# Energy density functional (Sec. 2.4) and regularisation (Sec. 2.6)
# ----------------------------------------------------------------------------
C_ASLDA = -11.11  # C(p) of the ASLDA functional


def aslda_A(p):
    """A_a(p) of the ASLDA functional (Sec. 2.4)."""
    return 1.094 + 0.156 * p * (1 - 2 * p ** 2 / 3 + p ** 4 / 5) - 0.532 * p ** 2 * (1 - p ** 2 + p ** 4 / 3)


def aslda_B(p):
    """B(p) of the ASLDA functional (Sec. 2.4); A_b(p) = A_a(-p)."""
    return 2 ** (2.0 / 3.0) * (0.357 + 0.642 * p ** 2 - aslda_A(p) * ((1 + p) / 2) ** (5.0 / 3.0)
                                - aslda_A(-p) * ((1 - p) / 2) ** (5.0 / 3.0))


B_SLDA = float(aslda_B(0.0))  # spin-symmetric SLDA value, approx -0.5273


def fermi_energy(rho_total):
    """eF(rho) = (3 pi^2 rho)^(2/3) / 2 with rho = rho_a + rho_b (Sec. 2.4)."""
    return 0.5 * (3 * np.pi ** 2 * rho_total) ** (2.0 / 3.0)


def lattice_cutoff(lat: Lattice) -> float:
    """Default cutoff energy of the regulator (Sec. 2.6).

    Reading R5: the evolved set is all M lattice states, whose kinetic energies
    reach the corner of the Brillouin zone, (pi^2/2)(1/dx^2 + 1/dy^2 + 1/dz^2)
    = 3 k_c^2 / 2 on a cubic lattice; Sec. 2.6 notes that energy conservation
    with all states needs E_c >= 3 k_c^2 / 2, so that value is the default."""
    return 0.5 * np.pi ** 2 * (1 / lat.dx ** 2 + 1 / lat.dy ** 2 + 1 / lat.dz ** 2)


def lambda_c(mu_minus_V, ec: float, A: float = 1.0):
    """Regulator Lambda_c of Eq. Creg (Sec. 2.6), pointwise.

    k_0 and k_c solve A k_0^2/2 + V - mu = 0 and A k_c^2/2 + V - mu = E_c.
    Lambda_c is the principal-value integral (1/2 pi^2) int_0^kc k^2 dk /
    (A k^2 - A k_0^2), which the printed logarithmic form evaluates for k_0^2 > 0.
    Reading R3: for k_0^2 < 0 (classically forbidden, mu < V) the same integral
    has no pole and gives 1 - (kappa/k_c) arctan(k_c/kappa), kappa^2 = -k_0^2;
    for k_c^2 <= 0 the regulator is 0."""
    x = np.asarray(mu_minus_V, dtype=np.float64)
    k0sq = 2.0 * x / A
    kcsq = 2.0 * (ec + x) / A
    out = np.zeros_like(x)
    ok = kcsq > 0
    kc = np.sqrt(np.where(ok, kcsq, 1.0))
    pos = ok & (k0sq > 0)
    neg = ok & (k0sq < 0)
    zer = ok & (k0sq == 0)
    k0 = np.sqrt(np.where(pos, k0sq, 0.0))
    kap = np.sqrt(np.where(neg, -k0sq, 0.0))
    pref = kc / (2 * np.pi ** 2 * A)
    with np.errstate(divide="ignore", invalid="ignore"):
        br_pos = 1.0 - (k0 / (2 * kc)) * np.log((kc + k0) / (kc - k0))
        br_neg = 1.0 - (kap / kc) * np.arctan2(kc, kap)
    out = np.where(pos, pref * br_pos, out)
    out = np.where(neg, pref * br_neg, out)
    out = np.where(zer, pref, out)
    return out


@dataclass
class Functional:
    """SLDA-type ('slda', Sec. 2.4) or BdG ('bdg').

    slda: E_0 + E_CM = sum_sigma [A/2 (tau_s - j_s^2/rho_s) + j_s^2/(2 rho_s)]
                       + 3/5 B rho eF(rho) + g_eff |nu|^2
          (Eqs. sldae-functional-generic, -CM, sldae-functional) with a constant
          A; A = 1 is the 'A_sigma = 1' option of Sec. 2.4 (last paragraph),
          where the current terms cancel. The spin-symmetric ASLDA has
          A = A_a(0) = 1.094, B = B(0), C = -11.11.
    bdg : A = 1, B = 0, coupling 4 pi a (Eq. HBdG)
    Reading R1: 1/g_eff = rho^(1/3)/C - Lambda_c (slda) or 1/(4 pi a) - Lambda_c
    (bdg); Delta = -g_eff nu (Eq. Delta)."""
    kind: str = "slda"
    B: float = B_SLDA
    C: float = C_ASLDA
    inv_4pi_a: float = 0.0
    mu: float = 0.0
    ec: float = -1.0          # <= 0 selects lattice_cutoff() (reading R5)
    rho_floor: float = 1e-12  # Reading R4
    A: float = 1.0            # inverse effective mass alpha = A_sigma (slda only)

    def cutoff(self, lat: Lattice) -> float:
        return self.ec if self.ec > 0 else lattice_cutoff(lat)

    @property
    def currents(self) -> bool:
        """Whether the current terms are present (A != 1, Sec. 2.4)."""
        return self.kind == "slda" and self.A != 1.0


def inverse_coupling(rho_sigma, lam, fn: Functional):
    """1/g_eff at each site (Eq. Creg, reading R1)."""
    if fn.kind == "slda":
        rho = np.maximum(2.0 * rho_sigma, fn.rho_floor)
        return rho ** (1.0 / 3.0) / fn.C - lam
    return fn.inv_4pi_a - lam


def mean_field(rho_sigma, delta, fn: Functional):
    """U = dE_0/d rho_sigma for A = 1 (derived from Eq. sldae-functional with
    Lambda_c held fixed): B eF(rho) - |Delta|^2 / (3 C rho^(2/3)); 0 for BdG."""
    if fn.kind == "slda":
        rho = np.maximum(2.0 * rho_sigma, fn.rho_floor)
        return fn.B * fermi_energy(rho) - np.abs(delta) ** 2 / (3.0 * fn.C * rho ** (2.0 / 3.0))
    return np.zeros_like(np.asarray(rho_sigma, dtype=np.float64))


def current_mean_field(rho_sigma, j, fn: Functional):
    """The part of U = dE/d rho_sigma that the current terms add for a
    constant A: d/d rho_s [(1 - A) j_s^2 / (2 rho_s)] = (A - 1) j_s^2 / (2 rho_s^2)
    (reading N1: rho_s floored at rho_floor)."""
    rs = np.maximum(rho_sigma, fn.rho_floor)
    return (fn.A - 1.0) * np.sum(j * j, axis=0) / (2.0 * rs * rs)


def current_potential(rho_sigma, j, fn: Functional):
    """Current potential A_sigma = dE/d j_sigma = (1 - A) j_s / rho_s
    (Sec. 2.2 list of potentials; reading N1 floor)."""
    rs = np.maximum(rho_sigma, fn.rho_floor)
    return (1.0 - fn.A) * j / rs[None, :]


def potentials(rho_sigma, nu, lam, fn: Functional, j=None):
    """(U, Delta, g_eff) from the densities with a given regulator field; `j`
    (the current of one spin, [3][M]) adds the current part of U when A != 1."""
    g = 1.0 / inverse_coupling(rho_sigma, lam, fn)
    delta = -g * nu
    U = mean_field(rho_sigma, delta, fn)
    if fn.currents and j is not None:
        U = U + current_mean_field(rho_sigma, j, fn)
    return U, delta, g


REGULATOR_ITERS = 60


def frozen_regulator(rho_sigma, nu, vext, fn: Functional, lat: Lattice, iters: int = REGULATOR_ITERS, j=None):
    """Reading R2: the regulator used during time evolution is fixed at t = 0.

    Lambda_c depends on V = U + V_ext (and on A_+ = A, Sec. 2.6), and U depends
    on Lambda_c through g_eff; the t = 0 value is the fixed point of that loop,
    reached by `iters` plain iterations started from U = 0 (the same count on
    the GPU side). With A != 1, U includes the current part from `j` at t = 0."""
    ec = fn.cutoff(lat)
    U = np.zeros_like(vext)
    for _ in range(iters):
        lam = lambda_c(fn.mu - U - vext, ec, fn.A)
        U, _, _ = potentials(rho_sigma, nu, lam, fn, j)
    return lambda_c(fn.mu - U - vext, ec, fn.A)


# ----------------------------------------------------------------------------
# Densities (Eqs. nab3D - jab3D, spin-symmetric, frozen weights Sec. 2.5)
# ----------------------------------------------------------------------------
def densities(phi, w_minus, w_plus):
    """rho_a = rho_b = sum_n w-_n |v_n|^2 + w+_n |u_n|^2;
    nu = sum_n (w-_n - w+_n) u_n v_n^*."""
    u, v = phi[:, 0, :], phi[:, 1, :]
    rho = np.einsum("n,nr->r", w_minus, np.abs(v) ** 2) + np.einsum("n,nr->r", w_plus, np.abs(u) ** 2)
    nu = np.einsum("n,nr->r", w_minus - w_plus, u * np.conj(v))
    return rho, nu


def kinetic_current_densities(phi, w_minus, w_plus, lat: Lattice):
    """tau_sigma and j_sigma (Eqs. nab3D-jab3D) with Nyquist-free gradients."""
    u, v = phi[:, 0, :], phi[:, 1, :]
    gu, gv = gradient(u, lat), gradient(v, lat)
    tau = sum(np.einsum("n,nr->r", w_minus, np.abs(gv[d]) ** 2)
              + np.einsum("n,nr->r", w_plus, np.abs(gu[d]) ** 2) for d in range(3))
    j = np.stack([np.einsum("n,nr->r", w_minus, np.imag(v * np.conj(gv[d])))
                  - np.einsum("n,nr->r", w_plus, np.imag(u * np.conj(gu[d]))) for d in range(3)])
    return tau, j


# ----------------------------------------------------------------------------
# Hamiltonian application and ABM right-hand side (Sec. 3.3)
# ----------------------------------------------------------------------------
@dataclass
class Fields:
    """Pointwise fields defining H (Eq. h_sigma, Eq. HpsiEpsi):
    W = U + V_ext - mu on the diagonal, D = Delta + Delta_ext off the diagonal,
    alpha the (constant) inverse effective mass, Avec [3][M] the current
    potential and divA its spectral divergence (None: no current term, as in
    Eq. h_sigma_A1)."""
    W: np.ndarray
    D: np.ndarray
    alpha: float = 1.0
    Avec: np.ndarray | None = None
    divA: np.ndarray | None = None


def current_term(f, F: Fields, lat: Lattice):
    """-(i/2){A, grad} f, the current term of h_sigma (Eq. h_sigma).

    Reading N2: the anticommutator is evaluated as 2 A.grad f + (div A) f with
    spectral, Nyquist-free first derivatives of f and of A (the gradient
    buffers Sec. 3.3 counts, with no transform of the product A f)."""
    g = gradient(f, lat)
    s = sum(F.Avec[d] * g[d] for d in range(3))
    return -1j * (s + 0.5 * F.divA * f)


def apply_H(phi, F: Fields, lat: Lattice):
    """(H phi)_u = h u - mu u + D v with h = -alpha/2 lap + U + V_ext - (i/2){A, grad};
    (H phi)_v = D^* u - h^* v + mu v  (Eqs. HpsiEpsi, h_sigma; spin-symmetric, so
    h_a = h_b). For a constant alpha, -1/2 grad.alpha grad = -alpha/2 lap
    (Eq. kinop-alpha with a constant alpha). h^* has the current term with the
    opposite sign, so -h^* v carries -(i/2){A, grad} v, the same term as h u."""
    u, v = phi[:, 0, :], phi[:, 1, :]
    a = F.alpha
    Hu = -0.5 * a * laplacian(u, lat) + F.W * u + F.D * v
    Hv = np.conj(F.D) * u + 0.5 * a * laplacian(v, lat) - F.W * v
    if F.Avec is not None:
        Hu = Hu + current_term(u, F, lat)
        Hv = Hv + current_term(v, F, lat)
    return np.stack([Hu, Hv], axis=1)


def expectation(phi, Hphi, lat: Lattice):
    """<H>_n = Re int phi_n^dagger H phi_n (reading I2: imaginary part is roundoff)."""
    return lat.dV * np.real(np.einsum("ncr,ncr->n", np.conj(phi), Hphi))


def norms(phi, lat: Lattice):
    return lat.dV * np.einsum("ncr,ncr->n", np.conj(phi), phi).real


def normalize(phi, lat: Lattice):
    return phi / np.sqrt(norms(phi, lat))[:, None, None]


def rhs_f(phi, F: Fields, lat: Lattice):
    """f(phi) = -i [H - <H>_n] phi (Eq. ABM-f, Eq. shorttdproblem-mod)."""
    Hphi = apply_H(phi, F, lat)
    En = expectation(phi, Hphi, lat)
    return -1j * (Hphi - En[:, None, None] * phi)


# ----------------------------------------------------------------------------
# Time-dependent system: densities -> potentials -> H, energy
# ----------------------------------------------------------------------------
AB4 = np.array([55.0, -59.0, 37.0, -9.0]) / 24.0                 # Eq. AB4
AM5 = np.array([251.0, 646.0, -264.0, 106.0, -19.0]) / 720.0     # Eq. AM5
AB3 = np.array([23.0, -16.0, 5.0]) / 12.0                         # Eq. AB3
AB5 = np.array([1901.0, -2774.0, 2616.0, -1274.0, 251.0]) / 720.0  # Eq. AB5
AM4 = np.array([9.0, 19.0, -5.0, 1.0]) / 24.0                     # Eq. AM4


@dataclass
class Friction:
    """Dissipative ("quantum friction") terms of Sec. 5.2.4 for the
    spin-symmetric system (Eqs. cooling_alpha, Deltadiss2):
      U_diss = -(alpha / rho0) div j_sigma,
      Delta_diss = Delta [beta sin(theta_nu - theta_B') + i gamma (N - N_req) / N_req],
      theta_B' = arg[-1/2 sum_n (u_n lap v_n^* + v_n^* lap u_n)],  theta_nu = arg nu.
    Reading Q1: div j_sigma is evaluated as sum_n [w-_n Im(v_n lap v_n^*)
    - w+_n Im(u_n lap u_n^*)] (the divergence of j by the product rule, the
    |grad v|^2 term being real), with the spectral Laplacian of H.
    Reading Q2: the sum in theta_B' carries the weights of nu, w-_n - w+_n.
    Reading Q3: rho0 (not defined in the text) is a parameter; N counts both
    spin species, N = int (rho_a + rho_b)."""
    alpha: float = 0.0
    beta: float = 0.0
    gamma: float = 0.0
    rho0: float = 1.0 / (6.0 * math.pi ** 2)
    n_req: float = 1.0

    def fields(self, phi, wm, wp, rho_sigma, nu, delta, lat: "Lattice"):
        u, v = phi[:, 0, :], phi[:, 1, :]
        lu, lv = laplacian(u, lat), laplacian(v, lat)
        div_j = (np.einsum("n,nr->r", wm, np.imag(v * np.conj(lv)))
                 - np.einsum("n,nr->r", wp, np.imag(u * np.conj(lu))))
        bp = -0.5 * np.einsum("n,nr->r", wm - wp, u * np.conj(lv) + np.conj(v) * lu)
        dU = -(self.alpha / self.rho0) * div_j
        n_tot = lat.dV * np.sum(2.0 * rho_sigma)
        g = self.gamma * (n_tot - self.n_req) / self.n_req
        dD = delta * (self.beta * np.sin(np.angle(nu) - np.angle(bp)) + 1j * g)
        return dU, dD


@dataclass
class TDSystem:
    lat: Lattice
    fn: Functional
    vext: np.ndarray                     # [M] real
    dext: np.ndarray | None = None       # [M] complex external pairing field
    w_minus: np.ndarray | None = None    # [n] frozen thermal weights f(-E_n)
    w_plus: np.ndarray | None = None     # [n] frozen thermal weights f(E_n)
    lam: np.ndarray | None = None        # frozen regulator (reading R2)
    freeze_fields: Fields | None = None  # testing aid: H held fixed
    friction: "Friction | None" = None   # dissipative terms (Sec. 5.2.4)

    def weights(self, n):
        wm = np.ones(n) if self.w_minus is None else self.w_minus
        wp = np.zeros(n) if self.w_plus is None else self.w_plus
        return wm, wp

    def current(self, phi):
        """j_sigma (Eq. jab3D) when the functional has current terms, else None."""
        if not self.fn.currents:
            return None
        wm, wp = self.weights(phi.shape[0])
        return kinetic_current_densities(phi, wm, wp, self.lat)[1]

    def init_regulator(self, phi):
        wm, wp = self.weights(phi.shape[0])
        rho, nu = densities(phi, wm, wp)
        self.lam = frozen_regulator(rho, nu, self.vext, self.fn, self.lat, j=self.current(phi))

    def potentials(self, phi, j=None):
        wm, wp = self.weights(phi.shape[0])
        rho, nu = densities(phi, wm, wp)
        U, delta, g = potentials(rho, nu, self.lam, self.fn, j)
        return rho, nu, U, delta, g

    def fields(self, phi) -> Fields:
        """Densities of all states -> potentials -> (W, D) and, for A != 1, the
        current potential and its divergence (Alg. 1 steps 3-4)."""
        if self.freeze_fields is not None:
            return self.freeze_fields
        j = self.current(phi)
        rho, nu, U, delta, _ = self.potentials(phi, j)
        if self.friction is not None:
            wm, wp = self.weights(phi.shape[0])
            dU, dD = self.friction.fields(phi, wm, wp, rho, nu, delta, self.lat)
            U = U + dU
            delta = delta + dD
        D = delta if self.dext is None else delta + self.dext
        if j is None:
            return Fields(W=U + self.vext - self.fn.mu, D=D)
        Avec = current_potential(rho, j, self.fn)
        divA = np.real(sum(gradient(Avec[d], self.lat)[d] for d in range(3)))
        return Fields(W=U + self.vext - self.fn.mu, D=D, alpha=self.fn.A, Avec=Avec, divA=divA)

    def f(self, phi):
        return rhs_f(phi, self.fields(phi), self.lat)

    def energy(self, phi) -> dict:
        """Energy terms of Sec. 3.2 (reading E1: the kinetic term uses the same
        Laplacian as H, via sum_n w <v|-lap|v>, times A). With A != 1 the
        current terms add e_cur = int sum_s (1 - A) j_s^2 / (2 rho_s). The
        quantity the evolution conserves is e_total - mu * n_part (Eq. E_tot)."""
        lat, fn = self.lat, self.fn
        wm, wp = self.weights(phi.shape[0])
        j = self.current(phi)
        rho_s, nu, U, delta, g = self.potentials(phi, j)
        u, v = phi[:, 0, :], phi[:, 1, :]
        lu, lv = laplacian(u, lat), laplacian(v, lat)
        a = fn.A if fn.kind == "slda" else 1.0
        e_kin = a * lat.dV * (np.einsum("n,nr->", wm, -np.conj(v) * lv).real
                              + np.einsum("n,nr->", wp, -np.conj(u) * lu).real)
        e_cur = 0.0
        if j is not None:
            rs = np.maximum(rho_s, fn.rho_floor)
            e_cur = lat.dV * np.sum((1.0 - fn.A) * np.sum(j * j, axis=0) / rs)
        rho = 2.0 * rho_s
        e_pot = lat.dV * np.sum(0.6 * fn.B * rho * fermi_energy(rho)) if fn.kind == "slda" else 0.0
        e_pair = -lat.dV * np.sum(np.real(np.conj(delta) * nu))
        e_ext = lat.dV * np.sum(self.vext * rho)
        e_pext = 0.0 if self.dext is None else -lat.dV * np.sum(2.0 * np.real(self.dext * np.conj(nu)))
        n_part = lat.dV * np.sum(rho)
        tot = e_kin + e_pot + e_pair + e_ext + e_pext + e_cur
        return dict(e_kin=e_kin, e_pot=e_pot, e_pair=e_pair, e_ext=e_ext, e_pair_ext=e_pext,
                    e_cur=e_cur, e_total=tot, n_part=n_part)


# ----------------------------------------------------------------------------
# Integrators: AB4AM5 (Alg. 2) and the Taylor start (Eq. Taylor-exp)
# ----------------------------------------------------------------------------
@dataclass
class ABMState:
    """The five buffers of Alg. 2: phi_{k-1} and f_{k-1} .. f_{k-4}."""
    phi: np.ndarray
    f1: np.ndarray
    f2: np.ndarray
    f3: np.ndarray
    f4: np.ndarray
    t: float = 0.0
    steps: int = 0


def ab4am5_step(sys: TDSystem, st: ABMState, dt: float) -> ABMState:
    """One pass of Integrator_AB4AM5 (Alg. 2), steps 1-10 in order."""
    lat = sys.lat
    # step 1: predictor (Eq. AB4) and corrector partial (Eq. AM5 without the new
    # term), both formed from the same phi_{k-1} before it is overwritten
    pred = st.phi + dt * (AB4[0] * st.f1 + AB4[1] * st.f2 + AB4[2] * st.f3 + AB4[3] * st.f4)
    corr = st.phi + dt * (AM5[1] * st.f1 + AM5[2] * st.f2 + AM5[3] * st.f3 + AM5[4] * st.f4)
    phi, f4 = pred, corr
    # step 2: normalise
    phi = normalize(phi, lat)
    # step 3: f(phi_p) (densities, potentials, H) into the phi buffer
    phi = sys.f(phi)
    # step 4: corrector completion
    phi = (AM5[0] * dt) * phi + f4
    # steps 5-7: shift the history
    f4, f3, f2 = st.f3, st.f2, st.f1
    # step 8: normalise
    phi = normalize(phi, lat)
    # step 9: f(phi_k) into f_{k-1}
    f1 = sys.f(phi)
    # step 10
    return ABMState(phi=phi, f1=f1, f2=f2, f3=f3, f4=f4, t=st.t + dt, steps=st.steps + 1)


def taylor_series(phi0, F: Fields, shift, h: float, r: int, lat: Lattice):
    """sum_{k=0}^{r} (-i h)^k / k! [H - shift]^k phi0 (Eq. Taylor-exp), term by term."""
    out = phi0.copy()
    term = phi0
    for k in range(1, r + 1):
        term = apply_H(term, F, lat) - shift[:, None, None] * term
        term = (-1j * h / k) * term
        out = out + term
    return out


def taylor_step(sys: TDSystem, phi, dt: float, r: int = 5):
    """Predictor-corrector Taylor step (Sec. 3.3, Eq. Taylor-exp).

    Reading T1: the series uses the shifted operator H - <H>_n of the ABM
    equations, the shift being the expectation value of that sub-step's H in
    phi(t) (the state the series is applied to), fixed over the r powers.
    Reading T2: normalise the midpoint state and the result."""
    lat = sys.lat
    F0 = sys.fields(phi)
    s0 = expectation(phi, apply_H(phi, F0, lat), lat)
    mid = normalize(taylor_series(phi, F0, s0, 0.5 * dt, r, lat), lat)
    Fm = sys.fields(mid)
    s1 = expectation(phi, apply_H(phi, Fm, lat), lat)
    return normalize(taylor_series(phi, Fm, s1, dt, r, lat), lat)


def start(sys: TDSystem, phi0, dt: float, stationary: bool, r: int = 5) -> ABMState:
    """ABM start-up (Sec. 3.3).

    stationary: reading S1, f_{k-2..k-4} = 0 and f_{k-1} = f(phi_0) (zero for an
    exact stationary state). Otherwise reading T2/T3: three Taylor steps give
    phi_1..phi_3, history f_0..f_3, and count as steps of the evolution."""
    lat = sys.lat
    phi = normalize(phi0, lat)
    if sys.lam is None:
        sys.init_regulator(phi)
    z = np.zeros_like(phi)
    if stationary:
        return ABMState(phi=phi, f1=sys.f(phi), f2=z, f3=z.copy(), f4=z.copy())
    hist = [sys.f(phi)]
    for _ in range(3):
        phi = taylor_step(sys, phi, dt, r)
        hist.append(sys.f(phi))
    return ABMState(phi=phi, f1=hist[3], f2=hist[2], f3=hist[1], f4=hist[0], t=3 * dt, steps=3)


def evolve(sys: TDSystem, st: ABMState, dt: float, nsteps: int) -> ABMState:
    for _ in range(nsteps):
        st = ab4am5_step(sys, st, dt)
    return st


# ----------------------------------------------------------------------------
# The other predictor-corrector pairs of Sec. 3.3: AB3AM4 and AB5AM5
# ----------------------------------------------------------------------------
SCHEMES = {"AB3AM4": (AB3, AM4), "AB4AM5": (AB4, AM5), "AB5AM5": (AB5, AM5)}


@dataclass
class ABMHistory:
    """phi_{k-1} and the history f_{k-1}, f_{k-2}, ..., f_{k-p} of an ABpAMq
    scheme (p = predictor order: p + 2 buffers in the in-place form, Sec. 3.3)."""
    phi: np.ndarray
    f: list
    t: float = 0.0
    steps: int = 0


def abm_step(sys: TDSystem, st: ABMHistory, dt: float, scheme: str) -> ABMHistory:
    """One step of the scheme, in the order of Alg. 2 (which Sec. 3.3 says the
    other schemes follow): predictor and corrector partial from phi_{k-1} and
    the history, normalise, f at the predictor, complete the corrector,
    shift the history, normalise, f at the new state."""
    b, a = SCHEMES[scheme]
    lat = sys.lat
    pred = st.phi + dt * sum(b[j] * st.f[j] for j in range(len(b)))
    corr = st.phi + dt * sum(a[j + 1] * st.f[j] for j in range(len(a) - 1))
    phi = normalize(pred, lat)
    phi = (a[0] * dt) * sys.f(phi) + corr
    phi = normalize(phi, lat)
    hist = [sys.f(phi)] + st.f[:-1]
    return ABMHistory(phi=phi, f=hist, t=st.t + dt, steps=st.steps + 1)


def start_scheme(sys: TDSystem, phi0, dt: float, stationary: bool, scheme: str, r: int = 5) -> ABMHistory:
    """Start-up for a scheme whose predictor uses p history values: a stationary
    start (f_{k-2..k-p} = 0) or p - 1 Taylor steps (readings S1, T2, T3)."""
    p = len(SCHEMES[scheme][0])
    lat = sys.lat
    phi = normalize(phi0, lat)
    if sys.lam is None:
        sys.init_regulator(phi)
    if stationary:
        return ABMHistory(phi=phi, f=[sys.f(phi)] + [np.zeros_like(phi) for _ in range(p - 1)])
    hist = [sys.f(phi)]
    for _ in range(p - 1):
        phi = taylor_step(sys, phi, dt, r)
        hist.insert(0, sys.f(phi))
    return ABMHistory(phi=phi, f=hist, t=(p - 1) * dt, steps=p - 1)


def evolve_scheme(sys: TDSystem, st: ABMHistory, dt: float, nsteps: int, scheme: str) -> ABMHistory:
    for _ in range(nsteps):
        st = abm_step(sys, st, dt, scheme)
    return st


# ----------------------------------------------------------------------------
# Uniform systems (Sec. 5.2.1 "inittype 0"): lattice seeds and continuum checks
# ----------------------------------------------------------------------------
def bcs_amplitudes(xi, delta):
    """U_k, V_k of the 2x2 problem [[xi, D], [D, -xi]] at E_k = sqrt(xi^2 + D^2) > 0."""
    E = np.sqrt(xi ** 2 + delta ** 2)
    Uk = np.sqrt(0.5 * (1 + xi / E))
    Vk = np.sign(delta) * np.sqrt(0.5 * (1 - xi / E))
    return Uk, Vk, E


def solve_mu_eff(lat: Lattice, delta: float, rho_sigma: float) -> float:
    """mu_eff = mu - U such that (1/V) sum_k V_k^2 = rho_sigma over all M lattice k."""
    from scipy.optimize import brentq
    k2 = lat.k2().reshape(-1)

    def dens(me):
        xi = 0.5 * k2 - me
        E = np.sqrt(xi ** 2 + delta ** 2)
        return np.sum(0.5 * (1 - xi / E)) / lat.volume - rho_sigma
    return brentq(dens, -50.0, 0.5 * k2.max() + 50.0, xtol=1e-15, rtol=1e-15, maxiter=500)


@dataclass
class UniformSeed:
    mu_eff: float
    delta: float
    mu: float
    U: float
    C: float
    lam: float
    inv_g: float
    rho_sigma: float


def uniform_slda_seed(lat: Lattice, delta0: float, rho_sigma: float, B: float = B_SLDA,
                      ec: float = -1.0) -> UniformSeed:
    """Self-consistent uniform SLDA (A = 1) state on the lattice k-set with the
    gap fixed to delta0: mu_eff from the number equation, 1/g_eff from the gap
    equation 1 = -g_eff (1/V) sum_k 1/(2E_k), C backed out of Eq. Creg, and
    U = B eF - Delta^2/(3 C rho^(2/3))."""
    me = solve_mu_eff(lat, delta0, rho_sigma)
    k2 = lat.k2().reshape(-1)
    E = np.sqrt((0.5 * k2 - me) ** 2 + delta0 ** 2)
    inv_g = -np.sum(1.0 / (2 * E)) / lat.volume
    ecut = ec if ec > 0 else lattice_cutoff(lat)
    lam = float(lambda_c(me, ecut))
    rho = 2 * rho_sigma
    C = rho ** (1.0 / 3.0) / (inv_g + lam)
    U = B * fermi_energy(rho) - delta0 ** 2 / (3 * C * rho ** (2.0 / 3.0))
    return UniformSeed(mu_eff=me, delta=delta0, mu=U + me, U=U, C=C, lam=lam, inv_g=inv_g,
                       rho_sigma=rho_sigma)


def uniform_bdg_seed(lat: Lattice, inv_4pi_a: float, rho_sigma: float, ec: float = -1.0) -> UniformSeed:
    """Uniform BdG (U = 0) on the lattice: solve the number equation and the gap
    equation 1/(4 pi a) - Lambda_c(mu) = -(1/V) sum_k 1/(2E_k) for (mu, Delta).
    The root taken is the first sign change of the gap residual on a log grid
    of Delta from 1e-6 to 8, refined by bisection."""
    from scipy.optimize import brentq
    k2 = lat.k2().reshape(-1)
    ecut = ec if ec > 0 else lattice_cutoff(lat)

    def gap_residual(delta):
        me = solve_mu_eff(lat, delta, rho_sigma)
        E = np.sqrt((0.5 * k2 - me) ** 2 + delta ** 2)
        return inv_4pi_a - float(lambda_c(me, ecut)) + np.sum(1.0 / (2 * E)) / lat.volume
    grid = np.geomspace(1e-6, 8.0, 80)
    vals = [gap_residual(d) for d in grid]
    for a, b, fa, fb in zip(grid[:-1], grid[1:], vals[:-1], vals[1:]):
        if fa > 0 >= fb:
            delta = brentq(gap_residual, a, b, xtol=1e-15, rtol=1e-15, maxiter=500)
            break
    else:
        raise ValueError("uniform BdG gap equation has no root on this lattice")
    me = solve_mu_eff(lat, delta, rho_sigma)
    E = np.sqrt((0.5 * k2 - me) ** 2 + delta ** 2)
    return UniformSeed(mu_eff=me, delta=delta, mu=me, U=0.0, C=float("nan"), lam=float(lambda_c(me, ecut)),
                       inv_g=-np.sum(1.0 / (2 * E)) / lat.volume, rho_sigma=rho_sigma)


def uniform_states(lat: Lattice, mu_eff: float, delta: float) -> np.ndarray:
    """All M positive-energy plane-wave quasiparticle states of the uniform
    system: u_k = U_k e^{ik.r}/sqrt(V), v_k = V_k e^{ik.r}/sqrt(V), with k in the
    flattened FFT order and r = site index * spacing."""
    kx, ky, kz = (lat.kaxis(a) for a in range(3))
    x = np.arange(lat.nx) * lat.dx
    y = np.arange(lat.ny) * lat.dy
    z = np.arange(lat.nz) * lat.dz
    ex = np.exp(1j * np.outer(kx, x))
    ey = np.exp(1j * np.outer(ky, y))
    ez = np.exp(1j * np.outer(kz, z))
    pw = np.einsum("ai,bj,ck->abcijk", ex, ey, ez).reshape(lat.M, lat.M) / np.sqrt(lat.volume)
    k2 = lat.k2().reshape(-1)
    Uk, Vk, _ = bcs_amplitudes(0.5 * k2 - mu_eff, delta)
    return np.stack([Uk[:, None] * pw, Vk[:, None] * pw], axis=1)


def _v2(xi, d):
    """V_k^2 = (1 - xi/E)/2, E = sqrt(xi^2 + d^2), written as d^2 / (2 E (E + xi))
    for xi > 0 so that the far tail (xi >> d, where 1 - xi/E cancels to a few
    digits) keeps full double precision."""
    E = math.hypot(xi, d)
    return 0.5 * d * d / (E * (E + xi)) if xi > 0 else 0.5 * (1.0 - xi / E)


def _continuum_solve(integrals, rho_s, C, inv_4pi_a, lam, rho):
    """(mu_eff, Delta) from the number equation n_s(mu_eff, Delta) = rho_s
    (solved for mu_eff at each Delta) and the gap equation
    1/g_eff + (1/V) sum_k 1/(2E_k) = 0 (solved for Delta), both by bracketed
    root finding."""
    from scipy.optimize import brentq

    def me_of(d):
        lo = -10.0
        while integrals(lo, d)[0] > rho_s:  # strong pairing: the density needs a lower mu_eff
            lo *= 2
        return brentq(lambda me: integrals(me, d)[0] - rho_s, lo, 10.0, xtol=1e-14, rtol=1e-14, maxiter=300)

    def gap(d):
        me = me_of(d)
        inv_g = (rho ** (1 / 3) / C - lam(me)) if C is not None else (inv_4pi_a - lam(me))
        return inv_g + integrals(me, d)[3]
    grid = np.geomspace(1e-3, 2.0, 40)
    vals = [gap(d) for d in grid]
    for a, b, fa, fb in zip(grid[:-1], grid[1:], vals[:-1], vals[1:]):
        if fa * fb <= 0:
            d = brentq(gap, a, b, xtol=1e-14, rtol=1e-14, maxiter=300)
            return me_of(d), d
    raise ValueError("no superfluid root of the continuum gap equation")


def uniform_continuum(A: float, B: float, C: float | None, inv_4pi_a: float | None,
                      kF: float = 1.0, ec_over_eF: float = 2000.0):
    """Self-consistent uniform continuum solution with the Eq. Creg regularisation
    (spherical cutoff E_c, A k_c^2/2 - mu_eff = E_c). Returns a dict with mu/eF,
    Delta/eF and E/E_FG (E_FG = 3/5 N eF). SLDA-type if C is given, BdG if
    inv_4pi_a is given (then B must be 0).

    The k integrals run over [0, k_c] split at k_0 (the quasiparticle minimum,
    where xi changes sign), at 1/4, 1 and 4 times w = 4 Delta/(A k_0) on either
    side of it (w is the width of the step of V_k^2) and at a few multiples of
    max(k_0, kF); V_k^2 uses
    the cancellation-free form of _v2, so every piece converges to the
    requested tolerance."""
    from scipy.integrate import quad
    rho = kF ** 3 / (3 * np.pi ** 2)
    rho_s = rho / 2
    eF = 0.5 * kF ** 2
    ec = ec_over_eF * eF

    def integrals(me, d):
        kc = math.sqrt(2 * (ec + me) / A)
        k0 = math.sqrt(max(2 * me / A, 0.0))
        kk = max(k0, kF)

        def xi(k):
            return 0.5 * A * k * k - me
        opts = dict(limit=200, epsabs=1e-13, epsrel=1e-11)
        w = 4 * d / (A * k0) if k0 > 0 else 0.0  # width of the step of V_k^2 at k_0
        near = [k0 + f * w for f in (-4, -1, -0.25, 0, 0.25, 1, 4)]
        segs = sorted(set(s for s in [0.0, *near, 2 * kk, 8 * kk, 64 * kk, kc] if 0 <= s <= kc))

        def q(fun):
            return sum(quad(fun, a, b, **opts)[0] for a, b in zip(segs[:-1], segs[1:]))
        c = 1.0 / (2 * np.pi ** 2)
        return (c * q(lambda k: k * k * _v2(xi(k), d)),
                c * q(lambda k: k * k * d / (2 * math.hypot(xi(k), d))),
                c * q(lambda k: k ** 4 * _v2(xi(k), d)),
                c * q(lambda k: k * k / (2 * math.hypot(xi(k), d))))

    me, d = _continuum_solve(integrals, rho_s, C, inv_4pi_a, lambda me: float(lambda_c(me, ec, A)), rho)
    n_s, nu, tau, ie = integrals(me, d)
    g = -1.0 / ie
    U = (B * fermi_energy(rho) - d ** 2 / (3 * C * rho ** (2 / 3))) if C is not None else 0.0
    e_dens = A * tau + 0.6 * B * rho * fermi_energy(rho) + g * nu ** 2
    return dict(mu_over_eF=(U + me) / eF, delta_over_eF=d / eF,
                E_over_EFG=e_dens / (0.6 * rho * eF), mu_eff=me, nu=nu, tau=tau)


def uniform_continuum_limit(A: float, B: float, C: float | None, inv_4pi_a: float | None, kF: float = 1.0):
    """The same uniform solution directly at infinite cutoff, without Lambda_c:
    the regulator is the principal value of (1/2 pi^2) int k^2 / (A k^2 - 2 mu_eff),
    whose part beyond k_c -> infinity differs from (1/2 pi^2) int 1/A by a
    principal-value integral of 1/(k^2 - k_0^2) over [0, inf), which vanishes.
    So Eq. Creg's gap equation becomes
        rho^(1/3)/C (or 1/(4 pi a)) = -(1/2 pi^2) int_0^inf k^2 [1/(2E) - 1/(A k^2)] dk,
    and the energy density A tau + g nu^2 = A tau - Delta nu becomes
        (1/2 pi^2) int_0^inf [A k^4 V_k^2 - k^2 Delta^2 / (2E)] dk,
    both absolutely convergent (integrands ~ k^-2). Evaluated on [0, inf) with
    the tail mapped by quad's infinite-range transformation; an independent
    route to the Richardson-extrapolated output of uniform_continuum."""
    from scipy.integrate import quad
    rho = kF ** 3 / (3 * np.pi ** 2)
    rho_s = rho / 2
    eF = 0.5 * kF ** 2

    def integrals(me, d):
        k0 = math.sqrt(max(2 * me / A, 0.0))
        kk = max(k0, kF)

        def xi(k):
            return 0.5 * A * k * k - me
        opts = dict(limit=200, epsabs=1e-13, epsrel=1e-11)
        w = 4 * d / (A * k0) if k0 > 0 else 0.0
        near = [k0 + f * w for f in (-4, -1, -0.25, 0, 0.25, 1, 4)]
        segs = sorted(set(s for s in [0.0, *near, 2 * kk, 8 * kk] if s >= 0))

        def q(fun):
            parts = [quad(fun, a, b, **opts)[0] for a, b in zip(segs[:-1], segs[1:])]
            return sum(parts) + quad(fun, segs[-1], np.inf, **opts)[0]
        c = 1.0 / (2 * np.pi ** 2)
        # k^2 [1/(2E) - 1/(A k^2)] and A k^4 V_k^2 - k^2 Delta^2/(2E); for xi > 0
        # both are rewritten with A k^2 = 2 xi + 2 mu_eff and E - xi = Delta^2/(E + xi)
        # so that no large terms cancel in the tail
        def reg(k):
            x = xi(k)
            E = math.hypot(x, d)
            if x > 0:
                return (me - d * d / (E + x)) / (A * E)
            return (A * k * k - 2 * E) / (2 * A * E)

        def ereg(k):
            x = xi(k)
            E = math.hypot(x, d)
            if x > 0:
                return (k * k * d * d / (2 * E)) * (2 * me - d * d / (E + x)) / (E + x)
            return A * k ** 4 * _v2(x, d) - k * k * d * d / (2 * E)
        return (c * q(lambda k: k * k * _v2(xi(k), d)), None, c * q(ereg), c * q(reg))

    me, d = _continuum_solve(integrals, rho_s, C, inv_4pi_a, lambda me: 0.0, rho)
    n_s, _, e_pair_kin, reg = integrals(me, d)
    U = (B * fermi_energy(rho) - d ** 2 / (3 * C * rho ** (2 / 3))) if C is not None else 0.0
    e_dens = e_pair_kin + 0.6 * B * rho * fermi_energy(rho)
    return dict(mu_over_eF=(U + me) / eF, delta_over_eF=d / eF, E_over_EFG=e_dens / (0.6 * rho * eF), mu_eff=me)


# ----------------------------------------------------------------------------
# Dense reduced BdG matrix (brute force on tiny lattices)
# ----------------------------------------------------------------------------
def dense_bdg(F: Fields, lat: Lattice) -> np.ndarray:
    """2M x 2M matrix of Eq. HpsiEpsi for A = 1 built from Eq. D2:
    [[-1/2 D2 + W, D], [D^*, 1/2 D2 - W]]."""
    L = dense_laplacian(lat)
    M = lat.M
    H = np.zeros((2 * M, 2 * M), dtype=np.complex128)
    H[:M, :M] = -0.5 * L + np.diag(F.W)
    H[M:, M:] = 0.5 * L - np.diag(F.W)
    H[:M, M:] = np.diag(F.D)
    H[M:, :M] = np.diag(np.conj(F.D))
    return H


def dense_rhs(sys: TDSystem, phi):
    """f(phi) through the dense matrix (independent of the FFT path)."""
    F = sys.fields(phi)
    H = dense_bdg(F, sys.lat)
    n = phi.shape[0]
    x = phi.reshape(n, -1)
    Hx = x @ H.T
    En = sys.lat.dV * np.real(np.einsum("ni,ni->n", np.conj(x), Hx))
    return (-1j * (Hx - En[:, None] * x)).reshape(phi.shape)


def rk4_reference(sys: TDSystem, phi0, T: float, nsub: int):
    """Classical RK4 on the modified equation (Eq. shorttdproblem-mod) with the
    dense matrix, used only as an independent fine-step reference."""
    h = T / nsub
    phi = phi0.copy()
    for _ in range(nsub):
        k1 = dense_rhs(sys, phi)
        k2 = dense_rhs(sys, phi + 0.5 * h * k1)
        k3 = dense_rhs(sys, phi + 0.5 * h * k2)
        k4 = dense_rhs(sys, phi + h * k3)
        phi = phi + (h / 6) * (k1 + 2 * k2 + 2 * k3 + k4)
    return phi
