"""Pins of the A != 1 (current-carrying) SLDA terms of the oracle.

The functional of Sec. 2.4 is Galilean invariant (E_0) plus the centre-of-mass
part E_CM, so a uniform boost u -> e^{iq.r} u, v -> e^{-iq.r} v acts on the
single-particle Hamiltonian exactly as for particles of bare mass 1, whatever A
is: h' e^{iq.r} = e^{iq.r} (h + q.p + q^2/2), p = -i grad. With mu' = mu + q^2/2
this gives H' B_q phi = B_q (H + q.p) phi, B_q = diag(e^{iq.r}, e^{-iq.r}), and
E' = E + q.P + N q^2 / 2 for the energy. Both identities need the kinetic
factor A, the current potential (1 - A) j / rho, the current part of U and the
sign of the anticommutator to be right together; with A = 1.094 (A_a(0) of the
ASLDA functional, Sec. 2.4) a dropped or mis-signed term breaks them. On a
lattice they are exact (to rounding) for states whose spectrum stays clear of
the Nyquist planes after the shift, which the inputs below are built to be.
"""
import numpy as np

from oracle import tdslda as o
from paper_2602_08982_b300 import inputs


def _band_limited_states(lat, n, seed, mmax=1):
    """n states (u, v) built from the modes |m_d| <= mmax with seeded
    coefficients, normalised."""
    u01 = inputs.uniform01(seed, 4 * n * (2 * mmax + 1) ** 3).reshape(n, 2, -1, 2)
    coef = (2 * u01[..., 0] - 1) + 1j * (2 * u01[..., 1] - 1)
    x = [np.arange(N) * d for N, d in zip(lat.shape, (lat.dx, lat.dy, lat.dz))]
    X, Y, Z = np.meshgrid(*x, indexing="ij")
    phi = np.zeros((n, 2, lat.M), dtype=complex)
    k = 0
    r = range(-mmax, mmax + 1)
    for mx in r:
        for my in r:
            for mz in r:
                kv = [2 * np.pi * m / (N * d) for m, N, d in zip((mx, my, mz), lat.shape, (lat.dx, lat.dy, lat.dz))]
                wave = np.exp(1j * (kv[0] * X + kv[1] * Y + kv[2] * Z)).reshape(-1)
                phi += coef[:, :, k, None] * wave[None, None, :]
                k += 1
    return o.normalize(phi, lat)


def _setup(A=o.aslda_A(0.0)):
    lat = o.Lattice(8, 8, 10, 1.0, 0.9, 1.1)
    n = 12
    phi = _band_limited_states(lat, n, seed=41)
    wm = 0.5 + 0.5 * inputs.uniform01(5, n)
    wp = 0.3 * inputs.uniform01(6, n)
    vext = inputs.harmonic_trap(lat.shape, 0.08)
    fn = o.Functional("slda", B=o.B_SLDA, C=o.C_ASLDA, mu=0.4, A=float(A))
    sys = o.TDSystem(lat, fn, vext=vext, w_minus=wm, w_plus=wp)
    sys.init_regulator(phi)
    mq = (1, 1, -1)
    q = np.array([2 * np.pi * m / (N * d) for m, N, d in zip(mq, lat.shape, (lat.dx, lat.dy, lat.dz))])
    x = [np.arange(N) * d for N, d in zip(lat.shape, (lat.dx, lat.dy, lat.dz))]
    X, Y, Z = np.meshgrid(*x, indexing="ij")
    ph = np.exp(1j * (q[0] * X + q[1] * Y + q[2] * Z)).reshape(-1)
    boosted = np.stack([phi[:, 0] * ph, phi[:, 1] * np.conj(ph)], axis=1)
    fnb = o.Functional("slda", B=o.B_SLDA, C=o.C_ASLDA, mu=0.4 + 0.5 * q @ q, A=float(A))
    sysb = o.TDSystem(lat, fnb, vext=vext, w_minus=wm, w_plus=wp, lam=sys.lam)
    return lat, phi, boosted, ph, q, sys, sysb


def _covariance_residual(lat, phi, boosted, ph, q, F, Fb):
    H = o.apply_H(phi, F, lat)
    g = o.gradient(phi, lat)
    qp = -1j * sum(q[d] * g[d] for d in range(3))   # q.p phi
    rhs = H + qp
    rhs = np.stack([rhs[:, 0] * ph, rhs[:, 1] * np.conj(ph)], axis=1)
    Hb = o.apply_H(boosted, Fb, lat)
    return np.abs(Hb - rhs).max() / np.abs(rhs).max()


def test_printed_effective_mass_is_used():
    assert o.aslda_A(0.0) == 1.094


def test_current_of_boosted_state_is_shifted_by_rho_q():
    lat, phi, boosted, ph, q, sys, sysb = _setup()
    wm, wp = sys.weights(phi.shape[0])
    rho, _ = o.densities(phi, wm, wp)
    j = sys.current(phi)
    jb = sysb.current(boosted)
    assert np.abs(j).max() > 1e-3          # the states carry currents
    assert np.abs(jb - (j + rho[None] * q[:, None])).max() < 1e-13


def test_hamiltonian_is_galilean_covariant_for_A_not_1():
    lat, phi, boosted, ph, q, sys, sysb = _setup()
    F, Fb = sys.fields(phi), sysb.fields(boosted)
    assert F.Avec is not None and np.abs(F.Avec).max() > 1e-4
    res = _covariance_residual(lat, phi, boosted, ph, q, F, Fb)
    assert res < 1e-12, res


def test_covariance_fails_without_the_current_terms():
    """Sensitivity of the pin: drop the current potential (keeping A) and the
    identity fails by orders of magnitude."""
    lat, phi, boosted, ph, q, sys, sysb = _setup()
    F, Fb = sys.fields(phi), sysb.fields(boosted)
    F0 = o.Fields(W=F.W, D=F.D, alpha=F.alpha)
    Fb0 = o.Fields(W=Fb.W, D=Fb.D, alpha=Fb.alpha)
    assert _covariance_residual(lat, phi, boosted, ph, q, F0, Fb0) > 1e-3
    # the current part of U alone (potential kept) also matters
    Fb1 = o.Fields(W=Fb.W - o.current_mean_field(o.densities(boosted, *sysb.weights(12))[0],
                                                 sysb.current(boosted), sysb.fn),
                   D=Fb.D, alpha=Fb.alpha, Avec=Fb.Avec, divA=Fb.divA)
    assert _covariance_residual(lat, phi, boosted, ph, q, F, Fb1) > 1e-3


def test_energy_changes_by_the_centre_of_mass_terms():
    """E' = E + q.P + N q^2 / 2 with P = int (j_a + j_b) and N = int (rho_a + rho_b)."""
    lat, phi, boosted, ph, q, sys, sysb = _setup()
    e, eb = sys.energy(phi), sysb.energy(boosted)
    P = 2.0 * lat.dV * sys.current(phi).sum(axis=1)
    want = e["e_total"] + q @ P + 0.5 * e["n_part"] * (q @ q)
    assert abs(eb["e_total"] - want) < 1e-12 * abs(want)
    assert abs(e["e_cur"]) > 1e-6


def test_A_equal_1_has_no_current_terms():
    lat, phi, boosted, ph, q, sys, sysb = _setup(A=1.0)
    F = sys.fields(phi)
    assert F.Avec is None and sys.current(phi) is None
    res = _covariance_residual(lat, phi, boosted, ph, q, F, sysb.fields(boosted))
    assert res < 1e-12, res
