"""Pins of the spin-imbalanced ASLDA oracle (oracle/aslda.py)."""
import numpy as np
import pytest

from cases import make_case, oracle_system
from oracle import aslda as a
from oracle import tdslda as o
from paper_2602_08982_b300 import inputs


def _random_densities(M=7, seed=21):
    r = lambda k: inputs.uniform01(seed + k, M)
    rho_a = 0.004 + 0.02 * r(0)
    rho_b = 0.002 + 0.015 * r(1)
    j_a = 0.002 * (2 * np.stack([r(2), r(3), r(4)]) - 1)
    j_b = 0.002 * (2 * np.stack([r(5), r(6), r(7)]) - 1)
    tau_a = np.sum(j_a ** 2, axis=0) / rho_a + 0.01 * (0.5 + r(8))
    tau_b = np.sum(j_b ** 2, axis=0) / rho_b + 0.01 * (0.5 + r(9))
    nu = 0.003 * ((2 * r(10) - 1) + 1j * (2 * r(11) - 1))
    lam = 0.04 + 0.03 * r(12)
    return a.Densities(rho_a, rho_b, tau_a, tau_b, nu, j_a, j_b), lam


def _shift(d, name, comp, h):
    """Copy of d with one density (component comp of a vector / complex part) moved by h."""
    f = {k: np.array(getattr(d, k), copy=True) for k in ("rho_a", "rho_b", "tau_a", "tau_b", "nu", "j_a", "j_b")}
    if name == "nu":
        f["nu"] = f["nu"] + (h if comp == 0 else 1j * h)
    elif name in ("j_a", "j_b"):
        f[name][comp] += h
    else:
        f[name] += h
    return a.Densities(**f)


def test_potentials_are_derivatives_of_the_energy_density():
    """V_s = dE/d rho_s, alpha_s = 2 dE/d tau_s, A_s = dE/d j_s, Delta = -dE/d nu^*
    (Sec. 2.2) against central differences of the pointwise energy density,
    with p varying from site to site (the A(p), B(p) derivative terms matter)."""
    d, lam = _random_densities()
    fn = a.ASLDA(mu_a=0.3, mu_b=0.2)
    P = a.potentials(d, lam, fn)
    _, _, _, p = a._floored(d, fn)
    assert np.ptp(p) > 0.3
    E = lambda dd: a.energy_density(dd, lam, fn)

    def fd(name, comp, scale):
        h = 1e-5 * scale
        return (E(_shift(d, name, comp, h)) - E(_shift(d, name, comp, -h))) / (2 * h)

    checks = [(fd("rho_a", 0, 0.01), P.V_a), (fd("rho_b", 0, 0.01), P.V_b),
              (fd("tau_a", 0, 0.01), 0.5 * P.alpha_a), (fd("tau_b", 0, 0.01), 0.5 * P.alpha_b),
              (fd("nu", 0, 0.003), -2 * P.Delta.real), (fd("nu", 1, 0.003), -2 * P.Delta.imag)]
    checks += [(fd("j_a", c, 0.002), P.Avec_a[c]) for c in range(3)]
    checks += [(fd("j_b", c, 0.002), P.Avec_b[c]) for c in range(3)]
    for k, (num, ana) in enumerate(checks):
        scale = max(np.abs(ana).max(), 1e-3)
        assert np.abs(num - ana).max() < 1e-7 * scale, (k, num, ana)
    # sensitivity: without the p-derivative terms V_a misses the central difference
    _, _, rt, _ = a._floored(d, fn)
    eF = o.fermi_energy(rt)
    V_plain = a.B(p) * eF - np.abs(P.Delta) ** 2 / (3 * fn.C * np.cbrt(rt) ** 2)
    assert np.abs(V_plain - fd("rho_a", 0, 0.01)).max() > 1e-3 * np.abs(P.V_a).max()


def test_normal_uniform_energies_of_the_parametrisation():
    """Uniform normal states (nu = 0, j = 0, tau_s of a free Fermi sea of each
    species): the printed A(p), B(p) give E = 2^(2/3) 0.357 E_FG unpolarised
    (the normal-state xi_N) and E = (0.357 + 0.642) E_free fully polarised."""
    fn = a.ASLDA(mu_a=0.0, mu_b=0.0)
    rho = 0.017
    tau = lambda r: 0.6 * r * (6 * np.pi ** 2 * r) ** (2.0 / 3.0)
    z = np.zeros((3, 1))
    half = a.Densities(np.array([rho / 2]), np.array([rho / 2]), np.array([tau(rho / 2)]),
                       np.array([tau(rho / 2)]), np.zeros(1, complex), z, z)
    e_fg = 0.6 * rho * o.fermi_energy(rho)
    assert abs(a.energy_density(half, 0.0, fn)[0] / e_fg - 2 ** (2 / 3) * 0.357) < 1e-12
    full = a.Densities(np.array([rho]), np.array([0.0]), np.array([tau(rho)]), np.array([0.0]),
                       np.zeros(1, complex), z, z)
    e_free = 0.5 * tau(rho)
    assert abs(a.energy_density(full, 0.0, fn)[0] / e_free - (0.357 + 0.642)) < 1e-12


def _trig_field(lat, seed, complex_=True, n=None, mmax=1):
    """Sum of the modes |m_d| <= mmax with seeded coefficients (band-limited)."""
    nm = (2 * mmax + 1) ** 3
    shape = (nm,) if n is None else (n, nm)
    u = inputs.uniform01(seed, 2 * int(np.prod(shape))).reshape(shape + (2,))
    c = (2 * u[..., 0] - 1) + (1j * (2 * u[..., 1] - 1) if complex_ else 0)
    x = [np.arange(N) * d for N, d in zip(lat.shape, (lat.dx, lat.dy, lat.dz))]
    X, Y, Z = np.meshgrid(*x, indexing="ij")
    r = range(-mmax, mmax + 1)
    waves = []
    for mx in r:
        for my in r:
            for mz in r:
                k = [2 * np.pi * m / (N * d) for m, N, d in zip((mx, my, mz), lat.shape, (lat.dx, lat.dy, lat.dz))]
                waves.append(np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z)).reshape(-1))
    f = np.tensordot(c, np.array(waves), axes=([-1], [0]))
    return f if complex_ else f.real


def test_kinetic_operator_of_eq_kinop_alpha():
    """For band-limited alpha and f (products clear of the Nyquist planes) the
    symmetrised form equals -1/2 sum_d d_d (alpha d_d f) exactly."""
    lat = o.Lattice(8, 8, 10, 1.0, 0.9, 1.1)
    alpha = 1.0 + 0.05 * _trig_field(lat, 3, complex_=False)
    f = _trig_field(lat, 5, n=3)
    gf = o.gradient(f, lat)
    ref = -0.5 * sum(o.gradient(alpha * gf[d], lat)[d] for d in range(3))
    got = a.kinetic(alpha, f, lat)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    # a constant alpha gives -alpha/2 lap
    assert np.abs(a.kinetic(np.full(lat.M, 1.094), f, lat) + 0.547 * o.laplacian(f, lat)).max() < 1e-13


def test_spin_symmetric_limit_reproduces_the_A_1094_oracle():
    """States of a spin-symmetric A = 1.094 case plus their partners
    [v^*, -u^*] (energy -E_n, weights swapped) in the imbalanced formulation
    with mu_a = mu_b: the same densities and potentials, the same f for the
    states, and the partner transform of f for the partners."""
    case = make_case((8, 8, 8), nstates=60, trap=0.08, seed=4, thermal=True, vortex=True, A=o.aslda_A(0.0))
    sysm = oracle_system(case)
    sysm.init_regulator(case.phi)
    j = sysm.current(case.phi)
    rho, nu, U, delta, _ = sysm.potentials(case.phi, j)
    f_sym = sysm.f(case.phi)
    u, v = case.phi[:, 0], case.phi[:, 1]
    phi = np.concatenate([case.phi, np.stack([np.conj(v), -np.conj(u)], axis=1)])
    fp = np.concatenate([case.wp, case.wm])
    fm = np.concatenate([case.wm, case.wp])
    fn = a.ASLDA(mu_a=case.fn.mu, mu_b=case.fn.mu, C=case.fn.C)
    sys_i = a.ImbalancedSystem(case.lat, fn, case.vext, case.vext, fp, fm)
    sys_i.init_regulator(phi)
    d = a.densities(phi, fp, fm, case.lat)
    P = a.potentials(d, sys_i.lam, fn)
    rel = lambda x, y: np.abs(x - y).max() / np.abs(y).max()
    assert np.abs(j).max() > 1e-6
    assert rel(sys_i.lam, sysm.lam) < 1e-13
    assert rel(d.rho_a, rho) < 1e-13 and rel(d.rho_b, rho) < 1e-13 and rel(d.nu, nu) < 1e-13
    assert rel(d.j_a, j) < 1e-12 and rel(d.j_b, j) < 1e-12
    assert rel(P.V_a, U) < 1e-12 and rel(P.V_b, U) < 1e-12 and rel(P.Delta, delta) < 1e-12
    f_i = sys_i.f(phi)
    n = case.phi.shape[0]
    assert rel(f_i[:n], f_sym) < 1e-12
    partner = np.stack([np.conj(f_sym[:, 1]), -np.conj(f_sym[:, 0])], axis=1)
    assert rel(f_i[n:], partner) < 1e-12


def test_energy_changes_by_the_centre_of_mass_terms_with_polarisation():
    """A boost u -> e^{iq.r} u, v -> e^{-iq.r} v of band-limited states with
    unequal species (p != 0): E' = E + q.P + (N_a + N_b) q^2 / 2."""
    lat = o.Lattice(8, 8, 10, 1.0, 0.9, 1.1)
    n = 10
    phi = o.normalize(np.stack([_trig_field(lat, 31, n=n), _trig_field(lat, 37, n=n)], axis=1), lat)
    fp = 0.7 * inputs.uniform01(41, n)
    fm = 0.3 + 0.7 * inputs.uniform01(43, n)
    fn = a.ASLDA(mu_a=0.3, mu_b=0.1)
    vext = inputs.harmonic_trap(lat.shape, 0.08)
    sys_i = a.ImbalancedSystem(lat, fn, vext, 0.5 * vext, fp, fm)
    sys_i.init_regulator(phi)
    d = a.densities(phi, fp, fm, lat)
    _, _, _, p = a._floored(d, fn)
    assert np.abs(p).max() > 0.05
    mq = (1, 1, -1)
    q = np.array([2 * np.pi * m / (N * dd) for m, N, dd in zip(mq, lat.shape, (lat.dx, lat.dy, lat.dz))])
    x = [np.arange(N) * dd for N, dd in zip(lat.shape, (lat.dx, lat.dy, lat.dz))]
    X, Y, Z = np.meshgrid(*x, indexing="ij")
    ph = np.exp(1j * (q[0] * X + q[1] * Y + q[2] * Z)).reshape(-1)
    boosted = np.stack([phi[:, 0] * ph, phi[:, 1] * np.conj(ph)], axis=1)
    e, eb = sys_i.energy(phi), sys_i.energy(boosted)
    want = e["e_total"] + q @ e["P"] + 0.5 * (e["n_a"] + e["n_b"]) * (q @ q)
    assert abs(eb["e_total"] - want) < 1e-12 * abs(want)
    db = a.densities(boosted, fp, fm, lat)
    assert np.abs(db.j_a - (d.j_a + d.rho_a[None] * q[:, None])).max() < 1e-13
    assert np.abs(db.j_b - (d.j_b + d.rho_b[None] * q[:, None])).max() < 1e-13


@pytest.mark.parametrize("stationary", [True, False])
def test_spin_symmetric_evolution_is_reproduced(stationary):
    """AB4AM5 steps (Alg. 2) after a stationary or Taylor start, of states plus
    partners in the imbalanced formulation, track the spin-symmetric
    A = 1.094 oracle: the states themselves, and the partner transform of them
    for the partners."""
    case = make_case((8, 8, 8), nstates=40, trap=0.08, seed=6, thermal=True, vortex=True, A=o.aslda_A(0.0))
    sysm = oracle_system(case)
    dt, nsteps = 0.01, 5
    st = o.start_scheme(sysm, case.phi, dt, stationary, "AB4AM5")
    st = o.evolve_scheme(sysm, st, dt, nsteps - st.steps, "AB4AM5")
    u, v = case.phi[:, 0], case.phi[:, 1]
    phi = np.concatenate([case.phi, np.stack([np.conj(v), -np.conj(u)], axis=1)])
    fp = np.concatenate([case.wp, case.wm])
    fm = np.concatenate([case.wm, case.wp])
    sys_i = a.ImbalancedSystem(case.lat, a.ASLDA(mu_a=case.fn.mu, mu_b=case.fn.mu, C=case.fn.C),
                               case.vext, case.vext, fp, fm)
    st_i = a.start(sys_i, phi, dt, stationary)
    st_i = a.evolve(sys_i, st_i, dt, nsteps - st_i.steps)
    n = case.phi.shape[0]
    ref = st.phi
    partner = np.stack([np.conj(ref[:, 1]), -np.conj(ref[:, 0])], axis=1)
    assert np.abs(st_i.phi[:n] - ref).max() < 1e-11 * np.abs(ref).max()
    assert np.abs(st_i.phi[n:] - partner).max() < 1e-11 * np.abs(ref).max()
    # the states moved: the comparison is not one of unchanged inputs
    assert np.abs(ref - o.normalize(case.phi, case.lat)).max() > 1e-4 * np.abs(ref).max()
