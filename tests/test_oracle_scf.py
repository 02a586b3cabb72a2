"""Pins of the static self-consistent solver oracle (Alg. 1, Sec. 3.2).

Each pin checks the oracle against something other than itself: the uniform
lattice seeds come from the number and gap equations solved as scalar root
problems over the k-set (no matrix, no eigensolver); the spectral symmetry and
the stationarity of a converged solution under the time-dependent right-hand
side are properties of the exact problem.
"""
import numpy as np
import pytest

from oracle import scf
from oracle import tdslda as o
from paper_2602_08982_b300 import inputs

RHO_S = 1.0 / (6 * np.pi ** 2)   # k_F = 1


def _bdg(lat, inv_kfa):
    sd = o.uniform_bdg_seed(lat, inv_kfa / (4 * np.pi), RHO_S)
    return sd, o.Functional("bdg", B=0.0, inv_4pi_a=inv_kfa / (4 * np.pi), mu=sd.mu)


def test_uniform_slda_seed_is_a_fixed_point_of_the_map():
    """The seed's C is backed out of the gap equation, so K must return the
    seed's (U, Delta) and its density exactly."""
    lat = o.Lattice(6, 6, 6)
    sd = o.uniform_slda_seed(lat, 0.25, RHO_S)
    fn = o.Functional("slda", B=o.B_SLDA, C=sd.C, mu=sd.mu)
    out = scf.map_K(lat, fn, np.zeros(lat.M), np.full(lat.M, sd.U), np.full(lat.M, sd.delta + 0j))
    assert np.abs(out.U - sd.U).max() < 1e-12 * abs(sd.U)
    assert np.abs(out.delta - sd.delta).max() < 1e-12 * sd.delta
    assert np.abs(out.rho - RHO_S).max() < 1e-12 * RHO_S
    assert np.abs(out.nu.imag).max() < 1e-14
    # every kept state has E > 0; the spectrum is the uniform BCS one
    k2 = lat.k2().reshape(-1)
    E_bcs = np.sort(np.sqrt((0.5 * k2 - sd.mu_eff) ** 2 + sd.delta ** 2))
    assert np.abs(np.sort(out.E) - E_bcs).max() < 1e-12


def test_uniform_bdg_iteration_converges_to_the_seed_gap():
    lat = o.Lattice(6, 6, 6)
    sd, fn = _bdg(lat, -0.5)
    r = scf.static_solve(lat, fn, np.zeros(lat.M), np.zeros(lat.M), np.full(lat.M, 0.5 * sd.delta),
                         eps_energy=1e-10, max_iters=300)
    assert r.converged
    assert np.abs(r.delta - sd.delta).max() < 1e-8 * sd.delta
    assert np.abs(r.U).max() == 0.0


def test_fixed_particle_number_mu_update_reaches_the_slda_seed():
    """Eq. update-mu with N_req = the seed's N: from 90% of the seed's
    potentials the iteration returns to the seed's (U, Delta, mu)."""
    lat = o.Lattice(6, 6, 6)
    sd = o.uniform_slda_seed(lat, 0.25, RHO_S)
    fn = o.Functional("slda", B=o.B_SLDA, C=sd.C, mu=sd.mu + 0.05)   # mu off by 0.05 at the start
    n_req = RHO_S * lat.volume
    r = scf.static_solve(lat, fn, np.zeros(lat.M), np.full(lat.M, 0.9 * sd.U), np.full(lat.M, 0.9 * sd.delta),
                         eps_energy=1e-9, max_iters=400, n_target=n_req, a_mu=0.5, eps_npart=1e-8)
    assert r.converged
    assert abs(lat.dV * r.last.rho.sum() - n_req) < 1e-8
    assert abs(r.mu - sd.mu) < 1e-7
    assert np.abs(r.U - sd.U).max() < 1e-7 and np.abs(r.delta - sd.delta).max() < 1e-7


def test_spectrum_is_plus_minus_symmetric_in_a_trap():
    lat = o.Lattice(6, 6, 8)
    sd, fn = _bdg(lat, 0.5)
    v = inputs.harmonic_trap(lat.shape, (0.15, 0.12, 0.1))
    delta = sd.delta * (1.0 + 0.3 * inputs.complex_noise(lat.shape, 5))   # complex, not symmetric
    out = scf.map_K(lat, fn, v, 0.1 * inputs.uniform01(6, lat.M), delta)
    ev = np.sort(out.evals)
    assert np.abs(ev + ev[::-1]).max() < 1e-12 * np.abs(ev).max()
    assert out.E.min() > 0


@pytest.fixture(scope="module")
def trapped():
    lat = o.Lattice(6, 6, 8)
    sd, fn = _bdg(lat, 1.0)
    v = inputs.harmonic_trap(lat.shape, (0.15, 0.12, 0.1))
    res = {m: scf.static_solve(lat, fn, v, np.zeros(lat.M), np.full(lat.M, sd.delta), mixing=m,
                               eps_energy=1e-9, max_iters=300) for m in (0.5, 1.0)}
    return lat, fn, v, res


def test_converged_trap_solution_is_a_fixed_point(trapped):
    lat, fn, v, res = trapped
    r = res[1.0]
    assert r.converged
    again = scf.map_K(lat, fn, v, r.U, r.delta)
    scale = np.abs(r.delta).max()
    assert np.abs(again.delta - r.delta).max() < 1e-8 * scale
    # the mixing parameter changes the path, not the fixed point
    assert res[0.5].converged
    assert np.abs(res[0.5].delta - r.delta).max() < 1e-8 * scale


def test_converged_trap_states_are_stationary_under_the_td_rhs(trapped):
    """Sec. 3.3: a self-consistent static solution does not evolve. With the
    regulator frozen at t = 0, f(phi) = -i (H - <H>_n) phi vanishes up to the
    self-consistency tolerance, and <H>_n is the quasiparticle energy."""
    lat, fn, v, res = trapped
    r = res[1.0]
    sysm = o.TDSystem(lat, fn, vext=v)
    sysm.init_regulator(r.phi)
    F = sysm.fields(r.phi)
    Hphi = o.apply_H(r.phi, F, lat)
    f = o.rhs_f(r.phi, F, lat)
    assert np.abs(f).max() < 1e-9 * np.abs(Hphi).max()
    assert np.abs(o.expectation(r.phi, Hphi, lat) - r.E).max() < 1e-9 * r.E.max()


def test_broyden_reaches_the_linear_mixing_fixed_point_faster(trapped):
    lat, fn, v, res = trapped
    sd, _ = _bdg(lat, 1.0)
    rb = scf.static_solve(lat, fn, v, np.zeros(lat.M), np.full(lat.M, sd.delta), mixing=0.5, eps_energy=1e-11,
                          max_iters=300, method="broyden")
    assert rb.converged and rb.iters < res[1.0].iters // 3
    scale = np.abs(res[1.0].delta).max()
    assert np.abs(rb.delta - res[1.0].delta).max() < 1e-8 * scale
    assert np.abs(np.sort(rb.E) - np.sort(res[1.0].E)).max() < 1e-9 * rb.E.max()


def test_broyden_with_mu_update_reaches_the_slda_seed():
    lat = o.Lattice(6, 6, 6)
    sd = o.uniform_slda_seed(lat, 0.25, RHO_S)
    fn = o.Functional("slda", B=o.B_SLDA, C=sd.C, mu=sd.mu + 0.05)
    n_req = RHO_S * lat.volume
    r = scf.static_solve(lat, fn, np.zeros(lat.M), np.full(lat.M, 0.9 * sd.U), np.full(lat.M, 0.9 * sd.delta),
                         eps_energy=1e-9, max_iters=100, n_target=n_req, a_mu=0.5, eps_npart=1e-8,
                         method="broyden")
    assert r.converged and r.iters < 40
    assert abs(r.mu - sd.mu) < 1e-8
    assert np.abs(r.U - sd.U).max() < 1e-8 and np.abs(r.delta - sd.delta).max() < 1e-8


def test_trapped_slda_converges_with_the_printed_C_and_not_with_the_seed_C():
    """Reading K6. The uniform A = 1 seed backs out C = +5.3 on these lattices
    (with the zone-corner cutoff of reading R5), which makes the density
    derivative of the pairing energy, -|Delta|^2 / (3 C rho^(2/3)), attractive
    and unbounded where rho -> 0: a trapped iteration with a particle-number
    target then oscillates. With the printed ASLDA C = -11.11 that term is
    repulsive, and the same iteration converges to a paired solution that is
    a fixed point of K with the requested N."""
    lat = o.Lattice(8, 8, 8)
    vext = inputs.harmonic_trap(lat.shape, 0.12)
    sd = o.uniform_slda_seed(o.Lattice(16, 16, 16), 0.25, RHO_S)
    assert sd.C > 0
    res = {}
    for C in (o.C_ASLDA, sd.C):
        fn = o.Functional("slda", B=o.B_SLDA, C=C, mu=sd.mu)
        res[C] = scf.static_solve(lat, fn, vext, np.full(lat.M, sd.U), np.full(lat.M, sd.delta), mixing=0.3,
                                  eps_energy=1e-6, max_iters=60, method="broyden", n_target=10.0, a_mu=0.5,
                                  eps_npart=1e-3)
    good, bad = res[o.C_ASLDA], res[sd.C]
    assert good.converged and good.iters < 45
    assert abs(lat.dV * good.last.rho.sum() - 10.0) < 1e-3
    assert np.abs(good.delta).max() > 0.05  # paired
    fn = o.Functional("slda", B=o.B_SLDA, C=o.C_ASLDA, mu=good.mu)
    again = scf.map_K(lat, fn, vext, good.U, good.delta)
    assert np.abs(again.U - good.U).max() < 1e-4 and np.abs(again.delta - good.delta).max() < 1e-4
    assert not bad.converged
