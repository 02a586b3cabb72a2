"""Static self-consistent solve on the GPU (Alg. 1) against the oracle.

The CUDA path diagonalises the 8 reflection-parity blocks of the BdG matrix;
the oracle diagonalises the full 2M x 2M matrix. Eigenvectors of degenerate
levels are not unique, so the comparison is on what is: the sorted
quasiparticle spectrum, the densities, the energy terms, mu and the
iteration count.
"""
import numpy as np
import pytest

from oracle import scf
from oracle import tdslda as o
from paper_2602_08982_b300 import inputs

pytestmark = pytest.mark.gpu

RHO_S = 1.0 / (6 * np.pi ** 2)


def _bdg_trap(shape, inv_kfa, omega):
    lat = o.Lattice(*shape)
    sd = o.uniform_bdg_seed(lat, inv_kfa / (4 * np.pi), RHO_S)
    fn = o.Functional("bdg", B=0.0, inv_4pi_a=inv_kfa / (4 * np.pi), mu=sd.mu)
    return lat, sd, fn, inputs.harmonic_trap(lat.shape, omega)


def _ctx(W, prec, lat, fn, vext):
    ctx = W.Context(prec)
    kind = W.SLDA_A1 if fn.kind == "slda" else W.BDG
    b = ctx.add_box(lat.shape, (lat.dx, lat.dy, lat.dz), kind=kind, B=fn.B, C=fn.C, inv_4pi_a=fn.inv_4pi_a,
                    mu=fn.mu, nstates=lat.M)
    ctx.set_vext(b, vext)
    return ctx, b


def _compare(res, E, rho, nu, ref, e_tol, f_tol=1e-11):
    assert np.abs(np.sort(E) - np.sort(ref.last.E)).max() < f_tol * ref.last.E.max()
    assert np.abs(rho - ref.last.rho).max() < f_tol * ref.last.rho.max()
    assert np.abs(nu - ref.last.nu).max() < f_tol * np.abs(ref.last.nu).max()
    for k in ("e_kin", "e_pot", "e_pair", "e_ext", "e_total", "n_part"):
        r = ref.history[-1][k]
        assert abs(res["energy"][k] - r) <= e_tol * max(1.0, abs(r)), k
    assert res["iters"] == ref.iters and res["converged"] == ref.converged
    assert abs(res["mu"] - ref.mu) < 1e-13


@pytest.mark.parametrize("shape,omega", [((8, 12, 16), (0.3, 0.2, 0.15)), ((8, 8, 8), (0.3, 0.25, 0.2))])
def test_fixed_iterations_match_oracle_fp64(shape, omega):
    from paper_2602_08982_b300 import wslda as W
    lat, sd, fn, v = _bdg_trap(shape, 1.0, omega)
    n_it = 3 if lat.M > 1000 else 6
    ref = scf.static_solve(lat, fn, v, np.zeros(lat.M), np.full(lat.M, sd.delta), eps_energy=0.0, max_iters=n_it)
    ctx, b = _ctx(W, W.FP64, lat, fn, v)
    res, E = ctx.static_solve(b, np.zeros(lat.M), np.full(lat.M, sd.delta), eps_energy=0.0, max_iters=n_it)
    rho, nu = ctx.get_densities(b)
    ctx.close()
    _compare(res, E, rho, nu, ref, 1e-10)


@pytest.fixture(scope="module")
def converged_8():
    lat, sd, fn, v = _bdg_trap((8, 8, 8), 1.0, (0.3, 0.25, 0.2))
    ref = scf.static_solve(lat, fn, v, np.zeros(lat.M), np.full(lat.M, sd.delta), mixing=1.0, eps_energy=1e-8,
                           max_iters=300)
    return lat, sd, fn, v, ref


def test_converged_solution_matches_oracle_and_is_stationary(converged_8):
    """Same iteration count and fixed point as the oracle; the eigenstates then
    stay put under the time-dependent step (Sec. 3.3 static-TD consistency)."""
    from paper_2602_08982_b300 import wslda as W
    lat, sd, fn, v, ref = converged_8
    assert ref.converged
    ctx, b = _ctx(W, W.FP64, lat, fn, v)
    res, E = ctx.static_solve(b, np.zeros(lat.M), np.full(lat.M, sd.delta), mixing=1.0, eps_energy=1e-8,
                              max_iters=300)
    rho, nu = ctx.get_densities(b)
    _compare(res, E, rho, nu, ref, 1e-9)
    ctx.start(True, 0.01)
    ctx.step(0.01, 20)
    rho2, nu2 = ctx.get_densities(b)
    ctx.close()
    assert np.abs(rho2 - rho).max() < 1e-8 * rho.max()
    assert np.abs(nu2 - nu).max() < 1e-8 * np.abs(nu).max()


def test_mixed_box_gets_rounded_eigenstates(converged_8):
    from paper_2602_08982_b300 import wslda as W
    lat, sd, fn, v, ref = converged_8
    ctx, b = _ctx(W, W.MIXED, lat, fn, v)
    res, E = ctx.static_solve(b, np.zeros(lat.M), np.full(lat.M, sd.delta), mixing=1.0, eps_energy=1e-8,
                              max_iters=300)
    rho, nu = ctx.get_densities(b)
    ctx.close()
    assert res["iters"] == ref.iters
    assert np.abs(rho - ref.last.rho).max() < 1e-6 * ref.last.rho.max()
    assert np.abs(nu - ref.last.nu).max() < 1e-6 * np.abs(ref.last.nu).max()


def test_fixed_particle_number_returns_to_the_uniform_slda_seed():
    """Eq. update-mu on an 8^3 uniform SLDA system started 10% off the
    self-consistent seed, with mu off by 0.05."""
    from paper_2602_08982_b300 import wslda as W
    lat = o.Lattice(8, 8, 8)
    sd = o.uniform_slda_seed(lat, 0.25, RHO_S)
    fn = o.Functional("slda", B=o.B_SLDA, C=sd.C, mu=sd.mu + 0.05)
    ctx, b = _ctx(W, W.FP64, lat, fn, np.zeros(lat.M))
    n_req = RHO_S * lat.volume
    res, E = ctx.static_solve(b, np.full(lat.M, 0.9 * sd.U), np.full(lat.M, 0.9 * sd.delta), eps_energy=1e-9,
                              max_iters=400, n_target=n_req, a_mu=0.5, eps_npart=1e-8)
    U, delta = ctx.get_fields(b)
    ctx.close()
    assert res["converged"]
    assert abs(res["n_sigma"] - n_req) < 1e-8
    assert abs(res["mu"] - sd.mu) < 1e-7
    assert np.abs(U - sd.U).max() < 1e-6 and np.abs(delta.real - sd.delta).max() < 1e-6
    k2 = lat.k2().reshape(-1)
    E_bcs = np.sort(np.sqrt((0.5 * k2 - sd.mu_eff) ** 2 + sd.delta ** 2))
    assert np.abs(np.sort(E) - E_bcs).max() < 1e-6


def test_broyden_iterations_match_oracle():
    from paper_2602_08982_b300 import wslda as W
    lat, sd, fn, v = _bdg_trap((8, 8, 8), 1.0, (0.3, 0.25, 0.2))
    ref = scf.static_solve(lat, fn, v, np.zeros(lat.M), np.full(lat.M, sd.delta), mixing=0.5, eps_energy=0.0,
                           max_iters=9, method="broyden")
    ctx, b = _ctx(W, W.FP64, lat, fn, v)
    res, E = ctx.static_solve(b, np.zeros(lat.M), np.full(lat.M, sd.delta), mixing=0.5, eps_energy=0.0,
                              max_iters=9, method="broyden")
    rho, nu = ctx.get_densities(b)
    ctx.close()
    # each Broyden step solves with w0^2 I + A, whose condition number reaches
    # (w0^2 + k) / w0^2 ~ 7e4 for w0 = 0.01 and k = 7 stored pairs, so rounding
    # differences between the two sides grow by up to that factor per step
    _compare(res, E, rho, nu, ref, 1e-9, f_tol=1e-9)


def test_broyden_with_mu_update_returns_to_the_uniform_slda_seed():
    from paper_2602_08982_b300 import wslda as W
    lat = o.Lattice(8, 8, 8)
    sd = o.uniform_slda_seed(lat, 0.25, RHO_S)
    fn = o.Functional("slda", B=o.B_SLDA, C=sd.C, mu=sd.mu + 0.05)
    ctx, b = _ctx(W, W.FP64, lat, fn, np.zeros(lat.M))
    n_req = RHO_S * lat.volume
    res, E = ctx.static_solve(b, np.full(lat.M, 0.9 * sd.U), np.full(lat.M, 0.9 * sd.delta), eps_energy=1e-10,
                              max_iters=100, n_target=n_req, a_mu=0.5, eps_npart=1e-9, method="broyden")
    ctx.close()
    assert res["converged"] and res["iters"] < 50
    assert abs(res["mu"] - sd.mu) < 1e-8


def test_rejected_inputs():
    from paper_2602_08982_b300 import wslda as W
    lat, sd, fn, v = _bdg_trap((8, 8, 8), 1.0, (0.3, 0.25, 0.2))
    U0, d0 = np.zeros(lat.M), np.full(lat.M, sd.delta)
    # a trap centred off the reflection point
    ctx, b = _ctx(W, W.FP64, lat, fn, np.roll(v, 1))
    with pytest.raises(W.WsldaError) as e:
        ctx.static_solve(b, U0, d0)
    assert e.value.status == 1
    ctx.close()
    # external pairing field
    ctx, b = _ctx(W, W.FP64, lat, fn, v)
    ctx.set_dext(b, np.full(lat.M, 1e-3 + 0j))
    with pytest.raises(W.WsldaError) as e:
        ctx.static_solve(b, U0, d0)
    assert e.value.status == 1
    ctx.close()
    # fewer states than lattice sites
    ctx = W.Context(W.FP64)
    b = ctx.add_box(lat.shape, kind=W.BDG, inv_4pi_a=fn.inv_4pi_a, mu=fn.mu, nstates=lat.M - 1)
    with pytest.raises(W.WsldaError) as e:
        ctx.static_solve(b, U0, d0)
    assert e.value.status == 1
    ctx.close()
    # bad mixing
    ctx, b = _ctx(W, W.FP64, lat, fn, v)
    with pytest.raises(W.WsldaError):
        ctx.static_solve(b, U0, d0, mixing=1.5)
    ctx.close()


def test_16cubed_trap_converges_and_stays_stationary():
    """GPU only (the dense oracle would need a 8192 x 8192 matrix per
    iteration): convergence, a positive spectrum, and stationarity."""
    from paper_2602_08982_b300 import wslda as W
    lat, sd, fn, v = _bdg_trap((16, 16, 16), 1.0, (0.12, 0.1, 0.08))
    ctx, b = _ctx(W, W.FP64, lat, fn, v)
    res, E = ctx.static_solve(b, np.zeros(lat.M), np.full(lat.M, sd.delta), mixing=0.5, eps_energy=1e-9,
                              max_iters=150, method="broyden")
    assert res["converged"] and E.min() > 0
    rho, nu = ctx.get_densities(b)
    assert abs(lat.dV * rho.sum() - res["n_sigma"]) < 1e-10 * res["n_sigma"]
    ctx.start(True, 0.01)
    ctx.step(0.01, 10)
    rho2, _ = ctx.get_densities(b)
    ctx.close()
    assert np.abs(rho2 - rho).max() < 1e-7 * rho.max()


def test_single_precision_warmup_reaches_the_double_fixed_point(converged_8):
    """Leading iterations diagonalised in float change the path, not the fixed
    point: the final double-precision iterations land where the double-only
    solve does."""
    from paper_2602_08982_b300 import wslda as W
    lat, sd, fn, v, ref = converged_8
    ctx, b = _ctx(W, W.FP64, lat, fn, v)
    res, E = ctx.static_solve(b, np.zeros(lat.M), np.full(lat.M, sd.delta), mixing=1.0, eps_energy=1e-8,
                              max_iters=300, fp32_iters=10)
    rho, nu = ctx.get_densities(b)
    ctx.close()
    assert res["converged"] and res["iters"] > 11
    assert np.abs(np.sort(E) - np.sort(ref.last.E)).max() < 1e-6 * ref.last.E.max()
    assert np.abs(rho - ref.last.rho).max() < 1e-6 * ref.last.rho.max()
    assert np.abs(nu - ref.last.nu).max() < 1e-6 * np.abs(ref.last.nu).max()


def test_trapped_slda_with_the_printed_C_matches_oracle_and_is_stationary():
    """Reading K6: trapped SLDA (A = 1, B(0), C = -11.11) with a particle-number
    target and Broyden mixing converges on the GPU to the oracle's fixed point
    (same iterations, spectrum, densities, mu), and the static states stay put
    under the time-dependent step."""
    from paper_2602_08982_b300 import wslda as W
    lat = o.Lattice(8, 8, 8)
    v = inputs.harmonic_trap(lat.shape, 0.12)
    sd = o.uniform_slda_seed(o.Lattice(16, 16, 16), 0.25, RHO_S)
    fn = o.Functional("slda", B=o.B_SLDA, C=o.C_ASLDA, mu=sd.mu)
    kw = dict(mixing=0.3, eps_energy=1e-7, max_iters=60, method="broyden", n_target=10.0, a_mu=0.5, eps_npart=1e-4)
    ref = scf.static_solve(lat, fn, v, np.full(lat.M, sd.U), np.full(lat.M, sd.delta), **kw)
    assert ref.converged
    ctx, b = _ctx(W, W.FP64, lat, fn, v)
    res, E = ctx.static_solve(b, np.full(lat.M, sd.U), np.full(lat.M, sd.delta), **kw)
    rho, nu = ctx.get_densities(b)
    _compare(res, E, rho, nu, ref, 1e-8, f_tol=1e-8)
    assert abs(res["n_sigma"] - 10.0) < 1e-4 and np.abs(nu).max() > 1e-3
    ctx.start(True, 0.01)
    ctx.step(0.01, 10)
    rho2, _ = ctx.get_densities(b)
    ctx.close()
    assert np.abs(rho2 - rho).max() < 1e-6 * rho.max()
