"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerances: the plain FP64 path must match the oracle within 1e-12 relative on
rho, nu, the states and the energy; the mixed path (complex float states and
FFTs, double reductions) within 1e-5 relative. Cases span several tiles and
ragged state counts, anisotropic lattices and spacings, thermal weights, both
functionals, cluster sizes 1-16 and pencils split over 1, 2 and 4 lanes.
"""
import os

import numpy as np
import pytest

from cases import gpu_context, make_case, oracle_evolve, oracle_system, rel
from oracle import tdslda as o

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def W():
    from paper_2602_08982_b300 import wslda
    return wslda


def _compare_f(W, case, prec, tol):
    ctx, box = gpu_context(case, prec)
    f_gpu = ctx.eval_f(box)
    sysm = oracle_system(case)
    sysm.init_regulator(case.phi)
    f_ref = sysm.f(case.phi)
    # the f of a plane-wave state in a trap is O(1); compare against the H scale
    scale = np.abs(o.apply_H(case.phi, sysm.fields(case.phi), case.lat)).max()
    err = np.abs(f_gpu - f_ref).max() / scale
    U_g, D_g = ctx.get_fields(box)
    rho_s, nu, U, delta, _ = sysm.potentials(case.phi)
    ctx.close()
    assert err < tol, err
    assert rel(U_g, U) < tol and rel(D_g, delta) < tol


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,spacing,kind,n", [
    ((8, 8, 8), (1, 1, 1), "slda", None),
    ((8, 12, 16), (1.0, 0.9, 1.1), "bdg", 301),
    ((12, 12, 12), (1, 1, 1), "slda", 700),
    ((16, 16, 16), (1, 1, 1), "slda", 513),
    ((32, 32, 32), (1, 1, 1), "slda", 300),
    ((12, 12, 48), (1, 1, 1), "slda", 200),
])
def test_f_matches_oracle(W, prec, shape, spacing, kind, n):
    """f(phi) = -i [H - <H>_n] phi (Eq. ABM-f) with potentials from the
    densities of all states, at t = 0, for a trap plus a pairing kick."""
    if not W.lattice_supported(prec, *shape):
        pytest.skip("shape not compiled for this precision")
    case = make_case(shape, spacing, kind=kind, nstates=n, trap=0.08, kick=0.05, seed=3)
    _compare_f(W, case, prec, TOL[prec] * (10 if prec == 0 else 1))


@pytest.mark.parametrize("shape", [(18, 18, 18), (20, 20, 20), (24, 24, 24), (24, 24, 96)])
def test_f_matches_oracle_mixed_more_shapes(W, shape):
    case = make_case(shape, kind="slda", nstates=150, trap=0.06, kick=0.05, seed=4, vortex=shape[2] == 96)
    _compare_f(W, case, 1, TOL[1])


def _evolve_and_compare(W, case, prec, dt, nsteps, stationary, tol):
    ctx, box = gpu_context(case, prec)
    ctx.start(stationary, dt)
    t0, s0 = ctx.get_time()
    ctx.step(dt, nsteps - s0)
    t, s = ctx.get_time()
    assert s == nsteps and abs(t - nsteps * dt) < 1e-12
    rho_g, nu_g = ctx.get_densities(box)
    e_g = ctx.get_energy(box)
    phi_g = ctx.get_states(box)
    ctx.close()
    ref_in = case.phi
    if prec == 1:  # the mixed path starts from the float-rounded states
        ref_in = case.phi.astype(np.complex64).astype(np.complex128)
    sysm, st = oracle_evolve(case, dt, nsteps, stationary, phi0=ref_in)
    rho_r, nu_r = o.densities(st.phi, case.wm, case.wp)
    e_r = sysm.energy(st.phi)
    errs = dict(rho=rel(rho_g, rho_r), nu=rel(nu_g, nu_r), states=rel(phi_g, st.phi),
                e_total=abs(e_g["e_total"] - e_r["e_total"]) / abs(e_r["e_total"]),
                e_kin=abs(e_g["e_kin"] - e_r["e_kin"]) / abs(e_r["e_kin"]),
                n_part=abs(e_g["n_part"] - e_r["n_part"]) / abs(e_r["n_part"]))
    bad = {k: v for k, v in errs.items() if not v < tol}
    assert not bad, errs
    return errs


@pytest.mark.parametrize("prec", [0, 1])
def test_taylor_start_and_steps_8cubed(W, prec):
    case = make_case((8, 8, 8), trap=0.1, kick=0.05, seed=5)
    _evolve_and_compare(W, case, prec, 0.01, 12, False, TOL[prec])


@pytest.mark.parametrize("prec", [0, 1])
def test_steps_anisotropic_bdg_thermal(W, prec):
    case = make_case((8, 12, 16), (1.0, 0.9, 1.1), kind="bdg", nstates=301, trap=0.1, kick=0.05, seed=6,
                     thermal=True)
    _evolve_and_compare(W, case, prec, 0.01, 10, False, TOL[prec])


@pytest.mark.parametrize("prec", [0, 1])
def test_stationary_start_32cubed_clusters(W, prec):
    """32^3 runs on clusters of 16 (double) and 8 (float) CTAs with the x pass
    over distributed shared memory; pencils split over 2 lanes in double."""
    case = make_case((32, 32, 32), nstates=257, trap=0.05, kick=0.02, seed=7)
    _evolve_and_compare(W, case, prec, 0.007, 4, True, TOL[prec])


def test_mixed_elongated_vortex(W):
    case = make_case((12, 12, 48), nstates=333, trap=0.064, kick=0.0, seed=8, vortex=True)
    _evolve_and_compare(W, case, 1, 0.007, 8, False, TOL[1])


@pytest.mark.parametrize("prec", [0, 1])
def test_uniform_seed_is_stationary_16cubed(W, prec):
    """All 4096 plane-wave states of the self-consistent uniform SLDA seed:
    f vanishes and the states do not move (Sec. 3.3)."""
    case = make_case((16, 16, 16), seed=9)
    ctx, box = gpu_context(case, prec)
    f = ctx.eval_f(box)
    assert np.abs(f).max() < (1e-11 if prec == 0 else 2e-5)
    ctx.start(True, 0.01)
    ctx.step(0.01, 5)
    phi = ctx.get_states(box)
    ctx.close()
    assert rel(phi, case.phi) < (1e-12 if prec == 0 else 1e-5)


@pytest.mark.parametrize("prec", [0, 1])
def test_c1_config_16cubed_20_steps(W, prec):
    """The plain FP64 uniform unitary gas on 16^3 (all 4096 states), seeded
    1e-3 pairing perturbation, Taylor start, 20 steps of dt = 0.01, against
    the stored oracle run (tests/golden/c1_100steps.npz, step 20): FP64 within
    1e-12; the mixed path, started from the same double states (its rounding
    to complex float included), within 1e-5."""
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "c1_100steps.npz"))
    case = make_case((16, 16, 16), kick=1e-3, seed=1)
    ctx, box = gpu_context(case, prec)
    ctx.start(False, 0.01)
    ctx.step(0.01, 17)
    rho, nu = ctx.get_densities(box)
    e = ctx.get_energy(box)
    ctx.close()
    errs = dict(rho=rel(rho, g["rho_20"]), nu=rel(nu, g["nu_20"]),
                e_total=abs(e["e_total"] - float(g["e_total_20"])) / abs(float(g["e_total_20"])))
    print("c1", prec, errs)
    assert all(v < TOL[prec] for v in errs.values()), errs


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,spacing,n", [((8, 12, 16), (1.0, 0.9, 1.1), 301), ((32, 32, 32), (1, 1, 1), 129)])
def test_tau_and_current_match_oracle(W, prec, shape, spacing, n):
    """tau and j (Eqs. nab3D..jab3D) with Nyquist-free spectral gradients, after
    a few steps so that j is non-zero (trap + pairing kick + thermal weights)."""
    case = make_case(shape, spacing, nstates=n, trap=0.1, kick=0.05, seed=12, thermal=True)
    ctx, box = gpu_context(case, prec)
    ctx.start(False, 0.01)
    ctx.step(0.01, 2)
    rho, nu, tau, j = ctx.get_densities(box, tau=True, current=True)
    ctx.close()
    ref_in = case.phi if prec == 0 else case.phi.astype(np.complex64).astype(np.complex128)
    sysm, st = oracle_evolve(case, 0.01, 5, False, phi0=ref_in)
    tau_r, j_r = o.kinetic_current_densities(st.phi, case.wm, case.wp, case.lat)
    assert rel(tau, tau_r) < TOL[prec]
    assert np.abs(j - j_r).max() / np.abs(j_r).max() < TOL[prec] * (10 if prec == 1 else 1)


def test_save_load_resume_is_bit_identical(W, tmp_path):
    case = make_case((8, 8, 8), trap=0.1, kick=0.05, seed=10)
    a, box = gpu_context(case, 0)
    a.start(False, 0.01)
    a.step(0.01, 3)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(0.01, 4)
    ref = a.get_states(box)
    a.close()
    b, box = gpu_context(case, 0)
    b.load(path)
    b.step(0.01, 4)
    got = b.get_states(box)
    b.close()
    assert np.array_equal(ref, got)


def test_conservation_diagnostics(W):
    """Energy (E_tot - mu N) and N drift checks of the TD codes (Sec. 4.5.1):
    small for a trapped evolution, and a zero tolerance trips WSLDA_EDRIFT
    (host-side fault injection, no GPU fault), which then sticks."""
    case = make_case((8, 8, 8), trap=0.1, seed=13)
    ctx, box = gpu_context(case, 0)
    ctx.start(False, 0.005)
    ctx.step(0.005, 20)
    de, dn = ctx.check_conservation(box, 1e-6, 1e-6)
    assert de < 1e-6 and dn < 1e-6
    with pytest.raises(W.WsldaError) as e:
        ctx.check_conservation(box, 0.0, 0.0)
    assert e.value.status == 5
    with pytest.raises(W.WsldaError) as e:
        ctx.step(0.005, 1)
    assert e.value.status == 7
    ctx.close()


def test_errors_are_status_codes(W):
    ctx = W.Context(W.FP64)
    with pytest.raises(W.WsldaError) as e:
        ctx.add_box((7, 8, 8), nstates=4)
    assert e.value.status == 1
    ctx.close()
    ctx = W.Context(W.FP64)
    with pytest.raises(W.WsldaError) as e:
        ctx.add_box((14, 14, 14), nstates=4)
    assert e.value.status == 8
    ctx.close()
    case = make_case((8, 8, 8), seed=11)
    bad = case.phi.copy()
    bad[3, 1, 5] = np.nan
    ctx = W.Context(W.FP64)
    box = ctx.add_box((8, 8, 8), C=case.fn.C, B=case.fn.B, mu=case.fn.mu, nstates=bad.shape[0])
    with pytest.raises(W.WsldaError) as e:
        ctx.load_states(box, bad)
    assert e.value.status == 4
    with pytest.raises(W.WsldaError) as e:
        ctx.step(0.01, 1)
    assert e.value.status == 7  # sticky error
    ctx.close()
    ctx = W.Context(W.MIXED)
    with pytest.raises(W.WsldaError) as e:
        ctx.add_box((32, 32, 32), nstates=10 ** 8)
    assert e.value.status == 2
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_complex_float_state_io(prec):
    """load_states_f32 / get_states_f32 carry the same states as the double
    calls: a mixed box stores exactly the rounded values either way, and the
    read-outs agree to float rounding."""
    c = make_case((8, 8, 8), kick=0.05, trap=0.1, seed=71)
    a, box = gpu_context(c, prec)
    a.start(False, 0.01)
    a.step(0.01, 2)
    ref = a.get_states(box)
    got = a.get_states_f32(box)
    a.close()
    assert got.dtype == np.complex64
    assert np.abs(got - ref).max() <= 2.0 ** -23 * np.abs(ref).max()
    from paper_2602_08982_b300 import wslda as W
    b = W.Context(prec)
    kind = W.SLDA_A1 if c.fn.kind == "slda" else W.BDG
    bx = b.add_box(c.lat.shape, kind=kind, B=c.fn.B, C=c.fn.C, inv_4pi_a=c.fn.inv_4pi_a, mu=c.fn.mu,
                   nstates=c.phi.shape[0])
    b.load_states_f32(bx, c.phi.astype(np.complex64))
    back = b.get_states(bx)
    b.close()
    assert np.array_equal(back, c.phi.astype(np.complex64).astype(np.complex128))


def test_fp64_rate_probes_measure_the_device():
    """The FP64 microbenchmarks behind the FP64 step's roofline: finite and
    positive, and an addition (one operation per instruction) issues no
    faster than an FMA delivers its two."""
    from paper_2602_08982_b300 import wslda as W
    fma = W.measure_fp64_rate(2)
    add = W.measure_fp64_add_rate(2)
    assert np.isfinite(fma) and np.isfinite(add) and fma > 0.1 and add > 0.05
    assert add < fma
