"""A != 1 SLDA step (current terms, Sec. 2.4 / Eq. h_sigma) of the CUDA path
against the oracle, element by element.

Tolerances as for the A = 1 path: the plain FP64 path within 1e-12 relative
(1e-11 for f, whose scale is set by H), the mixed path within 1e-5. The inputs
carry currents (a vortex phase imprint on u, a trap, a pairing kick and thermal
weights), so the per-stage current j, the current potential (1 - A) j / rho and
its divergence, the current part of U and the current term of H all enter.
A = 1.094 is A_a(0) of the ASLDA functional.
"""
import numpy as np
import pytest

from cases import gpu_context, make_case, oracle_system, rel
from oracle import tdslda as o

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}
A = o.aslda_A(0.0)


@pytest.fixture(scope="module")
def W():
    from paper_2602_08982_b300 import wslda
    return wslda


def _case(shape, spacing, n, seed=3):
    return make_case(shape, spacing, nstates=n, trap=0.08, kick=0.05, seed=seed, thermal=True, vortex=True, A=A)


def _ref_states(case, prec):
    # the mixed path starts from the states rounded to complex float
    return case.phi if prec == 0 else case.phi.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,spacing,n", [
    ((8, 12, 16), (1.0, 0.9, 1.1), 301),
    ((12, 12, 12), (1, 1, 1), 700),
    ((16, 16, 16), (1, 1, 1), 513),
    ((32, 32, 32), (1, 1, 1), 300),
])
def test_current_fields_and_f_match_oracle(W, prec, shape, spacing, n):
    """j (Eq. jab3D), U with its current part, Delta, and f = -i[H - <H>_n] phi
    with the current term, at t = 0 (regulator from the t = 0 fixed point)."""
    if not W.lattice_supported(prec, *shape):
        pytest.skip("shape not compiled for this precision")
    case = _case(shape, spacing, n)
    ctx, box = gpu_context(case, prec)
    f_gpu = ctx.eval_f(box)
    U_g, D_g = ctx.get_fields(box)
    _, _, _, j_g = ctx.get_densities(box, tau=True, current=True)
    e_g = ctx.get_energy(box)
    ctx.close()
    phi = _ref_states(case, prec)
    sysm = oracle_system(case)
    sysm.init_regulator(phi)
    F = sysm.fields(phi)
    j = sysm.current(phi)
    _, _, U, delta, _ = sysm.potentials(phi, j)
    f_ref = o.rhs_f(phi, F, case.lat)
    e_r = sysm.energy(phi)
    scale = np.abs(o.apply_H(phi, F, case.lat)).max()
    tol = TOL[prec]
    assert np.abs(j).max() > 1e-6 and np.abs(F.divA).max() > 1e-6   # currents and a non-zero div A
    errs = dict(j=rel(j_g, j), U=rel(U_g, U), delta=rel(D_g, delta),
                f=np.abs(f_gpu - f_ref).max() / scale,
                e_total=abs(e_g["e_total"] - e_r["e_total"]) / abs(e_r["e_total"]),
                e_cur=abs(e_g["e_cur"] - e_r["e_cur"]) / abs(e_r["e_cur"]))
    print("A != 1 fields", shape, prec, errs)
    assert errs["f"] < tol * (10 if prec == 0 else 1), errs
    assert all(v < tol for k, v in errs.items() if k != "f"), errs


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,spacing,n,stationary", [
    ((8, 12, 16), (1.0, 0.9, 1.1), 301, False),
    ((16, 16, 16), (1, 1, 1), 513, False),
    ((12, 12, 12), (1, 1, 1), 700, True),
])
def test_evolution_matches_oracle(W, prec, shape, spacing, n, stationary):
    """Taylor (or stationary) start and AB4AM5 steps (Alg. 2) with the current
    terms re-evaluated at every stage: rho, nu, the states and the energy."""
    if not W.lattice_supported(prec, *shape):
        pytest.skip("shape not compiled for this precision")
    case = _case(shape, spacing, n, seed=5)
    dt, nsteps = 0.01, 8
    ctx, box = gpu_context(case, prec)
    ctx.start(stationary, dt)
    ctx.step(dt, nsteps - (0 if stationary else 3))
    rho, nu = ctx.get_densities(box)
    phi = ctx.get_states(box)
    e = ctx.get_energy(box)
    ctx.close()
    sysm = oracle_system(case)
    st = o.start(sysm, _ref_states(case, prec), dt, stationary)
    st = o.evolve(sysm, st, dt, nsteps - st.steps)
    rho_r, nu_r = o.densities(st.phi, case.wm, case.wp)
    e_r = sysm.energy(st.phi)
    errs = dict(rho=rel(rho, rho_r), nu=rel(nu, nu_r), states=rel(phi, st.phi),
                e_total=abs(e["e_total"] - e_r["e_total"]) / abs(e_r["e_total"]),
                e_cur=abs(e["e_cur"] - e_r["e_cur"]) / abs(e_r["e_cur"]))
    print("A != 1 evolution", shape, prec, errs)
    assert all(v < TOL[prec] for v in errs.values()), errs


@pytest.fixture(scope="module")
def launch_form_case():
    """12^3 with 1000 states (more than the clusters resident at once, so the
    persistent form loops) and its oracle evolution, shared by both forms."""
    case = _case((12, 12, 12), (1, 1, 1), 1000, seed=7)
    sysm = oracle_system(case)
    st = o.start(sysm, _ref_states(case, 1), 0.01, False)
    st = o.evolve(sysm, st, 0.01, 6 - st.steps)
    return case, o.densities(st.phi, case.wm, case.wp)


@pytest.mark.parametrize("persist", ["0", "1"])
def test_both_launch_forms_match_oracle(W, monkeypatch, launch_form_case, persist):
    """One cluster per state and the persistent form (clusters looping over
    states) both match the oracle within the mixed tolerance."""
    monkeypatch.setenv("WSLDA_PERSIST", persist)
    monkeypatch.setenv("WSLDA_VARIANT", "0")
    case, (rho_r, nu_r) = launch_form_case
    ctx, box = gpu_context(case, 1)
    ctx.start(False, 0.01)
    ctx.step(0.01, 3)
    rho, nu = ctx.get_densities(box)
    ctx.close()
    assert rel(rho, rho_r) < TOL[1] and rel(nu, nu_r) < TOL[1]


@pytest.fixture(scope="module")
def mixed_variant_case():
    """16^3 with 300 states (compiled variants with clusters of 1 and of 2
    CTAs) and its oracle evolution."""
    case = _case((16, 16, 16), (1, 1, 1), 300, seed=11)
    sysm = oracle_system(case)
    st = o.start(sysm, _ref_states(case, 1), 0.01, False)
    st = o.evolve(sysm, st, 0.01, 6 - st.steps)
    rho_r, nu_r = o.densities(st.phi, case.wm, case.wp)
    return case, rho_r, nu_r, st.phi


@pytest.mark.parametrize("vx,vy", [(0, 2), (2, 0)])
def test_predictor_and_corrector_on_different_variants(W, monkeypatch, mixed_variant_case, vx, vy):
    """The autotuner may put the two stages on launch variants with different
    cluster sizes; the current term's <H>_n partials (one per CTA) must then
    come from a launch on the consuming stage's variant."""
    if max(vx, vy) >= W.lattice_variants(1, 16, 16, 16):
        pytest.skip("not enough compiled variants")
    monkeypatch.setenv("WSLDA_PERSIST", "0")
    monkeypatch.setenv("WSLDA_VARIANT", str(vx))
    monkeypatch.setenv("WSLDA_VARIANT_Y", str(vy))
    case, rho_r, nu_r, phi_r = mixed_variant_case
    ctx, box = gpu_context(case, 1)
    ctx.start(False, 0.01)
    ctx.step(0.01, 3)
    rho, nu = ctx.get_densities(box)
    phi = ctx.get_states(box)
    desc = ctx.get_variant(box)
    ctx.close()
    errs = dict(rho=rel(rho, rho_r), nu=rel(nu, nu_r), states=rel(phi, phi_r))
    print(desc, errs)
    assert all(v < TOL[1] for v in errs.values()), errs


def test_ab3am4_with_currents_matches_oracle(W):
    case = _case((12, 12, 12), (1, 1, 1), 400, seed=9)
    dt, nsteps = 0.01, 6
    ctx, box = gpu_context(case, 0, scheme="AB3AM4")
    ctx.start(False, dt)
    ctx.step(dt, nsteps - 2)
    rho, nu = ctx.get_densities(box)
    ctx.close()
    sysm = oracle_system(case)
    st = o.start_scheme(sysm, case.phi, dt, False, "AB3AM4")
    st = o.evolve_scheme(sysm, st, dt, nsteps - st.steps, "AB3AM4")
    rho_r, nu_r = o.densities(st.phi, case.wm, case.wp)
    assert rel(rho, rho_r) < TOL[0] and rel(nu, nu_r) < TOL[0]


def test_unsupported_combinations_fail_loudly(W):
    case = _case((12, 12, 12), (1, 1, 1), 100)
    ctx, box = gpu_context(case, 1)
    with pytest.raises(W.WsldaError):
        ctx.set_friction(box, 0.1, 0.0, 0.0)
    ctx.close()
