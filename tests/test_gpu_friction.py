"""Quantum friction (Sec. 5.2.4) on the GPU against the oracle's terms."""
import numpy as np
import pytest

from cases import gpu_context, make_case, oracle_system, rel
from oracle import tdslda as o

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def _case(shape=(8, 8, 8)):
    if shape == (8, 8, 8):
        return make_case(shape, kick=0.0, trap=0.12, seed=91)
    return make_case(shape, nstates=96, kick=0.0, trap=0.08, seed=92 + shape[0])


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 16, 16), (32, 32, 32)])
def test_friction_matches_oracle(prec, shape):
    """All three terms at once, after a Taylor start and five steps; 16^3 and
    32^3 run on the cluster launch variants (the x pass over distributed
    shared memory)."""
    c = _case(shape)
    n0 = c.lat.dV * np.sum(2.0 * o.densities(c.phi, c.wm, c.wp)[0])
    fr = o.Friction(alpha=5.0, beta=5.0, gamma=0.5, n_req=1.05 * n0)
    ctx, box = gpu_context(c, prec)
    ctx.set_friction(box, fr.alpha, fr.beta, fr.gamma, fr.rho0, fr.n_req)
    ctx.start(False, 0.01)
    ctx.step(0.01, 5)
    rho, nu = ctx.get_densities(box)
    desc = ctx.get_variant(box)
    ctx.close()
    ref_in = c.phi if prec == 0 else c.phi.astype(np.complex64).astype(np.complex128)
    sysm = oracle_system(c)
    sysm.friction = fr
    st = o.start(sysm, ref_in, 0.01, False)
    st = o.evolve(sysm, st, 0.01, 5)
    r, n = o.densities(st.phi, c.wm, c.wp)
    assert rel(rho, r) < TOL[prec] and rel(nu, n) < TOL[prec], (rel(rho, r), rel(nu, n), desc)


def test_zero_coefficients_are_the_conservative_step():
    c = _case()
    out = []
    for fric in (False, True):
        ctx, box = gpu_context(c, 0)
        if fric:
            ctx.set_friction(box, 0.0, 0.0, 0.0)
        ctx.start(False, 0.01)
        ctx.step(0.01, 4)
        out.append(ctx.get_states(box))
        ctx.close()
    assert np.array_equal(out[0], out[1])


def test_alpha_removes_energy_on_the_gpu():
    c = _case()
    drifts = []
    for alpha in (0.0, 5.0):
        ctx, box = gpu_context(c, 0)
        ctx.set_friction(box, alpha)
        ctx.start(False, 0.01)
        e0 = ctx.get_energy(box)
        ctx.step(0.01, 30)
        e1 = ctx.get_energy(box)
        ctx.close()
        drifts.append((e1["e_total"] - c.fn.mu * e1["n_part"]) - (e0["e_total"] - c.fn.mu * e0["n_part"]))
    assert abs(drifts[0]) < 1e-7 * abs(e0["e_total"]) + 1e-9
    assert drifts[1] < -1e-4
