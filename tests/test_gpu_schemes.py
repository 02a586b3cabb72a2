"""AB3AM4 and AB5AM5 (Sec. 3.3) on the GPU against the oracle's schemes.

Same fused stages as AB4AM5 with four or six state buffers; the start-up takes
two or four Taylor steps.
"""
import numpy as np
import pytest

from cases import gpu_context, make_case, oracle_system, rel
from oracle import tdslda as o

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def _case(shape):
    if shape == (8, 8, 8):
        return make_case(shape, kick=0.05, trap=0.1, seed=41)
    return make_case(shape, (1.0, 0.9, 1.1), nstates=300, kick=0.03, trap=0.08, seed=42, thermal=True)


@pytest.mark.parametrize("scheme", ["AB3AM4", "AB5AM5"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(8, 8, 8), (8, 12, 16)])
@pytest.mark.parametrize("stationary", [False, True])
def test_scheme_matches_oracle(scheme, prec, shape, stationary):
    c = _case(shape)
    dt, nsteps = 0.01, 9
    ctx, box = gpu_context(c, prec, scheme)
    ctx.start(stationary, dt)
    p = len(o.SCHEMES[scheme][0])
    ctx.step(dt, nsteps - (0 if stationary else p - 1))
    rho, nu = ctx.get_densities(box)
    phi = ctx.get_states(box)
    t, steps = ctx.get_time()
    ctx.close()
    ref_in = c.phi if prec == 0 else c.phi.astype(np.complex64).astype(np.complex128)
    sysm = oracle_system(c)
    st = o.start_scheme(sysm, ref_in, dt, stationary, scheme)
    st = o.evolve_scheme(sysm, st, dt, nsteps - st.steps, scheme)
    assert steps == nsteps and abs(t - nsteps * dt) < 1e-12
    r, n = o.densities(st.phi, c.wm, c.wp)
    assert rel(rho, r) < TOL[prec] and rel(nu, n) < TOL[prec]
    if prec == 0:
        assert rel(phi, st.phi) < 1e-12


@pytest.mark.parametrize("scheme", ["AB3AM4", "AB5AM5"])
def test_scheme_graph_replay_is_bitwise_direct(scheme):
    """Four-step graphs cycle through the slot phases of a three- or
    five-slot history rotation."""
    from paper_2602_08982_b300 import wslda as W
    cases = [make_case((8, 8, 8), kick=0.05, trap=0.1, seed=43),
             make_case((12, 12, 12), nstates=200, kick=0.05, seed=44)]

    def run(graph):
        ctx = W.Context(W.MIXED)
        ctx.set_integrator(scheme)
        ids = []
        for c in cases:
            b = ctx.add_box(c.lat.shape, kind=W.SLDA_A1, B=c.fn.B, C=c.fn.C, mu=c.fn.mu, nstates=c.phi.shape[0])
            ctx.set_vext(b, c.vext)
            ctx.set_dext(b, c.dext)
            ctx.load_states(b, c.phi)
            ids.append(b)
        if graph:
            ctx.set_graph(True, 2)
        ctx.start(True, 0.01)
        ctx.step(0.01, 13)
        out = [ctx.get_states(b) for b in ids]
        ctx.close()
        return out

    for g, d in zip(run(True), run(False)):
        assert np.array_equal(g, d)


def test_ab5am5_save_load_resume_is_bit_identical(tmp_path):
    c = _case((8, 8, 8))
    a, box = gpu_context(c, 0, "AB5AM5")
    a.start(False, 0.01)
    a.step(0.01, 2)
    path = str(tmp_path / "ck5.bin")
    a.save(path)
    a.step(0.01, 3)
    ref = a.get_states(box)
    a.close()
    b, box = gpu_context(c, 0, "AB5AM5")
    b.load(path)
    b.step(0.01, 3)
    got = b.get_states(box)
    b.close()
    assert np.array_equal(ref, got)


def test_integrator_is_fixed_before_boxes():
    from paper_2602_08982_b300 import wslda as W
    c = _case((8, 8, 8))
    ctx, box = gpu_context(c, 0)
    with pytest.raises(W.WsldaError) as e:
        ctx.set_integrator("AB3AM4")
    assert e.value.status == 7
    ctx.close()
    ctx = W.Context(W.FP64)
    with pytest.raises(KeyError):
        ctx.set_integrator("RK4")
    ctx.close()
