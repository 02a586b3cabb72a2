"""Several boxes of different shapes in one context, advanced together.

With batched execution on, every box of a step runs on its own forked stream
and four steps replay as one captured CUDA graph. Each box must match its own
oracle evolution, and the graph path must reproduce direct launches bit for bit.
"""
import numpy as np
import pytest

from cases import make_case, oracle_evolve, rel
from oracle import tdslda as o

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def _boxes():
    return [make_case((8, 8, 8), kind="bdg", inv_kfa=-0.6, kick=0.05, trap=0.1, seed=31),
            make_case((12, 12, 12), nstates=500, kick=0.05, trap=0.08, seed=32),
            make_case((8, 12, 16), (1.0, 0.9, 1.1), nstates=257, kick=0.03, seed=33, thermal=True)]


def _run(W, prec, cases, graph, dt, nsteps):
    ctx = W.Context(prec)
    ids = []
    for c in cases:
        kind = W.SLDA_A1 if c.fn.kind == "slda" else W.BDG
        b = ctx.add_box(c.lat.shape, (c.lat.dx, c.lat.dy, c.lat.dz), kind=kind, B=c.fn.B, C=c.fn.C,
                        inv_4pi_a=c.fn.inv_4pi_a, mu=c.fn.mu, nstates=c.phi.shape[0])
        ctx.set_vext(b, c.vext)
        if c.dext is not None:
            ctx.set_dext(b, c.dext)
        ctx.load_states(b, c.phi, c.wm, c.wp)
        ids.append(b)
    if graph:
        ctx.set_graph(True, 3)
    ctx.start(False, dt)
    ctx.step(dt, nsteps - 3)
    out = [(ctx.get_densities(b), ctx.get_states(b)) for b in ids]
    ctx.close()
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_boxes_match_oracle_and_direct_launches(prec):
    from paper_2602_08982_b300 import wslda as W
    cases = _boxes()
    dt, nsteps = 0.01, 11   # 3 Taylor steps, two 4-step graphs and nothing left over
    g = _run(W, prec, cases, True, dt, nsteps)
    d = _run(W, prec, cases, False, dt, nsteps)
    for (gd, gs), (dd, ds) in zip(g, d):
        assert np.array_equal(gs, ds)
        assert np.array_equal(gd[0], dd[0]) and np.array_equal(gd[1], dd[1])
    for c, ((rho, nu), _) in zip(cases, g):
        ref_in = c.phi if prec == 0 else c.phi.astype(np.complex64).astype(np.complex128)
        sysm, st = oracle_evolve(c, dt, nsteps, False, phi0=ref_in)
        r, n = o.densities(st.phi, c.wm, c.wp)
        assert rel(rho, r) < TOL[prec] and rel(nu, n) < TOL[prec]
