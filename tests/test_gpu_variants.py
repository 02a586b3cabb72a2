"""Every compiled launch variant (cluster size, threads, register budget) of
the mixed-precision lattices the workloads use, forced one at a time, against
the oracle on a sample of states (Taylor start and two ABM steps)."""
import functools

import numpy as np
import pytest

from cases import gpu_context, make_case, oracle_evolve, rel
from oracle import tdslda as o

pytestmark = pytest.mark.gpu

SHAPES = [(12, 12, 12), (16, 16, 16), (18, 18, 18), (20, 20, 20), (24, 24, 24), (32, 32, 32)]


@functools.lru_cache(maxsize=None)
def _reference(shape):
    c = make_case(shape, nstates=40, kick=0.05, trap=0.06, seed=81 + shape[0])
    ref_in = c.phi.astype(np.complex64).astype(np.complex128)
    _, st = oracle_evolve(c, 0.01, 5, False, phi0=ref_in)
    return c, o.densities(st.phi, c.wm, c.wp)


def _cases():
    from paper_2602_08982_b300 import wslda as W
    out = []
    for s in SHAPES:
        for v in range(W.lattice_variants(W.MIXED, *s)):
            for p in (0, 1):
                out.append((s, v, p))
    return out


@pytest.mark.parametrize("shape,variant,persist", _cases())
def test_variant_matches_oracle(shape, variant, persist, monkeypatch):
    from paper_2602_08982_b300 import wslda as W
    c, (r, n) = _reference(shape)
    monkeypatch.setenv("WSLDA_VARIANT", str(variant))
    monkeypatch.setenv("WSLDA_PERSIST", str(persist))
    ctx, box = gpu_context(c, W.MIXED)
    ctx.start(False, 0.01)
    ctx.step(0.01, 2)
    desc = ctx.get_variant(box)
    rho, nu = ctx.get_densities(box)
    ctx.close()
    assert rel(rho, r) < 1e-5 and rel(nu, n) < 1e-5, desc
