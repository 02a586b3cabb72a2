"""The elongated-trap workload's lattice (24 x 24 x 96, mixed precision) at
full size, every compiled launch variant, against the oracle on a sample of
48 states with a vortex imprinted on the pairing (reading P2)."""
import os

import numpy as np
import pytest

from cases import gpu_context, make_case, oracle_evolve, rel
from oracle import tdslda as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reference():
    c = make_case((24, 24, 96), nstates=48, kick=0.0, trap=0.0, seed=61, vortex=True)
    from paper_2602_08982_b300 import inputs
    c.vext = inputs.harmonic_trap(c.lat.shape, (0.064, 0.064, 0.016))
    ref_in = c.phi.astype(np.complex64).astype(np.complex128)
    _, st = oracle_evolve(c, 0.007, 6, False, phi0=ref_in)
    return c, st


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_every_variant_matches_oracle(reference, variant, monkeypatch):
    from paper_2602_08982_b300 import wslda as W
    c, st = reference
    monkeypatch.setenv("WSLDA_VARIANT", str(variant))
    monkeypatch.setenv("WSLDA_PERSIST", "0")
    ctx, box = gpu_context(c, W.MIXED)
    ctx.start(False, 0.007)
    ctx.step(0.007, 3)
    desc = ctx.get_variant(box)
    rho, nu = ctx.get_densities(box)
    ctx.close()
    r, n = o.densities(st.phi, c.wm, c.wp)
    assert rel(rho, r) < 1e-5 and rel(nu, n) < 1e-5, desc
