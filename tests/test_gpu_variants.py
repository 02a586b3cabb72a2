"""Every compiled launch variant (cluster size, threads, register budget) of
the lattices the workloads use (mixed precision, and FP64 at 32^3), in both
launch forms, forced one at a time, against the oracle on a sample of states
(Taylor start and two ABM steps)."""
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
    for prec, shapes in ((W.MIXED, SHAPES), (W.FP64, [(32, 32, 32)])):
        for s in shapes:
            for v in range(W.lattice_variants(prec, *s)):
                for p in (0, 1):
                    out.append((prec, s, v, p))
    return out


@functools.lru_cache(maxsize=None)
def _reference64(shape):
    c = make_case(shape, nstates=40, kick=0.05, trap=0.06, seed=81 + shape[0])
    _, st = oracle_evolve(c, 0.01, 5, False)
    return c, o.densities(st.phi, c.wm, c.wp)


@pytest.mark.parametrize("prec,shape,variant,persist", _cases())
def test_variant_matches_oracle(prec, shape, variant, persist, monkeypatch):
    from paper_2602_08982_b300 import wslda as W
    c, (r, n) = _reference(shape) if prec == W.MIXED else _reference64(shape)
    tol = 1e-5 if prec == W.MIXED else 1e-12
    monkeypatch.setenv("WSLDA_VARIANT", str(variant))
    monkeypatch.setenv("WSLDA_PERSIST", str(persist))
    ctx, box = gpu_context(c, prec)
    ctx.start(False, 0.01)
    ctx.step(0.01, 2)
    desc = ctx.get_variant(box)
    rho, nu = ctx.get_densities(box)
    ctx.close()
    assert rel(rho, r) < tol and rel(nu, n) < tol, desc


SCHEME_SHAPES = [(24, 24, 96), (32, 32, 32)]


@functools.lru_cache(maxsize=None)
def _scheme_reference(shape, scheme, prec):
    c = make_case(shape, nstates=24, kick=0.05, trap=0.06, seed=181 + shape[0], vortex=shape[2] == 96)
    ref_in = c.phi if prec == 0 else c.phi.astype(np.complex64).astype(np.complex128)
    from cases import oracle_system
    sysm = oracle_system(c)
    st = o.start_scheme(sysm, ref_in, 0.01, False, scheme)
    st = o.evolve_scheme(sysm, st, 0.01, 2, scheme)
    return c, o.densities(st.phi, c.wm, c.wp)


def _scheme_cases():
    from paper_2602_08982_b300 import wslda as W
    out = []
    for prec in (W.MIXED, W.FP64):
        for s in SCHEME_SHAPES:
            for v in range(W.lattice_variants(prec, *s)):
                for scheme in ("AB3AM4", "AB5AM5"):
                    for p in (0, 1):
                        out.append((prec, s, v, scheme, p))
    return out


@pytest.mark.parametrize("prec,shape,variant,scheme,persist", _scheme_cases())
def test_scheme_variant_matches_oracle(prec, shape, variant, scheme, persist, monkeypatch):
    """AB3AM4 / AB5AM5 predictor stages (two and four history reads) on every
    cluster variant of the large lattices, Taylor start and two steps."""
    from paper_2602_08982_b300 import wslda as W
    c, (r, n) = _scheme_reference(shape, scheme, prec)
    tol = 1e-5 if prec == W.MIXED else 1e-12
    monkeypatch.setenv("WSLDA_VARIANT", str(variant))
    monkeypatch.setenv("WSLDA_PERSIST", str(persist))
    ctx, box = gpu_context(c, prec, scheme)
    ctx.start(False, 0.01)
    ctx.step(0.01, 2)
    desc = ctx.get_variant(box)
    rho, nu = ctx.get_densities(box)
    ctx.close()
    assert rel(rho, r) < tol and rel(nu, n) < tol, desc


def test_corrector_variant_keeps_the_kinetic_table_layout(monkeypatch):
    """The kinetic tables of a box are ordered for the lanes per pencil of its
    launch variant (a pencil split over T lanes leaves its frequencies in a
    T-dependent order). A corrector variant with another split (here FP64
    32^3 with pencils over 2 lanes for the predictor, 4 for the requested
    corrector) must not be taken: the corrector stays on the predictor's
    layout and the step still matches the oracle."""
    from paper_2602_08982_b300 import wslda as W
    variants = W.lattice_variants(W.FP64, 32, 32, 32)
    assert variants >= 3
    c, (r, n) = _reference64((32, 32, 32))
    monkeypatch.setenv("WSLDA_VARIANT", "0")
    monkeypatch.setenv("WSLDA_VARIANT_Y", "2")
    monkeypatch.setenv("WSLDA_PERSIST", "0")
    ctx, box = gpu_context(c, W.FP64)
    ctx.start(False, 0.01)
    ctx.step(0.01, 2)
    desc = ctx.get_variant(box)
    rho, nu = ctx.get_densities(box)
    ctx.close()
    x_part, y_part = desc.split("; stage Y:")
    lanes = lambda d: d.split("lanes_per_pencil=")[1].split()[0]
    assert lanes(x_part) == lanes(y_part) == "2,2,2", desc
    assert rel(rho, r) < 1e-12 and rel(nu, n) < 1e-12, desc
