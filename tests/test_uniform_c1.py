"""Uniform BCS states (Sec. 5.2.1, "inittype 0"): the library's seed solver
and its device fill against the oracle.

wslda_uniform_solve is host code of the library (number and gap equations
over the lattice k-set, Eq. Creg), so its comparison with the oracle's seeds
runs without a GPU; wslda_fill_uniform_states writes the plane-wave states on
the device and is compared element by element with the oracle's states.
"""
import numpy as np
import pytest

from cases import RHO_S, DELTA0, plane_waves, rel
from oracle import tdslda as o
from paper_2602_08982_b300 import inputs

SHAPES = [((12, 12, 12), (1.0, 1.0, 1.0)), ((16, 16, 16), (1.0, 1.0, 1.0)), ((24, 24, 96), (1.0, 1.0, 1.0)),
          ((32, 32, 32), (1.0, 1.0, 1.0)), ((8, 12, 16), (1.0, 0.9, 1.1))]
KEYS = ("mu_eff", "delta", "mu", "U", "C", "lam", "inv_g")


def _lib():
    from paper_2602_08982_b300 import wslda as W
    return W


@pytest.mark.parametrize("shape,spacing", SHAPES)
def test_uniform_slda_seed_matches_oracle(shape, spacing):
    W = _lib()
    lat = o.Lattice(*shape, *spacing)
    ref = o.uniform_slda_seed(lat, DELTA0, RHO_S)
    got = W.uniform_solve(shape, spacing, kind=W.SLDA_A1, B=o.B_SLDA, rho_sigma=RHO_S, delta0=DELTA0)
    for k in KEYS:
        assert got[k] == pytest.approx(getattr(ref, k), rel=1e-12, abs=1e-14), k


@pytest.mark.parametrize("shape,spacing", SHAPES)
@pytest.mark.parametrize("inv_kfa", [-0.5, 0.0, 0.6])
def test_uniform_bdg_seed_matches_oracle(shape, spacing, inv_kfa):
    W = _lib()
    lat = o.Lattice(*shape, *spacing)
    ia = inv_kfa / (4 * np.pi)
    ref = o.uniform_bdg_seed(lat, ia, RHO_S)
    got = W.uniform_solve(shape, spacing, kind=W.BDG, inv_4pi_a=ia, rho_sigma=RHO_S)
    for k in ("mu_eff", "delta", "mu", "U", "lam", "inv_g"):
        assert got[k] == pytest.approx(getattr(ref, k), rel=1e-12, abs=1e-14), k


def test_uniform_solve_rejects_bad_input():
    W = _lib()
    with pytest.raises(W.WsldaError):
        W.uniform_solve((8, 8, 8), kind=W.SLDA_A1, B=o.B_SLDA, rho_sigma=RHO_S, delta0=0.0)
    with pytest.raises(W.WsldaError):
        W.uniform_solve((8, 8, 8), kind=W.BDG, rho_sigma=-1.0)


def _filled(W, prec, shape, spacing, mu_eff, delta, kidx):
    ctx = W.Context(prec)
    n = shape[0] * shape[1] * shape[2] if kidx is None else len(kidx)
    box = ctx.add_box(shape, spacing, kind=W.BDG, inv_4pi_a=0.0, mu=mu_eff, nstates=n)
    ctx.fill_uniform_states(box, mu_eff, delta, kidx)
    phi = ctx.get_states(box)
    ctx.close()
    return phi


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,spacing,nsub", [((12, 12, 12), (1, 1, 1), None), ((8, 12, 16), (1.0, 0.9, 1.1), None),
                                                ((16, 16, 16), (1, 1, 1), 700), ((24, 24, 96), (1, 1, 1), 150),
                                                ((32, 32, 32), (1, 1, 1), 64)])
def test_fill_uniform_states_matches_oracle(prec, shape, spacing, nsub):
    """All states (kidx NULL) on small lattices, a seeded k subset elsewhere;
    FP64 within 1e-12 of the oracle's plane waves, the mixed path within the
    rounding of the oracle's values to complex float."""
    from paper_2602_08982_b300 import wslda as W
    if not W.lattice_supported(prec, *shape):
        pytest.skip("shape not compiled for this precision")
    lat = o.Lattice(*shape, *spacing)
    seed = o.uniform_slda_seed(lat, DELTA0, RHO_S)
    if nsub is None:
        kidx = None
        ref = o.uniform_states(lat, seed.mu_eff, seed.delta)
    else:
        kidx = np.sort(np.argsort(inputs.uniform01(300 + shape[2], lat.M))[:nsub]).astype(np.int64)
        ref = plane_waves(lat, seed.mu_eff, seed.delta, kidx)
    got = _filled(W, prec, shape, spacing, seed.mu_eff, seed.delta, kidx)
    if prec == 0:
        assert rel(got, ref) < 1e-12
    else:
        assert rel(got, ref.astype(np.complex64).astype(np.complex128)) < 2e-7


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_imprint_phase_matches_host_imprint(prec):
    """The vortex start imprinted in the library (u e^{i theta/2}, v e^{-i theta/2},
    reading P2) equals the same factors applied to the oracle's states."""
    from paper_2602_08982_b300 import wslda as W
    shape = (12, 12, 48)
    lat = o.Lattice(*shape)
    seed = o.uniform_slda_seed(lat, DELTA0, RHO_S)
    kidx = np.sort(np.argsort(inputs.uniform01(404, lat.M))[:120]).astype(np.int64)
    ph = inputs.vortex_phase(shape, winding=0.5)
    ref = plane_waves(lat, seed.mu_eff, seed.delta, kidx)
    ref[:, 0, :] *= ph[None, :]
    ref[:, 1, :] *= np.conj(ph)[None, :]
    ctx = W.Context(prec)
    box = ctx.add_box(shape, kind=W.SLDA_A1, B=o.B_SLDA, C=seed.C, mu=seed.mu, nstates=len(kidx))
    ctx.fill_uniform_states(box, seed.mu_eff, seed.delta, kidx)
    ctx.imprint_phase(box, 0, ph)
    ctx.imprint_phase(box, 1, np.conj(ph))
    got = ctx.get_states(box)
    ctx.close()
    assert rel(got, ref) < (1e-12 if prec == 0 else 3e-7)
