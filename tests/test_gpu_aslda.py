"""Spin-imbalanced ASLDA (Secs. 2.3-2.4) on the GPU against oracle/aslda.py.

States: a spin-symmetric case with A = A_a(0) (trap, vortex phase, thermal
weights) plus the partner of every state, [v^*, -u^*], so that the set spans
both signs of E_n as in Eq. HpsiEpsi; the weights of the v rows are then
scaled down state by state (rho_b < rho_a, p != 0 and varying in space) and mu_a != mu_b, so that the
p-dependent A_a(p), A_b(p), B(p), the per-species currents and the varying
alpha of Eq. kinop-alpha all enter. FP64 within 1e-12 of the oracle, the mixed
path within 1e-5.
"""
import functools

import numpy as np
import pytest

from cases import make_case, rel
from oracle import aslda as a
from oracle import tdslda as o
from paper_2602_08982_b300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def _case(shape, spacing, n, seed):
    c = make_case(shape, spacing, nstates=n, trap=0.08, seed=seed, thermal=True, vortex=True, A=o.aslda_A(0.0))
    # smooth envelopes with seeded phases (different for u and v of each
    # state) make the densities, and so p, vary in space from the start
    x = [np.arange(N) * d for N, d in zip(c.lat.shape, (c.lat.dx, c.lat.dy, c.lat.dz))]
    X, Y, Z = (g.reshape(-1) for g in np.meshgrid(*x, indexing="ij"))
    th = 2 * np.pi * inputs.uniform01(seed + 5, 2 * n).reshape(2, n, 1)
    Lx, Lz = c.lat.nx * c.lat.dx, c.lat.nz * c.lat.dz
    env_u = 1.0 + 0.3 * np.cos(2 * np.pi * X[None, :] / Lx + th[0])
    env_v = 1.0 + 0.3 * np.cos(2 * np.pi * Z[None, :] / Lz + th[1])
    c.phi = o.normalize(np.stack([c.phi[:, 0] * env_u, c.phi[:, 1] * env_v], axis=1), c.lat)
    u, v = c.phi[:, 0], c.phi[:, 1]
    phi = np.concatenate([c.phi, np.stack([np.conj(v), -np.conj(u)], axis=1)])
    fp = np.concatenate([c.wp, c.wm])
    # state-dependent reduction of the v weights: rho_b < rho_a with a ratio
    # that varies from site to site, so alpha_a, alpha_b vary in space
    fm = np.concatenate([c.wm, c.wp]) * (0.2 + 0.3 * inputs.uniform01(seed + 7, 2 * n))
    fn = a.ASLDA(mu_a=c.fn.mu + 0.02, mu_b=c.fn.mu - 0.03, C=c.fn.C)
    sysm = a.ImbalancedSystem(c.lat, fn, c.vext, c.vext, fp, fm)
    return c, phi, fp, fm, fn, sysm


def _gpu(W, c, phi, fp, fm, fn, prec):
    ctx = W.Context(prec)
    box = ctx.add_box(c.lat.shape, (c.lat.dx, c.lat.dy, c.lat.dz), kind=W.ASLDA, C=fn.C, mu=fn.mu_a, mu_b=fn.mu_b,
                      nstates=phi.shape[0])
    ctx.set_vext(box, c.vext)
    ctx.load_states(box, phi, fm, fp)
    return ctx, box


SHAPES = [((8, 12, 16), (1.0, 0.9, 1.1), 60), ((32, 32, 32), (1.0, 1.0, 1.0), 16)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,spacing,n", SHAPES)
def test_aslda_fields_and_f_match_oracle(prec, shape, spacing, n):
    """Densities of both species, V_a, V_b, Delta and f(phi) = -i [H - <H>_n] phi
    of the loaded states (regulator frozen at these states)."""
    from paper_2602_08982_b300 import wslda as W
    c, phi, fp, fm, fn, sysm = _case(shape, spacing, n, 51)
    ctx, box = _gpu(W, c, phi, fp, fm, fn, prec)
    d = ctx.get_spin_densities(box)
    Va, Vb, D = ctx.get_spin_fields(box)
    f = ctx.eval_f(box)
    ctx.close()
    ref_in = phi if prec == 0 else phi.astype(np.complex64).astype(np.complex128)
    sysm.init_regulator(ref_in)
    dr = a.densities(ref_in, fp, fm, c.lat)
    P = a.potentials(dr, sysm.lam, fn)
    rho_t = dr.rho_a + dr.rho_b
    p = (dr.rho_a - dr.rho_b) / rho_t
    assert p.min() > 0.02 and np.ptp(p) > 0.02  # polarised everywhere, varying in space
    tol = TOL[prec]
    assert rel(d["rho_a"], dr.rho_a) < tol and rel(d["rho_b"], dr.rho_b) < tol and rel(d["nu"], dr.nu) < tol
    assert rel(d["tau_a"], dr.tau_a) < tol and rel(d["tau_b"], dr.tau_b) < tol
    assert rel(d["j_a"], dr.j_a) < 10 * tol and rel(d["j_b"], dr.j_b) < 10 * tol
    assert rel(Va, P.V_a) < tol and rel(Vb, P.V_b) < tol and rel(D, P.Delta) < tol
    f_ref = sysm.f(ref_in)
    scale = np.abs(a.apply_H(ref_in, sysm.fields(ref_in), c.lat)).max()
    assert np.abs(f - f_ref).max() / scale < 10 * tol


@functools.lru_cache(maxsize=None)
def _reference(shape, spacing, n, stationary, dt, nsteps):
    """Oracle evolution from the double states (the mixed path is held to its
    1e-5 against it, its own rounding of the start included)."""
    c, phi, fp, fm, fn, sysm = _case(shape, spacing, n, 53)
    st = a.start(sysm, phi, dt, stationary)
    st = a.evolve(sysm, st, dt, nsteps - st.steps)
    return st.phi, a.densities(st.phi, fp, fm, c.lat), sysm.energy(st.phi)


EVOLVE = [(SHAPES[0], False), (SHAPES[0], True), (SHAPES[1], False)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case,stationary", EVOLVE)
def test_aslda_evolution_matches_oracle(prec, case, stationary):
    """Taylor (or stationary) start and AB4AM5 steps (Alg. 2): states,
    per-species densities and the energy."""
    from paper_2602_08982_b300 import wslda as W
    shape, spacing, n = case
    c, phi, fp, fm, fn, sysm = _case(shape, spacing, n, 53)
    dt, nsteps = 0.01, 7
    ctx, box = _gpu(W, c, phi, fp, fm, fn, prec)
    ctx.start(stationary, dt)
    _, s0 = ctx.get_time()
    ctx.step(dt, nsteps - s0)
    d = ctx.get_spin_densities(box)
    e = ctx.get_energy(box)
    got = ctx.get_states(box)
    de, dn = ctx.check_conservation(box, 1.0, 1.0)
    ctx.close()
    ref, dr, er = _reference(shape, spacing, n, stationary, dt, nsteps)
    tol = TOL[prec]
    errs = dict(rho_a=rel(d["rho_a"], dr.rho_a), rho_b=rel(d["rho_b"], dr.rho_b), nu=rel(d["nu"], dr.nu),
                j_a=rel(d["j_a"], dr.j_a), states=rel(got, ref),
                e_total=abs(e["e_total"] - er["e_total"]) / abs(er["e_total"]))
    bad = {k: v for k, v in errs.items() if not v < (10 * tol if k == "j_a" else tol)}
    assert not bad, errs
    # the states moved: not a comparison of unchanged inputs
    assert rel(ref, o.normalize(phi, c.lat)) > 1e-4
    assert de < 1e-3 and dn < 1e-3


def test_aslda_rejects_static_solve_and_friction():
    from paper_2602_08982_b300 import wslda as W
    c, phi, fp, fm, fn, sysm = _case((8, 8, 8), (1.0, 1.0, 1.0), 20, 55)
    ctx, box = _gpu(W, c, phi, fp, fm, fn, 0)
    with pytest.raises(W.WsldaError) as e:
        ctx.set_friction(box, 1.0)
    assert e.value.status == 8
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_aslda_uniform_fill_is_states_and_partners(prec):
    """fill_uniform_states on an ASLDA box: n/2 plane-wave states, then their
    partners [v^*, -u^*], with the T = 0 weights of both signs of E (the
    densities then equal those of the spin-symmetric states: p = 0)."""
    from cases import plane_waves
    from paper_2602_08982_b300 import wslda as W
    lat = o.Lattice(12, 12, 12)
    seed = o.uniform_slda_seed(lat, 0.25, 1.0 / (6 * np.pi ** 2))
    h = 150
    kidx = np.sort(np.argsort(inputs.uniform01(606, lat.M))[:h]).astype(np.int64)
    pw = plane_waves(lat, seed.mu_eff, seed.delta, kidx)
    ref = np.concatenate([pw, np.stack([np.conj(pw[:, 1]), -np.conj(pw[:, 0])], axis=1)])
    ctx = W.Context(prec)
    box = ctx.add_box(lat.shape, kind=W.ASLDA, C=-11.11, mu=seed.mu, mu_b=seed.mu, nstates=2 * h)
    ctx.fill_uniform_states(box, seed.mu_eff, seed.delta, kidx)
    got = ctx.get_states(box)
    d = ctx.get_spin_densities(box)
    ctx.close()
    assert rel(got, ref) < (1e-12 if prec == 0 else 2e-7)
    fp = np.concatenate([np.zeros(h), np.ones(h)])
    fm = np.concatenate([np.ones(h), np.zeros(h)])
    dr = a.densities(ref, fp, fm, lat)
    tol = TOL[prec]
    assert rel(d["rho_a"], dr.rho_a) < tol and rel(d["rho_b"], dr.rho_b) < tol and rel(d["nu"], dr.nu) < tol
    assert rel(dr.rho_a, dr.rho_b) < 1e-13
