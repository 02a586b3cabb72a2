"""Pins of the dissipative ("quantum friction") terms of the oracle
(Sec. 5.2.4, Eqs. cooling_alpha, Deltadiss2)."""
import numpy as np
import pytest

from oracle import tdslda as o
from paper_2602_08982_b300 import inputs

RHO_S = 1.0 / (6 * np.pi ** 2)


def _case():
    lat = o.Lattice(4, 4, 4)
    seed = o.uniform_slda_seed(lat, 0.25, RHO_S)
    fn = o.Functional("slda", B=o.B_SLDA, C=seed.C, mu=seed.mu)
    phi0 = o.uniform_states(lat, seed.mu_eff, seed.delta)
    return lat, fn, phi0, inputs.harmonic_trap(lat.shape, 0.3)


def _history(friction, nsamples=10, every=4, dt=0.01):
    lat, fn, phi0, vext = _case()
    sysm = o.TDSystem(lat, fn, vext=vext, friction=friction)
    st = o.start(sysm, phi0, dt, stationary=False)
    out = []
    for _ in range(nsamples):
        e = sysm.energy(st.phi)
        out.append((e["e_total"] - fn.mu * e["n_part"], e["n_part"]))
        st = o.evolve(sysm, st, dt, every)
    return np.array(out)


def test_uniform_state_feels_no_friction():
    """A uniform BCS state carries no current and its anomalous kinetic
    density is in phase with nu: every dissipative field vanishes."""
    lat, fn, phi0, _ = _case()
    sysm = o.TDSystem(lat, fn, vext=np.zeros(lat.M))
    sysm.init_regulator(phi0)
    wm, wp = np.ones(lat.M), np.zeros(lat.M)
    rho, nu, U, delta, _ = sysm.potentials(phi0)
    dU, dD = o.Friction(alpha=5, beta=5).fields(phi0, wm, wp, rho, nu, delta, lat)
    assert np.abs(dU).max() < 1e-14 and np.abs(dD).max() < 1e-14


def test_zero_coefficients_leave_the_dynamics_unchanged():
    a = _history(None, 3)
    b = _history(o.Friction(), 3)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("friction", [o.Friction(alpha=5.0), o.Friction(beta=5.0)])
def test_friction_removes_energy_and_keeps_n(friction):
    """Without friction the trap quench conserves E - mu N (to 1e-7 over the
    run); with alpha or beta it falls at every sample and N stays put."""
    ref = _history(None)
    assert np.abs(ref[:, 0] - ref[0, 0]).max() < 1e-7
    h = _history(friction)
    assert np.all(np.diff(h[:, 0]) < 0)
    assert h[-1, 0] < ref[-1, 0] - 3e-4
    assert np.abs(h[:, 1] - h[0, 1]).max() < 1e-8


def test_gamma_drives_n_toward_the_request():
    lat, fn, phi0, _ = _case()
    n_req = 1.1 * lat.dV * 2 * RHO_S * lat.M
    h = _history(o.Friction(gamma=0.5, n_req=n_req))
    gap = np.abs(h[:, 1] - n_req)
    assert np.all(np.diff(gap) < 0)
