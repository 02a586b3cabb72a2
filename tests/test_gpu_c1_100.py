"""The uniform unitary gas on 16^3 (all 4096 states, seeded 1e-3 external
pairing kick) over 100 steps of dt = 0.01 against the stored oracle run
(tests/golden/c1_100steps.npz, written by tests/golden/make_c1_100steps.py,
which calls only the oracle).

Both paths start from the same double states (the mixed path rounds them to
complex float); the FP64 path must stay within 1e-12 of the oracle on rho, nu
and the energy after 20, 50 and 100 steps, the mixed path within 1e-5. The
energy drift |E(t) - E(0)| / |E(0)| of E_tot - mu N (conserved, Eq. E_tot)
is printed and bounded for both.
"""
import os

import numpy as np
import pytest

from cases import gpu_context, make_case, rel

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c1_100steps.npz")
TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def golden():
    return dict(np.load(GOLDEN))


@pytest.mark.parametrize("prec", [0, 1])
def test_c1_100_steps_against_oracle(golden, prec):
    g = golden
    c = make_case((16, 16, 16), kick=1e-3, seed=1)
    dt = float(g["dt"])
    mu = float(g["mu"])
    ctx, box = gpu_context(c, prec)
    e0 = ctx.get_energy(box)
    ctx.start(False, dt)
    errs = {}
    for mark in (20, 50, 100):
        _, steps = ctx.get_time()
        ctx.step(dt, mark - steps)
        rho, nu = ctx.get_densities(box)
        e = ctx.get_energy(box)
        errs[mark] = dict(rho=rel(rho, g[f"rho_{mark}"]), nu=rel(nu, g[f"nu_{mark}"]),
                          e_total=abs(e["e_total"] - g[f"e_total_{mark}"]) / abs(g[f"e_total_{mark}"]),
                          n_part=abs(e["n_part"] - g[f"n_part_{mark}"]) / abs(g[f"n_part_{mark}"]))
    econs0 = e0["e_total"] - mu * e0["n_part"]
    drift = abs((e["e_total"] - mu * e["n_part"]) - econs0) / abs(econs0)
    ref_drift = abs((g["e_total_100"] - mu * g["n_part_100"]) - (g["e0_total"] - mu * g["e0_n"])) / abs(
        g["e0_total"] - mu * g["e0_n"])
    ctx.close()
    print(f"precision {prec}: errors {errs}; energy drift after 100 steps {drift:.3e} (oracle {ref_drift:.3e})")
    for mark, d in errs.items():
        assert all(v < TOL[prec] for v in d.values()), (mark, d)
    assert drift < (1e-9 if prec == 0 else 1e-5), drift
