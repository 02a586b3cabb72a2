"""Writes tests/golden/c1_100steps.npz: the CPU oracle's result for the plain
uniform unitary gas on a 16^3 lattice (all 4096 states, seeded 1e-3 external
pairing kick, SLDA with A = 1), Taylor start (Sec. 3.3) and AB4AM5 steps
(Alg. 2) of dt = 0.01 up to 100 steps in total.

Stored: rho_sigma and nu at steps 20, 50 and 100, the energy terms at the
start and at those steps. Only oracle/ computes anything here (the inputs
come from the seeded generators through tests/cases.py). Run from the
repository root:  python tests/golden/make_c1_100steps.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

from cases import make_case, oracle_system  # noqa: E402
from oracle import tdslda as o  # noqa: E402

DT = 0.01
MARKS = (20, 50, 100)


def main():
    c = make_case((16, 16, 16), kick=1e-3, seed=1)
    sysm = oracle_system(c)
    sysm.init_regulator(c.phi)
    e0 = sysm.energy(c.phi)
    st = o.start(sysm, c.phi, DT, False)
    out = {"dt": DT, "e0_total": e0["e_total"], "e0_n": e0["n_part"], "mu": c.fn.mu}
    t0 = time.time()
    for mark in MARKS:
        st = o.evolve(sysm, st, DT, mark - st.steps)
        rho, nu = o.densities(st.phi, c.wm, c.wp)
        e = sysm.energy(st.phi)
        out[f"rho_{mark}"] = rho
        out[f"nu_{mark}"] = nu
        out[f"e_total_{mark}"] = e["e_total"]
        out[f"e_kin_{mark}"] = e["e_kin"]
        out[f"n_part_{mark}"] = e["n_part"]
        print(f"step {mark}: {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(os.path.join(HERE, "c1_100steps.npz"), **out)


if __name__ == "__main__":
    main()
