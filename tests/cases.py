"""Seeded test cases shared by the GPU parity tests.

Inputs come from the oracle's uniform-state construction (test
infrastructure) and the seeded generators of paper_2602_08982_b300.inputs;
the CUDA path receives them through the C ABI, and the oracle evolves the
same inputs on the CPU.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from oracle import tdslda as o
from paper_2602_08982_b300 import inputs

RHO_S = 1.0 / (6 * np.pi ** 2)   # per-spin density at kF = 1
DELTA0 = 0.25                     # 0.5 eF at kF = 1


@dataclass
class Case:
    lat: o.Lattice
    fn: o.Functional
    phi: np.ndarray
    vext: np.ndarray
    dext: np.ndarray | None
    wm: np.ndarray
    wp: np.ndarray
    delta0: float


def plane_waves(lat: o.Lattice, mu_eff: float, delta: float, idx: np.ndarray) -> np.ndarray:
    """Positive-energy uniform BCS states for the flattened k indices `idx`."""
    kx, ky, kz = (lat.kaxis(a) for a in range(3))
    ix, rem = np.divmod(idx, lat.ny * lat.nz)
    iy, iz = np.divmod(rem, lat.nz)
    x = np.arange(lat.nx) * lat.dx
    y = np.arange(lat.ny) * lat.dy
    z = np.arange(lat.nz) * lat.dz
    ex = np.exp(1j * np.outer(kx[ix], x))
    ey = np.exp(1j * np.outer(ky[iy], y))
    ez = np.exp(1j * np.outer(kz[iz], z))
    pw = np.einsum("ni,nj,nk->nijk", ex, ey, ez).reshape(len(idx), lat.M) / np.sqrt(lat.volume)
    k2 = kx[ix] ** 2 + ky[iy] ** 2 + kz[iz] ** 2
    Uk, Vk, _ = o.bcs_amplitudes(0.5 * k2 - mu_eff, delta)
    return np.stack([Uk[:, None] * pw, Vk[:, None] * pw], axis=1)


def make_case(shape, spacing=(1.0, 1.0, 1.0), kind="slda", nstates=None, trap=0.0, kick=0.0, seed=1,
              inv_kfa=-0.5, thermal=False, vortex=False, A=1.0) -> Case:
    """A != 1 (kind slda) switches on the current terms; the uniform A = 1
    seed then only supplies a start with the right density and gap scale."""
    lat = o.Lattice(*shape, *spacing)
    if kind == "slda":
        s = o.uniform_slda_seed(lat, DELTA0, RHO_S)
        fn = o.Functional("slda", B=o.B_SLDA, C=s.C, mu=s.mu, A=float(A))
    else:
        ia = inv_kfa / (4 * np.pi)
        s = o.uniform_bdg_seed(lat, ia, RHO_S)
        fn = o.Functional("bdg", inv_4pi_a=ia, mu=s.mu)
    if nstates is None or nstates >= lat.M:
        idx = np.arange(lat.M)
    else:
        r = inputs.uniform01(seed + 1000, lat.M)
        idx = np.sort(np.argsort(r)[:nstates])
    phi = plane_waves(lat, s.mu_eff, s.delta, idx)
    if vortex:  # reading P2: u e^{i theta/2}, v e^{-i theta/2}, so nu winds once
        half = inputs.vortex_phase(lat.shape, (lat.dx, lat.dy, lat.dz), 0.5)
        phi[:, 0, :] *= half[None, :]
        phi[:, 1, :] *= np.conj(half)[None, :]
    vext = inputs.harmonic_trap(lat.shape, trap, (lat.dx, lat.dy, lat.dz)) if trap else np.zeros(lat.M)
    dext = inputs.pairing_kick(lat.shape, seed, kick * s.delta) if kick else None
    n = len(idx)
    if thermal:
        r = inputs.uniform01(seed + 2000, n)
        wm = 1.0 - 0.2 * r
        wp = 0.2 * r
    else:
        wm, wp = np.ones(n), np.zeros(n)
    return Case(lat=lat, fn=fn, phi=phi, vext=vext, dext=dext, wm=wm, wp=wp, delta0=s.delta)


def oracle_system(c: Case) -> o.TDSystem:
    return o.TDSystem(c.lat, c.fn, vext=c.vext, dext=c.dext, w_minus=c.wm, w_plus=c.wp)


def oracle_evolve(c: Case, dt: float, nsteps: int, stationary: bool, phi0=None):
    sysm = oracle_system(c)
    st = o.start(sysm, c.phi if phi0 is None else phi0, dt, stationary)
    st = o.evolve(sysm, st, dt, nsteps - st.steps)
    return sysm, st


def gpu_context(c: Case, precision: int, scheme: str | None = None):
    from paper_2602_08982_b300 import wslda as W
    ctx = W.Context(precision)
    if scheme is not None:
        ctx.set_integrator(scheme)
    kind = (W.SLDA if c.fn.currents else W.SLDA_A1) if c.fn.kind == "slda" else W.BDG
    box = ctx.add_box(c.lat.shape, (c.lat.dx, c.lat.dy, c.lat.dz), kind=kind, B=c.fn.B, C=c.fn.C,
                      inv_4pi_a=c.fn.inv_4pi_a, mu=c.fn.mu, A=c.fn.A, nstates=c.phi.shape[0])
    ctx.set_vext(box, c.vext)
    if c.dext is not None:
        ctx.set_dext(box, c.dext)
    ctx.load_states(box, c.phi, c.wm, c.wp)
    return ctx, box


def rel(a, b) -> float:
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    return float(d / max(np.abs(np.asarray(b)).max(), 1e-300))
