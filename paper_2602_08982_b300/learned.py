"""Learned starting fields for the static self-consistent solver (Alg. 1).

Workflow around the wslda_net_* kernels and wslda_static_solve:
  * dataset(): seeded anisotropic harmonic traps on a periodic lattice, each
    solved to self-consistency (BdG functional, 1/(kF a) drawn per trap, mu
    of the uniform system at that coupling), giving input channels
    (V_ext / eF, 1/(kF a)) and target channels (U / eF, Delta / eF);
  * train(): Adam on the mean squared error, mini-batches in a seeded order;
  * predict(): the network's fields, averaged over the lattice reflections so
    that they have the symmetry the solver requires;
  * iterations(): self-consistent iterations from a given start, with the
    plain linear mixing that serves as the fallback and judge;
  * converged_td(): a static solve from a given start, then the
    mixed-precision time evolution of its states (the use the method makes
    of a converged state).
Device memory comes from torch; every arithmetic step runs in the library.
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs
from . import wslda as W

EF = 0.5                                  # Fermi energy at kF = 1
RHO_SIGMA = 1.0 / (6.0 * math.pi ** 2)    # per-spin density at kF = 1


def draw_trap(seed: int, omega_lo: float, omega_hi: float):
    """(omega_x, omega_y, omega_z) and 1/(kF a) in [0, 1) for one trap."""
    om = inputs.draw_trap_omegas(seed, omega_lo, omega_hi)
    inv_kfa = float(inputs.uniform01(seed ^ 0x5DEECE66D, 1)[0])
    return om, inv_kfa


def net_input(shape, om, inv_kfa):
    """Input channels [2][M]: V_ext / eF and the coupling."""
    M = int(np.prod(shape))
    x = np.empty((2, M), dtype=np.float32)
    x[0] = inputs.harmonic_trap(shape, om) / EF
    x[1] = inv_kfa
    return x


def _box(shape, om, inv_kfa, precision=W.FP64):
    u = W.uniform_solve(shape, kind=W.BDG, inv_4pi_a=inv_kfa / (4 * math.pi), rho_sigma=RHO_SIGMA)
    ctx = W.Context(precision)
    b = ctx.add_box(shape, kind=W.BDG, inv_4pi_a=inv_kfa / (4 * math.pi), mu=u["mu"],
                    nstates=int(np.prod(shape)))
    ctx.set_vext(b, inputs.harmonic_trap(shape, om))
    return ctx, b, u


def solve(shape, om, inv_kfa, U0=None, D0=None, method="broyden", mixing=0.5, eps=1e-6, max_iters=400):
    """Static solve of one trap; returns (result dict, U, Delta real)."""
    ctx, b, u = _box(shape, om, inv_kfa)
    M = int(np.prod(shape))
    U0 = np.zeros(M) if U0 is None else U0
    D0 = np.full(M, u["delta"]) if D0 is None else D0
    res, _ = ctx.static_solve(b, U0, D0, method=method, mixing=mixing, eps_energy=eps, max_iters=max_iters)
    U, D = ctx.get_fields(b)
    ctx.close()
    return res, U, D.real


def dataset(shape, n: int, seed: int, omega_lo=0.1, omega_hi=0.2):
    """n solved traps: inputs [n][2][M] and targets [n][2][M] (float32)."""
    M = int(np.prod(shape))
    X = np.empty((n, 2, M), dtype=np.float32)
    T = np.empty((n, 2, M), dtype=np.float32)
    iters = []
    for i in range(n):
        om, a = draw_trap(seed + i, omega_lo, omega_hi)
        res, U, D = solve(shape, om, a)
        if not res["converged"]:
            raise RuntimeError(f"training trap {i} did not converge")
        X[i] = net_input(shape, om, a)
        T[i, 0] = U / EF
        T[i, 1] = D / EF
        iters.append(res["iters"])
    return X, T, iters


def init_params(net: W.Net, seed: int):
    """Uniform(-s, s) weights with s = sqrt(3 / fan_in) / 2, zero biases, from SplitMix64."""
    theta = np.zeros(net.nparams, dtype=np.float32)
    chans = [2, net.hidden, net.hidden, net.hidden, 2]
    k = 0
    for l in range(4):
        co, ci = chans[l + 1], chans[l]
        nw = co * ci * 27
        s = 0.5 * math.sqrt(3.0 / (ci * 27))
        theta[k:k + nw] = (s * (2.0 * inputs.uniform01(seed + l, nw) - 1.0)).astype(np.float32)
        k += nw + co
    net.set_params(theta)


def train(net: W.Net, X, T, steps: int, batch: int, lr: float, seed: int):
    """Adam on mini-batches drawn in a seeded order; X, T are device tensors
    [n][2][M] (torch). Returns the loss history."""
    import torch
    n = X.shape[0]
    M = X.shape[2]
    xb = torch.empty((batch, 2, M), dtype=torch.float32, device=X.device)
    tb = torch.empty_like(xb)
    losses = []
    order = np.argsort(inputs.uniform01(seed, n))
    pos = 0
    for step in range(steps):
        if pos + batch > n:
            order = np.argsort(inputs.uniform01(seed + step + 1, n))
            pos = 0
        idx = torch.as_tensor(order[pos:pos + batch], device=X.device)
        pos += batch
        torch.index_select(X, 0, idx, out=xb)
        torch.index_select(T, 0, idx, out=tb)
        losses.append(net.loss_grad(xb, tb, batch))
        net.adam(lr)
    return losses


def predict(net: W.Net, x):
    """Network fields for one input [2][M] (numpy), mirror-averaged; returns
    (U, Delta) in code units (numpy float64)."""
    import torch
    M = x.shape[1]
    xd = torch.as_tensor(x[None], device="cuda")
    yd = torch.empty((1, 2, M), dtype=torch.float32, device="cuda")
    sd = torch.empty_like(yd)
    net.forward(xd, yd, 1)
    net.symmetrize(yd, sd, 2)
    y = sd.cpu().numpy()[0].astype(np.float64)
    return y[0] * EF, y[1] * EF


def iterations(shape, om, inv_kfa, U0=None, D0=None, mixing=0.5, eps=1e-6, max_iters=600):
    """Plain linear-mixing iterations to convergence from a start (None: the
    uniform system's fields)."""
    res, _, _ = solve(shape, om, inv_kfa, U0, D0, method="linear", mixing=mixing, eps=eps, max_iters=max_iters)
    return res["iters"], res["converged"]


def converged_td(shape, om, inv_kfa, U0, D0, steps: int = 100, dt: float = 0.007, eps: float = 1e-7,
                 max_iters: int = 400):
    """Static solve of one trap from (U0, D0) (Broyden mixing), then `steps`
    steps of the mixed-precision TD evolution (AB4AM5, stationary start) of its
    states. Returns (solve result, largest relative change of rho over the
    evolution, relative drift of E_tot - mu N)."""
    ctx, b, _ = _box(shape, om, inv_kfa)
    res, _ = ctx.static_solve(b, U0, D0, method="broyden", mixing=0.5, eps_energy=eps, max_iters=max_iters)
    rho0, _ = ctx.get_densities(b)
    phi = ctx.get_states(b)
    ctx.close()
    ctx, b, _ = _box(shape, om, inv_kfa, precision=W.MIXED)
    ctx.load_states(b, phi)
    ctx.start(True, dt)
    ctx.step(dt, steps)
    rho1, _ = ctx.get_densities(b)
    de, _ = ctx.check_conservation(b, float("inf"), float("inf"))
    ctx.close()
    return res, float(np.abs(rho1 - rho0).max() / np.abs(rho0).max()), float(de)
