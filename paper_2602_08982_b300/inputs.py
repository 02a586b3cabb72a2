"""Seeded synthetic inputs for the TDSLDA workloads.

This module holds only random-number generation and the shapes of the
synthetic workloads (trap potentials, perturbation fields, box-size draws).
It contains none of the method's arithmetic, so both the CUDA product path and
the CPU oracle's tests may use it.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated counter-style: the
i-th value of stream `seed` is the i-th output of the generator started at
state `seed`, so any element can be computed on its own.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of SplitMix64 started at state `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def centered_coords(shape, spacing=(1.0, 1.0, 1.0)):
    """Site coordinates x = dx (i - N/2) per axis, broadcastable to the lattice
    (the convention of the paper's custom-initialisation example, Sec. 5.2.1)."""
    out = []
    for ax, (n, d) in enumerate(zip(shape, spacing)):
        c = d * (np.arange(n, dtype=np.float64) - n // 2)
        s = [1, 1, 1]
        s[ax] = n
        out.append(c.reshape(s))
    return out


def harmonic_trap(shape, omega, spacing=(1.0, 1.0, 1.0)) -> np.ndarray:
    """V_ext = 1/2 (wx^2 x^2 + wy^2 y^2 + wz^2 z^2), centred on site N/2, flattened [M]."""
    if np.isscalar(omega):
        omega = (omega, omega, omega)
    x, y, z = centered_coords(shape, spacing)
    v = 0.5 * (omega[0] ** 2 * x ** 2 + omega[1] ** 2 * y ** 2 + omega[2] ** 2 * z ** 2)
    return np.ascontiguousarray(np.broadcast_to(v, tuple(shape)).reshape(-1))


def complex_noise(shape, seed: int) -> np.ndarray:
    """xi = a + i b with a, b uniform in [-1, 1), one pair per site, flattened [M]."""
    m = int(np.prod(shape))
    r = uniform01(seed, 2 * m)
    return (2.0 * r[0::2] - 1.0) + 1j * (2.0 * r[1::2] - 1.0)


def pairing_kick(shape, seed: int, amplitude: float) -> np.ndarray:
    """External pairing field Delta_ext(r) = amplitude * xi(r), flattened [M] complex."""
    return amplitude * complex_noise(shape, seed)


def vortex_phase(shape, spacing=(1.0, 1.0, 1.0), winding: float = 1.0) -> np.ndarray:
    """exp(i winding theta(x, y)) for a straight vortex line along z whose core
    sits half a cell off the central site, theta in (-pi, pi], flattened [M]
    complex. winding = 1/2 gives the factor that multiplies u (and its
    conjugate v) in the vortex start: the product u v^*, hence the pairing
    field, then winds once around the line."""
    x, y, _ = centered_coords(shape, spacing)
    theta = np.arctan2(y - 0.5 * spacing[1], x - 0.5 * spacing[0])
    ph = np.exp(1j * winding * theta)
    return np.ascontiguousarray(np.broadcast_to(ph, tuple(shape)).reshape(-1))


BOX_SIDES = (12, 16, 18, 20, 24)


def draw_box_sides(nboxes: int, seed: int) -> list[int]:
    """Cubic box sides for the batched workload, drawn uniformly from BOX_SIDES."""
    r = uniform01(seed, nboxes)
    return [BOX_SIDES[min(int(v * len(BOX_SIDES)), len(BOX_SIDES) - 1)] for v in r]


def draw_inv_kfa(nboxes: int, seed: int) -> np.ndarray:
    """Dimensionless couplings 1/(kF a) uniform in [-1, 1)."""
    return 2.0 * uniform01(seed, nboxes) - 1.0


def draw_trap_omegas(seed: int, lo: float = 0.04, hi: float = 0.08) -> tuple:
    """Anisotropic trap frequencies (wx, wy, wz) uniform in [lo, hi)."""
    r = uniform01(seed, 3)
    return tuple(lo + (hi - lo) * r)
