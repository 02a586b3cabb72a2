"""Pins of the learned starting-field network oracle (oracle/convnet.py)."""
import numpy as np

from oracle import convnet as cn
from paper_2602_08982_b300 import inputs


def _params(shapes, seed):
    n = cn.param_count(shapes)
    return 0.3 * (2.0 * inputs.uniform01(seed, n) - 1.0)


def test_periodic_convolution_is_a_circular_cross_correlation():
    """Each (out, in) channel pair against numpy's FFT: sum_s k[s] x[r + s]
    has the transform conj(K) X for a real kernel k."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 3, 6, 5, 4))
    W = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cn.conv(x, W, b)
    N = x.shape[2:]
    ref = np.zeros_like(y)
    for co in range(4):
        for ci in range(3):
            k = np.zeros(N)
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        k[dx % N[0], dy % N[1], dz % N[2]] += W[co, ci, dx + 1, dy + 1, dz + 1]
            K = np.fft.fftn(k)
            ref[:, co] += np.real(np.fft.ifftn(np.conj(K)[None] * np.fft.fftn(x[:, ci], axes=(1, 2, 3)),
                                               axes=(1, 2, 3)))
        ref[:, co] += b[co]
    assert np.abs(y - ref).max() < 1e-12


def test_gradient_matches_central_differences():
    shapes = cn.layer_shapes(2, 3, 2)
    theta = _params(shapes, 11)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 2, 4, 4, 4))
    t = rng.standard_normal((2, 2, 4, 4, 4))
    L, g = cn.gradient(theta, shapes, x, t, bf16=False)
    idx = np.unique(np.concatenate([np.arange(0, len(theta), 7), [len(theta) - 1]]))
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (cn.loss(cn.forward(tp, shapes, x, False)[0], t) - cn.loss(cn.forward(tm, shapes, x, False)[0], t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])), (i, fd, g[i])
    assert abs(L - cn.loss(cn.forward(theta, shapes, x, False)[0], t)) == 0.0


def test_bfloat16_rounding_follows_its_definition():
    one = 1.0
    half_ulp = 2.0 ** -8   # bfloat16 has 7 stored mantissa bits at 1.0: ulp 2^-7
    vals = np.array([one, one + half_ulp, one + 3 * half_ulp, one + half_ulp * 1.001, -2.5, 3.0e-3])
    got = cn.to_bf16(vals)
    assert got[0] == 1.0
    assert got[1] == 1.0                  # tie -> even mantissa
    assert got[2] == 1.0 + 2.0 ** -6      # tie between odd 1 + 2^-7 and even 1 + 2^-6
    assert got[3] == 1.0 + 2.0 ** -7      # above the tie rounds up
    assert got[4] == -2.5                 # representable
    assert abs(got[5] - 3.0e-3) <= 2.0 ** -8 * 3.0e-3   # half an ulp of 7 mantissa bits


def test_first_adam_step_has_its_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 2.0, 3.0, 4.0])
    opt = cn.Adam(4, lr=0.01)
    out = opt.step(th, g)
    assert np.allclose(out, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_mirror_average_projects_onto_reflection_symmetric_fields():
    rng = np.random.default_rng(9)
    y = rng.standard_normal((1, 2, 6, 8, 4))
    s = cn.mirror_average(y)
    assert np.abs(cn.mirror_average(s) - s).max() < 1e-15
    v = inputs.harmonic_trap((6, 8, 4), (0.3, 0.2, 0.1)).reshape(1, 1, 6, 8, 4)
    assert np.abs(cn.mirror_average(v) - v).max() < 1e-15
    i = (2, 5, 1)
    m = tuple((n - k) % n for k, n in zip(i, (6, 8, 4)))
    assert abs(s[0, 0][i] - s[0, 0][m]) < 1e-15
