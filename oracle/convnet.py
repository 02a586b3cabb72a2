"""Plain FP64 CPU oracle of the learned starting-field network.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import or run anything in this package; the
product path never does, and this module never imports the product.

The network maps per-site input channels (the trap potential V_ext / eF and the
coupling) on a periodic lattice to per-site outputs (U / eF, Delta / eF) that
start the static self-consistent iteration of Alg. 1 (Sec. 3.2). It is a stack
of 3x3x3 convolutions with periodic wrap-around (the lattice is periodic,
Sec. 3.1), tanh between layers and a linear last layer, trained on the mean
squared error with Adam (Kingma and Ba, arXiv:1412.6980). Weights are used in
bfloat16 (rounded to nearest even from the float32 master copy), and so is
every convolution operand: a layer's input enters its convolution rounded to
bfloat16, and the gradient of a layer's output enters both gradient
convolutions (with respect to the weights and to the input) rounded too,
the weight gradient pairing it with the rounded inputs (the operands of
bfloat16 tensor-core GEMMs with float32 accumulation). Everything else is
float64 here. With bf16=False nothing is rounded (the plain network).

Conventions: activations x[b, c, ix, iy, iz]; weights W[co, ci, dx, dy, dz]
with offsets d - 1 in {-1, 0, 1}; a layer computes
  y[b, co, r] = bias[co] + sum_ci sum_d W[co, ci, d] x[b, ci, r + d - 1]   (periodic).
Parameters are flattened layer by layer as (W, bias).

Pins (tests/test_oracle_convnet.py): the convolution equals a circular
cross-correlation computed with the FFT, analytic gradients equal central
finite differences, the first Adam step equals its closed form, bfloat16
rounding matches the definition (round to nearest, ties to even, of the top
16 bits of the float32 pattern).
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]


def layer_shapes(cin: int, hidden: int, cout: int, layers: int = 4):
    """[(c_out, c_in)] of each layer: cin -> hidden -> ... -> hidden -> cout."""
    chans = [cin] + [hidden] * (layers - 1) + [cout]
    return [(chans[i + 1], chans[i]) for i in range(layers)]


def param_count(shapes) -> int:
    return sum(co * ci * 27 + co for co, ci in shapes)


def unflatten(theta, shapes):
    out, k = [], 0
    for co, ci in shapes:
        W = theta[k:k + co * ci * 27].reshape(co, ci, 3, 3, 3)
        k += co * ci * 27
        b = theta[k:k + co]
        k += co
        out.append((W, b))
    return out


def to_bf16(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def shift(x, d):
    """x[..., r + d] with periodic wrap (d a 3-tuple of offsets)."""
    return np.roll(x, shift=(-d[0], -d[1], -d[2]), axis=(-3, -2, -1))


def conv(x, W, b):
    """One periodic 3x3x3 layer, summed offset by offset."""
    B = x.shape[0]
    y = np.zeros((B, W.shape[0]) + x.shape[2:])
    for d in OFFSETS:
        xs = shift(x, d)
        y += np.einsum("oc,bcxyz->boxyz", W[:, :, d[0] + 1, d[1] + 1, d[2] + 1], xs)
    return y + b[None, :, None, None, None]


def forward(theta, shapes, x, bf16: bool = True):
    """Returns the output and the list of layer inputs (for the backward pass)."""
    params = unflatten(theta, shapes)
    acts = [x]
    h = x
    for i, (W, b) in enumerate(params):
        Wq = to_bf16(W) if bf16 else W
        h = conv(to_bf16(h) if bf16 else h, Wq, b)
        if i < len(params) - 1:
            h = np.tanh(h)
        acts.append(h)
    return h, acts


def loss(y, t) -> float:
    """Mean squared error over every element."""
    return float(np.mean((y - t) ** 2))


def gradient(theta, shapes, x, t, bf16: bool = True):
    """Loss and its gradient with respect to the flattened parameters (the
    gradient of the bfloat16-rounded weights is applied to the master copy)."""
    params = unflatten(theta, shapes)
    y, acts = forward(theta, shapes, x, bf16)
    L = loss(y, t)
    g = 2.0 * (y - t) / y.size  # dL/dy
    grads = []
    for i in range(len(params) - 1, -1, -1):
        W, b = params[i]
        Wq = to_bf16(W) if bf16 else W
        if i < len(params) - 1:
            g = g * (1.0 - acts[i + 1] ** 2)  # through tanh
        xin = to_bf16(acts[i]) if bf16 else acts[i]
        gq = to_bf16(g) if bf16 else g
        gW = np.zeros_like(W)
        for d in OFFSETS:
            gW[:, :, d[0] + 1, d[1] + 1, d[2] + 1] = np.einsum("boxyz,bcxyz->oc", gq, shift(xin, d))
        gb = g.sum(axis=(0, 2, 3, 4))
        grads.append((gW, gb))
        # dL/dx[r] = sum_d W[:, :, d]^T g[r - d]
        gx = np.zeros_like(xin)
        for d in OFFSETS:
            gx += np.einsum("oc,boxyz->bcxyz", Wq[:, :, d[0] + 1, d[1] + 1, d[2] + 1],
                            shift(gq, (-d[0], -d[1], -d[2])))
        g = gx
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.reshape(-1))
        flat.append(gb)
    return L, np.concatenate(flat)


class Adam:
    """Adam with bias correction (Kingma and Ba), applied to the float64 copy."""

    def __init__(self, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, theta, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def mirror_average(y):
    """Average over the 8 reflections i -> N - i (mod N) of the three axes: the
    projection onto fields with the symmetry of a trap centred on site N/2."""
    out = np.zeros_like(y)
    for fx in (0, 1):
        for fy in (0, 1):
            for fz in (0, 1):
                z = y
                for ax, f in zip((-3, -2, -1), (fx, fy, fz)):
                    if f:
                        z = np.roll(np.flip(z, axis=ax), 1, axis=ax)
                out += z
    return out / 8.0
