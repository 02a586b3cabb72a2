"""The learned starting-field network on the GPU against its oracle, and what
it gains for the static solver."""
import numpy as np
import pytest

from oracle import convnet as cn
from paper_2602_08982_b300 import inputs

pytestmark = pytest.mark.gpu


def _setup(shape, hidden, batch, seed):
    import torch
    from paper_2602_08982_b300 import wslda as W
    net = W.Net(shape, hidden=hidden, max_batch=batch)
    shapes = cn.layer_shapes(2, hidden, 2)
    assert net.nparams == cn.param_count(shapes)
    theta = (0.4 * (2.0 * inputs.uniform01(seed, net.nparams) - 1.0)).astype(np.float32)
    net.set_params(theta)
    M = int(np.prod(shape))
    x = (2.0 * inputs.uniform01(seed + 1, batch * 2 * M) - 1.0).astype(np.float32).reshape(batch, 2, M)
    t = (0.5 * inputs.uniform01(seed + 2, batch * 2 * M)).astype(np.float32).reshape(batch, 2, M)
    xd, td = torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda")
    return net, shapes, theta, x, t, xd, td


@pytest.mark.parametrize("shape,hidden,batch", [((6, 6, 8), 8, 2), ((12, 12, 12), 32, 3), ((5, 7, 9), 32, 2),
                                                ((32, 32, 32), 32, 2)],
                         ids=["6x6x8", "12cubed", "5x7x9", "32cubed"])
def test_each_tensor_core_layer_matches_oracle(shape, hidden, batch):
    """Every layer of the forward pass (tensor-core implicit GEMM, bfloat16
    operands, float32 accumulation) against the oracle's layer fed the GPU's
    own layer input, so both sides round the same float32 values to
    bfloat16 and differ only in the accumulation. The bound is elementwise
    and follows from the arithmetic: the bfloat16 products are exact in
    float32, and any order of n float32 additions, each with a relative error
    of at most 2^-23 (round to nearest or toward zero), is within
    n 2^-23 sum |terms| of the exact sum; tanh does not enlarge it. The 5x7x9
    lattice leaves a ragged last tile of 128 sites."""
    import torch
    net, shapes, theta, x, t, xd, td = _setup(shape, hidden, batch, 303)
    y = torch.empty_like(xd)
    net.forward(xd, y, batch)
    params = cn.unflatten(theta.astype(np.float64), shapes)
    ins = [x] + [net.get_activation(l, batch) for l in range(3)]
    outs = ins[1:] + [y.cpu().numpy()]
    for l, (W, b) in enumerate(params):
        xin = ins[l].astype(np.float64).reshape((batch, -1) + shape)
        xq, Wq = cn.to_bf16(xin), cn.to_bf16(W)
        ref = cn.conv(xq, Wq, b)
        bound = (27 * xin.shape[1] + 1) * 2.0 ** -23 * cn.conv(np.abs(xq), np.abs(Wq), np.abs(b)) + 1e-6
        if l < 3:
            ref = np.tanh(ref)
        got = outs[l].reshape(ref.shape)
        err = np.abs(got - ref)
        assert (err <= bound).all(), (l, float(err.max()), float((err / bound).max()))
        assert err.max() < 1e-4 * max(np.abs(ref).max(), 1.0), l
    net.close()


@pytest.mark.parametrize("shape,hidden,batch", [((6, 6, 8), 8, 2), ((12, 12, 12), 32, 3)])
def test_forward_and_gradient_match_oracle(shape, hidden, batch):
    """The whole network and its gradient against the oracle run from the
    same parameters and inputs. Both round every convolution operand to
    bfloat16; an activation that lies within float32 rounding of a bfloat16
    rounding boundary can round differently on the two sides (the oracle
    carries it in double), which moves single outputs by up to ~1e-3 of the
    largest (6e-4 for the outputs, 1.1e-3 for the gradient in a float32
    emulation on the CPU), hence the tolerances."""
    import torch
    net, shapes, theta, x, t, xd, td = _setup(shape, hidden, batch, 101)
    y = torch.empty_like(xd)
    net.forward(xd, y, batch)
    th = theta.astype(np.float64)
    xo = x.astype(np.float64).reshape((batch, 2) + shape)
    to = t.astype(np.float64).reshape((batch, 2) + shape)
    yo, _ = cn.forward(th, shapes, xo)
    assert np.abs(y.cpu().numpy().reshape(yo.shape) - yo).max() < 3e-3 * np.abs(yo).max()
    loss, g = net.loss_grad(xd, td, batch, want_grad=True)
    Lo, go = cn.gradient(th, shapes, xo, to)
    assert abs(loss - Lo) < 1e-4 * Lo
    assert np.abs(g - go).max() < 5e-3 * np.abs(go).max()
    net.close()


@pytest.mark.parametrize("shape,hidden,batch", [((6, 6, 8), 8, 2), ((12, 12, 12), 32, 3)])
def test_last_layer_weight_gradient_matches_oracle(shape, hidden, batch):
    """The weight gradient of the last layer (split-K tensor-core GEMM) and
    its bias gradient against sums formed with the oracle's operations from
    the GPU's own float32 output and last hidden activation, so that both
    sides round the same values to bfloat16: within 1e-5 of the largest."""
    import torch
    net, shapes, theta, x, t, xd, td = _setup(shape, hidden, batch, 404)
    _, g = net.loss_grad(xd, td, batch, want_grad=True)
    y = torch.empty_like(xd)
    net.forward(xd, y, batch)
    y = y.cpu().numpy()
    a3 = net.get_activation(2, batch).astype(np.float64).reshape((batch, hidden) + shape)
    # dL/dy as the GPU forms it: float32 (2 / n) (y - t)
    gl = (np.float32(2.0 / y.size) * (y - t)).astype(np.float64).reshape((batch, 2) + shape)
    gq, aq = cn.to_bf16(gl), cn.to_bf16(a3)
    ref = np.zeros((2, hidden, 3, 3, 3))
    for d in cn.OFFSETS:
        ref[:, :, d[0] + 1, d[1] + 1, d[2] + 1] = np.einsum("boxyz,bcxyz->oc", gq, cn.shift(aq, d))
    off = cn.param_count(shapes[:3])
    got_w = g[off:off + ref.size].reshape(ref.shape)
    got_b = g[off + ref.size:off + ref.size + 2]
    assert np.abs(got_w - ref).max() < 1e-5 * np.abs(ref).max()
    ref_b = gl.sum(axis=(0, 2, 3, 4))
    assert np.abs(got_b - ref_b).max() < 1e-5 * np.abs(ref_b).max()
    net.close()


def test_adam_step_matches_oracle():
    net, shapes, theta, x, t, xd, td = _setup((6, 6, 8), 8, 2, 202)
    _, g = net.loss_grad(xd, td, 2, want_grad=True)
    net.adam(1e-3)
    got = net.get_params()
    opt = cn.Adam(net.nparams, lr=1e-3)
    ref = opt.step(theta.astype(np.float64), g.astype(np.float64))
    assert np.abs(got - ref).max() < 1e-6
    net.close()


def test_symmetrize_matches_mirror_average():
    import torch
    from paper_2602_08982_b300 import wslda as W
    shape = (6, 8, 4)
    net = W.Net(shape, hidden=8, max_batch=1)
    y = (2.0 * inputs.uniform01(7, 3 * 192) - 1.0).astype(np.float32).reshape(3, 192)
    yd = torch.as_tensor(y, device="cuda")
    out = torch.empty_like(yd)
    net.symmetrize(yd, out, 3)
    ref = cn.mirror_average(y.astype(np.float64).reshape((1, 3) + shape)).reshape(3, 192)
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-6
    net.close()


HELD_OUT = (5000, 5001, 5002, 5003, 5004)  # fixed before any run; every trap is counted


def test_trained_network_cuts_static_iterations():
    """Train on solved 12^3 traps, then start the fixed held-out traps from the
    network's fields and from the uniform system's, with plain linear mixing.
    A solve that reaches the iteration cap is a result, not an exclusion: it
    counts as the cap in the means and as a failure in the convergence count.
    The network's start must converge on at least as many traps, need fewer
    iterations on average over all of them, and at least 20% fewer on the
    traps that both starts solve."""
    import torch
    from paper_2602_08982_b300 import learned as L
    from paper_2602_08982_b300 import wslda as W
    shape = (12, 12, 12)
    cap = 400
    X, T, _ = L.dataset(shape, 32, seed=1000)
    net = W.Net(shape, hidden=32, max_batch=8)
    L.init_params(net, 77)
    losses = L.train(net, torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda"), steps=400, batch=8,
                     lr=2e-3, seed=5)
    assert losses[-1] < 0.2 * losses[0]
    rows = []
    for seed in HELD_OUT:
        om, a = L.draw_trap(seed, 0.1, 0.2)
        n0, ok0 = L.iterations(shape, om, a, eps=1e-5, max_iters=cap)
        U, D = L.predict(net, L.net_input(shape, om, a))
        # the BdG functional has no mean field: only Delta is taken from the network
        n1, ok1 = L.iterations(shape, om, a, U0=np.zeros_like(U), D0=D, eps=1e-5, max_iters=cap)
        rows.append((seed, n0 if ok0 else cap, ok0, n1 if ok1 else cap, ok1))
    # the pipeline the learned start feeds: a converged static solve from the
    # network's fields, then 100 mixed-precision TD steps of its states
    om, a = L.draw_trap(HELD_OUT[0], 0.1, 0.2)
    U, D = L.predict(net, L.net_input(shape, om, a))
    res, drho, de = L.converged_td(shape, om, a, np.zeros_like(U), D, steps=100)
    net.close()
    print("held-out traps (seed, uniform iters, converged, network iters, converged):", rows)
    for k, name in ((1, "uniform start"), (3, "network start")):
        it = [r[k] for r in rows]
        print(f"{name}: mean {np.mean(it):.1f}, median {np.median(it):.1f} iterations (cap {cap} counted)")
    print(f"100 mixed TD steps from the network-started solve ({res['iters']} Broyden iterations): "
          f"rho changes by {drho:.2e}, E - mu N drifts by {de:.2e}")
    assert res["converged"] and drho < 1e-3 and de < 1e-5
    assert sum(r[4] for r in rows) >= sum(r[2] for r in rows), rows
    assert np.mean([r[3] for r in rows]) < np.mean([r[1] for r in rows]), rows
    both = [r for r in rows if r[2] and r[4]]
    assert len(both) >= 3, rows
    assert np.mean([r[3] for r in both]) < 0.8 * np.mean([r[1] for r in both]), rows
