"""The allocation-free density entry point against the context-based one.

wslda_densities_noalloc serves callers that cannot call cudaMalloc (device
memory owned by their own pool allocator, or latency-critical paths where an
allocation's implicit synchronisation or failure is not acceptable). Its
results must agree with wslda_get_densities on the same states, and stay
correct when called twice in a row (the scratch array keeps the last call's
contents). This file is collected last so that a run stopping at its first
failure has already run every other test.
"""
import numpy as np
import pytest

from cases import gpu_context, make_case, rel

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_densities_match_context_path(prec):
    import torch
    from paper_2602_08982_b300 import wslda as W
    case = make_case((8, 12, 16), (1.0, 0.9, 1.1), kind="bdg", nstates=301, trap=0.1, kick=0.05, seed=21,
                     thermal=True)
    ctx, box = gpu_context(case, prec)
    rho_ref, nu_ref = ctx.get_densities(box)
    ctx.close()
    dev = torch.device("cuda")
    ctype = torch.complex64 if prec == W.MIXED else torch.complex128
    uv = torch.from_numpy(case.phi.astype(np.complex64 if prec == W.MIXED else np.complex128)).to(dev, ctype)
    wm = torch.from_numpy(case.wm).to(dev)
    wp = torch.from_numpy(case.wp).to(dev)
    M = case.lat.M
    results = []
    for _ in range(2):  # two calls in a row share the scratch array
        rho = torch.full((M,), float("nan"), dtype=torch.float64, device=dev)
        nu = torch.full((2 * M,), float("nan"), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        W.densities_noalloc(prec, uv, rho, nu, case.lat.shape, wm, wp, stream=stream)
        torch.cuda.synchronize()
        r = rho.cpu().numpy()
        n = nu.cpu().numpy().view(np.complex128)
        assert rel(r, rho_ref) < TOL[prec] and rel(n, nu_ref) < TOL[prec]
        results.append((r, n))
    assert np.array_equal(results[0][0], results[1][0]) and np.array_equal(results[0][1], results[1][1])


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch
    from paper_2602_08982_b300 import wslda as W
    dev = torch.device("cuda")
    shape = (128, 128, 64)
    M = shape[0] * shape[1] * shape[2]
    uv = torch.zeros((1, 2, M), dtype=torch.complex64, device=dev)
    rho = torch.zeros(M, dtype=torch.float64, device=dev)
    nu = torch.zeros(2 * M, dtype=torch.float64, device=dev)
    with pytest.raises(W.WsldaError) as e:
        W.densities_noalloc(W.MIXED, uv, rho, nu, shape)
    assert e.value.status == 2


def test_noalloc_binding_checks_shapes_and_dtypes():
    """The C call takes raw device pointers, so the binding refuses tensors
    whose dtype, shape or length would make the kernels step outside them."""
    import torch
    from paper_2602_08982_b300 import wslda as W
    dev = torch.device("cuda")
    shape = (8, 8, 8)
    M = 512
    uv = torch.zeros((3, 2, M), dtype=torch.complex64, device=dev)
    rho = torch.zeros(M, dtype=torch.float64, device=dev)
    nu = torch.zeros(2 * M, dtype=torch.float64, device=dev)
    bad = [
        (W.FP64, uv, rho, nu, None),                                   # complex64 states for FP64
        (W.MIXED, uv[:, :, :256], rho, nu, None),                      # wrong site count
        (W.MIXED, uv, rho[:100], nu, None),                            # rho too short
        (W.MIXED, uv, rho, nu[:M], None),                              # nu too short
        (W.MIXED, uv, rho, nu, torch.ones(2, dtype=torch.float64, device=dev)),  # weights too short
        (W.MIXED, uv.cpu(), rho, nu, None),                            # host tensor
    ]
    for prec, u, r, n, w in bad:
        with pytest.raises(ValueError):
            W.densities_noalloc(prec, u, r, n, shape, w, w)
