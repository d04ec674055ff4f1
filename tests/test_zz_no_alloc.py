"""The allocation-free entry point, gp_kernel_matvec_static_scratch, against
the workspace entry point, gp_kernel_matvec.

It serves callers that cannot allocate device memory when they call in (an
application that owns all device memory through its own pool, a
latency-critical loop that must avoid cudaMalloc's implicit synchronisation,
a plugin without access to its host's allocator). Its scratch is a static
device array shared by every call, so the test runs it twice in a row with
different inputs and checks each result. This file is collected last so that
a run stopping at the first failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import abi, api, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return abi.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def static_call(lib, q, s, v, ell, var, want_beta):
    cq, k1 = api.to_c_points(q)
    cs, k2 = api.to_c_points(s)
    out = torch.empty(cq.n, dtype=torch.float32, device="cuda")
    beta = torch.empty((cq.n, 2), dtype=torch.float32, device="cuda") if want_beta else None
    st = lib.gp_kernel_matvec_static_scratch(ctypes.byref(cq), ctypes.byref(cs) if cs is not None else None,
                                             v.data_ptr(), 1, ell, var, out.data_ptr(),
                                             beta.data_ptr() if beta is not None else None,
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    abi.check(st, "gp_kernel_matvec_static_scratch")
    return out, beta


def compare(lib, q, s, v, ell, var, want_beta=False):
    """The static-scratch call runs the same plan and kernels as
    gp_kernel_matvec, so its output must be the same bits; a stale word read
    from the shared array would show up as a difference."""
    got, gbeta = static_call(lib, q, s, v, ell, var, want_beta)
    ref, rbeta = api.gp_kernel_matvec(q, s, v, ell, var, want_beta=True) if want_beta else \
        (api.gp_kernel_matvec(q, s, v, ell, var), None)
    torch.cuda.synchronize()
    assert torch.equal(got, ref), float((got - ref).abs().max())
    if want_beta:
        assert torch.equal(gbeta, rbeta)


def test_fused_grid_two_calls_in_a_row(lib):
    p = W.realistic(seed=31, side=120, ss=2, n_sub=60)
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub))
    s = api.Points(grid=p.ygrid)
    size = api.matvec_workspace_size(q, s)
    assert 0 < size <= lib.lr_static_scratch_bytes()
    compare(lib, q, s, dev(p.v), p.lengthscale, p.variance, want_beta=False)
    v2 = np.random.default_rng(1).standard_normal(p.m).astype(np.float32)
    compare(lib, q, s, dev(v2), p.lengthscale, 0.7, want_beta=True)


def test_self_kernel_two_calls_in_a_row(lib):
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, (30000, 2)).astype(np.float32)
    for k in range(2):
        v = rng.standard_normal(30000).astype(np.float32)
        compare(lib, api.Points(xy=dev(x)), None, dev(v), 0.05 * (1 + k), 1.0)


def test_rejects_problems_beyond_the_static_scratch(lib):
    # a ray-traced query whose point scratch alone (8 bytes per point) is
    # larger than the static array, whatever its size
    cap = int(lib.lr_static_scratch_bytes())
    side = int(np.ceil(np.sqrt(cap / 8 + 1))) + 1
    g = W.Grid(side, side, 1, 0.01)
    assert 8 * g.n > cap
    lens = W.Lens(0.0, 0.0, 0.8, 0.2, 1.2, 2.0, 0.0, 0.0)
    cq, keep = api.to_c_points(api.Points(grid=g, lens=lens))
    cs, keep2 = api.to_c_points(api.Points(grid=W.Grid(4, 4, 1, 0.1)))
    # real buffers of the full sizes: validation must reject the call before
    # any launch, and no argument is a made-up or too-short address
    v = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(g.n, dtype=torch.float32, device="cuda")
    st = lib.gp_kernel_matvec_static_scratch(ctypes.byref(cq), ctypes.byref(cs), v.data_ptr(), 1, 0.1, 1.0,
                                             out.data_ptr(), None, None)
    assert st == abi.LR_ERR_INVALID_ARG
    assert b"static scratch" in lib.lr_last_error()
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
