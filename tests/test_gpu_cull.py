"""Culled reductions over explicit point sets against the FP64 oracle.

Covers several right-hand sides in one pass (forward and backward, each
column against the oracle, explicit, self and grid sources), ray-traced
pixels that carry their image layout (where the exact-zero skipping leaves
out most pairs), ragged layouts, length scales well above and well below the
point spacing, and the skipping itself: the same bits with
lr_set_pair_culling(0) as with it on."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import abi, api, workloads as W
from tests.gpu_util import assert_matvec_close, dev, host, need_gpu

pytestmark = pytest.mark.gpu

REL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    yield
    abi.load().lr_set_pair_culling(1)


def close(got, ref, scale, rel=REL, what=""):
    got, ref, scale = (np.asarray(a, np.float64) for a in (got, ref, scale))
    tol = rel * scale + 1e-30
    err = np.abs(got - ref)
    bad = err > tol
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} outside; worst ratio {np.max(err / tol):.2f}, "
                           f"err {err.flat[np.argmax(err / tol)]:.3e} scale {scale.flat[np.argmax(err / tol)]:.3e}")


def pts(rng, n, hw):
    return rng.uniform(-hw, hw, (n, 2)).astype(np.float32)


def traced(orc, p):
    """The oracle's ray-traced pixels of a workload, rounded to FP32 (both
    sides read the same points, which isolates the reduction)."""
    _, b = orc.raytrace(orc.grid_points(*p.xgrid.astuple()), p.lens.astuple(), p.sub)
    return b.astype(np.float32)


def oracle_bwd(orc, x, y, v, g, ell, var, self_kernel):
    """Per right-hand side oracle gradients, summed where the CUDA path sums."""
    R = [orc.kernel_matvec_vjp(x, x if self_kernel else y, v[:, r], ell, var, g[:, r].astype(np.float64),
                               self_kernel, with_abs=True) for r in range(v.shape[1])]
    out = {"d_v": np.stack([r["d_v"] for r in R], 1), "d_v_abs": np.stack([r["d_v_abs"] for r in R], 1)}
    for k in ("d_x", "d_len", "d_var") + (() if self_kernel else ("d_y",)):
        out[k] = sum(r[k] for r in R)
        out[k + "_abs"] = sum(r[k + "_abs"] for r in R)
    return out


@pytest.mark.parametrize("nrhs", [1, 2, 3, 4])
def test_multi_rhs_forward_explicit(orc, nrhs):
    rng = np.random.default_rng(100 + nrhs)
    x, y = pts(rng, 3001, 0.7), pts(rng, 2777, 0.7)
    v = rng.standard_normal((2777, nrhs)).astype(np.float32)
    got = host(api.gp_kernel_matvec(api.Points(xy=dev(x)), api.Points(xy=dev(y)), dev(v), 0.05, 1.2))
    assert got.shape == (3001, nrhs)
    for r in range(nrhs):
        ref, ab = orc.kernel_matvec(x, y, v[:, r], 0.05, 1.2)
        assert_matvec_close(got[:, r], ref, ab, what=f"rhs {r}")


@pytest.mark.parametrize("nrhs", [2, 4])
def test_multi_rhs_self_kernel_layout(orc, nrhs):
    """Ray-traced pixels with their image layout, self-kernel, nrhs columns."""
    p = W.realistic(seed=61, side=70, ss=2, n_sub=30)
    b = traced(orc, p)
    rng = np.random.default_rng(nrhs)
    v = rng.standard_normal((p.n, nrhs)).astype(np.float32)
    got = host(api.gp_kernel_matvec(api.Points(xy=dev(b), grid=p.xgrid), None, dev(v), 0.05, 1.0))
    for r in range(nrhs):
        ref, ab = orc.kernel_matvec(b, b, v[:, r], 0.05, 1.0)
        assert_matvec_close(got[:, r], ref, ab, what=f"self rhs {r}")


@pytest.mark.parametrize("nrhs", [1, 3])
def test_multi_rhs_backward_self(orc, nrhs):
    rng = np.random.default_rng(7 + nrhs)
    x = pts(rng, 5000, 0.9)
    v = rng.standard_normal((5000, nrhs)).astype(np.float32)
    g = rng.standard_normal((5000, nrhs)).astype(np.float32)
    G = api.gp_kernel_matvec_bwd(api.Points(xy=dev(x)), None, dev(v), 0.05, 1.1, dev(g),
                                 want=("v", "x", "lengthscale", "variance"))
    R = oracle_bwd(orc, x, None, v, g, 0.05, 1.1, True)
    close(host(G["v"]), R["d_v"], R["d_v_abs"], what="d_v")
    close(host(G["x"]), R["d_x"], R["d_x_abs"], what="d_x")
    close(host(G["lengthscale"]), [R["d_len"]], [R["d_len_abs"]], what="d_len")
    close(host(G["variance"]), [R["d_var"]], [R["d_var_abs"]], what="d_var")


@pytest.mark.parametrize("nrhs", [1, 2])
def test_multi_rhs_backward_explicit(orc, nrhs):
    rng = np.random.default_rng(17 + nrhs)
    x, y = pts(rng, 2100, 0.6), pts(rng, 2500, 0.6)
    v = rng.standard_normal((2500, nrhs)).astype(np.float32)
    g = rng.standard_normal((2100, nrhs)).astype(np.float32)
    G = api.gp_kernel_matvec_bwd(api.Points(xy=dev(x)), api.Points(xy=dev(y)), dev(v), 0.05, 0.8, dev(g),
                                 want=("v", "x", "y", "lengthscale", "variance"))
    R = oracle_bwd(orc, x, y, v, g, 0.05, 0.8, False)
    close(host(G["v"]), R["d_v"], R["d_v_abs"], what="d_v")
    close(host(G["x"]), R["d_x"], R["d_x_abs"], what="d_x")
    close(host(G["y"]), R["d_y"], R["d_y_abs"], what="d_y")
    close(host(G["lengthscale"]), [R["d_len"]], [R["d_len_abs"]], what="d_len")
    close(host(G["variance"]), [R["d_var"]], [R["d_var_abs"]], what="d_var")


@pytest.mark.parametrize("nx,ny,ell", [(77, 45, 0.05), (64, 32, 0.05), (50, 90, 0.002), (33, 33, 0.4)])
def test_layout_self_kernel_forward_backward(orc, nx, ny, ell):
    """Ragged image layouts (not multiples of the chunk, group or row-block
    tile); length scales well above the point spacing and at 2 mas, far
    below the 25 mas spacing, where a row's sum beyond its own point is made
    of far pairs (scaled distance^2 of 30 to 120) and a chunk spans many
    length scales."""
    lens = W.Lens(0.05, -0.03, 0.75, 0.4, 1.1, 2.05, 0.02, -0.01)
    g = W.Grid(nx, ny, 2, 0.05)
    _, b = orc.raytrace(orc.grid_points(*g.astuple()), lens.astuple())
    b = b.astype(np.float32)
    rng = np.random.default_rng(nx * ny)
    v = rng.standard_normal(g.n).astype(np.float32)
    gg = rng.standard_normal(g.n).astype(np.float32)
    q = api.Points(xy=dev(b), grid=g)
    got = host(api.gp_kernel_matvec(q, None, dev(v), ell, 0.9))
    ref, ab = orc.kernel_matvec(b, b, v, ell, 0.9)
    assert_matvec_close(got, ref, ab, what="layout self forward")
    G = api.gp_kernel_matvec_bwd(q, None, dev(v), ell, 0.9, dev(gg), want=("v", "x", "lengthscale", "variance"))
    R = orc.kernel_matvec_vjp(b, b, v, ell, 0.9, gg.astype(np.float64), True, with_abs=True)
    close(host(G["v"]), R["d_v"], R["d_v_abs"], what="d_v")
    close(host(G["x"]), R["d_x"], R["d_x_abs"], what="d_x")
    close(host(G["lengthscale"]), [R["d_len"]], [R["d_len_abs"]], what="d_len")
    close(host(G["variance"]), [R["d_var"]], [R["d_var_abs"]], what="d_var")


def test_layout_explicit_sources_backward(orc):
    """Ray-traced pixels (with layout) against another ray-traced pixel set
    (with its own layout): d_v and d_y run with the roles swapped."""
    p = W.realistic(seed=71, side=40, ss=2, n_sub=5)
    b = traced(orc, p)
    p2 = W.realistic(seed=72, side=30, ss=2, n_sub=0)
    y = traced(orc, p2)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(p2.n).astype(np.float32)
    gg = rng.standard_normal(p.n).astype(np.float32)
    q, s = api.Points(xy=dev(b), grid=p.xgrid), api.Points(xy=dev(y), grid=p2.xgrid)
    got = host(api.gp_kernel_matvec(q, s, dev(v), 0.07, 1.0))
    ref, ab = orc.kernel_matvec(b, y, v, 0.07, 1.0)
    assert_matvec_close(got, ref, ab, what="layout explicit forward")
    G = api.gp_kernel_matvec_bwd(q, s, dev(v), 0.07, 1.0, dev(gg), want=("v", "x", "y", "lengthscale", "variance"))
    R = orc.kernel_matvec_vjp(b, y, v, 0.07, 1.0, gg.astype(np.float64), False, with_abs=True)
    for k in ("v", "x", "y"):
        close(host(G[k]), R["d_" + k], R["d_" + k + "_abs"], what="d_" + k)
    close(host(G["lengthscale"]), [R["d_len"]], [R["d_len_abs"]], what="d_len")


def _both(fn):
    lib = abi.load()
    try:
        lib.lr_set_pair_culling(0)
        a = fn()
        lib.lr_set_pair_culling(1)
        b = fn()
    finally:
        lib.lr_set_pair_culling(1)
    return a, b


def test_culling_changes_no_bit(orc):
    """The skipped pairs are exact zeros: culled and unculled sweeps, in the
    same order, give bitwise equal forward outputs and gradients."""
    p = W.realistic(seed=81, side=120, ss=2, n_sub=20)
    beta = api.lens_raytrace(api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub)))
    rng = np.random.default_rng(9)
    v = dev(rng.standard_normal((p.n, 2)).astype(np.float32))
    g = dev(rng.standard_normal((p.n, 2)).astype(np.float32))
    q = api.Points(xy=beta, grid=p.xgrid)

    def run():
        out = api.gp_kernel_matvec(q, None, v, 0.05, 1.0)
        G = api.gp_kernel_matvec_bwd(q, None, v, 0.05, 1.0, g, want=("v", "x", "lengthscale", "variance"))
        torch.cuda.synchronize()
        return [out] + [G[k] for k in ("v", "x", "lengthscale", "variance")]

    off, on = _both(run)
    for a, b in zip(off, on):
        assert torch.equal(a, b)


def test_culling_changes_no_bit_explicit_sources(orc):
    p = W.realistic(seed=82, side=60, ss=2, n_sub=0)
    beta = api.lens_raytrace(api.Points(grid=p.xgrid, lens=p.lens))
    rng = np.random.default_rng(10)
    y = dev(pts(rng, 9000, 2.0))
    v = dev(rng.standard_normal(9000).astype(np.float32))
    g = dev(rng.standard_normal(p.n).astype(np.float32))
    q, s = api.Points(xy=beta, grid=p.xgrid), api.Points(xy=y)

    def run():
        out = api.gp_kernel_matvec(q, s, v, 0.05, 1.0)
        G = api.gp_kernel_matvec_bwd(q, s, v, 0.05, 1.0, g, want=("v", "x", "y", "lengthscale", "variance"))
        torch.cuda.synchronize()
        return [out] + [G[k] for k in ("v", "x", "y", "lengthscale", "variance")]

    off, on = _both(run)
    for a, b in zip(off, on):
        assert torch.equal(a, b)


def test_rejects_nrhs_outside_range():
    x = dev(np.zeros((4, 2)))
    with pytest.raises(abi.LensGPError):
        api.gp_kernel_matvec(api.Points(xy=x), None, torch.zeros((4, 5), device="cuda"), 0.1)
    with pytest.raises(abi.LensGPError):
        api.gp_kernel_matvec(api.Points(xy=x), api.Points(grid=W.Grid(4, 4, 1, 0.1)),
                             torch.zeros((16, 5), device="cuda"), 0.1)


@pytest.mark.parametrize("nrhs", [2, 4])
def test_multi_rhs_grid_sources(orc, nrhs):
    """Ray-traced pixels against a grid of inducing points with several
    right-hand sides: forward and backward, each column against the oracle."""
    p = W.realistic(seed=91, side=60, ss=2, n_sub=12, ygrid_side=40)
    b = traced(orc, p)
    rng = np.random.default_rng(nrhs)
    v = rng.standard_normal((p.m, nrhs)).astype(np.float32)
    g = rng.standard_normal((p.n, nrhs)).astype(np.float32)
    q, s = api.Points(xy=dev(b), grid=p.xgrid), api.Points(grid=p.ygrid)
    got = host(api.gp_kernel_matvec(q, s, dev(v), p.lengthscale, p.variance))
    yg = orc.grid_points(*p.ygrid.astuple())
    for r in range(nrhs):
        ref, ab = orc.kernel_matvec(b, yg, v[:, r], p.lengthscale, p.variance)
        assert_matvec_close(got[:, r], ref, ab, what=f"grid rhs {r}")
    G = api.gp_kernel_matvec_bwd(q, s, dev(v), p.lengthscale, p.variance, dev(g),
                                 want=("v", "x", "lengthscale", "variance"))
    R = oracle_bwd(orc, b, yg, v, g, p.lengthscale, p.variance, False)
    close(host(G["v"]), R["d_v"], R["d_v_abs"], what="d_v")
    close(host(G["x"]), R["d_x"], R["d_x_abs"], what="d_x")
    close(host(G["lengthscale"]), [R["d_len"]], [R["d_len_abs"]], what="d_len")
    close(host(G["variance"]), [R["d_var"]], [R["d_var_abs"]], what="d_var")


def test_no_fault_recorded():
    assert api.fault_status() == 0
