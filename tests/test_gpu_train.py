"""Parity of the training forward (gp_kernel_matvec_train: out plus the row
moments) and of the backward pass fed those moments, against the FP64
oracle, for grid sources on both sides of the split-exponent bound, explicit
sources and the fused ray-traced chain."""
import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import abi, api, workloads as W
from tests.gpu_util import (assert_close_tol, assert_matvec_close, chain_tol, dev, host, lens_chain_tols, need_gpu,
                            point_delta)
from tests.test_gpu_backward import close, fused_chain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def grid_case(ratio, seed):
    rng = np.random.default_rng(seed)
    g = W.Grid(260, 30, 1, 0.04)
    x = np.stack([rng.uniform(-5.6, 5.6, 2999), rng.uniform(-0.7, 0.7, 2999)], -1).astype(np.float32)
    return g, x, rng.standard_normal(g.n).astype(np.float32), rng.standard_normal(2999).astype(np.float32), ratio * 0.04


@pytest.mark.parametrize("ratio", [0.5, 1.2, 1.25, 1.5, 4.0])
def test_grid_source(orc, ratio):
    g, x, v, gout, ell = grid_case(ratio, int(10 * ratio))
    yg = orc.grid_points(*g.astuple())
    q, s = api.Points(xy=dev(x)), api.Points(grid=g)
    out, mom = api.gp_kernel_matvec_train(q, s, dev(v), ell, 0.8)
    ref, ab = orc.kernel_matvec(x, yg, v, ell, 0.8)
    assert_matvec_close(host(out), ref, ab, what="train forward")
    G = api.gp_kernel_matvec_bwd(q, s, dev(v), ell, 0.8, dev(gout), want=["v", "x", "lengthscale", "variance"],
                                 moments=mom)
    R = orc.kernel_matvec_vjp(x, yg, v, ell, 0.8, gout.astype(np.float64), False, with_abs=True)
    close(host(G["v"]), R["d_v"], R["d_v_abs"], what="d_v")
    close(host(G["x"]), R["d_x"], R["d_x_abs"], what="d_x")
    close(host(G["lengthscale"]), [R["d_len"]], [R["d_len_abs"]], what="d_len")
    close(host(G["variance"]), [R["d_var"]], [R["d_var_abs"]], what="d_var")


@pytest.mark.parametrize("ell", [0.03, 0.08])
def test_grid_query_odd_source_grid(orc, ell):
    """Pixel-grid queries (compact row blocks: the training forward's and the
    d_v sweep's tiles laid from each reach start) against a source grid of odd
    width and height, so that a tile's last quarter runs past the row end and
    reach intervals start off the quarter boundaries."""
    qg, sg = W.Grid(48, 40, 2, 0.05), W.Grid(131, 37, 1, 0.02)
    rng = np.random.default_rng(int(1000 * ell))
    v = rng.standard_normal(sg.n).astype(np.float32)
    xq, yg = orc.grid_points(*qg.astuple()), orc.grid_points(*sg.astuple())
    gout = rng.standard_normal(len(xq)).astype(np.float32)
    q, s = api.Points(grid=qg), api.Points(grid=sg)
    out, mom = api.gp_kernel_matvec_train(q, s, dev(v), ell, 0.9)
    ref, ab = orc.kernel_matvec(xq, yg, v, ell, 0.9)
    assert_matvec_close(host(out), ref, ab, what="train forward")
    G = api.gp_kernel_matvec_bwd(q, s, dev(v), ell, 0.9, dev(gout), want=["v", "x", "lengthscale", "variance"],
                                 moments=mom)
    R = orc.kernel_matvec_vjp(xq, yg, v, ell, 0.9, gout.astype(np.float64), False, with_abs=True)
    close(host(G["v"]), R["d_v"], R["d_v_abs"], what="d_v")
    close(host(G["x"]), R["d_x"], R["d_x_abs"], what="d_x")
    close(host(G["lengthscale"]), [R["d_len"]], [R["d_len_abs"]], what="d_len")
    close(host(G["variance"]), [R["d_var"]], [R["d_var_abs"]], what="d_var")


@pytest.mark.parametrize("n,m", [(1, 1), (700, 5003), (3001, 2500)])
def test_explicit_sources(orc, n, m):
    rng = np.random.default_rng(n + m)
    x, y = rng.uniform(-0.5, 0.5, (n, 2)).astype(np.float32), rng.uniform(-0.5, 0.5, (m, 2)).astype(np.float32)
    v, gout = rng.standard_normal(m).astype(np.float32), rng.standard_normal(n).astype(np.float32)
    q, s = api.Points(xy=dev(x)), api.Points(xy=dev(y))
    out, mom = api.gp_kernel_matvec_train(q, s, dev(v), 0.05, 1.3)
    ref, ab = orc.kernel_matvec(x, y, v, 0.05, 1.3)
    assert_matvec_close(host(out), ref, ab, what="train forward")
    want = ["v", "x", "y", "lengthscale", "variance"]
    G = api.gp_kernel_matvec_bwd(q, s, dev(v), 0.05, 1.3, dev(gout), want=want, moments=mom)
    R = orc.kernel_matvec_vjp(x, y, v, 0.05, 1.3, gout.astype(np.float64), False, with_abs=True)
    for k, rk in (("v", "d_v"), ("x", "d_x"), ("y", "d_y")):
        close(host(G[k]), R[rk], R[rk + "_abs"], what=rk)
    close(host(G["lengthscale"]), [R["d_len"]], [R["d_len_abs"]], what="d_len")
    close(host(G["variance"]), [R["d_var"]], [R["d_var_abs"]], what="d_var")


def test_fused_chain_with_moments(orc):
    """Ray-traced query (lens, shear, 200 tNFW) against grid inducing points:
    train forward, then the backward with the forward's points and moments,
    down to the lens and subhalo parameters."""
    p = W.realistic(seed=51, side=80, ss=2, n_sub=200)
    g = np.random.default_rng(3).standard_normal(p.n).astype(np.float32)
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub))
    s = api.Points(grid=p.ygrid)
    beta = torch.empty((p.n, 2), device="cuda")
    out, mom = api.gp_kernel_matvec_train(q, s, dev(p.v), p.lengthscale, p.variance, beta=beta)
    want = ["v", "x", "lengthscale", "variance", "lens", "sub"]
    G = api.gp_kernel_matvec_bwd(q, s, dev(p.v), p.lengthscale, p.variance, dev(g), want=want, beta=beta,
                                 moments=mom)
    xi, bref, yg = fused_chain(orc, p)
    ref, ab, sens = orc.kernel_matvec(bref, yg, p.v, p.lengthscale, p.variance, with_sens=True)
    delta = 1e-6 + np.spacing(np.abs(bref).max().astype(np.float32))
    assert_matvec_close(host(out), ref, ab, sens=sens, delta=delta, what="fused train forward")
    R = orc.kernel_matvec_vjp(bref, yg, p.v, p.lengthscale, p.variance, g.astype(np.float64), with_abs=True)
    delta = point_delta(bref)
    assert_close_tol(host(G["v"]), R["d_v"], chain_tol(R, "d_v", delta), what="d_v")
    assert_close_tol(host(G["x"]), R["d_x"], chain_tol(R, "d_x", delta), what="d_x")
    for k, rk in (("lengthscale", "d_len"), ("variance", "d_var")):
        assert_close_tol(host(G[k]), [R[rk]], [chain_tol(R, rk, delta)], what=rk)
    rl, rs, tl, ts = lens_chain_tols(orc, xi, p.lens.astuple(), p.sub, R, delta)
    assert_close_tol(host(G["lens"]), rl, tl, what="d_lens")
    assert_close_tol(host(G["sub"]), rs, ts, what="d_sub")


def test_deterministic_and_self_kernel_rejected():
    p = W.realistic(seed=52, side=40, ss=2, n_sub=30)
    q, s = api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub)), api.Points(grid=p.ygrid)
    g = dev(np.random.default_rng(0).standard_normal(p.n))
    a_out, a_mom = api.gp_kernel_matvec_train(q, s, dev(p.v), p.lengthscale, 1.0)
    b_out, b_mom = api.gp_kernel_matvec_train(q, s, dev(p.v), p.lengthscale, 1.0)
    assert torch.equal(a_out, b_out) and torch.equal(a_mom, b_mom)
    want = ["v", "x", "lengthscale", "variance", "lens", "sub"]
    ga = api.gp_kernel_matvec_bwd(q, s, dev(p.v), p.lengthscale, 1.0, g, want=want, moments=a_mom)
    gb = api.gp_kernel_matvec_bwd(q, s, dev(p.v), p.lengthscale, 1.0, g, want=want, moments=a_mom)
    for k in want:
        assert torch.equal(ga[k], gb[k]), k
    x = dev(np.zeros((8, 2)))
    with pytest.raises(abi.LensGPError, match="self-kernel"):
        api.gp_kernel_matvec_train(api.Points(xy=x), None, dev(np.ones(8)), 0.1, 1.0)
    with pytest.raises(abi.LensGPError, match="non-self"):
        api.gp_kernel_matvec_bwd(api.Points(xy=x), None, dev(np.ones(8)), 0.1, 1.0, dev(np.ones(8)),
                                 moments=torch.zeros((4, 8), device="cuda"))


def test_graph_capture_matches_direct_launches():
    """The training step captured into a CUDA graph (the backward forks its
    d_v branch onto a side stream) gives the bits of direct launches."""
    p = W.realistic(seed=5, side=96, ss=2, n_sub=30, ygrid_side=48)
    sub = torch.from_numpy(p.sub).cuda()
    q, s = api.Points(grid=p.xgrid, lens=p.lens, sub=sub), api.Points(grid=p.ygrid)
    v = torch.from_numpy(p.v).cuda()
    g = torch.from_numpy(np.random.default_rng(3).standard_normal(p.n).astype(np.float32)).cuda()
    want = ["v", "lengthscale", "variance", "lens", "sub"]
    out = torch.empty(p.n, dtype=torch.float32, device="cuda")
    beta = torch.empty((p.n, 2), dtype=torch.float32, device="cuda")
    mom = torch.empty((4, p.n), dtype=torch.float32, device="cuda")
    ws = torch.empty(max(api.train_workspace_size(q, s), 1), dtype=torch.uint8, device="cuda")

    def step():
        api.gp_kernel_matvec_train(q, s, v, p.lengthscale, p.variance, out=out, beta=beta, moments=mom, workspace=ws)
        return api.gp_kernel_matvec_bwd(q, s, v, p.lengthscale, p.variance, g, want=want, beta=beta, moments=mom)

    ref = {k: t.clone() for k, t in step().items()}
    ref_out = out.clone()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        G = step()
    out.zero_()
    for t in G.values():
        t.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref_out)
    for k in want:
        assert torch.equal(G[k], ref[k]), k
