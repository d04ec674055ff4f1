"""Parity of the CUDA backward pass with the FP64 oracle's analytic
gradients: the reduction alone on explicit points, grid inducing points, the
self-kernel; the ray-trace vector-Jacobian product alone; and the whole
fused chain down to the lens and subhalo parameters."""
import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import api, workloads as W
from tests.gpu_util import (assert_close_tol, chain_tol, dev, host, lens_chain_tols, need_gpu, point_delta,
                            ulp32)

pytestmark = pytest.mark.gpu

REL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def close(got, ref, scale, rel=REL, what=""):
    got, ref, scale = (np.asarray(a, np.float64) for a in (got, ref, scale))
    tol = rel * scale + 1e-30
    err = np.abs(got - ref)
    bad = err > tol
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} outside; worst ratio {np.max(err / tol):.2f}, "
                           f"err {err.flat[np.argmax(err / tol)]:.3e} scale {scale.flat[np.argmax(err / tol)]:.3e}")


def pts(rng, n, hw):
    return rng.uniform(-hw, hw, (n, 2)).astype(np.float32)


def check_reduction(orc, x, y, v, g, ell, var, self_kernel, grid=None):
    q = api.Points(xy=dev(x))
    s = None if self_kernel else (api.Points(grid=grid) if grid is not None else api.Points(xy=dev(y)))
    want = ["v", "x", "lengthscale", "variance"] + ([] if (self_kernel or grid is not None) else ["y"])
    G = api.gp_kernel_matvec_bwd(q, s, dev(v), ell, var, dev(g), want=want)
    R = orc.kernel_matvec_vjp(x, x if self_kernel else y, v, ell, var, g.astype(np.float64), self_kernel,
                              with_abs=True)
    close(host(G["v"]), R["d_v"], R["d_v_abs"], what="d_v")
    close(host(G["x"]), R["d_x"], R["d_x_abs"], what="d_x")
    if "y" in want:
        close(host(G["y"]), R["d_y"], R["d_y_abs"], what="d_y")
    close(host(G["lengthscale"]), [R["d_len"]], [R["d_len_abs"]], what="d_len")
    close(host(G["variance"]), [R["d_var"]], [R["d_var_abs"]], what="d_var")


@pytest.mark.parametrize("n,m", [(1, 1), (33, 31), (3001, 2500), (700, 5003)])
def test_reduction_explicit(orc, n, m):
    rng = np.random.default_rng(n + 3 * m)
    x, y = pts(rng, n, 0.5), pts(rng, m, 0.5)
    check_reduction(orc, x, y, rng.standard_normal(m).astype(np.float32), rng.standard_normal(n).astype(np.float32),
                    0.05, 1.3, False)


@pytest.mark.parametrize("gw,gh", [(128, 40), (300, 7)])
def test_reduction_grid_source(orc, gw, gh):
    rng = np.random.default_rng(gw)
    g = W.Grid(gw, gh, 1, 0.04, 0.01, -0.02)
    yg = orc.grid_points(*g.astuple())
    x = pts(rng, 4099, 0.8 * max(gw, gh) * 0.04 / 2)
    check_reduction(orc, x, yg, rng.standard_normal(g.n).astype(np.float32),
                    rng.standard_normal(4099).astype(np.float32), 0.053, 0.7, False, grid=g)


@pytest.mark.parametrize("ratio", [0.5, 1.2, 1.25, 1.5, 4.0])
def test_reduction_grid_lengthscale_to_spacing(orc, ratio):
    """Both forms of the grid path (split exponent from 1.24 grid spacings up)."""
    rng = np.random.default_rng(int(ratio * 10))
    g = W.Grid(260, 30, 1, 0.04)
    yg = orc.grid_points(*g.astuple())
    x = np.stack([rng.uniform(-5.6, 5.6, 2999), rng.uniform(-0.7, 0.7, 2999)], -1).astype(np.float32)
    check_reduction(orc, x, yg, rng.standard_normal(g.n).astype(np.float32),
                    rng.standard_normal(2999).astype(np.float32), ratio * 0.04, 0.8, False, grid=g)


def test_reduction_self_kernel(orc):
    rng = np.random.default_rng(5)
    x = pts(rng, 6000, 1.0)
    check_reduction(orc, x, x, rng.standard_normal(6000).astype(np.float32),
                    rng.standard_normal(6000).astype(np.float32), 0.05, 1.1, True)


@pytest.mark.parametrize("profile", [0, 1])
def test_raytrace_vjp(orc, profile):
    rng = np.random.default_rng(40 + profile)
    p = W.realistic(seed=41, side=60, ss=2, n_sub=150)
    sub = p.sub.copy()
    if profile == 1:
        sub[:, 2] = rng.uniform(0.01, 0.05, len(sub))
    xi = orc.grid_points(*p.xgrid.astuple())
    db = rng.standard_normal((p.n, 2)).astype(np.float32)
    d_lens, d_sub = api.lens_raytrace_vjp(api.Points(grid=p.xgrid, lens=p.lens, sub=dev(sub), profile=profile),
                                          dev(db))
    rl, rs, al, asub = orc.raytrace_vjp(xi, p.lens.astuple(), sub, db, profile, with_abs=True)
    close(host(d_lens), rl, al, what="d_lens")
    close(host(d_sub), rs, asub, what="d_sub")


@pytest.mark.parametrize("n_sub", [3, 4097])
def test_raytrace_vjp_subhalo_counts(orc, n_sub):
    """A few subhalos (several phases per subhalo) and more subhalos than a
    CTA orders by class (every slot in index order): the far-field series,
    the local expansion and the closed forms serve the sums, every gradient
    element against the oracle."""
    rng = np.random.default_rng(44)
    lens = W.draw_lens(rng)
    sub = W.draw_subhalos(rng, n_sub, lens, 1e6, 1e10)
    g = W.Grid(24, 24, 2, 0.1)
    xi = orc.grid_points(*g.astuple())
    db = rng.standard_normal((g.n, 2)).astype(np.float32)
    d_lens, d_sub = api.lens_raytrace_vjp(api.Points(grid=g, lens=lens, sub=dev(sub)), dev(db))
    rl, rs, al, asub = orc.raytrace_vjp(xi, lens.astuple(), sub, db, 0, with_abs=True)
    close(host(d_lens), rl, al, what="d_lens")
    close(host(d_sub), rs, asub, what="d_sub")


@pytest.mark.parametrize("name", ["hoags_object", "ngc4414"])
def test_raytrace_vjp_printed_lenses(orc, name):
    from tests.golden.lenses import paper_lenses
    L = W.Lens(*[float(np.float32(v)) for v in paper_lenses()[name].values()])
    g = W.Grid(48, 48, 2, 0.05, 0.0125, 0.0125)
    xi = orc.grid_points(*g.astuple())
    db = np.random.default_rng(7).standard_normal((g.n, 2)).astype(np.float32)
    d_lens, _ = api.lens_raytrace_vjp(api.Points(grid=g, lens=L), dev(db))
    rl, _, al, _ = orc.raytrace_vjp(xi, L.astuple(), None, db, 0, with_abs=True)
    close(host(d_lens), rl, al, what="d_lens")


def fused_chain(orc, p, rows=None):
    """Oracle gradients of sum_i g_i out_i through ray-trace + reduction."""
    xi = orc.grid_points(*p.xgrid.astuple())
    _, bref = orc.raytrace(xi, p.lens.astuple(), p.sub)
    yg = orc.grid_points(*p.ygrid.astuple())
    return xi, bref, yg


def test_fused_chain_reduced_differentiation_config(orc):
    """Differentiation workload recipe (power-law lens + shear + 200 tNFW,
    grid inducing points) at 80x80x2x2: every gradient against the oracle chain."""
    p = W.realistic(seed=51, side=80, ss=2, n_sub=200)
    rng = np.random.default_rng(3)
    g = rng.standard_normal(p.n).astype(np.float32)
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub))
    G = api.gp_kernel_matvec_bwd(q, api.Points(grid=p.ygrid), dev(p.v), p.lengthscale, p.variance, dev(g),
                                 want=["v", "x", "lengthscale", "variance", "lens", "sub"])
    xi, bref, yg = fused_chain(orc, p)
    R = orc.kernel_matvec_vjp(bref, yg, p.v, p.lengthscale, p.variance, g.astype(np.float64), with_abs=True)
    # the GPU's ray-traced points differ from the oracle's by at most delta per
    # coordinate; each gradient may move by 2 sqrt(2) delta times its
    # input-error sensitivity on top of the 2e-5 arithmetic bound
    delta = point_delta(bref)
    for k, rk in (("v", "d_v"), ("x", "d_x")):
        assert_close_tol(host(G[k]), R[rk], chain_tol(R, rk, delta), what=rk)
    for k, rk in (("lengthscale", "d_len"), ("variance", "d_var")):
        assert_close_tol(host(G[k]), [R[rk]], [chain_tol(R, rk, delta)], what=rk)
    rl, rs, tl, ts = lens_chain_tols(orc, xi, p.lens.astuple(), p.sub, R, delta)
    assert_close_tol(host(G["lens"]), rl, tl, what="d_lens")
    assert_close_tol(host(G["sub"]), rs, ts, what="d_sub")


def test_deterministic(orc):
    p = W.realistic(seed=52, side=40, ss=2, n_sub=30)
    g = dev(np.random.default_rng(0).standard_normal(p.n))
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub))
    want = ["v", "x", "lengthscale", "variance", "lens", "sub"]
    a = api.gp_kernel_matvec_bwd(q, api.Points(grid=p.ygrid), dev(p.v), p.lengthscale, 1.0, g, want=want)
    b = api.gp_kernel_matvec_bwd(q, api.Points(grid=p.ygrid), dev(p.v), p.lengthscale, 1.0, g, want=want)
    for k in want:
        assert torch.equal(a[k], b[k]), k


def test_empty_sets_give_zero_gradients():
    x = dev(np.zeros((5, 2)))
    e = torch.empty((0, 2), device="cuda")
    G = api.gp_kernel_matvec_bwd(api.Points(xy=x), api.Points(xy=e), torch.empty(0, device="cuda"), 0.1, 1.0,
                                 dev(np.ones(5)), want=["x", "lengthscale", "variance"])
    assert torch.all(G["x"] == 0) and G["lengthscale"].item() == 0 and G["variance"].item() == 0


def test_full_size_differentiation_system_sampled(orc):
    """One lens system of the differentiation workload at full size (200x200
    at 2x2 = 160k points, 200 subhalos, 16384 grid inducing points): every
    gradient against the oracle's full FP64 chain on its own ray-traced
    points, within 2e-5 of the absolute terms plus the derived input-error
    term."""
    p = W.diff_batch(batch=1)[0]
    rng = np.random.default_rng(9)
    g = rng.standard_normal(p.n).astype(np.float32)
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub))
    G = api.gp_kernel_matvec_bwd(q, api.Points(grid=p.ygrid), dev(p.v), p.lengthscale, p.variance, dev(g),
                                 want=["v", "x", "lengthscale", "variance", "lens", "sub"])
    xi, bref, yg = fused_chain(orc, p)
    R = orc.kernel_matvec_vjp(bref, yg, p.v, p.lengthscale, p.variance, g.astype(np.float64), with_abs=True)
    delta = point_delta(bref)
    assert_close_tol(host(G["v"]), R["d_v"], chain_tol(R, "d_v", delta), what="d_v")
    assert_close_tol(host(G["x"]), R["d_x"], chain_tol(R, "d_x", delta), what="d_x")
    for k, rk in (("lengthscale", "d_len"), ("variance", "d_var")):
        assert_close_tol(host(G[k]), [R[rk]], [chain_tol(R, rk, delta)], what=rk)
    rl, rs, tl, ts = lens_chain_tols(orc, xi, p.lens.astuple(), p.sub, R, delta)
    assert_close_tol(host(G["lens"]), rl, tl, what="d_lens")
    assert_close_tol(host(G["sub"]), rs, ts, what="d_sub")
