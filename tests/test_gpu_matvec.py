"""Parity of the CUDA kernel reduction with the FP64 oracle, on explicit
points, grid inducing points, the self-kernel and the fused ray-trace path."""
import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import api, workloads as W
from tests.gpu_util import assert_matvec_close, dev, host, need_gpu, ulp32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def pts(rng, n, hw):
    return rng.uniform(-hw, hw, (n, 2)).astype(np.float32)


@pytest.mark.parametrize("n,m", [(1, 1), (31, 33), (127, 129), (1000, 257), (3001, 2500), (5000, 7001)])
def test_explicit_points(orc, n, m):
    rng = np.random.default_rng(n * 7 + m)
    x, y = pts(rng, n, 0.6), pts(rng, m, 0.6)
    v = rng.standard_normal(m).astype(np.float32)
    got = host(api.gp_kernel_matvec(api.Points(xy=dev(x)), api.Points(xy=dev(y)), dev(v), 0.05, 1.3))
    ref, ab = orc.kernel_matvec(x, y, v, 0.05, 1.3)
    assert_matvec_close(got, ref, ab)


@pytest.mark.parametrize("gw,gh", [(128, 128), (100, 37), (300, 5), (1, 64)])
def test_grid_source(orc, gw, gh):
    rng = np.random.default_rng(gw + gh)
    g = W.Grid(gw, gh, 1, 0.04, 0.01, -0.02)
    yg = orc.grid_points(*g.astuple())
    x = pts(rng, 4099, 0.8 * max(gw, gh) * 0.04 / 2)
    v = rng.standard_normal(g.n).astype(np.float32)
    got = host(api.gp_kernel_matvec(api.Points(xy=dev(x)), api.Points(grid=g), dev(v), 0.053, 0.7))
    ref, ab = orc.kernel_matvec(x, yg, v, 0.053, 0.7)
    assert_matvec_close(got, ref, ab)


@pytest.mark.parametrize("ratio", [0.3, 0.9, 1.2, 1.25, 1.5, 4.0])
def test_grid_source_lengthscale_to_spacing(orc, ratio):
    """Length scales below and above 1.24 grid spacings: the grid path splits
    the exponent only above that (both forms are covered)."""
    rng = np.random.default_rng(int(ratio * 100))
    g = W.Grid(300, 40, 1, 0.04, 0.0, 0.0)
    yg = orc.grid_points(*g.astuple())
    x = np.stack([rng.uniform(-6.5, 6.5, 3001), rng.uniform(-0.9, 0.9, 3001)], -1).astype(np.float32)
    v = rng.standard_normal(g.n).astype(np.float32)
    ell = ratio * 0.04
    got = host(api.gp_kernel_matvec(api.Points(xy=dev(x)), api.Points(grid=g), dev(v), ell, 0.9))
    ref, ab = orc.kernel_matvec(x, yg, v, ell, 0.9)
    assert_matvec_close(got, ref, ab)


def test_self_kernel_explicit(orc):
    rng = np.random.default_rng(3)
    x = pts(rng, 6000, 1.0)
    v = rng.standard_normal(6000).astype(np.float32)
    got = host(api.gp_kernel_matvec(api.Points(xy=dev(x)), None, dev(v), 0.05, 1.0))
    ref, ab = orc.kernel_matvec(x, x, v, 0.05, 1.0)
    assert_matvec_close(got, ref, ab)


def test_tiny_config_fused(orc):
    """100x100 SIE + shear, self-kernel l = 0.05 over the ray-traced points (1e8 pairs), end to end."""
    p = W.tiny()
    got, beta = api.gp_kernel_matvec(api.Points(grid=p.xgrid, lens=p.lens), None, dev(p.v), p.lengthscale,
                                     p.variance, want_beta=True)
    xi = orc.grid_points(*p.xgrid.astuple())
    _, bref = orc.raytrace(xi, p.lens.astuple())
    ref, ab, sens = orc.kernel_matvec(bref, bref, p.v, p.lengthscale, p.variance, with_sens=True)
    delta = 1e-6 + ulp32(bref).max()
    assert_matvec_close(host(got), ref, ab, sens, delta, what="fused self-kernel")
    # reduction alone, on the oracle's beta rounded to FP32
    b32 = bref.astype(np.float32)
    got2 = host(api.gp_kernel_matvec(api.Points(xy=dev(b32)), None, dev(p.v), p.lengthscale, p.variance))
    ref2, ab2 = orc.kernel_matvec(b32, b32, p.v, p.lengthscale, p.variance)
    assert_matvec_close(got2, ref2, ab2, what="self-kernel reduction")


def test_realistic_recipe_fused_reduced_size(orc):
    p = W.realistic(seed=21, side=100, ss=2, n_sub=200)
    got, beta = api.gp_kernel_matvec(api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub)),
                                     api.Points(grid=p.ygrid), dev(p.v), p.lengthscale, p.variance, want_beta=True)
    xi = orc.grid_points(*p.xgrid.astuple())
    _, bref = orc.raytrace(xi, p.lens.astuple(), p.sub)
    yg = orc.grid_points(*p.ygrid.astuple())
    ref, ab, sens = orc.kernel_matvec(bref, yg, p.v, p.lengthscale, p.variance, with_sens=True)
    assert_matvec_close(host(got), ref, ab, sens, 1e-6 + ulp32(bref).max(), what="fused grid")


def test_full_size_realistic_sampled_rows(orc):
    """640k ray-traced points x 16384 grid inducing points, 200 subhalos: the
    benchmark's launch configuration; 1500 sampled rows against the oracle."""
    p = W.realistic()
    got = host(api.gp_kernel_matvec(api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub)),
                                    api.Points(grid=p.ygrid), dev(p.v), p.lengthscale, p.variance))
    rows = np.random.default_rng(1).choice(p.n, 1500, replace=False)
    xi = orc.grid_points(*p.xgrid.astuple())[rows]
    _, bref = orc.raytrace(xi, p.lens.astuple(), p.sub)
    yg = orc.grid_points(*p.ygrid.astuple())
    ref, ab, sens = orc.kernel_matvec(bref, yg, p.v, p.lengthscale, p.variance, with_sens=True)
    assert_matvec_close(got[rows], ref, ab, sens, 1e-6 + ulp32(bref).max(), what="realistic sampled")


def test_full_size_large_self_kernel_sampled_rows(orc):
    """2.56M-point self-kernel (6.55e12 pairs) on seeded points with the large
    workload's extent and density; 400 sampled rows against the oracle."""
    rng = np.random.default_rng(44)
    n = 1600 * 1600
    x = pts(rng, n, 20.0)
    v = rng.standard_normal(n).astype(np.float32)
    got = host(api.gp_kernel_matvec(api.Points(xy=dev(x)), None, dev(v), 0.05, 1.0))
    rows = rng.choice(n, 400, replace=False)
    ref, ab = orc.kernel_matvec(x, x, v, 0.05, 1.0, rows=rows)
    assert_matvec_close(got[rows], ref, ab, what="large self-kernel sampled")


def test_edge_cases(orc):
    rng = np.random.default_rng(2)
    x = pts(rng, 10, 0.1)
    # m = 0: zeros
    out = host(api.gp_kernel_matvec(api.Points(xy=dev(x)), api.Points(xy=torch.empty((0, 2), device="cuda")),
                                    torch.empty(0, device="cuda"), 0.1))
    assert np.all(out == 0)
    # n = 0: empty
    out = api.gp_kernel_matvec(api.Points(xy=torch.empty((0, 2), device="cuda")), api.Points(xy=dev(x)),
                               dev(np.ones(10)), 0.1)
    assert out.shape == (0,)
    # far-apart points: every contribution underflows; exact zeros
    far = np.array([[1000.0, 1000.0]], np.float32)
    out = host(api.gp_kernel_matvec(api.Points(xy=dev(far)), api.Points(xy=dev(x)), dev(np.ones(10)), 0.01))
    assert out[0] == 0.0
    # coincident points: k = variance exactly
    out = host(api.gp_kernel_matvec(api.Points(xy=dev(x[:1])), api.Points(xy=dev(x[:1])), dev(np.ones(1)), 0.1, 2.5))
    assert out[0] == np.float32(2.5)


def test_deterministic_and_stream_ordered(orc):
    rng = np.random.default_rng(4)
    x, v = pts(rng, 20000, 1.0), rng.standard_normal(20000).astype(np.float32)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = api.gp_kernel_matvec(api.Points(xy=dev(x)), None, dev(v), 0.05)
        b = api.gp_kernel_matvec(api.Points(xy=dev(x)), None, dev(v), 0.05)
    s.synchronize()
    np.testing.assert_array_equal(host(a), host(b))


def test_no_fault_recorded():
    assert api.fault_status() == 0


def test_evaluated_pairs_bounds():
    """The grid kernels leave out only pairs beyond the exact-zero radius: none
    for a length scale as large as the field, most for the realistic one."""
    p = W.realistic(seed=3, side=80, ss=2, n_sub=0)
    beta = api.lens_raytrace(api.Points(grid=p.xgrid, lens=p.lens))
    full = p.n * p.m
    assert api.grid_pairs_evaluated(beta, p.xgrid, p.ygrid, 100.0, 1024) == full
    some = api.grid_pairs_evaluated(beta, p.xgrid, p.ygrid, p.lengthscale, 1024)
    assert 0 < some < full
    # explicit order (no layout) evaluates at least as many pairs as image tiles
    assert api.grid_pairs_evaluated(beta, None, p.ygrid, p.lengthscale, 1024) >= some


def test_grid_source_with_image_layout(orc):
    """Explicit ray-traced pixels that carry their image grid (row blocks in
    image tiles, pairs beyond the exact-zero radius left out) against the oracle."""
    p = W.realistic(seed=5, side=64, ss=2, n_sub=10)
    # the oracle's ray-traced points, rounded to FP32, feed both sides
    _, bref = orc.raytrace(orc.grid_points(*p.xgrid.astuple()), p.lens.astuple(), p.sub)
    b = bref.astype(np.float32)
    yg = orc.grid_points(*p.ygrid.astuple())
    got = host(api.gp_kernel_matvec(api.Points(xy=dev(b), grid=p.xgrid), api.Points(grid=p.ygrid), dev(p.v),
                                    p.lengthscale, p.variance))
    ref, ab = orc.kernel_matvec(b, yg, p.v, p.lengthscale, p.variance)
    assert_matvec_close(got, ref, ab, what="grid source, image layout")
