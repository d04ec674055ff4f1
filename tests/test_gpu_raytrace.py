"""Parity of the CUDA ray-trace with the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import api, workloads as W
from tests.golden.lenses import paper_lenses
from tests.gpu_util import ALPHA_TOL, dev, host, need_gpu, ulp32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def run_both(orc, grid, lens, sub, profile=0, sub_offset=0):
    """GPU (alpha, beta) and oracle (alpha, beta) on the grid's FP32 points."""
    xi = orc.grid_points(*grid.astuple())
    if sub is not None and len(sub):
        # optional misalignment: place the records at an offset inside a larger buffer
        buf = np.zeros((len(sub) + sub_offset, 5), np.float32)
        buf[sub_offset:] = sub
        tb = dev(buf.reshape(-1))
        tsub = tb[5 * sub_offset:].view(-1, 5)
    else:
        tsub = None
    beta, alpha = api.lens_raytrace(api.Points(grid=grid, lens=lens, sub=tsub, profile=profile), want_alpha=True)
    a_ref, b_ref = orc.raytrace(xi, lens.astuple(), sub, profile)
    return host(alpha), host(beta), a_ref, b_ref, xi


def check(a, b, a_ref, b_ref, tol=ALPHA_TOL, ulps=0):
    """|alpha - alpha_ref| <= max(tol, ulps * ulp32(|alpha_ref|)) per component;
    beta additionally carries its own FP32 rounding."""
    lim = np.maximum(tol, ulps * ulp32(a_ref))
    da = np.abs(a - a_ref)
    assert np.all(da <= lim), f"max |alpha - alpha_ref| = {da.max():.3e} (excess ratio {(da / lim).max():.2f})"
    db = np.abs(b - b_ref)
    assert np.all(db <= lim + ulp32(b_ref)), f"max |beta - beta_ref| = {db.max():.3e}"
    return da.max()


def test_grid_points_bit_exact(orc):
    g = W.Grid(37, 23, 3, 0.05, 0.013, -0.021)
    out, beta = api.gp_kernel_matvec(api.Points(grid=g), api.Points(grid=W.Grid(4, 4, 1, 0.1)),
                                     dev(np.ones(16)), 0.1, want_beta=True)
    np.testing.assert_array_equal(host(beta).astype(np.float32), orc.grid_points(*g.astuple()))


def test_sie_plus_shear_tiny_config(orc):
    p = W.tiny()
    a, b, ar, br, _ = run_both(orc, p.xgrid, p.lens, None)
    check(a, b, ar, br)


@pytest.mark.parametrize("name", sorted(paper_lenses()))
def test_printed_lenses(orc, name):
    """The paper's printed lenses reach slopes of 2.48, where |alpha| grows to
    several arcsec next to the centre; there the bound is 4 FP32 ulps of
    |alpha| (1e-6 arcsec is below FP32 resolution for |alpha| > 8)."""
    L = W.Lens(*[float(np.float32(v)) for v in paper_lenses()[name].values()])
    a, b, ar, br, _ = run_both(orc, W.Grid(64, 64, 2, 0.05, 0.01, -0.02), L, None)
    check(a, b, ar, br, ulps=4)


@pytest.mark.parametrize("n_sub,offset", [(1, 0), (203, 0), (256, 0), (300, 1), (517, 3)])
def test_tnfw_subhalos(orc, n_sub, offset):
    rng = np.random.default_rng(n_sub)
    lens = W.draw_lens(rng)
    sub = W.draw_subhalos(rng, n_sub, lens, 1e7, 1e10)
    g = W.Grid(61, 53, 2, 0.05)  # ragged point count (12932)
    a, b, ar, br, _ = run_both(orc, g, lens, sub, 0, offset)
    check(a, b, ar, br)


def test_subhalo_centred_on_pixels_and_near_x_equals_one(orc):
    """Subhalos on pixel centres (R = 0), and pixels at R ~ theta_s (the x = 1 branch point)."""
    g = W.Grid(40, 40, 1, 0.05)
    xi = orc.grid_points(*g.astuple()).astype(np.float64)
    lens = W.Lens(0.0, 0.0, 0.8, 0.3, 1.2, 2.0, 0.01, 0.0)
    sub = np.array([[xi[820, 0], xi[820, 1], 0.02, 0.1, 10.0],   # exactly on a pixel
                    [0.3, 0.2, 0.015, 0.05 * math.sqrt(2.0), 4.0],  # theta_s = diagonal pixel offset
                    [-0.4, 0.1, 0.01, 0.05, 25.0]], np.float32)
    a, b, ar, br, _ = run_both(orc, g, lens, sub)
    check(a, b, ar, br)


@pytest.mark.parametrize("tau", [0.7, 3.0, 10.0, 40.0])
def test_tnfw_far_field_series_boundary(orc, tau):
    """Pixels on both sides of the far-field series radius x = 6 max(tau, 2)
    of heavy subhalos (the kernels switch from the closed form to the series
    there; both must match the FP64 closed form), in tiles that are entirely
    inside, entirely outside and across the radius."""
    theta_s = 0.08
    xT = 6 * max(tau, 2) * theta_s
    g = W.Grid(96, 96, 2, 2.2 * xT / 96)
    # one subhalo at the grid centre and three at the edges, with the
    # realistic-size normalisation kappa_s of a 1e10 Msun halo
    pos = [(0.0, 0.0), (0.9 * g.nx * g.pix / 2, 0.0), (0.0, -0.8 * g.ny * g.pix / 2), (0.31 * xT, 0.44 * xT)]
    sub = np.array([[x, y, 0.05, theta_s, tau] for x, y in pos], np.float32)
    lens = W.Lens(0.0, 0.0, 0.8, 0.3, 1.2, 2.0, 0.01, 0.02)
    a, b, ar, br, _ = run_both(orc, g, lens, sub)
    check(a, b, ar, br)


def test_point_mass_profile(orc):
    rng = np.random.default_rng(5)
    lens = W.draw_lens(rng)
    sub = np.stack([rng.uniform(-1, 1, 40), rng.uniform(-1, 1, 40), rng.uniform(0.01, 0.05, 40),
                    np.zeros(40), np.zeros(40)], 1).astype(np.float32)
    a, b, ar, br, _ = run_both(orc, W.Grid(50, 50, 2, 0.05, 0.0125, 0.0125), lens, sub, profile=1)
    check(a, b, ar, br)


def test_realistic_recipe_reduced_size(orc):
    p = W.realistic(seed=11, side=80, ss=2, n_sub=200)
    a, b, ar, br, _ = run_both(orc, p.xgrid, p.lens, p.sub)
    check(a, b, ar, br)


def test_explicit_points_and_edge_sizes(orc):
    rng = np.random.default_rng(9)
    lens = W.draw_lens(rng)
    sub = W.draw_subhalos(rng, 17, lens, 1e7, 1e10)
    for n in [1, 31, 33, 255, 257]:
        xi = rng.uniform(-3, 3, (n, 2)).astype(np.float32)
        beta, alpha = api.lens_raytrace(api.Points(xy=dev(xi), lens=lens, sub=dev(sub)), want_alpha=True)
        ar, br = orc.raytrace(xi, lens.astuple(), sub)
        check(host(alpha), host(beta), ar, br)


def test_empty_input_is_a_noop():
    lens = W.Lens(0, 0, 0.8, 0.1, 1.2, 2.0, 0, 0)
    beta = api.lens_raytrace(api.Points(xy=torch.empty((0, 2), device="cuda"), lens=lens))
    assert beta.shape == (0, 2)


def test_deterministic(orc):
    p = W.realistic(seed=12, side=40, ss=2, n_sub=50)
    pts = api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub))
    b1 = host(api.lens_raytrace(pts))
    b2 = host(api.lens_raytrace(pts))
    np.testing.assert_array_equal(b1, b2)


def test_full_size_sampled_rows_large(orc):
    """800x800 at 2x2 (2.56M points) with 2000 subhalos, in the launch
    configuration of the benchmark; 2000 sampled pixels against the oracle."""
    p = W.large()
    beta, alpha = api.lens_raytrace(api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub)), want_alpha=True)
    rows = np.random.default_rng(0).choice(p.n, 2000, replace=False)
    xi = orc.grid_points(*p.xgrid.astuple())[rows]
    ar, br = orc.raytrace(xi, p.lens.astuple(), p.sub)
    check(host(alpha)[rows], host(beta)[rows], ar, br)
