"""Parity of the CUDA pixel windows and windowed transmission reduction with
the FP64 oracle, on a lensed pixel grid like the paper's image-plane model."""
import numpy as np
import pytest

from paper_2105_09465_gb300 import api, workloads as W
from tests.gpu_util import assert_matvec_close, dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def lensed_grid(orc, side=60, pix=0.05, seed=3):
    rng = np.random.default_rng(seed)
    lens = W.draw_lens(rng)
    g = W.Grid(side, side, 1, pix)
    _, b = orc.raytrace(orc.grid_points(*g.astuple()), lens.astuple())
    return g, b.astype(np.float32)


def test_pixel_shapes(orc):
    g, b = lensed_grid(orc)
    z = host(api.pixel_shapes(dev(b), g.nx, g.ny))
    zr = orc.pixel_shapes(b, g.nx, g.ny)
    scale = np.abs(zr).max(axis=1, keepdims=True)
    assert np.all(np.abs(z - zr) <= 1e-5 * scale + 1e-12), float(np.max(np.abs(z - zr) / scale))


@pytest.mark.parametrize("source", ["grid", "explicit", "self"])
def test_windowed_transmission(orc, source):
    g, b = lensed_grid(orc, side=70)
    zr = orc.pixel_shapes(b, g.nx, g.ny).astype(np.float32)  # oracle windows feed both sides
    rng = np.random.default_rng(4)
    ell = 0.05
    if source == "grid":
        yg = W.Grid(40, 40, 1, 0.1)
        q = orc.grid_points(*yg.astuple())
        src = api.Points(grid=yg)
    elif source == "explicit":
        q = rng.uniform(-2, 2, (3000, 2)).astype(np.float32)
        src = api.Points(xy=dev(q))
    else:
        q = b
        src = api.Points(xy=dev(b))
    v = rng.standard_normal(len(q)).astype(np.float32)
    got = host(api.gp_windowed_matvec(dev(b), dev(zr), src, dev(v), ell))
    ref, ab = orc.windowed_matvec(b, zr, q, v, ell)
    assert_matvec_close(got, ref, ab, what=f"windowed ({source})")


def test_zero_windows_reduce_to_the_point_kernel():
    rng = np.random.default_rng(5)
    x = rng.uniform(-0.5, 0.5, (2000, 2)).astype(np.float32)
    v = rng.standard_normal(2000).astype(np.float32)
    z = np.zeros((2000, 3), np.float32)
    a = host(api.gp_windowed_matvec(dev(x), dev(z), api.Points(xy=dev(x)), dev(v), 0.08))
    b = host(api.gp_kernel_matvec(api.Points(xy=dev(x)), None, dev(v), 0.08 / np.sqrt(2.0), 1.0 / (np.pi * 0.0064)))
    np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-5 * np.abs(b).max())


def test_windowed_grid_realistic_scales(orc):
    """Pixel windows of a lensed 120 x 120 image at the realistic pixel size
    (0.05 arcsec) against a 128 x 128 source grid over the field padded by 20 %,
    length scale 4/3 of its spacing: the grid path's completed square at the
    workload's coordinate magnitudes."""
    p = W.realistic(seed=11, side=120, ss=1, n_sub=0)
    g = p.xgrid
    _, b = orc.raytrace(orc.grid_points(*g.astuple()), p.lens.astuple())
    b = b.astype(np.float32)
    zr = orc.pixel_shapes(b, g.nx, g.ny).astype(np.float32)
    yg = p.ygrid
    q = orc.grid_points(*yg.astuple())
    v = np.random.default_rng(12).standard_normal(len(q)).astype(np.float32)
    got = host(api.gp_windowed_matvec(dev(b), dev(zr), api.Points(grid=yg), dev(v), p.lengthscale))
    ref, ab = orc.windowed_matvec(b, zr, q, v, p.lengthscale)
    assert_matvec_close(got, ref, ab, what="windowed (realistic grid)")


def _close(got, ref, scale, rel, what):
    got, ref, scale = (np.asarray(a, np.float64) for a in (got, ref, scale))
    bad = np.abs(got - ref) > rel * scale + 1e-30
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(got - ref) / (scale + 1e-300))))


@pytest.mark.parametrize("self_points", [False, True])
def test_windowed_backward(orc, self_points):
    """Every gradient of sum_i g_i out_i against the FP64 oracle, on a lensed
    pixel grid with its windows; sources explicit or the pixels themselves
    (the image-plane layer)."""
    g_, b = lensed_grid(orc, side=50)
    zr = orc.pixel_shapes(b, g_.nx, g_.ny).astype(np.float32)
    rng = np.random.default_rng(21)
    q = b if self_points else rng.uniform(-1.2, 1.2, (2000, 2)).astype(np.float32)
    v = rng.standard_normal(len(q)).astype(np.float32)
    gout = rng.standard_normal(len(b)).astype(np.float32)
    ell = 0.05
    G = api.gp_windowed_matvec_bwd(dev(b), dev(zr), api.Points(xy=dev(q)), dev(v), ell, dev(gout))
    R = orc.windowed_vjp(b, zr, q, v, ell, gout, with_abs=True)
    rel = 2e-5  # of the sum of |terms|, the reduction tolerance
    _close(host(G["v"]), R["d_v"], R["d_v_abs"], rel, "d_v")
    _close(host(G["p"]), R["d_p"], R["d_p_abs"], rel, "d_p")
    _close(host(G["q"]), R["d_q"], R["d_q_abs"], rel, "d_q")
    _close(host(G["z"]), R["d_z"], R["d_z_abs"], rel, "d_z")
    _close(host(G["lengthscale"]), [R["d_len"]], [R["d_len_abs"]], rel, "d_len")


def test_pixel_shapes_vjp(orc):
    g_, b = lensed_grid(orc, side=40)
    dz = np.random.default_rng(22).standard_normal((len(b), 3)).astype(np.float32)
    got = host(api.pixel_shapes_vjp(dev(b), g_.nx, g_.ny, dev(dz)))
    ref = orc.pixel_shapes_vjp(b, g_.nx, g_.ny, dz)
    np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-5 * np.abs(ref).max())
