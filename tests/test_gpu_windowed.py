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
