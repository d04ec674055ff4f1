"""Parity of the multi-layer reduction with the oracle's sum of layers, on
the paper's printed three-layer image-plane configuration and on grid sources."""
from pathlib import Path

import numpy as np
import pytest

from paper_2105_09465_gb300 import api, workloads as W
from tests.gpu_util import assert_matvec_close, dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def paper_layers():
    rows = [l.split() for l in (Path(__file__).parent / "golden" / "paper_layers.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    return {r[0]: (float(r[1]), float(r[2])) for r in rows}


def oracle_layers(orc, x, y, v, ls, vs):
    out = np.zeros(len(x))
    ab = np.zeros(len(x))
    for l in range(len(ls)):
        o, a = orc.kernel_matvec(x, y, v[l], float(np.float32(ls[l])), float(np.float32(vs[l])))
        out += o
        ab += np.abs(a)
    return out, ab


def test_paper_three_image_plane_layers_self_kernel(orc):
    """12.5 mas pixels ray-traced through a Hoag-like lens; the three printed layers."""
    P = paper_layers()
    ls = [P[k][0] for k in ("image0", "image1", "image2")]
    vs = [P[k][1] ** 2 for k in ("image0", "image1", "image2")]
    g = W.Grid(120, 100, 1, 0.0125)
    lens = W.Lens(-0.0704, -0.0193, 0.2753, 1.742, 1.1847, 2.2193, -0.0227, 0.0047)
    lens = W.Lens(*[float(np.float32(t)) for t in lens.astuple()])
    rng = np.random.default_rng(12)
    v = rng.standard_normal((3, g.n)).astype(np.float32)
    # the oracle's ray-traced points, rounded to FP32, feed both sides
    _, bref = orc.raytrace(orc.grid_points(*g.astuple()), lens.astuple())
    b = bref.astype(np.float32)
    out = api.gp_kernel_matvec_layers(api.Points(xy=dev(b)), None, dev(v), ls, vs)
    ref, ab = oracle_layers(orc, b, b, v, ls, vs)
    assert_matvec_close(host(out), ref, ab, what="3-layer self-kernel")


@pytest.mark.parametrize("L", [1, 2, 4])
def test_grid_and_explicit_sources(orc, L):
    rng = np.random.default_rng(L)
    g = W.Grid(70, 50, 1, 0.03)
    yg = orc.grid_points(*g.astuple())
    x = rng.uniform(-1.0, 1.0, (3001, 2)).astype(np.float32)
    v = rng.standard_normal((L, g.n)).astype(np.float32)
    ls = list(np.float32(0.05 * 1.7 ** np.arange(L)))
    vs = list(np.float32(1.0 + 0.3 * np.arange(L)))
    ref, ab = oracle_layers(orc, x, yg, v, ls, vs)
    got = host(api.gp_kernel_matvec_layers(api.Points(xy=dev(x)), api.Points(grid=g), dev(v), ls, vs))
    assert_matvec_close(got, ref, ab, what=f"{L} layers, grid")
    got = host(api.gp_kernel_matvec_layers(api.Points(xy=dev(x)), api.Points(xy=dev(yg)), dev(v), ls, vs))
    assert_matvec_close(got, ref, ab, what=f"{L} layers, explicit")


def test_one_layer_matches_single_layer_entry_point():
    rng = np.random.default_rng(5)
    x = rng.uniform(-0.5, 0.5, (2000, 2)).astype(np.float32)
    v = rng.standard_normal(2000).astype(np.float32)
    a = host(api.gp_kernel_matvec_layers(api.Points(xy=dev(x)), None, dev(v[None, :]), [0.04], [1.3]))
    b = host(api.gp_kernel_matvec(api.Points(xy=dev(x)), None, dev(v), 0.04, 1.3))
    np.testing.assert_allclose(a, b, rtol=3e-6, atol=1e-6 * np.abs(b).max())


@pytest.mark.parametrize("L,nrhs", [(1, 2), (3, 4), (4, 3), (2, 4)])
@pytest.mark.parametrize("source", ["grid", "explicit", "self"])
def test_several_right_hand_sides(orc, L, nrhs, source):
    """v of shape (L, m, nrhs): every column of out against the oracle's sum
    of layers for that column (one exp2 per pair and layer serves all the
    right-hand sides); ragged sizes that leave partial tiles and row blocks."""
    rng = np.random.default_rng(10 * L + nrhs)
    g = W.Grid(61, 37, 1, 0.035)
    yg = orc.grid_points(*g.astuple())
    x = rng.uniform(-1.0, 1.0, (2777, 2)).astype(np.float32)
    src = {"grid": api.Points(grid=g), "explicit": api.Points(xy=dev(yg)), "self": None}[source]
    y = x if source == "self" else yg
    v = rng.standard_normal((L, len(y), nrhs)).astype(np.float32)
    ls = list(np.float32(0.04 * 1.6 ** np.arange(L)))
    vs = list(np.float32(1.0 + 0.25 * np.arange(L)))
    got = host(api.gp_kernel_matvec_layers(api.Points(xy=dev(x)), src, dev(v), ls, vs))
    assert got.shape == (len(x), nrhs)
    for h in range(nrhs):
        ref, ab = oracle_layers(orc, x, y, np.ascontiguousarray(v[:, :, h]), ls, vs)
        assert_matvec_close(got[:, h], ref, ab, what=f"{L} layers, {source}, right-hand side {h}")
