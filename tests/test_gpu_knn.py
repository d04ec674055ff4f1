"""Parity of the CUDA k-nearest-neighbour inducing-point density and
transmission weights with the FP64 oracle (same FP32 points on both sides)."""
import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import abi, api, workloads as W
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu
R2_REL = 1e-6  # FP32 squared distances of FP32 points: a few 2^-24 relative


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def check(orc, q, k, rows=None):
    q = np.ascontiguousarray(q, np.float32)
    r2 = host(api.knn_density(dev(q), k))
    ref = orc.knn_r2(q, k, rows)
    got = r2 if rows is None else r2[rows]
    bad = np.abs(got - ref) > R2_REL * ref
    assert not bad.any(), (int(bad.sum()), got[bad][:5], ref[bad][:5])
    return r2


@pytest.mark.parametrize("k", [1, 5, 20, 32])
def test_uniform_random(orc, k):
    q = np.random.default_rng(k).uniform(-3, 3, (6000, 2))
    check(orc, q, k)


def test_lattice_ties(orc):
    g = ((np.arange(64) - 31.5) * 0.05).astype(np.float32)
    q = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2)
    r2 = check(orc, q, 20)
    inner = np.array([r * 64 + c for r in range(4, 60) for c in range(4, 60)])
    np.testing.assert_allclose(r2[inner], 5 * 0.05 ** 2, rtol=1e-6)


def test_lensed_pixels(orc):
    """The image-plane inducing points: ray-traced pixel centres, dense in
    the magnified regions of the source plane."""
    rng = np.random.default_rng(8)
    lens = W.draw_lens(rng)
    _, b = orc.raytrace(orc.grid_points(200, 200, 1, 0.02), lens.astuple())
    rows = np.sort(rng.choice(len(b), 3000, replace=False))
    check(orc, b, 20, rows)


def test_coincident_line_and_outlier(orc):
    rng = np.random.default_rng(9)
    q = rng.uniform(-1, 1, (3000, 2))
    q[100:200] = q[0:100]
    r2 = check(orc, q, 1)
    assert np.all(r2[0:200] == 0.0)
    line = np.stack([rng.uniform(-5, 5, 2000), np.zeros(2000)], -1)
    check(orc, line, 20)
    clump = np.concatenate([rng.normal(0, 1e-3, (2000, 2)), [[500.0, -300.0]]])
    check(orc, clump, 20)


def test_transmission_weights(orc):
    q = np.random.default_rng(10).uniform(-2, 2, (5000, 2)).astype(np.float32)
    r2, a = api.knn_density(dev(q), 20, lengthscale=0.07)
    ref = orc.transmission_weights(q, 0.07, 20)
    np.testing.assert_allclose(host(a), ref, rtol=2e-6)
    assert host(r2).shape == (5000,)


def test_arguments_are_validated():
    q = torch.zeros((20, 2), device="cuda")
    with pytest.raises(abi.LensGPError, match="other neighbour"):
        api.knn_density(q, 20)
    with pytest.raises(abi.LensGPError, match="outside"):
        api.knn_density(torch.zeros((100, 2), device="cuda"), 33)
