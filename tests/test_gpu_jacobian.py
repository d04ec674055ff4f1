"""Parity of the CUDA lens Jacobian / magnification with the FP64 oracle."""
import numpy as np
import pytest

from paper_2105_09465_gb300 import api, workloads as W
from tests.golden.lenses import paper_lenses
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def check(orc, grid, lens, sub, profile=0):
    jac, mu = api.lens_jacobian(api.Points(grid=grid, lens=lens, sub=dev(sub) if sub is not None else None,
                                           profile=profile))
    xi = orc.grid_points(*grid.astuple())
    jr, mr = orc.lens_jacobian(xi, lens.astuple(), sub, profile)
    j, m = host(jac), host(mu)
    # FP32 derivative terms: relative 2e-6 of the largest entry of d alpha/d xi at that point
    scale = 1.0 + np.abs(jr - np.eye(2)).max(axis=(1, 2))
    err = np.abs(j - jr).max(axis=(1, 2))
    assert np.all(err <= 2e-6 * scale), float(np.max(err / scale))
    # det A from the returned magnification: element errors of 2e-6 S propagate
    # to det as ~4e-6 S^2 with S the largest |A_ij| (cancellation near critical curves)
    det_r = 1.0 / mr
    det = 1.0 / m
    S = np.abs(jr).max(axis=(1, 2))
    assert np.all(np.abs(det - det_r) <= 1e-5 * S * S)


def test_sie_shear(orc):
    p = W.tiny()
    check(orc, p.xgrid, p.lens, None)


@pytest.mark.parametrize("name", ["hoags_object", "arp148"])
def test_printed_lenses(orc, name):
    L = W.Lens(*[float(np.float32(v)) for v in paper_lenses()[name].values()])
    check(orc, W.Grid(50, 50, 2, 0.05, 0.0125, 0.0125), L, None)


def test_realistic_with_subhalos(orc):
    p = W.realistic(seed=71, side=60, ss=2, n_sub=200)
    check(orc, p.xgrid, p.lens, p.sub)


def test_point_masses(orc):
    rng = np.random.default_rng(3)
    lens = W.draw_lens(rng)
    sub = np.stack([rng.uniform(-1, 1, 30), rng.uniform(-1, 1, 30), rng.uniform(0.01, 0.05, 30),
                    np.zeros(30), np.zeros(30)], 1).astype(np.float32)
    check(orc, W.Grid(40, 40, 2, 0.05, 0.0125, 0.0125), lens, sub, profile=1)
