"""The ray-trace backward above one wave of tiles, against the FP64 oracle.

Above a full wave of resident CTA slots (608 on a GB300) the backward cuts
its points into several waves of tiles. For tNFW subhalos a plan sorts each
tile's subhalos and launches the tiles heaviest first. The full-size tests
cover a pixel grid with tNFW subhalos. Here, at 640k points (two waves):

- explicit points, whose tiles are contiguous index ranges, with a plan;
- point-mass subhalos on a pixel grid, without a plan;
- repeated calls, which give the same bits.

Every lens and subhalo gradient is compared element by element at the
stated 2e-5 of the sum of absolute terms.
"""
import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import api, workloads as W
from tests.gpu_util import GRAD_REL, assert_close_tol, dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def check(orc, xi, q, lens, sub, profile, db):
    d_lens, d_sub = api.lens_raytrace_vjp(q, dev(db))
    rl, rs, al, asub = orc.raytrace_vjp(xi, lens.astuple(), sub, db, profile, with_abs=True)
    assert_close_tol(host(d_lens), rl, GRAD_REL * al, what="d_lens")
    assert_close_tol(host(d_sub), rs, GRAD_REL * asub, what="d_sub")
    return d_lens, d_sub


def test_explicit_points_several_waves(orc):
    rng = np.random.default_rng(71)
    lens = W.draw_lens(rng)
    sub = W.draw_subhalos(rng, 40, lens, 1e6, 1e10)
    xi = rng.uniform(-6.0, 6.0, (640_000, 2)).astype(np.float32)
    db = rng.standard_normal(xi.shape).astype(np.float32)
    check(orc, xi, api.Points(xy=dev(xi), lens=lens, sub=dev(sub)), lens, sub, 0, db)


def test_point_masses_on_a_grid_several_waves(orc):
    rng = np.random.default_rng(72)
    lens = W.draw_lens(rng)
    g = W.Grid(400, 400, 2, 0.05)
    sub = np.stack([rng.uniform(-2, 2, 40), rng.uniform(-2, 2, 40), rng.uniform(0.005, 0.05, 40),
                    np.zeros(40), np.zeros(40)], 1).astype(np.float32)
    xi = orc.grid_points(*g.astuple())
    db = rng.standard_normal(xi.shape).astype(np.float32)
    check(orc, xi, api.Points(grid=g, lens=lens, sub=dev(sub), profile=1), lens, sub, 1, db)


def test_planned_calls_repeat_bitwise():
    p = W.large(seed=9, side=400)
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub))
    db = dev(np.random.default_rng(73).standard_normal((p.n, 2)).astype(np.float32))
    a = api.lens_raytrace_vjp(q, db)
    b = api.lens_raytrace_vjp(q, db)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
