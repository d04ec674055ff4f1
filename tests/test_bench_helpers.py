"""Host-side helpers of bench.py: the ray-trace kernels' op-count model and
the backward's tiling mirror, exercised on the CPU so that an error in them
surfaces before a GPU run."""
import importlib
import sys

import pytest

from paper_2105_09465_gb300 import workloads as W


@pytest.fixture(scope="module")
def bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        yield importlib.import_module("bench")
    finally:
        sys.argv = argv


def test_vjp_bands_divide_the_tiles(bench):
    for nblk, w, h in [(4864, 1600, 1600), (1216, 800, 800), (608, 1600, 1600), (8, 32, 32), (7, 10, 3)]:
        r = bench.vjp_bands(nblk, w, h)
        assert nblk % r == 0 and 1 <= r <= max(1, min(nblk, h))


def test_vjp_phases(bench):
    assert bench.vjp_phases(2_560_000, 4864, 2000) == 1  # one phase: 2048 slots waste 2.3 %
    assert bench.vjp_phases(640_000, 1216, 200) == 3     # 600 slots fill 640 threads
    assert bench.vjp_phases(1024, 8, 1) == 1             # 128-point tiles keep one phase


@pytest.mark.parametrize("side", [64, 128])
def test_cost_models_are_shares(bench, side):
    p = W.large(side=side)
    nblk = max(1, (p.n + 127) // 128)
    for mufu, lanes, sh in (bench.raytrace_cost(p), bench.vjp_cost(p, nblk)):
        total = sum(v for k, v in sh.items() if k != "expansion_lanes")
        assert total == pytest.approx(1.0, abs=1e-9)
        assert 0 < lanes < 60 and 0 < mufu <= 4
        assert "closed form" in bench._shares_text(sh)
