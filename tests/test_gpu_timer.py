"""The library's launch timer: events around the pair-sweep launches only,
none while it is off or while a stream is captured into a graph."""
import pytest
import torch

from paper_2105_09465_gb300 import api, workloads as W
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def small():
    return W.realistic(seed=3, side=64, ss=1, n_sub=10, ygrid_side=32)


def test_timer_counts_the_timed_kernels_only():
    p = small()
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=torch.from_numpy(p.sub).cuda())
    s = api.Points(grid=p.ygrid)
    v = torch.from_numpy(p.v).cuda()
    api.lens_raytrace(q)  # warm-up: not recorded
    api.kernel_timer_enable(True)
    for _ in range(3):
        api.lens_raytrace(q)
    api.gp_kernel_matvec(api.Points(grid=p.xgrid), s, v, p.lengthscale, p.variance)
    api.kernel_timer_enable(False)
    api.lens_raytrace(q)  # timer off: not recorded
    n, ms, dropped = api.kernel_timer_read("raytrace")
    assert (n, dropped) == (3, 0) and ms > 0.0
    n, ms, _ = api.kernel_timer_read("matvec")
    assert n == 1 and ms > 0.0
    for k in ("train_rows", "bwd_rows", "dv_rows", "raytrace_vjp", "windowed"):
        assert api.kernel_timer_read(k)[0] == 0
    # enabling again clears the records
    api.kernel_timer_enable(True)
    api.kernel_timer_enable(False)
    assert api.kernel_timer_read("raytrace")[0] == 0


def test_timer_skips_graph_capture():
    p = small()
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=torch.from_numpy(p.sub).cuda())
    api.lens_raytrace(q)
    torch.cuda.synchronize()
    api.kernel_timer_enable(True)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        beta = api.lens_raytrace(q)
    g.replay()
    torch.cuda.synchronize()
    api.kernel_timer_enable(False)
    assert api.kernel_timer_read("raytrace")[0] == 0
    assert torch.equal(api.lens_raytrace(q), beta)
