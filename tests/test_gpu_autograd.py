"""The autograd wrapper returns exactly the CUDA backward's gradients, and
agrees with finite differences of the CUDA forward where FP32 allows."""
import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import api, workloads as W
from paper_2105_09465_gb300.autograd import lensed_gp_matvec
from tests.gpu_util import dev, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def setup(seed=61):
    p = W.realistic(seed=seed, side=40, ss=2, n_sub=25)
    v = dev(p.v).requires_grad_(True)
    lens = torch.tensor(p.lens.astuple(), dtype=torch.float64, requires_grad=True)
    sub = dev(p.sub).requires_grad_(True)
    ell = torch.tensor(p.lengthscale, dtype=torch.float64, requires_grad=True)
    var = torch.tensor(1.3, dtype=torch.float64, requires_grad=True)
    return p, v, lens, sub, ell, var


def test_autograd_matches_direct_backward():
    p, v, lens, sub, ell, var = setup()
    out = lensed_gp_matvec(v, lens, sub, ell, var, p.xgrid, p.ygrid)
    g = dev(np.random.default_rng(1).standard_normal(p.n))
    (out * g).sum().backward()
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=sub.detach())
    s = api.Points(grid=p.ygrid)
    # the wrapper's path: training forward (row moments), then the backward with them
    beta = torch.empty((p.n, 2), device="cuda")
    _, mom = api.gp_kernel_matvec_train(q, s, v.detach(), p.lengthscale, 1.3, beta=beta)
    G = api.gp_kernel_matvec_bwd(q, s, v.detach(), p.lengthscale, 1.3, g,
                                 want=["v", "lens", "sub", "lengthscale", "variance"], beta=beta, moments=mom)
    assert torch.equal(v.grad, G["v"])
    assert torch.equal(lens.grad[[0, 1, 2, 3, 4, 6, 7]], G["lens"].cpu())
    assert lens.grad[5] == 0
    assert torch.equal(sub.grad[:, :4], G["sub"].float())
    assert torch.all(sub.grad[:, 4] == 0)
    assert ell.grad.item() == G["lengthscale"].item() and var.grad.item() == G["variance"].item()


def test_finite_differences_on_gpu_forward():
    """Central differences of the FP32 forward (informational precision: the
    step is large enough to dominate FP32 noise, the tolerance is loose). The
    inducing grid is coarse (l = 0.15 arcsec) so that a 1e-3 arcsec step stays
    in the linear regime (with l = 0.025 the central difference at that step
    is 25% off even in FP64)."""
    p, v, lens, sub, ell, var = setup(62)
    p.ygrid = W.Grid(24, 24, 1, 0.1)
    v = dev(np.random.default_rng(3).standard_normal(p.ygrid.n)).requires_grad_(True)
    ell = torch.tensor(0.15, dtype=torch.float64, requires_grad=True)
    g = dev(np.random.default_rng(2).standard_normal(p.n))
    out = lensed_gp_matvec(v, lens, sub, ell, var, p.xgrid, p.ygrid)
    (out * g).sum().backward()

    def loss(lens_t=lens, ell_t=ell, var_t=var):
        with torch.no_grad():
            o = lensed_gp_matvec(v, lens_t, sub, ell_t, var_t, p.xgrid, p.ygrid)
            return float((o.double() * g.double()).sum())

    h = 1e-3
    fd = (loss(var_t=var + h) - loss(var_t=var - h)) / (2 * h)
    assert abs(fd - var.grad.item()) <= 1e-3 * abs(fd) + 1e-3
    fd = (loss(ell_t=ell + h * ell) - loss(ell_t=ell - h * ell)) / (2 * h * ell.item())
    assert abs(fd - ell.grad.item()) <= 2e-2 * abs(fd) + 1e-2
    for k, hk in [(0, 1e-3), (2, 1e-3), (4, 1e-3)]:
        e = torch.zeros(8, dtype=torch.float64)
        e[k] = hk
        fd = (loss(lens_t=lens + e) - loss(lens_t=lens - e)) / (2 * hk)
        assert abs(fd - lens.grad[k].item()) <= 5e-2 * abs(fd) + 5e-2 * torch.abs(lens.grad).max().item(), k
