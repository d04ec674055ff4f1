"""A lens prepared on the device (lr_lens_prepare) from device-resident
parameters, as an SVI step draws them: the same deflection and gradients as
the host-side lens, and an out-of-domain draw reported in the fault word
without a GPU fault (Sec. 2.2 lens model; Sec. 4.2 proposal over the lens
parameters)."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import api, workloads as W
from tests.golden.lenses import paper_lenses
from tests.gpu_util import ALPHA_TOL, GRAD_REL, assert_close_tol, dev, host, need_gpu, ulp32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def theta7(lens: W.Lens) -> torch.Tensor:
    return dev(np.array([lens.x0, lens.y0, lens.q, lens.phi, lens.theta_e, lens.g1, lens.g2], np.float32))


def record(lens: W.Lens) -> torch.Tensor:
    return api.lens_prepare(theta7(lens), lens.gamma)


@pytest.mark.parametrize("name", sorted(paper_lenses()))
def test_record_ray_trace_matches_oracle_and_host_lens(orc, name):
    """The printed lenses (FP32-rounded parameters, as the device holds them)
    with subhalos; the bound of the host-lens ray-trace test: 1e-6 arcsec or
    4 FP32 ulps of |alpha| where the steep slopes make |alpha| large."""
    lens = W.Lens(*[float(np.float32(v)) for v in paper_lenses()[name].values()])
    p = W.realistic(seed=5, side=60, n_sub=50)
    sub = dev(p.sub)
    api.fault_status(clear=True)
    b_rec, a_rec = (host(t) for t in api.lens_raytrace(api.Points(grid=p.xgrid, lens_record=record(lens), sub=sub),
                                                       want_alpha=True))
    b_host = host(api.lens_raytrace(api.Points(grid=p.xgrid, lens=lens, sub=sub)))
    xi = orc.grid_points(*p.xgrid.astuple())
    a_ref, b_ref = orc.raytrace(xi, lens.astuple(), p.sub)
    lim = np.maximum(ALPHA_TOL, 4 * ulp32(a_ref))
    assert np.all(np.abs(a_rec - a_ref) <= lim), float(np.max(np.abs(a_rec - a_ref) / lim))
    assert np.all(np.abs(b_rec - b_ref) <= lim + ulp32(b_ref))
    # the constants come from the same FP64 formulas on either side; a last
    # FP64 digit of cos, sin or pow may differ once rounded to FP32
    assert np.all(np.abs(b_rec - b_host) <= lim + ulp32(b_ref))
    assert api.fault_status() == 0


def test_record_vjp_matches_oracle(orc):
    p = W.realistic(seed=6, side=60, n_sub=40)
    sub = dev(p.sub)
    d_beta = np.random.default_rng(7).standard_normal((p.xgrid.n, 2)).astype(np.float32)
    pts = api.Points(grid=p.xgrid, lens_record=record(p.lens), sub=sub)
    d_lens, d_sub = api.lens_raytrace_vjp(pts, dev(d_beta))
    xi = orc.grid_points(*p.xgrid.astuple())
    rl, rs, al, asub = orc.raytrace_vjp(xi, p.lens.astuple(), p.sub, d_beta.astype(np.float64), 0, with_abs=True)
    assert_close_tol(host(d_lens), rl, GRAD_REL * al, what="d_lens")
    assert_close_tol(host(d_sub), rs, GRAD_REL * asub, what="d_sub")
    h_lens, h_sub = api.lens_raytrace_vjp(api.Points(grid=p.xgrid, lens=p.lens, sub=sub), dev(d_beta))
    assert_close_tol(host(d_lens), host(h_lens), GRAD_REL * al, what="d_lens vs host lens")


def test_record_in_the_fused_self_kernel():
    """gp_kernel_matvec with the ray-trace fused in takes the record too."""
    p = W.realistic(seed=8, side=50, n_sub=30)
    sub = dev(p.sub)
    v = dev(np.random.default_rng(9).standard_normal(p.xgrid.n).astype(np.float32))
    out_r = api.gp_kernel_matvec(api.Points(grid=p.xgrid, lens_record=record(p.lens), sub=sub), None, v, 0.05)
    out_h = api.gp_kernel_matvec(api.Points(grid=p.xgrid, lens=p.lens, sub=sub), None, v, 0.05)
    scale = float(torch.sum(torch.abs(v)))
    assert float(torch.max(torch.abs(out_r - out_h))) <= 1e-5 * scale


@pytest.mark.parametrize("bad", [("q", 1.5), ("q", 0.0), ("theta_e", -0.1), ("x0", float("nan"))])
def test_out_of_domain_draw_sets_fault_code_2(bad):
    """A draw outside the lens domain cannot be refused at the call (its
    parameters never reach the host): the ray-trace records code 2 and
    writes finite values; a valid record afterwards records nothing."""
    ok = W.Lens(0.01, -0.02, 0.8, 0.3, 1.2, 2.0, 0.01, 0.02)
    lens = dataclasses.replace(ok, **{bad[0]: bad[1]})
    g = W.Grid(20, 20, 1, 0.1)
    api.fault_status(clear=True)
    beta = api.lens_raytrace(api.Points(grid=g, lens_record=record(lens)))
    torch.cuda.synchronize()
    assert api.fault_status(clear=True) == 2
    assert bool(torch.isfinite(beta).all())
    api.lens_raytrace(api.Points(grid=g, lens_record=record(ok)))
    torch.cuda.synchronize()
    assert api.fault_status() == 0
