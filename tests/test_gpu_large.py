"""The large workload against the FP64 oracle.

800x800 image at 2x2 supersampling (2.56M ray-traced points), power-law lens
+ shear + 2000 truncated-NFW subhalos, self-kernel with l = 0.05 arcsec
(6.55e12 pairs), forward and backward in the benchmark's launch
configuration: the ray-trace fused into the forward call, the backward with
the forward's points, down to the lens and subhalo parameters.

At full size the oracle checks a seeded sample of 10,000 rows element by
element: the ray-traced points, the reduction, d_v and both roles of d_x (on
the GPU's own points, which isolates the reduction). The lens gradient and a
sample of subhalo gradients are checked by running the oracle's ray-trace VJP
on the GPU's dL/dbeta over every point. d_variance is checked against its
identity sum_i g_i out_i / var. A reduced-size copy of the same recipe runs
the whole chain against the oracle's own FP64 chain, with the derived
input-error tolerances."""
import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import api, workloads as W
from tests.gpu_util import (ALPHA_TOL, GRAD_REL, assert_close_tol, assert_matvec_close, chain_tol, dev, host,
                            lens_chain_tols, need_gpu, point_delta, ulp32)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def run_gpu(p, g):
    sub = dev(p.sub)
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=sub)
    v = dev(p.v)
    out, beta = api.gp_kernel_matvec(q, None, v, p.lengthscale, p.variance, want_beta=True)
    G = api.gp_kernel_matvec_bwd(q, None, v, p.lengthscale, p.variance, dev(g),
                                 want=("v", "x", "lengthscale", "variance", "lens", "sub"), beta=beta)
    return host(out), host(beta).astype(np.float32), {k: host(t) for k, t in G.items()}


@pytest.fixture(scope="module")
def large(orc):
    p = W.large()
    g = np.random.default_rng(404).standard_normal(p.n).astype(np.float32)
    out, beta, G = run_gpu(p, g)
    return p, g, out, beta, G


def test_large_ray_trace_sampled_rows(orc, large):
    p, g, out, beta, G = large
    rows = np.random.default_rng(4).choice(p.n, 10000, replace=False)
    xi = orc.grid_points(*p.xgrid.astuple())[rows]
    _, bref = orc.raytrace(xi, p.lens.astuple(), p.sub)
    err = np.abs(beta[rows].astype(np.float64) - bref)
    tol = ALPHA_TOL + ulp32(bref)
    assert np.all(err <= tol), float(np.max(err / tol))


def test_large_reduction_and_gradients_sampled_rows(orc, large):
    """out, d_v and d_x (both roles) on 10,000 seeded rows, each against all
    2.56M points, on the GPU's ray-traced points: 2e-5 of the absolute terms."""
    p, g, out, beta, G = large
    rows = np.random.default_rng(4).choice(p.n, 10000, replace=False)
    R = orc.self_vjp_rows(beta, p.v, g, p.lengthscale, p.variance, rows)
    assert_matvec_close(out[rows], R["out"], R["out_abs"], what="large self-kernel forward")
    assert_close_tol(G["v"][rows], R["d_v"], GRAD_REL * R["d_v_abs"], what="d_v")
    assert_close_tol(G["x"][rows], R["d_x"], GRAD_REL * R["d_x_abs"], what="d_x")


def test_large_lens_and_subhalo_gradients(orc, large):
    """The GPU's lens gradient and 40 sampled subhalo gradients against the
    oracle's ray-trace VJP of the GPU's own dL/dbeta over all 2.56M points (a
    subhalo's gradient depends only on its own deflection, the lens gradient
    only on the main deflector and the shear)."""
    p, g, out, beta, G = large
    xi = orc.grid_points(*p.xgrid.astuple())
    pick = np.sort(np.random.default_rng(6).choice(len(p.sub), 40, replace=False))
    rl, _, al, _ = orc.raytrace_vjp(xi, p.lens.astuple(), None, G["x"], 0, with_abs=True)
    assert_close_tol(G["lens"], rl, GRAD_REL * al, what="d_lens")
    _, rs, _, asub = orc.raytrace_vjp(xi, p.lens.astuple(), p.sub[pick], G["x"], 0, with_abs=True)
    assert_close_tol(G["sub"][pick], rs, GRAD_REL * asub, what="d_sub")


def test_large_variance_gradient_identity(large):
    """d_var = sum_i g_i out_i / var holds at any size."""
    p, g, out, beta, G = large
    ref = float(np.sum(g.astype(np.float64) * out) / p.variance)
    scale = float(np.sum(np.abs(g.astype(np.float64) * out)) / abs(p.variance))
    assert abs(float(G["variance"][0]) - ref) <= GRAD_REL * scale


def test_large_recipe_reduced_size_full_chain(orc):
    """The large recipe (power-law lens, shear, 2000 tNFW on [1e6, 1e10]
    Msun, self-kernel l = 0.05) at 100x100 pixels x 2x2: every output and
    gradient against the oracle's FP64 chain on its own ray-traced points."""
    p = W.large(seed=14, side=100)
    g = np.random.default_rng(15).standard_normal(p.n).astype(np.float32)
    out, beta, G = run_gpu(p, g)
    xi = orc.grid_points(*p.xgrid.astuple())
    _, bref = orc.raytrace(xi, p.lens.astuple(), p.sub)
    delta = point_delta(bref)
    ref, ab, sens = orc.kernel_matvec(bref, bref, p.v, p.lengthscale, p.variance, with_sens=True)
    assert_matvec_close(out, ref, ab, sens, delta, what="fused self-kernel")
    R = orc.kernel_matvec_vjp(bref, bref, p.v, p.lengthscale, p.variance, g.astype(np.float64), True, with_abs=True)
    assert_close_tol(G["v"], R["d_v"], chain_tol(R, "d_v", delta), what="d_v")
    assert_close_tol(G["x"], R["d_x"], chain_tol(R, "d_x", delta), what="d_x")
    for k, rk in (("lengthscale", "d_len"), ("variance", "d_var")):
        assert_close_tol(G[k], [R[rk]], [chain_tol(R, rk, delta)], what=rk)
    rl, rs, tl, ts = lens_chain_tols(orc, xi, p.lens.astuple(), p.sub, R, delta)
    assert_close_tol(G["lens"], rl, tl, what="d_lens")
    assert_close_tol(G["sub"], rs, ts, what="d_sub")


def test_large_pairs_evaluated(large):
    """The culled sweeps evaluate a small fraction of the 6.55e12 logical
    pairs, and at least every pair within the exact-zero radius (counted on
    a sample of rows)."""
    p = large[0]
    beta = torch.from_numpy(large[3]).cuda()
    q = api.Points(xy=beta, grid=p.xgrid)
    fwd, fwd_slots = api.cull_pairs_evaluated(q, None, p.lengthscale, 0)
    bwd, bwd_slots = api.cull_pairs_evaluated(q, None, p.lengthscale, 1)
    assert 0 < fwd <= fwd_slots and 0 < bwd <= bwd_slots
    assert fwd < 0.01 * p.n * p.n and bwd < 0.01 * p.n * p.n
    # lower bound: pairs whose exponent is above -126 must all be evaluated
    b = large[3].astype(np.float64)
    rows = np.random.default_rng(8).choice(p.n, 200, replace=False)
    c = np.log2(np.e) / (2 * p.lengthscale ** 2)
    need = sum(int(np.count_nonzero(c * ((b - b[i]) ** 2).sum(1) <= 126.0)) for i in rows)
    assert fwd >= need * (p.n / 200) * 0.5
