"""The row-partitioned self-kernel step on one GPU: row bands run one after
the other (the exchanges done in-process: concatenating the bands' ray-traced
points, summing their parameter-gradient shares). At the large workload's
size (where no call splits its source groups) two bands give the unsharded
call's row results bitwise; on a small case with three bands, every result
is checked against the FP64 oracle. Summed parameter gradients differ from
the unsharded ones only by the reduction order's rounding."""
import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import api, shard, workloads as W
from tests.gpu_util import GRAD_REL, assert_close_tol, assert_matvec_close, dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def run_bands(p, world, align, v, g):
    sub = dev(p.sub)
    shards = [shard.RowShard(p.xgrid, p.lens, sub, r, world, align=align) for r in range(world)]
    beta_all = torch.cat([S.trace() for S in shards]).contiguous()
    parts = [S.reduce(beta_all, v, g, p.lengthscale, p.variance) for S in shards]
    share = sum(q[3] for q in parts)
    cat = [torch.cat([q[k] for q in parts]) for k in range(3)]
    return beta_all, cat, shard.unpack_share(share), sub


def test_two_bands_full_size_bitwise(orc):
    p = W.large()
    rng = np.random.default_rng(5)
    v, g = dev(rng.standard_normal(p.n)), dev(rng.standard_normal(p.n))
    beta_all, (out_b, dv_b, dx_b), (d_len, d_var, d_lens, d_sub), sub = run_bands(p, 2, 32, v, g)
    q = api.Points(xy=api.grid_points(p.xgrid), grid=p.xgrid, lens=p.lens, sub=sub)
    out = api.gp_kernel_matvec(api.Points(xy=beta_all, grid=p.xgrid), None, v, p.lengthscale, p.variance)
    G = api.gp_kernel_matvec_bwd(q, None, v, p.lengthscale, p.variance, g,
                                 want=("v", "x", "lengthscale", "variance", "lens", "sub"), beta=beta_all)
    torch.cuda.synchronize()
    assert torch.equal(out_b, out)
    assert torch.equal(dv_b, G["v"])
    assert torch.equal(dx_b, G["x"])
    for got, ref in ((d_len, G["lengthscale"].item()), (d_var, G["variance"].item())):
        assert abs(got - ref) <= 1e-6 * abs(ref)
    # the summed lens and subhalo shares against the oracle's ray-trace VJP of
    # the same dL/dbeta (40 sampled subhalos), as the unsharded result is
    xi = orc.grid_points(*p.xgrid.astuple())
    dx = host(G["x"])
    pick = np.sort(np.random.default_rng(6).choice(len(p.sub), 40, replace=False))
    rl, _, al, _ = orc.raytrace_vjp(xi, p.lens.astuple(), None, dx, 0, with_abs=True)
    _, rs, _, asub = orc.raytrace_vjp(xi, p.lens.astuple(), p.sub[pick], dx, 0, with_abs=True)
    for lens_g, sub_g, what in ((host(d_lens), host(d_sub), "bands"), (host(G["lens"]), host(G["sub"]), "whole")):
        assert_close_tol(lens_g, rl, GRAD_REL * al, what=f"{what} d_lens")
        assert_close_tol(sub_g[pick], rs, GRAD_REL * asub, what=f"{what} d_sub")
    # the bands' points are the unsharded ray-trace's, to the deflection tolerance
    assert float((beta_all - api.lens_raytrace(q)).abs().max()) <= 2e-6


def test_three_bands_against_the_oracle(orc):
    p = W.large(seed=21, side=120)
    rng = np.random.default_rng(6)
    vn, gn = rng.standard_normal(p.n).astype(np.float32), rng.standard_normal(p.n).astype(np.float32)
    beta_all, (out_b, dv_b, dx_b), (d_len, d_var, d_lens, d_sub), _ = run_bands(p, 3, 16, dev(vn), dev(gn))
    b = host(beta_all).astype(np.float32)
    ref, ab = orc.kernel_matvec(b, b, vn, p.lengthscale, p.variance)
    assert_matvec_close(host(out_b), ref, ab, what="bands forward")
    R = orc.kernel_matvec_vjp(b, b, vn, p.lengthscale, p.variance, gn.astype(np.float64), True, with_abs=True)
    assert_close_tol(host(dv_b), R["d_v"], GRAD_REL * R["d_v_abs"], what="bands d_v")
    assert_close_tol(host(dx_b), R["d_x"], GRAD_REL * R["d_x_abs"], what="bands d_x")
    assert_close_tol([d_len], [R["d_len"]], [GRAD_REL * R["d_len_abs"]], what="bands d_len")
    assert_close_tol([d_var], [R["d_var"]], [GRAD_REL * R["d_var_abs"]], what="bands d_var")
    xi = orc.grid_points(*p.xgrid.astuple())
    rl, rs, al, asub = orc.raytrace_vjp(xi, p.lens.astuple(), p.sub, host(dx_b), 0, with_abs=True)
    assert_close_tol(host(d_lens), rl, GRAD_REL * al, what="bands d_lens")
    assert_close_tol(host(d_sub), rs, GRAD_REL * asub, what="bands d_sub")
