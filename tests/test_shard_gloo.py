"""The row-partitioned self-kernel step on the host: two gloo ranks run
paper_2105_09465_gb300.shard with the FP64 oracle standing in for the CUDA
kernels (test-only), exchange beta by all-gather and the parameter gradients
by all-reduce, and together give the unsharded oracle's results."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2105_09465_gb300 import shard, workloads as W


class OracleKernels:
    """The oracle behind the interface of shard.GpuKernels (FP64, host)."""

    def __init__(self):
        import oracle
        oracle.build()
        self.o = oracle

    def grid_points(self, grid):
        return torch.from_numpy(self.o.grid_points(*grid.astuple()).astype(np.float64))

    def raytrace(self, xi, layout, lens, sub):
        return torch.from_numpy(self.o.raytrace(xi.numpy(), lens.astuple(), sub)[1])

    def forward(self, beta_own, own_layout, beta_all, all_layout, v, ell, var):
        return torch.from_numpy(self.o.kernel_matvec(beta_own.numpy(), beta_all.numpy(), v.numpy(), ell, var)[0])

    def backward(self, beta_own, own_layout, beta_all, all_layout, row0, v, g, ell, var):
        n = beta_own.shape[0]
        rows = row0 + np.arange(n)
        R = self.o.self_vjp_rows(beta_all.numpy(), v.numpy(), g.numpy(), ell, var, rows)
        # the rows' share of d_l and d_var: the row sums of these rows
        S = self.o.kernel_matvec_vjp(beta_own.numpy(), beta_all.numpy(), v.numpy(), ell, var, g.numpy()[rows])
        return (torch.from_numpy(R["d_v"]), torch.from_numpy(R["d_x"]),
                torch.tensor([S["d_len"]], dtype=torch.float64), torch.tensor([S["d_var"]], dtype=torch.float64))

    def vjp(self, xi_own, own_layout, lens, sub, d_x):
        dl, ds = self.o.raytrace_vjp(xi_own.numpy(), lens.astuple(), sub, d_x.numpy())
        return torch.from_numpy(dl), torch.from_numpy(ds)


def case():
    p = W.realistic(seed=9, side=24, ss=2, n_sub=6)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(p.n)
    g = rng.standard_normal(p.n)
    return p, v, g, 0.05, 1.2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, v, g, ell, var = case()
    R = shard.self_kernel_step(p.xgrid, p.lens, p.sub, torch.from_numpy(v), torch.from_numpy(g), ell, var, rank,
                               world, kernels=OracleKernels(), align=8)
    out[rank] = {"rows": R.rows, "out": R.out.numpy(), "d_v": R.d_v.numpy(), "d_x": R.d_x.numpy(),
                 "d_len": R.d_lengthscale, "d_var": R.d_variance, "d_lens": R.d_lens.numpy(),
                 "d_sub": R.d_sub.numpy(), "beta_all": R.beta_all.numpy()}
    dist.barrier()
    dist.destroy_process_group()


def test_row_bands_partition_the_image():
    g = W.Grid(100, 75, 2, 0.05)
    for world in (1, 2, 3, 8):
        b = shard.row_bands(g, world)
        assert b[0][0] == 0 and b[-1][1] == 150
        assert all(b[k][1] == b[k + 1][0] for k in range(world - 1))
        assert all((r1 - r0) % 2 == 0 for r0, r1 in b)


@pytest.mark.timeout(300)
def test_two_gloo_ranks_equal_the_unsharded_oracle(orc):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert r0["rows"][0] == 0 and r0["rows"][1] == r1["rows"][0]
    p, v, g, ell, var = case()
    assert r1["rows"][1] == p.n
    np.testing.assert_array_equal(r0["beta_all"], r1["beta_all"])  # the all-gather gave both ranks every point
    xi = orc.grid_points(*p.xgrid.astuple())
    _, b = orc.raytrace(xi, p.lens.astuple(), p.sub)
    np.testing.assert_array_equal(r0["beta_all"], b)
    ref, _ = orc.kernel_matvec(b, b, v, ell, var)
    R = orc.kernel_matvec_vjp(b, b, v, ell, var, g, True)
    dl, ds = orc.raytrace_vjp(xi, p.lens.astuple(), p.sub, R["d_x"])
    cat = lambda k: np.concatenate([r0[k], r1[k]])
    np.testing.assert_allclose(cat("out"), ref, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(cat("d_v"), R["d_v"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(cat("d_x"), R["d_x"], rtol=1e-10, atol=1e-12)
    for rk in (r0, r1):  # the all-reduced parameter gradients, the same on both ranks
        assert rk["d_len"] == pytest.approx(R["d_len"], rel=1e-10)
        assert rk["d_var"] == pytest.approx(R["d_var"], rel=1e-10)
        np.testing.assert_allclose(rk["d_lens"], dl, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(rk["d_sub"], ds, rtol=1e-9, atol=1e-12)
