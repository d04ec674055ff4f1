"""The self-kernel step with its rows split across the ranks of a process
group (one rank per GPU): the path's one real exchange.

The pair sum out_i = sum_j k(beta_i, beta_j) v_j (Sec. 3.1 RBF kernel over
the ray-traced pixels, Sec. 3.3 lazy reduction) needs every point as a
source but each output row only once. Rank r owns a band of whole image rows
(points [p0_r, p1_r) in row-major order, bands cut at multiples of the
supersampling so that each band is itself a pixel grid):

  1. ray-trace its own points through the lens and subhalos (Sec. 2.1);
  2. all-gather beta: every rank then holds all the points as sources
     (8 bytes per point: 20 MB for 2.56M points);
  3. forward: out for its rows against all points;
  4. backward with dL/dout for all points (replicated, or all-gathered by
     the caller): d_v of its rows, dL/dbeta of its rows with both roles
     (the row role and the column role, which needs g at every source), and
     its rows' share of d_lengthscale and d_variance;
  5. the ray-trace VJP of its rows: its share of the 7 lens and 4 S subhalo
     gradients;
  6. all-reduce (sum) of the 2 + 7 + 4 S parameter gradients.

No other data crosses ranks: out, d_v and dL/dbeta stay with the rank that
owns the rows. Sums of a partition of the rows are the whole self-kernel's
gradients. A row's reductions are bitwise the same in a band as in the whole
problem whenever neither call splits its source groups across CTAs (the row
blocks alone fill the GPU, as at the large workload's sizes): the culled
sweeps visit a row's chunks in the sources' order and fold only nonzero chunk
sums, so the row block a row lands in changes no bit.

The kernel calls go through a `kernels` object (GpuKernels by default, the
library's CUDA entry points); the collectives through torch.distributed, so
the same orchestration runs over NCCL on GPUs or, with other kernels, over
gloo on the host (the tests do that).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from .workloads import Grid, Lens


def row_bands(grid: Grid, world: int, align: int = 32) -> list[tuple[int, int]]:
    """Bands of supersampled image rows [r0, r1) per rank: contiguous, whole
    rows, cut at multiples of `align` rows (rounded down to a multiple of the
    supersampling; the row-block tiles of the sweeps are 32 rows high), as
    even as that allows; empty bands when there are more ranks than blocks."""
    H = grid.ny * grid.ss
    step = max(align, grid.ss)
    step -= step % grid.ss
    blocks = (H + step - 1) // step
    out = []
    for r in range(world):
        b0, b1 = r * blocks // world, (r + 1) * blocks // world
        out.append((min(b0 * step, H), min(b1 * step, H)))
    return out


def band_grid(grid: Grid, r0: int, r1: int) -> Grid:
    """The layout of a band of rows as a grid of its own (only its shape is
    used: explicit points carry it to order their row blocks and chunks)."""
    return Grid(grid.nx, (r1 - r0) // grid.ss, grid.ss, grid.pix, grid.cx, grid.cy)


class GpuKernels:
    """The library's CUDA entry points."""

    def __init__(self):
        from . import api
        self.api = api

    def grid_points(self, grid: Grid) -> torch.Tensor:
        return self.api.grid_points(grid)

    def raytrace(self, xi: torch.Tensor, layout: Grid, lens: Lens, sub: torch.Tensor | None) -> torch.Tensor:
        return self.api.lens_raytrace(self.api.Points(xy=xi, grid=layout, lens=lens, sub=sub))

    def forward(self, beta_own, own_layout, beta_all, all_layout, v, ell, var):
        api = self.api
        return api.gp_kernel_matvec(api.Points(xy=beta_own, grid=own_layout), api.Points(xy=beta_all, grid=all_layout),
                                    v, ell, var)

    def backward(self, beta_own, own_layout, beta_all, all_layout, row0, v, g, ell, var):
        api = self.api
        G = api.gp_kernel_matvec_bwd(api.Points(xy=beta_own, grid=own_layout),
                                     api.Points(xy=beta_all, grid=all_layout), v, ell, var, g,
                                     want=("v", "x", "lengthscale", "variance"), source_rows=row0)
        return G["v"], G["x"], G["lengthscale"], G["variance"]

    def vjp(self, xi_own, own_layout, lens, sub, d_x):
        api = self.api
        return api.lens_raytrace_vjp(api.Points(xy=xi_own, grid=own_layout, lens=lens, sub=sub), d_x)


@dataclass
class ShardResult:
    rows: tuple[int, int]      # this rank's points [p0, p1)
    beta_all: torch.Tensor     # (n, 2) every ray-traced point
    out: torch.Tensor          # (p1 - p0,) this rank's rows of K v
    d_v: torch.Tensor          # (p1 - p0,) this rank's rows of dL/dv
    d_x: torch.Tensor          # (p1 - p0, 2) dL/dbeta of this rank's points (both roles)
    d_lengthscale: float       # all-reduced
    d_variance: float
    d_lens: torch.Tensor       # (7,) all-reduced
    d_sub: torch.Tensor        # (S, 4) all-reduced


class RowShard:
    """Rank r's share of the step: its band of rows (steps 1 and 3-5 of the
    module docstring); the exchanges (steps 2 and 6) are the caller's."""

    def __init__(self, grid: Grid, lens: Lens, sub, rank: int, world: int, kernels=None, align: int = 32):
        self.K = kernels or GpuKernels()
        self.grid, self.lens, self.sub = grid, lens, sub
        self.bands = row_bands(grid, world, align)
        W = grid.nx * grid.ss
        r0, r1 = self.bands[rank]
        self.rows = (r0 * W, r1 * W)
        self.counts = [(b1 - b0) * W for b0, b1 in self.bands]
        self.layout = band_grid(grid, r0, r1)
        self.xi = self.K.grid_points(grid)[self.rows[0]:self.rows[1]].contiguous()

    def trace(self):
        """Step 1: the band's ray-traced points."""
        self.beta = self.K.raytrace(self.xi, self.layout, self.lens, self.sub)
        return self.beta

    def reduce(self, beta_all, v, g, lengthscale: float, variance: float):
        """Steps 3-5 with every ray-traced point: (out, d_v, d_x) of the band
        and its share (FP64 vector d_l, d_var, 7 lens, 4 S subhalo) of the
        parameter gradients."""
        K = self.K
        out = K.forward(self.beta, self.layout, beta_all, self.grid, v, lengthscale, variance)
        d_v, d_x, d_len, d_var = K.backward(self.beta, self.layout, beta_all, self.grid, self.rows[0], v, g,
                                            lengthscale, variance)
        d_lens, d_sub = K.vjp(self.xi, self.layout, self.lens, self.sub, d_x)
        share = torch.cat([torch.as_tensor(d_len).reshape(1).double(), torch.as_tensor(d_var).reshape(1).double(),
                           torch.as_tensor(d_lens).reshape(-1).double(), torch.as_tensor(d_sub).reshape(-1).double()])
        return out, d_v, d_x, share


def unpack_share(share: torch.Tensor):
    """(d_lengthscale, d_variance, d_lens (7,), d_sub (S, 4)) of a summed share vector."""
    ns = (share.numel() - 9) // 4
    return float(share[0]), float(share[1]), share[2:9], share[9:].reshape(ns, 4)


def self_kernel_step(grid: Grid, lens: Lens, sub, v: torch.Tensor, g: torch.Tensor, lengthscale: float,
                     variance: float, rank: int, world: int, group=None, kernels=None,
                     align: int = 32) -> ShardResult:
    """One forward + backward of the self-kernel over the ray-traced pixels of
    `grid`, rows split across `world` ranks (see the module docstring). v and
    g cover all points on every rank; collectives use `group` (the default
    process group when None; none at all when world == 1)."""
    import torch.distributed as dist

    S = RowShard(grid, lens, sub, rank, world, kernels, align)
    beta_own = S.trace()
    # step 2: all-gather beta (bands may differ in size: gather padded bands)
    if world > 1:
        pad = torch.zeros((max(S.counts), 2), dtype=beta_own.dtype, device=beta_own.device)
        pad[: beta_own.shape[0]] = beta_own
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        beta_all = torch.cat([parts[k][: S.counts[k]] for k in range(world)]).contiguous()
    else:
        beta_all = beta_own
    out, d_v, d_x, share = S.reduce(beta_all, v, g, lengthscale, variance)
    # step 6: all-reduce of the parameter gradients (FP64)
    if world > 1:
        dist.all_reduce(share, op=dist.ReduceOp.SUM, group=group)
    d_len, d_var, d_lens, d_sub = unpack_share(share)
    return ShardResult(rows=S.rows, beta_all=beta_all, out=out, d_v=d_v, d_x=d_x, d_lengthscale=d_len,
                       d_variance=d_var, d_lens=d_lens, d_sub=d_sub)
