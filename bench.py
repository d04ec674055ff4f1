"""Benchmark: fused lens ray-trace + Gaussian-kernel reduction on one GB300.

Headline workload (the largest configuration that fits one GPU): one
800x800 image at 2x2 supersampling (2.56M points), ray-traced through a
power-law lens + shear + 2000 truncated-NFW subhalos; the squared-exponential
self-kernel of the 2.56M ray-traced points (6.55e12 logical pairs), forward
and backward down to the lens and subhalo parameters. One step = the forward
call (ray-trace fused into it) and the backward call.

A second section times the realistic workload (400x400 at 2x2 = 640k points,
200 subhalos, against a 128x128 grid of inducing points) with its own kernel
table, then the serving trace and the kernels beyond the step.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on
a bounded sample of the headline workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "Gpair-evals/s fused raytrace+GP kernel matvec (fwd, fwd+bwd); p50/p99 req latency"
FILL_PAIRS = 8_000_000_000  # pairs per iteration that fill the GPU (about a 384-px request at 2x2 on 128^2)
UNIT = "Gpair/s"
SM_MAX_MHZ_DEFAULT = 2070.0
# Work per point-subhalo pair, counted operation by operation from the
# kernels' source (FP32 lanes; packed f32x2 operations count 2 lanes for 2
# pairs). Forward, far-side closed form (x^2 >= 1.05): 2 offsets, 3 for R^2
# and x^2, 22 for the shared far terms (arctan polynomial 12; the record's
# (tau^2-1)/tau carries the ln(2)/2 of the log), 7 for the mass bracket, 2 to
# accumulate both components, 1.25 for the Kahan fold after every 8
# subhalos; MUFU: 2 rsqrt, 1 rcp, 1 lg2. Forward, far-field series to y^K
# (a subhalo whose series radius clears the CTA's whole tile): 2 + 3, 1 for
# y^2, K - 2 + 1 for the Horner steps, 2 for m = A y^2 Q, 2 to accumulate
# and 0.31 for the Kahan fold after every 32 subhalos; MUFU: 1 rsqrt.
# Backward, subhalos near the tile's points (far-side closed form): 5 + 22,
# 12 for the G and H brackets, 11 for the four subhalo sums (their constant
# factors, 1/theta_s^2 of the q terms included, applied once per fold or
# slot), 0.3 for the Kahan folds; 4 MUFU. Backward, subhalos whose gradient
# series radius clears every point of the tile (far-field series of G and of
# x dG/dx to y^K): 5, 1 for y^2, 2 (K - 2) for the two Horner chains, 2 + 2
# for G and x dG/dx, 10 for the four sums, 0.3 for the folds; 1 MUFU.
# Culled reductions over explicit points (the self-kernel), per evaluated
# pair: forward 2 differences, the squared distance (2), the scale (1) and
# the accumulation (1); self-kernel backward the same 6 before the
# accumulation, then k w and k g (2) and 7 accumulations (A, B, C of v; A, B
# of g). One MUFU.EX2 each.
CULL_FWD_MUFU, CULL_FWD_LANES = 1, 6.0
CULL_SELF_MUFU, CULL_SELF_LANES = 1, 14.0
RT_MUFU, RT_LANES = 4, 37.3
VJ_MUFU, VJ_LANES = 4, 50.3
SER_MUFU = 1
# series degrees K and the x^2 / max(tau^2, 4) from which each serves a
# whole CTA (fewest terms first)
RT_DEGREES = ((3, 6400.0), (4, 1024.0), (5, 324.0), (7, 64.0), (9, 36.0))
VJ_DEGREES = ((3, 6400.0), (4, 1024.0), (5, 324.0), (7, 64.0))


def rt_ser_lanes(k: int) -> float:
    return 9.31 + k


def vj_ser_lanes(k: int) -> float:
    return 20.3 + 2 * (k - 2)


# The backward's local expansion of a far subhalo about a tile's centre: 15
# to 36 terms (by the tile's size against its distance) of 40 FP32
# operations each (7 series terms of the coefficient, 4 real parts of
# products with the tile's moments, the next power of u) and 30 to set up,
# per tile and subhalo, whatever the tile's point count; its moments add
# about 31 operations per point and term, once per tile (not counted).
VJ_EXP_LANES_PER_TERM = 40.0


def _grid_axes(g):
    w, hgt = g.nx * g.ss, g.ny * g.ss
    h = g.pix / g.ss
    xs = (np.arange(w) - (w - 1) / 2) * h + g.cx
    ys = (np.arange(hgt) - (hgt - 1) / 2) * h + g.cy
    return w, hgt, xs, ys


def _degree_shares(p, boxes, counts, degrees, expand=False) -> dict:
    """Share of the point-subhalo pairs by the series degree that serves a
    CTA's whole box (x_lo, y_lo, x_hi, y_hi) of `counts` points; 0: the
    closed forms. With `expand`, the pairs of a far subhalo whose distance
    from the box's centre is at least 12.5 half-diagonals go to the key
    "expansion" (the ray-trace backward's local expansion)."""
    sub = p.sub.astype(np.float64)
    its2 = 1.0 / sub[:, 3] ** 2
    m = np.maximum(sub[:, 4] ** 2, 4.0)
    tot = {k: 0.0 for k, _ in degrees}
    tot[0] = 0.0
    tot["expansion"] = 0.0
    exp_lanes = 0.0
    for c in range(0, len(boxes), 1024):
        bx, cn = boxes[c:c + 1024], counts[c:c + 1024].astype(np.float64)
        dx = np.maximum(np.maximum(bx[:, 0, None] - sub[None, :, 0], sub[None, :, 0] - bx[:, 2, None]), 0.0)
        dy = np.maximum(np.maximum(bx[:, 1, None] - sub[None, :, 1], sub[None, :, 1] - bx[:, 3, None]), 0.0)
        x2 = (dx * dx + dy * dy) * its2[None, :] / m[None, :]
        left = np.ones(x2.shape, dtype=bool)
        if expand:
            hd2 = 0.25 * ((bx[:, 2] - bx[:, 0]) ** 2 + (bx[:, 3] - bx[:, 1]) ** 2)
            cx = 0.5 * (bx[:, 0] + bx[:, 2])[:, None] - sub[None, :, 0]
            cy = 0.5 * (bx[:, 1] + bx[:, 3])[:, None] - sub[None, :, 1]
            c2 = cx * cx + cy * cy
            hit = (x2 >= degrees[-1][1]) & (hd2[:, None] <= 0.0064 * c2) & (cn[:, None] <= 2048)
            tot["expansion"] += float((hit.sum(1) * cn).sum())
            # terms of the expansion's order: 15, 21, 28 or 36 for (half-diagonal / |c|) up to 0.01, 0.03, 0.05, 0.08
            r2 = hd2[:, None] / c2
            terms = np.where(r2 <= 1e-4, 15, np.where(r2 <= 9e-4, 21, np.where(r2 <= 2.5e-3, 28, 36)))
            exp_lanes += float(np.sum(np.where(hit, VJ_EXP_LANES_PER_TERM * terms + 30.0, 0.0)))
            left &= ~hit
        for k, r2 in degrees:
            hit = left & (x2 >= r2)
            tot[k] += float((hit.sum(1) * cn).sum())
            left &= ~hit
        tot[0] += float((left.sum(1) * cn).sum())
    n = float(counts.sum()) * len(sub)
    out = {k: v / n for k, v in tot.items()}
    out["expansion_lanes"] = exp_lanes / n
    return out


def raytrace_cost(p):
    """(MUFU, FP32 lanes) per point-subhalo pair of the forward ray-trace on
    a pixel grid, and the pairs' shares by series degree: a CTA takes a
    16 x 16 tile of pixels, a subhalo takes the series of the degree that
    serves the whole tile, the others the far-side closed form."""
    w, hgt, xs, ys = _grid_axes(p.xgrid)
    tw, th = (w + 15) // 16, (hgt + 15) // 16
    ty, tx = np.divmod(np.arange(tw * th), tw)
    r0, c0 = ty * 16, tx * 16
    r1, c1 = np.minimum(r0 + 16, hgt) - 1, np.minimum(c0 + 16, w) - 1
    boxes = np.stack([xs[c0], ys[r0], xs[c1], ys[r1]], 1)
    sh = _degree_shares(p, boxes, (r1 - r0 + 1) * (c1 - c0 + 1), RT_DEGREES)
    mufu = sh[0] * RT_MUFU + (1 - sh[0]) * SER_MUFU
    lanes = sh[0] * RT_LANES + sum(sh[k] * rt_ser_lanes(k) for k, _ in RT_DEGREES)
    return mufu, lanes, sh


def vjp_bands(nblk: int, w: int, hgt: int) -> int:
    """Bands of image rows of the ray-trace backward's CTA tiles: the divisor
    R of nblk whose tiles are closest to square, preferring equal bands."""
    best, best_s = 1, float("inf")
    for r in range(1, min(nblk, hgt) + 1):
        if nblk % r:
            continue
        th, tw = hgt / r, w * r / nblk
        sc = abs(float(np.log(th / tw))) + 2.0 * (((hgt + r - 1) // r) / th - 1.0)
        if sc < best_s:
            best, best_s = r, sc
    return best


def vjp_phases(n: int, nblk: int, n_sub: int) -> int:
    """Slots per subhalo of the ray-trace backward: 1 when n_sub slots waste
    at most 5 % of the last 128 threads, else the P in [1, 8] whose n_sub P
    wastes the fewest of them, keeping 128 points per slot (the local
    expansion needs P = 1)."""
    per = -(-n // nblk)
    if -(-n_sub // 128) * 128 <= 1.05 * n_sub:
        return 1
    best, best_w = 1, float("inf")
    for P in range(1, 9):
        if P > 1 and per // P < 128:
            break
        sl = n_sub * P
        w = (-(-sl // 128) * 128) / sl
        if w < best_w - 1e-9:
            best, best_w = P, w
    return best


def vjp_cost(p, nblk: int):
    """(MUFU, FP32 lanes) per point-subhalo pair of the ray-trace backward on
    a pixel grid, and the pairs' shares by series degree: nblk tiles (bands
    of rows, each band's points split in column-major order), a subhalo takes
    the gradient series of the degree that serves the whole tile's bounding
    box, the others the far-side closed form."""
    w, hgt, xs, ys = _grid_axes(p.xgrid)
    bands = vjp_bands(nblk, w, hgt)
    per = nblk // bands
    b, c = np.divmod(np.arange(nblk, dtype=np.int64), per)
    row0 = b * hgt // bands
    rows = (b + 1) * hgt // bands - row0
    nb = rows * w
    u0, u1 = c * nb // per, (c + 1) * nb // per
    col0, col1 = u0 // rows, (u1 - 1) // rows
    one = col0 == col1
    rlo = np.where(one, u0 % rows, 0)
    rhi = np.where(one, (u1 - 1) % rows, rows - 1)
    boxes = np.stack([xs[col0], ys[row0 + rlo], xs[col1], ys[row0 + rhi]], 1)
    sh = _degree_shares(p, boxes, u1 - u0, VJ_DEGREES, expand=vjp_phases(p.n, nblk, len(p.sub)) == 1)
    mufu = sh[0] * VJ_MUFU + sum(sh[k] for k, _ in VJ_DEGREES) * SER_MUFU
    lanes = (sh[0] * VJ_LANES + sum(sh[k] * vj_ser_lanes(k) for k, _ in VJ_DEGREES) + sh["expansion_lanes"])
    return mufu, lanes, sh


def _shares_text(sh: dict) -> str:
    ser = ", ".join(f"y^{k}: {v:.3f}" for k, v in sh.items() if isinstance(k, int) and k)
    exp = f"local expansion: {sh['expansion']:.3f}, " if "expansion" in sh else ""
    return exp + ser + f"; closed form: {sh[0]:.3f}"


def vjp_tiles(dev, n: int) -> int:
    """Tiles (CTAs) of the ray-trace backward for n points, with 4 CTAs
    resident per SM (128 registers and 45 KB of shared memory each): one per
    128 points below a full wave, above it whole waves (at most 8) of tiles
    of at least 512 points."""
    import torch

    slots = 4 * torch.cuda.get_device_properties(dev).multi_processor_count
    nb = (n + 127) // 128
    if nb < slots:
        return nb
    return min(max(n // (slots * 512), 1), 8) * slots


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-extensions", action="store_true", help="skip timing the kernels beyond the fused step")
    ap.add_argument("--no-graph", action="store_true", help="launch the step's kernels directly, not from a CUDA graph")
    ap.add_argument("--profile", action="store_true",
                    help="headline step only, direct launches: W warm-up and K timed steps, then exit (profiler runs)")
    ap.add_argument("--profile-side", type=int, default=800,
                    help="with --profile: pixels per side of the large workload's image (800: the workload itself; "
                         "smaller sides give profiler captures of the same recipe)")
    ap.add_argument("--profile-layer", action="store_true",
                    help="the image-plane layer's windowed forward and backward only (400x400 ray-traced pixels "
                         "against themselves, l = 0.05 arcsec): W warm-up and K timed calls, then exit (profiler runs)")
    ap.add_argument("--serving-requests", type=int, default=32)
    ap.add_argument("--serving-iters", type=int, default=50)
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target oracle CPU time for cpu_baseline")
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="target oracle CPU time of a whole --impl reference run (each step 0.2 to 2 s)")
    return ap.parse_args()


def measured_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu capture, if the kernel's
    sources are unchanged since it was taken (else None)."""
    import hashlib
    try:
        d = json.loads((ROOT / "profiles" / "traffic.json").read_text())[kernel]
        h = hashlib.sha256()
        for f in d["csrc_files"]:
            h.update((ROOT / "paper_2105_09465_gb300" / "csrc" / f).read_bytes())
        return d["dram_bytes_per_launch"] if h.hexdigest() == d["csrc_sha256"] else None
    except Exception:
        return None


def workload_config(p) -> dict:
    return {"workload": f"realistic: {p.xgrid.nx}x{p.xgrid.ny} image, {p.xgrid.ss}x{p.xgrid.ss} supersampling "
                        f"({p.n} points), power-law lens + shear + {len(p.sub)} tNFW subhalos, "
                        f"{p.ygrid.nx}x{p.ygrid.ny} grid inducing points ({p.m})",
            "n_points": p.n, "m_inducing": p.m, "n_subhalos": int(len(p.sub)), "pairs_per_step": p.pairs,
            "lengthscale": p.lengthscale, "variance": p.variance,
            "l2": "flushed between timed steps (256 MiB device write outside the timed region)"}


def large_config(p) -> dict:
    return {"workload": f"large: {p.xgrid.nx}x{p.xgrid.ny} image, {p.xgrid.ss}x{p.xgrid.ss} supersampling "
                        f"({p.n} points), power-law lens + shear + {len(p.sub)} tNFW subhalos "
                        f"(1e6-1e10 Msun), self-kernel of the ray-traced points",
            "n_points": p.n, "n_subhalos": int(len(p.sub)), "pairs_per_step": p.pairs,
            "lengthscale": p.lengthscale, "variance": p.variance,
            "l2": "inputs larger than L2 and a 256 MiB device write between timed steps (outside the timed region)"}


# --------------------------------------------------------------------------
class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def start(self):
        try:
            self._proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                           "--format=csv,noheader,nounits", "-lms", "100"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._proc = None
            return

        def run():
            for line in self._proc.stdout:
                self.rows.append([c.strip() for c in line.split(",")])
        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()

    def stop(self) -> dict:
        if getattr(self, "_proc", None) is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        if self._t:
            self._t.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# --------------------------------------------------------------------------
class OracleSampler:
    """The FP64 oracle on row samples of workload p: ray-trace, kernel
    reduction, reduction gradients and ray-trace gradients of the sampled
    rows against all inducing points (the same per-pair work as the GPU
    step)."""

    def __init__(self, p, g=None):
        import oracle

        oracle.build()
        self.oracle, self.p = oracle, p
        self.xi_all = oracle.grid_points(*p.xgrid.astuple())
        self.yg = oracle.grid_points(*p.ygrid.astuple())
        self.rng = np.random.default_rng(0)
        self.g = self.rng.standard_normal(p.n) if g is None else g
        self.run(self.rng.choice(p.n, 64, replace=False))  # warm-up (library load, page-in)

    def run(self, rows) -> float:
        o, p = self.oracle, self.p
        t = time.perf_counter()
        xi = self.xi_all[rows]
        _, b = o.raytrace(xi, p.lens.astuple(), p.sub)
        o.kernel_matvec(b, self.yg, p.v, p.lengthscale, p.variance)
        R = o.kernel_matvec_vjp(b, self.yg, p.v, p.lengthscale, p.variance, self.g[rows])
        o.raytrace_vjp(xi, p.lens.astuple(), p.sub, R["d_x"])
        return time.perf_counter() - t

    def rows_for(self, seconds: float) -> int:
        """Rows that take about `seconds` (from a 256-row calibration)."""
        dt = self.run(self.rng.choice(self.p.n, 256, replace=False))
        return int(min(self.p.n, max(256, 256 * seconds / max(dt, 1e-3))))

    def step(self, k: int) -> float:
        return self.run(self.rng.choice(self.p.n, k, replace=False))

    def describe(self, k: int, dt: float) -> str:
        return (f"{k} random rows of the workload x all {self.p.m} inducing points ({k * self.p.m:.3e} pairs): "
                f"ray-trace, reduction, reduction gradients and ray-trace gradients, {dt:.1f} s")


class LargeOracleSampler:
    """The FP64 oracle on row samples of the large workload: per sampled row,
    the ray-trace through the lens and 2000 subhalos, the self-kernel row
    against all 2.56M points (out, d_v and both roles of d_x), and the
    ray-trace gradients of that row. The rows' sources are the pixels
    ray-traced through the main lens and the shear (the subhalos move them by
    milli-arcseconds, which leaves the reduction's cost unchanged); that
    ray-trace is a fixed cost of the full problem counted once per step in
    its share n_sample / n."""

    def __init__(self, p, g=None):
        import oracle

        oracle.build()
        self.oracle, self.p = oracle, p
        self.xi_all = oracle.grid_points(*p.xgrid.astuple())
        self.rng = np.random.default_rng(0)
        self.g = self.rng.standard_normal(p.n) if g is None else g
        _, self.beta_src = oracle.raytrace(self.xi_all, p.lens.astuple(), None)
        self.run(self.rng.choice(p.n, 16, replace=False))  # warm-up

    def run(self, rows) -> float:
        o, p = self.oracle, self.p
        t = time.perf_counter()
        xi = self.xi_all[rows]
        o.raytrace(xi, p.lens.astuple(), p.sub)
        R = o.self_vjp_rows(self.beta_src, p.v, self.g, p.lengthscale, p.variance, rows)
        o.raytrace_vjp(xi, p.lens.astuple(), p.sub, R["d_x"])
        return time.perf_counter() - t

    def rows_for(self, seconds: float) -> int:
        dt = self.run(self.rng.choice(self.p.n, 64, replace=False))
        return int(min(self.p.n, max(64, 64 * seconds / max(dt, 1e-3))))

    def step(self, k: int) -> float:
        return self.run(self.rng.choice(self.p.n, k, replace=False))

    def describe(self, k: int, dt: float) -> str:
        return (f"{k} random rows of the large workload x all {self.p.n} points ({k * self.p.n:.3e} pairs): "
                f"ray-trace (2000 subhalos), self-kernel row with d_v and d_x, ray-trace gradients, {dt:.1f} s; "
                f"extrapolated to all {self.p.n} rows")


def cpu_sample_large(p, seconds: float, g=None, one_core_seconds: float = 0.0) -> dict:
    """Oracle throughput on a bounded sample (about `seconds` of CPU work) on
    all host cores, and, with one_core_seconds > 0, on one core."""
    S = LargeOracleSampler(p, g)
    k = S.rows_for(seconds)
    total, done = 0.0, 0
    while total < 0.8 * seconds and done < p.n:
        total += S.step(k)
        done += k
    out = {"value": done * p.n / total / 1e9, "unit": UNIT, "cores": S.oracle.num_threads(), "kind": "oracle",
           "sample": S.describe(done, total), "seconds": total}
    if one_core_seconds > 0:
        cores = S.oracle.num_threads()
        S.oracle.set_num_threads(1)
        try:
            k1 = S.rows_for(one_core_seconds)
            t1 = S.step(k1)
        finally:
            S.oracle.set_num_threads(cores)
        out["one_core"] = {"value": k1 * p.n / t1 / 1e9, "unit": UNIT, "cores": 1,
                           "sample": S.describe(k1, t1)}
    return out


def cpu_sample(p, seconds: float, g=None) -> dict:
    """Oracle throughput on a bounded sample of about `seconds` of CPU work."""
    S = OracleSampler(p, g)
    k = S.rows_for(seconds)
    total, done = 0.0, 0
    while total < 0.8 * seconds and done < p.n:
        total += S.step(k)
        done += k
    pairs = done * p.m
    return {"value": pairs / total / 1e9, "unit": UNIT, "cores": S.oracle.num_threads(), "kind": "oracle",
            "sample": S.describe(done, total), "seconds": total}


# --------------------------------------------------------------------------
def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores. Each
    of the W + K steps is a bounded row sample of the large workload (the same
    rows count every step, about ref_seconds / (W + K) seconds each); the K
    timed steps give the whole-job rate, pairs over seconds."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2105_09465_gb300 import workloads as W

    p = W.large()
    S = LargeOracleSampler(p)
    per_step = min(2.0, max(0.2, args.ref_seconds / max(1, args.steps + args.warmup)))
    k = S.rows_for(per_step)
    for _ in range(args.warmup):
        S.step(k)
    secs = [S.step(k) for _ in range(args.steps)]
    total = float(np.sum(secs))
    val = k * p.n * len(secs) / total / 1e9
    ms = p.pairs / (val * 1e9) * 1e3
    sample = (f"each step {k} random rows of the large workload x all {p.n} points ({k * p.n:.3e} pairs, "
              f"{total / len(secs):.2f} s): ray-trace (2000 subhalos), self-kernel row with d_v and d_x, ray-trace "
              f"gradients; ms_per_step is the full workload at this rate")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": large_config(p),
            "cpu_baseline": {"kind": "oracle", "cores": S.oracle.num_threads(), "sample": sample, "value": val,
                             "unit": UNIT},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------------
def run_serving(n_req: int, iters: int) -> dict:
    """Serving trace (sides 64-512 px at 2x2, 0-500 subhalos, 128x128 inducing
    grid, `iters` fwd+bwd+update iterations each) through the session engine:
    all requests at t = 0 with continuous batching (16 slots) and one at a
    time (1 slot, per-request launches), then Poisson arrivals at 70 % of the
    measured batched capacity through both."""
    import threading as th

    from paper_2105_09465_gb300 import workloads as W
    from paper_2105_09465_gb300.serving import Session

    trace = W.serving_trace(seed=3, n_requests=n_req, iters=iters)
    rng = np.random.default_rng(33)
    datas = [rng.standard_normal(r["problem"].n).astype(np.float32) for r in trace]
    pairs = sum(r["problem"].n * r["problem"].m for r in trace) * iters
    step = 1e-3

    def pct(lat):
        return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(np.mean(lat))}

    out = {"trace": f"{n_req} requests (seed 3): square images of side U{{64,128,256,384,512}} px at 2x2, "
                    f"0-500 tNFW subhalos, 128x128 inducing grid, {iters} iterations of ray-trace + reduction + "
                    f"backward + update each; {pairs:.3e} pairs of forward+backward work",
           "unit": UNIT}
    with Session(max_slots=2) as S:  # warm-up (module load, pools)
        p = trace[0]["problem"]
        S.poll(S.submit(p, datas[0], 2, step))
    # three engines: 16 slots; one request at a time; 16 slots admitted only
    # while the active requests' pairs per iteration stay within FILL_PAIRS
    # (requests that fill the GPU alone run alone, small ones share it)
    modes = (("batched", 16, 0), ("unbatched", 1, 0), ("filled", 16, FILL_PAIRS))
    for mode, slots, fill in modes:
        with Session(max_slots=slots, fill_pairs=fill) as S:
            t0 = time.perf_counter()
            ts = [S.submit(r["problem"], d, iters, step) for r, d in zip(trace, datas)]
            res = [S.poll(t, timeout_s=600, want=()) for t in ts]
            wall = time.perf_counter() - t0
            st = S.stats()
        assert all(r.status == 0 for r in res), [r.status for r in res]
        lat = [r.latency for r in res]
        out[mode] = {"value": pairs / wall / 1e9, "wall_s": wall, "req_per_s": n_req / wall,
                     "batched_launches": st["launches"], "iterations": st["iterations"], **pct(lat)}
    out["speedup_batched_vs_unbatched"] = out["batched"]["value"] / out["unbatched"]["value"]
    # Poisson arrivals (the serving workload's stream, its rate scaled to this
    # GPU: 70 % of the measured batched capacity), the same arrival times for
    # the batched engine and for one request at a time
    rate = 0.7 * out["batched"]["req_per_s"]
    arr = np.cumsum(np.random.default_rng(5).exponential(1.0 / rate, n_req))
    for mode, slots, fill in modes:
        with Session(max_slots=slots, fill_pairs=fill) as S:
            tickets = [None] * n_req
            t0 = time.perf_counter()

            def feeder():
                for k, (r, d) in enumerate(zip(trace, datas)):
                    dt = arr[k] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                    tickets[k] = S.submit(r["problem"], d, iters, step)

            f = th.Thread(target=feeder)
            f.start()
            res = []
            for k in range(n_req):
                while tickets[k] is None:
                    time.sleep(0.0005)
                res.append(S.poll(tickets[k], timeout_s=600, want=()))
            f.join()
            wall = time.perf_counter() - t0
        assert all(r.status == 0 for r in res), [r.status for r in res]
        out[f"poisson_70pct_{mode}"] = {"rate_req_per_s": rate, "value": pairs / wall / 1e9, "wall_s": wall,
                                        **pct([r.latency for r in res])}
    out["speedup_filled_vs_unbatched"] = out["filled"]["value"] / out["unbatched"]["value"]
    out["latency_note"] = ("most requests of this trace fill the GPU alone, so sharing it among 16 stretches each "
                           "one (all-at-once p50 above one-at-a-time FIFO's); admission by pairs per iteration "
                           "batches only the small ones")
    return out


def event_time(fn, n, stream, flush):
    """Mean CUDA-event time (ms) of fn() over n calls, L2 flushed before each."""
    import torch
    evs = []
    for k in range(n):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in evs]))


def kernel_time(fn, n, stream, flush, kernel):
    """Mean device time (ms) of one library kernel alone over n calls of fn
    (the library's launch timer: CUDA events around that kernel's launches on
    its stream), and the mean CUDA-event time of the whole call."""
    from paper_2105_09465_gb300 import api
    api.kernel_timer_enable(True)
    call_ms = event_time(fn, n, stream, flush)
    api.kernel_timer_enable(False)
    cnt, tot, dropped = api.kernel_timer_read(kernel)
    if cnt != n or dropped:
        raise RuntimeError(f"launch timer saw {cnt} launches of {kernel} for {n} calls ({dropped} dropped)")
    return tot / cnt, call_ms


def run_extensions(p, dev, rates, sm_max, flush, stream) -> dict:
    """Kernels beyond the fused step, each timed alone on realistic-shaped
    inputs (same lens, same inducing grid): windowed transmission over the
    ray-traced pixel centres, three image-plane layers, k-NN density, lens
    Jacobian, likelihood and ELBO terms."""
    import torch

    from paper_2105_09465_gb300 import api, workloads as W

    ex2, fma, nsm = rates["ex2_per_clk"], rates["ffma2_lanes_per_clk"], rates["sm_count"]

    def roof(pairs, ms, n_ex2, lanes):
        per_clk = min(ex2 / n_ex2, fma / lanes)
        peak = per_clk * nsm * sm_max * 1e6 / 1e9
        ach = pairs / (ms * 1e-3) / 1e9
        return {"ms": ms, "achieved": ach, "peak": peak, "unit": UNIT, "frac": ach / peak,
                "basis": f"{n_ex2} MUFU.EX2 + {lanes} FP32 lanes per pair"}

    nk = 20
    out = {}
    sub = torch.from_numpy(p.sub).to(dev)
    pix = W.Grid(p.xgrid.nx, p.xgrid.ny, 1, p.xgrid.pix)
    bp = api.lens_raytrace(api.Points(grid=pix, lens=p.lens, sub=sub))
    z = api.pixel_shapes(bp, pix.nx, pix.ny)
    s = api.Points(grid=p.ygrid)
    v = torch.from_numpy(p.v).to(dev)
    ms = event_time(lambda: api.gp_windowed_matvec(bp, z, s, v, p.lengthscale), nk, stream, flush)
    out["windowed_matvec<grid>"] = dict(roof(pix.n * p.m, ms, 1, 3), n=pix.n, m=p.m,
                                        workload=f"{pix.nx}x{pix.ny} ray-traced pixel centres with their "
                                                 f"window covariances x {p.ygrid.nx}x{p.ygrid.ny} grid")
    out["pixel_shapes"] = {"ms": event_time(lambda: api.pixel_shapes(bp, pix.nx, pix.ny), nk, stream, flush)}
    # the image-plane layer: the pixels' own windowed reduction (explicit
    # sources = the pixels, in their image layout), at the workloads' 0.05
    # arcsec and at the paper's narrowest image-plane kernel, 2 mas; pairs
    # whose exponent is below -126 are skipped, so the roofline counts the
    # evaluated pairs (forward 8 lanes, backward rows 19, columns 14 per pair)
    vp = torch.randn(pix.n, generator=torch.Generator().manual_seed(6)).to(dev)
    gp = torch.randn(pix.n, generator=torch.Generator().manual_seed(7)).to(dev)
    selfp = api.Points(xy=bp, grid=pix)
    for ell in (0.05, 0.002):
        ev = [api.windowed_pairs_evaluated(bp, z, selfp, ell, sw, layout=pix)[0] for sw in (0, 1, 2)]
        ms = event_time(lambda: api.gp_windowed_matvec(bp, z, selfp, vp, ell, layout=pix), nk, stream, flush)
        out[f"windowed_matvec<explicit> image-plane layer l={ell}"] = dict(
            roof(ev[0], ms, 1, 8), n=pix.n, m=pix.n, logical_pairs=pix.n * pix.n, evaluated_pairs=ev[0])
        ms = event_time(lambda: api.gp_windowed_matvec_bwd(bp, z, selfp, vp, ell, gp, layout=pix), nk, stream,
                        flush)
        rr, rc = roof(ev[1], 1.0, 1, 19), roof(ev[2], 1.0, 1, 14)
        bound_ms = ev[1] / (rr["peak"] * 1e9) * 1e3 + ev[2] / (rc["peak"] * 1e9) * 1e3
        out[f"windowed backward (rows + columns) image-plane layer l={ell}"] = {
            "ms": ms, "frac": bound_ms / ms, "evaluated_pairs": {"rows": ev[1], "columns": ev[2]},
            "logical_pairs": 2 * pix.n * pix.n,
            "basis": "time at the FMA bound of both sweeps (19 and 14 lanes per evaluated pair) / measured"}
    # one SVI step of the model at this size: every step on the device, no host wait inside
    from paper_2105_09465_gb300 import svi
    mc = svi.ModelConfig(pixels=pix, source_grid=p.ygrid, sigma_sp=p.lengthscale * 1.4142135, sigma_layers=[0.05],
                         alpha_sp=1.0, alpha_layers=[0.5], noise=0.1, gamma=p.lens.gamma)
    M = p.m
    th = torch.tensor([p.lens.x0, p.lens.y0, p.lens.q, p.lens.phi, p.lens.theta_e, p.lens.g1, p.lens.g2])
    gd = svi.Guide(mu=torch.cat([th, torch.zeros(M)]).to(dev), L=(torch.eye(7) * 1e-3).to(dev),
                   C=torch.zeros((M, 7), device=dev), sd_sp=torch.full((M,), 0.05, device=dev),
                   mu_layers=[torch.zeros(pix.n, device=dev)], sd_layers=[torch.full((pix.n,), 0.01, device=dev)])
    gen = torch.Generator().manual_seed(8)
    data = torch.randn(pix.n, generator=gen).to(dev)
    e_sp = torch.randn(7 + M, generator=gen).to(dev)
    e_l = [torch.randn(pix.n, generator=gen).to(dev)]
    for _ in range(3):
        svi.loss_and_grads(mc, gd, data, e_sp, e_l)
    ms = event_time(lambda: svi.loss_and_grads(mc, gd, data, e_sp, e_l), 5, stream, flush)
    out["svi_step"] = {"ms": ms,
                       "workload": f"{pix.nx}x{pix.ny} pixels, {p.ygrid.nx}x{p.ygrid.ny} source grid, one "
                                   "image-plane layer: draws, ray-trace, both layers, likelihood and every gradient",
                       "timing": "CUDA events around the step on its stream, L2 flushed before each; the drawn lens "
                                 "parameters stay on the device (lens record), so nothing waits on the host"}
    # three image-plane layers (the paper's 10 / 4.47 / 2 mas ratios) on the supersampled points
    beta = api.lens_raytrace(api.Points(grid=p.xgrid, lens=p.lens, sub=sub))
    vl = torch.randn((3, p.m), generator=torch.Generator().manual_seed(5)).to(dev)
    ls = [p.lengthscale, p.lengthscale * 0.447, p.lengthscale * 0.2]
    ms = event_time(lambda: api.gp_kernel_matvec_layers(api.Points(xy=beta), s, vl, ls, [1.0, 0.5, 0.25]), nk,
                    stream, flush)
    out["matvec_layers<grid> x3"] = dict(roof(p.pairs, ms, 3, 10), layers=3,
                                         note="pairs counted once; 3 exponentials per pair")
    # four draws of the three layers' weights in one pass (the exponentials
    # shared) beside four one-draw passes
    vl4 = torch.randn((3, p.m, 4), generator=torch.Generator().manual_seed(9)).to(dev)
    ms4 = event_time(lambda: api.gp_kernel_matvec_layers(api.Points(xy=beta), s, vl4, ls, [1.0, 0.5, 0.25]), nk,
                     stream, flush)
    out["matvec_layers<grid> x3, 4 right-hand sides"] = {
        "ms": ms4, "ms_four_single_passes": 4 * ms, "speedup": 4 * ms / ms4,
        "note": "v (3 layers, m, 4): one exp2 per pair and layer, 4 FMAs"}
    out["knn_density k=20"] = {"ms": event_time(lambda: api.knn_density(beta, 20, lengthscale=p.lengthscale), nk,
                                                stream, flush), "points": p.n}
    qj = api.Points(grid=p.xgrid, lens=p.lens, sub=sub)
    out["lens_jacobian"] = {"ms": event_time(lambda: api.lens_jacobian(qj), nk, stream, flush), "points": p.n,
                            "subhalo_pairs": p.n * len(p.sub)}
    f = torch.randn(p.n, device=dev)
    d = torch.randn(p.xgrid.nx * p.xgrid.ny, device=dev)
    out["gaussian_nll"] = {"ms": event_time(lambda: api.gaussian_nll(f, d, 0.1, grid=p.xgrid), nk, stream, flush),
                           "pixels": int(d.numel()), "subpixels": p.n}
    m3 = 3 * p.n
    mu, sd, eps = torch.randn(m3, device=dev), torch.rand(m3, device=dev) + 0.01, torch.randn(m3, device=dev)
    out["diag_normal_draw+vjp"] = {
        "ms": event_time(lambda: (api.diag_normal_draw(mu, sd, eps, 1.0), api.diag_normal_vjp(mu, sd, eps, 1.0, eps)),
                         nk, stream, flush), "params": m3}
    D, M = 7, p.m
    L = (torch.eye(D) * 0.01).to(dev)
    C = torch.randn((M, D), device=dev) * 0.01
    sd2, e2 = torch.rand(M, device=dev) + 0.01, torch.randn(D + M, device=dev)
    out["partial_mvn_draw+vjp"] = {
        "ms": event_time(lambda: (api.partial_mvn_draw(e2, L, C, sd2, e2), api.partial_mvn_vjp(L, sd2, e2, e2)), nk,
                         stream, flush), "D": D, "M": M}
    return out


def run_profile_layer(args, dev) -> dict:
    """The image-plane layer of the realistic workload (the pixels' own
    windowed reduction, forward then backward) with direct launches: the
    launch sequence a profiler sees."""
    import torch

    from paper_2105_09465_gb300 import api, workloads as W

    p = W.realistic()
    sub = torch.from_numpy(p.sub).to(dev)
    pix = W.Grid(p.xgrid.nx, p.xgrid.ny, 1, p.xgrid.pix)
    bp = api.lens_raytrace(api.Points(grid=pix, lens=p.lens, sub=sub))
    z = api.pixel_shapes(bp, pix.nx, pix.ny)
    gen = torch.Generator().manual_seed(6)
    vp = torch.randn(pix.n, generator=gen).to(dev)
    gp = torch.randn(pix.n, generator=gen).to(dev)
    selfp = api.Points(xy=bp, grid=pix)

    def call():
        api.gp_windowed_matvec(bp, z, selfp, vp, 0.05, layout=pix)
        api.gp_windowed_matvec_bwd(bp, z, selfp, vp, 0.05, gp, layout=pix)

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    return {"profile": "image-plane layer", "ms_per_call": e0.elapsed_time(e1) / max(args.steps, 1),
            "workload": f"{pix.nx}x{pix.ny} ray-traced pixels with their windows, self sources, l = 0.05"}


def run_realistic(args, dev, rates, clk) -> dict:
    """The realistic workload's training step (grid inducing points, row
    moments in the forward, the d_v-only sweep in the backward) with its
    kernel table, timed like the headline step (one GPU)."""
    import torch

    from paper_2105_09465_gb300 import api, replicas, workloads as W

    world = 1
    dist = None
    p = W.realistic()
    g_np = np.random.default_rng(100).standard_normal(p.n).astype(np.float32)
    sub = torch.from_numpy(p.sub).to(dev)
    v = torch.from_numpy(p.v).to(dev)
    g = torch.from_numpy(g_np).to(dev)
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=sub)
    s = api.Points(grid=p.ygrid)
    want = ["v", "lengthscale", "variance", "lens", "sub"]
    out = torch.empty(p.n, dtype=torch.float32, device=dev)
    beta_buf = torch.empty((p.n, 2), dtype=torch.float32, device=dev)
    mom = torch.empty((4, p.n), dtype=torch.float32, device=dev)
    ws = torch.empty(max(api.train_workspace_size(q, s), 1), dtype=torch.uint8, device=dev)
    bws = torch.empty(1, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    grads = {}

    # training step: the forward also leaves the row moments, the backward
    # sweeps the pairs once more for d_v only
    def fwd():
        api.gp_kernel_matvec_train(q, s, v, p.lengthscale, p.variance, out=out, beta=beta_buf, moments=mom,
                                   workspace=ws)

    def bwd():
        nonlocal bws
        G = api.gp_kernel_matvec_bwd(q, s, v, p.lengthscale, p.variance, g, want=want, workspace=bws, beta=beta_buf,
                                     moments=mom)
        grads.update(G)

    def step():
        fwd()
        bwd()

    # size the backward workspace once (the call allocates it on first use)
    bws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    from paper_2105_09465_gb300 import abi as _abi
    import ctypes
    cq, _k1 = api.to_c_points(q)
    cs, _k2 = api.to_c_points(s)
    gr = _abi.lr_grads()
    # the size query reads only which gradients are requested; real buffers
    # stand for them so that no argument is a made-up address
    _req = [torch.empty(64, dtype=torch.float64, device=dev) for _ in range(7)]
    (gr.d_v, gr.d_lengthscale, gr.d_variance, gr.d_lens, gr.d_sub, gr.beta_in,
     gr.moments_in) = [t.data_ptr() for t in _req]
    b = ctypes.c_size_t(0)
    _abi.check(_abi.load().lr_matvec_bwd_workspace_size(ctypes.byref(cq), ctypes.byref(cs), 1, ctypes.byref(gr),
                                                         ctypes.byref(b)), "lr_matvec_bwd_workspace_size")
    bws = torch.empty(max(int(b.value), 1), dtype=torch.uint8, device=dev)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # the step's launches captured once into a CUDA graph and replayed (no
    # host launch overhead between kernels); --no-graph launches them directly
    run_step = step
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        torch.cuda.synchronize()
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        run_step = graph.replay

    # ---- timed region: device-resident inputs, forward + backward per step
    n_steps = max(20, min(args.steps, 200))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
    torch.cuda.synchronize()
    for k in range(n_steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        run_step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = replicas.max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), dev)
    value = replicas.aggregate_rate(p.pairs, ms * 1e-3, world) / 1e9
    nk = max(5, min(args.steps, 50))
    fwd_ms = event_time(fwd, nk, stream, flush)
    bwd_ms = event_time(bwd, nk, stream, flush)

    # ---- where the step's time goes: the launch timer around each heavy
    # kernel over nk directly launched steps
    api.kernel_timer_enable(True)
    direct_ms = event_time(step, nk, stream, flush)
    api.kernel_timer_enable(False)
    breakdown = {}
    for kname in ("raytrace", "train_rows", "dv_rows", "raytrace_vjp"):
        cnt, tot, _ = api.kernel_timer_read(kname)
        breakdown[kname] = tot / cnt if cnt else None
    breakdown["step (direct launches, timer on)"] = direct_ms
    breakdown["note"] = ("each kernel's own span (events on its stream); the backward's d_v branch (dv_rows) runs on "
                         "a side stream concurrently with the row gradients and raytrace_vjp, so the spans overlap "
                         "and do not add up to the step")

    # ---- kernels in isolation (same launch configuration as inside the step)
    # Each entry: (ms, pairs, pairs per SM clock at the binding pipe, note, in the step?).
    beta = api.lens_raytrace(q)
    qx = api.Points(xy=beta, grid=p.xgrid)  # the ray-traced pixels, in the step's row-block layout
    # pairs the grid kernels evaluate: the others are exactly zero in FP32 and left out
    ev = {r: api.grid_pairs_evaluated(beta, p.xgrid, p.ygrid, p.lengthscale, r) for r in (512, 1024)}
    ws2 = torch.empty(max(api.train_workspace_size(qx, s), 1), dtype=torch.uint8, device=dev)
    ws3 = torch.empty(max(api.matvec_workspace_size(qx, s), 1), dtype=torch.uint8, device=dev)
    mom2 = torch.empty((4, p.n), dtype=torch.float32, device=dev)
    dbeta = torch.from_numpy(np.random.default_rng(7).standard_normal((p.n, 2)).astype(np.float32)).to(dev)
    kern = {}
    kern["bwd_rows_kernel<grid, split> (training forward: out + row moments)"] = (
        *kernel_time(lambda: api.gp_kernel_matvec_train(qx, s, v, p.lengthscale, p.variance, out=out, moments=mom2,
                                                        workspace=ws2), nk, stream, flush, "train_rows"),
        ev[512], 1, 4.6, "pairs: 1 MUFU.EX2 + 4.6 FP32 lanes each (split exponent: 4 per pair, 0.56 "
        "per-sub-segment moment conversion)", True)
    kern["dv_rows_kernel<split> (backward: d_v)"] = (
        *kernel_time(lambda: api.gp_kernel_matvec_bwd(qx, s, v, p.lengthscale, p.variance, g, want=["v"],
                                                      moments=mom2), nk, stream, flush, "dv_rows"),
        ev[1024], 1, 2.1, "pairs: 1 MUFU.EX2 + 2.1 FP32 lanes each (split exponent: 2 per pair, 0.12 d_v "
        "reduce-scatter)", True)
    kern["matvec_kernel<grid> (inference forward, not in the step)"] = (
        *kernel_time(lambda: api.gp_kernel_matvec(qx, s, v, p.lengthscale, p.variance, out=out, workspace=ws3), nk,
                     stream, flush, "matvec"),
        ev[1024], 1, 2.0, "pairs: 1 MUFU.EX2 + 2 FP32 lanes each (split exponent)", False)
    kern["bwd_rows_kernel<grid, split, fused d_v> (backward without moments, not in the step)"] = (
        *kernel_time(lambda: api.gp_kernel_matvec_bwd(qx, s, v, p.lengthscale, p.variance, g, want=["x", "v"]), nk,
                     stream, flush, "bwd_rows"),
        ev[1024], 1, 5.7, "pairs: 1 MUFU.EX2 + 5.7 FP32 lanes each (split exponent: 5 per pair, 0.56 "
        "per-sub-segment moments, 0.12 d_v reduce-scatter)", False)
    rt_ms, rt_call_ms = kernel_time(lambda: api.lens_raytrace(q), nk, stream, flush, "raytrace")
    vjp_ms, vjp_call_ms = kernel_time(lambda: api.lens_raytrace_vjp(q, dbeta), nk, stream, flush, "raytrace_vjp")
    # the ray-trace kernels' unit is the point-subhalo pair; counts are those
    # of the far-side tNFW form that nearly every pair takes
    sub_pairs = p.n * len(p.sub)
    rt_mufu, rt_lanes, rt_sh = raytrace_cost(p)
    kern["raytrace_kernel<tNFW> (forward ray-trace; unit: point-subhalo pair)"] = (
        rt_ms, rt_call_ms, sub_pairs, rt_mufu, rt_lanes,
        f"pairs: {rt_mufu:.2f} MUFU + {rt_lanes:.1f} FP32 lanes each on average; shares of the pairs by the "
        f"far-field series degree that serves the CTA's tile ({SER_MUFU} MUFU + 9.31 + K lanes) and the far-side "
        f"closed form ({RT_MUFU} MUFU + {RT_LANES} lanes): {_shares_text(rt_sh)}; the SPLE and shear terms, once "
        "per point, are not counted", True)
    vj_mufu, vj_lanes, vj_sh = vjp_cost(p, vjp_tiles(dev, p.n))
    kern["raytrace_vjp_kernel<tNFW> (ray-trace backward; unit: point-subhalo pair)"] = (
        vjp_ms, vjp_call_ms, sub_pairs, vj_mufu, vj_lanes,
        f"pairs: {vj_mufu:.2f} MUFU + {vj_lanes:.1f} FP32 lanes each on average; shares of the pairs by the "
        f"degree of the series of G and x dG/dx that serves the CTA's tile ({SER_MUFU} MUFU + 20.3 + 2 (K - 2) "
        f"lanes) and the far-side closed form ({VJ_MUFU} MUFU + {VJ_LANES} lanes): {_shares_text(vj_sh)}; the "
        "per-point SPLE and shear gradient terms are not counted", True)

    # ---- end to end through the public API with host buffers
    v_host = torch.from_numpy(p.v).pin_memory()
    g_host = torch.from_numpy(g_np).pin_memory()
    sub_host = torch.from_numpy(p.sub).pin_memory()
    out_host = torch.empty(p.n, dtype=torch.float32).pin_memory()
    dv_host = torch.empty(p.m, dtype=torch.float32).pin_memory()
    dl_host = torch.empty(7, dtype=torch.float64).pin_memory()
    ds_host = torch.empty((len(p.sub), 4), dtype=torch.float64).pin_memory()
    sc_host = torch.empty(2, dtype=torch.float64).pin_memory()
    v_d, g_d, sub_d = torch.empty_like(v), torch.empty_like(g), torch.empty_like(sub)
    qe = api.Points(grid=p.xgrid, lens=p.lens, sub=sub_d)

    # the two large transfers overlap the compute on a second stream: dL/dout
    # (needed only by the backward) comes in during the forward, and out goes
    # back during the backward; events order them against the step
    copy_stream = torch.cuda.Stream(device=dev)
    ev_start, ev_g, ev_out, ev_out_done = (torch.cuda.Event() for _ in range(4))

    def e2e_step():
        cur = torch.cuda.current_stream()
        ev_start.record(cur)
        v_d.copy_(v_host, non_blocking=True)
        sub_d.copy_(sub_host, non_blocking=True)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev_start)
            g_d.copy_(g_host, non_blocking=True)
            ev_g.record(copy_stream)
        api.gp_kernel_matvec_train(qe, s, v_d, p.lengthscale, p.variance, out=out, beta=beta_buf, moments=mom,
                                   workspace=ws)
        ev_out.record(cur)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev_out)
            out_host.copy_(out, non_blocking=True)
            ev_out_done.record(copy_stream)
        cur.wait_event(ev_g)
        G = api.gp_kernel_matvec_bwd(qe, s, v_d, p.lengthscale, p.variance, g_d, want=want, workspace=bws,
                                     beta=beta_buf, moments=mom)
        dv_host.copy_(G["v"], non_blocking=True)
        dl_host.copy_(G["lens"], non_blocking=True)
        ds_host.copy_(G["sub"], non_blocking=True)
        sc_host[0:1].copy_(G["lengthscale"], non_blocking=True)
        sc_host[1:2].copy_(G["variance"], non_blocking=True)
        cur.wait_event(ev_out_done)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    n_e2e = max(5, min(args.steps, 100))
    e_direct_ms = replicas.max_over_ranks(event_time(e2e_step, n_e2e, stream, flush), dev)
    # as for `value`: the whole step, host copies included, captured once into
    # a CUDA graph and replayed; every replay copies the inputs in from the
    # pinned host buffers and the results out to them
    run_e2e = e2e_step
    if not args.no_graph:
        e2e_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(e2e_graph):
            e2e_step()
        torch.cuda.synchronize()
        for _ in range(2):
            e2e_graph.replay()
        torch.cuda.synchronize()
        run_e2e = e2e_graph.replay
    e_ms = replicas.max_over_ranks(event_time(run_e2e, n_e2e, stream, flush), dev) if not args.no_graph else e_direct_ms
    e2e_val = replicas.aggregate_rate(p.pairs, e_ms * 1e-3, world) / 1e9
    h2d = (v_host.numel() + g_host.numel() + sub_host.numel()) * 4
    d2h = out_host.numel() * 4 + dv_host.numel() * 4 + (dl_host.numel() + ds_host.numel() + 2) * 8

    sm_mhz = clk["sm_mhz"] or SM_MAX_MHZ_DEFAULT
    sm_max = clk["sm_max_mhz"] or SM_MAX_MHZ_DEFAULT
    nsm = rates["sm_count"]
    ex2 = rates["ex2_per_clk"]
    fma = rates["ffma2_lanes_per_clk"]
    table = {}
    for name, (kms, call_ms, pairs, mufu, lanes, note, in_step) in kern.items():
        # MUFU (XU pipe, measured at its EX2 rate) or the FP32 FMA pipe binds
        per_clk = min(ex2 / mufu, fma / lanes)
        peak = per_clk * nsm * sm_max * 1e6 / 1e9
        ach = pairs / (kms * 1e-3) / 1e9
        table[name] = {"ms": kms, "call_ms": call_ms, "achieved": ach, "peak": peak, "frac": ach / peak,
                       "per_sm_clk": per_clk, "pairs_evaluated": pairs,
                       "pairs_logical": p.pairs if "raytrace" not in name else pairs, "note": note,
                       "in_step": in_step,
                       "timing": "kernel alone (launch-timer events around its launches); call_ms: the whole "
                                 "entry point (row-block pre-pass and merges included)"}
    dom = max((k for k in table if table[k]["in_step"]), key=lambda k: table[k]["ms"])
    d = table[dom]
    return {
        "value": value, "unit": UNIT, "ms_per_step": ms, "steps": n_steps,
        "config": workload_config(p),
        "pass": "forward + backward (grid, ray-trace, reduction with the row moments; gradients for v, "
                "lengthscale, variance, 7 lens parameters, 200x4 subhalo parameters)",
        "fwd": {"ms": fwd_ms, "value": p.pairs / (fwd_ms * 1e-3) / 1e9, "unit": UNIT},
        "bwd": {"ms": bwd_ms},
        "pairs": {"logical_per_step": p.pairs, "evaluated_training_forward": ev[512],
                  "evaluated_dv_sweep": ev[1024],
                  "note": "value counts every logical (i, j) pair; the grid kernels leave out the pairs whose "
                          "FP32 exp2 flushes to exactly 0 (scaled distance^2 > 170), so results are identical to "
                          "evaluating all of them; the roofline counts evaluated pairs"},
        "roofline": {"bound": "alu", "achieved": d["achieved"], "peak": d["peak"], "unit": UNIT,
                     "frac": d["frac"], "traffic": measured_traffic("realistic: " + dom), "kernel": dom,
                     "peak_basis": f"min(MUFU {ex2:.2f}/clk/SM / MUFU per pair, FFMA2 {fma:.1f} lanes/clk/SM / lanes "
                                   f"per pair) x {nsm} SMs x {sm_max:.0f} MHz (max clock; probe-measured rates); "
                                   f"{d['note']}"},
        "kernels": table,
        "step_breakdown_ms": breakdown,
        "raytrace": {"ms": rt_ms, "vjp_ms": vjp_ms, "vjp_call_ms": vjp_call_ms, "points": p.n,
                     "subhalo_pairs": p.n * len(p.sub),
                     "hbm_gbs": p.n * 8 / (rt_ms * 1e-3) / 1e9,
                     "note": "ALU/XU-bound with subhalos (8 B written per point)"},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e_ms, "ms_per_step_direct_launches": e_direct_ms},
        "gpu_launches_per_step": 13,
    }


def run_large(args, rank, local, world, dist, dev):
    """The headline step on the large workload; returns (line fields, rates,
    clocks) on every rank."""
    import torch

    from paper_2105_09465_gb300 import api, replicas, workloads as W

    # each rank owns an independent lens system of the large recipe (weak scaling)
    p = W.large(seed=4 + rank, side=args.profile_side if args.profile else 800)
    g_np = np.random.default_rng(400 + rank).standard_normal(p.n).astype(np.float32)
    sub = torch.from_numpy(p.sub).to(dev)
    v = torch.from_numpy(p.v).to(dev)
    g = torch.from_numpy(g_np).to(dev)
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=sub)
    want = ("v", "lengthscale", "variance", "lens", "sub")
    out = torch.empty(p.n, dtype=torch.float32, device=dev)
    beta_buf = torch.empty((p.n, 2), dtype=torch.float32, device=dev)
    ws = torch.empty(max(api.matvec_workspace_size(q, None), 1), dtype=torch.uint8, device=dev)
    bws = torch.empty(max(api.matvec_bwd_workspace_size(q, None, want=want, beta=True), 1), dtype=torch.uint8,
                      device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    grads = {}

    def fwd():
        api.gp_kernel_matvec(q, None, v, p.lengthscale, p.variance, out=out, beta=beta_buf, workspace=ws)

    def bwd():
        grads.update(api.gp_kernel_matvec_bwd(q, None, v, p.lengthscale, p.variance, g, want=want, workspace=bws,
                                              beta=beta_buf))

    def step():
        fwd()
        bwd()

    if args.profile:
        # the launch sequence a profiler sees: W warm-up steps, K timed steps
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        return {"profile": True, "ms_per_step": e0.elapsed_time(e1) / max(args.steps, 1),
                "launches_per_step": LARGE_STEP_LAUNCHES}, None, None, p, g_np
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    run_step = step
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        torch.cuda.synchronize()
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        run_step = graph.replay

    # ---- timed region: device-resident inputs, forward + backward per step
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        run_step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = replicas.max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), dev)
    value = replicas.aggregate_rate(p.pairs, ms * 1e-3, world) / 1e9
    nk = max(5, min(args.steps, 30))
    fwd_ms = replicas.max_over_ranks(event_time(fwd, nk, stream, flush), dev)
    bwd_ms = event_time(bwd, nk, stream, flush)

    # ---- where the step's time goes: the launch timer around each heavy
    # kernel over nk directly launched steps
    api.kernel_timer_enable(True)
    direct_ms = event_time(step, nk, stream, flush)
    api.kernel_timer_enable(False)
    breakdown = {}
    for kname in ("raytrace", "matvec", "bwd_rows", "raytrace_vjp"):
        cnt, tot, _ = api.kernel_timer_read(kname)
        breakdown[kname] = tot / cnt if cnt else None
    breakdown["step (direct launches, timer on)"] = direct_ms
    breakdown["note"] = ("matvec: the culled self-kernel forward sweep; bwd_rows: the culled self-kernel backward "
                         "sweep; each kernel's own span (events on its stream)")

    # ---- four right-hand sides in one pass (one exp2 per pair for all four):
    # the step with v and dL/dout of four draws that share the lens
    v4 = torch.from_numpy(np.random.default_rng(40).standard_normal((p.n, 4)).astype(np.float32)).to(dev)
    g4 = torch.from_numpy(np.random.default_rng(41).standard_normal((p.n, 4)).astype(np.float32)).to(dev)
    out4 = torch.empty((p.n, 4), dtype=torch.float32, device=dev)
    ws4 = torch.empty(max(api.matvec_workspace_size(q, None, nrhs=4), 1), dtype=torch.uint8, device=dev)
    bws4 = torch.empty(max(api.matvec_bwd_workspace_size(q, None, want=want, beta=True, nrhs=4), 1),
                       dtype=torch.uint8, device=dev)

    def step4():
        api.gp_kernel_matvec(q, None, v4, p.lengthscale, p.variance, out=out4, beta=beta_buf, workspace=ws4)
        api.gp_kernel_matvec_bwd(q, None, v4, p.lengthscale, p.variance, g4, want=want, workspace=bws4,
                                 beta=beta_buf)

    step4()
    ms4 = event_time(step4, nk, stream, flush)
    ms1 = event_time(step, nk, stream, flush)
    multi_rhs = {"nrhs": 4, "ms_per_step": ms4, "ms_one_rhs": ms1, "ms_four_one_rhs_steps": 4 * ms1,
                 "speedup_vs_four_steps": 4 * ms1 / ms4,
                 "note": "v and dL/dout with 4 columns that share the ray-traced points: the forward and the "
                         "self-kernel backward evaluate each pair's exp2 once for all four; the ray-trace and its "
                         "VJP (dL/dbeta summed over the columns) run once; direct launches"}

    # ---- pairs the culled sweeps evaluate (the rest are exact zeros in FP32)
    beta = api.lens_raytrace(q)
    qx = api.Points(xy=beta, grid=p.xgrid)
    pf, sf = api.cull_pairs_evaluated(qx, None, p.lengthscale, 0)
    pb, sb = api.cull_pairs_evaluated(qx, None, p.lengthscale, 1)

    # ---- kernels alone (same launch configuration as inside the step)
    dbeta = torch.from_numpy(np.random.default_rng(7).standard_normal((p.n, 2)).astype(np.float32)).to(dev)
    kern = {}
    kern["cull_kernel<forward> (self-kernel forward)"] = (
        *kernel_time(fwd, nk, stream, flush, "matvec"), pf, CULL_FWD_MUFU, CULL_FWD_LANES,
        f"evaluated pairs ({sf:.3e} pair slots with row-block padding and empty chunk slots): 1 MUFU.EX2 + "
        f"{CULL_FWD_LANES:g} FP32 lanes each; call_ms includes the ray-trace fused into the call", True)
    kern["cull_kernel<self backward> (d_v, d_x both roles, d_l, d_var)"] = (
        *kernel_time(bwd, nk, stream, flush, "bwd_rows"), pb, CULL_SELF_MUFU, CULL_SELF_LANES,
        f"evaluated pairs ({sb:.3e} pair slots): 1 MUFU.EX2 + {CULL_SELF_LANES:g} FP32 lanes each; call_ms "
        "includes the ray-trace VJP", True)
    rt_ms, rt_call_ms = kernel_time(lambda: api.lens_raytrace(q), nk, stream, flush, "raytrace")
    vjp_ms, vjp_call_ms = kernel_time(lambda: api.lens_raytrace_vjp(q, dbeta), nk, stream, flush, "raytrace_vjp")
    sub_pairs = p.n * len(p.sub)
    rt_mufu, rt_lanes, rt_sh = raytrace_cost(p)
    kern["raytrace_kernel<tNFW> (forward ray-trace; unit: point-subhalo pair)"] = (
        rt_ms, rt_call_ms, sub_pairs, rt_mufu, rt_lanes,
        f"pairs: {rt_mufu:.2f} MUFU + {rt_lanes:.1f} FP32 lanes each on average; shares of the pairs by the "
        f"far-field series degree that serves the CTA's tile ({SER_MUFU} MUFU + 9.31 + K lanes) and the far-side "
        f"closed form ({RT_MUFU} MUFU + {RT_LANES} lanes): {_shares_text(rt_sh)}", True)
    vj_mufu, vj_lanes, vj_sh = vjp_cost(p, vjp_tiles(dev, p.n))
    kern["raytrace_vjp_kernel<tNFW> (ray-trace backward; unit: point-subhalo pair)"] = (
        vjp_ms, vjp_call_ms, sub_pairs, vj_mufu, vj_lanes,
        f"pairs: {vj_mufu:.2f} MUFU + {vj_lanes:.1f} FP32 lanes each on average; shares of the pairs by the "
        f"degree of the series of G and x dG/dx that serves the CTA's tile ({SER_MUFU} MUFU + 20.3 + 2 (K - 2) "
        f"lanes) and the far-side closed form ({VJ_MUFU} MUFU + {VJ_LANES} lanes): {_shares_text(vj_sh)}", True)

    # ---- end to end through the public API with host buffers
    v_host = torch.from_numpy(p.v).pin_memory()
    g_host = torch.from_numpy(g_np).pin_memory()
    sub_host = torch.from_numpy(p.sub).pin_memory()
    out_host = torch.empty(p.n, dtype=torch.float32).pin_memory()
    dv_host = torch.empty(p.n, dtype=torch.float32).pin_memory()
    dl_host = torch.empty(7, dtype=torch.float64).pin_memory()
    ds_host = torch.empty((len(p.sub), 4), dtype=torch.float64).pin_memory()
    sc_host = torch.empty(2, dtype=torch.float64).pin_memory()
    v_d, g_d, sub_d = torch.empty_like(v), torch.empty_like(g), torch.empty_like(sub)
    qe = api.Points(grid=p.xgrid, lens=p.lens, sub=sub_d)
    copy_stream = torch.cuda.Stream(device=dev)
    ev_start, ev_g, ev_out, ev_out_done = (torch.cuda.Event() for _ in range(4))

    def e2e_step():
        # dL/dout (needed only by the backward) comes in on a second stream
        # during the forward; out goes back during the backward
        cur = torch.cuda.current_stream()
        ev_start.record(cur)
        v_d.copy_(v_host, non_blocking=True)
        sub_d.copy_(sub_host, non_blocking=True)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev_start)
            g_d.copy_(g_host, non_blocking=True)
            ev_g.record(copy_stream)
        api.gp_kernel_matvec(qe, None, v_d, p.lengthscale, p.variance, out=out, beta=beta_buf, workspace=ws)
        ev_out.record(cur)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev_out)
            out_host.copy_(out, non_blocking=True)
            ev_out_done.record(copy_stream)
        cur.wait_event(ev_g)
        G = api.gp_kernel_matvec_bwd(qe, None, v_d, p.lengthscale, p.variance, g_d, want=want, workspace=bws,
                                     beta=beta_buf)
        dv_host.copy_(G["v"], non_blocking=True)
        dl_host.copy_(G["lens"], non_blocking=True)
        ds_host.copy_(G["sub"], non_blocking=True)
        sc_host[0:1].copy_(G["lengthscale"], non_blocking=True)
        sc_host[1:2].copy_(G["variance"], non_blocking=True)
        cur.wait_event(ev_out_done)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    n_e2e = max(5, min(args.steps, 50))
    e_direct_ms = replicas.max_over_ranks(event_time(e2e_step, n_e2e, stream, flush), dev)
    run_e2e = e2e_step
    if not args.no_graph:
        e2e_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(e2e_graph):
            e2e_step()
        torch.cuda.synchronize()
        for _ in range(2):
            e2e_graph.replay()
        torch.cuda.synchronize()
        run_e2e = e2e_graph.replay
    e_ms = replicas.max_over_ranks(event_time(run_e2e, n_e2e, stream, flush), dev) if not args.no_graph else e_direct_ms
    e2e_val = replicas.aggregate_rate(p.pairs, e_ms * 1e-3, world) / 1e9
    h2d = (v_host.numel() + g_host.numel() + sub_host.numel()) * 4
    d2h = out_host.numel() * 4 + dv_host.numel() * 4 + (dl_host.numel() + ds_host.numel() + 2) * 8

    rates = api.probe_pipe_rates(local)
    sm_mhz = clk["sm_mhz"] or SM_MAX_MHZ_DEFAULT
    sm_max = clk["sm_max_mhz"] or SM_MAX_MHZ_DEFAULT
    nsm, ex2, fma = rates["sm_count"], rates["ex2_per_clk"], rates["ffma2_lanes_per_clk"]
    table = {}
    for name, (kms, call_ms, pairs, mufu, lanes, note, in_step) in kern.items():
        per_clk = min(ex2 / mufu, fma / lanes)
        peak = per_clk * nsm * sm_max * 1e6 / 1e9
        ach = pairs / (kms * 1e-3) / 1e9
        table[name] = {"ms": kms, "call_ms": call_ms, "achieved": ach, "peak": peak, "frac": ach / peak,
                       "per_sm_clk": per_clk, "pairs_evaluated": pairs,
                       "pairs_logical": p.pairs if "raytrace" not in name else pairs, "note": note,
                       "in_step": in_step,
                       "timing": "kernel alone (launch-timer events around its launches); call_ms: the whole "
                                 "entry point"}
    dom = max((k for k in table if table[k]["in_step"]), key=lambda k: table[k]["ms"])
    d = table[dom]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; see workloads.py)",
        "config": dict(large_config(p), parallelism=f"independent lens system per GPU x{world}"),
        "pass": "forward + backward: ray-trace fused into the forward call, the culled self-kernel forward, "
                "the culled self-kernel backward (d_v, dL/dbeta of both roles, d_lengthscale, d_variance) and "
                "the ray-trace backward (7 lens parameters, 2000x4 subhalo parameters)",
        "fwd": {"ms": fwd_ms, "value": replicas.aggregate_rate(p.pairs, fwd_ms * 1e-3, world) / 1e9, "unit": UNIT,
                "note": "forward alone: ray-trace + self-kernel reduction"},
        "bwd": {"ms": bwd_ms},
        "pairs": {"logical_per_step": p.pairs, "evaluated_forward": pf, "evaluated_backward": pb,
                  "slots_forward": sf, "slots_backward": sb,
                  "note": "value counts every logical (i, j) pair, as the metric defines it; the culled sweeps "
                          "leave out the pairs whose FP32 exp2 flushes to exactly 0 (scaled distance^2 > 170), so "
                          "results are bitwise those of evaluating all of them (tested); the roofline counts the "
                          "evaluated pairs"},
        "roofline": {"bound": "alu", "achieved": d["achieved"], "peak": d["peak"], "unit": UNIT,
                     "frac": d["frac"], "traffic": measured_traffic("large: " + dom), "kernel": dom,
                     "peak_basis": f"min(MUFU {ex2:.2f}/clk/SM / MUFU per pair, FFMA2 {fma:.1f} lanes/clk/SM / lanes "
                                   f"per pair) x {nsm} SMs x {sm_max:.0f} MHz (max clock; probe-measured rates); "
                                   f"{d['note']}",
                     "frac_at_measured_clock": d["frac"] * sm_max / sm_mhz},
        "kernels": table,
        "step_breakdown_ms": breakdown,
        "multi_rhs": multi_rhs,
        "raytrace": {"ms": rt_ms, "vjp_ms": vjp_ms, "points": p.n, "subhalo_pairs": sub_pairs,
                     "hbm_gbs": p.n * 8 / (rt_ms * 1e-3) / 1e9,
                     "note": "ALU/XU-bound with subhalos (8 B written per point)"},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e_ms, "ms_per_step_direct_launches": e_direct_ms,
                "launch": ("CUDA graph of the step with its 3 host-to-device and 6 device-to-host copies, replayed"
                           if not args.no_graph else "direct launches")},
        "gpu_launches": LARGE_STEP_LAUNCHES * args.steps,
        "launch": (f"CUDA graph of the step's {LARGE_STEP_LAUNCHES} launches, replayed" if not args.no_graph
                   else "direct launches"),
        "clocks": clk,
        "pipe_rates": rates,
    }
    return line, rates, clk, p, g_np


# Kernels of one headline step: forward = ray-trace, chunk prepare, group
# boxes, culled sweep; backward = chunk prepare, group boxes, culled sweep,
# scalar sum, ray-trace VJP and its final sums.
LARGE_STEP_LAUNCHES = 12


def run_ours(args):
    import torch

    from paper_2105_09465_gb300 import replicas

    rank, local, world = replicas.world()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    if args.profile_layer:
        if rank == 0:
            print(json.dumps(run_profile_layer(args, dev)))
        if dist:
            dist.destroy_process_group()
        return
    line, rates, clk, p, g_np = run_large(args, rank, local, world, dist, dev)
    if args.profile:
        if rank == 0:
            print(json.dumps(line))
        if dist:
            dist.destroy_process_group()
        return
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    if world == 1:
        line["realistic"] = run_realistic(args, dev, rates, clk)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        sm_max = clk["sm_max_mhz"] or SM_MAX_MHZ_DEFAULT
        if not args.no_extensions:
            from paper_2105_09465_gb300 import workloads as W
            line["extensions"] = run_extensions(W.realistic(), dev, rates, sm_max, flush,
                                                torch.cuda.current_stream())
        if not args.no_serving:
            line["serving"] = run_serving(args.serving_requests, args.serving_iters)
            # request latency as a service sees it: Poisson arrivals, the
            # engine that admits by pairs per iteration
            line["p50_latency_s"] = line["serving"]["poisson_70pct_filled"]["p50_s"]
            line["p99_latency_s"] = line["serving"]["poisson_70pct_filled"]["p99_s"]
        if not args.no_cpu_baseline:
            cb = cpu_sample_large(p, args.cpu_seconds, g_np.astype(np.float64), one_core_seconds=args.cpu_seconds / 2)
            cb.pop("seconds", None)
            line["cpu_baseline"] = cb
    print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
