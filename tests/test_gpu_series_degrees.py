"""The ray-trace kernels' far-field series of a tNFW subhalo, degree by degree.

A CTA sums a subhalo by the terms of its far-field series up to y^K (y =
1/x, x = R / theta_s) when the whole bounding box of the CTA's points lies
beyond that degree's radius: the forward from x = 6, 8, 18, 32, 80
max(tau, 2) with K = 9, 7, 5, 4, 3, the backward from 8, 18, 32, 80 with
K = 7, 5, 4, 3. Where the tile is small against its distance, the backward
sums the same series by its local expansion about the tile's centre. Here one heavy subhalo sits at the origin and a small image
grid lies wholly inside one distance band at a time; the main deflector is
negligible (theta_E = 1e-9) and the shear zero, so every deflection is the
subhalo's. The FP64 oracle evaluates the closed form (Baltz, Marshall & Oguri
2009), and the kernels must match it to relative precision, far tighter than
the absolute 1e-6 arcsec of the deflection tolerance: 1.5e-6 for the
deflections (about ten FP32 roundings and the 2^-22.9 of the reciprocal
square root) and 4e-6 for the gradient's subhalo sums, whose two parts
cancel to a third of their size in the far field, so that a wrong or dropped
term of relative size 1e-5 fails. The gradient's dL/dbeta has one sign
everywhere, so each point's term of a subhalo sum has the same sign.
"""
import numpy as np
import pytest

from paper_2105_09465_gb300 import api, workloads as W
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu

THETA_S, TAU = 0.05, 10.0  # R = x theta_s, max(tau, 2) = 10: R = 0.5 r arcsec at x = r max(tau, 2)
# grid centres R (arcsec) inside each band of r = x / max(tau, 2), the grid
# spanning +-0.2 arcsec: forward bands [6, 8) [8, 18) [18, 32) [32, 80) [80, inf),
# backward (closed forms below 8) [8, 18) [18, 32) [32, 80) [80, inf)
CENTRES = [3.5, 6.0, 12.0, 25.0, 60.0, 400.0]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def setup(cx):
    g = W.Grid(16, 16, 2, 0.025, cx, 0.0)
    lens = W.Lens(0.0, 0.0, 0.9, 0.2, 1e-9, 2.0, 0.0, 0.0)
    sub = np.array([[0.0, 0.0, 0.05, THETA_S, TAU]], np.float32)
    return g, lens, sub


@pytest.mark.parametrize("cx", CENTRES)
def test_forward_series_degree(orc, cx):
    g, lens, sub = setup(cx)
    xi = orc.grid_points(*g.astuple())
    _, alpha = api.lens_raytrace(api.Points(grid=g, lens=lens, sub=dev(sub)), want_alpha=True)
    a_ref, _ = orc.raytrace(xi, lens.astuple(), sub, 0)
    a = host(alpha).astype(np.float64)
    err = np.hypot(*(a - a_ref).T) / np.hypot(*a_ref.T)
    assert err.max() <= 1.5e-6, f"max relative deflection error {err.max():.3e}"


@pytest.mark.parametrize("copies", [1, 4097])
@pytest.mark.parametrize("cx", CENTRES)
def test_vjp_series_degree(orc, cx, copies):
    """One subhalo: the backward's local expansion about each tile's centre
    serves every band but the nearest; 4097 copies of it (more than a tile
    orders): every pair takes the series or the closed forms directly."""
    g, lens, sub = setup(cx)
    sub = np.repeat(sub, copies, axis=0)
    xi = orc.grid_points(*g.astuple())
    rng = np.random.default_rng(3)
    db = rng.uniform(0.5, 1.5, (g.n, 2)).astype(np.float32)
    _, d_sub = api.lens_raytrace_vjp(api.Points(grid=g, lens=lens, sub=dev(sub)), dev(db))
    _, rs, _, asub = orc.raytrace_vjp(xi, lens.astuple(), sub, db, 0, with_abs=True)
    got, rs, asub = host(d_sub).astype(np.float64).ravel(), np.ravel(rs), np.ravel(asub)
    # one sign per sum over the points: the sums of absolute terms are the sums themselves
    assert np.all(np.abs(rs) >= 0.999 * asub)
    err = np.abs(got - rs) / asub
    assert err.max() <= 4e-6, f"relative subhalo-gradient errors {err}"


# Off-axis tiles near the local expansion's limit: a light subhalo (theta_s =
# 0.01 arcsec) with the grid's centre at distance D in direction 40 degrees,
# so that the tiles' half-diagonals are 0.01 to 0.08 of their distance and
# every term delta^k conj(delta)^l of the expansion, and its phase, counts.
@pytest.mark.parametrize("dist", [3.6, 8.0, 25.0])
def test_expansion_off_axis(orc, dist):
    ang = np.deg2rad(40.0)
    g = W.Grid(16, 16, 2, 0.05, dist * np.cos(ang), dist * np.sin(ang))
    lens = W.Lens(0.0, 0.0, 0.9, 0.2, 1e-9, 2.0, 0.0, 0.0)
    sub = np.array([[0.0, 0.0, 0.3, 0.01, TAU]], np.float32)
    xi = orc.grid_points(*g.astuple())
    _, alpha = api.lens_raytrace(api.Points(grid=g, lens=lens, sub=dev(sub)), want_alpha=True)
    a_ref, _ = orc.raytrace(xi, lens.astuple(), sub, 0)
    a = host(alpha).astype(np.float64)
    err = np.hypot(*(a - a_ref).T) / np.hypot(*a_ref.T)
    assert err.max() <= 1.5e-6, f"max relative deflection error {err.max():.3e}"
    db = np.random.default_rng(5).uniform(0.5, 1.5, (g.n, 2)).astype(np.float32)
    _, d_sub = api.lens_raytrace_vjp(api.Points(grid=g, lens=lens, sub=dev(sub)), dev(db))
    _, rs, _, asub = orc.raytrace_vjp(xi, lens.astuple(), sub, db, 0, with_abs=True)
    got, rs, asub = host(d_sub).astype(np.float64).ravel(), np.ravel(rs), np.ravel(asub)
    err = np.abs(got - rs) / asub
    assert err.max() <= 4e-6, f"relative subhalo-gradient errors {err}"
