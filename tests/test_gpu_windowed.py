"""Parity of the CUDA pixel windows and windowed transmission reduction with
the FP64 oracle, on a lensed pixel grid like the paper's image-plane model."""
import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import abi, api, workloads as W
from tests.gpu_util import assert_matvec_close, dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def lensed_grid(orc, side=60, pix=0.05, seed=3):
    rng = np.random.default_rng(seed)
    lens = W.draw_lens(rng)
    g = W.Grid(side, side, 1, pix)
    _, b = orc.raytrace(orc.grid_points(*g.astuple()), lens.astuple())
    return g, b.astype(np.float32)


def test_pixel_shapes(orc):
    g, b = lensed_grid(orc)
    z = host(api.pixel_shapes(dev(b), g.nx, g.ny))
    zr = orc.pixel_shapes(b, g.nx, g.ny)
    scale = np.abs(zr).max(axis=1, keepdims=True)
    assert np.all(np.abs(z - zr) <= 1e-5 * scale + 1e-12), float(np.max(np.abs(z - zr) / scale))


@pytest.mark.parametrize("source", ["grid", "explicit", "self"])
def test_windowed_transmission(orc, source):
    g, b = lensed_grid(orc, side=70)
    zr = orc.pixel_shapes(b, g.nx, g.ny).astype(np.float32)  # oracle windows feed both sides
    rng = np.random.default_rng(4)
    ell = 0.05
    if source == "grid":
        yg = W.Grid(40, 40, 1, 0.1)
        q = orc.grid_points(*yg.astuple())
        src = api.Points(grid=yg)
    elif source == "explicit":
        q = rng.uniform(-2, 2, (3000, 2)).astype(np.float32)
        src = api.Points(xy=dev(q))
    else:
        q = b
        src = api.Points(xy=dev(b))
    v = rng.standard_normal(len(q)).astype(np.float32)
    got = host(api.gp_windowed_matvec(dev(b), dev(zr), src, dev(v), ell))
    ref, ab = orc.windowed_matvec(b, zr, q, v, ell)
    assert_matvec_close(got, ref, ab, what=f"windowed ({source})")


def test_zero_windows_reduce_to_the_point_kernel():
    rng = np.random.default_rng(5)
    x = rng.uniform(-0.5, 0.5, (2000, 2)).astype(np.float32)
    v = rng.standard_normal(2000).astype(np.float32)
    z = np.zeros((2000, 3), np.float32)
    a = host(api.gp_windowed_matvec(dev(x), dev(z), api.Points(xy=dev(x)), dev(v), 0.08))
    b = host(api.gp_kernel_matvec(api.Points(xy=dev(x)), None, dev(v), 0.08 / np.sqrt(2.0), 1.0 / (np.pi * 0.0064)))
    np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-5 * np.abs(b).max())


def test_windowed_grid_realistic_scales(orc):
    """Pixel windows of a lensed 120 x 120 image at the realistic pixel size
    (0.05 arcsec) against a 128 x 128 source grid over the field padded by 20 %,
    length scale 4/3 of its spacing: the grid path's completed square at the
    workload's coordinate magnitudes."""
    p = W.realistic(seed=11, side=120, ss=1, n_sub=0)
    g = p.xgrid
    _, b = orc.raytrace(orc.grid_points(*g.astuple()), p.lens.astuple())
    b = b.astype(np.float32)
    zr = orc.pixel_shapes(b, g.nx, g.ny).astype(np.float32)
    yg = p.ygrid
    q = orc.grid_points(*yg.astuple())
    v = np.random.default_rng(12).standard_normal(len(q)).astype(np.float32)
    got = host(api.gp_windowed_matvec(dev(b), dev(zr), api.Points(grid=yg), dev(v), p.lengthscale))
    ref, ab = orc.windowed_matvec(b, zr, q, v, p.lengthscale)
    assert_matvec_close(got, ref, ab, what="windowed (realistic grid)")


def _close(got, ref, scale, rel, what, floor=0.0):
    got, ref, scale = (np.asarray(a, np.float64) for a in (got, ref, scale))
    tol = rel * scale + floor + 1e-30
    ratio = np.abs(got - ref) / tol
    if np.any(ratio > 1):
        k = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
        raise AssertionError(f"{what}: {int(np.sum(ratio > 1))} outside tolerance; worst {k}: got {got[k]!r} "
                             f"ref {ref[k]!r} tol {np.broadcast_to(tol, ratio.shape)[k]!r}")


@pytest.mark.parametrize("self_points", [False, True])
def test_windowed_backward(orc, self_points):
    """Every gradient of sum_i g_i out_i against the FP64 oracle, on a lensed
    pixel grid with its windows; sources explicit or the pixels themselves
    (the image-plane layer)."""
    g_, b = lensed_grid(orc, side=50)
    zr = orc.pixel_shapes(b, g_.nx, g_.ny).astype(np.float32)
    rng = np.random.default_rng(21)
    q = b if self_points else rng.uniform(-1.2, 1.2, (2000, 2)).astype(np.float32)
    v = rng.standard_normal(len(q)).astype(np.float32)
    gout = rng.standard_normal(len(b)).astype(np.float32)
    ell = 0.05
    G = api.gp_windowed_matvec_bwd(dev(b), dev(zr), api.Points(xy=dev(q)), dev(v), ell, dev(gout))
    R = orc.windowed_vjp(b, zr, q, v, ell, gout, with_abs=True)
    rel = 2e-5  # of the sum of |terms|, the reduction tolerance
    _close(host(G["v"]), R["d_v"], R["d_v_abs"], rel, "d_v")
    _close(host(G["p"]), R["d_p"], R["d_p_abs"], rel, "d_p")
    _close(host(G["q"]), R["d_q"], R["d_q_abs"], rel, "d_q")
    _close(host(G["z"]), R["d_z"], R["d_z_abs"], rel, "d_z")
    _close(host(G["lengthscale"]), [R["d_len"]], [R["d_len_abs"]], rel, "d_len")


def test_pixel_shapes_vjp(orc):
    g_, b = lensed_grid(orc, side=40)
    dz = np.random.default_rng(22).standard_normal((len(b), 3)).astype(np.float32)
    got = host(api.pixel_shapes_vjp(dev(b), g_.nx, g_.ny, dev(dz)))
    ref, ab = orc.pixel_shapes_vjp(b, g_.nx, g_.ny, dz, with_abs=True)
    # FP32 products and a gather of up to four neighbours' terms: 16 u of the absolute terms
    _close(got, ref, ab, 16 * 2.0 ** -24, "pixel-window VJP")


# ---- the image-plane layer with exact skipping of far pairs

FLUSH = 2.0 ** -125  # FP32 exp2 returns 0 below 2^-126; one binade of margin
U32 = 2.0 ** -24     # FP32 unit roundoff


def windowed_tols(orc, p, z, q, v, g, ell):
    """Per-output tolerances of the FP32 windowed path: 2e-5 of the sum of
    absolute terms, twice the FP32 rounding sensitivity of the far pairs'
    exponents (oracle windowed_rounding: the rounded difference and window
    constants, amplified by the exponent and the window's elongation), and
    the flush floor."""
    A = orc.windowed_vjp(p, z, q, v, ell, g, with_abs=True)
    ref, ab = orc.windowed_matvec(p, z, q, v, ell)
    S = orc.windowed_rounding(p, z, q, v, ell, g)
    F = flush_floors(p, z, q, v, g, ell)
    T = {"out": 2e-5 * ab + 2 * U32 * S["s_out"] + F["out"]}
    for k, sk in (("d_v", "s_v"), ("d_p", "s_p"), ("d_q", "s_q"), ("d_z", "s_z"), ("d_len", "s_len")):
        T[k] = 2e-5 * np.asarray(A[k + "_abs"]) + 2 * U32 * np.asarray(S[sk]) + F[k]
    A["out"] = ref
    return A, T


def check_windowed(G, out, R, T, what):
    for key, rk in (("v", "d_v"), ("p", "d_p"), ("q", "d_q"), ("z", "d_z")):
        if key in G:
            _close(host(G[key]), R[rk], 0.0, 0.0, f"{what} {rk}", T[rk])
    if "lengthscale" in G:
        _close(host(G["lengthscale"]), [R["d_len"]], [0.0], 0.0, f"{what} d_len", T["d_len"])
    if out is not None:
        _close(out, R["out"], 0.0, 0.0, f"{what} out", T["out"])


def flush_floors(p, z, q, v, g, ell):
    """Per-output bounds of the terms the FP32 kernels drop: a pair whose
    Gaussian factor exp(-d^T C^-1 d / 2) is below 2^-126 contributes exactly
    0 there, and at most FLUSH times its other factors in FP64 (N_i, v_k,
    g_i, u = C_i^-1 d, C_i^-1). Rows far from every source have only such
    terms, where the windows' large N and |u| lift them past a fixed floor."""
    p, q, z = (np.asarray(a, np.float64) for a in (p, q, z))
    v, g = np.abs(np.asarray(v, np.float64)), np.abs(np.asarray(g, np.float64))
    hs = 0.5 * ell * ell
    cxx, cxy, cyy = z[:, 0] + hs, z[:, 1], z[:, 2] + hs
    det = cxx * cyy - cxy * cxy
    ixx, ixy, iyy = cyy / det, -cxy / det, cxx / det
    N = 1.0 / (2 * np.pi * np.sqrt(det))
    dx = p[:, None, 0] - q[None, :, 0]
    dy = p[:, None, 1] - q[None, :, 1]
    ux = np.abs(ixx[:, None] * dx + ixy[:, None] * dy)
    uy = np.abs(ixy[:, None] * dx + iyy[:, None] * dy)
    w = FLUSH * N[:, None]
    F = {"out": (w * v[None, :]).sum(1)}
    gw = g[:, None] * w
    F["d_p"] = np.stack([(gw * v * ux).sum(1), (gw * v * uy).sum(1)], 1)
    mz = 0.5 * gw * v
    F["d_z"] = np.stack([(mz * (ux * ux + np.abs(ixx)[:, None])).sum(1),
                         (2 * mz * (ux * uy + np.abs(ixy)[:, None])).sum(1),
                         (mz * (uy * uy + np.abs(iyy)[:, None])).sum(1)], 1)
    F["d_v"] = gw.sum(0)
    F["d_q"] = np.stack([(gw * ux).sum(0) * v, (gw * uy).sum(0) * v], 1)
    F["d_len"] = ell * float(F["d_z"][:, 0].sum() + F["d_z"][:, 2].sum())
    return F

def image_layer(orc, side, ell, seed=30):
    """A lensed side x side pixel grid (0.05 arcsec pixels) with its windows,
    its own points as the sources, weights and output gradients."""
    g, b = lensed_grid(orc, side=side, seed=seed)
    zr = orc.pixel_shapes(b, g.nx, g.ny).astype(np.float32)
    rng = np.random.default_rng(seed + 1)
    v = rng.standard_normal(len(b)).astype(np.float32)
    gout = rng.standard_normal(len(b)).astype(np.float32)
    return g, b, zr, v, gout


@pytest.mark.parametrize("ell", [0.002, 0.00447, 0.01, 0.05])
@pytest.mark.parametrize("layout", [False, True])
def test_image_plane_layer_at_the_papers_scales(orc, ell, layout):
    """The image-plane layers' kernel sizes (10, 4.47 and 2 mas, and the
    0.05 arcsec of the workloads) on an 80 x 80 lensed grid, forward and every
    gradient element by element against the FP64 oracle; with the pixels'
    image layout and in index order."""
    g, b, zr, v, gout = image_layer(orc, 80, ell)
    lay = g if layout else None
    src = api.Points(xy=dev(b), grid=g if layout else None)
    got = host(api.gp_windowed_matvec(dev(b), dev(zr), src, dev(v), ell, layout=lay))
    G = api.gp_windowed_matvec_bwd(dev(b), dev(zr), src, dev(v), ell, dev(gout), layout=lay)
    R, T = windowed_tols(orc, b, zr, b, v, gout, ell)
    check_windowed(G, got, R, T, f"image-plane layer l = {ell}")


@pytest.mark.parametrize("ell", [0.002, 0.00447, 0.01])
def test_grid_sources_with_narrow_kernels(orc, ell):
    """Grid sources at the image-plane layers' kernel sizes (10, 4.47 and
    2 mas), spaced 3/4 of the length scale, 270 columns (two tiles, the
    second ragged) by 10 rows, against a lensed 60 x 60 image whose
    windows are most elongated relative to the kernel there: every output
    against the FP64 oracle within the derived FP32 tolerance."""
    g, b, zr, v, _ = image_layer(orc, 60, ell, seed=33)
    yg = W.Grid(270, 10, 1, 0.75 * ell)
    q = orc.grid_points(*yg.astuple())
    w = np.random.default_rng(34).standard_normal(len(q)).astype(np.float32)
    got = host(api.gp_windowed_matvec(dev(b), dev(zr), api.Points(grid=yg), dev(w), ell))
    R, T = windowed_tols(orc, b, zr, q, w, np.zeros(len(b), np.float32), ell)
    near = R["out"] != 0
    assert int(np.sum(np.abs(R["out"]) > 1e-3 * np.abs(R["out"]).max())) >= 20  # rows that meet the grid
    _close(got, R["out"], 0.0, 0.0, f"grid sources l = {ell}", T["out"])
    assert np.all(got[~near] == 0)


@pytest.mark.parametrize("ell", [0.002, 0.05])
def test_skipping_is_exact_bitwise(orc, ell):
    """With exact skipping switched off every pair is evaluated, in the same
    order: every output and gradient is bitwise the same."""
    g, b, zr, v, gout = image_layer(orc, 72, ell, seed=40)
    args = (dev(b), dev(zr), api.Points(xy=dev(b), grid=g), dev(v), ell)
    lib = abi.load()
    try:
        lib.lr_set_pair_culling(0)
        f0 = api.gp_windowed_matvec(*args, layout=g)
        G0 = api.gp_windowed_matvec_bwd(*args, dev(gout), layout=g)
        torch.cuda.synchronize()
    finally:
        lib.lr_set_pair_culling(1)
    f1 = api.gp_windowed_matvec(*args, layout=g)
    G1 = api.gp_windowed_matvec_bwd(*args, dev(gout), layout=g)
    torch.cuda.synchronize()
    assert torch.equal(f0, f1)
    for k in G0:
        assert torch.equal(G0[k], G1[k]), k


def test_explicit_sources_ragged_sizes(orc):
    """Query and source counts that leave partial chunks and row blocks,
    sources scattered without a layout, a narrow kernel."""
    g, b = lensed_grid(orc, side=37, seed=9)
    zr = orc.pixel_shapes(b, g.nx, g.ny).astype(np.float32)
    rng = np.random.default_rng(10)
    for m in (1, 31, 33, 1000):
        q = (b[rng.choice(len(b), m, replace=False)] + rng.normal(0, 0.02, (m, 2))).astype(np.float32)
        v = rng.standard_normal(m).astype(np.float32)
        gout = rng.standard_normal(len(b)).astype(np.float32)
        got = host(api.gp_windowed_matvec(dev(b), dev(zr), api.Points(xy=dev(q)), dev(v), 0.01, layout=g))
        G = api.gp_windowed_matvec_bwd(dev(b), dev(zr), api.Points(xy=dev(q)), dev(v), 0.01, dev(gout), layout=g)
        R, T = windowed_tols(orc, b, zr, q, v, gout, 0.01)
        check_windowed(G, got, R, T, f"windowed m = {m}")


def test_windowed_pairs_evaluated(orc):
    """On the 400 x 400 image of the workloads (0.05 arcsec pixels) at a 2 mas
    kernel the sweeps evaluate a small fraction of the n^2 pairs, and at least
    every pair whose exponent is above -126 (counted by brute force on
    sampled rows). The fraction is set by the boxes of the source chunks
    (8 x 4 pixels) and of a warp's rows against the source-plane region the
    image maps to."""
    g, b, zr, v, gout = image_layer(orc, 400, 0.002, seed=50)
    n = len(b)
    src = api.Points(xy=dev(b), grid=g)
    counts = [api.windowed_pairs_evaluated(dev(b), dev(zr), src, 0.002, s, layout=g) for s in (0, 1, 2)]
    for pairs, slots in counts:
        assert 0 < pairs <= slots and pairs < 0.01 * n * n
    # brute force over sampled rows: exponent = -(log2 e / 2) d^T C^-1 d
    rows = np.random.default_rng(51).choice(n, 300, replace=False)
    bb = b.astype(np.float64)
    need = 0
    for i in rows:
        c = zr[i].astype(np.float64) + np.array([0.5 * 0.002 ** 2, 0.0, 0.5 * 0.002 ** 2])
        det = c[0] * c[2] - c[1] ** 2
        d = bb - bb[i]
        q = (c[2] * d[:, 0] ** 2 - 2 * c[1] * d[:, 0] * d[:, 1] + c[0] * d[:, 1] ** 2) / det
        need += int(np.count_nonzero(0.5 * np.log2(np.e) * q <= 126.0))
    assert counts[0][0] >= need * (n / 300) * 0.5


@pytest.mark.parametrize("with_f_in", [False, True])
def test_likelihood_in_the_epilogue(orc, with_f_in):
    """gp_windowed_matvec_nll: the model total, dL/df and the Gaussian nll
    formed where the windowed reduction finishes each row, against the
    oracle's windowed reduction and Gaussian likelihood (Sec. 3.3)."""
    g_, b, zr, v, _ = image_layer(orc, 70, 0.01, seed=60)
    rng = np.random.default_rng(61)
    n = len(b)
    f_in = rng.standard_normal(n).astype(np.float32) if with_f_in else None
    data = rng.standard_normal(n).astype(np.float32)
    sigma = 0.3
    src = api.Points(xy=dev(b), grid=g_)
    out, g, nll = api.gp_windowed_matvec_nll(dev(b), dev(zr), src, dev(v), 0.01, dev(data), sigma,
                                             f_in=dev(f_in) if with_f_in else None, layout=g_)
    R, T = windowed_tols(orc, b, zr, b, v, np.zeros(n), 0.01)
    ref = R["out"] + (f_in.astype(np.float64) if with_f_in else 0.0)
    tol_out = T["out"] + 4 * 2.0 ** -24 * (np.abs(f_in) if with_f_in else 0.0)
    _close(host(out), ref, 0.0, 0.0, "model total", tol_out)
    r = ref - data.astype(np.float64)
    _close(host(g), r / sigma ** 2, 0.0, 0.0, "dL/df", (tol_out + 4 * 2.0 ** -24 * np.abs(r)) / sigma ** 2)
    ref_nll = float(np.sum(0.5 * r * r) / sigma ** 2 + n * np.log(sigma) + 0.5 * n * np.log(2 * np.pi))
    tol_nll = float(np.sum(np.abs(r) * tol_out) / sigma ** 2) + 1e-6 * abs(ref_nll)
    assert abs(float(nll) - ref_nll) <= tol_nll, (float(nll), ref_nll, tol_nll)
