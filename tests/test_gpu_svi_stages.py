"""One SVI step checked element by element, stage by stage.

The step (paper_2105_09465_gb300.svi) is a chain: draw (Sec. 4.2 partial
MVN), ray-trace (Sec. 2.1), pixel windows (Sec. 3.2), transmission weights
(Sec. 3.4 density), the source-plane and image-plane reductions (Sec. 3.3,
3.4), the Gaussian likelihood (Sec. 3.3), their VJPs down to the guide
parameters (Sec. 3.6). Each stage is compared with the FP64 oracle on the
GPU's own inputs to that stage (taken from the step's trace), every output
element against that stage's tolerance:
  - elementwise FP32 steps (draws, weights, dL/df, gradient assembly):
    8 u of the sum of the absolute terms (u = 2^-24);
  - the ray-trace: 1e-6 arcsec plus the ulp of beta;
  - the windows and the k-th-neighbour weights: 1e-5 of their scale;
  - the reductions and their VJPs: 2e-5 of the sum of absolute terms, plus,
    for the windowed ones, the derived FP32 rounding term and flush floor
    of the windowed tests.
The whole-chain FP64 comparison lives in test_gpu_svi."""
import math

import numpy as np
import pytest

from oracle import elbo as E
from paper_2105_09465_gb300 import svi, workloads as W
from tests.gpu_util import ALPHA_TOL, GRAD_REL, dev, host, need_gpu, ulp32
from tests.svi_case import case
from tests.test_gpu_windowed import windowed_tols

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def close(got, ref, tol, what):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    tol = np.broadcast_to(np.asarray(tol, np.float64), ref.shape) + 1e-30
    ratio = np.abs(got - ref) / tol
    if np.any(ratio > 1):
        k = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
        raise AssertionError(f"{what}: {int(np.sum(ratio > 1))} of {ratio.size} outside tolerance; worst {k}: "
                             f"got {got[k]!r} ref {ref[k]!r} tol {tol[k]!r}")


@pytest.fixture(scope="module")
def step():
    cfg, guide, data, eps_sp, eps_l = case()
    nx, ny, pix = cfg["pixels"]
    mc = svi.ModelConfig(pixels=W.Grid(nx, ny, 1, pix), source_grid=W.Grid(*cfg["source_grid"]),
                         sigma_sp=cfg["sigma_sp"], sigma_layers=cfg["sigma_layers"], alpha_sp=cfg["alpha_sp"],
                         alpha_layers=cfg["alpha_layers"], noise=cfg["noise"], gamma=cfg["gamma"],
                         knn_k=cfg["knn_k"])
    gd = svi.Guide(mu=dev(guide["mu"]), L=dev(guide["L"]), C=dev(guide["C"]), sd_sp=dev(guide["sd_sp"]),
                   mu_layers=[dev(a) for a in guide["mu_layers"]], sd_layers=[dev(a) for a in guide["sd_layers"]])
    T = {}
    loss, G = svi.loss_and_grads(mc, gd, dev(data), dev(eps_sp), [dev(e) for e in eps_l], trace=T)
    tr = {}
    for k, v in T.items():
        if isinstance(v, list):
            tr[k] = [({kk: host(vv) for kk, vv in x.items()} if isinstance(x, dict) else host(x)) for x in v]
        elif isinstance(v, dict):
            tr[k] = {kk: host(vv) for kk, vv in v.items()}
        else:
            tr[k] = host(v)
    grads = {k: (host(v) if not isinstance(v, list) else [host(x) for x in v]) for k, v in G.items()}
    return cfg, guide, data, eps_sp, eps_l, tr, grads


def test_draw(step):
    cfg, guide, data, eps_sp, eps_l, tr, G = step
    x, _ = E.partial_mvn_draw(guide["mu"], guide["L"], guide["C"], guide["sd_sp"], eps_sp)
    S = E.partial_mvn_scale(guide["L"], guide["C"], guide["sd_sp"])
    ab = np.abs(guide["mu"].astype(np.float64)) + np.abs(S) @ np.abs(eps_sp.astype(np.float64))
    close(tr["x"], x, 8 * U * ab, "partial MVN draw")
    for y, mu, sd, e in zip(tr["ys"], guide["mu_layers"], guide["sd_layers"], eps_l):
        ref = mu.astype(np.float64) + sd.astype(np.float64) * e
        close(y, ref, 8 * U * (np.abs(mu) + np.abs(sd * e)), "layer draw")


def test_ray_trace_windows_and_weights(orc, step):
    cfg, guide, data, eps_sp, eps_l, tr, G = step
    nx, ny, pix = cfg["pixels"]
    xi = orc.grid_points(nx, ny, 1, pix)
    th = tr["x"][:7].astype(np.float64)
    lens = (th[0], th[1], th[2], th[3], th[4], cfg["gamma"], th[5], th[6])
    _, bref = orc.raytrace(xi, lens)
    close(tr["beta"], bref, ALPHA_TOL + ulp32(bref), "ray-traced pixels")
    b = tr["beta"]
    zref = orc.pixel_shapes(b, nx, ny)
    close(tr["z"], zref, 1e-5 * np.abs(zref).max(axis=1, keepdims=True) + 1e-12, "pixel windows")
    for a_k, s in zip(tr["a_layers"], cfg["sigma_layers"]):
        aref = orc.transmission_weights(b, s, cfg["knn_k"])
        close(a_k, aref, 1e-5 * np.abs(aref), "transmission weights")


def source_plane(cfg, orc):
    yg = orc.grid_points(*cfg["source_grid"]).astype(np.float64)
    return yg, cfg["sigma_sp"] / math.sqrt(2.0)


def test_fluxes_and_likelihood(orc, step):
    """f = T_sp w_sp + sum_l T_l w_l on the GPU's points, windows and weights;
    dL/df and the nll from the GPU's f."""
    cfg, guide, data, eps_sp, eps_l, tr, G = step
    b, z = tr["beta"], tr["z"]
    yg, ell_sp = source_plane(cfg, orc)
    ref, ab = orc.kernel_matvec(b, yg, tr["w_sp"], ell_sp, 1.0)
    tol = 2e-5 * ab
    for w, s in zip(tr["w_layers"], cfg["sigma_layers"]):
        R, T = windowed_tols(orc, b, z, b, w, np.zeros(len(b)), s)
        ref = ref + R["out"]
        tol = tol + T["out"]
    close(tr["f"], ref, tol, "model fluxes")
    f = tr["f"].astype(np.float64)
    nll, g, _ = E.gaussian_nll(f, data, cfg["noise"])
    close(tr["g"], g, 8 * U * (np.abs(f) + np.abs(data)) / cfg["noise"] ** 2, "dL/df")
    assert abs(float(tr["nll"]) - nll) <= 1e-6 * abs(nll)


def test_reduction_gradients(orc, step):
    """The image-plane layer's and the source-plane layer's VJPs for the GPU's
    dL/df, element by element."""
    cfg, guide, data, eps_sp, eps_l, tr, G = step
    b, z, g = tr["beta"], tr["z"], tr["g"]
    for w, s, Gl in zip(tr["w_layers"], cfg["sigma_layers"], tr["layer_grads"]):
        R, T = windowed_tols(orc, b, z, b, w, g, s)
        for key, rk in (("v", "d_v"), ("p", "d_p"), ("q", "d_q"), ("z", "d_z")):
            close(Gl[key], R[rk], T[rk], f"image-plane layer {rk}")
    yg, ell_sp = source_plane(cfg, orc)
    Rs = orc.kernel_matvec_vjp(b, yg, tr["w_sp"], ell_sp, 1.0, g.astype(np.float64), with_abs=True)
    close(tr["source_grads"]["v"], Rs["d_v"], GRAD_REL * Rs["d_v_abs"], "source-plane d_v")
    close(tr["source_grads"]["x"], Rs["d_x"], GRAD_REL * Rs["d_x_abs"], "source-plane d_beta")


def test_lens_and_guide_gradients(orc, step):
    """dL/dbeta assembled from the layers, the lens gradient through the
    ray-trace VJP, and the guide gradients through the proposals' VJPs, each
    from the GPU's own inputs."""
    cfg, guide, data, eps_sp, eps_l, tr, G = step
    nx, ny, pix = cfg["pixels"]
    b = tr["beta"]
    parts = [tr["source_grads"]["x"]]
    dz = None
    for Gl in tr["layer_grads"]:
        parts += [Gl["p"], Gl["q"]]
        dz = Gl["z"] if dz is None else dz + Gl["z"]
    pv, pv_ab = orc.pixel_shapes_vjp(b, nx, ny, dz, with_abs=True)
    ref = sum(p.astype(np.float64) for p in parts) + pv
    ab = sum(np.abs(p.astype(np.float64)) for p in parts) + pv_ab
    close(G["d_beta"], ref, 8 * U * ab, "dL/dbeta")
    xi = orc.grid_points(nx, ny, 1, pix)
    th = tr["x"][:7].astype(np.float64)
    lens = (th[0], th[1], th[2], th[3], th[4], cfg["gamma"], th[5], th[6])
    rl, _, al, _ = orc.raytrace_vjp(xi, lens, None, G["d_beta"].astype(np.float64), 0, with_abs=True)
    close(G["d_lens"], rl, GRAD_REL * al, "lens gradient")
    # d_x = [d_lens, a_sp d_v + y_sp / alpha^2] and the partial-MVN VJP
    h = cfg["source_grid"][3] / cfg["source_grid"][2]
    s_sp = cfg["sigma_sp"]
    a_sp = math.sqrt(2.0 * math.pi) * s_sp * h / (math.pi * s_sp ** 2)
    y_sp = tr["x"][7:].astype(np.float64)
    dv = tr["source_grads"]["v"].astype(np.float64)
    d_ysp = a_sp * dv + y_sp / cfg["alpha_sp"] ** 2
    close(tr["d_x"][7:], d_ysp, 8 * U * (np.abs(a_sp * dv) + np.abs(y_sp) / cfg["alpha_sp"] ** 2), "dL/dy_sp")
    close(tr["d_x"][:7], G["d_lens"], 2 * U * np.abs(G["d_lens"]), "dL/dtheta packed")
    d_x = tr["d_x"].astype(np.float64)
    d_mu, d_L, d_C, d_sd = E.partial_mvn_vjp(guide["L"], guide["C"], guide["sd_sp"], eps_sp, d_x, 1.0)
    eps = np.abs(eps_sp.astype(np.float64))
    Gab = np.outer(np.abs(d_x), eps)
    D = 7
    L_ab = np.tril(Gab[:D, :D]) + np.diag(1.0 / np.abs(np.diag(guide["L"].astype(np.float64))))
    close(G["mu"], d_mu, 8 * U * np.abs(d_x), "d_mu")
    close(G["L"], d_L, 8 * U * L_ab, "d_L")
    close(G["C"], d_C, 8 * U * Gab[D:, :D], "d_C")
    close(G["sd_sp"], d_sd, 8 * U * (np.diag(Gab[D:, D:]) + 1.0 / np.abs(guide["sd_sp"])), "d_sd_sp")
    for a_k, Gl, mu, sd, e, al, gm, gs in zip(tr["a_layers"], tr["layer_grads"], guide["mu_layers"],
                                              guide["sd_layers"], eps_l, cfg["alpha_layers"], G["layers_mu"],
                                              G["layers_sd"]):
        d_y = (a_k * Gl["v"]).astype(np.float64)  # the product the step forms in FP32, exactly
        r_mu, r_sd, _ = E.diag_normal_vjp(mu, sd, e, al, d_y, 1.0, 1.0)
        y = mu.astype(np.float64) + sd.astype(np.float64) * e
        t_ab = np.abs(d_y) + np.abs(y) / al ** 2
        close(gm, r_mu, 8 * U * t_ab, "layer d_mu")
        close(gs, r_sd, 8 * U * (t_ab * np.abs(e) + 1.0 / np.abs(sd)), "layer d_sd")
