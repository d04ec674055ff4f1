"""One stochastic-variational-inference step of the paper's lensed-GP model,
composed from the library's kernels (Sec. 3.3 generative model, Sec. 3.4
transmission, Sec. 3.6 ELBO, Sec. 4.2 proposals).

Model for one draw:
  theta (7 lens and shear parameters) and the source-plane layer y_sp are
  drawn jointly from the partial multivariate-normal proposal; every
  image-plane layer y_l from its diagonal-normal proposal;
  beta = ray-trace of the pixel centres through theta;
  f = T_sp y_sp + sum_l T_l y_l with
    T_sp: the stationary reduction of beta against the source grid
          (length scale sigma_sp / sqrt(2), weights A |pi Sigma|^-1/2 y_sp,
          A from the grid's exact density),
    T_l:  the windowed reduction of beta against beta itself (the
          image-plane layer), windows from the projected pixel grid, weights
          A_k y_l with A_k from the k = 20 nearest-neighbour density;
  loss = nll(d | f) - ln p(y | alpha) + ln q, minus the ELBO estimate.
The lens priors are uniform (constant inside their domain) and left out;
the transmission weights A_k are held fixed within a step.

Every numerical step runs in the library's CUDA kernels, the elementwise
ones (A y, the sum of the layers, dL/dbeta summed over the layers, the
source-plane prior gradient y_sp / alpha^2, the loss's sum of terms)
included; the last image-plane layer forms the likelihood in its epilogue.
The 7 drawn lens parameters stay on the device (lens_prepare turns them
into the ray-trace's lens record). This module only orders the calls and
allocates their outputs; nothing is copied to the host, so a step can be
timed with CUDA events or captured in a graph.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from . import api
from .workloads import Grid, Lens

N_LENS = 7  # x0, y0, q, phi, theta_e, g1, g2 (the slope is held fixed)


@dataclass
class ModelConfig:
    pixels: Grid                 # image pixel centres (ss = 1)
    source_grid: Grid            # source-plane inducing points
    sigma_sp: float              # source-plane layer kernel size
    sigma_layers: list[float]    # image-plane layer kernel sizes
    alpha_sp: float              # prior scale of y_sp
    alpha_layers: list[float]    # prior scales of the image-plane layers
    noise: float                 # pixel noise standard deviation
    gamma: float = 2.0           # fixed SPLE slope
    knn_k: int = 20


@dataclass
class Guide:
    """Variational parameters (Table 2): partial MVN over (theta, y_sp),
    diagonal normals over the image-plane layers. All float32 CUDA."""
    mu: torch.Tensor             # (7 + M,)
    L: torch.Tensor              # (7, 7) lower triangular, positive diagonal
    C: torch.Tensor              # (M, 7)
    sd_sp: torch.Tensor          # (M,)
    mu_layers: list[torch.Tensor] = field(default_factory=list)
    sd_layers: list[torch.Tensor] = field(default_factory=list)


def lens_from(theta: list[float], gamma: float) -> Lens:
    x0, y0, q, phi, te, g1, g2 = theta
    return Lens(x0, y0, q, phi, te, gamma, g1, g2)


_UNIT = {}


def _unit_draw(M: int, dev) -> tuple[torch.Tensor, torch.Tensor]:
    """(ones, zeros) of length M: the draw y = y_sp with sd 1 and eps 0 gives
    the source-plane prior term -ln p(y_sp | alpha_sp)."""
    key = (M, str(dev))
    if key not in _UNIT:
        _UNIT[key] = (torch.ones(M, device=dev), torch.zeros(M, device=dev))
    return _UNIT[key]


def loss_and_grads(cfg: ModelConfig, guide: Guide, data: torch.Tensor, eps_sp: torch.Tensor,
                   eps_layers: list[torch.Tensor], trace: dict | None = None) -> tuple[torch.Tensor, dict]:
    """Loss of one reparameterised draw (given the standard-normal draws), as
    a (1,) float64 device tensor, and its gradients with respect to every
    guide parameter. `trace`, when given, receives the step's intermediate
    device tensors (the draw, the ray-traced pixels, windows, weights, model
    fluxes, dL/df and the layers' gradients) for inspection."""
    dev = data.device
    M = guide.sd_sp.numel()
    W, H = cfg.pixels.nx, cfg.pixels.ny
    # ---- draws and their log densities
    x, logq_sp = api.partial_mvn_draw(guide.mu, guide.L, guide.C, guide.sd_sp, eps_sp)
    lens_rec = api.lens_prepare(x[:N_LENS], cfg.gamma)
    y_sp = x[N_LENS:]
    ys, terms = [], []
    for mu, sd, e, a in zip(guide.mu_layers, guide.sd_layers, eps_layers, cfg.alpha_layers):
        y, t = api.diag_normal_draw(mu, sd, e, a)
        ys.append(y)
        terms.append(t)
    ones_sp, zeros_sp = _unit_draw(M, dev)
    _, prior_sp = api.diag_normal_draw(y_sp, ones_sp, zeros_sp, cfg.alpha_sp)

    # ---- forward
    pix = api.Points(grid=cfg.pixels, lens_record=lens_rec)
    beta = api.lens_raytrace(pix)
    h = cfg.source_grid.pix / cfg.source_grid.ss
    a_sp = math.sqrt(2.0 * math.pi) * cfg.sigma_sp * h / (math.pi * cfg.sigma_sp ** 2)  # A |pi Sigma|^-1/2
    src = api.Points(grid=cfg.source_grid)
    w_sp = api.vec_axpby(a_sp, y_sp)
    f = api.gp_kernel_matvec(api.Points(xy=beta), src, w_sp, cfg.sigma_sp / math.sqrt(2.0), 1.0)
    z = api.pixel_shapes(beta, W, H)
    self_pts = api.Points(xy=beta, grid=cfg.pixels)  # the pixels in their image layout
    a_layers, w_layers = [], []
    nll = g = None
    for li, (y, s) in enumerate(zip(ys, cfg.sigma_layers)):
        a_k = api.knn_density(beta, cfg.knn_k, lengthscale=s, want_r2=False)
        w = api.vec_mul(a_k, y)
        if li + 1 < len(ys):
            api.vec_axpby(1.0, f, 1.0, api.gp_windowed_matvec(beta, z, self_pts, w, s, layout=cfg.pixels), out=f)
        else:
            # the last layer: the model total, dL/df and the likelihood in its epilogue
            f, g, nll = api.gp_windowed_matvec_nll(beta, z, self_pts, w, s, data, cfg.noise, f_in=f,
                                                   layout=cfg.pixels)
        a_layers.append(a_k)
        w_layers.append(w)
    if nll is None:
        nll, g, _ = api.gaussian_nll(f, data, cfg.noise)
    if trace is not None:
        trace.update(x=x, beta=beta, z=z, f=f, g=g, nll=nll, ys=ys, a_layers=a_layers, w_layers=w_layers,
                     w_sp=w_sp)

    # ---- backward: dL/dbeta summed over the layers (in place)
    d_beta = d_z = None
    grads = {"layers_mu": [], "layers_sd": []}
    for y, s, a_k, w, mu, sd, e, al in zip(ys, cfg.sigma_layers, a_layers, w_layers, guide.mu_layers,
                                           guide.sd_layers, eps_layers, cfg.alpha_layers):
        G = api.gp_windowed_matvec_bwd(beta, z, self_pts, w, s, g, want=("v", "p", "q", "z"), layout=cfg.pixels)
        if d_beta is None:
            d_beta = api.vec_axpby(1.0, G["p"], 1.0, G["q"])
            d_z = G["z"]
        else:
            api.vec_axpby(1.0, d_beta, 1.0, G["p"], out=d_beta)
            api.vec_axpby(1.0, d_beta, 1.0, G["q"], out=d_beta)
            api.vec_axpby(1.0, d_z, 1.0, G["z"], out=d_z)
        if trace is not None:
            trace.setdefault("layer_grads", []).append(G)
        d_mu, d_sd, _ = api.diag_normal_vjp(mu, sd, e, al, api.vec_mul(a_k, G["v"]), 1.0, 1.0)
        grads["layers_mu"].append(d_mu)
        grads["layers_sd"].append(d_sd)
    Gs = api.gp_kernel_matvec_bwd(api.Points(xy=beta), src, w_sp, cfg.sigma_sp / math.sqrt(2.0), 1.0, g,
                                  want=("v", "x"))
    if d_beta is None:
        d_beta = api.vec_axpby(1.0, Gs["x"])
    else:
        api.vec_axpby(1.0, d_beta, 1.0, api.pixel_shapes_vjp(beta, W, H, d_z), out=d_beta)
        api.vec_axpby(1.0, d_beta, 1.0, Gs["x"], out=d_beta)
    d_lens, _ = api.lens_raytrace_vjp(pix, d_beta)
    if trace is not None:
        trace.update(source_grads=Gs)
    # the source-plane layer's weights and its prior: d(-ln p)/dy_sp = y_sp / alpha^2
    d_ysp = api.vec_axpby(a_sp, Gs["v"], 1.0 / cfg.alpha_sp ** 2, y_sp)
    d_x = api.vec_pack(d_lens, d_ysp)
    if trace is not None:
        trace.update(d_x=d_x)
    d_mu, d_L, d_C, d_sd = api.partial_mvn_vjp(guide.L, guide.sd_sp, eps_sp, d_x, 1.0)
    grads.update(mu=d_mu, L=d_L, C=d_C, sd_sp=d_sd, d_lens=d_lens, d_beta=d_beta)

    parts = [nll.reshape(1), prior_sp[0:1], logq_sp.reshape(1)]
    for t in terms:
        parts += [t[0:1], t[1:2]]
    loss = api.sum_scalars(parts)
    return loss, grads
