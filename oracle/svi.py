"""ORACLE for one SVI step of the lensed-GP model: the loss of one
reparameterised draw and its gradients, composed in FP64 from the oracle's
ray-trace, reductions, windows, density estimate and ELBO terms, in the
order the model defines (Sec. 3.3 generative model, Sec. 3.4 transmission,
Sec. 3.6 ELBO, Sec. 4.2 proposals).

THIS IS TEST INFRASTRUCTURE: only the test suite, the smoke check and the
benchmark's CPU legs may import it.

Conventions (the same as the library's driver): the source-plane layer
uses the stationary kernel with length scale sigma/sqrt(2) and weights
A |pi Sigma|^-1/2 y with A = sqrt(2 pi) sigma h from the grid's exact
density 1/h^2; image-plane layers use the windowed kernel of the projected
pixels against themselves with weights A_k y, A_k from the k-nearest
neighbour density; A is held fixed within a step; lens priors are uniform.
"""
import math

import numpy as np

from . import elbo as E

N_LENS = 7


def _lens(theta, gamma):
    x0, y0, q, phi, te, g1, g2 = theta
    return (x0, y0, q, phi, te, gamma, g1, g2)


def loss_and_grads(orc, cfg, guide, data, eps_sp, eps_layers, A_fixed=None):
    """cfg: dict(pixels=(nx, ny, pix), source_grid=(nx, ny, ss, pix, cx, cy),
    sigma_sp, sigma_layers, alpha_sp, alpha_layers, noise, gamma, knn_k);
    guide: dict(mu, L, C, sd_sp, mu_layers, sd_layers) of numpy arrays;
    A_fixed: optional per-layer weights to use instead of the density
    estimate (the gradients treat the weights as fixed either way).
    Returns (loss, grads dict); grads["A"] holds the weights used."""
    nx, ny, pix = cfg["pixels"]
    xi = orc.grid_points(nx, ny, 1, pix).astype(np.float64)
    yg = orc.grid_points(*cfg["source_grid"]).astype(np.float64)
    h = cfg["source_grid"][3] / cfg["source_grid"][2]
    x, logq_sp = E.partial_mvn_draw(guide["mu"], guide["L"], guide["C"], guide["sd_sp"], eps_sp)
    theta, y_sp = x[:N_LENS], x[N_LENS:]
    lens = _lens(theta, cfg["gamma"])
    _, beta = orc.raytrace(xi, lens)
    s_sp = cfg["sigma_sp"]
    a_sp = math.sqrt(2.0 * math.pi) * s_sp * h / (math.pi * s_sp ** 2)
    f, _ = orc.kernel_matvec(beta, yg, a_sp * y_sp, s_sp / math.sqrt(2.0), 1.0)
    z = orc.pixel_shapes(beta, nx, ny)
    ys, loss_terms, A = [], 0.0, []
    for li, (mu, sd, e, al, s) in enumerate(zip(guide["mu_layers"], guide["sd_layers"], eps_layers,
                                               cfg["alpha_layers"], cfg["sigma_layers"])):
        y, nlp, lq = E.diag_normal_draw(mu, sd, e, al)
        a_k = orc.transmission_weights(beta, s, cfg["knn_k"]) if A_fixed is None else A_fixed[li]
        f = f + orc.windowed_matvec(beta, z, beta, a_k * y, s)[0]
        ys.append(y)
        A.append(a_k)
        loss_terms += nlp + lq
    nll, g, _ = E.gaussian_nll(f, data, cfg["noise"])
    al_sp = cfg["alpha_sp"]
    prior_sp = np.sum(y_sp ** 2) / (2 * al_sp ** 2) + y_sp.size * (math.log(al_sp) + 0.5 * E.LOG_2PI)
    loss = nll + prior_sp + logq_sp + loss_terms

    d_beta = np.zeros_like(beta)
    d_z = np.zeros_like(z)
    grads = {"layers_mu": [], "layers_sd": []}
    for y, a_k, mu, sd, e, al, s in zip(ys, A, guide["mu_layers"], guide["sd_layers"], eps_layers,
                                        cfg["alpha_layers"], cfg["sigma_layers"]):
        R = orc.windowed_vjp(beta, z, beta, a_k * y, s, g)
        d_beta += R["d_p"] + R["d_q"]
        d_z += R["d_z"]
        d_mu, d_sd, _ = E.diag_normal_vjp(mu, sd, e, al, a_k * R["d_v"], 1.0, 1.0)
        grads["layers_mu"].append(d_mu)
        grads["layers_sd"].append(d_sd)
    d_beta += orc.pixel_shapes_vjp(beta, nx, ny, d_z)
    Rs = orc.kernel_matvec_vjp(beta, yg, a_sp * y_sp, s_sp / math.sqrt(2.0), 1.0, g)
    d_beta += Rs["d_x"]
    d_lens, _ = orc.raytrace_vjp(xi, lens, None, d_beta)
    d_x = np.concatenate([d_lens, a_sp * Rs["d_v"] + y_sp / al_sp ** 2])
    d_mu, d_L, d_C, d_sd = E.partial_mvn_vjp(guide["L"], guide["C"], guide["sd_sp"], eps_sp, d_x, 1.0)
    grads.update(mu=d_mu, L=d_L, C=d_C, sd_sp=d_sd, d_lens=d_lens, d_beta=d_beta, A=A)
    return loss, grads
