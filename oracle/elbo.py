"""ORACLE for the likelihood and ELBO terms: plain FP64 numpy definitions.

THIS IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the CUDA library never
calls it and shares no code with it.

Generative model (Sec. 3.3): d ~ N(f, diag(sigma^2)), f = T y,
y ~ N(0, alpha^2 I). The observed pixel is the local average of its S x S
supersampled model fluxes (Sec. 4.1 makes mock images that way). The ELBO
(Sec. 3.6) for one reparameterised draw is
    ln p(d | f) + ln p(y) - ln q(y),
so the loss minimised is
    nll(d | f) - ln p(y | alpha) + ln q(y).
Proposals: a diagonal normal per source parameter (Sec. 3.7, mean-field
proposal), and the "partial" multivariate normal over the lens parameters and
the source-plane layer (Sec. 4.2): x = mu + L_full eps with
    L_full = [[L, 0], [C, diag(sd)]],
L lower triangular with a positive diagonal. Uniform lens priors (Table 1)
add a constant and are left out.
"""
import numpy as np

LOG_2PI = np.log(2.0 * np.pi)


def pixel_average(f, nx, ny, ss):
    """Pixel model fluxes: mean of each ss x ss block of the (nx ss) x (ny ss)
    supersampled grid (row-major over y, like the grid points)."""
    f = np.asarray(f, np.float64).reshape(ny * ss, nx * ss)
    out = np.zeros((ny, nx))
    for a in range(ss):
        for b in range(ss):
            out += f[a::ss, b::ss]
    return (out / (ss * ss)).reshape(-1)


def gaussian_nll(f, data, sigma, nx=None, ny=None, ss=1):
    """(nll, g, model): nll = sum_p [ (m_p - d_p)^2 / (2 sigma_p^2) + ln sigma_p ]
    + (P/2) ln 2 pi over the P pixels with model m = pixel_average(f), and
    g = d nll / d f per supersampled point = (m_p - d_p) / (sigma_p^2 ss^2)."""
    f = np.asarray(f, np.float64)
    d = np.asarray(data, np.float64).reshape(-1)
    if nx is None:
        nx, ny, ss = d.size, 1, 1
    m = pixel_average(f, nx, ny, ss)
    s = np.broadcast_to(np.asarray(sigma, np.float64), d.shape)
    r = m - d
    nll = np.sum(0.5 * r * r / (s * s) + np.log(s)) + 0.5 * d.size * LOG_2PI
    gp = (r / (s * s) / (ss * ss)).reshape(ny, nx)
    g = np.repeat(np.repeat(gp, ss, axis=0), ss, axis=1).reshape(-1)
    return nll, g, m


def diag_normal_draw(mu, sd, eps, alpha):
    """(y, neg_log_prior, log_q): y = mu + sd eps;
    -ln p(y | alpha) = sum y^2 / (2 alpha^2) + M ln alpha + (M/2) ln 2 pi;
    ln q(y) = sum [ -eps^2/2 - ln sd ] - (M/2) ln 2 pi."""
    mu, sd, eps = (np.asarray(a, np.float64) for a in (mu, sd, eps))
    y = mu + sd * eps
    M = y.size
    nlp = np.sum(y * y) / (2 * alpha * alpha) + M * np.log(alpha) + 0.5 * M * LOG_2PI
    logq = np.sum(-0.5 * eps * eps - np.log(sd)) - 0.5 * M * LOG_2PI
    return y, nlp, logq


def diag_normal_vjp(mu, sd, eps, alpha, d_y, w_prior=1.0, w_q=1.0):
    """Gradients of  Loss = L(y) + w_prior (-ln p(y | alpha)) + w_q ln q(y)
    with dL/dy = d_y, through y = mu + sd eps at fixed eps:
    (d_mu, d_sd, d_alpha)."""
    mu, sd, eps, d_y = (np.asarray(a, np.float64) for a in (mu, sd, eps, d_y))
    y = mu + sd * eps
    t = d_y + w_prior * y / (alpha * alpha)
    d_alpha = w_prior * (y.size / alpha - np.sum(y * y) / alpha ** 3)
    return t, t * eps - w_q / sd, d_alpha


def partial_mvn_scale(L, C, sd):
    """The full lower-triangular scale matrix [[L, 0], [C, diag(sd)]]."""
    L, C, sd = (np.asarray(a, np.float64) for a in (L, C, sd))
    D, M = L.shape[0], sd.size
    S = np.zeros((D + M, D + M))
    S[:D, :D] = np.tril(L)
    S[D:, :D] = C
    S[D:, D:] = np.diag(sd)
    return S


def partial_mvn_draw(mu, L, C, sd, eps):
    """(x, log_q): x = mu + L_full eps, ln q(x) = -|eps|^2/2 - sum ln diag(L)
    - sum ln sd - ((D + M)/2) ln 2 pi (the density of N(mu, L_full L_full^T))."""
    S = partial_mvn_scale(L, C, sd)
    eps = np.asarray(eps, np.float64)
    x = np.asarray(mu, np.float64) + S @ eps
    logq = -0.5 * eps @ eps - np.sum(np.log(np.diag(S))) - 0.5 * eps.size * LOG_2PI
    return x, logq


def partial_mvn_vjp(L, C, sd, eps, d_x, w_q=1.0):
    """Gradients of Loss = L(x) + w_q ln q(x) with dL/dx = d_x through
    x = mu + L_full eps at fixed eps: (d_mu, d_L (lower part, D x D), d_C, d_sd)."""
    L = np.asarray(L, np.float64)
    D = L.shape[0]
    eps, d_x = np.asarray(eps, np.float64), np.asarray(d_x, np.float64)
    G = np.outer(d_x, eps)  # d x / d L_full contracted with d_x
    d_L = np.tril(G[:D, :D])
    d_L[np.diag_indices(D)] -= w_q / np.diag(L)
    d_C = G[D:, :D]
    d_sd = np.diag(G[D:, D:]) - w_q / np.asarray(sd, np.float64)
    return d_x.copy(), d_L, d_C, d_sd
