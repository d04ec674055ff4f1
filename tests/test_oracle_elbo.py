"""Pins of the likelihood and ELBO-term oracle (Sec. 3.3, 3.6, 3.7, 4.2)
against library densities, closed forms and FP64 central differences."""
import numpy as np
import pytest
from scipy import stats

from oracle import elbo as E


def cdiff(fn, x, h=1e-6):
    x = np.array(x, np.float64)
    g = np.zeros_like(x)
    for i in np.ndindex(x.shape):
        a, b = x.copy(), x.copy()
        a[i] += h
        b[i] -= h
        g[i] = (fn(a) - fn(b)) / (2 * h)
    return g


def test_nll_is_the_gaussian_log_density():
    rng = np.random.default_rng(0)
    f, d, s = rng.normal(size=50), rng.normal(size=50), rng.uniform(0.5, 2, 50)
    nll, g, m = E.gaussian_nll(f, d, s)
    assert nll == pytest.approx(-stats.norm.logpdf(d, f, s).sum(), rel=1e-13)
    np.testing.assert_allclose(m, f)
    np.testing.assert_allclose(g, (f - d) / s ** 2, rtol=1e-14)


def test_pixel_average_of_a_linear_field_is_its_value_at_the_pixel_centre(orc):
    """Subpixel centres are symmetric about the pixel centre, so averaging a
    linear field over them gives the field at the centre (nx != ny pins the
    block layout)."""
    nx, ny, ss, pix = 7, 5, 3, 0.1
    xs = orc.grid_points(nx, ny, ss, pix).astype(np.float64)
    xp = orc.grid_points(nx, ny, 1, pix).astype(np.float64)
    f = 0.3 + 1.7 * xs[:, 0] - 2.1 * xs[:, 1]
    np.testing.assert_allclose(E.pixel_average(f, nx, ny, ss), 0.3 + 1.7 * xp[:, 0] - 2.1 * xp[:, 1], atol=1e-6)


def test_nll_gradient_by_central_differences():
    rng = np.random.default_rng(1)
    nx, ny, ss = 4, 3, 2
    f = rng.normal(size=nx * ny * ss * ss)
    d, s = rng.normal(size=nx * ny), rng.uniform(0.5, 2, nx * ny)
    _, g, _ = E.gaussian_nll(f, d, s, nx, ny, ss)
    np.testing.assert_allclose(g, cdiff(lambda z: E.gaussian_nll(z, d, s, nx, ny, ss)[0], f), rtol=1e-7, atol=1e-9)


def test_diag_normal_terms_are_library_log_densities():
    rng = np.random.default_rng(2)
    mu, sd, eps = rng.normal(size=40), rng.uniform(0.1, 1, 40), rng.normal(size=40)
    y, nlp, logq = E.diag_normal_draw(mu, sd, eps, 0.7)
    np.testing.assert_allclose(y, mu + sd * eps)
    assert nlp == pytest.approx(-stats.norm.logpdf(y, 0, 0.7).sum(), rel=1e-13)
    assert logq == pytest.approx(stats.norm.logpdf(y, mu, sd).sum(), rel=1e-13)


def test_diag_normal_vjp_by_central_differences():
    rng = np.random.default_rng(3)
    M = 12
    mu, sd, eps, w = rng.normal(size=M), rng.uniform(0.2, 1, M), rng.normal(size=M), rng.normal(size=M)
    alpha, wp, wq = 0.8, 0.6, 1.3

    def loss(mu_, sd_, a_):
        y, nlp, lq = E.diag_normal_draw(mu_, sd_, eps, a_)
        return w @ y + wp * nlp + wq * lq

    d_mu, d_sd, d_a = E.diag_normal_vjp(mu, sd, eps, alpha, w, wp, wq)
    np.testing.assert_allclose(d_mu, cdiff(lambda z: loss(z, sd, alpha), mu), rtol=1e-7)
    np.testing.assert_allclose(d_sd, cdiff(lambda z: loss(mu, z, alpha), sd), rtol=1e-7)
    assert d_a == pytest.approx(cdiff(lambda z: loss(mu, sd, z[0]), [alpha])[0], rel=1e-7)


def partial(rng, D=7, M=30):
    L = np.tril(rng.normal(0, 0.3, (D, D)))
    L[np.diag_indices(D)] = rng.uniform(0.2, 1.0, D)
    return rng.normal(size=D + M), L, rng.normal(0, 0.2, (M, D)), rng.uniform(0.1, 0.5, M), rng.normal(size=D + M)


def test_partial_mvn_log_q_is_the_library_mvn_density():
    """Sec. 4.2: ln q of the draw equals the N(mu, L_full L_full^T) log density."""
    mu, L, C, sd, eps = partial(np.random.default_rng(4))
    x, logq = E.partial_mvn_draw(mu, L, C, sd, eps)
    S = E.partial_mvn_scale(L, C, sd)
    assert logq == pytest.approx(stats.multivariate_normal.logpdf(x, mu, S @ S.T), rel=1e-10)
    # lens block covariance L L^T, source block sd^2 + C C^T (Sec. 4.2)
    cov = S @ S.T
    np.testing.assert_allclose(cov[:7, :7], L @ L.T)
    np.testing.assert_allclose(cov[7:, 7:], np.diag(sd ** 2) + C @ C.T)


def test_partial_mvn_vjp_by_central_differences():
    rng = np.random.default_rng(5)
    mu, L, C, sd, eps = partial(rng, D=3, M=5)
    w, wq = rng.normal(size=8), 0.9

    def loss(mu_, L_, C_, sd_):
        x, lq = E.partial_mvn_draw(mu_, L_, C_, sd_, eps)
        return w @ x + wq * lq

    d_mu, d_L, d_C, d_sd = E.partial_mvn_vjp(L, C, sd, eps, w, wq)
    np.testing.assert_allclose(d_mu, cdiff(lambda z: loss(z, L, C, sd), mu), rtol=1e-7)
    np.testing.assert_allclose(d_L, np.tril(cdiff(lambda z: loss(mu, z, C, sd), L)), rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(d_C, cdiff(lambda z: loss(mu, L, z, sd), C), rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(d_sd, cdiff(lambda z: loss(mu, L, C, z), sd), rtol=1e-7)


def test_svi_step_gradients_by_central_differences(orc):
    """The oracle's composed SVI loss (ray-trace, both GP layers, windows,
    likelihood, prior and proposal terms) against its own analytic
    gradients, weights held fixed: lens means, source weights, scale
    parameters and image-plane layer parameters."""
    from oracle import svi
    from tests.svi_case import case
    cfg, guide, data, eps_sp, eps_l = case()
    g64 = {k: (np.asarray(v, np.float64) if not isinstance(v, list) else [np.asarray(x, np.float64) for x in v])
           for k, v in guide.items()}
    loss, G = svi.loss_and_grads(orc, cfg, g64, data, eps_sp, eps_l)
    A = G["A"]

    def L_of(key, idx, val, sub=None):
        gg = {k: (v.copy() if not isinstance(v, list) else [x.copy() for x in v]) for k, v in g64.items()}
        arr = gg[key] if sub is None else gg[key][sub]
        arr[idx] = val
        return svi.loss_and_grads(orc, cfg, gg, data, eps_sp, eps_l, A_fixed=A)[0]

    def fd(key, idx, h, sub=None):
        base = (g64[key] if sub is None else g64[key][sub])[idx]
        return (L_of(key, idx, base + h, sub) - L_of(key, idx, base - h, sub)) / (2 * h)

    for j in range(7):
        assert G["mu"][j] == pytest.approx(fd("mu", j, 1e-6), rel=2e-5, abs=1e-3), f"mu[{j}]"
    for j in (7, 50, 200):
        assert G["mu"][j] == pytest.approx(fd("mu", j, 1e-5), rel=1e-6, abs=1e-6), f"mu[{j}]"
    assert G["L"][4, 4] == pytest.approx(fd("L", (4, 4), 1e-6), rel=2e-5)
    assert G["C"][10, 2] == pytest.approx(fd("C", (10, 2), 1e-6), rel=2e-5, abs=1e-6)
    assert G["sd_sp"][3] == pytest.approx(fd("sd_sp", 3, 1e-6), rel=1e-6)
    for j in (0, 300):
        assert G["layers_mu"][0][j] == pytest.approx(fd("mu_layers", j, 1e-5, sub=0), rel=1e-6, abs=1e-6)
        assert G["layers_sd"][0][j] == pytest.approx(fd("sd_layers", j, 1e-7, sub=0), rel=1e-5, abs=1e-5)
