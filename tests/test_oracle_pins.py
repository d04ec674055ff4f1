"""Pins of the FP64 oracle against facts fixed independently of it: closed
forms, library special functions, quadrature of the 3-D density, the
divergence theorem for lensing (div alpha = 2 kappa), finite differences and
brute force. Every case is chosen so that a plausible slip (dropped term,
wrong sign, swapped operand, wrong frame or normalisation) fails it."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_2105_09465_gb300 import workloads as W

RNG = np.random.default_rng(1234)


def lens(**kw):
    base = dict(x0=0.0, y0=0.0, q=1.0, phi=0.0, theta_e=1.2, gamma=2.0, g1=0.0, g2=0.0)
    base.update(kw)
    return base


def pts(n, hw=3.0, rng=RNG):
    return rng.uniform(-hw, hw, size=(n, 2))


# ---------------------------------------------------------------- pixel grid
def test_grid_points_definition(orc):
    xi = orc.grid_points(3, 2, 2, 0.05, 0.25, -0.5).astype(np.float64)
    assert xi.shape == (6 * 4, 2)
    # row-major over y, x fastest; spacing pix/ss; centred on (cx, cy)
    g = xi.reshape(4, 6, 2)
    assert np.all(np.diff(g[..., 0], axis=1) > 0) and np.all(np.diff(g[..., 1], axis=0) > 0)
    np.testing.assert_allclose(np.diff(g[..., 0], axis=1), 0.025, rtol=1e-6)
    np.testing.assert_allclose(g[..., 0].mean(), 0.25, atol=1e-7)
    np.testing.assert_allclose(g[..., 1].mean(), -0.5, atol=1e-7)


def test_grid_supersampling_averages_to_coarse_centres(orc):
    """S x S subpixel centres average to the coarse pixel centre."""
    coarse = orc.grid_points(10, 8, 1, 0.05).astype(np.float64).reshape(8, 10, 2)
    fine = orc.grid_points(10, 8, 2, 0.05).astype(np.float64).reshape(8, 2, 10, 2, 2)
    np.testing.assert_allclose(fine.mean(axis=(1, 3)), coarse, atol=2e-8)


def test_grid_points_are_fp32_values(orc):
    xi = orc.grid_points(7, 5, 3, 0.05, 0.1, 0.2)
    assert xi.dtype == np.float32
    # symmetric about the centre (cx, cy) up to one FP32 rounding
    g = xi.astype(np.float64).reshape(15, 21, 2)
    np.testing.assert_allclose(g[..., 0] + g[:, ::-1, 0], 0.2, atol=1e-7)


# ---------------------------------------------------------------- SPLE
def test_sis_constant_magnitude(orc):
    """q = 1, gamma = 2: |alpha| = theta_E everywhere, radial."""
    x = pts(500)
    a, b = orc.raytrace(x, lens(theta_e=1.3))
    np.testing.assert_allclose(np.hypot(a[:, 0], a[:, 1]), 1.3, rtol=1e-13)
    np.testing.assert_allclose(a[:, 0] * x[:, 1] - a[:, 1] * x[:, 0], 0.0, atol=1e-12)
    np.testing.assert_allclose(b, x - a, atol=0)


@pytest.mark.parametrize("gamma", [1.5, 1.8, 2.2, 2.7])
def test_circular_power_law(orc, gamma):
    """q = 1: alpha = R kappa_bar(<R) = theta_E (theta_E / R)^(gamma-2), radial."""
    x = pts(300) + np.array([0.3, -0.2])
    a, _ = orc.raytrace(x, lens(x0=0.3, y0=-0.2, gamma=gamma, phi=0.7))
    d = x - np.array([0.3, -0.2])
    R = np.hypot(d[:, 0], d[:, 1])
    mag = 1.2 * (1.2 / R) ** (gamma - 2)
    np.testing.assert_allclose(a, d / R[:, None] * mag[:, None], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("q,phi", [(0.8, math.pi / 6), (0.2753, 1.1), (0.5, -0.4)])
def test_sie_artanh_closed_form(orc, q, phi):
    """gamma = 2: 2F1(1, 1/2; 3/2; z) = artanh(sqrt z)/sqrt z (textbook)."""
    x = pts(300)
    a, _ = orc.raytrace(x, lens(q=q, phi=phi))
    c, s = math.cos(phi), math.sin(phi)
    u = c * x[:, 0] + s * x[:, 1]
    v = -s * x[:, 0] + c * x[:, 1]
    Rx, Ry = math.sqrt(q) * u, v / math.sqrt(q)
    e = (Rx + 1j * Ry) / np.hypot(Rx, Ry)
    z = -(1 - q) / (1 + q) * e ** 2
    F = np.arctanh(np.sqrt(z)) / np.sqrt(z)
    ap = 1.2 * 2 * math.sqrt(q) / (1 + q) * F * e
    ab = ap * (c + 1j * s)  # rotate back by +phi
    np.testing.assert_allclose(a[:, 0] + 1j * a[:, 1], ab, rtol=1e-12)


@pytest.mark.parametrize("gamma,q", [(1.8, 0.6), (2.2, 0.9), (2.05, 0.3)])
def test_sple_matches_scipy_hyp2f1(orc, gamma, q):
    x = pts(200)
    phi = 0.3
    a, _ = orc.raytrace(x, lens(q=q, phi=phi, gamma=gamma))
    c, s = math.cos(phi), math.sin(phi)
    u = c * x[:, 0] + s * x[:, 1]
    v = -s * x[:, 0] + c * x[:, 1]
    Rx, Ry = math.sqrt(q) * u, v / math.sqrt(q)
    R = np.hypot(Rx, Ry)
    e = (Rx + 1j * Ry) / R
    z = -(1 - q) / (1 + q) * e ** 2
    F = special.hyp2f1(1.0, (gamma - 1) / 2, (5 - gamma) / 2, z)
    ap = 1.2 * 2 * math.sqrt(q) / (1 + q) * (1.2 / R) ** (gamma - 2) * F * e
    np.testing.assert_allclose(a[:, 0] + 1j * a[:, 1], ap * (c + 1j * s), rtol=1e-10)


def _div_curl(orc, x, L, sub=None, profile=0, h=1e-5):
    def alpha(p):
        return orc.raytrace(p, L, sub, profile)[0]
    ex, ey = np.array([h, 0.0]), np.array([0.0, h])
    axp, axm = alpha(x + ex), alpha(x - ex)
    ayp, aym = alpha(x + ey), alpha(x - ey)
    div = (axp[:, 0] - axm[:, 0] + ayp[:, 1] - aym[:, 1]) / (2 * h)
    curl = (axp[:, 1] - axm[:, 1] - (ayp[:, 0] - aym[:, 0])) / (2 * h)
    return div, curl


@pytest.mark.parametrize("gamma,q,phi", [(2.0, 0.8, 0.52), (1.8, 0.6, 2.0), (2.2, 0.35, -1.0)])
def test_sple_divergence_is_twice_convergence(orc, gamma, q, phi):
    """Poisson equation: div alpha = 2 kappa with kappa from the SPLE surface
    density; curl alpha = 0. Pins the frame, rotation and normalisation."""
    L = lens(x0=0.1, y0=-0.05, q=q, phi=phi, gamma=gamma)
    x = pts(200, 2.5)
    x = x[np.hypot(x[:, 0] - 0.1, x[:, 1] + 0.05) > 0.2]
    div, curl = _div_curl(orc, x, L)
    kap = np.array([orc.sple_kappa(p[0], p[1], L) for p in x])
    np.testing.assert_allclose(div, 2 * kap, rtol=1e-6)
    np.testing.assert_allclose(curl, 0.0, atol=1e-6 * np.max(kap))


def test_sple_zero_at_centre(orc):
    a, _ = orc.raytrace(np.array([[0.1, -0.2]]), lens(x0=0.1, y0=-0.2, q=0.7))
    assert np.all(a == 0.0)


# ---------------------------------------------------------------- external shear
def test_shear_linear_symmetric_traceless(orc):
    L = lens(theta_e=0.0, g1=0.03, g2=-0.02)
    x1, x2 = pts(50), pts(50)
    a1 = orc.raytrace(x1, L)[0]
    a2 = orc.raytrace(x2, L)[0]
    a12 = orc.raytrace(2.5 * x1 - 0.7 * x2, L)[0]
    np.testing.assert_allclose(a12, 2.5 * a1 - 0.7 * a2, atol=1e-14)
    e = orc.raytrace(np.array([[1.0, 0.0], [0.0, 1.0]]), L)[0]
    np.testing.assert_allclose(e, [[0.03, -0.02], [-0.02, -0.03]], atol=1e-16)
    # about the origin, not the lens centre
    L2 = dict(L, x0=0.5, y0=0.5)
    np.testing.assert_allclose(orc.raytrace(x1, L2)[0], a1, atol=1e-15)


def test_superposition(orc):
    """Linearity of thin-lens deflections: the total is the sum of parts."""
    x = pts(100)
    sub = np.array([[0.3, 0.4, 0.02, 0.2, 10.0], [-1.0, 0.5, 0.01, 0.5, 5.0]])
    full = orc.raytrace(x, lens(q=0.7, phi=0.3, g1=0.02, g2=0.01), sub)[0]
    main = orc.raytrace(x, lens(q=0.7, phi=0.3))[0]
    shear = orc.raytrace(x, lens(theta_e=0.0, g1=0.02, g2=0.01))[0]
    s0 = orc.raytrace(x, lens(theta_e=0.0), sub[:1])[0]
    s1 = orc.raytrace(x, lens(theta_e=0.0), sub[1:])[0]
    np.testing.assert_allclose(full, main + shear + s0 + s1, atol=1e-14)


# ---------------------------------------------------------------- subhalos
def _tnfw_rho(r, ks, ts, tau):
    """3-D truncated NFW density in units of Sigma_cr per arcsec (theta_s = r_s)."""
    t = r / ts
    return (ks / ts) / (t * (1 + t) ** 2) * tau ** 2 / (tau ** 2 + t ** 2)


def _tnfw_alpha_quad(R, ks, ts, tau):
    """alpha(R) = M_cyl(R) / (pi R): projected mass inside radius R by quadrature
    of the 3-D density over the cylinder (sphere part + outer shells)."""
    f = lambda r: 4 * math.pi * r * r * _tnfw_rho(r, ks, ts, tau)
    inner = integrate.quad(f, 0, R, limit=400, epsabs=0, epsrel=1e-12)[0]
    g = lambda r: f(r) * (1 - math.sqrt(1 - (R / r) ** 2))
    brk = [R * 1.0001, R * 1.01, 2 * R, 10 * R, 100 * R]
    outer = 0.0
    lo = R
    for hi in brk:
        outer += integrate.quad(g, lo, hi, limit=400, epsabs=0, epsrel=1e-12)[0]
        lo = hi
    outer += integrate.quad(g, lo, np.inf, limit=400, epsabs=0, epsrel=1e-12)[0]
    return (inner + outer) / (math.pi * R)


@pytest.mark.parametrize("tau", [2.0, 10.0])
@pytest.mark.parametrize("x", [0.02, 0.4, 0.9995, 1.0, 1.0004, 2.5, 40.0])
def test_tnfw_against_quadrature(orc, tau, x):
    ks, ts = 0.02, 0.3
    R = x * ts
    sub = np.array([[0.1, -0.2, ks, ts, tau]])
    p = np.array([[0.1 + R * 0.6, -0.2 + R * 0.8]])
    a = orc.raytrace(p, lens(theta_e=0.0), sub)[0][0]
    ref = _tnfw_alpha_quad(R, ks, ts, tau)
    np.testing.assert_allclose(np.hypot(*a), ref, rtol=2e-8)
    np.testing.assert_allclose(a / np.hypot(*a), [0.6, 0.8], atol=1e-12)  # radial, outward


def test_tnfw_nfw_limit(orc):
    """tau -> infinity: untruncated NFW, alpha = 4 kappa_s theta_s h(x)/x with
    h(x) = ln(x/2) + arccosh(1/x)/sqrt(1-x^2) (x<1), ln(x/2) + arccos(1/x)/sqrt(x^2-1) (x>1)."""
    ks, ts, tau = 0.02, 0.3, 1e5
    for x in [0.1, 0.7, 1.6, 5.0]:
        h = math.log(x / 2) + (math.acosh(1 / x) / math.sqrt(1 - x * x) if x < 1 else math.acos(1 / x) / math.sqrt(x * x - 1))
        a = orc.raytrace(np.array([[x * ts, 0.0]]), lens(theta_e=0.0), np.array([[0, 0, ks, ts, tau]]))[0][0]
        np.testing.assert_allclose(a[0], 4 * ks * ts * h / x, rtol=2e-8)


def test_tnfw_far_field_total_mass(orc):
    """Far outside the truncation radius the deflection is that of a point of the total mass."""
    ks, ts, tau = 0.02, 0.3, 3.0
    mtot = integrate.quad(lambda r: 4 * math.pi * r * r * _tnfw_rho(r, ks, ts, tau), 0, np.inf, limit=400)[0]
    R = 3e4 * ts
    a = orc.raytrace(np.array([[R, 0.0]]), lens(theta_e=0.0), np.array([[0, 0, ks, ts, tau]]))[0][0]
    np.testing.assert_allclose(a[0] * R, mtot / math.pi, rtol=1e-6)


def test_tnfw_divergence_is_twice_convergence(orc):
    ks, ts, tau = 0.02, 0.3, 10.0
    sub = np.array([[0.0, 0.0, ks, ts, tau]])
    for x in [0.2, 0.8, 1.3, 4.0]:
        p = np.array([[x * ts * 0.8, x * ts * 0.6]])
        div, curl = _div_curl(orc, p, lens(theta_e=0.0), sub, h=1e-6)
        R = x * ts
        sig = 2 * integrate.quad(lambda z: _tnfw_rho(math.hypot(R, z), ks, ts, tau), 0, np.inf, limit=400,
                                 epsrel=1e-12)[0]
        np.testing.assert_allclose(div[0], 2 * sig, rtol=1e-5)
        assert abs(curl[0]) < 1e-6 * sig


def test_point_mass(orc):
    x = pts(50) + 0.01
    sub = np.array([[0.2, -0.1, 0.05, 0.0, 0.0]])
    a = orc.raytrace(x, lens(theta_e=0.0), sub, profile=1)[0]
    d = x - np.array([0.2, -0.1])
    np.testing.assert_allclose(a, 0.05 ** 2 * d / (d ** 2).sum(1)[:, None], rtol=1e-13)


# ---------------------------------------------------------------- ray-trace gradients
@pytest.mark.parametrize("profile", [0, 1])
def test_raytrace_vjp_against_central_differences(orc, profile):
    rng = np.random.default_rng(7)
    x = rng.uniform(-2, 2, (60, 2))
    L = lens(x0=0.05, y0=-0.03, q=0.7, phi=0.4, theta_e=1.25, gamma=2.1, g1=0.02, g2=-0.01)
    sub = np.array([[0.4, 0.3, 0.02, 0.25, 10.0], [-0.5, 0.9, 0.015, 0.4, 4.0]])
    gb = rng.standard_normal((60, 2))
    d_lens, d_sub = orc.raytrace_vjp(x, L, sub, gb, profile)
    keys = ["x0", "y0", "q", "phi", "theta_e", "g1", "g2"]
    h = 1e-6
    for k, key in enumerate(keys):
        Lp, Lm = dict(L), dict(L)
        Lp[key] += h
        Lm[key] -= h
        fd = (np.sum(gb * orc.raytrace(x, Lp, sub, profile)[1]) - np.sum(gb * orc.raytrace(x, Lm, sub, profile)[1])) / (2 * h)
        np.testing.assert_allclose(d_lens[k], fd, rtol=1e-6, atol=1e-7, err_msg=key)
    for hh in range(2):
        for k in range(4 if profile == 0 else 3):
            sp, sm = sub.copy(), sub.copy()
            sp[hh, k] += h
            sm[hh, k] -= h
            fd = (np.sum(gb * orc.raytrace(x, L, sp, profile)[1]) - np.sum(gb * orc.raytrace(x, L, sm, profile)[1])) / (2 * h)
            np.testing.assert_allclose(d_sub[hh, k], fd, rtol=1e-6, atol=1e-7)


# ---------------------------------------------------------------- kernel reduction
def test_matvec_brute_force_long_double(orc):
    rng = np.random.default_rng(3)
    x, y = rng.uniform(-0.2, 0.2, (37, 2)), rng.uniform(-0.2, 0.2, (53, 2))
    v = rng.standard_normal(53)
    out, ab = orc.kernel_matvec(x, y, v, 0.07, 1.7)
    X, Y = x.astype(np.longdouble), y.astype(np.longdouble)
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    K = np.longdouble(1.7) * np.exp(-d2 / (2 * np.longdouble(0.07) ** 2))
    np.testing.assert_allclose(out, (K @ v.astype(np.longdouble)).astype(np.float64), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(ab, (np.abs(K * v[None, :]).sum(1)).astype(np.float64), rtol=1e-13)


def test_matvec_symmetric_psd(orc):
    rng = np.random.default_rng(4)
    x = rng.uniform(-0.3, 0.3, (120, 2))
    K = np.stack([orc.kernel_matvec(x, x, np.eye(120)[j], 0.1, 1.0)[0] for j in range(120)], axis=1)
    np.testing.assert_allclose(K, K.T, atol=1e-15)
    np.linalg.cholesky(K + 1e-12 * np.trace(K) * np.eye(120))
    np.testing.assert_allclose(np.diag(K), 1.0, atol=0)


def test_matvec_limits(orc):
    rng = np.random.default_rng(5)
    x, y, v = rng.uniform(-1, 1, (10, 2)), rng.uniform(-1, 1, (20, 2)), rng.standard_normal(20)
    out, _ = orc.kernel_matvec(x, y, v, 1e6, 2.0)
    np.testing.assert_allclose(out, 2.0 * v.sum(), rtol=1e-10)
    # two points at distance d: var * exp(-d^2 / (2 l^2))
    out, _ = orc.kernel_matvec(np.array([[0.0, 0.0]]), np.array([[0.03, 0.04]]), np.array([1.0]), 0.05, 3.0)
    np.testing.assert_allclose(out[0], 3.0 * math.exp(-0.0025 / 0.005), rtol=1e-15)


def test_matvec_riemann_sum_pins_length_scale_convention(orc):
    """sum_j k(x, y_j) h^2 -> 2 pi l^2 var on a fine grid (Sigma = l^2 I, factor 1/2 in the exponent)."""
    h = 0.004
    g = np.arange(-60, 61) * h
    Y = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2)
    out, _ = orc.kernel_matvec(np.array([[0.001, -0.0013]]), Y, np.full(len(Y), h * h), 0.03, 1.5)
    np.testing.assert_allclose(out[0], 2 * math.pi * 0.03 ** 2 * 1.5, rtol=1e-9)


def test_matvec_rows_matches_full(orc):
    rng = np.random.default_rng(6)
    x, y, v = rng.uniform(-1, 1, (80, 2)), rng.uniform(-1, 1, (90, 2)), rng.standard_normal(90)
    out, ab = orc.kernel_matvec(x, y, v, 0.2)
    rows = np.array([0, 17, 79, 3])
    o2, a2 = orc.kernel_matvec_rows(x, rows, y, v, 0.2)
    np.testing.assert_array_equal(o2, out[rows])
    np.testing.assert_array_equal(a2, ab[rows])


# ---------------------------------------------------------------- reduction gradients
@pytest.mark.parametrize("self_kernel", [False, True])
def test_matvec_vjp_against_central_differences(orc, self_kernel):
    rng = np.random.default_rng(8)
    n, m = 25, 31
    x = rng.uniform(-0.15, 0.15, (n, 2))
    y = x.copy() if self_kernel else rng.uniform(-0.15, 0.15, (m, 2))
    m = len(y)
    v = rng.standard_normal(m)
    g = rng.standard_normal(n)
    ell, var = 0.08, 1.3
    G = orc.kernel_matvec_vjp(x, y, v, ell, var, g, self_kernel)

    def loss(x_, y_, v_, l_, s_):
        return float(np.dot(g, orc.kernel_matvec(x_, y_, v_, l_, s_)[0]))

    h = 1e-6
    fd = (loss(x, y, v, ell + h, var) - loss(x, y, v, ell - h, var)) / (2 * h)
    np.testing.assert_allclose(G["d_len"], fd, rtol=1e-7)
    fd = (loss(x, y, v, ell, var + h) - loss(x, y, v, ell, var - h)) / (2 * h)
    np.testing.assert_allclose(G["d_var"], fd, rtol=1e-7)
    for j in [0, 5, m - 1]:
        vp, vm = v.copy(), v.copy()
        vp[j] += h
        vm[j] -= h
        np.testing.assert_allclose(G["d_v"][j], (loss(x, y, vp, ell, var) - loss(x, y, vm, ell, var)) / (2 * h),
                                   rtol=1e-7, atol=1e-9)
    for i in [0, 7, n - 1]:
        for c in range(2):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            yp, ym = (xp, xm) if self_kernel else (y, y)
            fd = (loss(xp, yp, v, ell, var) - loss(xm, ym, v, ell, var)) / (2 * h)
            np.testing.assert_allclose(G["d_x"][i, c], fd, rtol=1e-6, atol=1e-8)
    if not self_kernel:
        for j in [1, m - 2]:
            for c in range(2):
                yp, ym = y.copy(), y.copy()
                yp[j, c] += h
                ym[j, c] -= h
                fd = (loss(x, yp, v, ell, var) - loss(x, ym, v, ell, var)) / (2 * h)
                np.testing.assert_allclose(G["d_y"][j, c], fd, rtol=1e-6, atol=1e-8)


def test_self_vjp_rows_against_central_differences(orc):
    """The rows-only self-kernel gradients (used for sampled parity at full
    size) against FP64 central differences of the forward oracle: moving point
    p moves both its row and its column of the kernel."""
    rng = np.random.default_rng(18)
    n = 40
    x = rng.uniform(-0.12, 0.12, (n, 2))
    v, g = rng.standard_normal(n), rng.standard_normal(n)
    ell, var = 0.06, 0.9

    def loss(x_, v_):
        return float(np.dot(g, orc.kernel_matvec(x_, x_, v_, ell, var)[0]))

    rows = np.array([0, 3, 17, n - 1])
    R = orc.self_vjp_rows(x, v, g, ell, var, rows)
    h = 1e-6
    for r, i in enumerate(rows):
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        np.testing.assert_allclose(R["d_v"][r], (loss(x, vp) - loss(x, vm)) / (2 * h), rtol=1e-7, atol=1e-9)
        for c in range(2):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            np.testing.assert_allclose(R["d_x"][r, c], (loss(xp, v) - loss(xm, v)) / (2 * h), rtol=1e-6, atol=1e-8)
        assert np.all(R["d_x_abs"][r] >= np.abs(R["d_x"][r]))


@pytest.mark.parametrize("self_kernel", [False, True])
def test_matvec_vjp_sensitivities_bound_point_errors(orc, self_kernel):
    """The input-error sensitivities bound how far each gradient moves when
    every point moves by up to delta per coordinate (first order: with
    delta = 1e-5 l the second-order rest is far below the 1 % slack)."""
    rng = np.random.default_rng(28 + self_kernel)
    n, m = 30, 34
    x = rng.uniform(-0.2, 0.2, (n, 2))
    y = x.copy() if self_kernel else rng.uniform(-0.2, 0.2, (m, 2))
    v, g = rng.standard_normal(len(y)), rng.standard_normal(n)
    ell, var = 0.07, 1.1
    G = orc.kernel_matvec_vjp(x, y, v, ell, var, g, self_kernel, with_abs=True)
    delta = 1e-5 * ell
    D = 2 * np.sqrt(2) * delta
    worst = {k: 0.0 for k in ("d_v", "d_x", "d_y", "d_len", "d_var")}
    for trial in range(20):
        dx = rng.uniform(-delta, delta, x.shape)
        xp = x + dx
        yp = xp.copy() if self_kernel else y + rng.uniform(-delta, delta, y.shape)
        P = orc.kernel_matvec_vjp(xp, yp, v, ell, var, g, self_kernel)
        for k in worst:
            if G[k] is None:
                continue
            ratio = np.max(np.abs(np.asarray(P[k]) - np.asarray(G[k])) / (D * np.asarray(G[k + "_sens"]) + 1e-300))
            worst[k] = max(worst[k], float(ratio))
    assert all(r <= 1.01 for r in worst.values()), worst
    # the per-point bounds are not vacuous: some perturbation moves those
    # outputs by a sizeable fraction of them (the scalar sums' bounds add the
    # pairs' worst cases, which random perturbations mostly cancel)
    assert worst["d_x"] > 0.05 and worst["d_v"] > 0.05, worst


def test_self_vjp_rows_sensitivities_match_full(orc):
    rng = np.random.default_rng(38)
    x = rng.uniform(-0.2, 0.2, (50, 2))
    v, g = rng.standard_normal(50), rng.standard_normal(50)
    F = orc.kernel_matvec_vjp(x, x, v, 0.05, 1.0, g, True, with_abs=True)
    rows = np.arange(0, 50, 7)
    R = orc.self_vjp_rows(x, v, g, 0.05, 1.0, rows)
    out, ab = orc.kernel_matvec(x, x, v, 0.05, 1.0)
    np.testing.assert_allclose(R["out"], out[rows], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(R["out_abs"], ab[rows], rtol=1e-12)
    for k in ("d_v", "d_x"):
        np.testing.assert_allclose(R[k], F[k][rows], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(R[k + "_abs"], F[k + "_abs"][rows], rtol=1e-12)
        np.testing.assert_allclose(R[k + "_sens"], F[k + "_sens"][rows], rtol=1e-12)


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_a_planted_sign_error(orc):
    """The divergence pin rejects a deflection with a flipped rotation (a
    plausible frame slip), computed here by mirroring the oracle's output."""
    L = lens(q=0.6, phi=0.9)
    x = pts(40, 2.0)
    a = orc.raytrace(x, L)[0]
    c, s = math.cos(2 * 0.9), math.sin(2 * 0.9)
    wrong = np.stack([c * a[:, 0] + s * a[:, 1], s * a[:, 0] - c * a[:, 1]], 1)  # reflect about the major axis
    kap = np.array([orc.sple_kappa(p[0], p[1], L) for p in x])
    # finite-difference divergence of the mirrored field breaks div = 2 kappa
    h = 1e-5
    def wrongf(p):
        aa = orc.raytrace(p, L)[0]
        return np.stack([c * aa[:, 0] + s * aa[:, 1], s * aa[:, 0] - c * aa[:, 1]], 1)
    div = ((wrongf(x + [h, 0])[:, 0] - wrongf(x - [h, 0])[:, 0]) + (wrongf(x + [0, h])[:, 1] - wrongf(x - [0, h])[:, 1])) / (2 * h)
    assert np.max(np.abs(div - 2 * kap) / (2 * kap)) > 1e-2


# ---------------------------------------------------------------- the paper's printed lenses
from tests.golden.lenses import paper_lenses  # noqa: E402


@pytest.mark.parametrize("name", sorted(paper_lenses()))
def test_printed_lenses_divergence_and_shear(orc, name):
    """For each lens the paper prints, div alpha = 2 kappa + 0 (shear is traceless)
    and curl alpha = 0, over the image field away from the centre."""
    L = paper_lenses()[name]
    rng = np.random.default_rng(11)
    x = rng.uniform(-2.5, 2.5, (120, 2))
    x = x[np.hypot(x[:, 0] - L["x0"], x[:, 1] - L["y0"]) > 0.3]
    div, curl = _div_curl(orc, x, L)
    kap = np.array([orc.sple_kappa(p[0], p[1], L) for p in x])
    np.testing.assert_allclose(div, 2 * kap, rtol=2e-6)
    np.testing.assert_allclose(curl, 0.0, atol=2e-6 * np.max(kap))


# ---------------------------------------------------------------- lens Jacobian / magnification
def test_jacobian_sis_magnification_closed_form(orc):
    """SIS: det(d beta / d xi) = 1 - theta_E / R (tangential eigenvalue; radial is 1)."""
    x = pts(200, 3.0)
    x = x[np.hypot(x[:, 0], x[:, 1]) > 0.05]
    jac, mu = orc.lens_jacobian(x, lens(theta_e=1.3))
    R = np.hypot(x[:, 0], x[:, 1])
    np.testing.assert_allclose(1.0 / mu, 1 - 1.3 / R, rtol=1e-11, atol=1e-13)
    # radial direction is an eigenvector with eigenvalue 1
    n = x / R[:, None]
    np.testing.assert_allclose(np.einsum("nij,nj->ni", jac, n), n, atol=1e-12)


def test_jacobian_point_mass_closed_form(orc):
    """Point mass: mu = (1 - theta^4 / R^4)^-1."""
    x = pts(100, 1.0) + 0.02
    sub = np.array([[0.0, 0.0, 0.4, 0.0, 0.0]])
    _, mu = orc.lens_jacobian(x, lens(theta_e=0.0), sub, profile=1)
    R = np.hypot(x[:, 0], x[:, 1])
    np.testing.assert_allclose(mu, 1.0 / (1 - 0.4 ** 4 / R ** 4), rtol=1e-10)


@pytest.mark.parametrize("name", ["hoags_object", "arp142"])
def test_jacobian_trace_and_symmetry_and_shear(orc, name):
    """Paper's lens-Jacobian form: A = (1 - kappa) I - [[g1, g2], [g2, -g1]]_local, i.e.
    tr A = 2 - 2 kappa and A symmetric; with subhalos also against finite differences of beta."""
    L = paper_lenses()[name]
    x = pts(120, 2.5)
    x = x[np.hypot(x[:, 0] - L["x0"], x[:, 1] - L["y0"]) > 0.2]
    sub = np.array([[0.4, 0.3, 0.02, 0.25, 10.0], [-0.5, 0.9, 0.015, 0.4, 4.0]])
    jac, mu = orc.lens_jacobian(x, L)
    kap = np.array([orc.sple_kappa(p[0], p[1], L) for p in x])
    np.testing.assert_allclose(jac[:, 0, 0] + jac[:, 1, 1], 2 - 2 * kap, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(jac[:, 0, 1], jac[:, 1, 0], atol=1e-12)
    jac2, _ = orc.lens_jacobian(x, L, sub)
    h = 1e-6
    bx = (orc.raytrace(x + [h, 0], L, sub)[1] - orc.raytrace(x - [h, 0], L, sub)[1]) / (2 * h)
    by = (orc.raytrace(x + [0, h], L, sub)[1] - orc.raytrace(x - [0, h], L, sub)[1]) / (2 * h)
    np.testing.assert_allclose(jac2[:, :, 0], bx, atol=1e-7)
    np.testing.assert_allclose(jac2[:, :, 1], by, atol=1e-7)


# ---------------------------------------------------------------- pixel windows (next: windowed kernel)
def test_pixel_window_normalisation_appendix_c(orc):
    """App. C: the window with Z = (a a^T + b b^T)/4pi has integral of w^2 equal to
    1/|det(a, b)| (the inverse projected pixel area); checked by 2-D quadrature."""
    rng = np.random.default_rng(21)
    a, b = rng.normal(0, 0.05, 2), rng.normal(0, 0.05, 2)
    grid = np.array([[i * a + j * b for i in range(3)] for j in range(3)]).reshape(-1, 2)
    z = orc.pixel_shapes(grid, 3, 3)[4]  # centre pixel: both neighbours present
    Z = np.array([[z[0], z[1]], [z[1], z[2]]])
    Zi = np.linalg.inv(Z)
    L = 8 * np.sqrt(np.max(np.linalg.eigvalsh(Z)))
    h = L / 400
    xs = np.arange(-L, L, h)
    X, Y = np.meshgrid(xs, xs)
    r = np.stack([X, Y], -1)
    w = np.exp(-0.5 * np.einsum("...i,ij,...j", r, Zi, r)) / (2 * np.pi * np.sqrt(np.linalg.det(Z)))
    np.testing.assert_allclose((w ** 2).sum() * h * h, 1 / abs(a[0] * b[1] - a[1] * b[0]), rtol=1e-6)
    np.testing.assert_allclose(w.sum() * h * h, 1.0, rtol=1e-6)


def test_pixel_shapes_border_uses_the_single_neighbour(orc):
    grid = np.array([[c * 0.1, r * 0.2] for r in range(2) for c in range(3)])
    z = orc.pixel_shapes(grid, 3, 2)
    k = 1 / (4 * np.pi)
    for i in range(6):
        np.testing.assert_allclose(z[i], [k * 0.01, 0.0, k * 0.04], atol=1e-15)


def test_windowed_point_limit_is_the_rbf_kernel(orc):
    """Z_i -> 0: G(d, l^2/2 I) = exp(-d^2/l^2)/(pi l^2), the RBF with length l/sqrt2."""
    rng = np.random.default_rng(22)
    p, q, v = rng.uniform(-0.3, 0.3, (20, 2)), rng.uniform(-0.3, 0.3, (30, 2)), rng.standard_normal(30)
    out, _ = orc.windowed_matvec(p, np.zeros((20, 3)), q, v, 0.1)
    ref, _ = orc.kernel_matvec(p, q, v, 0.1 / np.sqrt(2), 1 / (np.pi * 0.01))
    np.testing.assert_allclose(out, ref, rtol=1e-12)


def test_transmission_factorises_the_windowed_covariance(orc):
    """Sec. 3.4: with A_k = |2 pi Sigma|^(1/4) / sqrt(n_q) on a dense grid,
    sum_k T_ik T_jk -> |2 pi Sigma|^(1/2) G(p_i - p_j, Z_i + Sigma + Z_j) = K_ij / var (eq. covariance)."""
    rng = np.random.default_rng(23)
    ell = 0.1
    p = rng.uniform(-0.1, 0.1, (5, 2))
    z = np.abs(rng.normal(0, 1e-3, (5, 3)))
    z[:, 1] = 0.3 * np.sqrt(z[:, 0] * z[:, 2])
    h = 0.008
    g = np.arange(-0.7, 0.7 + h / 2, h)
    Q = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2)
    _, _, T = orc.windowed_matvec(p, z, Q, None, ell, dense=True)
    S = ell * ell
    A2 = 2 * np.pi * S * h * h  # A_k^2 = |2 pi Sigma|^(1/2) / n_q with |2 pi Sigma|^(1/2) = 2 pi l^2
    lhs = A2 * T @ T.T
    ref = np.empty((5, 5))
    for i in range(5):
        for j in range(5):
            C = np.array([[z[i, 0] + z[j, 0] + S, z[i, 1] + z[j, 1]], [z[i, 1] + z[j, 1], z[i, 2] + z[j, 2] + S]])
            d = p[i] - p[j]
            ref[i, j] = 2 * np.pi * S * np.exp(-0.5 * d @ np.linalg.solve(C, d)) / (2 * np.pi * np.sqrt(np.linalg.det(C)))
    np.testing.assert_allclose(lhs, ref, rtol=1e-6)


# ---------------------------------------------------------------- inducing-point density
def _lattice(side, h):
    g = (np.arange(side) - (side - 1) / 2) * h
    return np.stack(np.meshgrid(g, g), -1).reshape(-1, 2)


@pytest.mark.parametrize("k,shell", [(1, 1), (4, 1), (5, 2), (8, 2), (12, 4), (13, 5), (20, 5), (24, 8), (28, 9)])
def test_knn_radius_on_the_square_lattice(orc, k, shell):
    """Neighbour shells of the square lattice (spacing h, interior points):
    4 at h^2, 4 at 2h^2, 4 at 4h^2, 8 at 5h^2, 4 at 8h^2, 4 at 9h^2, so the
    k-th closest other point sits at shell * h^2 (k = 20 -> r^2 = 5 h^2)."""
    side, h = 15, 0.1
    q = _lattice(side, h)
    inner = [r * side + c for r in range(4, side - 4) for c in range(4, side - 4)]
    r2 = orc.knn_r2(q, k, inner)
    np.testing.assert_allclose(r2, shell * h * h, rtol=1e-12)


def test_knn_radius_matches_a_full_sort(orc):
    """Brute force by a library sort of every row of the distance matrix
    (self excluded), on random points with coincident pairs."""
    rng = np.random.default_rng(31)
    q = rng.uniform(-1, 1, (300, 2))
    q[50:60] = q[40:50]  # ten coincident pairs
    d2 = ((q[:, None, :] - q[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    srt = np.sort(d2, axis=1)
    for k in (1, 2, 7, 20, 33):
        np.testing.assert_array_equal(orc.knn_r2(q, k), srt[:, k - 1])
    assert np.all(orc.knn_r2(q, 1)[40:60] == 0.0)


def test_knn_density_of_a_uniform_lattice_corner_and_interior(orc):
    """rho = k / (pi r_k^2): 20 / (5 pi h^2) in the lattice interior. The
    corner point sees one quadrant, squared distances (a^2 + b^2) h^2 over
    a, b >= 0 not both zero, whose 20th smallest is 20 h^2."""
    side, h = 15, 0.1
    q = _lattice(side, h)
    rho = orc.knn_density(q, 20, [side * 7 + 7, 0])
    c = np.sort([(a * a + b * b) for a in range(side) for b in range(side) if a or b])[19]
    np.testing.assert_allclose(rho, [20 / (np.pi * 5 * h * h), 20 / (np.pi * c * h * h)], rtol=1e-12)


def test_transmission_weights_reproduce_the_rbf_kernel(orc):
    """Sec. 3.4: with A_k = |2 pi Sigma|^(1/4) / sqrt(rho) and the exact
    density 1/h^2 of a fine lattice, sum_k A_k^2 G(p_i - q_k, Sigma/2)
    G(p_j - q_k, Sigma/2) equals exp(-|p_i - p_j|^2 / (2 l^2)), the unit
    variance Gaussian RBF (Sec. 3.1)."""
    rng = np.random.default_rng(37)
    ell, h = 0.1, 0.02
    p = rng.uniform(-0.15, 0.15, (6, 2))
    Q = _lattice(101, h)
    A = orc.transmission_weights(Q, ell, density=np.full(len(Q), 1 / (h * h)))
    _, _, T = orc.windowed_matvec(p, np.zeros((6, 3)), Q, None, ell, dense=True)
    lhs = (T * A) @ (T * A).T
    d2 = ((p[:, None, :] - p[None, :, :]) ** 2).sum(-1)
    np.testing.assert_allclose(lhs, np.exp(-d2 / (2 * ell * ell)), rtol=1e-9)


# ---------------------------------------------------------------- windowed reduction gradients
def _cd(f, x, h):
    x = np.array(x, np.float64)
    out = np.zeros_like(x)
    for i in np.ndindex(x.shape):
        a, b = x.copy(), x.copy()
        a[i] += h
        b[i] -= h
        out[i] = (f(a) - f(b)) / (2 * h)
    return out


def test_windowed_vjp_by_central_differences(orc):
    """Every gradient of sum_i g_i out_i through the windowed transmission,
    against FP64 central differences of the forward oracle."""
    rng = np.random.default_rng(41)
    n, m, ell = 5, 7, 0.07
    p = rng.uniform(-0.1, 0.1, (n, 2))
    q = rng.uniform(-0.1, 0.1, (m, 2))
    z = np.stack([rng.uniform(1e-4, 4e-4, n), rng.uniform(-5e-5, 5e-5, n), rng.uniform(1e-4, 4e-4, n)], -1)
    v, g = rng.normal(size=m), rng.normal(size=n)
    L = lambda p_, z_, q_, v_, l_: g @ orc.windowed_matvec(p_, z_, q_, v_, l_)[0]
    R = orc.windowed_vjp(p, z, q, v, ell, g)
    np.testing.assert_allclose(R["d_p"], _cd(lambda a: L(a, z, q, v, ell), p, 1e-6), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(R["d_q"], _cd(lambda a: L(p, z, a, v, ell), q, 1e-6), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(R["d_v"], _cd(lambda a: L(p, z, q, a, ell), v, 1e-4), rtol=1e-8)
    np.testing.assert_allclose(R["d_z"], _cd(lambda a: L(p, a, q, v, ell), z, 1e-8), rtol=1e-5, atol=1e-3)
    assert R["d_len"] == pytest.approx(_cd(lambda a: L(p, z, q, v, a[0]), [ell], 1e-7)[0], rel=1e-6)


def test_pixel_shapes_vjp_by_central_differences(orc):
    rng = np.random.default_rng(43)
    W, H = 5, 4
    g = (np.arange(W) - 2.0) * 0.05
    P = np.stack(np.meshgrid(g, (np.arange(H) - 1.5) * 0.05), -1).reshape(-1, 2) + rng.normal(0, 0.01, (W * H, 2))
    dz = rng.normal(size=(W * H, 3))
    f = lambda a: np.sum(dz * orc.pixel_shapes(a, W, H))
    np.testing.assert_allclose(orc.pixel_shapes_vjp(P, W, H, dz), _cd(f, P, 1e-6), rtol=1e-7, atol=1e-9)


# ---- FP32 rounding sensitivities of the windowed reduction (a tolerance term)

def test_windowed_rounding_isotropic_closed_form(orc):
    """Without windows (Z = 0, C = l^2/2 I) R is diagonal, w^ = |w| and the
    relative error bound of a Gaussian factor is rho = 3 q with q = 2 |d|^2 / l^2."""
    rng = np.random.default_rng(1)
    p = rng.uniform(-0.3, 0.3, (40, 2))
    q = rng.uniform(-0.3, 0.3, (25, 2))
    v = rng.standard_normal(25)
    ell = 0.07
    S = orc.windowed_rounding(p, np.zeros((40, 3)), q, v, ell)
    d2 = ((p[:, None, :] - q[None, :, :]) ** 2).sum(-1)
    qq = 2.0 * d2 / ell ** 2
    G = np.exp(-0.5 * qq) / (np.pi * ell ** 2)
    np.testing.assert_allclose(S["s_out"], (np.abs(G * v) * 3 * qq).sum(1), rtol=1e-12)


def test_windowed_rounding_bounds_an_fp32_evaluation(orc):
    """The bound holds for a plain FP32 evaluation of the Cholesky form with
    rounded differences and constants, on thin windows (condition numbers up
    to 1e3) and pairs out to exponents near the FP32 range."""
    rng = np.random.default_rng(2)
    n, m, ell = 60, 400, 0.002
    p = rng.uniform(-0.2, 0.2, (n, 2)).astype(np.float32)
    q = rng.uniform(-0.2, 0.2, (m, 2)).astype(np.float32)
    th = rng.uniform(0, np.pi, n)
    l1, l2 = 10 ** rng.uniform(-4, -3, n), 10 ** rng.uniform(-7, -5, n)
    c, s_ = np.cos(th), np.sin(th)
    z = np.stack([l1 * c * c + l2 * s_ * s_, (l1 - l2) * c * s_, l1 * s_ * s_ + l2 * c * c], 1).astype(np.float32)
    v = rng.standard_normal(m).astype(np.float32)
    ref, _ = orc.windowed_matvec(p, z, q, v, ell)
    S = orc.windowed_rounding(p, z, q, v, ell)
    # FP32: constants from FP64 rounded once, differences and the form in FP32
    zz = z.astype(np.float64)
    hs = 0.5 * ell * ell
    cxx, cxy, cyy = zz[:, 0] + hs, zz[:, 1], zz[:, 2] + hs
    det = cxx * cyy - cxy * cxy
    k = np.sqrt(np.log2(np.e) / 2)
    a = (k * np.sqrt(cyy / det)).astype(np.float32)
    b = (-k * cxy / np.sqrt(cyy * det)).astype(np.float32)
    cc = (k / np.sqrt(cyy)).astype(np.float32)
    N = 1.0 / (2 * np.pi * np.sqrt(det))
    dx = (q[None, :, 0] - p[:, None, 0]).astype(np.float32)
    dy = (q[None, :, 1] - p[:, None, 1]).astype(np.float32)
    w1 = (a[:, None] * dx + b[:, None] * dy).astype(np.float32)
    w2 = (cc[:, None] * dy).astype(np.float32)
    t = (w1 * w1 + w2 * w2).astype(np.float32)
    G = np.exp2(-t.astype(np.float64)) * N[:, None]
    out = (G * v[None, :].astype(np.float64)).sum(1)
    err = np.abs(out - ref)
    assert np.all(err <= 2 * 2.0 ** -24 * S["s_out"] + 1e-300)
    assert np.max(err / (2 * 2.0 ** -24 * S["s_out"] + 1e-300)) > 1e-3  # the bound is not vacuous
