"""Truncation bounds of the ray-trace kernels' far-field series and local
expansion, checked on the host against the truncated-NFW closed form.

The kernels sum a tNFW subhalo's deflection factor G = B(x) / x^2 by its
series in y = 1/x, G = y^2 (q0 + sum_{j>=2} q_j y^j), cut after y^K from
x = r_K max(tau, 2) on (Baltz, Marshall & Oguri 2009 for B; the q_j from
expanding its logarithm and arccosine in 1/x). The ray-trace backward also
needs x dG/dx, the same series with coefficients -(j + 2) q_j. Far from a
small tile, the backward sums the series by its local expansion about the
tile's centre, to total order N in delta and conj(delta).

This file checks the stated bounds with independent arithmetic:
- the series truncation, in extended precision (mpmath), within 1.4e-8
  relative for tau from 0.5 to 30;
- the expansion, in FP64 against the analytic per-point gradients, within
  5e-9 of the sums of absolute terms.
"""
import math

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")


def closed_G(x, tau):
    """G = B / x^2 of the truncated NFW profile (x > 1)."""
    t2 = tau * tau
    F = mp.acos(1 / x) / mp.sqrt(x * x - 1)
    L = mp.log(x / (mp.sqrt(t2 + x * x) + tau))
    B = (t2 + 1 + 2 * (x * x - 1)) * F + tau * mp.pi + (t2 - 1) * mp.log(tau) + mp.sqrt(t2 + x * x) * (
        -mp.pi + (t2 - 1) / tau * L)
    return B / (x * x)


def series_q(tau):
    """q0 .. q9 of G = y^2 sum_j q_j y^j (q1 = 0)."""
    T = mp.mpf(tau) ** 2
    T1 = T + 1
    C = (T - 1) * mp.log(tau) + tau * mp.pi
    return [C - T1, 0, -T1 ** 2 / 3, mp.pi * T1 ** 2 / 8, 2 * (T ** 3 - T ** 2 - 5 * T - 3) / 15,
            mp.pi * (-T ** 3 + 3 * T + 2) / 16, 8 * (-T ** 4 + T ** 3 - 7 * T - 5) / 105,
            5 * mp.pi * (T ** 4 + 4 * T + 3) / 128, 16 * (T ** 5 - T ** 4 - 9 * T - 7) / 315,
            7 * mp.pi * (-T ** 5 + 5 * T + 4) / 256]


@pytest.mark.parametrize("K, r", [(9, 6), (7, 8), (5, 18), (4, 32), (3, 80)])
def test_far_field_series_radii(K, r):
    mp.mp.dps = 40
    worst = mp.mpf(0)
    for tau in (0.5, 2.0, 10.0, 30.0):
        q = series_q(tau)
        for f in (1.0, 1.5, 3.0):
            x = mp.mpf(r * max(tau, 2.0) * f)
            y = 1 / x
            g = closed_G(x, tau)
            hg = x * mp.diff(lambda s: closed_G(s, tau), x)
            gs = y * y * sum(q[j] * y ** j for j in range(K + 1))
            hs = y * y * sum(-(j + 2) * q[j] * y ** j for j in range(K + 1))
            worst = max(worst, abs(gs / g - 1), abs(hs / hg - 1) if K <= 7 else 0)
    assert worst <= 1.4e-8, float(worst)


def binom(a, k):
    out = 1.0
    for i in range(k):
        out *= (a - i) / (i + 1)
    return out


def expansion_sums(pts, g, xh, A, kappa, ts, q, K, N):
    """The four subhalo sums by the local expansion about the points' centre."""
    cen = pts.mean()
    c, d = cen - xh, pts - cen
    W = {(k, l): np.sum(np.conj(g) * d ** k * np.conj(d) ** l) for k in range(N + 1) for l in range(N + 1 - k)}
    u, ub, yc = 1 / c, np.conj(1 / c), ts / abs(c)
    L = Lt = X = Y = 0.0
    for k in range(N + 1):
        for l in range(N + 1 - k):
            ckl = sum(q[j] * yc ** j * binom(-j / 2, k) * binom(-(j + 2) / 2, l) for j in range(K + 1) if j != 1)
            ctl = sum((j + 2) * q[j] * yc ** j * binom(-j / 2, k) * binom(-(j + 2) / 2, l)
                      for j in range(K + 1) if j != 1)
            Q = u ** k * ub ** (l + 1)
            wa = W[(k - 1, l)] if k else 0
            wb = W[(k, l - 1)] if l else 0
            L += ckl * (Q * W[(k, l)]).real
            Lt += ctl * (Q * W[(k, l)]).real
            X += ckl * (Q * (k * wa + l * wb)).real
            Y += ckl * (Q * 1j * (k * wa - l * wb)).real
    s = A * ts * ts
    return np.array([s * X, s * Y, -s * L / kappa, -s * Lt / ts])


def direct_sums(pts, g, xh, A, kappa, ts, q, K):
    """The same sums point by point from the series (analytic derivatives), and their absolute terms."""
    d = pts - xh
    R, dx, dy, gx, gy = np.abs(d), d.real, d.imag, g.real, g.imag
    T = np.zeros((4, pts.size))
    for j in range(K + 1):
        if j == 1:
            continue
        a = A * q[j] * ts ** (j + 2)
        f, fp = a * R ** (-(j + 2)), -(j + 2) * a * R ** (-(j + 4))
        T[0] += gx * (f + fp * dx * dx) + gy * (fp * dx * dy)
        T[1] += gx * (fp * dx * dy) + gy * (f + fp * dy * dy)
        T[2] -= (gx * f * dx + gy * f * dy) / kappa
        T[3] -= (j + 2) / ts * (gx * f * dx + gy * f * dy)
    return T.sum(1), np.abs(T).sum(1)


@pytest.mark.parametrize("N, ratio", [(4, 0.01), (5, 0.03), (6, 0.05), (7, 0.08)])
def test_local_expansion_orders(N, ratio):
    rng = np.random.default_rng(N)
    q = [float(v) for v in series_q(10.0)]
    worst = 0.0
    for ts, K in ((0.015, 3), (0.015, 4), (0.05, 5), (0.2, 7)):
        for ang in (0.3, 2.1, 4.0):
            xs, ys = (np.arange(21) - 10) * 0.025, (np.arange(25) - 12) * 0.025
            X, Y = np.meshgrid(xs, ys)
            cen = math.hypot(0.25, 0.3) / ratio * np.exp(1j * ang)
            pts = (X + 1j * Y).ravel() + cen
            g = rng.standard_normal(pts.size) + 1j * rng.standard_normal(pts.size)
            ref, ab = direct_sums(pts, g, 0j, 0.002, 0.05, ts, q, K)
            got = expansion_sums(pts, g, 0j, 0.002, 0.05, ts, q, K, N)
            worst = max(worst, float(np.max(np.abs(got - ref) / ab)))
    assert worst <= 5e-9, worst
