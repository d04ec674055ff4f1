"""Parity of the CUDA likelihood and ELBO-term kernels with the FP64 oracle
(oracle/elbo.py) on the same FP32 inputs. The kernels form each term in FP32
(FP32 log and reciprocal, a few ulp) and sum in FP64, so a scalar agrees
within SCALAR_REL of the sum of its terms' magnitudes."""
import numpy as np
import pytest
import torch

from oracle import elbo as E
from paper_2105_09465_gb300 import abi, api, workloads as W
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


SCALAR_REL = 1e-6
ALPHA = np.float32(0.7)  # the FP32 value both sides use


def f32(a):
    return np.asarray(a, np.float32)


def close(got, ref, scale):
    assert abs(float(got) - ref) <= SCALAR_REL * scale, (float(got), ref, scale)


@pytest.mark.parametrize("nx,ny,ss,per_pixel", [(37, 23, 2, True), (400, 400, 2, False), (19, 11, 3, True),
                                                 (1000, 1, 1, False)])
def test_gaussian_nll(nx, ny, ss, per_pixel):
    rng = np.random.default_rng(nx + ss)
    n, P = nx * ny * ss * ss, nx * ny
    f, d = f32(rng.normal(size=n)), f32(rng.normal(size=P))
    s = f32(rng.uniform(0.05, 0.3, P)) if per_pixel else np.float32(0.1)
    grid = W.Grid(nx, ny, ss, 0.05) if ss > 1 or ny > 1 else None
    nll, g, model = api.gaussian_nll(dev(f), dev(d), dev(s) if per_pixel else float(s), grid=grid, want_model=True)
    ref, gref, mref = E.gaussian_nll(f, d, s, nx, ny, ss)
    m = E.pixel_average(f, nx, ny, ss)
    sb = np.broadcast_to(np.float64(s) if not per_pixel else s.astype(np.float64), m.shape)
    close(nll, ref, np.sum(0.5 * (m - d) ** 2 / sb ** 2 + np.abs(np.log(sb))) + P)
    np.testing.assert_allclose(host(model), mref, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(host(g), gref, rtol=2e-6, atol=1e-6 * np.abs(gref).max())


def test_nll_is_reproducible():
    rng = np.random.default_rng(3)
    f, d = dev(rng.normal(size=640000)), dev(rng.normal(size=160000))
    grid = W.Grid(400, 400, 2, 0.05)
    a = [float(api.gaussian_nll(f, d, 0.1, grid=grid)[0]) for _ in range(3)]
    assert a[0] == a[1] == a[2]


@pytest.mark.parametrize("m", [1, 1000, 300000])
def test_diag_normal(m):
    rng = np.random.default_rng(m)
    mu, sd, eps, dy = f32(rng.normal(size=m)), f32(rng.uniform(0.01, 1, m)), f32(rng.normal(size=m)), \
        f32(rng.normal(size=m))
    y, terms = api.diag_normal_draw(dev(mu), dev(sd), dev(eps), ALPHA)
    yr, nlp, lq = E.diag_normal_draw(mu, sd, eps, ALPHA)
    np.testing.assert_allclose(host(y), yr, rtol=1e-6, atol=1e-7)
    t = host(terms)
    a = np.float64(ALPHA)
    close(t[0], nlp, np.sum(yr ** 2) / (2 * a * a) + m * (abs(np.log(a)) + 1))
    close(t[1], lq, np.sum(0.5 * eps.astype(np.float64) ** 2 + np.abs(np.log(sd))) + m)
    d_mu, d_sd, d_a = api.diag_normal_vjp(dev(mu), dev(sd), dev(eps), ALPHA, dev(dy), 0.5, 1.5)
    rm, rs, ra = E.diag_normal_vjp(mu, sd, eps, ALPHA, dy, 0.5, 1.5)
    np.testing.assert_allclose(host(d_mu), rm, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(host(d_sd), rs, rtol=1e-6, atol=1e-6 * np.abs(rs).max())
    close(d_a, ra, 0.5 * (m / a + np.sum(yr ** 2) / a ** 3))


@pytest.mark.parametrize("D,M", [(7, 1600), (7, 16384), (3, 0), (32, 500)])
def test_partial_mvn(D, M):
    """The paper's configuration: 7 lens parameters and a 40 x 40
    source-plane grid (Table 2), and a 128 x 128 one."""
    rng = np.random.default_rng(D * 1000 + M)
    L = np.tril(rng.normal(0, 0.05, (D, D)))
    L[np.diag_indices(D)] = rng.uniform(0.005, 0.02, D)
    L, C, sd = f32(L), f32(rng.normal(0, 0.01, (M, D))), f32(rng.uniform(0.005, 0.02, M))
    mu, eps, dx = f32(rng.normal(size=D + M)), f32(rng.normal(size=D + M)), f32(rng.normal(size=D + M))
    x, lq = api.partial_mvn_draw(dev(mu), dev(L), dev(C), dev(sd), dev(eps))
    xr, lqr = E.partial_mvn_draw(mu, L, C, sd, eps)
    np.testing.assert_allclose(host(x), xr, rtol=1e-6, atol=1e-6)
    e64 = eps.astype(np.float64)
    close(lq, lqr, np.sum(0.5 * e64 ** 2) + np.sum(np.abs(np.log(np.diag(L)))) + np.sum(np.abs(np.log(sd))) + D + M)
    g = api.partial_mvn_vjp(dev(L), dev(sd), dev(eps), dev(dx), 0.8)
    for got, ref in zip(g, E.partial_mvn_vjp(L, C, sd, eps, dx, 0.8)):
        if ref.size:
            np.testing.assert_allclose(host(got).reshape(ref.shape), ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def test_validation():
    z = torch.zeros(4, device="cuda")
    with pytest.raises(abi.LensGPError, match="alpha"):
        api.diag_normal_draw(z, z + 1, z, 0.0)
    with pytest.raises(abi.LensGPError, match="sigma0"):
        api.gaussian_nll(z, z, 0.0)
