"""A small seeded instance of the lensed-GP SVI model (shared by the oracle
pin and the GPU parity test): 24 x 24 pixels of 0.1 arcsec, a 16 x 16
source grid, one image-plane layer, SPLE + shear near the workloads'
priors. No arithmetic of the method lives here."""
import numpy as np


def case(seed=7):
    rng = np.random.default_rng(seed)
    nx = ny = 24
    pix = 0.1
    src = (16, 16, 1, 0.18, 0.0, 0.0)
    cfg = dict(pixels=(nx, ny, pix), source_grid=src, sigma_sp=0.24, sigma_layers=[0.06], alpha_sp=1.0,
               alpha_layers=[0.5], noise=0.2, gamma=2.0, knn_k=20)
    M = 16 * 16
    theta = np.array([0.02, -0.03, 0.8, 0.5, 0.7, 0.02, -0.01])
    L = np.diag(np.full(7, 0.01))
    L[3, 1] = 0.002
    mu = np.concatenate([theta, rng.normal(0, 1, M)])
    guide = dict(mu=mu, L=L, C=rng.normal(0, 0.01, (M, 7)), sd_sp=np.full(M, 0.05),
                 mu_layers=[rng.normal(0, 0.5, nx * ny)], sd_layers=[np.full(nx * ny, 0.02)])
    data = rng.normal(0, 1, nx * ny)
    eps_sp = rng.normal(size=7 + M)
    eps_layers = [rng.normal(size=nx * ny)]
    f32 = lambda a: np.asarray(a, np.float32)
    guide = {k: (f32(v) if not isinstance(v, list) else [f32(x) for x in v]) for k, v in guide.items()}
    return cfg, guide, f32(data), f32(eps_sp), [f32(e) for e in eps_layers]
