"""Seeded synthetic inputs shaped like the paper's lensing workloads.

This module only draws inputs: grids, lens parameters, subhalo populations,
source weights. It holds none of the ray-trace or kernel-reduction arithmetic,
and both the CUDA path and the FP64 oracle read the arrays it returns, so the
two sides always see bit-identical inputs.

Workloads (sizes in arcseconds, seeds explicit):
  tiny        100x100 image, 0.05" pixels, no supersampling; SIE (theta_E 1.2,
              q 0.8, PA 30 deg) + shear (0.03, 0); no subhalos; self-kernel,
              length scale 0.05, variance 1; 1e8 pairs.
  realistic   400x400 image, 0.05" pixels, 2x2 supersampling (640k points);
              power-law lens (slope U(1.8,2.2), theta_E U(1,1.5), q
              U(0.6,0.95), PA U(0,pi)), shear magnitude U(0,0.05); 200
              truncated-NFW subhalos, dN/dM ~ M^-1.9 on [1e7, 1e10] Msun,
              uniform in the disc of radius 2 theta_E; 128x128 source-plane
              inducing grid; 1.05e10 pairs.
  diff        8 lens systems of 200x200 at 2x2 supersampling with the
              realistic geometry, each against a 128x128 inducing grid.
  large       800x800 at 2x2 (2.56M points); 2000 tNFW subhalos on
              [1e6, 1e10] Msun; self-kernel; 6.55e12 pairs.
  serving     Poisson request stream (mean 200/s); square images with side
              drawn from {64,128,256,384,512} px at 2x2; 0-500 subhalos each.

Subhalo masses become angular tNFW parameters (kappa_s, theta_s, tau) through
a fixed host-side recipe (NFW M200 with the Duffy et al. 2008 concentration,
flat LCDM with Planck 2015 parameters, lens at z=0.6, source at z=2.5,
truncation tau = r_t/r_s = 10). The recipe is part of the input definition,
not of the method: the kernels only ever see the angular parameters.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

ARCSEC_PER_RAD = 180.0 / math.pi * 3600.0


@dataclass(frozen=True)
class Grid:
    """(nx*ss) x (ny*ss) grid of FP32 centres, spacing pix/ss, centred on (cx, cy)."""
    nx: int
    ny: int
    ss: int
    pix: float
    cx: float = 0.0
    cy: float = 0.0

    @property
    def n(self) -> int:
        return self.nx * self.ss * self.ny * self.ss

    def astuple(self):
        return (self.nx, self.ny, self.ss, self.pix, self.cx, self.cy)


@dataclass(frozen=True)
class Lens:
    """SPLE + external shear parameters in the order the paper lists them."""
    x0: float
    y0: float
    q: float
    phi: float
    theta_e: float
    gamma: float
    g1: float
    g2: float

    def astuple(self):
        return dataclasses.astuple(self)

    def asdict(self):
        return dataclasses.asdict(self)


@dataclass
class Problem:
    """One lens system: image grid -> ray-trace -> kernel reduction against `ygrid`
    (or against its own ray-traced points when `ygrid` is None: self-kernel)."""
    name: str
    xgrid: Grid
    lens: Lens
    sub: np.ndarray              # (S, 5) float32: x, y, kappa_s, theta_s, tau
    profile: int                 # 0 = truncated NFW, 1 = point mass
    ygrid: Grid | None           # inducing grid; None = self-kernel
    lengthscale: float
    variance: float
    v: np.ndarray                # (M,) float32 source weights
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.xgrid.n

    @property
    def m(self) -> int:
        return self.n if self.ygrid is None else self.ygrid.n

    @property
    def pairs(self) -> int:
        return self.n * self.m


# --------------------------------------------------------------------------
# Host-side subhalo recipe (input definition only).
_C_KM_S = 299792.458
_G_MPC_MSUN = 4.30091727e-9        # G in Mpc (km/s)^2 / Msun
_H0 = 67.74                         # Planck 2015 (TT,TE,EE+lowP+lensing+ext)
_OM = 0.3089
_Z_L, _Z_S = 0.6, 2.5
_TAU = 10.0


def _comoving(z1: float, z2: float, n: int = 4096) -> float:
    """Comoving distance between z1 < z2 in Mpc (flat LCDM), Simpson's rule."""
    z = np.linspace(z1, z2, n + 1)
    e = np.sqrt(_OM * (1 + z) ** 3 + (1 - _OM))
    f = 1.0 / e
    w = np.ones(n + 1)
    w[1:-1:2] = 4
    w[2:-1:2] = 2
    return float((_C_KM_S / _H0) * (z2 - z1) / (3 * n) * np.dot(w, f))


def _cosmo():
    dc_l = _comoving(0.0, _Z_L)
    dc_s = _comoving(0.0, _Z_S)
    d_l = dc_l / (1 + _Z_L)
    d_s = dc_s / (1 + _Z_S)
    d_ls = (dc_s - dc_l) / (1 + _Z_S)
    c2_4piG = _C_KM_S ** 2 / (4 * math.pi * _G_MPC_MSUN)          # Msun / Mpc
    sigma_cr = c2_4piG * d_s / (d_l * d_ls)                         # Msun / Mpc^2
    hz2 = _H0 ** 2 * (_OM * (1 + _Z_L) ** 3 + (1 - _OM))
    rho_crit = 3 * hz2 / (8 * math.pi * _G_MPC_MSUN)                # Msun / Mpc^3
    return d_l, sigma_cr, rho_crit


def tnfw_params_from_mass(m200: np.ndarray, tau: float = _TAU) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """M200 [Msun] -> (kappa_s, theta_s [arcsec], tau) for the truncated NFW profile."""
    d_l, sigma_cr, rho_crit = _cosmo()
    m = np.asarray(m200, np.float64)
    h = _H0 / 100.0
    conc = 5.71 * (m * h / 2e12) ** -0.084 * (1 + _Z_L) ** -0.47
    r200 = (3 * m / (4 * math.pi * 200 * rho_crit)) ** (1 / 3)
    rs = r200 / conc
    rho_s = m / (4 * math.pi * rs ** 3 * (np.log1p(conc) - conc / (1 + conc)))
    kappa_s = rho_s * rs / sigma_cr
    theta_s = rs / d_l * ARCSEC_PER_RAD
    return kappa_s, theta_s, np.full_like(m, tau)


def draw_masses(rng: np.random.Generator, n: int, lo: float, hi: float, slope: float = -1.9) -> np.ndarray:
    """Inverse-CDF draw from dN/dM ~ M^slope on [lo, hi]."""
    a = slope + 1.0
    u = rng.random(n)
    return (lo ** a + u * (hi ** a - lo ** a)) ** (1.0 / a)


def draw_subhalos(rng: np.random.Generator, n: int, lens: Lens, mlo: float, mhi: float) -> np.ndarray:
    """(n, 5) float32 tNFW records uniform in the disc of radius 2 theta_E around the lens centre."""
    if n == 0:
        return np.zeros((0, 5), np.float32)
    r = 2.0 * lens.theta_e * np.sqrt(rng.random(n))
    t = 2.0 * math.pi * rng.random(n)
    m = draw_masses(rng, n, mlo, mhi)
    ks, ts, tau = tnfw_params_from_mass(m)
    rec = np.stack([lens.x0 + r * np.cos(t), lens.y0 + r * np.sin(t), ks, ts, tau], axis=1)
    return rec.astype(np.float32)


def draw_lens(rng: np.random.Generator) -> Lens:
    """Power-law lens and shear with the realistic-workload priors."""
    gamma = rng.uniform(1.8, 2.2)
    te = rng.uniform(1.0, 1.5)
    q = rng.uniform(0.6, 0.95)
    phi = rng.uniform(0.0, math.pi)
    gmag = rng.uniform(0.0, 0.05)
    psi = rng.uniform(0.0, math.pi)
    vals = [0.0, 0.0, q, phi, te, gamma, gmag * math.cos(2 * psi), gmag * math.sin(2 * psi)]
    return Lens(*[float(np.float32(v)) for v in vals])


def inducing_grid(xgrid: Grid, side: int = 128, pad: float = 1.2) -> Grid:
    """side x side source-plane grid covering the image field of view padded by 20%.
    A converging lens maps the field of view inside itself, so the grid covers
    every ray-traced point."""
    fov = max(xgrid.nx, xgrid.ny) * xgrid.pix
    return Grid(side, side, 1, float(np.float32(pad * fov / side)), xgrid.cx, xgrid.cy)


def draw_v(rng: np.random.Generator, m: int) -> np.ndarray:
    return rng.standard_normal(m, dtype=np.float32)


# --------------------------------------------------------------------------
def tiny(seed: int = 0) -> Problem:
    rng = np.random.default_rng(seed)
    g = Grid(100, 100, 1, 0.05)
    lens = Lens(0.0, 0.0, 0.8, float(np.float32(math.pi / 6)), 1.2, 2.0, 0.03, 0.0)
    return Problem("tiny", g, lens, np.zeros((0, 5), np.float32), 0, None, 0.05, 1.0, draw_v(rng, g.n), seed)


def realistic(seed: int = 1, side: int = 400, ss: int = 2, n_sub: int = 200, mlo: float = 1e7,
              mhi: float = 1e10, ygrid_side: int = 128) -> Problem:
    rng = np.random.default_rng(seed)
    g = Grid(side, side, ss, 0.05)
    lens = draw_lens(rng)
    sub = draw_subhalos(rng, n_sub, lens, mlo, mhi)
    yg = inducing_grid(g, ygrid_side)
    # length scale: the paper's source-plane ratio sigma / spacing = 40 mas / 30 mas
    ell = float(np.float32(yg.pix * 4.0 / 3.0))
    return Problem("realistic", g, lens, sub, 0, yg, ell, 1.0, draw_v(rng, yg.n), seed)


def diff_batch(seed: int = 2, batch: int = 8, side: int = 200) -> list[Problem]:
    out = []
    for b in range(batch):
        p = realistic(seed=1000 * seed + b, side=side, ss=2, n_sub=200)
        p.name = f"diff[{b}]"
        out.append(p)
    return out


def large(seed: int = 4, side: int = 800) -> Problem:
    rng = np.random.default_rng(seed)
    g = Grid(side, side, 2, 0.05)
    lens = draw_lens(rng)
    sub = draw_subhalos(rng, 2000, lens, 1e6, 1e10)
    return Problem("large", g, lens, sub, 0, None, 0.05, 1.0, draw_v(rng, g.n), seed)


def scaled(p_fn, **kw) -> Problem:
    """A workload with the same recipe at another size (parity tests)."""
    return p_fn(**kw)


def serving_trace(seed: int = 3, n_requests: int = 500, rate_hz: float = 200.0,
                  sides=(64, 128, 256, 384, 512), max_sub: int = 500, iters: int = 50) -> list[dict]:
    """Arrival-time-ordered request list: each with a Problem (grid inducing points) and iterations."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    reqs = []
    for k in range(n_requests):
        side = int(rng.choice(sides))
        lens = draw_lens(rng)
        sub = draw_subhalos(rng, int(rng.integers(0, max_sub + 1)), lens, 1e7, 1e10)
        g = Grid(side, side, 2, 0.05)
        yg = inducing_grid(g, 128)
        ell = float(np.float32(yg.pix * 4.0 / 3.0))
        p = Problem(f"req{k}", g, lens, sub, 0, yg, ell, 1.0, draw_v(rng, yg.n), seed)
        reqs.append({"t_arrival": float(t[k]), "problem": p, "iters": iters})
    return reqs


def random_points(rng: np.random.Generator, n: int, half_width: float) -> np.ndarray:
    """(n, 2) float32 points uniform in a square (kernel-only parity cases)."""
    return rng.uniform(-half_width, half_width, size=(n, 2)).astype(np.float32)
