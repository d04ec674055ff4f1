"""FP64 CPU oracle for the lens ray-trace and Gaussian-kernel reduction.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` load it. The product path (the CUDA library
and its Python binding) never imports it and shares no code with it.

The arithmetic lives in ``lensgp_oracle.c`` (plain C, FP64, OpenMP over
independent rows); this module compiles it with gcc and wraps it with ctypes
and numpy. Every function cites the passage of Karchev, Coogan & Weniger
(arXiv:2105.09465) it follows.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  grid_points       — pinned: exact definition, checked element-wise
  raytrace (SPLE)   — pinned: SIS limit, q=1 power law, SIE artanh closed form,
                      scipy 2F1, divergence = 2 kappa, zero curl
  raytrace (shear)  — pinned: linearity and superposition
  raytrace (tNFW)   — pinned: quadrature of the 3-D profile, NFW limit,
                      far-field total mass, divergence = 2 kappa
  raytrace (point)  — pinned: closed form
  raytrace_vjp      — pinned: FP64 central differences of raytrace
  kernel_matvec     — pinned: dense long-double brute force, symmetry, PSD,
                      l -> infinity, two-point value, Riemann-sum integral
  kernel_matvec_vjp — pinned: FP64 central differences of kernel_matvec; its
                      input-error sensitivities by perturbing the points
  self_vjp_rows     — pinned: FP64 central differences of kernel_matvec (both
                      roles of the listed points)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "lensgp_oracle.c"
LIB = HERE / "liblensgp_oracle.so"

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (FP64, -O2, OpenMP; no FP contraction)."""
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        tmp = LIB.with_suffix(".so.tmp")
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               "-std=c11", str(SRC), "-o", str(tmp), "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"oracle build failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


class OrcGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("ss", ctypes.c_int32),
                ("pix", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class OrcLens(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("x0", "y0", "q", "phi", "theta_e", "gamma", "g1", "g2")]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(str(build()))
        L.orc_grid_points.argtypes = [ctypes.POINTER(OrcGrid), _P]
        L.orc_sple_kappa.argtypes = [_D, _D, ctypes.POINTER(OrcLens)]
        L.orc_sple_kappa.restype = _D
        L.orc_raytrace.argtypes = [_P, _I64, ctypes.POINTER(OrcLens), _P, _I32, _I32, _P, _P]
        L.orc_raytrace_vjp.argtypes = [_P, _I64, ctypes.POINTER(OrcLens), _P, _I32, _I32, _P, _P, _P, _P, _P]
        L.orc_lens_jacobian.argtypes = [_P, _I64, ctypes.POINTER(OrcLens), _P, _I32, _I32, _P, _P]
        L.orc_pixel_shapes.argtypes = [_P, _I32, _I32, _P]
        L.orc_windowed_matvec.argtypes = [_P, _P, _I64, _P, _I64, _P, _D, _P, _P, _P]
        L.orc_knn_r2.argtypes = [_P, _I64, _I32, _P, _I64, _P]
        L.orc_windowed_vjp.argtypes = [_P, _P, _I64, _P, _I64, _P, _D, _P] + [_P] * 10
        L.orc_windowed_rounding.argtypes = [_P, _P, _I64, _P, _I64, _P, _D, _P] + [_P] * 6
        L.orc_pixel_shapes_vjp.argtypes = [_P, _I32, _I32, _P, _P, _P]
        L.orc_kernel_matvec.argtypes = [_P, _I64, _P, _I64, _P, _D, _D, _P, _I64, _P, _P, _P]
        L.orc_kernel_matvec_vjp.argtypes = [_P, _I64, _P, _I64, _P, _D, _D, _P, _I32, _P, _P, _P, _P, _P, _P]
        L.orc_self_vjp_rows.argtypes = [_P, _I64, _P, _P, _D, _D, _P, _I64] + [_P] * 8
        L.orc_num_threads.restype = _I32
        L.orc_set_num_threads.argtypes = [_I32]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _pairs(a) -> np.ndarray:
    """(n, 2) FP64 points; FP32 inputs widen exactly."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.ndim == 2 and a.shape[1] == 2, a.shape
    return a


def _lens(lens) -> OrcLens:
    """lens: mapping or sequence in the order (x0, y0, q, phi, theta_e, gamma, g1, g2)."""
    keys = ("x0", "y0", "q", "phi", "theta_e", "gamma", "g1", "g2")
    vals = [lens[k] for k in keys] if isinstance(lens, dict) else list(lens)
    return OrcLens(*[float(v) for v in vals])


def _subs(sub):
    if sub is None or len(sub) == 0:
        return np.zeros((0, 5), np.float64), 0
    s = np.ascontiguousarray(sub, dtype=np.float64)
    assert s.ndim == 2 and s.shape[1] == 5
    return s, s.shape[0]


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on."""
    lib().orc_set_num_threads(int(n))


def grid_points(nx, ny, ss, pix, cx=0.0, cy=0.0) -> np.ndarray:
    """FP32 pixel centres of the (nx ss) x (ny ss) supersampled grid, row-major over y."""
    g = OrcGrid(nx, ny, ss, pix, cx, cy)
    out = np.empty((nx * ss * ny * ss, 2), np.float32)
    lib().orc_grid_points(ctypes.byref(g), _ptr(out))
    return out


def sple_kappa(x, y, lens) -> float:
    """SPLE convergence (Sec. 2.2)."""
    L = _lens(lens)
    return float(lib().orc_sple_kappa(float(x), float(y), ctypes.byref(L)))


def raytrace(xi, lens, sub=None, profile=0):
    """Ray-trace beta = xi - alpha(xi): returns (alpha, beta), FP64 (n, 2) arrays."""
    xi = _pairs(xi)
    s, ns = _subs(sub)
    L = _lens(lens)
    alpha = np.empty(xi.shape, np.float64)
    beta = np.empty(xi.shape, np.float64)
    lib().orc_raytrace(_ptr(xi), xi.shape[0], ctypes.byref(L), _ptr(s), ns, profile, _ptr(alpha), _ptr(beta))
    return alpha, beta


def raytrace_vjp(xi, lens, sub, d_beta, profile=0, with_abs=False):
    """Gradient of sum(d_beta * beta) w.r.t. (x0, y0, q, phi, theta_e, g1, g2) and per subhalo
    (x_h, y_h, kappa_s | theta_pm, theta_s). With `with_abs`, also the sums of absolute
    per-point terms (tolerance scales)."""
    xi = _pairs(xi)
    s, ns = _subs(sub)
    L = _lens(lens)
    db = np.ascontiguousarray(d_beta, dtype=np.float64)
    d_lens = np.empty(7, np.float64)
    d_sub = np.empty((ns, 4), np.float64)
    a_lens = np.empty(7, np.float64)
    a_sub = np.empty((ns, 4), np.float64)
    lib().orc_raytrace_vjp(_ptr(xi), xi.shape[0], ctypes.byref(L), _ptr(s), ns, profile, _ptr(db), _ptr(d_lens),
                           _ptr(d_sub) if ns else None, _ptr(a_lens), _ptr(a_sub) if ns else None)
    return (d_lens, d_sub, a_lens, a_sub) if with_abs else (d_lens, d_sub)


def lens_jacobian(xi, lens, sub=None, profile=0):
    """(jac (n, 2, 2) = d beta / d xi, mu (n,) = 1/det) from the paper's lens-Jacobian definition."""
    xi = _pairs(xi)
    s, ns = _subs(sub)
    L = _lens(lens)
    jac = np.empty((xi.shape[0], 4), np.float64)
    mu = np.empty(xi.shape[0], np.float64)
    lib().orc_lens_jacobian(_ptr(xi), xi.shape[0], ctypes.byref(L), _ptr(s), ns, profile, _ptr(jac), _ptr(mu))
    return jac.reshape(-1, 2, 2), mu


def pixel_shapes(p, W, H):
    """(W*H, 3) window covariances (Zxx, Zxy, Zyy) of a W x H grid of projected pixel centres."""
    p = _pairs(p)
    assert p.shape[0] == W * H
    z = np.empty((W * H, 3), np.float64)
    lib().orc_pixel_shapes(_ptr(p), W, H, _ptr(z))
    return z


def windowed_matvec(p, z, q, v, lengthscale, dense=False):
    """(out, absout[, T]) of out_i = sum_k G(p_i - q_k, Z_i + l^2/2 I) v_k."""
    p, q = _pairs(p), _pairs(q)
    z = np.ascontiguousarray(z, np.float64)
    v = None if v is None else np.ascontiguousarray(v, np.float64).reshape(-1)
    n, m = p.shape[0], q.shape[0]
    out = np.empty(n, np.float64)
    ab = np.empty(n, np.float64)
    T = np.empty((n, m), np.float64) if dense else None
    lib().orc_windowed_matvec(_ptr(p), _ptr(z), n, _ptr(q), m, _ptr(v), lengthscale, _ptr(out), _ptr(ab), _ptr(T))
    return (out, ab, T) if dense else (out, ab)


def windowed_vjp(p, z, q, v, lengthscale, g, with_abs=False):
    """Gradients of Loss = sum_i g_i out_i through windowed_matvec: dict with
    d_v (m), d_p (n, 2), d_q (m, 2), d_z (n, 3: Zxx, Zxy, Zyy; the off-diagonal
    entry counted in both positions), d_len; with_abs adds *_abs scales."""
    p, q = _pairs(p), _pairs(q)
    z = np.ascontiguousarray(z, np.float64)
    v = np.ascontiguousarray(v, np.float64).reshape(-1)
    g = np.ascontiguousarray(g, np.float64).reshape(-1)
    n, m = p.shape[0], q.shape[0]
    R = {"d_v": np.empty(m), "d_p": np.empty((n, 2)), "d_q": np.empty((m, 2)), "d_z": np.empty((n, 3)),
         "d_len": np.empty(1)}
    A = {k + "_abs": np.empty_like(a) for k, a in R.items()} if with_abs else {}
    ab = [A.get(k + "_abs") for k in ("d_v", "d_p", "d_q", "d_z", "d_len")]
    lib().orc_windowed_vjp(_ptr(p), _ptr(z), n, _ptr(q), m, _ptr(v), lengthscale, _ptr(g), _ptr(R["d_v"]),
                           _ptr(R["d_p"]), _ptr(R["d_q"]), _ptr(R["d_z"]), _ptr(R["d_len"]), *map(_ptr, ab))
    R["d_len"] = float(R["d_len"][0])
    if with_abs:
        A["d_len_abs"] = float(A["d_len_abs"][0])
        R.update(A)
    return R


def windowed_rounding(p, z, q, v, lengthscale, g=None):
    """FP32 rounding sensitivities (in units of u = 2^-24) of windowed_matvec
    and windowed_vjp: dict s_out (n), s_v (m), s_p (n, 2), s_q (m, 2),
    s_z (n, 3), s_len; the gradient entries need g. Test infrastructure: a
    tolerance term, not the method."""
    p, q = _pairs(p), _pairs(q)
    z = np.ascontiguousarray(z, np.float64)
    v = np.ascontiguousarray(v, np.float64).reshape(-1)
    g = None if g is None else np.ascontiguousarray(g, np.float64).reshape(-1)
    n, m = p.shape[0], q.shape[0]
    S = {"s_out": np.empty(n), "s_v": np.empty(m), "s_p": np.empty((n, 2)), "s_q": np.empty((m, 2)),
         "s_z": np.empty((n, 3)), "s_len": np.empty(1)}
    lib().orc_windowed_rounding(_ptr(p), _ptr(z), n, _ptr(q), m, _ptr(v), lengthscale, _ptr(g),
                                *[_ptr(S[k]) for k in ("s_out", "s_v", "s_p", "s_q", "s_z", "s_len")])
    S["s_len"] = float(S["s_len"][0])
    return S


def pixel_shapes_vjp(p, W, H, dz, with_abs=False):
    """dL/dp (W*H, 2) through pixel_shapes given dL/dZ (W*H, 3); with
    `with_abs`, also the sums of absolute terms (a tolerance scale)."""
    p = _pairs(p)
    dz = np.ascontiguousarray(dz, np.float64)
    dp = np.empty((W * H, 2), np.float64)
    ab = np.empty((W * H, 2), np.float64) if with_abs else None
    lib().orc_pixel_shapes_vjp(_ptr(p), W, H, _ptr(dz), _ptr(dp), _ptr(ab))
    return (dp, ab) if with_abs else dp


def knn_r2(q, k, rows=None):
    """Squared distance from each point (or each listed row) of q to its k-th
    closest other point of q, FP64 (k <= 64)."""
    q = _pairs(q)
    assert 1 <= k <= 64
    r = None if rows is None else np.ascontiguousarray(rows, np.int64)
    n = q.shape[0] if r is None else len(r)
    out = np.empty(n, np.float64)
    lib().orc_knn_r2(_ptr(q), q.shape[0], k, _ptr(r), n, _ptr(out))
    return out


def knn_density(q, k=20, rows=None):
    """Inducing-point density rho = k / (pi r_k^2) (Sec. 3.4 footnote)."""
    return k / (np.pi * knn_r2(q, k, rows))


def transmission_weights(q, lengthscale, k=20, rows=None, density=None):
    """A_k = |2 pi Sigma|^(1/4) / sqrt(rho(q_k)) with Sigma = l^2 I in two
    dimensions, i.e. sqrt(2 pi l^2 / rho) (Sec. 3.4). `density` overrides
    the k-nearest-neighbour estimate."""
    rho = knn_density(q, k, rows) if density is None else np.asarray(density, np.float64)
    return np.sqrt(2.0 * np.pi * lengthscale ** 2 / rho)


def kernel_matvec(x, y, v, lengthscale, variance=1.0, rows=None, with_sens=False):
    """Gaussian-kernel reduction: (out, absout[, sens]), FP64, out_i = sum_j var exp(-|x_i-y_j|^2/(2 l^2)) v_j.
    With `rows`, only those rows of x are evaluated (sampled parity at full size)."""
    x, y = _pairs(x), _pairs(y)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    assert v.shape[0] == y.shape[0]
    if rows is not None:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        assert rows.size == 0 or (rows.min() >= 0 and rows.max() < x.shape[0])
    cnt = x.shape[0] if rows is None else rows.shape[0]
    out = np.empty(cnt, np.float64)
    ab = np.empty(cnt, np.float64)
    sens = np.empty(cnt, np.float64) if with_sens else None
    lib().orc_kernel_matvec(_ptr(x), x.shape[0], _ptr(y), y.shape[0], _ptr(v), lengthscale, variance, _ptr(rows),
                            0 if rows is None else rows.shape[0], _ptr(out), _ptr(ab), _ptr(sens))
    return (out, ab, sens) if with_sens else (out, ab)


def kernel_matvec_rows(x, rows, y, v, lengthscale, variance=1.0):
    """The reduction on the rows `rows` of x only: (out, absout) of length len(rows)."""
    return kernel_matvec(x, y, v, lengthscale, variance, rows=rows)


def kernel_matvec_vjp(x, y, v, lengthscale, variance, g, self_kernel=False, with_abs=False):
    """Reduction gradients: dict with d_v, d_x, d_y (None for a self-kernel), d_len, d_var for Loss = sum_i g_i out_i.
    With `with_abs`, also the matching sums of absolute terms under keys *_abs
    and the input-error sensitivities under *_sens: if every point moves by at
    most delta per coordinate, each output moves by at most
    2 sqrt(2) delta * sens (first order)."""
    x, y = _pairs(x), _pairs(y)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
    n, m = x.shape[0], y.shape[0]
    d_v = np.empty(m, np.float64)
    d_x = np.empty((n, 2), np.float64)
    d_y = None if self_kernel else np.empty((m, 2), np.float64)
    d_len = np.zeros(1, np.float64)
    d_var = np.zeros(1, np.float64)
    sc = [np.empty(m), np.empty((n, 2)), np.empty((m, 2)), np.zeros(1), np.zeros(1),
          np.empty(m), np.empty((n, 2)), np.empty((m, 2)), np.zeros(1), np.zeros(1)]
    arr = (ctypes.c_void_p * 10)(*[a.ctypes.data for a in sc]) if with_abs else None
    lib().orc_kernel_matvec_vjp(_ptr(x), n, _ptr(y), m, _ptr(v), lengthscale, variance, _ptr(g), int(self_kernel),
                                _ptr(d_v), _ptr(d_x), _ptr(d_y), _ptr(d_len), _ptr(d_var), arr)
    out = {"d_v": d_v, "d_x": d_x, "d_y": d_y, "d_len": float(d_len[0]), "d_var": float(d_var[0])}
    if with_abs:
        out.update({"d_v_abs": sc[0], "d_x_abs": sc[1], "d_y_abs": None if self_kernel else sc[2],
                    "d_len_abs": float(sc[3][0]), "d_var_abs": float(sc[4][0]),
                    "d_v_sens": sc[5], "d_x_sens": sc[6], "d_y_sens": None if self_kernel else sc[7],
                    "d_len_sens": float(sc[8][0]), "d_var_sens": float(sc[9][0])})
    return out


def self_vjp_rows(x, v, g, lengthscale, variance, rows):
    """Self-kernel reduction and gradients on the listed rows only: dict with
    out (r,) and its out_abs scale, d_v (r,), d_x (r, 2) (both roles of each
    listed point), their *_abs scales and *_sens input-error sensitivities
    (as kernel_matvec_vjp)."""
    x = _pairs(x)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    assert rows.size == 0 or (rows.min() >= 0 and rows.max() < x.shape[0])
    k = rows.shape[0]
    keys = ("out", "out_abs", "d_v", "d_x", "d_v_abs", "d_x_abs", "d_v_sens", "d_x_sens")
    R = {key: np.empty((k, 2) if key.startswith("d_x") else k) for key in keys}
    lib().orc_self_vjp_rows(_ptr(x), x.shape[0], _ptr(v), _ptr(g), lengthscale, variance, _ptr(rows), k,
                            *[_ptr(R[key]) for key in keys])
    return R
