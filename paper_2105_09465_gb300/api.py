"""Python entry points over the C ABI, with torch tensors for device memory.

These functions only marshal arguments: pointers of CUDA tensors, the current
torch stream and plain structs go to liblensgp.so, which does all the work.
They raise when CUDA or the library is unavailable (no CPU fallback).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import abi
from .workloads import Grid, Lens


@dataclass
class Points:
    """A point set for the C ABI: explicit (n, 2) float32 CUDA positions or a
    grid, optionally ray-traced through a lens with subhalos."""
    xy: torch.Tensor | None = None
    grid: Grid | None = None
    lens: Lens | None = None
    sub: torch.Tensor | None = None   # (S, 5) float32 CUDA
    profile: int = abi.LR_PROFILE_TNFW
    lens_record: torch.Tensor | None = None  # a device lens (lens_prepare) in place of `lens`

    @property
    def n(self) -> int:
        return int(self.xy.shape[0]) if self.xy is not None else self.grid.n


def _require_cuda(t: torch.Tensor | None, name: str, shape_tail=None) -> None:
    if t is None:
        return
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if shape_tail is not None and tuple(t.shape[1:]) != shape_tail:
        raise ValueError(f"{name} must have shape (n, {', '.join(map(str, shape_tail))})")


def _stream_handle(stream: torch.cuda.Stream | None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def to_c_points(p: Points | None):
    """Builds the lr_points struct; returns (struct or None, objects to keep alive)."""
    if p is None:
        return None, ()
    _require_cuda(p.xy, "xy", (2,))
    _require_cuda(p.sub, "sub", (5,))
    c = abi.lr_points()
    keep = []
    if p.xy is not None:
        c.xy = p.xy.data_ptr()
        c.n = p.xy.shape[0]
        if p.grid is not None:  # explicit points laid out on this grid (row-block order only)
            c.grid = abi.lr_grid(*p.grid.astuple())
    else:
        c.xy = None
        c.grid = abi.lr_grid(*p.grid.astuple())
        c.n = p.grid.n
    if p.lens is not None or p.lens_record is not None:
        if p.lens is not None:
            L = abi.lr_lens(*p.lens.astuple())
            keep.append(L)
            c.lens = ctypes.pointer(L)
        else:
            c.lens_record = p.lens_record.data_ptr()
        c.sub = p.sub.data_ptr() if (p.sub is not None and p.sub.numel()) else None
        c.n_sub = int(p.sub.shape[0]) if p.sub is not None else 0
        c.profile = int(p.profile)
    return c, keep


def lens_raytrace(pts: Points, want_alpha: bool = False, stream=None):
    """beta = xi - alpha(xi) for every point (pts.lens required). Returns beta (and alpha)."""
    lib = abi.load()
    c, keep = to_c_points(pts)
    n = c.n
    dev = pts.xy.device if pts.xy is not None else torch.device("cuda", torch.cuda.current_device())
    beta = torch.empty((n, 2), dtype=torch.float32, device=dev)
    alpha = torch.empty((n, 2), dtype=torch.float32, device=dev) if want_alpha else None
    st = lib.lens_raytrace(ctypes.byref(c), beta.data_ptr(), alpha.data_ptr() if alpha is not None else None,
                           _stream_handle(stream))
    abi.check(st, "lens_raytrace")
    return (beta, alpha) if want_alpha else beta


def grid_points(grid: Grid, stream=None) -> torch.Tensor:
    """(n, 2) float32 CUDA tensor of the grid's points, as the kernels generate them."""
    lib = abi.load()
    out = torch.empty((grid.n, 2), dtype=torch.float32, device=torch.device("cuda", torch.cuda.current_device()))
    g = abi.lr_grid(*grid.astuple())
    abi.check(lib.lr_grid_points(ctypes.byref(g), out.data_ptr(), _stream_handle(stream)), "lr_grid_points")
    return out


def lens_prepare(theta7: torch.Tensor, gamma: float, record: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Device lens record from device-resident parameters theta7 (x0, y0, q,
    phi, theta_e, g1, g2; float32 CUDA, 7 values) with the slope fixed at
    gamma: pass it as Points(lens_record=...). No host synchronisation."""
    lib = abi.load()
    _require_cuda(theta7, "theta7")
    if theta7.numel() != 7:
        raise ValueError("theta7 must hold 7 values")
    nb = int(lib.lr_lens_record_bytes())
    if record is None:
        record = torch.empty((nb + 15) // 16 * 4, dtype=torch.float32, device=theta7.device)
    abi.check(lib.lr_lens_prepare(theta7.data_ptr(), float(gamma), record.data_ptr(), _stream_handle(stream)),
              "lr_lens_prepare")
    return record


def vec_axpby(a: float, x: torch.Tensor, b: float = 0.0, y: torch.Tensor | None = None,
              out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """a x + b y (or a x) elementwise, in the library."""
    lib = abi.load()
    _require_cuda(x, "x")
    _require_cuda(y, "y")
    if y is not None and y.numel() != x.numel():
        raise ValueError("x and y differ in size")
    out = torch.empty_like(x) if out is None else out
    abi.check(lib.lr_vec_axpby(x.numel(), float(a), x.data_ptr(), float(b), y.data_ptr() if y is not None else None,
                               out.data_ptr(), _stream_handle(stream)), "lr_vec_axpby")
    return out


def vec_mul(a: torch.Tensor, b: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """a * b elementwise, in the library."""
    lib = abi.load()
    _require_cuda(a, "a")
    _require_cuda(b, "b")
    if a.numel() != b.numel():
        raise ValueError("a and b differ in size")
    out = torch.empty_like(a) if out is None else out
    abi.check(lib.lr_vec_mul(a.numel(), a.data_ptr(), b.data_ptr(), out.data_ptr(), _stream_handle(stream)),
              "lr_vec_mul")
    return out


def vec_pack(head: torch.Tensor, tail: torch.Tensor, stream=None) -> torch.Tensor:
    """[float32(head), tail] with head float64, tail float32 (CUDA)."""
    lib = abi.load()
    _require_cuda(tail, "tail")
    if head.dtype != torch.float64 or not head.is_cuda or not head.is_contiguous():
        raise ValueError("head must be a contiguous float64 CUDA tensor")
    out = torch.empty(head.numel() + tail.numel(), dtype=torch.float32, device=tail.device)
    abi.check(lib.lr_vec_pack(head.data_ptr(), head.numel(), tail.data_ptr(), tail.numel(), out.data_ptr(),
                              _stream_handle(stream)), "lr_vec_pack")
    return out


def sum_scalars(parts, stream=None) -> torch.Tensor:
    """(1,) float64 CUDA tensor: the sum of the first element of each float64
    CUDA tensor in `parts`, in order, in the library."""
    lib = abi.load()
    ptrs = (ctypes.c_void_p * max(len(parts), 1))(*[t.data_ptr() for t in parts])
    dev = parts[0].device if parts else torch.device("cuda", torch.cuda.current_device())
    out = torch.empty(1, dtype=torch.float64, device=dev)
    for t in parts:
        if t.dtype != torch.float64 or not t.is_cuda:
            raise ValueError("parts must be float64 CUDA tensors")
    abi.check(lib.lr_sum_scalars(ptrs, len(parts), out.data_ptr(), _stream_handle(stream)), "lr_sum_scalars")
    return out


def lens_jacobian(pts: Points, stream=None):
    """(jac (n, 2, 2) = d beta / d xi, mu (n,) magnification) for every point (pts.lens required)."""
    lib = abi.load()
    c, keep = to_c_points(pts)
    dev = pts.xy.device if pts.xy is not None else torch.device("cuda", torch.cuda.current_device())
    jac = torch.empty((c.n, 4), dtype=torch.float32, device=dev)
    mu = torch.empty(c.n, dtype=torch.float32, device=dev)
    abi.check(lib.lens_jacobian(ctypes.byref(c), jac.data_ptr(), mu.data_ptr(), _stream_handle(stream)),
              "lens_jacobian")
    return jac.view(-1, 2, 2), mu


def _nrhs(v: torch.Tensor) -> int:
    """Right-hand sides of a weight tensor: (m,) is one, (m, r) is r."""
    return 1 if v.dim() == 1 else int(v.shape[1])


def matvec_workspace_size(query: Points, source: Points | None, nrhs: int = 1) -> int:
    lib = abi.load()
    cq, k1 = to_c_points(query)
    cs, k2 = to_c_points(source)
    b = ctypes.c_size_t(0)
    st = lib.lr_matvec_workspace_size(ctypes.byref(cq), ctypes.byref(cs) if cs is not None else None, nrhs,
                                      ctypes.byref(b))
    abi.check(st, "lr_matvec_workspace_size")
    return int(b.value)


def gp_kernel_matvec(query: Points, source: Points | None, v: torch.Tensor, lengthscale: float,
                     variance: float = 1.0, want_beta: bool = False, out: torch.Tensor | None = None,
                     workspace: torch.Tensor | None = None, stream=None, beta: torch.Tensor | None = None):
    """out_i = sum_j variance exp(-|x_i - y_j|^2 / (2 lengthscale^2)) v_j.

    `source=None` is the self-kernel. `v` is (m,) or (m, nrhs) with up to four
    right-hand sides (explicit sources); out then has shape (n,) or (n, nrhs).
    Returns out (and the ray-traced query points when want_beta and the query
    carries a lens or a grid). `beta`, if given, is an (n, 2) float32 buffer
    that receives the ray-traced points."""
    lib = abi.load()
    _require_cuda(v, "v")
    nrhs = _nrhs(v)
    cq, k1 = to_c_points(query)
    cs, k2 = to_c_points(source)
    n = cq.n
    dev = v.device
    if out is None:
        out = torch.empty((n,) if v.dim() == 1 else (n, nrhs), dtype=torch.float32, device=dev)
    if beta is None and want_beta:
        beta = torch.empty((n, 2), dtype=torch.float32, device=dev)
    _require_cuda(beta, "beta", (2,))
    b = ctypes.c_size_t(0)
    abi.check(lib.lr_matvec_workspace_size(ctypes.byref(cq), ctypes.byref(cs) if cs is not None else None, nrhs,
                                           ctypes.byref(b)), "lr_matvec_workspace_size")
    need = int(b.value)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty((max(need, 1),), dtype=torch.uint8, device=dev)
    st = lib.gp_kernel_matvec(ctypes.byref(cq), ctypes.byref(cs) if cs is not None else None, v.data_ptr(), nrhs,
                              float(lengthscale), float(variance), out.data_ptr(),
                              beta.data_ptr() if beta is not None else None, workspace.data_ptr(),
                              workspace.numel(), _stream_handle(stream))
    abi.check(st, "gp_kernel_matvec")
    return (out, beta) if want_beta else out


def gp_kernel_matvec_layers(query: Points, source: Points | None, v: torch.Tensor, lengthscales, variances,
                            want_beta: bool = False, stream=None):
    """out[i, h] = sum_l variances[l] sum_j exp(-|x_i - y_j|^2 / (2 lengthscales[l]^2)) v[l, j, h];
    v is (L, m) (one right-hand side, out (n,)) or (L, m, nrhs) (out (n, nrhs))."""
    import numpy as np

    lib = abi.load()
    L = int(v.shape[0])
    nrhs = int(v.shape[2]) if v.dim() == 3 else 1
    _require_cuda(v, "v")
    cq, k1 = to_c_points(query)
    cs, k2 = to_c_points(source)
    ls = np.ascontiguousarray(lengthscales, np.float32)
    vs = np.ascontiguousarray(variances, np.float32)
    assert ls.shape == (L,) and vs.shape == (L,)
    n = cq.n
    out = torch.empty((n, nrhs) if v.dim() == 3 else (n,), dtype=torch.float32, device=v.device)
    beta = torch.empty((n, 2), dtype=torch.float32, device=v.device) if want_beta else None
    ps = ctypes.byref(cs) if cs is not None else None
    b = ctypes.c_size_t(0)
    abi.check(lib.lr_matvec_layers_workspace_size(ctypes.byref(cq), ps, L, nrhs, ctypes.byref(b)),
              "lr_matvec_layers_workspace_size")
    ws = torch.empty(max(int(b.value), 1), dtype=torch.uint8, device=v.device)
    st = lib.gp_kernel_matvec_layers(ctypes.byref(cq), ps, L, ls.ctypes.data, vs.ctypes.data, v.data_ptr(), nrhs,
                                     out.data_ptr(), beta.data_ptr() if beta is not None else None, ws.data_ptr(),
                                     ws.numel(), _stream_handle(stream))
    abi.check(st, "gp_kernel_matvec_layers")
    return (out, beta) if want_beta else out


def pixel_shapes(p: torch.Tensor, W: int, H: int, stream=None) -> torch.Tensor:
    """(W*H, 3) window covariances (Zxx, Zxy, Zyy) of a W x H grid of projected pixel centres p."""
    lib = abi.load()
    _require_cuda(p, "p", (2,))
    z = torch.empty((p.shape[0], 3), dtype=torch.float32, device=p.device)
    abi.check(lib.gp_pixel_shapes(p.data_ptr(), W, H, z.data_ptr(), _stream_handle(stream)), "gp_pixel_shapes")
    return z


def _layout(layout: Grid | None):
    return ctypes.byref(abi.lr_grid(*layout.astuple())) if layout is not None else None


def gp_windowed_matvec(p: torch.Tensor, z: torch.Tensor, source: Points, v: torch.Tensor, lengthscale: float,
                       layout: Grid | None = None, stream=None) -> torch.Tensor:
    """out_i = sum_k G(p_i - q_k, Z_i + l^2/2 I) v_k (windowed transmission);
    layout: the image grid the query points p come from (orders the work)."""
    lib = abi.load()
    _require_cuda(p, "p", (2,))
    _require_cuda(z, "z", (3,))
    _require_cuda(v, "v")
    cs, k = to_c_points(source)
    n = p.shape[0]
    out = torch.empty(n, dtype=torch.float32, device=p.device)
    b = ctypes.c_size_t(0)
    abi.check(lib.lr_windowed_workspace_size(n, _layout(layout), ctypes.byref(cs), ctypes.byref(b)),
              "lr_windowed_workspace_size")
    ws = torch.empty(max(int(b.value), 1), dtype=torch.uint8, device=p.device)
    st = lib.gp_windowed_matvec(p.data_ptr(), z.data_ptr(), n, _layout(layout), ctypes.byref(cs), v.data_ptr(),
                                float(lengthscale), out.data_ptr(), ws.data_ptr(), ws.numel(), _stream_handle(stream))
    abi.check(st, "gp_windowed_matvec")
    return out


def gp_windowed_matvec_nll(p: torch.Tensor, z: torch.Tensor, source: Points, v: torch.Tensor, lengthscale: float,
                           data: torch.Tensor, sigma: float, f_in: torch.Tensor | None = None,
                           layout: Grid | None = None, stream=None):
    """(out, g, nll): out = f_in + the windowed reduction, g = (out - data) / sigma^2,
    nll (float64 0-d device tensor) the Gaussian likelihood's negative log, formed
    in the reduction's epilogue."""
    lib = abi.load()
    _require_cuda(p, "p", (2,))
    _require_cuda(z, "z", (3,))
    _require_cuda(v, "v")
    _require_cuda(data, "data")
    _require_cuda(f_in, "f_in")
    cs, k = to_c_points(source)
    n = p.shape[0]
    out = torch.empty(n, dtype=torch.float32, device=p.device)
    g = torch.empty(n, dtype=torch.float32, device=p.device)
    nll = torch.empty((), dtype=torch.float64, device=p.device)
    b = ctypes.c_size_t(0)
    abi.check(lib.lr_windowed_workspace_size(n, _layout(layout), ctypes.byref(cs), ctypes.byref(b)),
              "lr_windowed_workspace_size")
    ws = torch.empty(max(int(b.value), 1), dtype=torch.uint8, device=p.device)
    st = lib.gp_windowed_matvec_nll(p.data_ptr(), z.data_ptr(), n, _layout(layout), ctypes.byref(cs), v.data_ptr(),
                                    float(lengthscale), f_in.data_ptr() if f_in is not None else None,
                                    data.data_ptr(), float(sigma), out.data_ptr(), g.data_ptr(), nll.data_ptr(),
                                    ws.data_ptr(), ws.numel(), _stream_handle(stream))
    abi.check(st, "gp_windowed_matvec_nll")
    return out, g, nll


def knn_density(q: torch.Tensor, k: int = 20, lengthscale: float | None = None, want_r2: bool = True,
                workspace: torch.Tensor | None = None, stream=None):
    """k-th-neighbour squared radius r2 (and, with a lengthscale, the
    transmission weights A = pi l sqrt(2 r2 / k)) of every point of q.
    Returns r2, A or (r2, A)."""
    lib = abi.load()
    _require_cuda(q, "q", (2,))
    m = q.shape[0]
    b = ctypes.c_size_t(0)
    abi.check(lib.lr_knn_workspace_size(m, ctypes.byref(b)), "lr_knn_workspace_size")
    if workspace is None or workspace.numel() < b.value:
        workspace = torch.empty(max(int(b.value), 1), dtype=torch.uint8, device=q.device)
    r2 = torch.empty(m, dtype=torch.float32, device=q.device) if want_r2 else None
    a = torch.empty(m, dtype=torch.float32, device=q.device) if lengthscale is not None else None
    st = lib.gp_knn_density(q.data_ptr(), m, int(k), float(lengthscale or 0.0),
                            r2.data_ptr() if r2 is not None else None, a.data_ptr() if a is not None else None,
                            workspace.data_ptr(), workspace.numel(), _stream_handle(stream))
    abi.check(st, "gp_knn_density")
    if r2 is not None and a is not None:
        return r2, a
    return r2 if r2 is not None else a


# ---------------------------------------------------------------- likelihood and ELBO terms
def _elbo_ws(device) -> torch.Tensor:
    return torch.empty(int(abi.load().lr_elbo_workspace_size()), dtype=torch.uint8, device=device)


def _f32(t: torch.Tensor | None, name: str, n: int | None = None):
    if t is None:
        return None
    _require_cuda(t, name)
    if n is not None and t.numel() != n:
        raise ValueError(f"{name}: {t.numel()} elements, {n} expected")
    return t.data_ptr()


def gaussian_nll(f: torch.Tensor, data: torch.Tensor, sigma: torch.Tensor | float, grid=None, want_g: bool = True,
                 want_model: bool = False, stream=None):
    """(nll: float64 0-d device tensor, g, model) of the Gaussian pixel
    likelihood of supersampled fluxes f (grid: the supersampled Grid, or None
    for one value per pixel)."""
    lib = abi.load()
    n = f.numel()
    P = data.numel()
    dev_ = f.device
    nll = torch.empty((), dtype=torch.float64, device=dev_)
    g = torch.empty(n, dtype=torch.float32, device=dev_) if want_g else None
    model = torch.empty(P, dtype=torch.float32, device=dev_) if want_model else None
    sig_t = sigma if isinstance(sigma, torch.Tensor) else None
    cg = ctypes.byref(abi.lr_grid(*grid.astuple())) if grid is not None else None
    ws = _elbo_ws(dev_)
    st = lib.gp_gaussian_nll(_f32(f, "f"), n, cg, _f32(data, "data"), _f32(sig_t, "sigma", P),
                             float(0.0 if sig_t is not None else sigma), g.data_ptr() if g is not None else None,
                             model.data_ptr() if model is not None else None, nll.data_ptr(), ws.data_ptr(),
                             ws.numel(), _stream_handle(stream))
    abi.check(st, "gp_gaussian_nll")
    return nll, g, model


def diag_normal_draw(mu, sd, eps, alpha: float, stream=None):
    """(y, terms[2] float64 = [-ln p(y | alpha), ln q(y)])."""
    lib = abi.load()
    m = mu.numel()
    y = torch.empty(m, dtype=torch.float32, device=mu.device)
    terms = torch.empty(2, dtype=torch.float64, device=mu.device)
    ws = _elbo_ws(mu.device)
    st = lib.gp_diag_normal_draw(_f32(mu, "mu"), _f32(sd, "sd", m), _f32(eps, "eps", m), m, float(alpha),
                                 y.data_ptr(), terms.data_ptr(), ws.data_ptr(), ws.numel(), _stream_handle(stream))
    abi.check(st, "gp_diag_normal_draw")
    return y, terms


def diag_normal_vjp(mu, sd, eps, alpha: float, d_y, w_prior: float = 1.0, w_q: float = 1.0, stream=None):
    """(d_mu, d_sd, d_alpha float64 0-d)."""
    lib = abi.load()
    m = mu.numel()
    d_mu = torch.empty(m, dtype=torch.float32, device=mu.device)
    d_sd = torch.empty(m, dtype=torch.float32, device=mu.device)
    d_a = torch.empty((), dtype=torch.float64, device=mu.device)
    ws = _elbo_ws(mu.device)
    st = lib.gp_diag_normal_vjp(_f32(mu, "mu"), _f32(sd, "sd", m), _f32(eps, "eps", m), m, float(alpha),
                                _f32(d_y, "d_y", m), float(w_prior), float(w_q), d_mu.data_ptr(), d_sd.data_ptr(),
                                d_a.data_ptr(), ws.data_ptr(), ws.numel(), _stream_handle(stream))
    abi.check(st, "gp_diag_normal_vjp")
    return d_mu, d_sd, d_a


def partial_mvn_draw(mu, L, C, sd, eps, stream=None):
    """(x[D+M], logq float64 0-d) of the partial MVN proposal."""
    lib = abi.load()
    D = L.shape[0]
    M = sd.numel()
    x = torch.empty(D + M, dtype=torch.float32, device=mu.device)
    lq = torch.empty((), dtype=torch.float64, device=mu.device)
    ws = _elbo_ws(mu.device)
    st = lib.gp_partial_mvn_draw(_f32(mu, "mu", D + M), _f32(L, "L", D * D), _f32(C, "C", M * D), _f32(sd, "sd"),
                                 _f32(eps, "eps", D + M), D, M, x.data_ptr(), lq.data_ptr(), ws.data_ptr(),
                                 ws.numel(), _stream_handle(stream))
    abi.check(st, "gp_partial_mvn_draw")
    return x, lq


def partial_mvn_vjp(L, sd, eps, d_x, w_q: float = 1.0, stream=None):
    """(d_mu[D+M], d_L[D, D], d_C[M, D], d_sd[M])."""
    lib = abi.load()
    D = L.shape[0]
    M = sd.numel()
    dv_ = L.device
    d_mu = torch.empty(D + M, dtype=torch.float32, device=dv_)
    d_L = torch.empty((D, D), dtype=torch.float32, device=dv_)
    d_C = torch.empty((M, D), dtype=torch.float32, device=dv_)
    d_sd = torch.empty(M, dtype=torch.float32, device=dv_)
    st = lib.gp_partial_mvn_vjp(_f32(L, "L", D * D), _f32(sd, "sd"), _f32(eps, "eps", D + M), D, M,
                                _f32(d_x, "d_x", D + M), float(w_q), d_mu.data_ptr(), d_L.data_ptr(),
                                d_C.data_ptr(), d_sd.data_ptr(), _stream_handle(stream))
    abi.check(st, "gp_partial_mvn_vjp")
    return d_mu, d_L, d_C, d_sd


def gp_windowed_matvec_bwd(p: torch.Tensor, z: torch.Tensor, source: Points, v: torch.Tensor, lengthscale: float,
                           g: torch.Tensor, want=("v", "p", "q", "z", "lengthscale"), layout: Grid | None = None,
                           stream=None) -> dict:
    """Gradients of sum_i g_i out_i through gp_windowed_matvec (explicit sources)."""
    lib = abi.load()
    _require_cuda(p, "p", (2,))
    _require_cuda(z, "z", (3,))
    _require_cuda(v, "v")
    _require_cuda(g, "g")
    cs, k = to_c_points(source)
    n, m = p.shape[0], cs.n
    dev_ = p.device
    shapes = {"v": (m,), "p": (n, 2), "q": (m, 2), "z": (n, 3)}
    out = {key: torch.empty(shapes[key], dtype=torch.float32, device=dev_) for key in want if key in shapes}
    if "lengthscale" in want:
        out["lengthscale"] = torch.empty(1, dtype=torch.float64, device=dev_)
    b = ctypes.c_size_t(0)
    abi.check(lib.lr_windowed_bwd_workspace_size(n, _layout(layout), ctypes.byref(cs), ctypes.byref(b)),
              "lr_windowed_bwd_workspace_size")
    ws = torch.empty(max(int(b.value), 1), dtype=torch.uint8, device=dev_)
    ptr = lambda key: out[key].data_ptr() if key in out else None
    st = lib.gp_windowed_matvec_bwd(p.data_ptr(), z.data_ptr(), n, _layout(layout), ctypes.byref(cs), v.data_ptr(),
                                    float(lengthscale), g.data_ptr(), ptr("v"), ptr("p"), ptr("q"), ptr("z"),
                                    ptr("lengthscale"), ws.data_ptr(), ws.numel(), _stream_handle(stream))
    abi.check(st, "gp_windowed_matvec_bwd")
    return out


def windowed_pairs_evaluated(p: torch.Tensor, z: torch.Tensor, source: Points, lengthscale: float, sweep: int = 0,
                             layout: Grid | None = None, stream=None) -> tuple[int, int]:
    """(pairs, slots) the windowed sweeps over explicit sources evaluate
    (sweep 0: forward; 1: backward rows; 2: backward columns)."""
    lib = abi.load()
    _require_cuda(p, "p", (2,))
    _require_cuda(z, "z", (3,))
    cs, k = to_c_points(source)
    pairs, slots = ctypes.c_int64(0), ctypes.c_int64(0)
    abi.check(lib.lr_windowed_pairs_evaluated(p.data_ptr(), z.data_ptr(), p.shape[0], _layout(layout),
                                              ctypes.byref(cs), float(lengthscale), int(sweep), ctypes.byref(pairs),
                                              ctypes.byref(slots), _stream_handle(stream)),
              "lr_windowed_pairs_evaluated")
    return int(pairs.value), int(slots.value)


def pixel_shapes_vjp(p: torch.Tensor, W: int, H: int, dz: torch.Tensor, stream=None) -> torch.Tensor:
    """dL/dp (W*H, 2) through pixel_shapes given dL/dZ (W*H, 3)."""
    lib = abi.load()
    _require_cuda(p, "p", (2,))
    _require_cuda(dz, "dz", (3,))
    dp = torch.empty_like(p)
    abi.check(lib.gp_pixel_shapes_vjp(p.data_ptr(), W, H, dz.data_ptr(), dp.data_ptr(), _stream_handle(stream)),
              "gp_pixel_shapes_vjp")
    return dp


GRADS = ("v", "x", "y", "lengthscale", "variance", "lens", "sub")


def grid_pairs_evaluated(x: torch.Tensor, query_grid: Grid | None, source_grid: Grid, lengthscale: float,
                         rows_per_cta: int = 1024, stream=None) -> int:
    """Pairs the grid-source kernels evaluate (the rest are exactly zero)."""
    lib = abi.load()
    _require_cuda(x, "x", (2,))
    qg = ctypes.byref(abi.lr_grid(*query_grid.astuple())) if query_grid is not None else None
    out = ctypes.c_int64(0)
    abi.check(lib.lr_grid_pairs_evaluated(x.data_ptr(), x.shape[0], qg, ctypes.byref(abi.lr_grid(*source_grid.astuple())),
                                          float(lengthscale), int(rows_per_cta), ctypes.byref(out),
                                          _stream_handle(stream)), "lr_grid_pairs_evaluated")
    return int(out.value)


def train_workspace_size(query: Points, source: Points) -> int:
    lib = abi.load()
    cq, k1 = to_c_points(query)
    cs, k2 = to_c_points(source)
    b = ctypes.c_size_t(0)
    ps = ctypes.byref(cs) if cs is not None else None
    abi.check(lib.lr_matvec_train_workspace_size(ctypes.byref(cq), ps, 1, ctypes.byref(b)),
              "lr_matvec_train_workspace_size")
    return int(b.value)


def gp_kernel_matvec_train(query: Points, source: Points, v: torch.Tensor, lengthscale: float, variance: float = 1.0,
                           out: torch.Tensor | None = None, beta: torch.Tensor | None = None,
                           moments: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None):
    """Forward of a training step: (out, moments). out equals gp_kernel_matvec's;
    moments (4, n) are the row sums to pass to gp_kernel_matvec_bwd(moments=...).
    `beta` optionally receives the ray-traced query points."""
    lib = abi.load()
    _require_cuda(v, "v")
    cq, k1 = to_c_points(query)
    cs, k2 = to_c_points(source)
    n = cq.n
    dev = v.device
    out = torch.empty((n,), dtype=torch.float32, device=dev) if out is None else out
    moments = torch.empty((4, n), dtype=torch.float32, device=dev) if moments is None else moments
    _require_cuda(beta, "beta", (2,))
    b = ctypes.c_size_t(0)
    ps = ctypes.byref(cs) if cs is not None else None
    abi.check(lib.lr_matvec_train_workspace_size(ctypes.byref(cq), ps, 1, ctypes.byref(b)),
              "lr_matvec_train_workspace_size")
    need = int(b.value)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty((max(need, 1),), dtype=torch.uint8, device=dev)
    st = lib.gp_kernel_matvec_train(ctypes.byref(cq), ps, v.data_ptr(), 1, float(lengthscale),
                                    float(variance), out.data_ptr(), beta.data_ptr() if beta is not None else None,
                                    moments.data_ptr(), workspace.data_ptr(), workspace.numel(),
                                    _stream_handle(stream))
    abi.check(st, "gp_kernel_matvec_train")
    return out, moments


def gp_kernel_matvec_bwd(query: Points, source: Points | None, v: torch.Tensor, lengthscale: float,
                         variance: float, g_out: torch.Tensor, want=("v", "x", "lengthscale", "variance"),
                         workspace: torch.Tensor | None = None, stream=None, beta: torch.Tensor | None = None,
                         moments: torch.Tensor | None = None, source_rows: int | None = None) -> dict:
    """Gradients of Loss = sum_i g_out_i out_i (recompute-only backward).

    `want` selects among v, x (query points after ray-tracing), y (explicit
    non-self sources), lengthscale, variance, lens (7: x0, y0, q, phi,
    theta_e, g1, g2) and sub (S x 4). `beta` (optional) passes the query's
    ray-traced points from the forward pass instead of recomputing them;
    `moments` (optional) the row sums of gp_kernel_matvec_train, which leaves
    only the column sums to sweep. `v` and `g_out` are (m,) and (n,), or
    (m, nrhs) and (n, nrhs) (explicit sources); d_v has v's shape.
    `source_rows=r0` says the query points are the points r0 .. r0 + n - 1
    of `source` (one rank's rows of a self-kernel split by rows): g_out then
    covers all m source points, x gets both roles of the query points and v
    (the gradient) the query rows only. Returns a dict of CUDA tensors (the
    scalar and parameter gradients are float64)."""
    lib = abi.load()
    _require_cuda(v, "v")
    _require_cuda(g_out, "g_out")
    nrhs = _nrhs(v)
    if _nrhs(g_out) != nrhs:
        raise ValueError("v and g_out must have the same number of right-hand sides")
    cq, k1 = to_c_points(query)
    cs, k2 = to_c_points(source)
    n, m = cq.n, (cs.n if cs is not None else cq.n)
    dev = v.device
    out = {}
    nv = n if source_rows is not None else m
    if "v" in want:
        out["v"] = torch.empty((nv,) if v.dim() == 1 else (nv, nrhs), dtype=torch.float32, device=dev)
    if "x" in want:
        out["x"] = torch.empty((n, 2), dtype=torch.float32, device=dev)
    if "y" in want:
        out["y"] = torch.empty((m, 2), dtype=torch.float32, device=dev)
    for k in ("lengthscale", "variance"):
        if k in want:
            out[k] = torch.empty(1, dtype=torch.float64, device=dev)
    if "lens" in want:
        out["lens"] = torch.empty(7, dtype=torch.float64, device=dev)
    if "sub" in want:
        ns = query.sub.shape[0] if query.sub is not None else 0
        out["sub"] = torch.empty((ns, 4), dtype=torch.float64, device=dev)
    gr = abi.lr_grads()
    gr.d_v = out["v"].data_ptr() if "v" in out else None
    gr.d_x = out["x"].data_ptr() if "x" in out else None
    gr.d_y = out["y"].data_ptr() if "y" in out else None
    gr.d_lengthscale = out["lengthscale"].data_ptr() if "lengthscale" in out else None
    gr.d_variance = out["variance"].data_ptr() if "variance" in out else None
    gr.d_lens = out["lens"].data_ptr() if "lens" in out else None
    gr.d_sub = out["sub"].data_ptr() if ("sub" in out and out["sub"].numel()) else None
    if beta is not None:
        _require_cuda(beta, "beta", (2,))
        gr.beta_in = beta.data_ptr()
    if moments is not None:
        _require_cuda(moments, "moments")
        if moments.numel() != 4 * n:
            raise ValueError("moments must hold 4 x n values")
        gr.moments_in = moments.data_ptr()
    if source_rows is not None:
        gr.source_rows = 1
        gr.row0 = int(source_rows)
    b = ctypes.c_size_t(0)
    ps = ctypes.byref(cs) if cs is not None else None
    abi.check(lib.lr_matvec_bwd_workspace_size(ctypes.byref(cq), ps, nrhs, ctypes.byref(gr), ctypes.byref(b)),
              "lr_matvec_bwd_workspace_size")
    need = int(b.value)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty((max(need, 1),), dtype=torch.uint8, device=dev)
    st = lib.gp_kernel_matvec_bwd(ctypes.byref(cq), ps, v.data_ptr(), nrhs, float(lengthscale), float(variance),
                                  g_out.data_ptr(), ctypes.byref(gr), workspace.data_ptr(), workspace.numel(),
                                  _stream_handle(stream))
    abi.check(st, "gp_kernel_matvec_bwd")
    return out


def cull_pairs_evaluated(query: Points, source: Points | None, lengthscale: float, sweep: int = 0,
                         stream=None) -> tuple[int, int]:
    """(valid pairs, pair slots) the culled sweeps over explicit or self
    sources evaluate; sweep 0 = forward, 1 = backward."""
    lib = abi.load()
    cq, k1 = to_c_points(query)
    cs, k2 = to_c_points(source)
    pr, sl = ctypes.c_int64(0), ctypes.c_int64(0)
    abi.check(lib.lr_cull_pairs_evaluated(ctypes.byref(cq), ctypes.byref(cs) if cs is not None else None,
                                          float(lengthscale), int(sweep), ctypes.byref(pr), ctypes.byref(sl),
                                          _stream_handle(stream)), "lr_cull_pairs_evaluated")
    return int(pr.value), int(sl.value)


def matvec_bwd_workspace_size(query: Points, source: Points | None, want=("v", "x", "lengthscale", "variance"),
                              beta: bool = False, moments: bool = False, nrhs: int = 1) -> int:
    """Workspace bytes gp_kernel_matvec_bwd needs for these point sets, the
    requested gradients (`want`, as in gp_kernel_matvec_bwd) and whether the
    forward's points (`beta`) and row moments (`moments`) are passed. The
    size depends only on which pointers are set: one small real device buffer
    stands for all of them."""
    lib = abi.load()
    cq, k1 = to_c_points(query)
    cs, k2 = to_c_points(source)
    stand_in = torch.empty(64, dtype=torch.float64, device="cuda").data_ptr()
    gr = abi.lr_grads()
    for key, field in (("v", "d_v"), ("x", "d_x"), ("y", "d_y"), ("lengthscale", "d_lengthscale"),
                       ("variance", "d_variance"), ("lens", "d_lens"), ("sub", "d_sub")):
        setattr(gr, field, stand_in if key in want else None)
    gr.beta_in = stand_in if beta else None
    gr.moments_in = stand_in if moments else None
    b = ctypes.c_size_t(0)
    abi.check(lib.lr_matvec_bwd_workspace_size(ctypes.byref(cq), ctypes.byref(cs) if cs is not None else None, nrhs,
                                               ctypes.byref(gr), ctypes.byref(b)), "lr_matvec_bwd_workspace_size")
    return int(b.value)


def lens_raytrace_vjp(pts: Points, d_beta: torch.Tensor, stream=None):
    """(d_lens[7], d_sub[S, 4]) float64 for Loss with dL/dbeta = d_beta."""
    lib = abi.load()
    _require_cuda(d_beta, "d_beta", (2,))
    c, keep = to_c_points(pts)
    dev = d_beta.device
    d_lens = torch.empty(7, dtype=torch.float64, device=dev)
    ns = pts.sub.shape[0] if pts.sub is not None else 0
    d_sub = torch.empty((ns, 4), dtype=torch.float64, device=dev)
    b = ctypes.c_size_t(0)
    abi.check(lib.lr_raytrace_vjp_workspace_size(ctypes.byref(c), ctypes.byref(b)), "lr_raytrace_vjp_workspace_size")
    ws = torch.empty((max(int(b.value), 1),), dtype=torch.uint8, device=dev)
    st = lib.lens_raytrace_vjp(ctypes.byref(c), d_beta.data_ptr(), d_lens.data_ptr(),
                               d_sub.data_ptr() if ns else None, ws.data_ptr(), ws.numel(), _stream_handle(stream))
    abi.check(st, "lens_raytrace_vjp")
    return d_lens, d_sub


def probe_pipe_rates(device: int = 0) -> dict:
    """Measured per-SM-clock rates: FFMA lanes, FFMA2 lanes, MUFU.EX2; and SM count."""
    lib = abi.load()
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_int32()
    abi.check(lib.lr_probe_pipe_rates(device, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(n)),
              "lr_probe_pipe_rates")
    return {"ffma_lanes_per_clk": a.value, "ffma2_lanes_per_clk": b.value, "ex2_per_clk": c.value, "sm_count": n.value}


# Kernel ids of the launch timer (LR_KT_* in the C header).
TIMED_KERNELS = {"matvec": 0, "train_rows": 1, "bwd_rows": 2, "dv_rows": 3, "raytrace": 4, "raytrace_vjp": 5,
                 "windowed": 6}


def kernel_timer_enable(enable: bool = True) -> None:
    """Start (clearing earlier records) or stop the library's launch timer on
    the current device: CUDA events around each pair-sweep launch."""
    abi.check(abi.load().lr_kernel_timer_enable(int(enable)), "lr_kernel_timer_enable")


def kernel_timer_read(kernel: str) -> tuple[int, float, int]:
    """(launches, summed device milliseconds, launches not recorded) of one
    timed kernel since the timer was last enabled; waits for its events."""
    lib = abi.load()
    n, ms, dropped = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    abi.check(lib.lr_kernel_timer_read(TIMED_KERNELS[kernel], ctypes.byref(n), ctypes.byref(ms), ctypes.byref(dropped)),
              "lr_kernel_timer_read")
    return int(n.value), float(ms.value), int(dropped.value)


def fault_status(clear: bool = False) -> int:
    lib = abi.load()
    code = ctypes.c_int32()
    abi.check(lib.lr_fault_status(ctypes.byref(code), int(clear)), "lr_fault_status")
    return int(code.value)
