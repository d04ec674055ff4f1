"""torch.autograd.Function over the fused ray-trace + kernel reduction.

Forward: out = K(beta(xi; lens, subhalos), y; l, var) v with the image-plane
grid `xgrid` ray-traced through the lens, against the inducing grid `ygrid`
(or the ray-traced points themselves when ygrid is None). Backward: the
hand-written recompute-only CUDA backward, returning gradients for v, the lens
parameters (x0, y0, q, phi, theta_e, gamma, g1, g2; the slope's gradient is
reported as zero because the library holds it fixed), the subhalo records
(x_h, y_h, kappa_s, theta_s, tau; tau's gradient is zero), the length scale
and the variance. Both directions run in liblensgp; this module only wires
them into autograd.
"""
from __future__ import annotations

import torch

from . import api
from .workloads import Grid, Lens


class RaytraceKernelMatvec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, lens_params, sub, lengthscale, variance, xgrid: Grid, ygrid: Grid | None, profile: int):
        lens = Lens(*[float(t) for t in lens_params.detach().cpu().tolist()])
        ell = float(lengthscale)
        var = float(variance)
        q = api.Points(grid=xgrid, lens=lens, sub=sub.detach().contiguous() if sub is not None else None,
                       profile=profile)
        s = api.Points(grid=ygrid) if ygrid is not None else None
        if s is not None:
            # training forward: also keeps the row moments, so the backward
            # sweeps the pairs only for d_v
            beta = torch.empty((q.n, 2), dtype=torch.float32, device=v.device)
            out, mom = api.gp_kernel_matvec_train(q, s, v.detach().contiguous(), ell, var, beta=beta)
        else:
            out, beta = api.gp_kernel_matvec(q, s, v.detach().contiguous(), ell, var, want_beta=True)
            mom = torch.empty(0, device=v.device)
        ctx.save_for_backward(v, sub if sub is not None else torch.empty(0), beta, mom)
        ctx.meta = (q, s, ell, var, lens_params.dtype, lens_params.device)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        v, sub, beta, mom = ctx.saved_tensors
        q, s, ell, var, ldtype, ldev = ctx.meta
        need = ctx.needs_input_grad
        want = []
        if need[0]:
            want.append("v")
        if need[1]:
            want.append("lens")
        if need[2] and sub.numel():
            want.append("sub")
        if need[3]:
            want.append("lengthscale")
        if need[4]:
            want.append("variance")
        if not want:
            return (None,) * 8
        G = api.gp_kernel_matvec_bwd(q, s, v.detach().contiguous(), ell, var, grad_out.contiguous().float(),
                                     want=want, beta=beta, moments=mom if mom.numel() else None)
        gv = G.get("v")
        gl = None
        if "lens" in G:
            g7 = G["lens"].to(ldev, ldtype)
            z = torch.zeros(1, dtype=ldtype, device=ldev)
            gl = torch.cat([g7[:5], z, g7[5:]])  # slope held fixed
        gs = None
        if "sub" in G:
            gs = torch.zeros_like(sub)
            gs[:, :4] = G["sub"].to(sub.dtype)
        gell = G["lengthscale"].reshape(()) if "lengthscale" in G else None
        gvar = G["variance"].reshape(()) if "variance" in G else None
        return gv, gl, gs, gell, gvar, None, None, None


def lensed_gp_matvec(v, lens_params, sub, lengthscale, variance, xgrid: Grid, ygrid: Grid | None = None,
                     profile: int = 0):
    """Differentiable fused ray-trace + kernel reduction (see module docstring)."""
    return RaytraceKernelMatvec.apply(v, lens_params, sub, lengthscale, variance, xgrid, ygrid, profile)
