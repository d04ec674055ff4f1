"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np
import pytest
import torch

ALPHA_TOL = 1e-6     # arcsec, deflection tolerance
MATVEC_REL = 2e-5    # of sum_j |k_ij v_j| per output
ABS_FLOOR = 1e-30    # FP32 exp flushes contributions below ~1e-38 to zero


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_09465_gb300 import abi
    abi.load()


def ulp32(a):
    a = np.abs(np.asarray(a, np.float64)).astype(np.float32)
    return np.spacing(a).astype(np.float64)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def assert_matvec_close(got, ref, absout, sens=None, delta=0.0, rel=MATVEC_REL, what="matvec"):
    tol = rel * absout + ABS_FLOOR
    if sens is not None:
        tol = tol + 2.0 * delta * sens
    err = np.abs(got - ref)
    bad = err > tol
    if bad.any():
        i = int(np.argmax(err / tol))
        raise AssertionError(f"{what}: {bad.sum()} of {len(got)} outside tolerance; worst row {i}: got {got[i]!r} "
                             f"ref {ref[i]!r} |err| {err[i]:.3e} tol {tol[i]:.3e} absout {absout[i]:.3e}")
    return float(np.max(err / np.maximum(absout, 1e-300)))


GRAD_REL = 2e-5      # of the sum of absolute terms per gradient


def point_delta(beta_ref):
    """Per-coordinate bound on |beta_gpu - beta_oracle|: the deflection
    tolerance plus one FP32 ulp of the largest |beta|."""
    return ALPHA_TOL + float(ulp32(beta_ref).max())


def chain_tol(R, key, delta, rel=GRAD_REL):
    """Tolerance of a reduction gradient computed on the GPU's ray-traced
    points against the oracle's gradient on its own points: rel times the sum
    of absolute terms, plus the first-order change the point error delta can
    cause, 2 sqrt(2) delta times the oracle's input-error sensitivity."""
    return rel * np.asarray(R[key + "_abs"]) + 2.0 * np.sqrt(2.0) * delta * np.asarray(R[key + "_sens"])


def assert_close_tol(got, ref, tol, what=""):
    got, ref, tol = (np.asarray(a, np.float64) for a in (got, ref, tol))
    err = np.abs(got - ref)
    bad = err > tol + 1e-30
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} outside; worst ratio "
                           f"{np.max(err / (tol + 1e-30)):.2f}, err {err.flat[np.argmax(err / (tol + 1e-30))]:.3e} "
                           f"tol {tol.flat[np.argmax(err / (tol + 1e-30))]:.3e}")


def lens_chain_tols(orc, xi, lens, sub, R, delta, profile=0):
    """Tolerances of the lens and subhalo gradients at the end of the chain:
    the ray-trace VJP's own (rel times its sum of absolute terms with the
    oracle's dL/dbeta) plus the VJP of the dL/dbeta tolerance itself, summed
    in absolute value (the raytrace_vjp abs sums with the tolerance vector as
    dL/dbeta)."""
    rl, rs, al, asub = orc.raytrace_vjp(xi, lens, sub, R["d_x"], profile, with_abs=True)
    tx = chain_tol(R, "d_x", delta)
    _, _, cl, csub = orc.raytrace_vjp(xi, lens, sub, tx, profile, with_abs=True)
    return rl, rs, GRAD_REL * al + cl, GRAD_REL * asub + csub
