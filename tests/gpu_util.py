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
