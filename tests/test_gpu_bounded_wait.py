"""The bounded waits give up instead of hanging: a kernel that waits on an
mbarrier whose transaction bytes never arrive returns after its budget,
records the time-out in the fault word, and leaves the context usable."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import abi, api
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def test_wait_runs_out_and_returns():
    lib = abi.load()
    code, fault = ctypes.c_int32(-1), ctypes.c_int32(-1)
    assert lib.lr_fault_status(ctypes.byref(fault), 1) == abi.LR_OK  # start clean
    # about 1e5 SM clocks (~50 us): the wait cannot complete, so it runs out
    abi.check(lib.lr_selftest_bounded_wait(100000, ctypes.byref(code)), "lr_selftest_bounded_wait")
    assert code.value == 1
    assert lib.lr_fault_status(ctypes.byref(fault), 1) == abi.LR_OK
    assert fault.value == 1  # kFaultBarrierTimeout
    assert lib.lr_fault_status(ctypes.byref(fault), 0) == abi.LR_OK and fault.value == 0
    # the context is still usable: a reduction runs and is correct
    x = np.array([[0.0, 0.0], [0.01, 0.0]], np.float32)
    out = host(api.gp_kernel_matvec(api.Points(xy=dev(x)), None, dev(np.ones(2)), 0.05, 1.0))
    ref = 1.0 + np.exp(-0.01 ** 2 / (2 * 0.05 ** 2))
    assert np.allclose(out, ref, rtol=1e-5)
    assert api.fault_status() == 0


def test_budget_is_validated():
    code = ctypes.c_int32(0)
    assert abi.load().lr_selftest_bounded_wait(0, ctypes.byref(code)) == abi.LR_ERR_INVALID_ARG
