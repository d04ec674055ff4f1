"""CPU checks of the C ABI: the library builds, loads, exports every symbol
that include/lensgp.h declares, and rejects bad arguments before touching the
GPU. No compute call runs here."""
import ctypes
import re
from pathlib import Path

import pytest

from paper_2105_09465_gb300 import abi

ROOT = Path(__file__).resolve().parent.parent


def declared_symbols():
    syms = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text):
            name = m.group(1)
            before = text[: m.start()].rstrip()
            if name in ("sizeof", "defined") or before.endswith("typedef"):
                continue
            # function declarations: a return type precedes the name
            if re.search(r"(lr_status|const char\s*\*|void|int32_t|size_t)\s*$", before):
                syms.add(name)
    return syms


@pytest.fixture(scope="module")
def lib():
    return abi.load()


_KEEP = []


def dbuf(offset=0):
    """Address for an argument that validation must reject before any launch.

    With a GPU present it points into a real 1 KiB device allocation (plus
    `offset` bytes, e.g. 4 for a misaligned pointer), so that no call can
    ever reach a made-up address. Without one no call reaches a device and a
    placeholder stands in."""
    try:
        import torch
        if torch.cuda.is_available():
            t = torch.empty(1024, dtype=torch.uint8, device="cuda")
            _KEEP.append(t)
            return ctypes.c_void_p(t.data_ptr() + offset)
    except ImportError:
        pass
    return ctypes.c_void_p(256 + offset)


def test_library_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert {"lens_raytrace", "gp_kernel_matvec", "lr_last_error"} <= syms
    for s in syms:
        assert hasattr(lib, s), f"liblensgp.so does not export {s}"
    assert set(abi.SIGNATURES) >= syms, f"binding lacks {syms - set(abi.SIGNATURES)}"


def test_status_names(lib):
    assert lib.lr_status_name(0) == b"LR_OK"
    assert lib.lr_status_name(1) == b"LR_ERR_INVALID_ARG"
    assert lib.lr_status_name(99) == b"LR_UNKNOWN_STATUS"


def test_raytrace_rejects_bad_arguments_without_gpu(lib):
    assert lib.lens_raytrace(None, None, None, None) == abi.LR_ERR_INVALID_ARG
    assert b"NULL" in lib.lr_last_error()
    p = abi.lr_points()
    p.xy = None
    p.grid = abi.lr_grid(10, 10, 1, 0.05, 0.0, 0.0)
    p.n = 99  # grid has 100 points
    L = abi.lr_lens(0, 0, 0.8, 0.5, 1.2, 2.0, 0, 0)
    p.lens = ctypes.pointer(L)
    assert lib.lens_raytrace(ctypes.byref(p), dbuf(), None, None) == abi.LR_ERR_INVALID_ARG
    assert b"grid has 100 points" in lib.lr_last_error()
    p.n = 100
    for bad in [dict(q=0.0), dict(q=1.5), dict(gamma=3.0), dict(gamma=1.0), dict(theta_e=-1.0),
                dict(x0=float("nan")), dict(q=0.05)]:
        L2 = abi.lr_lens(0, 0, 0.8, 0.5, 1.2, 2.0, 0, 0)
        for k, val in bad.items():
            setattr(L2, k, val)
        p.lens = ctypes.pointer(L2)
        assert lib.lens_raytrace(ctypes.byref(p), dbuf(), None, None) == abi.LR_ERR_INVALID_ARG, bad
    p.lens = ctypes.pointer(L)
    p.n_sub = 3
    p.sub = None
    assert lib.lens_raytrace(ctypes.byref(p), dbuf(), None, None) == abi.LR_ERR_INVALID_ARG
    p.n_sub = 0
    p.profile = 7
    assert lib.lens_raytrace(ctypes.byref(p), dbuf(), None, None) == abi.LR_ERR_INVALID_ARG


def test_matvec_rejects_bad_arguments_without_gpu(lib):
    q = abi.lr_points()
    q.xy = dbuf(4)  # misaligned
    q.n = 10
    assert lib.gp_kernel_matvec(ctypes.byref(q), None, None, 1, 0.1, 1.0, None, None, None, 0, None) == \
        abi.LR_ERR_INVALID_ARG
    q.xy = dbuf()
    for nrhs in (0, 5):
        assert lib.gp_kernel_matvec(ctypes.byref(q), None, None, nrhs, 0.1, 1.0, None, None, None, 0, None) == \
            abi.LR_ERR_INVALID_ARG  # nrhs outside 1..4
        assert b"nrhs" in lib.lr_last_error()
    q.n = -1
    assert lib.gp_kernel_matvec(ctypes.byref(q), None, None, 1, 0.1, 1.0, None, None, None, 0, None) == \
        abi.LR_ERR_INVALID_ARG


def test_kernel_timer_without_gpu(lib):
    n, ms, dropped = ctypes.c_int64(-1), ctypes.c_double(-1.0), ctypes.c_int64(-1)
    assert lib.lr_kernel_timer_enable(0) == 0
    assert lib.lr_kernel_timer_read(99, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(dropped)) == 1
    assert lib.lr_kernel_timer_read(-1, ctypes.byref(n), ctypes.byref(ms), None) == 1
    assert lib.lr_kernel_timer_read(0, None, ctypes.byref(ms), None) == 1
    # nothing recorded: no event is touched
    assert lib.lr_kernel_timer_read(0, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(dropped)) == 0
    assert (n.value, ms.value, dropped.value) == (0, 0.0, 0)
