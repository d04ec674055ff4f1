"""Python handle on the serving engine (solve_session_* in the C ABI).

The engine itself (admission, continuous batching, device state, completion
tracking) runs in liblensgp's worker thread; this class only marshals
requests and results between numpy arrays and the C structs.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import abi
from .workloads import Problem


@dataclass
class Result:
    ticket: int
    status: int
    out: np.ndarray | None
    v: np.ndarray | None
    d_lens: np.ndarray | None
    d_sub: np.ndarray | None
    d_lengthscale: float
    d_variance: float
    loss: float
    t_submit: float
    t_admit: float
    t_done: float

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


class Session:
    def __init__(self, max_slots: int = 16, hbm_budget_bytes: int = 0, device: int = 0, fill_pairs: int = 0):
        self.lib = abi.load()
        cfg = abi.lr_session_cfg(hbm_budget_bytes, max_slots, device, int(fill_pairs))
        h = ctypes.c_void_p()
        abi.check(self.lib.solve_session_create(ctypes.byref(cfg), ctypes.byref(h)), "solve_session_create")
        self.h = h
        self._shapes = {}

    def submit(self, p: Problem, data: np.ndarray, iters: int, step: float) -> int:
        """Queues problem p (grid inducing points) with observed fluxes `data`."""
        assert p.ygrid is not None, "serving requests use a grid of inducing points"
        sub = np.ascontiguousarray(p.sub, np.float32)
        v0 = np.ascontiguousarray(p.v, np.float32)
        d = np.ascontiguousarray(data, np.float32)
        assert v0.shape == (p.m,) and d.shape == (p.n,)
        q = abi.lr_request()
        q.grid = abi.lr_grid(*p.xgrid.astuple())
        q.lens = abi.lr_lens(*p.lens.astuple())
        q.sub = sub.ctypes.data if len(sub) else None
        q.n_sub = len(sub)
        q.profile = p.profile
        q.ygrid = abi.lr_grid(*p.ygrid.astuple())
        q.v0 = v0.ctypes.data
        q.data = d.ctypes.data
        q.lengthscale = p.lengthscale
        q.variance = p.variance
        q.step = step
        q.iters = iters
        t = ctypes.c_uint64()
        abi.check(self.lib.solve_session_submit(self.h, ctypes.byref(q), ctypes.byref(t)), "solve_session_submit")
        self._shapes[t.value] = (p.n, p.m, len(sub))
        return int(t.value)

    def poll(self, ticket: int, timeout_s: float = 60.0, want=("out", "v", "d_lens", "d_sub")) -> Result:
        early = getattr(self, "_early", {}).pop(ticket, None)
        if early is not None:
            out, v, r = early
            self._shapes.pop(ticket, None)
            return Result(ticket, abi.LR_OK, out, v, None, None, r.d_lengthscale, r.d_variance, r.loss,
                          r.t_submit_s, r.t_admit_s, r.t_done_s)
        n, m, ns = self._shapes[ticket]
        out = np.empty(n, np.float32) if "out" in want else None
        v = np.empty(m, np.float32) if "v" in want else None
        dl = np.empty(7, np.float64) if "d_lens" in want else None
        ds = np.empty((ns, 4), np.float64) if "d_sub" in want else None
        r = abi.lr_result()
        r.out = out.ctypes.data if out is not None else None
        r.v = v.ctypes.data if v is not None else None
        r.d_lens = dl.ctypes.data if dl is not None else None
        r.d_sub = ds.ctypes.data if (ds is not None and ns) else None
        st = self.lib.solve_session_poll(self.h, ticket, ctypes.byref(r), int(timeout_s * 1e6))
        if st in (abi.LR_PENDING, abi.LR_ERR_TIMEOUT):
            abi.check(st, "solve_session_poll")
        if st != abi.LR_OK:
            self._shapes.pop(ticket, None)
            return Result(ticket, st, None, None, None, None, 0.0, 0.0, 0.0, r.t_submit_s, r.t_admit_s, r.t_done_s)
        self._shapes.pop(ticket, None)
        return Result(ticket, st, out, v, dl, ds, r.d_lengthscale, r.d_variance, r.loss, r.t_submit_s, r.t_admit_s,
                      r.t_done_s)

    def poll_status(self, ticket: int, timeout_s: float = 0.0) -> int:
        """Status of an unfinished ticket without consuming a finished result:
        LR_PENDING / LR_ERR_TIMEOUT while it runs. Use poll() to collect it."""
        r = abi.lr_result()
        n, m, ns = self._shapes[ticket]
        out = np.empty(n, np.float32)
        v = np.empty(m, np.float32)
        r.out, r.v = out.ctypes.data, v.ctypes.data
        st = self.lib.solve_session_poll(self.h, ticket, ctypes.byref(r), int(timeout_s * 1e6))
        if st == abi.LR_OK:  # it had finished: keep what was collected for a later poll()
            self._early = getattr(self, "_early", {})
            self._early[ticket] = (out, v, r)
        return st

    def cancel(self, ticket: int) -> int:
        st = self.lib.solve_session_cancel(self.h, ticket)
        if st == abi.LR_OK:
            self._shapes.pop(ticket, None)
        return st

    def inject_fault(self) -> None:
        abi.check(self.lib.solve_session_inject_fault(self.h), "solve_session_inject_fault")

    def stats(self) -> dict:
        s = abi.lr_session_stats()
        abi.check(self.lib.solve_session_stats(self.h, ctypes.byref(s)), "solve_session_stats")
        return {k: getattr(s, k) for k, _ in abi.lr_session_stats._fields_}

    def close(self) -> None:
        if self.h:
            self.lib.solve_session_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
