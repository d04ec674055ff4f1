"""Serving engine: results against the oracle and against the single-problem
entry points, bit-identical alone vs in a mix vs one-at-a-time, admission by
device-memory budget, poll/timeout/cancel semantics and host-side fault
injection."""
import time

import numpy as np
import pytest
import torch

from paper_2105_09465_gb300 import abi, api, workloads as W
from paper_2105_09465_gb300.serving import Session
from tests.gpu_util import (GRAD_REL, MATVEC_REL, assert_close_tol, chain_tol, dev, host, need_gpu, point_delta,
                            ulp32)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def problem(seed, side, n_sub, yside=32):
    rng = np.random.default_rng(seed)
    lens = W.draw_lens(rng)
    sub = W.draw_subhalos(rng, n_sub, lens, 1e7, 1e10)
    g = W.Grid(side, side, 2, 0.05)
    yg = W.inducing_grid(g, yside)
    ell = float(np.float32(yg.pix * 4.0 / 3.0))
    p = W.Problem(f"s{seed}", g, lens, sub, 0, yg, ell, 1.0, W.draw_v(rng, yg.n), seed)
    data = rng.standard_normal(p.n).astype(np.float32)
    return p, data


def oracle_iteration(orc, p, data, step):
    """The oracle's iteration of the engine (ray-trace, out = K v, g = out -
    data, the backward of 0.5 |out - data|^2, v <- v - step d_v) with the
    per-element tolerance of each result: 2e-5 of its sum of absolute terms,
    the first-order effect of the GPU's point error delta (the oracle's
    input-error sensitivities), and, for the gradients, the effect of the
    error in g = out - data itself (the backward of the out tolerance, in
    absolute value: every kernel value is positive)."""
    xi = orc.grid_points(*p.xgrid.astuple())
    yg = orc.grid_points(*p.ygrid.astuple())
    v = p.v.astype(np.float64)
    _, b = orc.raytrace(xi, p.lens.astuple(), p.sub)
    delta = point_delta(b)
    out, ab, sens = orc.kernel_matvec(b, yg, v, p.lengthscale, p.variance, with_sens=True)
    t_out = MATVEC_REL * ab + 2.0 * delta * sens
    g = out - data
    R = orc.kernel_matvec_vjp(b, yg, v, p.lengthscale, p.variance, g, with_abs=True)
    E = orc.kernel_matvec_vjp(b, yg, v, p.lengthscale, p.variance, t_out, with_abs=True)
    tol = {k: chain_tol(R, k, delta) + E[k + "_abs"] for k in ("d_v", "d_x", "d_len", "d_var")}
    dl, ds, al, asub = orc.raytrace_vjp(xi, p.lens.astuple(), p.sub, R["d_x"], 0, with_abs=True)
    _, _, cl, csub = orc.raytrace_vjp(xi, p.lens.astuple(), p.sub, tol["d_x"], 0, with_abs=True)
    ref = {"out": out, "v": v - step * R["d_v"], "d_lens": dl, "d_sub": ds, "d_len": R["d_len"],
           "d_var": R["d_var"], "loss": 0.5 * np.sum(g ** 2)}
    tols = {"out": t_out, "v": step * tol["d_v"], "d_lens": GRAD_REL * al + cl, "d_sub": GRAD_REL * asub + csub,
            "d_len": tol["d_len"], "d_var": tol["d_var"], "loss": float(np.sum(np.abs(g) * t_out))}
    return ref, tols


def check_result(R, ref, tols, what):
    assert R.status == abi.LR_OK, what
    assert_close_tol(R.out, ref["out"], tols["out"], what=f"{what} out")
    # v comes back in FP32: one ulp of its value on top
    assert_close_tol(R.v, ref["v"], tols["v"] + ulp32(ref["v"]), what=f"{what} v")
    assert_close_tol(R.d_lens, ref["d_lens"], tols["d_lens"], what=f"{what} d_lens")
    assert_close_tol(R.d_sub, ref["d_sub"], tols["d_sub"], what=f"{what} d_sub")
    assert_close_tol([R.d_lengthscale], [ref["d_len"]], [tols["d_len"]], what=f"{what} d_len")
    assert_close_tol([R.d_variance], [ref["d_var"]], [tols["d_var"]], what=f"{what} d_var")
    assert abs(R.loss - ref["loss"]) <= tols["loss"] + 1e-12 * ref["loss"], what


def test_matches_oracle_one_iteration(orc):
    """Every result of one engine iteration against the oracle, element by
    element."""
    p, data = problem(1, 16, 6, 12)
    step = 0.5
    with Session(max_slots=4) as S:
        R = S.poll(S.submit(p, data, 1, step))
    ref, tols = oracle_iteration(orc, p, data.astype(np.float64), step)
    check_result(R, ref, tols, "one request")


def test_differentiation_batch_of_eight(orc):
    """The differentiation workload as a batch: 8 lens systems of 200x200 at
    2x2 (160k points each, 200 tNFW subhalos, 128x128 inducing grid) in one
    session, so that every stage is one batched launch for all eight; each
    system's output and gradients against the oracle element by element."""
    probs = W.diff_batch()
    assert len(probs) == 8
    rng = np.random.default_rng(22)
    datas = [rng.standard_normal(p.n).astype(np.float32) for p in probs]
    step = 0.5
    with Session(max_slots=8) as S:
        ts = [S.submit(p, d, 1, step) for p, d in zip(probs, datas)]
        res = [S.poll(t, timeout_s=300) for t in ts]
        st = S.stats()
    # the eight share batched launches (fewer iterations than requests)
    assert st["iterations"] < 8, st
    for k, (p, d, R) in enumerate(zip(probs, datas, res)):
        ref, tols = oracle_iteration(orc, p, d.astype(np.float64), step)
        check_result(R, ref, tols, f"system {k}")


def test_one_iteration_equals_single_problem_calls():
    """Batched launches inside the engine give exactly what the single-problem
    entry points give for the same iteration."""
    p, data = problem(2, 24, 9, 32)
    with Session(max_slots=4) as S:
        t = S.submit(p, data, 1, 0.0)
        R = S.poll(t)
    q = api.Points(grid=p.xgrid, lens=p.lens, sub=dev(p.sub))
    s = api.Points(grid=p.ygrid)
    out, mom = api.gp_kernel_matvec_train(q, s, dev(p.v), p.lengthscale, p.variance)
    g = out - dev(data)
    G = api.gp_kernel_matvec_bwd(q, s, dev(p.v), p.lengthscale, p.variance, g,
                                 want=["v", "lengthscale", "variance", "lens", "sub"], moments=mom)
    assert np.array_equal(R.out, host(out).astype(np.float32))
    assert np.array_equal(R.v, p.v)
    assert np.array_equal(R.d_lens, host(G["lens"]))
    # the subhalo sums of the batched and the single-problem ray-trace VJP
    # kernels are separate compilations of the same code and may round the
    # last bit of a term differently; the engine itself is bit-reproducible
    # (see the alone-versus-mix tests)
    ds, dref = R.d_sub, host(G["sub"])
    assert np.all(np.abs(ds - dref) <= 1e-6 * np.abs(dref).max())
    assert R.d_lengthscale == G["lengthscale"].item() and R.d_variance == G["variance"].item()


def run(reqs, max_slots, iters=4, step=0.02, budget=0, fill_pairs=0):
    with Session(max_slots=max_slots, hbm_budget_bytes=budget, fill_pairs=fill_pairs) as S:
        ts = [S.submit(p, d, iters, step) for p, d in reqs]
        return [S.poll(t) for t in ts]


def same(a, b):
    return (np.array_equal(a.out, b.out) and np.array_equal(a.v, b.v) and np.array_equal(a.d_lens, b.d_lens)
            and np.array_equal(a.d_sub, b.d_sub) and a.d_lengthscale == b.d_lengthscale
            and a.d_variance == b.d_variance)


def test_alone_vs_mix_vs_one_at_a_time_bit_identical():
    reqs = [problem(10 + k, side, ns, ys) for k, (side, ns, ys) in
            enumerate([(16, 0, 32), (40, 25, 64), (24, 7, 32), (64, 40, 128), (32, 3, 16), (20, 12, 48)])]
    mix = run(reqs, max_slots=8)
    fifo = run(reqs, max_slots=1)
    alone = [run([r], max_slots=1)[0] for r in reqs[:3]]
    for k in range(len(reqs)):
        assert mix[k].status == abi.LR_OK
        assert same(mix[k], fifo[k]), k
    for k in range(3):
        assert same(mix[k], alone[k]), k


def test_admission_by_pairs_per_iteration():
    """With fill_pairs the active requests' pairs per iteration stay within
    the limit (a request larger than it runs alone); results are bitwise
    those of one request at a time."""
    reqs = [problem(80 + k, side, ns, ys) for k, (side, ns, ys) in
            enumerate([(64, 10, 128), (16, 2, 32), (20, 0, 32), (48, 6, 64), (12, 3, 16), (40, 8, 64)])]
    work = [p.n * p.m for p, _ in reqs]
    fill = sorted(work)[-2] + min(work)  # the largest runs alone, smaller ones share
    with Session(max_slots=8, fill_pairs=fill) as S:
        ts = [S.submit(p, d, 6, 0.02) for p, d in reqs]
        res = [S.poll(t) for t in ts]
        peak = S.stats()["peak_active_pairs"]
    # the largest request alone, or requests within the limit, never more
    assert peak <= max(fill, max(work)) and peak >= max(work)
    fifo = run(reqs, max_slots=1, iters=6)
    for a, b in zip(res, fifo):
        assert a.status == abi.LR_OK and same(a, b)


def test_more_requests_than_one_batched_launch():
    """17+ active requests split every stage into several batched launches."""
    reqs = [problem(40 + k, 12 + (k % 5) * 4, k % 4, 16) for k in range(20)]
    mix = run(reqs, max_slots=20, iters=2)
    fifo = run(reqs, max_slots=1, iters=2)
    for a, b in zip(mix, fifo):
        assert a.status == abi.LR_OK and same(a, b)


def test_admission_respects_memory_budget():
    reqs = [problem(60 + k, 48, 10, 64) for k in range(6)]
    # footprint of one request: measure with a generous session and its stats
    with Session(max_slots=1) as S:
        t = S.submit(*reqs[0], 2, 0.01)
        peak = 0
        while True:
            peak = max(peak, S.stats()["used_bytes"])
            st = S.poll_status(t, 0.0)
            if st != abi.LR_PENDING:
                break
            time.sleep(0.001)
        S.poll(t)
    one = peak
    assert one > 0
    budget = int(2.5 * one)
    with Session(max_slots=8, hbm_budget_bytes=budget) as S:
        ts = [S.submit(p, d, 6, 0.01) for p, d in reqs]
        seen_active = 0
        for _ in range(2000):
            st = S.stats()
            assert st["used_bytes"] <= budget
            seen_active = max(seen_active, st["active"])
            if st["pending"] == 0 and st["active"] == 0:
                break
            time.sleep(0.002)
        res = [S.poll(t) for t in ts]
    assert all(r.status == abi.LR_OK for r in res)
    assert seen_active <= 2


def test_request_larger_than_budget_is_rejected():
    p, data = problem(70, 64, 5, 64)
    with Session(max_slots=2, hbm_budget_bytes=1 << 20) as S:
        with pytest.raises(abi.LensGPError) as e:
            S.submit(p, data, 2, 0.0)
        assert e.value.status == abi.LR_ERR_OUT_OF_MEMORY


def test_poll_pending_timeout_and_cancel():
    big, bd = problem(80, 200, 50, 128)
    small, sd = problem(81, 16, 2, 16)
    with Session(max_slots=1) as S:
        t1 = S.submit(big, bd, 40, 0.0)
        t2 = S.submit(small, sd, 2, 0.0)
        assert S.poll_status(t1, 0.0) == abi.LR_PENDING
        assert S.poll_status(t1, 0.001) == abi.LR_ERR_TIMEOUT
        assert S.cancel(t2) == abi.LR_OK  # still queued behind t1 (one slot)
        assert S.lib.solve_session_poll(S.h, t2, abi.lr_result(), 0) == abi.LR_ERR_NOT_FOUND
        r1 = S.poll(t1)
        assert r1.status == abi.LR_OK
        assert S.cancel(t1) == abi.LR_ERR_NOT_FOUND


def test_fault_injection_fails_the_iteration_and_the_session_recovers():
    a, ad = problem(90, 24, 4, 32)
    c, cd = problem(91, 24, 4, 32)
    with Session(max_slots=4) as S:
        S.inject_fault()
        ta = S.submit(a, ad, 3, 0.0)
        ra = S.poll(ta)
        assert ra.status == abi.LR_ERR_CUDA
        tc = S.submit(c, cd, 3, 0.0)
        rc = S.poll(tc)
        assert rc.status == abi.LR_OK
        assert S.stats()["used_bytes"] == 0
    assert api.fault_status() == 0  # no device-side fault was recorded
