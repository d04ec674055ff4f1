"""The multi-process (replica) path on CPU: two gloo ranks, each with its own
lens system seed, reduce their step times to the maximum and report the
whole-job rate the way bench.py does under torchrun."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2105_09465_gb300 import replicas, workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, ws = replicas.world()
    p = W.realistic(seed=replicas.rank_seed(r), side=16, ss=1, n_sub=3)
    my_time = 0.010 * (1 + r)  # the slower rank sets the job time
    t = replicas.max_over_ranks(my_time)
    rate = replicas.aggregate_rate(p.pairs, t, ws)
    dist.barrier()
    out[rank] = (ws, t, rate, p.lens.q)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_max_time_and_weak_scaling():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    ws0, t0, rate0, q0 = out[0]
    ws1, t1, rate1, q1 = out[1]
    assert ws0 == ws1 == 2
    assert t0 == t1 == pytest.approx(0.020)
    pairs = W.realistic(seed=1, side=16, ss=1, n_sub=3).pairs
    assert rate0 == rate1 == pytest.approx(2 * pairs / 0.020)
    assert q0 != q1  # each rank owns a different lens system


def test_single_process_identity():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.aggregate_rate(10.0, 2.0, 1) == 5.0
