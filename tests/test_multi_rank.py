"""The multi-GPU bench path on the CPU: two gloo ranks.

The hot path shards by perturbation blocks with no data-path exchange (each rank applies
chi0bar to its own block); the only collective is the max over ranks of the step times. These
tests run that host logic with world size 2 on the gloo backend.
"""

import multiprocessing as mp
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    import synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = synth.make_system("tiny")
        phi = synth.make_perturbations(s, 4, bench.rank_block_seed(rank))
        local = [10.0 + 5.0 * rank, 20.0 - 3.0 * rank]  # per-rank step times (ms)
        ms = bench.reduce_step_times(local)
        q.put((rank, phi, ms, bench.job_throughput(world, 64, ms[0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict()
    for _ in range(2):
        r, phi, ms, thr = q.get(timeout=120)
        out[r] = (phi, ms, thr)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the max over ranks of each step time
    assert out[0][1] == out[1][1] == [15.0, 20.0]
    # whole-job throughput: all ranks' units over the slowest time
    assert out[0][2] == pytest.approx(2 * 64 / 15e-3)
    # ranks own different perturbation blocks (independent work, no exchange)
    assert np.abs(out[0][0] - out[1][0]).max() > 0.1
