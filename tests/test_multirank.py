"""The multi-rank bench path on CPU: two gloo ranks.

Batched scoring shards by candidates with no exchange on the data path;
each rank generates its own workload from its rank seed, and the job's
throughput is every rank's units over the slowest rank's time (one MAX
all-reduce of the timing).  This checks that aggregation and that the
rank-seeded workloads differ, with two processes on 127.0.0.1.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2601_11626_gb300 import synth
        value, ms = bench.job_throughput(10.0 + 5.0 * rank, 4096, world)
        w = synth.scoring_c4(r=16, seed=rank, n_states=2, appends=1, per_state=2, m=256,
                             k_lo=16, k_hi=40)
        sig = torch.tensor([float(w["candidates"][0].double().sum())], dtype=torch.float64)
        sigs = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(sigs, sig)
        out[rank] = (value, ms, [float(x) for x in sigs])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_shard():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    assert set(out.keys()) == {0, 1}
    for rank in range(world):
        value, ms, sigs = out[rank]
        assert ms == pytest.approx(15.0)  # the slowest rank's time
        assert value == pytest.approx(world * 4096 / 0.015)
        assert sigs[0] != sigs[1]  # each rank scores its own shard
