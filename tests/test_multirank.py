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


# --------------------------------------------- sharded Alg. 3 candidate queue
class _OracleBackend:
    """The sharded driver's backend interface over the FP64 oracle (CPU): the
    same scan logic as on GPUs, with the oracle's merge evaluation."""

    def __init__(self, blocks, r, eps):
        import numpy as np
        self.np = np
        self.blocks = [b.double().numpy() for b in blocks]
        self.m = self.blocks[0].shape[0]
        self.r, self.eps = r, eps

    def energy(self, j):
        return float(self.np.sum(self.blocks[j] ** 2))

    def new_state(self, anchor):
        from oracle import incremental as oinc
        st = oinc.IncrementalSVD(self.m, self.r)
        st.append(self.blocks[anchor])
        return st

    def score(self, st, idx):
        tails, flags = [], []
        for j in idx:
            _, t, ok, _ = st.evaluate(self.blocks[j], self.eps)
            tails.append(t)
            flags.append(ok)
        return tails, flags

    def commit(self, st, j):
        st.append(self.blocks[j])

    def export(self, st):
        return [torch.tensor(st.Q), torch.tensor(st.s),
                torch.tensor([st.energy, st.discarded], dtype=torch.float64)]

    def shapes(self, st):
        rk = st.Q.shape[1]
        return [((self.m, rk), torch.float64), ((rk,), torch.float64), ((2,), torch.float64)]

    def load(self, st, parts):
        U, s, scal = parts
        st.Q, st.s = U.numpy().copy(), s.numpy().copy()
        st.energy, st.discarded = float(scal[0]), float(scal[1])

    def estimate_sq(self, st):
        return st.tail_sq()


def _sharded_worker(rank, world, port, out, chunk):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2601_11626_gb300 import sharded, synth
        col = synth.small_c1()
        be = _OracleBackend(col.blocks, col.meta["r"], col.meta["eps"])
        scored = []
        inner = be.score

        def counting(st, idx):
            scored.extend(idx)
            return inner(st, idx)

        be.score = counting
        labels, clusters, est = sharded.cluster_approx_sharded(be, len(col.blocks),
                                                               col.meta["eps"], chunk=chunk)
        out[rank] = (labels, clusters, est, sorted(scored))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("chunk", [3, 64])
def test_sharded_alg3_scan_equals_single_rank(chunk):
    """Two gloo ranks run Alg. 3 (frobenius scan) on the small recipe with the
    candidate queue dealt to the ranks by position, and the cluster state
    broadcast after each commit: labels, members in joining order and the
    per-cluster estimates equal the single-process oracle clustering, every
    rank returns the same result, and both ranks do scoring work.  A chunk
    of 3 puts accepts in the middle of chunks (stale scores discarded)."""
    from oracle import cluster as ocluster
    from paper_2601_11626_gb300 import synth
    col = synth.small_c1()
    want = ocluster.cluster(col.blocks, col.meta["r"], col.meta["eps"], "approx", "frobenius")
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_sharded_worker, args=(world, _free_port(), out, chunk), nprocs=world,
                       join=True, start_method="spawn")
    assert set(out.keys()) == {0, 1}
    for rank in range(world):
        labels, clusters, est, scored = out[rank]
        assert labels == want["labels"]
        assert clusters == want["clusters"]
        for a, b in zip(est, want["estimate_sq"]):
            assert a == pytest.approx(b, rel=1e-9, abs=1e-12)
        assert len(scored) > 0
    assert len(want["clusters"]) > 1 and max(len(c) for c in want["clusters"]) > 1
