"""The multi-rank paths on CPU, as gloo ranks on 127.0.0.1.

Batched scoring shards by candidates with no exchange on the data path;
each rank generates its own workload from its rank seed, and the job's
throughput is every rank's units over the slowest rank's time (one MAX
all-reduce of the timing).  The sharded Alg. 3 scan deals each chunk of
candidates to the ranks and must reproduce the single-process clustering
with two or three ranks, and a failing rank must make the others fail fast.
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


@pytest.mark.parametrize("world,chunk", [(2, 3), (2, 64), (3, 3)])
def test_sharded_alg3_scan_equals_single_rank(world, chunk):
    """Two or three gloo ranks run Alg. 3 (frobenius scan) on the small recipe
    with the candidate queue dealt to the ranks by position, and the cluster
    state broadcast after each commit: labels, members in joining order and
    the per-cluster estimates equal the single-process oracle clustering,
    every rank returns the same result, and every rank does scoring work.  A
    chunk of 3 puts accepts in the middle of chunks (stale scores
    discarded)."""
    from oracle import cluster as ocluster
    from paper_2601_11626_gb300 import synth
    col = synth.small_c1()
    want = ocluster.cluster(col.blocks, col.meta["r"], col.meta["eps"], "approx", "frobenius")
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_sharded_worker, args=(world, _free_port(), out, chunk), nprocs=world,
                       join=True, start_method="spawn")
    assert set(out.keys()) == set(range(world))
    for rank in range(world):
        labels, clusters, est, scored = out[rank]
        assert labels == want["labels"]
        assert clusters == want["clusters"]
        for a, b in zip(est, want["estimate_sq"]):
            assert a == pytest.approx(b, rel=1e-9, abs=1e-12)
        assert len(scored) > 0
    assert len(want["clusters"]) > 1 and max(len(c) for c in want["clusters"]) > 1


def _failing_worker(rank, world, port, out):
    """Rank 1's scoring raises on its first call; every rank records how it
    ended instead of exiting with the exception."""
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    try:
        from paper_2601_11626_gb300 import sharded, synth
        col = synth.small_c1()
        be = _OracleBackend(col.blocks, col.meta["r"], col.meta["eps"])
        if rank == 1:
            def broken(st, idx):
                raise RuntimeError("planted scoring failure")
            be.score = broken
        sharded.cluster_approx_sharded(be, len(col.blocks), col.meta["eps"], chunk=4)
        out[rank] = ("finished", "")
    except Exception as e:  # noqa: BLE001 -- the test inspects how each rank ended
        out[rank] = ("error", f"{type(e).__name__}: {e}"[:300])
    finally:
        dist.destroy_process_group()


def test_sharded_scan_fails_fast_when_a_rank_fails():
    """A rank whose scoring raises leaves the scan between collectives; the
    other rank's next collective ends with an error (the peer closed its
    connection, or the 20 s process-group timeout) instead of waiting for
    ever, and neither rank reports a result."""
    import time
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.start_processes(_failing_worker, args=(world, _free_port(), out), nprocs=world,
                             join=False, start_method="spawn")
    t0 = time.time()
    for p in ctx.processes:
        p.join(timeout=90)
    alive = [p for p in ctx.processes if p.is_alive()]
    for p in alive:
        p.terminate()
    assert not alive, "a rank hung after its peer failed"
    assert time.time() - t0 < 90
    assert out[1][0] == "error" and "planted scoring failure" in out[1][1]
    assert out[0][0] == "error", out[0]
