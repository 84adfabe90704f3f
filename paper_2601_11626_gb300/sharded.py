"""Alg. 3 (approximate incremental clustering, Appendix E) with the candidate
queue sharded across ranks.

One process per GPU.  Every rank holds the whole block collection (inputs
are replicated); the cluster state is replicated too and kept identical by
a broadcast from rank 0 after every commit.  What is split is the merge
scoring, the expensive part of the scan: a chunk of candidates taken in scan
order is dealt to the ranks by position (rank p scores positions p, p + W,
...), each rank scores its share against the current state in one batched
call, and one all-gather returns the accept flag of every candidate of the
chunk to every rank.  All ranks then take the same decision -- the first accepted
candidate in scan order joins the cluster (Alg. 3 step 3(e)) -- so the
decisions equal those of a single rank scanning candidate by candidate
(a merge score does not depend on the batch it is scored in), and the scan
resumes after the accepted position with the new state.

The scan order is the ``frobenius`` one of the single-GPU driver: ascending
||A_j||_F, repeated passes until a pass accepts nothing; anchors are the
largest remaining block, ties to the lowest index.

The scoring itself goes through a backend (``CsvdBackend`` below: the
library's batched merge evaluation on this rank's GPU); the exchange
through ``torch.distributed`` (NCCL between GPUs).  Only torch tensors and
plain Python values cross ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


class CsvdBackend:
    """Cluster states and batched merge scoring on this rank's GPU through the
    C ABI (csvd_incr_* and csvd_score)."""

    def __init__(self, blocks, r, eps, precision="mixed"):
        from . import csvd
        self.csvd = csvd
        self.blocks = blocks
        self.m = int(blocks[0].shape[0])
        self.r, self.eps, self.precision = r, eps, precision
        self.device = blocks[0].device

    def energy(self, j):
        return float(self.csvd.block_energy([self.blocks[j]])[0])

    def new_state(self, anchor):
        st = self.csvd.IncrSVD(self.m, self.r)
        st.append(self.blocks[anchor])
        return st

    def score(self, st, idx):
        """E~^2 and accept flags of candidates ``idx`` against ``st``."""
        if not idx:
            return [], []
        _, tail, _, acc = self.csvd.score([st], [0] * len(idx), [self.blocks[j] for j in idx],
                                          self.eps, self.precision)
        return tail.cpu().tolist(), [bool(a) for a in acc.cpu().tolist()]

    def commit(self, st, j):
        st.append(self.blocks[j])

    def export(self, st):
        te = st.tail_error()
        U = st.basis().contiguous()
        sig = torch.as_tensor(st.sigma(), dtype=torch.float32, device=U.device)
        scal = torch.tensor([te["energy"], te["tail_sq"]], dtype=torch.float64, device=U.device)
        return [U, sig, scal]

    def shapes(self, st):
        rk = st.rank
        return [((self.m, rk), torch.float32), ((rk,), torch.float32), ((2,), torch.float64)]

    def load(self, st, parts):
        U, sig, scal = parts
        st.load(U.to(self.device), sig.cpu().numpy(), float(scal[0]), float(scal[1]))

    def estimate_sq(self, st):
        return st.tail_error()["tail_sq"]


def _share(chunk, rank, world):
    return chunk[rank::world]


def _broadcast_state(backend, st, rank, group, device):
    """Rank 0's state to every rank (ranks agree on the shapes: the state's
    rank is the same on every rank, since every rank committed the same
    blocks)."""
    shapes = backend.shapes(st)
    if rank == 0:
        parts = [p.to(device) for p in backend.export(st)]
    else:
        parts = [torch.empty(s, dtype=dt, device=device) for s, dt in shapes]
    for p in parts:
        dist.broadcast(p, src=0, group=group)
    if rank != 0:
        backend.load(st, parts)


def cluster_approx_sharded(backend, n_blocks, eps, chunk=None, group=None, device="cpu"):
    """Alg. 3 with the frobenius scan, the merge scoring of each chunk split
    across the ranks of ``group``.  Returns (labels, clusters, estimate_sq).
    Every rank returns the same values."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    chunk = chunk or 64 * world
    norms = [backend.energy(j) for j in range(n_blocks)]
    # the energies decide every order: rank 0's values for everyone
    nt = torch.tensor(norms, dtype=torch.float64, device=device)
    dist.broadcast(nt, src=0, group=group)
    norms = nt.cpu().tolist()
    remaining = sorted(range(n_blocks), key=lambda j: (-norms[j], j))
    labels = [-1] * n_blocks
    clusters, estimates = [], []
    while remaining:
        anchor = remaining.pop(0)
        st = backend.new_state(anchor)
        _broadcast_state(backend, st, rank, group, device)
        members = [anchor]
        while True:
            order = sorted(remaining, key=lambda j: (norms[j], j))
            accepted_any = False
            pos = 0
            while pos < len(order):
                cand = order[pos:pos + chunk]
                mine = _share(list(range(len(cand))), rank, world)
                tails, flags = backend.score(st, [cand[i] for i in mine])
                # (position in chunk, flag) of every rank's share, gathered
                buf = torch.full((2, (len(cand) + world - 1) // world), -1.0, dtype=torch.float64,
                                 device=device)
                for t, (i, f) in enumerate(zip(mine, flags)):
                    buf[0, t] = float(i)
                    buf[1, t] = 1.0 if f else 0.0
                bufs = [torch.empty_like(buf) for _ in range(world)]
                dist.all_gather(bufs, buf, group=group)
                first = None
                for b in bufs:
                    for i, f in zip(b[0].tolist(), b[1].tolist()):
                        if i >= 0 and f > 0.5 and (first is None or i < first):
                            first = int(i)
                if first is None:
                    pos += len(cand)
                    continue
                j = cand[first]
                backend.commit(st, j)
                _broadcast_state(backend, st, rank, group, device)
                members.append(j)
                remaining.remove(j)
                accepted_any = True
                # the pass resumes after the accepted candidate, against the
                # new state (scores after it in this chunk are stale)
                pos = pos + first + 1
            if not accepted_any or not remaining:
                break
        cid = len(clusters)
        for j in members:
            labels[j] = cid
        clusters.append(members)
        estimates.append(backend.estimate_sq(st))
    return labels, clusters, estimates
