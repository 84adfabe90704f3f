"""Greedy error-constrained clustering, Algorithms 1-3 of Appendix E (FP64).

Test infrastructure (see the package docstring).

All three share one loop: the largest-norm unassigned block anchors a new
cluster; remaining blocks are offered in a candidate order; a block joins
when its merge certificate holds (relative error of the enlarged cluster
<= eps, i.e. bound^2 <= eps^2 * ||M_{C u j}||_F^2); when no block can join,
the next cluster starts.  They differ in the certificate:

* Alg. 1 (max-norm, Weyl): Thm. 1 on norms and top-r block energies.
* Alg. 2 (residual): Cor. 1 with a full-span cluster basis Q_C.
* Alg. 3 (approximate): the plug-in estimate of a rank-r incremental SVD.

Readings (paper silent or ambiguous):
* Ties in any ordering are broken by ascending block index; anchors are the
  largest ||A||_F, ties to the lowest index.
* Candidate order ``frobenius``: ascending ||A_j||_F.  One scan offers every
  remaining block once, in that order, and the cluster state is updated after
  each accepted block; scans repeat until one accepts nothing.
* Candidate order ``residual``: ascending ||(I - Q_C Q_C^T) A_j||_F with
  respect to the current basis; after every accepted block the residual norms
  of all remaining blocks are recomputed, and the smallest-residual block
  whose certificate holds joins; the cluster closes when none holds.
* Alg. 1's head: the anchor and then the next-largest blocks join while their
  cumulative width stays <= r (the head has rank <= r, so its top-r energy is
  ||head||_F^2, and Thm. 1 applied to {head, other blocks} gives
  bound^2 = S - S_head).  If the anchor alone is wider than r there is no
  head and bound^2 = S - max_{j in C} sum_{i<=r} sigma_i^2(A_j) (general
  Thm. 1).  Alg. 1 uses the ``frobenius`` scan.
* Alg. 2 basis: the full column space of the cluster (Thm. 2's hypothesis),
  not its leading rank-r subspace.
* Compression ratio (Section 4): a cluster with N_c columns stores
  min(m N_c, r_eff (m + N_c)) numbers, r_eff = min(r, N_c, m) -- a cluster
  that would not shrink is stored raw; ratio = sum m N_c / sum stored.
"""
from __future__ import annotations

import numpy as np

from .bounds import ResidualState, top_r_energy
from .exact import _f64
from .incremental import IncrementalSVD


def _norms_sq(blocks):
    return [float(np.sum(_f64(b) ** 2)) for b in blocks]


def _desc_order(norms):
    return sorted(range(len(norms)), key=lambda j: (-norms[j], j))


class _Weyl:
    """Alg. 1 cluster state."""

    def __init__(self, blocks, norms, r, members, head):
        self.blocks, self.norms, self.r = blocks, norms, r
        self.members = list(members)
        self.energy = sum(norms[j] for j in members)
        self.head_energy = sum(norms[j] for j in head) if head else None
        self.top = (max(top_r_energy(blocks[j], r) for j in members)
                    if not head else None)

    def bound_sq(self, j):
        energy = self.energy + self.norms[j]
        if self.head_energy is not None:
            return max(0.0, energy - self.head_energy), energy, None
        top = max(self.top, top_r_energy(self.blocks[j], self.r))
        return max(0.0, energy - top), energy, top

    def accept(self, j, info):
        self.members.append(j)
        self.energy += self.norms[j]
        if info is not None:
            self.top = info

    def estimate_sq(self):
        if self.head_energy is not None:
            return max(0.0, self.energy - self.head_energy)
        return max(0.0, self.energy - self.top)


class _Residual:
    """Alg. 2 cluster state (full-span basis and residual spectrum)."""

    def __init__(self, blocks, m, r, anchor):
        self.blocks, self.r = blocks, r
        self.st = ResidualState(m)
        self.st.append(blocks[anchor])
        self.members = [anchor]

    def bound_sq(self, j):
        nxt = self.st.step(self.blocks[j])
        return self.st.bound_sq(self.r, nxt), nxt[2], nxt

    def accept(self, j, nxt):
        self.st.commit(nxt)
        self.members.append(j)

    def residual_norm_sq(self, j):
        R = self.st.residual(self.blocks[j])
        return float(np.sum(R * R))

    def estimate_sq(self):
        return self.st.bound_sq(self.r)


class _Approx:
    """Alg. 3 cluster state (rank-r incremental SVD)."""

    def __init__(self, blocks, m, r, anchor):
        self.blocks, self.r = blocks, r
        self.st = IncrementalSVD(m, r)
        self.st.append(blocks[anchor])
        self.members = [anchor]

    def bound_sq(self, j):
        nxt, _ = self.st.step(self.blocks[j])
        _, s_new, energy, _ = nxt
        return max(0.0, energy - float(np.sum(s_new ** 2))), energy, nxt

    def accept(self, j, nxt):
        self.st.commit(nxt)
        self.members.append(j)

    def residual_norm_sq(self, j):
        A = _f64(self.blocks[j])
        Q = self.st.Q
        R = A - Q @ (Q.T @ A)
        R = R - Q @ (Q.T @ R)
        return float(np.sum(R * R))

    def estimate_sq(self):
        return self.st.tail_sq()


def _grow(state, remaining, norms, eps, sort_mode, log):
    """Offer the remaining blocks to one cluster until none can join."""
    e2 = eps * eps
    if sort_mode == "frobenius":
        while True:
            order = sorted(remaining, key=lambda j: (norms[j], j))
            accepted_any = False
            for j in order:
                b2, energy, info = state.bound_sq(j)
                ok = b2 <= e2 * energy
                log.append((len(state.members), j, b2, energy, ok))
                if ok:
                    state.accept(j, info)
                    remaining.remove(j)
                    accepted_any = True
            if not accepted_any or not remaining:
                return
    elif sort_mode == "residual":
        while remaining:
            order = sorted(remaining, key=lambda j: (state.residual_norm_sq(j), j))
            for j in order:
                b2, energy, info = state.bound_sq(j)
                ok = b2 <= e2 * energy
                log.append((len(state.members), j, b2, energy, ok))
                if ok:
                    state.accept(j, info)
                    remaining.remove(j)
                    break
            else:
                return
    else:
        raise ValueError(sort_mode)


def cluster(blocks, r, eps, algo="approx", sort_mode="frobenius"):
    """Run Alg. 1 (``weyl``), Alg. 2 (``residual``) or Alg. 3 (``approx``).

    Returns dict(labels, clusters (member lists in order of joining),
    estimate_sq (per cluster, the certificate's bound / estimate),
    energy (per cluster), compression_ratio, log)."""
    m = int(blocks[0].shape[0])
    norms = _norms_sq(blocks)
    desc = _desc_order(norms)
    remaining = list(desc)
    labels = [-1] * len(blocks)
    clusters, est, energies, log = [], [], [], []
    widths = [int(b.shape[1]) for b in blocks]
    while remaining:
        anchor = remaining[0]
        remaining.remove(anchor)
        if algo == "weyl":
            head = []
            if widths[anchor] <= r:
                head, width = [anchor], widths[anchor]
                for j in [x for x in desc if x in remaining]:
                    if width + widths[j] > r:
                        break
                    head.append(j)
                    width += widths[j]
                    remaining.remove(j)
            state = _Weyl(blocks, norms, r, head if head else [anchor], head)
            _grow(state, remaining, norms, eps, "frobenius", log)
        elif algo == "residual":
            state = _Residual(blocks, m, r, anchor)
            _grow(state, remaining, norms, eps, sort_mode, log)
        elif algo == "approx":
            state = _Approx(blocks, m, r, anchor)
            _grow(state, remaining, norms, eps, sort_mode, log)
        else:
            raise ValueError(algo)
        cid = len(clusters)
        for j in state.members:
            labels[j] = cid
        clusters.append(list(state.members))
        est.append(state.estimate_sq())
        energies.append(sum(norms[j] for j in state.members))
    return dict(labels=labels, clusters=clusters, estimate_sq=est, energy=energies,
                compression_ratio=compression_ratio(clusters, widths, m, r), log=log)


def compression_ratio(clusters, widths, m, r):
    """Original numbers / stored numbers (Section 4 'Compression ratio')."""
    raw = stored = 0
    for c in clusters:
        n_c = sum(widths[j] for j in c)
        r_eff = min(r, n_c, m)
        raw += m * n_c
        stored += min(m * n_c, r_eff * (m + n_c))
    return raw / stored
