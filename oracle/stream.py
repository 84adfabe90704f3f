"""Streaming cluster assignment (FP64), the incremental setting the paper's
discussion section names as future work: matrices arrive one at a time and
each joins an existing cluster or starts a new one by its predicted
compression error.

Test infrastructure (see the package docstring).

Reading (the paper gives no algorithm): block A_t is tentatively appended to
every open cluster's rank-r incremental state (Lemma 1, Cor. 3); a cluster
accepts when the plug-in estimate of the merged cluster meets the constraint,
E~^2 <= eps^2 ||M_{C u t}||_F^2 (Cor. 2, with E~^2 as the accumulated
discarded energy); among the accepting clusters the one with the smallest
estimated relative error E~^2 / ||M||_F^2 receives A_t (ties to the lowest
cluster index); when none accepts, A_t starts a new cluster.  Clusters are
numbered in order of creation.
"""
from __future__ import annotations

from .exact import _f64
from .incremental import IncrementalSVD


def assign(blocks, r, eps):
    """Labels of the blocks in arrival order, the cluster states and, per
    block, the evaluations against the clusters open when it arrived:
    (cluster, E~^2, ||M||^2, accepted)."""
    states, labels, log = [], [], []
    e2 = eps * eps
    for A in blocks:
        A = _f64(A)
        m = A.shape[0]
        best, best_rel, best_nxt = -1, None, None
        scores = []
        for c, st in enumerate(states):
            nxt, _ = st.step(A)
            energy, discarded = nxt[2], nxt[3]
            ok = discarded <= e2 * energy
            scores.append((c, discarded, energy, ok))
            rel = discarded / energy if energy > 0 else 0.0
            if ok and (best < 0 or rel < best_rel):
                best, best_rel, best_nxt = c, rel, nxt
        if best < 0:
            st = IncrementalSVD(m, r)
            st.append(A)
            states.append(st)
            best = len(states) - 1
        else:
            states[best].commit(best_nxt)
        labels.append(best)
        log.append(scores)
    return dict(labels=labels, states=states, log=log)
