"""Pins of the oracle's clustering (Algorithms 1-3) and compression ratio.

Hand-derived partitions, feasibility against the exact SVD, and exhaustive
search over all partitions of tiny collections.  CPU only.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import cluster, exact
from paper_2601_11626_gb300 import synth


def _orth(rng, m, n):
    q, rr = np.linalg.qr(rng.standard_normal((m, n)))
    return q * np.sign(np.diag(rr))


def test_weyl_head_hand_derived():
    """Alg. 1 with rank-one blocks of norms 10, 9, 1e-3, 2e-3 and r = 2: the
    head {10, 9} has rank 2; bound^2 = S - S_head."""
    rng = np.random.default_rng(0)
    U = _orth(rng, 5, 4)
    blocks = [U[:, [j]] * s for j, s in enumerate([10.0, 9.0, 1e-3, 2e-3])]
    out = cluster.cluster(blocks, 2, 1e-3, "weyl")
    assert out["clusters"] == [[0, 1, 2, 3]]
    # eps^2 = 1e-8: 1e-6/181 passes, (1e-6 + 4e-6)/181 does not
    out = cluster.cluster(blocks, 2, 1e-4, "weyl")
    assert out["clusters"] == [[0, 1, 2], [3]]


def test_approx_recovers_exact_subspaces():
    """Alg. 3 on noiseless blocks from three orthogonal rank-2 subspaces
    with r = 2 merges exactly the blocks of each subspace."""
    rng = np.random.default_rng(1)
    Q = _orth(rng, 12, 6)
    blocks, lat = [], []
    for j in range(9):
        c = j % 3
        blocks.append(Q[:, 2 * c:2 * c + 2] @ rng.standard_normal((2, 3)) * (1 + 0.1 * j))
        lat.append(c)
    for mode in ("frobenius", "residual"):
        out = cluster.cluster(blocks, 2, 1e-6, "approx", mode)
        parts = sorted(sorted(c) for c in out["clusters"])
        want = sorted(sorted(j for j in range(9) if lat[j] == c) for c in range(3))
        assert parts == want


def test_residual_merges_orthogonal_growth_only_up_to_rank():
    """Alg. 2 with r = 4 and rank-2 blocks from mutually orthogonal
    subspaces: the anchor takes exactly one partner (mu gets 4 values, the
    bound is 0); a third block leaves two residual directions out."""
    rng = np.random.default_rng(2)
    Q = _orth(rng, 12, 6)
    scales = [3.0, 2.0, 1.0]
    blocks = [Q[:, 2 * c:2 * c + 2] * scales[c] for c in range(3)]
    out = cluster.cluster(blocks, 4, 0.1, "residual", "frobenius")
    # anchor 0 (largest); candidates ascending: 2 (norm 1) joins first
    assert out["clusters"] == [[0, 2], [1]]
    assert out["estimate_sq"][0] < 1e-20


@pytest.mark.parametrize("algo,mode", [("weyl", "frobenius"), ("residual", "frobenius"),
                                       ("residual", "residual"), ("approx", "frobenius"),
                                       ("approx", "residual")])
def test_clusters_satisfy_constraint_c1(algo, mode):
    """Every cluster of every algorithm meets E_r(M_C) <= eps ||M_C||_F,
    checked with the exact SVD (Alg. 1/2 by their theorems; Alg. 3 because
    its plug-in estimate never falls below the true error)."""
    col = synth.small_c1()
    r, eps = col.meta["r"], col.meta["eps"]
    out = cluster.cluster(col.blocks, r, eps, algo, mode)
    assert sorted(j for c in out["clusters"] for j in c) == list(range(16))
    for c in out["clusters"]:
        bl = [col.blocks[j] for j in c]
        assert exact.rel_error(bl, r) <= eps * (1 + 1e-9)


def test_c1_approx_groups_latent_pairs():
    """On the small recipe (4 rank-8 latent subspaces, r = 16) two latent
    subspaces fit in rank 16, so no Alg. 3 cluster mixes more than two."""
    col = synth.small_c1()
    out = cluster.cluster(col.blocks, 16, 0.05, "approx", "frobenius")
    for c in out["clusters"]:
        assert len({col.latent[j] for j in c}) <= 2
    assert len(out["clusters"]) < 16


def _partitions(items):
    if not items:
        yield []
        return
    first, rest = items[0], items[1:]
    for p in _partitions(rest):
        yield [[first]] + p
        for i in range(len(p)):
            yield p[:i] + [[first] + p[i]] + p[i + 1:]


def test_exhaustive_tiny():
    """All partitions of 6 tiny blocks: the greedy outputs are feasible and
    never store fewer numbers than the best feasible partition."""
    rng = np.random.default_rng(3)
    Q = _orth(rng, 6, 4)
    blocks = [Q[:, (j % 2) * 2:(j % 2) * 2 + 2] @ rng.standard_normal((2, 2))
              + 1e-3 * rng.standard_normal((6, 2)) for j in range(6)]
    r, eps, m = 2, 0.05, 6
    widths = [2] * 6
    best = None
    for p in _partitions(list(range(6))):
        if all(exact.rel_error([blocks[j] for j in c], r) <= eps for c in p):
            cr = cluster.compression_ratio(p, widths, m, r)
            best = cr if best is None else max(best, cr)
    for algo, mode in [("weyl", "frobenius"), ("residual", "frobenius"), ("approx", "frobenius"),
                       ("approx", "residual")]:
        out = cluster.cluster(blocks, r, eps, algo, mode)
        for c in out["clusters"]:
            assert exact.rel_error([blocks[j] for j in c], r) <= eps * (1 + 1e-9)
        assert out["compression_ratio"] <= best + 1e-12
    # Alg. 3 finds the two latent groups here, which is the optimum
    out = cluster.cluster(blocks, r, eps, "approx", "frobenius")
    assert math.isclose(out["compression_ratio"], best)


def test_exhaustive_eight_blocks():
    """All 4140 partitions (Bell(8)) of 8 blocks drawn from three latent
    2-dim subspaces of R^8 (r = 2): the greedy outputs are feasible, none
    stores fewer numbers than the best feasible partition, and Alg. 3 with
    the norm order reaches that optimum (one cluster per latent subspace)."""
    rng = np.random.default_rng(8)
    Q = _orth(rng, 8, 6)
    groups = [0, 1, 2, 0, 1, 2, 0, 1]
    blocks = [Q[:, 2 * g:2 * g + 2] @ rng.standard_normal((2, 2)) * rng.uniform(0.5, 2)
              + 1e-4 * rng.standard_normal((8, 2)) for g in groups]
    r, eps, m = 2, 0.05, 8
    widths = [2] * 8
    feasible = {}

    def ok(c):
        key = frozenset(c)
        if key not in feasible:
            feasible[key] = exact.rel_error([blocks[j] for j in c], r) <= eps
        return feasible[key]

    best, n_parts = None, 0
    for p in _partitions(list(range(8))):
        n_parts += 1
        if all(ok(c) for c in p):
            cr = cluster.compression_ratio(p, widths, m, r)
            best = cr if best is None else max(best, cr)
    assert n_parts == 4140
    for algo, mode in [("weyl", "frobenius"), ("residual", "frobenius"), ("approx", "frobenius"),
                       ("approx", "residual")]:
        out = cluster.cluster(blocks, r, eps, algo, mode)
        for c in out["clusters"]:
            assert exact.rel_error([blocks[j] for j in c], r) <= eps * (1 + 1e-9)
        assert out["compression_ratio"] <= best + 1e-12
    out = cluster.cluster(blocks, r, eps, "approx", "frobenius")
    assert math.isclose(out["compression_ratio"], best)
    assert sorted(sorted(c) for c in out["clusters"]) == [[0, 3, 6], [1, 4, 7], [2, 5]]


def test_compression_ratio_closed_form():
    """Section 4: K blocks of m x n at rank r store r (m + K n) numbers;
    clusters that would not shrink are stored raw."""
    m, n, r = 100, 20, 5
    got = cluster.compression_ratio([[0, 1, 2, 3]], [n] * 4, m, r)
    assert math.isclose(got, 4 * m * n / (r * (m + 4 * n)))
    got = cluster.compression_ratio([[0], [1]], [3, 3], 10, 5)
    assert got == 1.0


def test_frobenius_scan_repeats_until_nothing_joins():
    """Alg. 3, r = 1, eps = 0.09, blocks 10 e1 (anchor), 1 e2, 5 e1.  The
    ascending scan first offers 1 e2: one direction is discarded (energy 1 of
    101, relative error 0.0995 > 0.09) and it is refused; 5 e1 joins with
    nothing discarded; the next scan offers 1 e2 again, now 1 of 126
    (0.0891 <= 0.09), and it joins."""
    e = np.eye(3)
    blocks = [10.0 * e[:, [0]], 1.0 * e[:, [1]], 5.0 * e[:, [0]]]
    out = cluster.cluster(blocks, 1, 0.09, "approx", "frobenius")
    assert out["clusters"] == [[0, 2, 1]]
    first = out["log"][0]
    assert first[1] == 1 and not first[4]
    assert first[2] == pytest.approx(1.0) and first[3] == pytest.approx(101.0)
    assert out["estimate_sq"][0] == pytest.approx(1.0)
