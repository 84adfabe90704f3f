"""Pins for the streaming-assignment oracle (no GPU): cases whose labels
follow from the definition by hand."""
import numpy as np
import pytest

from oracle import stream as ostream


def _coord_blocks(m, dims, seq, k, seed):
    """Blocks k columns wide inside coordinate subspaces: subspace c spans
    coordinates [sum(dims[:c]), sum(dims[:c+1]))."""
    rng = np.random.default_rng(seed)
    starts = np.cumsum([0] + list(dims))
    out = []
    for c in seq:
        b = np.zeros((m, k))
        b[starts[c]:starts[c + 1], :] = rng.standard_normal((dims[c], k))
        out.append(b)
    return out


def test_loose_constraint_keeps_one_cluster():
    """eps = 1: E~^2 <= ||M||^2 always holds, so every block joins cluster 0."""
    rng = np.random.default_rng(0)
    blocks = [rng.standard_normal((20, 3)) for _ in range(7)]
    assert ostream.assign(blocks, 2, 1.0)["labels"] == [0] * 7


def test_no_truncation_keeps_one_cluster_even_at_eps_zero():
    """r at least the rank of everything: nothing is discarded, E~^2 = 0."""
    rng = np.random.default_rng(1)
    blocks = [rng.standard_normal((30, 2)) for _ in range(5)]
    assert ostream.assign(blocks, 10, 0.0)["labels"] == [0] * 5


def test_orthogonal_subspaces_give_one_cluster_each():
    """Blocks inside three orthogonal 3-dim coordinate subspaces, r = 3: a
    block joins its own subspace's cluster with E~ = 0, and any other merge
    has rank > 3 with a large discarded share, so labels follow the order of
    first appearance of the subspaces."""
    seq = [2, 0, 2, 1, 0, 1, 2, 0]
    blocks = _coord_blocks(12, [3, 3, 3], seq, 2, 2)
    first = {}
    want = [first.setdefault(c, len(first)) for c in seq]
    out = ostream.assign(blocks, 3, 0.01)
    assert out["labels"] == want
    for st in out["states"]:
        assert st.discarded == pytest.approx(0.0, abs=1e-20)


def test_best_fit_not_first_fit():
    """Cluster 0 spans {e1, e3}, cluster 1 spans {e1, e2} (r = 2; the two
    cannot merge).  The block e1 + 0.1 e2 fits both (relative error 0 for
    cluster 1, about 0.1 / sqrt(3) for cluster 0 at eps = 0.2) and must go
    to cluster 1, the smaller estimate, not to the first accepting one."""
    m = 6
    e = np.eye(m)
    b0 = np.stack([e[0], e[2]], axis=1)
    b1 = np.stack([e[0], e[1]], axis=1)
    b2 = (e[0] + 0.1 * e[1])[:, None]
    out = ostream.assign([b0, b1, b2], 2, 0.2)
    assert out["labels"] == [0, 1, 1]
    (c0, d0, n0, ok0), (c1, d1, n1, ok1) = out["log"][2]
    assert ok0 and ok1 and d1 < d0
    # the estimate against cluster 0: merged singular values of
    # [e1, e3, e1 + 0.1 e2] beyond rank 2, computed by hand from the Gram
    M = np.concatenate([b0, b2], axis=1)
    s = np.linalg.svd(M, compute_uv=False)
    assert d0 == pytest.approx(float(np.sum(s[2:] ** 2)), rel=1e-10)


def test_state_grows_with_each_join():
    """e1, e2, e3 join one cluster (rank 3 = r, nothing discarded); 0.5 e4
    would discard 0.25 of 3.25, a relative error of 0.277 > 0.2, so it
    starts cluster 1.  Against a cluster holding only e1 it would fit."""
    e = np.eye(6)
    blocks = [e[0][:, None], e[1][:, None], e[2][:, None], 0.5 * e[3][:, None]]
    out = ostream.assign(blocks, 3, 0.2)
    assert out["labels"] == [0, 0, 0, 1]
    assert out["states"][0].energy == pytest.approx(3.0)
    assert out["states"][1].energy == pytest.approx(0.25)
    (_, d, n, ok), = out["log"][3]
    assert not ok and d == pytest.approx(0.25) and n == pytest.approx(3.25)


PINS = [test_loose_constraint_keeps_one_cluster, test_no_truncation_keeps_one_cluster_even_at_eps_zero,
        test_orthogonal_subspaces_give_one_cluster_each, test_best_fit_not_first_fit,
        test_state_grows_with_each_join]


@pytest.mark.parametrize("old,new", [
    ("if ok and (best < 0 or rel < best_rel):", "if ok and best < 0:"),        # first fit
    ("ok = discarded <= e2 * energy", "ok = True"),                            # no constraint
    ("states[best].commit(best_nxt)", "pass"),                                 # state not updated
    ("e2 = eps * eps", "e2 = eps"),                                            # eps not squared
])
def test_pins_catch_planted_mistakes(old, new, monkeypatch):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(ostream.assign))
    assert old in src
    ns = dict(ostream.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    monkeypatch.setattr(ostream, "assign", ns["assign"])
    failed = 0
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed > 0, f"no pin caught the mutant {new!r}"
