"""Pins of the randomized range-finder estimator (oracle/randomized.py):
never below the exact tail (Eckart-Young) for any draw, exact when the
collection's rank is at most r, converging to the exact tail with power
iterations on a gapped collection, equal to a hand-built two-block case,
and planted mistakes (a projector from the sketch's last vectors, a missing
block in the residual, a residual measured against the sketch instead of
its singular basis) caught."""
import numpy as np
import pytest

from oracle import exact
from oracle import randomized as rnd
from paper_2601_11626_gb300 import synth


def _blocks(seed, widths=(12, 9, 15), m=40, rank=None, decay=0.8):
    return [b.double().numpy() for b in synth.random_blocks(m, list(widths), seed=seed,
                                                            rank=rank, decay=decay)]


@pytest.mark.parametrize("seed", range(6))
def test_never_below_exact_tail(seed):
    blocks = _blocks(seed)
    for r in (2, 5, 9):
        om = rnd.gaussian_omegas([b.shape[1] for b in blocks], r + 4, seed + 100)
        for q in (0, 1):
            assert rnd.tail_sq(blocks, om, r, q) >= exact.tail_sq(blocks, r) * (1 - 1e-12) - 1e-12


def test_exact_when_rank_at_most_r():
    blocks = _blocks(3, rank=2)   # each block rank 2, 3 blocks: rank <= 6
    r = 6
    om = rnd.gaussian_omegas([b.shape[1] for b in blocks], r + 2, 7)
    assert rnd.tail_sq(blocks, om, r, 0) <= 1e-13 * exact.energy(blocks)


def test_power_iterations_converge_on_gapped_data():
    """M = U diag(s) V^T with a gap of 20 after r = 8: each power iteration
    shrinks the sketch's angle to the top-8 subspace by (1/20)^2, and the
    estimate reaches the exact tail."""
    rng = np.random.default_rng(4)
    m, N, r = 60, 60, 8
    u, _ = np.linalg.qr(rng.standard_normal((m, m)))
    v, _ = np.linalg.qr(rng.standard_normal((N, N)))
    s = np.array([10.0] * r + [0.5] * (m - r))
    M = (u * s) @ v.T
    blocks = [M[:, :20], M[:, 20:45], M[:, 45:]]
    om = rnd.gaussian_omegas([b.shape[1] for b in blocks], r + 4, 3)
    want = exact.tail_sq(blocks, r)
    assert want == pytest.approx(0.25 * (m - r), rel=1e-12)
    errs = [rnd.tail_sq(blocks, om, r, q) / want - 1 for q in (0, 1, 3)]
    assert errs[0] >= errs[1] >= errs[2] >= -1e-12
    assert errs[2] < 1e-9


def test_hand_built_orthogonal_case():
    """A_1 = 3 e_1, A_2 = [2 e_2, e_3] (singular values 3, 2, 1), r = 2, and
    a draw whose sketch has no e_3 component: Y spans e_1, e_2, so does every
    power iteration, U_r = {e_1, e_2} and the estimate is e_3's energy, 1 =
    the exact tail."""
    m = 5
    a1 = np.zeros((m, 1)); a1[0, 0] = 3.0
    a2 = np.zeros((m, 2)); a2[1, 0] = 2.0; a2[2, 1] = 1.0
    om = [np.array([[1.0, 0.5]]), np.array([[0.3, 1.0], [0.0, 0.0]])]
    for q in (0, 1):
        assert rnd.tail_sq([a1, a2], om, 2, q) == pytest.approx(1.0, rel=1e-12)
    assert exact.tail_sq([a1, a2], 2) == pytest.approx(1.0, rel=1e-12)
    # a draw that does see e_3 (and no power iteration) pays for it
    om2 = [np.array([[1.0, 0.5]]), np.array([[0.3, 1.0], [2.0, 0.1]])]
    assert rnd.tail_sq([a1, a2], om2, 2, 0) > 1.0 + 1e-3


def _bad_last_vectors(blocks, om, r, q):
    Y = rnd.sketch(blocks, om)
    for _ in range(q):
        Y = rnd.power_step(blocks, Y)
    u, _, _ = np.linalg.svd(Y, full_matrices=False)
    U = u[:, -r:]
    return sum(float(np.sum((a - U @ (U.T @ a)) ** 2)) for a in blocks)


def _bad_missing_block(blocks, om, r, q):
    return rnd.tail_sq(blocks[:-1], om[:-1], r, q)


def _bad_sketch_residual(blocks, om, r, q):
    Y = rnd.sketch(blocks, om)
    Q, _ = np.linalg.qr(Y)
    return sum(float(np.sum((a - Q @ (Q.T @ a)) ** 2)) for a in blocks)


@pytest.mark.parametrize("bad", [_bad_last_vectors, _bad_missing_block, _bad_sketch_residual])
def test_planted_mistakes_are_caught(bad):
    blocks = _blocks(11, widths=(10, 14, 8), m=30, decay=0.7)
    r = 4
    om = rnd.gaussian_omegas([b.shape[1] for b in blocks], r + 6, 5)
    good = rnd.tail_sq(blocks, om, r, 1)
    ex = exact.tail_sq(blocks, r)
    wrong = bad(blocks, om, r, 1)
    # the pins above: >= exact always, close to exact after an iteration
    caught = wrong < ex * (1 - 1e-9) or abs(wrong - good) > 1e-3 * good
    assert caught
