"""Pins of the oracle's exact SVD, incremental estimator and bounds.

Each check compares the oracle with something other than itself: matrices
built from prescribed singular values, an independent tiny Jacobi solver,
closed forms of the paper's worked examples, and the paper's theorems as
invariants.  CPU only.
"""
import math
import os

import numpy as np
import pytest

from oracle import bounds, exact, incremental
from tests import _jacobi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _orth(rng, m, n):
    q, rr = np.linalg.qr(rng.standard_normal((m, n)))
    return q * np.sign(np.diag(rr))


def _prescribed(rng, m, n, s):
    """M = U diag(s) V^T with Haar U, V: singular values are s (plus zeros)."""
    k = len(s)
    return _orth(rng, m, k) @ np.diag(s) @ _orth(rng, n, k).T


def _split(M, widths):
    out, c = [], 0
    for w in widths:
        out.append(M[:, c:c + w])
        c += w
    return out


# --------------------------------------------------------------- exact (O1)
def test_singular_values_prescribed():
    rng = np.random.default_rng(1)
    s = np.array([5.0, 3.0, 2.5, 1.0, 0.25, 1e-3])
    M = _prescribed(rng, 17, 40, s)
    got = exact.singular_values(_split(M, [7, 13, 20]))
    np.testing.assert_allclose(got[:6], s, rtol=1e-12, atol=1e-14)
    assert np.all(got[6:] < 1e-13)
    for r in range(0, 7):
        assert math.isclose(exact.tail_sq(_split(M, [7, 13, 20]), r),
                            float(np.sum(s[r:] ** 2)), rel_tol=1e-12, abs_tol=1e-26)


def test_singular_values_vs_tiny_jacobi():
    rng = np.random.default_rng(2)
    for _ in range(20):
        m, n = rng.integers(2, 7), rng.integers(2, 9)
        M = rng.standard_normal((m, n))
        ref = _jacobi.singular_values(M)
        got = exact.singular_values([M])
        np.testing.assert_allclose(got, ref[:len(got)], rtol=1e-10, atol=1e-12)


def test_eckart_young_optimality():
    """Thm. 4: no rank-r approximation beats the tail; a random rank-r
    projection never does better than E_r^2."""
    rng = np.random.default_rng(3)
    M = rng.standard_normal((9, 14))
    for r in range(1, 5):
        t = exact.tail_sq([M], r)
        for _ in range(30):
            q = _orth(rng, 9, r)
            assert np.sum((M - q @ (q.T @ M)) ** 2) >= t - 1e-12


def test_energy_identity_and_weyl_monotonicity():
    """||M||_F^2 = sum sigma^2 and sigma_i([A B]) >= sigma_i(A) (Thm. 3)."""
    rng = np.random.default_rng(4)
    A, B = rng.standard_normal((8, 5)), rng.standard_normal((8, 3))
    s = exact.singular_values([A, B])
    assert math.isclose(float(np.sum(s ** 2)), exact.energy([A, B]), rel_tol=1e-13)
    sa = exact.singular_values([A])
    assert np.all(s[:len(sa)] >= sa - 1e-12)


def test_tail_gradient_finite_differences():
    rng = np.random.default_rng(5)
    s = np.array([4.0, 3.0, 2.0, 0.5, 0.3, 0.1])   # gap sigma_3/sigma_4 = 4
    M = _prescribed(rng, 10, 12, s)
    blocks = _split(M, [5, 7])
    g = exact.tail_grad(blocks, 3)
    h = 1e-4
    for _ in range(5):
        d = [rng.standard_normal(b.shape) for b in blocks]
        fp = exact.tail_sq([b + h * x for b, x in zip(blocks, d)], 3)
        fm = exact.tail_sq([b - h * x for b, x in zip(blocks, d)], 3)
        fd = (fp - fm) / (2 * h)
        an = sum(float(np.sum(gi * di)) for gi, di in zip(g, d))
        assert math.isclose(fd, an, rel_tol=2e-5, abs_tol=1e-9)


# ------------------------------------------------------ incremental (O2)
def test_incremental_exact_without_truncation():
    """Cor. 2: with no truncation the plug-in estimate is exact; the
    retained sigma~ are the prescribed singular values."""
    rng = np.random.default_rng(6)
    s = np.array([3.0, 2.0, 1.5, 1.0, 0.5, 0.2, 0.05])
    M = _prescribed(rng, 20, 24, s)
    blocks = _split(M, [4, 6, 3, 11])
    st, steps = incremental.run(blocks, r=10)
    np.testing.assert_allclose(st.s[:7], s, rtol=1e-11)
    for r in range(0, 8):
        st_r, _ = incremental.run(blocks, r=max(r, 7))
        assert math.isclose(st_r.energy - float(np.sum(st_r.s[:r] ** 2)),
                            float(np.sum(s[r:] ** 2)), rel_tol=1e-9, abs_tol=1e-12)


def test_lemma1_gram_identity():
    """Lemma 1: M_{t+1} M_{t+1}^T = [Q_t Q_res] K K^T [Q_t Q_res]^T before the
    truncation, whenever the state was exact."""
    rng = np.random.default_rng(7)
    A1, A2 = rng.standard_normal((12, 3)), rng.standard_normal((12, 4))
    st = incremental.IncrementalSVD(12, r=12)
    st.append(A1)
    _, d = st.step(A2)
    Qf = np.hstack([st.Q, d["Qres"]])
    lhs = A1 @ A1.T + A2 @ A2.T
    rhs = Qf @ d["K"] @ d["K"].T @ Qf.T
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
    np.testing.assert_allclose(Qf.T @ Qf, np.eye(Qf.shape[1]), atol=1e-13)
    np.testing.assert_allclose(d["R"], d["Qres"] @ d["B"], atol=1e-13)


def test_cor3_truncation_errors():
    """Cor. 3 (as the mathematics gives it): ||G - G~||_F^2 = sum_{j>r}
    lambda_j^2 and ||G - G~||_2 = lambda_{r+1}, G = M M^T of an exact state."""
    rng = np.random.default_rng(8)
    A1, A2 = rng.standard_normal((10, 3)), rng.standard_normal((10, 4))
    st = incremental.IncrementalSVD(10, r=10)
    st.append(A1)
    st.r = 3
    nxt, d = st.step(A2)
    Q3, s3 = nxt[0], nxt[1]
    G = A1 @ A1.T + A2 @ A2.T
    Gt = Q3 @ np.diag(s3 ** 2) @ Q3.T
    lam = np.sort(np.linalg.eigvalsh(G))[::-1]
    assert math.isclose(np.sum((G - Gt) ** 2), float(np.sum(lam[3:] ** 2)), rel_tol=1e-10)
    assert math.isclose(np.linalg.norm(G - Gt, 2), lam[3], rel_tol=1e-10)


def test_two_tail_routes_agree():
    rng = np.random.default_rng(9)
    blocks = [rng.standard_normal((30, w)) for w in (5, 8, 3, 9, 6)]
    st, steps = incremental.run(blocks, r=6)
    for s, paper, discard in steps:
        assert math.isclose(paper, discard, rel_tol=1e-10, abs_tol=1e-12)


def test_pw_restatement_tiny():
    """Each step equals the top-r SVD of [Q_t diag(s_t), A] (since
    [Q_t diag(s), A] = [Q_t Q_res] K); checked with the independent Jacobi."""
    rng = np.random.default_rng(10)
    for _ in range(10):
        m = int(rng.integers(4, 8))
        blocks = [rng.standard_normal((m, int(rng.integers(1, 4)))) for _ in range(4)]
        r = int(rng.integers(1, m))
        st = incremental.IncrementalSVD(m, r)
        for b in blocks:
            X = np.hstack([st.Q * st.s, b])
            ref = _jacobi.singular_values(X)[:r]
            st.append(b)
            np.testing.assert_allclose(st.s, ref[:len(st.s)], rtol=1e-9, atol=1e-12)


def test_plugin_never_below_true_error():
    """The retained Gram never exceeds the true Gram (truncation drops a PSD
    part; Lemma 1 + Thm. 3), so E~_r >= E_r for every order and every step."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        m = int(rng.integers(2, 8))
        blocks = [rng.standard_normal((m, int(rng.integers(1, 4)))) * rng.uniform(0.01, 3)
                  for _ in range(int(rng.integers(2, 6)))]
        r = int(rng.integers(1, m + 1))
        st, steps = incremental.run(blocks, r)
        for t, (_, paper, _) in enumerate(steps):
            ex = exact.tail_sq(blocks[:t + 1], r)
            assert paper >= ex - 1e-10 * exact.energy(blocks[:t + 1])


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split(None, 1)
                vals[k] = v
    return vals


def test_negative_slack_example_closed_forms():
    """Appendix D, Example 2 -- closed forms of the true error and of the
    energy discarded at steps 2 and 3; the plug-in estimate of Cor. 2 equals
    the sum of the discards (>= the true error), while the last step's
    discard alone is ~ half of it."""
    g = _golden("negative_slack.txt")
    a, b, th = float(g["alpha"]), float(g["beta"]), float(g["theta"])
    tol = float(g["leading_order_rel_tol"])
    u = np.array([math.cos(th), math.sin(th)])
    blocks = [np.array([[a], [0.0]]), (b * u)[:, None], (b * u)[:, None]]
    true_lead = 2 * b * b * math.sin(th) ** 2
    disc_lead = b * b * math.sin(th) ** 2
    # exact smaller eigenvalue of the 2x2 true Gram by the quadratic formula
    c, s = math.cos(th), math.sin(th)
    G = np.array([[a * a + 2 * b * b * c * c, 2 * b * b * s * c],
                  [2 * b * b * s * c, 2 * b * b * s * s]])
    tr, det = G[0, 0] + G[1, 1], G[0, 0] * G[1, 1] - G[0, 1] ** 2
    lam_min = det / (tr / 2 + math.sqrt(tr * tr / 4 - det))
    ex = exact.tail_sq(blocks, 1)
    assert math.isclose(ex, lam_min, rel_tol=1e-9)
    assert math.isclose(ex, true_lead, rel_tol=tol)
    st = incremental.IncrementalSVD(2, 1)
    st.append(blocks[0])
    st.append(blocks[1])
    step2 = st.discarded
    st.append(blocks[2])
    step3 = st.discarded - step2
    assert math.isclose(step2, disc_lead, rel_tol=tol)
    assert math.isclose(step3, disc_lead, rel_tol=tol)
    # the paper form S - s_1^2 cancels (S ~ 1, tail ~ 2e-8): agreement to
    # ~ 1e-16 * S / tail only
    assert math.isclose(st.tail_sq(), step2 + step3, rel_tol=1e-6)
    assert st.discarded >= ex * (1 - 1e-9)
    assert math.isclose(st.discarded, true_lead, rel_tol=tol)
    assert step3 < ex


# ------------------------------------------------------------ bounds (O3)
def test_bounds_are_upper_bounds_random():
    rng = np.random.default_rng(12)
    for _ in range(300):
        m = int(rng.integers(2, 8))
        blocks = [rng.standard_normal((m, int(rng.integers(1, 4)))) * rng.uniform(0.1, 2)
                  for _ in range(int(rng.integers(1, 5)))]
        r = int(rng.integers(1, m + 1))
        ex = exact.tail_sq(blocks, r)
        w, res, plug, en = bounds.all_bounds(blocks, r)
        assert math.isclose(en, exact.energy(blocks), rel_tol=1e-13)
        eps = 1e-10 * en
        assert w >= ex - eps and res >= ex - eps and plug >= ex - eps


def test_bounds_are_upper_bounds_ten_thousand_tiny():
    """10^4 tiny collections (m <= 6, up to four blocks of up to three
    columns), a quarter of them degenerate: a block repeated (nested
    ranges), a block scaled from another, a zero block, or blocks of rank
    one.  The Weyl, residual and plug-in values never fall below the exact
    Eckart-Young tail, and the energies agree."""
    rng = np.random.default_rng(2026)
    for i in range(10_000):
        m = int(rng.integers(2, 7))
        blocks = [rng.standard_normal((m, int(rng.integers(1, 4)))) * rng.uniform(0.1, 2)
                  for _ in range(int(rng.integers(1, 5)))]
        kind = i % 8
        if kind == 1 and len(blocks) > 1:
            blocks[-1] = blocks[0].copy()
        elif kind == 3 and len(blocks) > 1:
            blocks[-1] = blocks[0] * rng.uniform(-3, 3)
        elif kind == 5:
            blocks[int(rng.integers(len(blocks)))] = np.zeros((m, 2))
        elif kind == 7:
            blocks = [np.outer(rng.standard_normal(m), rng.standard_normal(b.shape[1]))
                      for b in blocks]
        r = int(rng.integers(1, m + 1))
        ex = exact.tail_sq(blocks, r)
        w, res, plug, en = bounds.all_bounds(blocks, r)
        assert math.isclose(en, exact.energy(blocks), rel_tol=1e-12, abs_tol=1e-300)
        tol = 1e-10 * max(en, 1e-300)
        assert w >= ex - tol and res >= ex - tol and plug >= ex - tol, (i, w, res, plug, ex)


def test_weyl_rank_one_example():
    """Appendix D, Example 1: shared left vector -> E_1 = 0 but the Weyl
    bound equals sum s_j^2 - max s_j^2."""
    rng = np.random.default_rng(13)
    u = _orth(rng, 6, 1)[:, 0]
    s = [3.0, 1.0, 2.0, 0.5]
    blocks = [np.outer(u, sj * _orth(rng, 4, 1)[:, 0]) for sj in s]
    assert exact.tail_sq(blocks, 1) < 1e-24
    assert math.isclose(bounds.weyl_bound_sq(blocks, 1),
                        sum(x * x for x in s) - max(s) ** 2, rel_tol=1e-12)


def test_residual_bound_exact_under_orthogonal_growth():
    """Proposition 1 (exactness): mutually orthogonal residual subspaces."""
    rng = np.random.default_rng(14)
    Q = _orth(rng, 16, 12)
    blocks = [Q[:, 4 * i:4 * i + 4] @ rng.standard_normal((4, 5)) for i in range(3)]
    for r in range(0, 13):
        res, _ = bounds.residual_bound_sq(blocks, r)
        assert math.isclose(res, exact.tail_sq(blocks, r), rel_tol=1e-10, abs_tol=1e-12)


def test_residual_bound_degenerate_under_nesting():
    """Proposition 1 (degeneracy): nested ranges give R_i = 0 for i >= 2 and
    the bound sum_{i>=2} ||A_i||^2 when r >= rank(A_1)."""
    rng = np.random.default_rng(15)
    Q = _orth(rng, 10, 4)
    A1 = Q @ rng.standard_normal((4, 6))
    A2 = Q[:, :3] @ rng.standard_normal((3, 5))
    A3 = Q[:, :2] @ rng.standard_normal((2, 2))
    res, mu = bounds.residual_bound_sq([A1, A2, A3], 4)
    assert math.isclose(res, float(np.sum(A2 ** 2) + np.sum(A3 ** 2)), rel_tol=1e-10)
    np.testing.assert_allclose(mu[:4], np.linalg.svd(A1, compute_uv=False)[:4], rtol=1e-10)
    assert np.all(mu[4:] < 1e-12)


def test_residual_mu_is_union_and_monotone():
    """Thm. 2: mu are the singular values of [R_1 ... R_K] (computed here
    directly from the concatenated residual matrix), and mu_j never
    decreases as blocks are added."""
    rng = np.random.default_rng(16)
    blocks = [rng.standard_normal((9, w)) for w in (3, 2, 4, 3)]
    st = bounds.ResidualState(9)
    Rs, prev = [], None
    for b in blocks:
        Rs.append(st.residual(b))
        st.append(b)
        direct = np.linalg.svd(np.hstack(Rs), compute_uv=False)
        np.testing.assert_allclose(st.mu[:len(direct)], direct, atol=1e-12)
        if prev is not None:
            n = len(prev)
            assert np.all(st.mu[:n] >= prev - 1e-12)
        prev = st.mu.copy()


def test_thm2_individual_inequality_fails_but_cor1_holds():
    """Thm. 2 claims sigma_j(M) >= mu_j for every j; its proof drops the
    cross terms Q B R^T, which vanish only when the row spaces are
    orthogonal.  Counterexample: A_1 = e_1, A_2 = e_1 + e_2 gives mu = (1, 1)
    but sigma = (golden ratio, 1/golden ratio).  The summed form (Cor. 1)
    still holds: with W the top-r eigenvectors of [R_1..R_K][R_1..R_K]^T
    chosen inside the residual ranges, ||W^T M||^2 >= sum_{j<=r} mu_j^2."""
    A1 = np.array([[1.0], [0.0]])
    A2 = np.array([[1.0], [1.0]])
    res1, mu = bounds.residual_bound_sq([A1, A2], 1)
    sig = exact.singular_values([A1, A2])
    phi = (1 + math.sqrt(5)) / 2
    np.testing.assert_allclose(mu, [1.0, 1.0], atol=1e-14)
    np.testing.assert_allclose(sig, [phi, 1 / phi], rtol=1e-13)
    assert sig[1] < mu[1]
    for r in (0, 1, 2):
        b, _ = bounds.residual_bound_sq([A1, A2], r)
        assert b >= exact.tail_sq([A1, A2], r) - 1e-14
