"""Pins of the final per-cluster decomposition (oracle/decomp.py) against
facts that do not come from its own code: the Eckart-Young-Mirsky theorem
(Thm. 4, Appendix A), the SVD's orthonormal right factor, Pythagoras, and
exact reconstruction of blocks inside the basis."""
import numpy as np

from oracle import decomp, exact


def _blocks(rng, m, widths, rank):
    basis = np.linalg.qr(rng.standard_normal((m, rank)))[0]
    out = []
    for k in widths:
        out.append(basis @ (rng.standard_normal((rank, k)) * np.linspace(2.0, 0.1, rank)[:, None])
                   + 1e-2 * rng.standard_normal((m, k)))
    return out


def _svd(blocks, r):
    M = np.hstack(blocks)
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    return U[:, :r], s[:r], Vt[:r].T


def test_exact_svd_gives_the_eckart_young_tail_and_the_svd_factors():
    rng = np.random.default_rng(0)
    blocks = _blocks(rng, 120, [7, 13, 20, 5], rank=12)
    for r in (1, 6, 12, 30):
        U, s, V = _svd(blocks, r)
        Ut, Vs, res, en = decomp.decompose(U, s, blocks)
        # total residual = sum of the discarded squared singular values (Thm. 4)
        assert np.isclose(res.sum(), exact.tail_sq(blocks, r), rtol=1e-10, atol=1e-12)
        assert np.isclose(decomp.rel_error(res, en), exact.rel_error(blocks, r), rtol=1e-10)
        # the stacked coefficient blocks are the SVD's right factor: orthonormal columns
        Vc = np.vstack(Vs)
        assert np.allclose(Vc, V, atol=1e-9)
        assert np.allclose(Vc.T @ Vc, np.eye(r), atol=1e-9)
        assert np.allclose(Ut, U * s[None, :])
        assert decomp.memory(120, r, [b.shape[1] for b in blocks]) == r * (120 + 45)


def test_pythagoras_and_exact_blocks_inside_the_basis():
    rng = np.random.default_rng(1)
    m, r = 64, 8
    U = np.linalg.qr(rng.standard_normal((m, r)))[0]
    s = np.linspace(3.0, 0.5, r)
    inside = [U @ rng.standard_normal((r, k)) for k in (3, 9)]
    outside = [rng.standard_normal((m, k)) for k in (4, 6)]
    Ut, Vs, res, en = decomp.decompose(U, s, inside + outside)
    for i, A in enumerate(inside + outside):
        Ahat = Ut @ Vs[i].T
        assert np.isclose(np.sum(Ahat * Ahat) + res[i], en[i], rtol=1e-12)  # Pythagoras
        assert np.isclose(res[i], np.sum((A - Ahat) ** 2), rtol=1e-10, atol=1e-12)
    assert res[0] < 1e-20 * en[0] and res[1] < 1e-20 * en[1]  # A^ = A inside span(U)
    assert np.all(res[2:] > 0.5 * en[2:] * (1 - r / m) * 0.5)


def test_zero_singular_values_give_zero_coefficients():
    rng = np.random.default_rng(2)
    U = np.linalg.qr(rng.standard_normal((30, 4)))[0]
    s = np.array([2.0, 1.0, 0.0, 0.0])
    _, Vs, res, en = decomp.decompose(U, s, [rng.standard_normal((30, 5))])
    assert np.all(Vs[0][:, 2:] == 0.0) and np.all(np.isfinite(Vs[0]))


def _decomp_pins_hold(fn):
    """The pins above, run against a replacement of decomp.decompose."""
    orig = decomp.decompose
    decomp.decompose = fn
    try:
        for test in (test_exact_svd_gives_the_eckart_young_tail_and_the_svd_factors,
                     test_pythagoras_and_exact_blocks_inside_the_basis):
            try:
                test()
            except AssertionError:
                return False
        return True
    finally:
        decomp.decompose = orig


def test_planted_mistakes_are_caught():
    orig = decomp.decompose

    def no_inverse_scaling(U, s, blocks):  # V_i = A_i^T U (S^-1 dropped)
        Ut, V, res, en = orig(U, s, blocks)
        return Ut, [v * np.asarray(s)[None, :] for v in V], res, en

    def residual_from_wrong_side(U, s, blocks):  # ||A - U U^T A|| replaced by ||A U||-based
        Ut, V, res, en = orig(U, s, blocks)
        return Ut, V, np.array([max(e - float(np.sum((np.asarray(b) @ np.ones((np.asarray(b).shape[1], 1))) ** 2)), 0.0)
                                 for b, e in zip(blocks, en)]), en

    def unscaled_left_factor(U, s, blocks):  # U~ = U instead of U diag(s)
        Ut, V, res, en = orig(U, s, blocks)
        return np.asarray(U, dtype=np.float64), V, res, en

    assert _decomp_pins_hold(orig)
    for bad in (no_inverse_scaling, residual_from_wrong_side, unscaled_left_factor):
        assert not _decomp_pins_hold(bad), bad.__name__
