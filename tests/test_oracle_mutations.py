"""Plant plausible mistakes in the oracle (on the CPU) and check that the
pins catch each one: a flipped sign, a dropped term, a transposed operand,
an off-by-one truncation.  This shows the pins constrain the oracle rather
than restate it.
"""
import inspect
import textwrap

import numpy as np
import pytest

from oracle import bounds, exact, incremental


def _prescribed(rng, m, n, s):
    def orth(a, b):
        q, rr = np.linalg.qr(rng.standard_normal((a, b)))
        return q * np.sign(np.diag(rr))
    k = len(s)
    return orth(m, k) @ np.diag(s) @ orth(n, k).T


def _pins_hold(step_fn):
    """A compact subset of the incremental pins, run with a replaced step."""
    orig = incremental.IncrementalSVD.step
    incremental.IncrementalSVD.step = step_fn
    try:
        rng = np.random.default_rng(0)
        s = np.array([3.0, 2.0, 1.0, 0.5, 0.1])
        M = _prescribed(rng, 12, 15, s)
        blocks = [M[:, :4], M[:, 4:9], M[:, 9:]]
        st, steps = incremental.run(blocks, r=6)
        if not np.allclose(st.s[:5], s, rtol=1e-9):
            return False
        rng = np.random.default_rng(1)
        for _ in range(40):
            m = int(rng.integers(3, 7))
            bl = [rng.standard_normal((m, int(rng.integers(1, 4)))) for _ in range(3)]
            r = int(rng.integers(1, m))
            st, steps = incremental.run(bl, r)
            for t, (_, paper, disc) in enumerate(steps):
                ex = exact.tail_sq(bl[:t + 1], r)
                if paper < ex - 1e-9 or abs(paper - disc) > 1e-8 * (1 + paper):
                    return False
        return True
    except (ValueError, IndexError, np.linalg.LinAlgError):
        return False
    finally:
        incremental.IncrementalSVD.step = orig


def _mutant(old, new):
    src = textwrap.dedent(inspect.getsource(incremental.IncrementalSVD.step))
    assert old in src, old
    src = src.replace(old, new, 1)
    ns = dict(incremental.__dict__)
    exec(compile(src, "<mutant>", "exec"), ns)
    return ns["step"]


def test_unmutated_passes():
    assert _pins_hold(incremental.IncrementalSVD.step)


@pytest.mark.parametrize("old,new", [
    ("R = A - Q @ Y", "R = A + Q @ Y"),                               # sign
    ("K[rt:, rt:] = B", "K[rt:, rt:] = B.T if B.shape[0] == B.shape[1] else B[:, ::-1]"),  # transposed
    ("K[:rt, :rt] = np.diag(s)", "K[:rt, :rt] = np.diag(s) * 0"),      # dropped state
    ("K[:rt, rt:] = Y", "K[:rt, rt:] = 0 * Y"),                        # dropped projection
    ("r_new = min(self.r, rt + kp)", "r_new = min(self.r + 1, rt + kp)"),  # off by one
    ("energy = self.energy + float(np.sum(A * A))", "energy = self.energy"),
    ("discarded = self.discarded + float(np.sum(sig[r_new:] ** 2))",
     "discarded = self.discarded + float(np.sum(sig[r_new + 1:] ** 2))"),
])
def test_mutants_are_caught(old, new):
    assert not _pins_hold(_mutant(old, new))


def test_bound_mutant_is_caught():
    """Residual spectrum taken from the blocks instead of their residuals:
    still an upper bound (any union of block spectra is one), but the
    nested-range pin of Proposition 1 catches it."""
    orig = bounds.ResidualState.step

    def mutant(self, A):
        Q, mu, energy = orig(self, A)
        sv = np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False)
        return Q, np.sort(np.concatenate([self.mu, sv]))[::-1], energy

    rng = np.random.default_rng(2)
    q, _ = np.linalg.qr(rng.standard_normal((10, 4)))
    A1 = q @ rng.standard_normal((4, 6))
    A2 = q[:, :3] @ rng.standard_normal((3, 5))
    want = float(np.sum(A2 ** 2))
    got, _ = bounds.residual_bound_sq([A1, A2], 4)
    assert abs(got - want) < 1e-9 * want
    bounds.ResidualState.step = mutant
    try:
        got, _ = bounds.residual_bound_sq([A1, A2], 4)
        assert abs(got - want) > 1e-3 * want
    finally:
        bounds.ResidualState.step = orig
