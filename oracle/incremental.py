"""Incremental truncated SVD of a concatenation, one block at a time (FP64).

Test infrastructure (see the package docstring).

Follows Lemma 1 (exact incremental Gram factorisation, Appendix B), Cor. 3
(truncated top-r approximation, Appendix B) and Cor. 2 (plug-in estimator,
Section 3.3), in the paper's notation:

    state after t blocks:  M_t M_t^T ~ Q_t S_t Q_t^T,  S_t = diag(s_t^2)
    append A = A_{t+1} (m x k):
        Y   = Q_t^T A                        (projection)
        R   = A - Q_t Y                      (residual)
        R   = Q_res B                        (thin QR of the residual)
        S_{t+1} = [[S_t + Y Y^T, Y B^T], [B Y^T, B B^T]]
    Because S_t is kept diagonal, S_{t+1} = K K^T with the core
        K = [[diag(s_t), Y], [0, B]],
    so the eigenpairs of S_{t+1} are the squared singular values and left
    singular vectors of K.  Truncation keeps the top r of them (Cor. 3):
        Q_{t+1} <- [Q_t Q_res] W_r,   s_{t+1} <- sigma_1..r(K).
    Plug-in estimate (Cor. 2):  E~_r^2 = sum_i ||A_i||_F^2 - sum_{j<=r} s_j^2.

Readings (paper silent or ambiguous):
* The residual is re-orthogonalised once against Q_t (classical Gram-Schmidt
  twice); Y absorbs the correction.  In exact arithmetic this changes nothing.
* The thin QR keeps k' = min(k, m - r_t) columns and applies no rank
  threshold: Q_res is taken from a Householder QR of [Q_t R], which makes it
  orthonormal and orthogonal to Q_t even when R is rank deficient, and
  B = Q_res^T R.  When R has full column rank this is the thin QR of R.
* The retained rank is r_{t+1} = min(r, r_t + k'), i.e. min(r, sum k, m);
  zero singular values are kept.
* The tail is reported in two forms that agree in exact arithmetic:
  the paper's  S - sum s_j^2  (clamped at 0), and the accumulated discard
  sum_t sum_{j>r} sigma_j(K_t)^2, which follows from tr(S_{t+1}) =
  tr(S_t) + ||A||_F^2 (Lemma 1).
* The merge certificate accepts when E~^2 <= eps^2 * ||M_{C u j}||_F^2
  (inclusive, relative to the post-merge norm; Alg. 3 step 3(e)).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .exact import _f64


@dataclass
class IncrementalSVD:
    """Rank-r incremental state (Q_t, s_t, energy, discarded)."""
    m: int
    r: int
    Q: np.ndarray = None          # m x r_t, orthonormal columns
    s: np.ndarray = None          # r_t retained singular values, non-increasing
    energy: float = 0.0           # sum_i ||A_i||_F^2
    discarded: float = 0.0        # accumulated discarded sigma^2
    n_blocks: int = 0
    history: list = field(default_factory=list)

    def __post_init__(self):
        if self.Q is None:
            self.Q = np.zeros((self.m, 0))
            self.s = np.zeros(0)

    # -- one step of Lemma 1 + Cor. 3 ---------------------------------------
    def step(self, A):
        """Return the would-be next state and the step's diagnostics without
        modifying ``self``."""
        A = _f64(A)
        m, k = A.shape
        assert m == self.m, "row count mismatch"
        Q, s = self.Q, self.s
        rt = Q.shape[1]
        # projection and residual (Lemma 1), one re-orthogonalisation pass
        Y = Q.T @ A
        R = A - Q @ Y
        Y2 = Q.T @ R
        R = R - Q @ Y2
        Y = Y + Y2
        # thin QR of the residual, Q_res orthogonal to Q_t
        kp = min(k, m - rt)
        if kp > 0:
            qfull, _ = np.linalg.qr(np.hstack([Q, R]))
            Qres = qfull[:, rt:rt + kp]
            B = Qres.T @ R
        else:
            Qres = np.zeros((m, 0))
            B = np.zeros((0, k))
        # core K = [[diag(s), Y], [0, B]]; K K^T = S_{t+1}
        K = np.zeros((rt + kp, rt + k))
        K[:rt, :rt] = np.diag(s)
        K[:rt, rt:] = Y
        K[rt:, rt:] = B
        W, sig, _ = np.linalg.svd(K, full_matrices=False)
        # truncation (Cor. 3)
        r_new = min(self.r, rt + kp)
        Qnew = np.hstack([Q, Qres]) @ W[:, :r_new]
        s_new = sig[:r_new].copy()
        energy = self.energy + float(np.sum(A * A))
        discarded = self.discarded + float(np.sum(sig[r_new:] ** 2))
        diag = dict(Y=Y, R=R, Qres=Qres, B=B, K=K, sigma_core=sig, W=W, kp=kp)
        return (Qnew, s_new, energy, discarded), diag

    def commit(self, nxt):
        self.Q, self.s, self.energy, self.discarded = nxt
        self.n_blocks += 1

    def append(self, A):
        nxt, diag = self.step(A)
        self.commit(nxt)
        self.history.append(self.tail_sq())
        return diag

    # -- plug-in estimate (Cor. 2) ------------------------------------------
    def tail_sq(self):
        """Paper form: sum ||A_i||^2 - sum_{j<=r} s_j^2, clamped at zero."""
        return max(0.0, self.energy - float(np.sum(self.s ** 2)))

    def tail_sq_discard(self):
        """Accumulated-discard form of the same quantity."""
        return self.discarded

    def rel_tail(self):
        return float(np.sqrt(self.tail_sq() / self.energy)) if self.energy > 0 else 0.0

    def evaluate(self, A, eps):
        """One merge evaluation: tentative append of A, returning
        (sigma~ (r values), E~^2, accept flag, next state)."""
        nxt, _ = self.step(A)
        _, s_new, energy, _ = nxt
        tail = max(0.0, energy - float(np.sum(s_new ** 2)))
        accept = tail <= eps * eps * energy
        return s_new, tail, bool(accept), nxt

    def copy(self):
        c = IncrementalSVD(self.m, self.r, self.Q.copy(), self.s.copy(),
                           self.energy, self.discarded, self.n_blocks)
        return c


def run(blocks, r):
    """Sequential incremental SVD over ``blocks`` in order; returns the state
    and per-step (sigma~, tail paper form, tail discard form)."""
    m = int(blocks[0].shape[0])
    st = IncrementalSVD(m, r)
    steps = []
    for b in blocks:
        st.append(b)
        steps.append((st.s.copy(), st.tail_sq(), st.tail_sq_discard()))
    return st, steps
