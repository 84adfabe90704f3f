"""Certified upper bounds on E_r^2 of a concatenation (FP64).

Test infrastructure (see the package docstring).

* Thm. 1 (Weyl-type bound, Section 3.1):
      E_r^2(M) <= sum_j ||A_j||_F^2 - max_j sum_{i<=r} sigma_i^2(A_j),
  which becomes sum_j ||A_j||^2 - max_j ||A_j||^2 when r >= rank(A_j).
* Thm. 2 / Cor. 1 (residual bound, Section 3.2): with Q_{i-1} an orthonormal
  basis of range(M_{i-1}) and R_i = (I - Q_{i-1} Q_{i-1}^T) A_i, the singular
  values mu of [R_1 ... R_K] are the multiset union of the singular values of
  the R_i (proof of Thm. 2, step 4), and
      E_r^2(M) <= sum_i ||A_i||_F^2 - sum_{j<=r} mu_j^2.

Readings:
* Q_{i-1} spans all of range(M_{i-1}) (Thm. 2's hypothesis).  Numerical rank
  uses the tolerance tol = 1e-12 * ||M_{i}||_F on the residual's singular
  values; directions below it are treated as already spanned.
* The residual is formed with one re-orthogonalisation pass.
* Bounds are clamped at zero.
"""
from __future__ import annotations

import numpy as np

from .exact import _f64


def top_r_energy(A, r):
    """sum_{i<=r} sigma_i^2(A)."""
    s = np.linalg.svd(_f64(A), compute_uv=False)
    return float(np.sum(s[:r] ** 2))


def weyl_bound_sq(blocks, r):
    """Right-hand side of Thm. 1."""
    energies = [float(np.sum(_f64(b) ** 2)) for b in blocks]
    top = max(top_r_energy(b, r) for b in blocks)
    return max(0.0, sum(energies) - top)


class ResidualState:
    """Full-span basis Q, the residual singular-value multiset mu and the
    energy S, updated block by block (Thm. 2)."""

    def __init__(self, m, tol_rel=1e-12):
        self.m = m
        self.Q = np.zeros((m, 0))
        self.mu = np.zeros(0)
        self.energy = 0.0
        self.tol_rel = tol_rel

    def residual(self, A):
        A = _f64(A)
        R = A - self.Q @ (self.Q.T @ A)
        R = R - self.Q @ (self.Q.T @ R)
        return R

    def step(self, A):
        """Would-be (Q, mu, energy) after appending A."""
        A = _f64(A)
        R = self.residual(A)
        u, sv, _ = np.linalg.svd(R, full_matrices=False)
        energy = self.energy + float(np.sum(A * A))
        tol = self.tol_rel * np.sqrt(energy)
        keep = sv > tol
        Q = np.hstack([self.Q, u[:, keep]])
        mu = np.sort(np.concatenate([self.mu, sv]))[::-1]
        return Q, mu, energy

    def commit(self, nxt):
        self.Q, self.mu, self.energy = nxt

    def append(self, A):
        self.commit(self.step(A))

    def bound_sq(self, r, nxt=None):
        Q, mu, energy = nxt if nxt is not None else (self.Q, self.mu, self.energy)
        return max(0.0, energy - float(np.sum(mu[:r] ** 2)))


def residual_bound_sq(blocks, r):
    """Right-hand side of Cor. 1 for the blocks in the given order."""
    st = ResidualState(int(blocks[0].shape[0]))
    for b in blocks:
        st.append(b)
    return st.bound_sq(r), st.mu


def plugin_sq(blocks, r):
    """Plug-in estimate E~_r^2 of Cor. 2 for the blocks in the given order."""
    from .incremental import run
    st, _ = run(blocks, r)
    return st.tail_sq()


def all_bounds(blocks, r):
    """(weyl, residual, plug-in, energy) for the blocks in the given order."""
    res, _ = residual_bound_sq(blocks, r)
    energy = float(sum(np.sum(_f64(b) ** 2) for b in blocks))
    return weyl_bound_sq(blocks, r), res, plugin_sq(blocks, r), energy
