"""Exact quantities of the concatenation M = [A_1 ... A_K] (FP64).

Test infrastructure (see the package docstring).

* ``singular_values(blocks)`` -- sigma_1 >= sigma_2 >= ... of M.  The SVD is a
  library primitive (LAPACK through numpy); it serves as one step.
* ``tail_sq(blocks, r)`` -- E_r^2(M) = sum_{j>r} sigma_j^2(M), the optimal
  rank-r Frobenius error (Thm. 4, Eckart-Young-Mirsky, Appendix A; the cluster
  loss L_c of the Problem Formulation section).
* ``rel_error(blocks, r)`` -- E_r(M) / ||M||_F, the relative reconstruction
  error of the evaluation section.
* ``tail_grad(blocks, r)`` -- d E_r^2 / d A_j = 2 (I - U_r U_r^T) A_j with U_r the
  exact top-r left singular vectors (valid when sigma_r > sigma_{r+1}).
"""
from __future__ import annotations

import numpy as np


def _f64(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().double().numpy()
    return np.asarray(a, dtype=np.float64)


def concat(blocks):
    """M = [A_1 ... A_K] (horizontal concatenation, Problem Formulation)."""
    return np.hstack([_f64(b) for b in blocks])


def singular_values(blocks):
    """All min(m, N) singular values of M, non-increasing."""
    return np.linalg.svd(concat(blocks), compute_uv=False)


def energy(blocks):
    """||M||_F^2 = sum_i ||A_i||_F^2 (Frobenius norm of a concatenation)."""
    return float(sum(np.sum(_f64(b) ** 2) for b in blocks))


def tail_sq(blocks, r):
    """E_r^2(M) = sum_{j>r} sigma_j^2(M) (Thm. 4)."""
    s = singular_values(blocks)
    return float(np.sum(s[r:] ** 2))


def rel_error(blocks, r):
    """E_r(M) / ||M||_F (relative Frobenius reconstruction error)."""
    return float(np.sqrt(tail_sq(blocks, r) / energy(blocks)))


def top_left_basis(blocks, r):
    """Exact top-r left singular vectors U_r (m x r) of M."""
    u, s, _ = np.linalg.svd(concat(blocks), full_matrices=False)
    return u[:, :r], s


def tail_grad(blocks, r):
    """Gradient of E_r^2(M) with respect to each block: 2 (I - U_r U_r^T) A_j.

    E_r^2(M) = ||(I - U_r U_r^T) M||_F^2 at the optimal U_r; the dependence of
    U_r on M contributes nothing at the optimum (envelope argument), which
    needs sigma_r > sigma_{r+1}."""
    u, _ = top_left_basis(blocks, r)
    out = []
    for b in blocks:
        a = _f64(b)
        out.append(2.0 * (a - u @ (u.T @ a)))
    return out
