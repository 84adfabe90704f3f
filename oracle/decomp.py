"""Final decomposition of a cluster (FP64).

Test infrastructure (see the package docstring).

The Problem Formulation section keeps, for each cluster C_c with blocks
A_i (m x n_i) and rank r_c, the two factors of a rank-r_c truncated SVD
M_c ~ U_c S_c V_c^T: U~_c = U_c S_c (m x r_c) and V_c (N_c x r_c), split
row-wise into the coefficient blocks V_{c,i} (n_i x r_c) of the blocks, so
that A^_i = U~_c V_{c,i}^T, stored in r_c (m + N_c) numbers.  The
evaluation section measures the relative Frobenius error
||X - X^||_F / ||X||_F of the concatenation X of a cluster's blocks.

Reading (for a basis that is not an exact SVD, e.g. the incremental
estimator's U and sigma~): V_{c,i} = A_i^T U_c S_c^-1 (zero columns where a
singular value is zero), the coefficients that make A^_i = U_c U_c^T A_i, the
orthogonal projection of A_i on span(U_c) -- the best reconstruction of A_i
from that basis; with U_c, S_c the exact truncated SVD this is exactly the
SVD's V_c.

* ``decompose(U, s, blocks)`` -- (U~, [V_i], resid_sq, energy): U~ = U diag(s),
  V_i as above, resid_sq[i] = ||A_i - A^_i||_F^2 from the explicit residual,
  energy[i] = ||A_i||_F^2.
* ``rel_error(resid_sq, energy)`` -- sqrt(sum resid_sq / sum energy).
* ``memory(m, r, widths)`` -- r (m + sum n_i).
"""
from __future__ import annotations

import numpy as np


def _f64(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().double().numpy()
    return np.asarray(a, dtype=np.float64)


def decompose(U, s, blocks):
    U = _f64(U)
    s = _f64(s).ravel()
    inv = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
    Ut = U * s[None, :]
    V, res, en = [], [], []
    for b in blocks:
        A = _f64(b)
        V.append((A.T @ U) * inv[None, :])
        R = A - U @ (U.T @ A)
        res.append(float(np.sum(R * R)))
        en.append(float(np.sum(A * A)))
    return Ut, V, np.array(res), np.array(en)


def rel_error(resid_sq, energy):
    tot = float(np.sum(energy))
    return float(np.sqrt(np.sum(resid_sq) / tot)) if tot > 0 else 0.0


def memory(m, r, widths):
    return int(r * (m + sum(int(k) for k in widths)))
