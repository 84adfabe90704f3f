"""Randomized range-finder estimator of the rank-r tail (FP64).

Test infrastructure (see the package docstring).

The discussion section names a randomized SVD or range-finder as a possible
replacement of the incremental estimator, and notes that randomized
approximations do not by themselves give conservative bounds.  This module
states the variant the library implements, in steps:

1. sketch: Y = M Omega = sum_i A_i Omega_i, with Omega_i the k_i x l rows of
   a random test matrix (l = r + oversampling) that the caller draws;
2. q power iterations: Y <- M M^T Q with Q an orthonormal basis of range(Y)
   (re-orthonormalised before each product);
3. U_r = the top-r left singular vectors of the final Y;
4. the estimate is the explicit residual energy of that rank-r basis,
   E~_rand^2 = sum_i ||(I - U_r U_r^T) A_i||_F^2.

Step 4 makes the estimate a certificate: for any rank-r orthogonal
projector the residual is at least the optimal one (Thm. 4,
Eckart-Young-Mirsky), so E~_rand >= E_r(M) for every draw; the randomness
affects only how close it is.

Readings (the paper gives no algorithm):
* Omega is an input (Gaussian entries drawn by the caller), so the same
  draw can be given to the oracle and to the GPU.
* The basis of step 2 is the left singular vectors of Y (ordered), and of
  step 3 its first r: for rank(M) <= r the residual is zero, and with many
  power iterations U_r tends to the exact top-r basis.
"""
from __future__ import annotations

import numpy as np

from .exact import _f64


def sketch(blocks, omegas):
    """Y = sum_i A_i Omega_i (m x l)."""
    Y = None
    for a, o in zip(blocks, omegas):
        t = _f64(a) @ _f64(o)
        Y = t if Y is None else Y + t
    return Y


def left_basis(Y, r):
    """First r left singular vectors of Y (a library SVD as one step)."""
    u, _, _ = np.linalg.svd(Y, full_matrices=False)
    return u[:, :r]


def power_step(blocks, Y):
    """M M^T Q for Q the orthonormal left singular basis of Y."""
    Q = left_basis(Y, Y.shape[1])
    out = None
    for a in blocks:
        a = _f64(a)
        t = a @ (a.T @ Q)
        out = t if out is None else out + t
    return out


def basis(blocks, omegas, r, power_iters=1):
    Y = sketch(blocks, omegas)
    for _ in range(power_iters):
        Y = power_step(blocks, Y)
    return left_basis(Y, r)


def tail_sq(blocks, omegas, r, power_iters=1):
    """E~_rand^2 = sum_i ||(I - U_r U_r^T) A_i||_F^2 (step 4)."""
    U = basis(blocks, omegas, r, power_iters)
    t = 0.0
    for a in blocks:
        a = _f64(a)
        res = a - U @ (U.T @ a)
        t += float(np.sum(res * res))
    return t


def gaussian_omegas(widths, l, seed):
    """Test matrices for the given block widths (float32 values, so that the
    same numbers can be handed to the GPU)."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((k, l)).astype(np.float32) for k in widths]
