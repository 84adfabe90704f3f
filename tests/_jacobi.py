"""Independent tiny reference: cyclic two-sided Jacobi eigenvalues.

A textbook algorithm written with plain Python loops, used only to pin the
oracle (which calls LAPACK) on tiny inputs.  Not for sizes above ~16.
"""
import math

import numpy as np


def sym_eigvals(a, sweeps=60, tol=1e-15):
    a = [list(map(float, row)) for row in np.asarray(a, dtype=np.float64)]
    n = len(a)
    for _ in range(sweeps):
        off = sum(a[i][j] ** 2 for i in range(n) for j in range(n) if i != j)
        scale = sum(a[i][i] ** 2 for i in range(n)) + off
        if off <= tol * tol * max(scale, 1e-300):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if a[p][q] == 0.0:
                    continue
                theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q])
                t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                for k in range(n):
                    akp, akq = a[k][p], a[k][q]
                    a[k][p] = c * akp - s * akq
                    a[k][q] = s * akp + c * akq
                for k in range(n):
                    apk, aqk = a[p][k], a[q][k]
                    a[p][k] = c * apk - s * aqk
                    a[q][k] = s * apk + c * aqk
    return sorted((a[i][i] for i in range(n)), reverse=True)


def singular_values(m):
    """Singular values of a small matrix via Jacobi on the smaller Gram."""
    m = np.asarray(m, dtype=np.float64)
    g = m @ m.T if m.shape[0] <= m.shape[1] else m.T @ m
    ev = sym_eigvals(g)
    return [math.sqrt(max(e, 0.0)) for e in ev]
