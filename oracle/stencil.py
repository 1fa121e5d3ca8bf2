"""Oracle: finite-difference weights of the kinetic-energy stencil (Sec. V.A).

TEST INFRASTRUCTURE.  The paper's Laplacian is a star stencil of 25 points
in 3D, i.e. 8 neighbours per axis, half-width m = 4.  The 1-D central
second-derivative weights c_j (j = -m..m) are fixed by Taylor expansion:
requiring sum_j c_j f(x + j h) = h^2 f''(x) for every polynomial of degree
<= 2m gives the Vandermonde system  sum_j c_j j^k = 2 delta_{k,2},
k = 0..2m, solved here in exact rational arithmetic.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def fd_weights_exact(m: int) -> list[Fraction]:
    """Exact weights [c_0, c_1, ..., c_m] (c_{-j} = c_j) of the 2m+1 point
    central second derivative."""
    js = list(range(-m, m + 1))
    n = len(js)
    A = [[Fraction(j) ** k for j in js] for k in range(n)]
    b = [Fraction(2) if k == 2 else Fraction(0) for k in range(n)]
    # Gauss-Jordan elimination with exact fractions
    M = [row[:] + [b[k]] for k, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [v / pv for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * c for a, c in zip(M[r], M[col])]
    c = [M[r][n] for r in range(n)]
    return [c[m + j] for j in range(m + 1)]


def fd_weights(m: int = 4) -> np.ndarray:
    """FP64 weights [c_0..c_m]."""
    return np.array([float(x) for x in fd_weights_exact(m)])
