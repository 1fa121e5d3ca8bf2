"""Oracle: orthogonalisation and subspace diagonalisation (Sec. VI).

TEST INFRASTRUCTURE.  Orbitals are the columns of Psi[np, nst]; the inner
product is <a|b> = dV * sum_p a(p) b(p).  Matrix products use numpy's
matmul as a library primitive; the Cholesky factorisation, the triangular
inverse and the symmetric eigensolver are the textbook loops of
``ora_core.c``.
"""
from __future__ import annotations

import numpy as np

from . import _native


class NotPositiveDefinite(ArithmeticError):
    pass


def overlap(X: np.ndarray, Y: np.ndarray, dV: float) -> np.ndarray:
    """S_jk = <x_j | y_k> = dV * sum_p x_j(p) y_k(p), Eq. (5)."""
    return dV * (X.T @ Y)


def cholesky_upper(S: np.ndarray) -> np.ndarray:
    """S = U^T U with U upper triangular (the paper's S = U^dagger U)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    n = S.shape[0]
    U = np.empty_like(S)
    rc = _native.lib().ora_cholesky(n, _native.ptr(S), _native.ptr(U))
    if rc != 0:
        raise NotPositiveDefinite(f"pivot {rc - 1} not positive")
    return U


def tri_inv_upper(U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    X = np.empty_like(U)
    if _native.lib().ora_tri_inv_upper(U.shape[0], _native.ptr(U), _native.ptr(X)) != 0:
        raise ZeroDivisionError("singular triangular matrix")
    return X


def jacobi_eigh(A: np.ndarray, max_sweeps: int = 60, tol: float = 1e-15):
    """Eigenvalues (ascending) and eigenvectors (columns) of a real symmetric
    matrix by cyclic Jacobi rotations."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    n = A.shape[0]
    w = np.empty(n)
    V = np.empty((n, n))
    sweeps = _native.lib().ora_jacobi_eig(n, _native.ptr(A), _native.ptr(w), _native.ptr(V), max_sweeps, tol)
    if sweeps < 0:
        raise ArithmeticError("Jacobi did not converge")
    return w, V


def orthonormalize(Psi: np.ndarray, dV: float):
    """Sec. VI: S = <Psi|Psi>, S = U^T U, and the new orbitals from
    Eq. (6) read as phi_j = sum_k U_kj phibar_k, i.e. Psi = Psibar U, so
    Psibar = Psi U^{-1} (the reading that makes <Psibar|Psibar> = I).
    Returns (Psibar, U^{-1})."""
    S = overlap(Psi, Psi, dV)
    U = cholesky_upper(S)
    Ui = tri_inv_upper(U)
    return Psi @ Ui, Ui


def subspace_diag(apply_h, Psi: np.ndarray, dV: float, HPsi: np.ndarray | None = None):
    """Sec. VI, Eqs. (7)-(8): h_jk = <phi_j|H|phi_k> (symmetrised), h xi =
    xi diag(eps) with eps ascending, phibar_k = sum_j xi_jk phi_j.
    Returns (eps, Psi xi, H Psi xi, xi)."""
    if HPsi is None:
        HPsi = apply_h(Psi)
    h = overlap(Psi, HPsi, dV)
    h = 0.5 * (h + h.T)
    eps, xi = jacobi_eigh(h)
    return eps, Psi @ xi, HPsi @ xi, xi
