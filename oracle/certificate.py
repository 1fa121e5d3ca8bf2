"""Oracle: the FP64 certificate of a converged subspace and its smoothed form.

TEST INFRASTRUCTURE.

No counterpart in the paper: these are the checks a caller runs where no
reference solution exists.

Certificate.  The Rayleigh-Ritz step of Sec. VI (Eq. 7) on the columns of X:
with S = <X|X> and h = <X|H X> (grid integrals, weight dV), the generalized
symmetric problem h y_k = eps_k S y_k, normalised y_k^T S y_k = 1, gives the
Ritz pairs (eps_k, x_k = X y_k), <x_k|x_k> = 1, and their residual norms
r_k = ||H x_k - eps_k x_k||.  For a symmetric H an eigenvalue lies within
r_k of eps_k (and within r_k^2 / gap_k when gap_k separates eps_k from the
rest of the spectrum).

Smoothing.  Before the certificate, n damped Richardson steps on each column
with its own step length,
    x_k <- x_k - (H x_k - theta_k x_k) / (lam - theta_k),
theta_k the column's current eigenvalue estimate and lam >= the largest
eigenvalue of H.  Along an eigenvector of H with eigenvalue mu the step
multiplies the component by 1 - (mu - theta_k) / (lam - theta_k): 1 at
mu = theta_k, 0 at mu = lam.  It removes the high-energy part of rounding
noise in the orbitals.

Largest eigenvalue of H: a library Lanczos solve (ARPACK through scipy) on
the oracle's H.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse.linalg


def ritz_certificate(apply_h, X: np.ndarray, dV: float):
    """FP64 Rayleigh-Ritz of span(X) and the residual norms of the Ritz
    pairs.  Returns (eps ascending, res, Ritz vectors)."""
    HX = apply_h(X)
    S = dV * (X.T @ X)
    h = dV * (X.T @ HX)
    h = 0.5 * (h + h.T)
    eps, Y = scipy.linalg.eigh(h, 0.5 * (S + S.T))
    Xr, HXr = X @ Y, HX @ Y
    res = np.sqrt(dV * ((HXr - Xr * eps) ** 2).sum(axis=0))
    return eps, res, Xr


def richardson_smooth(apply_h, X: np.ndarray, theta: np.ndarray, lam: float, n: int) -> np.ndarray:
    """n damped Richardson steps per column (step length 1/(lam - theta_k))."""
    X = np.array(X, dtype=np.float64, copy=True)
    theta = np.asarray(theta, dtype=np.float64)
    for _ in range(n):
        X = X - (apply_h(X) - X * theta) / (lam - theta)
    return X


def smoothed_certificate(apply_h, X: np.ndarray, theta: np.ndarray, lam: float, n: int, dV: float):
    """ritz_certificate after richardson_smooth."""
    return ritz_certificate(apply_h, richardson_smooth(apply_h, X, theta, lam, n), dV)


def largest_eigenvalue(apply_h, npts: int) -> float:
    """Largest eigenvalue of H (Lanczos, tolerance 1e-12)."""
    op = scipy.sparse.linalg.LinearOperator((npts, npts), matvec=lambda v: apply_h(v.reshape(-1, 1)).ravel(),
                                            dtype=np.float64)
    w = scipy.sparse.linalg.eigsh(op, k=1, which="LA", tol=1e-12, return_eigenvectors=False,
                                  v0=np.ones(npts))
    return float(w[0])
