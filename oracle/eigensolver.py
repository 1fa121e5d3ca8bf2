"""Oracle: block eigensolver and the plain filter preconditioner.

TEST INFRASTRUCTURE.

The paper's eigensolver is RMM-DIIS with a Saad-type filter preconditioner
(Sec. III), working on blocks of orbitals (Sec. IV) and stopping a block
only when every state in it is converged (Sec. VIII).  The block
conjugate-gradient solver used here is LOBPCG (Knyazev 2001) applied block
by block, with the paper's orthogonalisation and subspace diagonalisation
(Sec. VI) after every sweep over the blocks.  One sweep, for each block X
(nb columns) of Psi:

  1. lambda_k = <x_k|H x_k> / <x_k|x_k>,  R = H X - X diag(lambda),
     ||r_k|| = sqrt(<r_k|r_k>); if every ||r_k|| <= tol the block is
     converged and left alone.
  2. W = K R (preconditioner).
  3. Y = [W, P] (P: the block's previous search directions, if any) is
     orthogonalised against Psi[:, :end of block] by classical Gram-Schmidt
     done twice, and each column is normalised.
  4. Rayleigh-Ritz on Z = [X, Y]: G = <Z|Z>, A = <Z|H Z> (symmetrised),
     G = U^T U; if the factorisation fails or a pivot falls below
     1e-12 of its diagonal, P is dropped (and the block skipped if W alone
     fails).  The nb lowest eigenpairs of U^-T A U^-1 give C = U^-1 Y_nb.
  5. X <- Z C,  P <- Z[:, nb:] C[nb:, :].
After the sweep: Psi <- orthonormalize(Psi) and Psi <- subspace_diag(Psi);
P is carried through the same two linear maps.

Filter preconditioner (Sec. III cites Saad et al. without giving its
form): a low-pass smoothing filter over the six face neighbours,
  (K r)(p) = alpha r(p) + (1-alpha)/6 * sum_{6 face neighbours n} r(n),
alpha = 1/2, r = 0 off the grid.

Kinetic preconditioner (used only to reach reference eigenvalues in fewer
sweeps): K r = a fixed number of CG iterations on (-1/2 Lap + sigma) x = r.
A preconditioner changes the path of the iteration, never the eigenvalues
it converges to.
"""
from __future__ import annotations

import numpy as np

from .hamiltonian import Hamiltonian
from .linalg import (NotPositiveDefinite, cholesky_upper, jacobi_eigh, orthonormalize, overlap,
                     subspace_diag, tri_inv_upper)

CHOL_REL = 1e-12


class FilterPreconditioner:
    def __init__(self, grid, alpha: float = 0.5):
        self.alpha = alpha
        self.nbr = grid.neighbours(1).reshape(grid.npts, 6)

    def __call__(self, R: np.ndarray) -> np.ndarray:
        acc = np.zeros_like(R)
        for t in range(6):
            q = self.nbr[:, t]
            ok = q >= 0
            acc[ok] += R[q[ok]]
        return self.alpha * R + (1.0 - self.alpha) / 6.0 * acc


class KineticPreconditioner:
    def __init__(self, grid, sigma: float = 1.0, n_iter: int = 10):
        self.grid, self.sigma, self.n_iter = grid, sigma, n_iter

    def __call__(self, R: np.ndarray) -> np.ndarray:
        from .precond import shifted_poisson_cg
        return shifted_poisson_cg(self.grid, R, self.sigma, self.n_iter)


def _chol_checked(G: np.ndarray) -> np.ndarray:
    U = cholesky_upper(G)
    if np.min(np.diag(U) ** 2 / np.diag(G)) <= CHOL_REL:
        raise NotPositiveDefinite("ill-conditioned Gram matrix")
    return U


def _normalise_columns(Y: np.ndarray, dV: float) -> np.ndarray:
    n = np.sqrt(dV * np.sum(Y * Y, axis=0))
    n[n == 0] = 1.0
    return Y / n


class BlockCG:
    """LOBPCG swept block by block over the state set (see module doc)."""

    def __init__(self, ham: Hamiltonian, Psi0: np.ndarray, nb: int, precond=None, tol: float = 1e-9):
        self.ham = ham
        self.dV = ham.grid.dV
        self.nb = nb
        self.tol = tol
        self.precond = precond if precond is not None else FilterPreconditioner(ham.grid)
        nst = Psi0.shape[1]
        assert nst % nb == 0
        Psi, _ = orthonormalize(np.array(Psi0, dtype=np.float64), self.dV)
        self.eps, self.Psi, self.HPsi, _ = subspace_diag(ham.apply, Psi, self.dV)
        self.P = np.zeros_like(self.Psi)
        self.resnorm = np.full(nst, np.inf)
        self.iterations = 0

    def _block(self, b: int):
        nb, dV = self.nb, self.dV
        sl = slice(b * nb, (b + 1) * nb)
        X = self.Psi[:, sl]
        HX = self.HPsi[:, sl]
        lam = np.sum(X * HX, axis=0) / np.sum(X * X, axis=0)
        R = HX - X * lam
        res = np.sqrt(dV * np.sum(R * R, axis=0))
        self.resnorm[sl] = res
        if np.all(res <= self.tol):
            return
        W = self.precond(R)
        Q = self.Psi[:, :sl.stop]
        Pb = self.P[:, sl]
        use_p = bool(np.any(Pb != 0.0))
        Y = np.concatenate([W, Pb], axis=1) if use_p else W
        for _ in range(2):
            Y = Y - Q @ overlap(Q, Y, dV)
        Y = _normalise_columns(Y, dV)
        HY = self.ham.apply(Y)
        Z = np.concatenate([X, Y], axis=1)
        HZ = np.concatenate([HX, HY], axis=1)
        G = overlap(Z, Z, dV)
        A = overlap(Z, HZ, dV)
        G = 0.5 * (G + G.T)
        A = 0.5 * (A + A.T)
        for ncols in ((Z.shape[1], 2 * nb) if use_p else (2 * nb,)):
            try:
                U = _chol_checked(G[:ncols, :ncols])
                break
            except NotPositiveDefinite:
                U = None
        if U is None:
            return
        Ui = tri_inv_upper(U)
        At = Ui.T @ A[:ncols, :ncols] @ Ui
        At = 0.5 * (At + At.T)
        _, Yv = jacobi_eigh(At)
        C = Ui @ Yv[:, :nb]
        Zc = Z[:, :ncols]
        self.Psi[:, sl] = Zc @ C
        self.P[:, sl] = Zc[:, nb:] @ C[nb:, :]

    def step(self):
        """One sweep over all blocks, then orthonormalise + subspace
        diagonalisation.  Returns (eps, resnorm, n_converged)."""
        nblk = self.Psi.shape[1] // self.nb
        for b in range(nblk):
            self._block(b)
        self.Psi, Ui = orthonormalize(self.Psi, self.dV)
        self.P = self.P @ Ui
        self.eps, self.Psi, self.HPsi, xi = subspace_diag(self.ham.apply, self.Psi, self.dV)
        self.P = self.P @ xi
        self.iterations += 1
        return self.eps.copy(), self.resnorm.copy(), int(np.sum(self.resnorm <= self.tol))

    def solve(self, max_iter: int = 1000, judged: int | None = None, callback=None):
        judged = self.Psi.shape[1] if judged is None else judged
        for _ in range(max_iter):
            eps, res, nconv = self.step()
            if callback is not None:
                callback(self)
            if np.all(res[:judged] <= self.tol):
                break
        return self.eps[:judged].copy()
