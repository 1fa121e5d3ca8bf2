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

    def set_potential(self, v: np.ndarray):
        """New local potential of the Hamiltonian (an SCF step): the subspace
        is rediagonalised with it and the search directions are dropped."""
        self.ham.V = np.ascontiguousarray(v, dtype=np.float64)
        self.eps, self.Psi, self.HPsi, _ = subspace_diag(self.ham.apply, self.Psi, self.dV)
        self.P[:] = 0.0

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


def diis_coefficients(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """The DIIS combination of RMM-DIIS (Kresse and Furthmueller 1996, after
    Wood and Zunger 1985): the coefficients alpha that minimise the norm of
    the combined residual sum_i alpha_i r_i relative to the norm of the
    combined vector sum_i alpha_i x_i, i.e. the eigenvector of the lowest
    eigenvalue of the generalized problem A alpha = mu B alpha with
    A_ij = <r_i|r_j>, B_ij = <x_i|x_j>; normalised so that <xbar|xbar> = 1 and
    signed so that sum_i alpha_i >= 0.  When the iterates are numerically
    dependent (a Cholesky pivot of B below 1e-12 of its diagonal) the latest
    iterate alone is kept."""
    try:
        U = _chol_checked(0.5 * (B + B.T))
    except NotPositiveDefinite:
        a = np.zeros(len(B))
        a[-1] = 1.0
        return a
    Ui = tri_inv_upper(U)
    C = Ui.T @ A @ Ui
    w, V = jacobi_eigh(0.5 * (C + C.T))
    a = Ui @ V[:, int(np.argmin(w))]
    return a if a.sum() >= 0 else -a


def rayleigh_step(xx, xp, pp, xhx, xhp, php) -> float:
    """The lambda that minimises the Rayleigh quotient of x + lambda p: the
    lower eigenvector (c0, c1) of the 2x2 pencil
    [[<x|Hx>, <x|Hp>], [<x|Hp>, <p|Hp>]] c = mu [[<x|x>, <x|p>], [<x|p>, <p|p>]] c,
    lambda = c1 / c0 (0 when the pencil is degenerate or c0 vanishes)."""
    B = np.array([[xx, xp], [xp, pp]])
    A = np.array([[xhx, xhp], [xhp, php]])
    try:
        U = _chol_checked(B)
    except NotPositiveDefinite:
        return 0.0
    Ui = tri_inv_upper(U)
    C = Ui.T @ A @ Ui
    w, V = jacobi_eigh(0.5 * (C + C.T))
    c = Ui @ V[:, int(np.argmin(w))]
    return float(c[1] / c[0]) if c[0] != 0 else 0.0


class RMMDIIS:
    """RMM-DIIS, the eigensolver the paper uses (Sec. III, refs. Wood 1985,
    Kresse 1996), with the filter preconditioner and the orthonormalisation
    and subspace diagonalisation of Sec. VI after every sweep.  Every state
    is refined on its own (block by block only for the bookkeeping of the
    per-block convergence rule, Sec. VIII):

      x_0 = psi, e_i = <x_i|H x_i>/<x_i|x_i>, r_i = H x_i - e_i x_i;
      a block whose states all have ||r_0|| <= tol is left alone;
      step 0: p = K r_0, the trial step lambda minimises the Rayleigh quotient of
              x_0 + lambda p (the lower Ritz pair of span{x_0, p}),
              x_1 = x_0 + lambda p;
      steps m = 1 .. n_steps - 1: alpha = diis_coefficients over x_0..x_m,
              xbar = sum alpha_i x_i, rbar = sum alpha_i r_i,
              x_{m+1} = xbar + lambda K rbar (the same lambda);
      psi <- x_{n_steps}.
    H is applied once per step (H x_{m+1} = H xbar + lambda H p by linearity)."""

    def __init__(self, ham: Hamiltonian, Psi0: np.ndarray, nb: int, precond=None, tol: float = 1e-9,
                 n_steps: int = 3):
        self.ham = ham
        self.dV = ham.grid.dV
        self.nb = nb
        self.tol = tol
        self.n_steps = n_steps
        self.precond = precond if precond is not None else FilterPreconditioner(ham.grid)
        nst = Psi0.shape[1]
        assert nst % nb == 0 and n_steps >= 1
        Psi, _ = orthonormalize(np.array(Psi0, dtype=np.float64), self.dV)
        self.eps, self.Psi, self.HPsi, _ = subspace_diag(ham.apply, Psi, self.dV)
        self.resnorm = np.full(nst, np.inf)
        self.iterations = 0

    def _dots(self, a, b):
        return self.dV * np.sum(a * b, axis=0)

    def _block(self, b: int):
        sl = slice(b * self.nb, (b + 1) * self.nb)
        x, hx = self.Psi[:, sl].copy(), self.HPsi[:, sl].copy()
        e = self._dots(x, hx) / self._dots(x, x)
        r = hx - x * e
        res = np.sqrt(self._dots(r, r))
        self.resnorm[sl] = res
        if np.all(res <= self.tol):
            return
        xs, hxs, rs = [x], [hx], [r]
        p = self.precond(r)
        hp = self.ham.apply(p)
        lam = np.zeros(x.shape[1])
        for j in range(x.shape[1]):
            if res[j] <= self.tol:
                continue          # a converged state is not moved
            lam[j] = rayleigh_step(self._dots(x[:, j], x[:, j]), self._dots(x[:, j], p[:, j]),
                                   self._dots(p[:, j], p[:, j]), self._dots(x[:, j], hx[:, j]),
                                   self._dots(x[:, j], hp[:, j]), self._dots(p[:, j], hp[:, j]))
        for m in range(self.n_steps):
            if m > 0:
                k = len(xs)
                alpha = np.empty((k, x.shape[1]))
                for j in range(x.shape[1]):
                    A = np.array([[self._dots(rs[i][:, j], rs[l][:, j]) for l in range(k)] for i in range(k)])
                    B = np.array([[self._dots(xs[i][:, j], xs[l][:, j]) for l in range(k)] for i in range(k)])
                    alpha[:, j] = diis_coefficients(A, B)
                x = sum(alpha[i] * xs[i] for i in range(k))
                hx = sum(alpha[i] * hxs[i] for i in range(k))
                r = sum(alpha[i] * rs[i] for i in range(k))
                p = self.precond(r)
                hp = self.ham.apply(p)
            x = x + lam * p
            hx = hx + lam * hp
            e = self._dots(x, hx) / self._dots(x, x)
            xs.append(x)
            hxs.append(hx)
            rs.append(hx - x * e)
        self.Psi[:, sl] = xs[-1]

    def set_potential(self, v: np.ndarray):
        """New local potential of the Hamiltonian (an SCF step): the subspace
        is rediagonalised with it."""
        self.ham.V = np.ascontiguousarray(v, dtype=np.float64)
        self.eps, self.Psi, self.HPsi, _ = subspace_diag(self.ham.apply, self.Psi, self.dV)

    def step(self):
        """One sweep over all blocks, then orthonormalise + subspace
        diagonalisation.  Returns (eps, resnorm, n_converged)."""
        for b in range(self.Psi.shape[1] // self.nb):
            self._block(b)
        self.Psi, _ = orthonormalize(self.Psi, self.dV)
        self.eps, self.Psi, self.HPsi, _ = subspace_diag(self.ham.apply, self.Psi, self.dV)
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
