"""Oracle: the Kohn-Sham Hamiltonian in operator form (Sec. V, Eq. 3).

TEST INFRASTRUCTURE.  H = T + V_local + V_nl is never assembled as a
matrix (except for tiny grids in the tests); it is applied to a block of
orbitals psi[np, nst] (state index fastest, Sec. IV) by the plain-C loops
of ``ora_core.c``.

Nonlocal projectors (Eq. 4, Kleinman-Bylander form).  The paper leaves the
projector shapes and energies to the pseudopotential; the synthetic ones
used here are, for every atom A at R_A:
  g(d)       = exp(-d^2 / (2 r_c^2)),   d = |r - R_A|
  gamma_s    = N_s g(d)
  gamma_p,x  = N_x (x - X_A) g(d)   (likewise y, z: real l=1 harmonics)
restricted to the grid points with d^2 <= r_cut^2 (FP64, same expression as
the grid), each normalised on its own point list so that
dV * sum gamma^2 = 1; one coupling E_{A,l} per atom and channel (s, p).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import _native
from .grid import Grid
from .stencil import fd_weights


@dataclass
class Projectors:
    n_atoms: int
    sph_off: np.ndarray    # [n_atoms+1] int64
    sph_idx: np.ndarray    # [sum len] int32 grid point ids (ascending per atom)
    gam: np.ndarray        # [4 * sum len] float64, per atom: 4 rows of len
    E: np.ndarray          # [n_atoms, 4] float64 (s, p, p, p)

    def gamma(self, A: int) -> np.ndarray:
        o, e = self.sph_off[A], self.sph_off[A + 1]
        return self.gam[4 * o:4 * e].reshape(4, e - o)

    def points(self, A: int) -> np.ndarray:
        return self.sph_idx[self.sph_off[A]:self.sph_off[A + 1]]


def make_projectors(grid: Grid, atoms: np.ndarray, E_l: np.ndarray, r_c: float, r_cut: float) -> Projectors:
    atoms = np.asarray(atoms, dtype=np.float64)
    offs = [0]
    idx, gam = [], []
    x, y, z = grid.coords[:, 0], grid.coords[:, 1], grid.coords[:, 2]
    for A, (X, Y, Z) in enumerate(atoms):
        dx = x - X
        dy = y - Y
        dz = z - Z
        d2 = (dx * dx + dy * dy) + dz * dz
        sel = np.nonzero(d2 <= r_cut * r_cut)[0]
        g = np.exp(-d2[sel] / (2.0 * r_c * r_c))
        rows = np.stack([g, dx[sel] * g, dy[sel] * g, dz[sel] * g])
        norm = np.sqrt(grid.dV * (rows * rows).sum(axis=1))
        rows = rows / norm[:, None]
        idx.append(sel.astype(np.int32))
        gam.append(rows.ravel())
        offs.append(offs[-1] + len(sel))
    E = np.repeat(np.asarray(E_l, dtype=np.float64), [1, 3], axis=1)
    return Projectors(len(atoms), np.array(offs, dtype=np.int64),
                      np.concatenate(idx) if idx else np.zeros(0, np.int32),
                      np.concatenate(gam) if gam else np.zeros(0), np.ascontiguousarray(E))


@dataclass
class Hamiltonian:
    grid: Grid
    V: np.ndarray                       # [np] local potential
    proj: Projectors | None = None
    m: int = 4                          # stencil half-width (25-point star)
    cw: np.ndarray = field(default=None)
    nbr: np.ndarray = field(default=None, repr=False)

    def __post_init__(self):
        if self.cw is None:
            self.cw = fd_weights(self.m)
        self.nbr = np.ascontiguousarray(self.grid.neighbours(self.m))
        self.V = np.ascontiguousarray(self.V, dtype=np.float64)

    def apply(self, psi: np.ndarray, local_only: bool = False) -> np.ndarray:
        """H psi for psi[np, nst] (or [np])."""
        vec = psi.ndim == 1
        P = np.ascontiguousarray(psi.reshape(len(psi), -1), dtype=np.float64)
        out = np.empty_like(P)
        pr = None if local_only else self.proj
        L = _native.lib()
        if pr is None or pr.n_atoms == 0:
            z64 = np.zeros(1, np.int64)
            z32 = np.zeros(1, np.int32)
            zf = np.zeros(4)
            rc = L.ora_apply_h(self.grid.npts, P.shape[1], self.m, _native.ptr(self.nbr), _native.ptr(self.cw),
                               self.grid.h, _native.ptr(self.V), 0, _native.ptr(z64), _native.ptr(z32),
                               _native.ptr(zf), _native.ptr(zf), self.grid.dV, _native.ptr(P), _native.ptr(out))
        else:
            rc = L.ora_apply_h(self.grid.npts, P.shape[1], self.m, _native.ptr(self.nbr), _native.ptr(self.cw),
                               self.grid.h, _native.ptr(self.V), pr.n_atoms, _native.ptr(pr.sph_off),
                               _native.ptr(pr.sph_idx), _native.ptr(pr.gam), _native.ptr(pr.E), self.grid.dV,
                               _native.ptr(P), _native.ptr(out))
        if rc != 0:
            raise MemoryError("ora_apply_h failed")
        return out.ravel() if vec else out

    def dense(self) -> np.ndarray:
        """H as a dense matrix, assembled column by column as H e_i (tiny grids)."""
        n = self.grid.npts
        if n > 6000:
            raise ValueError("dense assembly is for tiny grids only")
        return self.apply(np.eye(n))

    def nonlocal_dense(self) -> np.ndarray:
        """V_nl alone as a dense matrix (tiny grids), from its definition."""
        n = self.grid.npts
        M = np.zeros((n, n))
        if self.proj is None:
            return M
        for A in range(self.proj.n_atoms):
            pts = self.proj.points(A)
            g = self.proj.gamma(A)
            for q in range(4):
                M[np.ix_(pts, pts)] += self.proj.E[A, q] * self.grid.dV * np.outer(g[q], g[q])
        return M
