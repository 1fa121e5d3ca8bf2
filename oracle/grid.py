"""Oracle: real-space grids (Sec. II, Fig. 1; Sec. XI).

TEST INFRASTRUCTURE.  Points are kept in lexicographic order of their
integer lattice coordinates (i slowest, k fastest); the GPU library may use
any order and is matched point by point through the integer coordinates.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

HALO = 4  # margin of the bounding-box map: the star stencil's half-width


@dataclass
class Grid:
    h: float
    ijk: np.ndarray        # [np, 3] int64 lattice coordinates, lexicographic
    coords: np.ndarray     # [np, 3] float64 positions (Bohr)
    origin: np.ndarray     # [3] int64, lattice coordinate of map[0,0,0]
    map: np.ndarray        # [nx, ny, nz] int64 point index or -1

    @property
    def npts(self) -> int:
        return len(self.ijk)

    @property
    def dV(self) -> float:
        return self.h ** 3

    def lookup(self, ijk: np.ndarray) -> np.ndarray:
        """Point index of lattice coordinates (-1 outside the grid)."""
        rel = np.asarray(ijk) - self.origin
        shp = np.array(self.map.shape)
        ok = np.all((rel >= 0) & (rel < shp), axis=1)
        out = np.full(len(rel), -1, dtype=np.int64)
        r = rel[ok]
        out[ok] = self.map[r[:, 0], r[:, 1], r[:, 2]]
        return out

    def neighbours(self, m: int) -> np.ndarray:
        """Star-stencil neighbour table [np, 3, 2m]: along each axis the
        points at offsets -m..-1, 1..m, or -1 where that lattice point is not
        a grid point."""
        offs = [j for j in range(-m, m + 1) if j != 0]
        nbr = np.empty((self.npts, 3, 2 * m), dtype=np.int32)
        for a in range(3):
            for t, j in enumerate(offs):
                e = np.zeros(3, dtype=np.int64)
                e[a] = j
                nbr[:, a, t] = self.lookup(self.ijk + e)
        return nbr


def _finish(h: float, ijk: np.ndarray, coords: np.ndarray) -> Grid:
    order = np.lexsort((ijk[:, 2], ijk[:, 1], ijk[:, 0]))
    ijk = ijk[order]
    coords = coords[order]
    origin = ijk.min(axis=0) - HALO
    shape = ijk.max(axis=0) - origin + 1 + HALO
    mp = np.full(tuple(shape), -1, dtype=np.int64)
    rel = ijk - origin
    mp[rel[:, 0], rel[:, 1], rel[:, 2]] = np.arange(len(ijk))
    return Grid(h=h, ijk=ijk, coords=coords, origin=origin, map=mp)


def sphere_union_grid(atoms: np.ndarray, radius: float, h: float) -> Grid:
    """Uniform grid on the union of spheres of ``radius`` around the atoms
    (Sec. II).  Lattice points r = h*(i,j,k); a point belongs to the grid iff
    for some atom A, (x-X)^2 + (y-Y)^2 + (z-Z)^2 <= radius^2, evaluated in
    FP64 in that order with x = h*i."""
    atoms = np.asarray(atoms, dtype=np.float64)
    lo = np.floor((atoms.min(axis=0) - radius) / h).astype(np.int64) - 1
    hi = np.ceil((atoms.max(axis=0) + radius) / h).astype(np.int64) + 1
    r2 = radius * radius
    jj, kk = np.meshgrid(np.arange(lo[1], hi[1] + 1), np.arange(lo[2], hi[2] + 1), indexing="ij")
    jj = jj.ravel()
    kk = kk.ravel()
    y = h * jj.astype(np.float64)
    z = h * kk.astype(np.float64)
    pts = []
    for i in range(lo[0], hi[0] + 1):
        x = h * float(i)
        inside = np.zeros(len(jj), dtype=bool)
        for X, Y, Z in atoms:
            dx = x - X
            dy = y - Y
            dz = z - Z
            inside |= (dx * dx + dy * dy) + dz * dz <= r2
        if inside.any():
            sel = np.nonzero(inside)[0]
            pts.append(np.stack([np.full(len(sel), i), jj[sel], kk[sel]], axis=1))
    ijk = np.concatenate(pts).astype(np.int64)
    return _finish(h, ijk, h * ijk.astype(np.float64))


def box_grid(n: int, h: float) -> Grid:
    """Full n^3 box, x_i = (i - (n-1)/2) h, zero outside (harmonic oscillator)."""
    i = np.arange(n)
    I, J, K = np.meshgrid(i, i, i, indexing="ij")
    ijk = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.int64)
    coords = (ijk.astype(np.float64) - (n - 1) / 2.0) * h
    return _finish(h, ijk, coords)
