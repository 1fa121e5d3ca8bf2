"""Oracle: the Hartree potential by fast Fourier transforms (Sec. X, "The
Hartree potential"; Eq. 2, the Poisson equation lap V_H = -4 pi n).

TEST INFRASTRUCTURE.  The paper's steps: copy the density from the grid to
a cube, forward FFT, multiply by the Coulomb-interaction kernel, inverse
FFT, copy the potential back to the grid.  Free boundary conditions come
from an enlarged cube and a modified kernel (Rozzi et al. 2006); the
reading taken here is their spherical cutoff, the Coulomb potential 1/r cut
off at r = R_c, whose Fourier transform is

    v(G) = 4 pi (1 - cos(|G| R_c)) / |G|^2,   v(0) = 2 pi R_c^2.

With R_c at least the largest distance D between two grid points and a
cube of N_a points along axis a with N_a h >= (extent of the grid along a)
+ R_c, no periodic image of the density lies within R_c of the density, so
the periodic convolution equals the free-space one for every grid point.
N_a is the smallest size with no prime factor other than 2 and 3 (the
radices of the paper's GPU FFT).  numpy's FFT is the library primitive.
"""
from __future__ import annotations

import math

import numpy as np

from .grid import Grid


def smooth_size(n: int) -> int:
    """Smallest integer >= n of the form 2^p 3^q."""
    best = None
    p2 = 1
    while p2 < 2 * n + 2:
        p3 = p2
        while p3 < 2 * n + 2:
            if p3 >= n and (best is None or p3 < best):
                best = p3
            p3 *= 3
        p2 *= 2
    return best


def cube_geometry(grid: Grid):
    """(lattice coordinate of cube element 0, cube shape, R_c) for a grid:
    R_c = D + h (D: the largest distance between two points of the grid's
    bounding box), N_a = smooth_size(extent_a + ceil(R_c / h) + 1)."""
    lo = grid.ijk.min(axis=0)
    hi = grid.ijk.max(axis=0)
    ext = hi - lo
    D = grid.h * float(np.sqrt(np.sum(ext.astype(np.float64) ** 2)))
    Rc = D + grid.h
    shape = tuple(smooth_size(int(ext[a]) + int(math.ceil(Rc / grid.h)) + 1) for a in range(3))
    return lo, shape, Rc


def coulomb_kernel(shape, h: float, Rc: float) -> np.ndarray:
    """v(G) on the cube's FFT frequencies (numpy order)."""
    g = [2.0 * np.pi * np.fft.fftfreq(n, d=h) for n in shape]
    G2 = g[0][:, None, None] ** 2 + g[1][None, :, None] ** 2 + g[2][None, None, :] ** 2
    G = np.sqrt(G2)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = 4.0 * np.pi * (1.0 - np.cos(G * Rc)) / G2
    v[0, 0, 0] = 2.0 * np.pi * Rc * Rc
    return v


def hartree(grid: Grid, n: np.ndarray) -> np.ndarray:
    """V_H at every grid point for the density n (one value per point):
    cube <- n, FFT, times v(G), inverse FFT, back to the grid."""
    lo, shape, Rc = cube_geometry(grid)
    cube = np.zeros(shape)
    rel = grid.ijk - lo
    cube[rel[:, 0], rel[:, 1], rel[:, 2]] = n
    V = np.fft.ifftn(np.fft.fftn(cube) * coulomb_kernel(shape, grid.h, Rc))
    return V.real[rel[:, 0], rel[:, 1], rel[:, 2]]
