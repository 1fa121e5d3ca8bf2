"""Shared test plumbing: building the same synthetic system on both sides
(oracle and library) and matching their points by integer lattice
coordinates.  Holds no arithmetic of the method."""
from __future__ import annotations

import functools

import numpy as np

import workloads as wl


def lib_to_oracle_index(ora_grid, lib_ijk: np.ndarray) -> np.ndarray:
    """For every library point, the index of the same lattice point in the
    oracle grid (all must exist)."""
    idx = ora_grid.lookup(lib_ijk.astype(np.int64))
    assert np.all(idx >= 0), "library point missing from the oracle grid"
    return idx


@functools.lru_cache(maxsize=8)
def oracle_system(kind: str, *params):
    """Oracle grid + Hamiltonian for a named synthetic system (cached)."""
    from oracle import grid as og, hamiltonian as oh
    if kind == "box":
        n, h, omega = params
        g = og.box_grid(n, h)
        return g, oh.Hamiltonian(g, wl.harmonic_potential(g.coords, omega)), None, None
    if kind == "mol":
        spec = params[0]
        atoms = wl.atom_positions(spec)
        E = wl.kb_couplings(spec)
        g = og.sphere_union_grid(atoms, spec.radius, spec.h)
        pr = oh.make_projectors(g, atoms, E, spec.r_c, spec.r_cut)
        V = wl.local_potential(g.coords, atoms)
        return g, oh.Hamiltonian(g, V, pr), atoms, E
    if kind == "atoms":
        atoms, E, radius, h = params
        atoms = np.array(atoms)
        E = np.array(E)
        g = og.sphere_union_grid(atoms, radius, h)
        pr = oh.make_projectors(g, atoms, E, 1.0, 3.0)
        V = wl.local_potential(g.coords, atoms)
        return g, oh.Hamiltonian(g, V, pr), atoms, E
    raise ValueError(kind)


# a small molecule whose projector spheres overlap heavily and touch the grid edge
SMALL_ATOMS = ((0.0, 0.0, 0.0), (1.9, 0.3, -0.2), (0.4, 1.7, 0.8), (-2.1, 0.5, 1.1), (0.3, -1.2, 2.6))
SMALL_E = ((1.3, 0.7), (0.5, 1.9), (1.1, 1.4), (0.9, 0.6), (1.8, 1.2))
SMALL_RADIUS, SMALL_H = 3.4, 0.3
