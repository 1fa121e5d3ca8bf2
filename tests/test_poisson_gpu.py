"""The FFT Hartree solver on the GPU (through the C ABI) against the FP64
oracle (same cube, same kernel: agreement to FFT rounding, 1e-11 relative)
and against the closed form of a Gaussian charge."""
import numpy as np
import pytest

import workloads as wl
from tests.helpers import lib_to_oracle_index, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_poisson_gaussian_closed_form():
    from scipy.special import erf
    from oracle import grid as og, poisson as op
    from paper_1306_2953_gb300 import api
    h, n = 0.25, 53
    g = og.box_grid(n, h)
    lg = api.Grid.box(n, n, n, h)
    idx = lib_to_oracle_index(g, lg.ijk())
    r = np.linalg.norm(g.coords, axis=1)
    rho = np.exp(-r * r / 2.0) / (2 * np.pi) ** 1.5
    P = api.Poisson(lg)
    shape, rc, _ = P.info()
    lo, oshape, orc = op.cube_geometry(g)
    assert tuple(shape) == tuple(oshape) and abs(rc - orc) <= 1e-12 * orc
    V = P.solve(torch.from_numpy(np.ascontiguousarray(rho[idx])).cuda()).cpu().numpy()
    ref = np.where(r > 0, erf(r / np.sqrt(2)) / np.where(r > 0, r, 1), np.sqrt(2 / np.pi))[idx]
    assert np.abs(V - ref).max() <= 1e-9 * ref.max()


@pytest.mark.parametrize("name", ["mol20_h0.35", "mol100_h0.3"])
def test_poisson_matches_oracle_on_molecule_grids(name):
    """A smooth synthetic density on the union-of-spheres grids (a Gaussian
    per atom): the GPU solve equals the oracle's to 1e-11 of max |V_H|."""
    from oracle import poisson as op
    from paper_1306_2953_gb300 import api
    w = wl.WORKLOADS[name]
    s = w.system
    g_ora, _, atoms, _ = oracle_system("mol", s)
    lg = api.Grid.spheres(atoms, s.radius, s.h)
    idx = lib_to_oracle_index(g_ora, lg.ijk())
    rho = np.zeros(g_ora.npts)
    for a in atoms:
        rho += np.exp(-((g_ora.coords - a) ** 2).sum(axis=1) / 1.5)
    ref = op.hartree(g_ora, rho)
    P = api.Poisson(lg)
    V = P.solve(torch.from_numpy(np.ascontiguousarray(rho[idx])).cuda()).cpu().numpy()
    assert np.abs(V - ref[idx]).max() <= 1e-11 * np.abs(ref).max()
