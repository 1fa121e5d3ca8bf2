"""Tensor-core (tcgen05) overlap and rotation of FP32 orbitals against the
FP64 oracle's contraction of the same FP32 values.

Each FP32 operand is split exactly into three BF16 pieces; the six retained
piece products are exact and accumulated in FP32.  The dropped products
are below 3 * 2^-24 of |x||y| and FP32 accumulation adds ~2^-24 per term,
so every entry is within 2e-6 * sum_p |x_p| |y_p| (the natural scale of the
contraction) of the exact value -- the bound asserted here.
"""
import numpy as np
import pytest

import workloads as wl
from tests.helpers import SMALL_ATOMS, SMALL_E, SMALL_H, SMALL_RADIUS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _grid():
    from paper_1306_2953_gb300 import api
    return api.Grid.spheres(np.array(SMALL_ATOMS), SMALL_RADIUS, SMALL_H)


@pytest.mark.parametrize("nx,ny", [(128, 128), (32, 48), (96, 96), (256, 64), (130, 200)])
def test_overlap_tc_parity(nx, ny):
    from oracle import linalg as ol
    from paper_1306_2953_gb300 import api
    g = _grid()
    X = wl.random_block(g.npts, nx, 3).astype(np.float32)
    Y = wl.random_block(g.npts, ny, 4).astype(np.float32)
    S = api.overlap_tc(g, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()).cpu().numpy()
    ref = ol.overlap(X.astype(np.float64), Y.astype(np.float64), g.dV)
    scale = g.dV * np.abs(X.astype(np.float64)).T @ np.abs(Y.astype(np.float64))
    assert np.all(np.abs(S - ref) <= 2e-6 * scale)


@pytest.mark.parametrize("n,m", [(64, 64), (32, 96), (256, 256), (100, 40)])
def test_rotate_parity(n, m):
    from paper_1306_2953_gb300 import api
    g = _grid()
    X = wl.random_block(g.npts, n, 5).astype(np.float32)
    C = np.random.default_rng(6).standard_normal((n, m))
    Y = api.rotate(torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()).cpu().numpy()
    ref = X.astype(np.float64) @ C
    scale = np.abs(X.astype(np.float64)) @ np.abs(C)
    assert np.all(np.abs(Y - ref) <= 2e-6 * scale)


def test_rotate_in_place():
    from paper_1306_2953_gb300 import api
    g = _grid()
    X = wl.random_block(g.npts, 64, 7).astype(np.float32)
    C = np.random.default_rng(8).standard_normal((64, 64))
    Xd = torch.from_numpy(X).cuda()
    api.rotate(Xd, torch.from_numpy(C).cuda(), Y=Xd)
    ref = X.astype(np.float64) @ C
    assert np.all(np.abs(Xd.cpu().numpy() - ref) <= 2e-6 * (np.abs(X.astype(np.float64)) @ np.abs(C)))
