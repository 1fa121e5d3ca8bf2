"""The allocation-free orthonormalisation entry point.

rs_orthonormalize_noalloc is for callers that cannot allocate device memory
when they need the operation (frameworks that own every device buffer and
hand out no workspace, loops that forbid cudaMalloc after start-up).  It keeps its scratch in a fixed device array inside the library.
This test calls it through the C ABI and checks it against the workspace
entry point rs_orthonormalize, on two calls in a row with different sizes
and precisions (the second call must not be disturbed by what the first left
in the shared scratch), and checks that sizes beyond its limit are refused.

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as wl
from tests.helpers import SMALL_ATOMS, SMALL_E, SMALL_H, SMALL_RADIUS, lib_to_oracle_index, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(grid, P):
    from paper_1306_2953_gb300 import _lib
    from paper_1306_2953_gb300.api import _stream, dtype_code
    _lib.call("rs_orthonormalize_noalloc", grid._h, ctypes.c_void_p(P.data_ptr()), P.stride(0), P.shape[1],
              dtype_code(P), _stream())


def test_noalloc_matches_workspace_entry_point_twice():
    from paper_1306_2953_gb300 import api
    g_ora, _, _, _ = oracle_system("atoms", SMALL_ATOMS, SMALL_E, SMALL_RADIUS, SMALL_H)
    lg = api.Grid.spheres(np.array(SMALL_ATOMS), SMALL_RADIUS, SMALL_H)
    idx = lib_to_oracle_index(g_ora, lg.ijk())
    cases = [(48, torch.float64, 1e-10), (24, torch.float32, 1e-5)]
    for call, (nst, dt, tol) in enumerate(cases):
        psi = wl.random_block(g_ora.npts, nst, 40 + call)[idx]
        a = torch.from_numpy(np.ascontiguousarray(psi)).to(dt).cuda()
        b = a.clone()
        _noalloc(lg, a)
        api.orthonormalize(lg, b)
        torch.cuda.synchronize()
        A, B = a.double().cpu().numpy(), b.double().cpu().numpy()
        assert np.abs(A - B).max() <= tol * np.abs(B).max(), f"call {call}"
        S = lg.dV * A.T @ A
        assert np.abs(S - np.eye(nst)).max() <= (1e-12 if dt == torch.float64 else 1e-5)


def test_noalloc_rejects_oversized():
    from paper_1306_2953_gb300 import api
    from paper_1306_2953_gb300._lib import RS_EINVAL, RsError
    lg = api.Grid.box(6, 6, 6, 0.3)
    P = torch.zeros((lg.npts, 257), dtype=torch.float64, device="cuda")
    with pytest.raises(RsError) as e:
        _noalloc(lg, P)
    assert e.value.code == RS_EINVAL
