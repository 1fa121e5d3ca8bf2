"""Overlap, Cholesky orthonormalisation and subspace diagonalisation (Sec. VI)
on the GPU against the FP64 oracle.

Tolerances: FP64 data, <= 1e-12 relative on overlaps and 1e-10 on the
orthonormalised orbitals (a triangular solve amplifies rounding by the
condition number of S, ~10 here).  FP32 data: the overlap's products are
exact and the accumulation compensated, so it matches the oracle's FP64
contraction of the same FP32 values to <= 1e-12; the subspace eigenvalues
inherit the FP32 rounding of H psi (relative <= 2e-6 per state, see
test_ham_gpu), i.e. <= 2e-6 * ||H psi|| absolute.
"""
import numpy as np
import pytest

import workloads as wl
from tests.helpers import SMALL_ATOMS, SMALL_E, SMALL_H, SMALL_RADIUS
from tests.test_ham_gpu import _lib_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SYS = ("atoms", (SMALL_ATOMS, SMALL_E, SMALL_RADIUS, SMALL_H))


def _dev(a, t=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(t).cuda()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny", [(16, 16), (40, 24), (1, 7), (96, 130)])
def test_overlap_parity(dtype, nx, ny):
    from paper_1306_2953_gb300 import api
    from oracle import linalg as ol
    lg, H, g_ora, H_ora, idx = _lib_system(*SYS)
    X = wl.random_block(g_ora.npts, nx, 1)[idx]
    Y = wl.gaussian_sum_block(g_ora.coords, ny, 2)[idx]
    t = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        X, Y = X.astype(np.float32).astype(np.float64), Y.astype(np.float32).astype(np.float64)
    S = api.overlap(lg, _dev(X, t), _dev(Y, t)).cpu().numpy()
    ref = ol.overlap(X, Y, g_ora.dV)
    assert np.abs(S - ref).max() <= 1e-12 * np.abs(ref).max()


def test_overlap_full_size_mol100_f32():
    """The 100-atom molecule at full size, 32 x 32 FP32 overlap."""
    from paper_1306_2953_gb300 import api
    from oracle import linalg as ol
    lg, H, g_ora, H_ora, idx = _lib_system("mol", (wl.MOL100.system,))
    X = wl.random_block(g_ora.npts, 32, 5)[idx].astype(np.float32)
    S = api.overlap(lg, _dev(X, torch.float32), _dev(X, torch.float32)).cpu().numpy()
    ref = ol.overlap(X.astype(np.float64), X.astype(np.float64), g_ora.dV)
    assert np.abs(S - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("nst", [16, 48, 256, 400])
def test_orthonormalize_parity_f64(nst):
    """Up to 160 states the Cholesky runs in one CTA; above, blocked over
    many (400: a ragged last block of 16 rows)."""
    from paper_1306_2953_gb300 import api
    from oracle import linalg as ol
    lg, H, g_ora, H_ora, idx = _lib_system(*SYS)
    psi = wl.random_block(g_ora.npts, nst, 11)[idx]
    P = _dev(psi)
    Ui = api.orthonormalize(lg, P).cpu().numpy()
    ref, Ui_ref = ol.orthonormalize(psi, g_ora.dV)
    out = P.cpu().numpy()
    assert np.abs(Ui - Ui_ref).max() <= 1e-10 * np.abs(Ui_ref).max()
    assert np.abs(out - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.abs(ol.overlap(out, out, g_ora.dV) - np.eye(nst)).max() < 1e-12


def test_orthonormalize_not_spd():
    from paper_1306_2953_gb300 import api
    from paper_1306_2953_gb300._lib import RS_ENOTSPD, RsError
    lg, H, g_ora, H_ora, idx = _lib_system(*SYS)
    psi = wl.random_block(g_ora.npts, 8, 3)[idx]
    psi[:, 5] = psi[:, 2]            # linearly dependent columns
    P = _dev(psi)
    before = P.clone()
    with pytest.raises(RsError) as e:
        api.orthonormalize(lg, P)
    assert e.value.code == RS_ENOTSPD
    assert torch.equal(P, before)


def test_orthonormalize_not_spd_blocked():
    """A dependent column past the first block row of the blocked Cholesky
    (state 250 of 300): RS_ENOTSPD and the orbitals untouched."""
    from paper_1306_2953_gb300 import api
    from paper_1306_2953_gb300._lib import RS_ENOTSPD, RsError
    lg, H, g_ora, H_ora, idx = _lib_system(*SYS)
    psi = wl.random_block(g_ora.npts, 300, 3)[idx]
    psi[:, 250] = psi[:, 10]
    P = _dev(psi)
    before = P.clone()
    with pytest.raises(RsError) as e:
        api.orthonormalize(lg, P)
    assert e.value.code == RS_ENOTSPD
    assert torch.equal(P, before)


def _align_signs(V, R):
    s = np.sign(np.sum(V * R, axis=0))
    s[s == 0] = 1
    return V * s


@pytest.mark.parametrize("dtype,nst", [("f64", 24), ("f32", 24), ("f64", 256)])
def test_subspace_diag_parity(dtype, nst):
    from paper_1306_2953_gb300 import api
    from oracle import linalg as ol
    lg, H, g_ora, H_ora, idx = _lib_system(*SYS)
    psi = wl.gaussian_sum_block(g_ora.coords, nst, 12) if nst <= 32 else wl.random_block(g_ora.npts, nst, 12)
    psi, _ = ol.orthonormalize(psi, g_ora.dV)
    t = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        psi = psi.astype(np.float32).astype(np.float64)
    P = _dev(psi[idx], t)
    eps, xi, HP = api.subspace_diag(H, P, nb=8)
    eps = eps.cpu().numpy()
    # the oracle's Rayleigh-Ritz of the same orbitals (not re-orthonormalised)
    h = ol.overlap(psi, H_ora.apply(psi), g_ora.dV)
    h = 0.5 * (h + h.T)
    ref_eps, ref_xi = ol.jacobi_eigh(h)
    if dtype == "f64":
        assert np.abs(eps - ref_eps).max() <= 1e-10 * np.abs(ref_eps).max()
        rot = P.cpu().numpy()
        ref_rot = (psi @ ref_xi)[idx]
        assert np.abs(_align_signs(rot, ref_rot) - ref_rot).max() <= 1e-8 * np.abs(ref_rot).max()
    else:
        hn = np.linalg.norm(H_ora.apply(psi), axis=0).max() * np.sqrt(g_ora.dV)
        assert np.abs(eps - ref_eps).max() <= 2e-6 * hn


def test_linalg_bad_arguments():
    from paper_1306_2953_gb300 import api
    from paper_1306_2953_gb300._lib import RsError
    lg, H, g_ora, H_ora, idx = _lib_system(*SYS)
    P = torch.zeros((g_ora.npts, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(RsError):
        api.subspace_diag(H, P, nb=3)
