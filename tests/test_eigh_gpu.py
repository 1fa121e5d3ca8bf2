"""Dense symmetric eigensolver (the Rayleigh-Ritz diagonalisation of Sec. VI)
on the GPU against the oracle's cyclic Jacobi, for the sizes the solver uses
(one CTA in shared memory while the packed triangle fits, about n = 330 in
FP32 and 234 in FP64; the cooperative multi-CTA variant above, so 256 in
FP64 and 400 and 1024 in both) and all three modes.  FP64 modes: eigenvalues to
1e-12 of the spectral radius and A V = V diag(w) to 1e-11; FP32 Jacobi
alone stops at its rounding floor: 1e-5 of the Frobenius norm."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _matrix(n, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    w = np.sort(rng.uniform(-spread, spread, n))
    w[n // 3] = w[n // 3 + 1] + 1e-9          # a nearly degenerate pair
    return (Q * w) @ Q.T


@pytest.mark.parametrize("n", [16, 48, 96, 130, 192, 256, 400])
@pytest.mark.parametrize("refine", [2, 0, -1])
def test_eigh_matches_oracle(n, refine):
    from oracle import linalg as ol
    from paper_1306_2953_gb300 import api
    A = _matrix(n, n + 7, 40.0)
    w, V = api.eigh(torch.from_numpy(A).cuda(), refine=refine)
    w, V = w.cpu().numpy(), V.cpu().numpy()
    # the rounding floor of the oracle's FP64 rotations grows with the order:
    # above 256 its stopping test is set at 1e-14 of the Frobenius norm
    ref, _ = ol.jacobi_eigh(A, tol=1e-14 if n > 256 else 1e-15)
    if refine < 0:
        # FP32 Jacobi alone stops at its rounding floor, ~1e-6 of the Frobenius norm
        fro = np.linalg.norm(A)
        assert np.abs(w - ref).max() <= 1e-5 * fro
        assert np.abs(A @ V - V * w).max() <= 1e-5 * fro
    else:
        assert np.abs(w - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(A @ V - V * w).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("refine", [2, 0, -1])
def test_eigh_order_1024(refine):
    """The order of the 300-atom subspace matrix (1024), on the multi-CTA
    Jacobi in all three modes (FP32 then FP64 refinement; FP64 alone; FP32
    alone, as the mixed eigensolver's inner steps use it), against the
    library eigensolver (LAPACK through numpy) of the same matrix.  FP32
    alone: eigenvalues and residuals within its stopping floor, 1e-5 of the
    Frobenius norm, and eigenvectors orthogonal to 1e-4."""
    from paper_1306_2953_gb300 import api
    A = _matrix(1024, 5, 60.0)
    w, V = api.eigh(torch.from_numpy(A).cuda(), refine=refine)
    w, V = w.cpu().numpy(), V.cpu().numpy()
    ref = np.linalg.eigvalsh(A)
    if refine < 0:
        fro = np.linalg.norm(A)
        assert np.abs(w - ref).max() <= 1e-5 * fro
        assert np.abs(A @ V - V * w).max() <= 1e-5 * fro
        assert np.abs(V.T @ V - np.eye(1024)).max() <= 1e-4
    else:
        assert np.abs(w - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(A @ V - V * w).max() <= 1e-11 * np.abs(ref).max()
        assert np.abs(V.T @ V - np.eye(1024)).max() <= 1e-12
