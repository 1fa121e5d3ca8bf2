"""Block-CG eigensolver on the GPU against the FP64 oracle.

Bars (FP64 mode): eigenvalues within 1e-8 Ha of the oracle's converged
values (tests/golden/, written by make_golden.py from oracle/ only), and
sweep-by-sweep Ritz values equal to the oracle's own block CG from the same
start vectors to 1e-9 Ha (same algorithm, different rounding order).
"""
import json
import os

import numpy as np
import pytest

import workloads as wl
from tests.helpers import lib_to_oracle_index, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, f"eigs_{name}.json")) as f:
        return json.load(f)


def _system(w):
    from paper_1306_2953_gb300 import api
    s = w.system
    if isinstance(s, wl.BoxSpec):
        g_ora, H_ora, _, _ = oracle_system("box", s.n, s.h, s.omega)
        lg = api.Grid.box(s.n, s.n, s.n, s.h)
        idx = lib_to_oracle_index(g_ora, lg.ijk())
        return lg, api.Hamiltonian(lg, H_ora.V[idx]), g_ora, H_ora, idx
    g_ora, H_ora, atoms, E = oracle_system("mol", s)
    lg = api.Grid.spheres(atoms, s.radius, s.h)
    idx = lib_to_oracle_index(g_ora, lg.ijk())
    return lg, api.Hamiltonian(lg, H_ora.V[idx], api.Projectors(lg, atoms, E, s.r_c, s.r_cut)), g_ora, H_ora, idx


def test_block_cg_steps_match_oracle_f64():
    from oracle import eigensolver
    from paper_1306_2953_gb300 import api
    w = wl.HO32
    lg, H, g_ora, H_ora, idx = _system(w)
    psi0 = wl.random_block(g_ora.npts, w.n_states, w.seed)
    ora = eigensolver.BlockCG(H_ora, psi0, w.block, tol=1e-12)
    S = api.Solver(H, torch.from_numpy(np.ascontiguousarray(psi0[idx])).cuda(), w.block, 1e-12)
    for it in range(3):
        e_ora, r_ora, _ = ora.step()
        eps, res, _ = S.step()
        e = eps.cpu().numpy()
        # the judged states are separated from the rest; the block's top states cut
        # through the 10-fold n=3 shell, where the selected Ritz span is ill-determined
        assert np.abs(e[:w.judged] - e_ora[:w.judged]).max() <= 1e-9, f"sweep {it}"
        assert np.abs(e - e_ora).max() <= 1e-6, f"sweep {it}"
        assert np.abs(res.cpu().numpy()[:w.judged] - r_ora[:w.judged]).max() <= 1e-7 * max(1.0, np.abs(r_ora).max())


def _solve(S, judged, tol, max_iter):
    for it in range(max_iter):
        eps, res, _ = S.step()
        r = res.cpu().numpy()
        if np.all(r[:judged] <= tol):
            return eps.cpu().numpy(), it + 1
    raise AssertionError(f"not converged in {max_iter} sweeps; max residual {r[:judged].max():.2e}")


def test_harmonic_oscillator_f64_converges_to_oracle():
    from paper_1306_2953_gb300 import api
    w = wl.HO32
    lg, H, g_ora, H_ora, idx = _system(w)
    psi0 = wl.random_block(g_ora.npts, w.n_states, w.seed)
    S = api.Solver(H, torch.from_numpy(np.ascontiguousarray(psi0[idx])).cuda(), w.block, 1e-6)
    eps, iters = _solve(S, w.judged, 1e-6, 300)
    ref = np.array(golden(w.name)["eigenvalues"])
    assert np.abs(eps[:w.judged] - ref).max() <= 1e-8
    # and the analytic (n + 3/2) omega levels, within the discretisation error
    assert np.abs(eps[:w.judged] - np.array([1.5] + [2.5] * 3 + [3.5] * 6)).max() < 1e-4


def test_mol20_f64_converges_to_oracle():
    from paper_1306_2953_gb300 import api
    w = wl.MOL20
    lg, H, g_ora, H_ora, idx = _system(w)
    psi0 = wl.random_block(g_ora.npts, w.n_states, w.seed)
    S = api.Solver(H, torch.from_numpy(np.ascontiguousarray(psi0[idx])).cuda(), w.block, 1e-6)
    eps, iters = _solve(S, w.judged, 1e-6, 600)
    ref = np.array(golden(w.name)["eigenvalues"])
    assert np.abs(eps[:w.judged] - ref).max() <= 1e-8


def test_solver_bad_config():
    from paper_1306_2953_gb300 import api
    from paper_1306_2953_gb300._lib import RsError
    w = wl.HO32
    lg, H, g_ora, H_ora, idx = _system(w)
    psi0 = torch.zeros((g_ora.npts, 12), dtype=torch.float64, device="cuda")
    with pytest.raises(RsError):
        api.Solver(H, psi0, 8, 1e-6)          # nst not a multiple of nb


def test_mol20_mixed_precision_within_1e6_of_oracle():
    """FP32 orbitals, H psi and inner iterations (tensor-core contractions),
    FP64 Gram matrices, Cholesky, Rayleigh-Ritz and eigenvalues, closed by one
    FP64 Rayleigh-Ritz of the converged subspace: every state within 1e-6 Ha
    of the oracle's FP64 eigenvalues.  Without the closing step the FP32
    rounding of H itself (potential ~40 Ha stored to 6e-8) leaves ~2e-6 Ha."""
    from paper_1306_2953_gb300 import api
    w = wl.MOL20
    lg, H, g_ora, H_ora, idx = _system(w)
    psi0 = wl.random_block(g_ora.npts, w.n_states, w.seed)
    S = api.Solver(H, torch.from_numpy(np.ascontiguousarray(psi0[idx])).float().cuda(), w.block, 1e-4)
    ref = np.array(golden(w.name)["eigenvalues"])
    for it in range(600):
        eps, res, _ = S.step()
        if np.all(res.cpu().numpy()[:w.judged] <= 1e-4):
            break
    e = S.rayleigh_ritz_f64().cpu().numpy()
    assert np.abs(e[:w.judged] - ref).max() <= 1e-6


def test_mol20_mixed_cg_preconditioner_fewer_sweeps():
    """Five CG iterations on (-1/2 Lap + 2) W = R as the preconditioner: the
    FP32 solve reaches the oracle's eigenvalues (1e-6 Ha after the closing
    FP64 Rayleigh-Ritz) in fewer sweeps than the filter from the same start."""
    from paper_1306_2953_gb300 import api
    w = wl.MOL20
    lg, H, g_ora, H_ora, idx = _system(w)
    Hs = api.Hamiltonian(lg, np.full(lg.npts, 2.0))
    psi0 = torch.from_numpy(np.ascontiguousarray(wl.random_block(g_ora.npts, w.n_states, w.seed)[idx])).float().cuda()
    ref = np.array(golden(w.name)["eigenvalues"])
    sweeps = {}
    for kind in ("filter", "cg"):
        S = api.Solver(H, psi0, w.block, 1e-4)
        if kind == "cg":
            S.set_precond_cg(Hs, 5)
        for it in range(600):
            eps, res, _ = S.step()
            if np.all(res.cpu().numpy()[:w.judged] <= 1e-4):
                break
        sweeps[kind] = it + 1
        e = S.rayleigh_ritz_f64().cpu().numpy()
        assert np.abs(e[:w.judged] - ref).max() <= 1e-6, kind
    assert sweeps["cg"] < sweeps["filter"], sweeps
