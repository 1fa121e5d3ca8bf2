"""H psi on the GPU (through the C ABI) against the FP64 oracle.

Tolerances: FP64 mode, relative error per state <= 1e-12 (the FP64 hot-path
target).  FP32 mode: the oracle is fed the same FP32-rounded inputs; an
output is a sum of ~30 products of magnitude up to |w_0 psi| ~ 4.3/h^2 |psi|
plus the potential, so FP32 rounding bounds its error by roughly
30 * 2^-24 * max|term|; per state this gives a relative norm error below
2e-6 for random orbitals and below 3e-5 for smooth ones, where the Laplacian
cancels most of the terms (the bounds asserted below).

Element-wise FP32 bound (full-size molecules).  With u = 2^-24, every
output element of the FP32 kernel differs from the FP64 value of the same
FP32 inputs by at most u (c_loc M_loc + c_nl M_nl), where the oracle gives
the term magnitudes at that element:
  M_loc = 1/(2h^2) sum_taps |c_j| |psi| + |V| |psi|   (stencil and potential),
  M_nl  = sum_{A,q} |gamma_Aq(p)| |E_Aq| dV sum_{p'} |gamma_Aq(p')| |psi(p')|.
The local part is a recursive sum of 27 terms whose inputs (weights, V) are
themselves rounded once: c_loc = 32 covers (27 - 1) + 2 roundings.  The
projection integral sums a sphere of ~4200 products in FP32 partial sums
and atomics; its error grows like sqrt(n) u for rounding errors of random
sign (~65 u) and its worst case is n u: c_nl = 512 is eight times the
typical growth.  A wrong or missing nonlocal entry changes an element by a
term of size ~M_nl, 2^24 / 512 = 32768 times this bound.
"""
import os

import numpy as np
import pytest

import workloads as wl
from tests.helpers import SMALL_ATOMS, SMALL_E, SMALL_H, SMALL_RADIUS, lib_to_oracle_index, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib_system(kind, params):
    from paper_1306_2953_gb300 import api
    g_ora, H_ora, atoms, E = oracle_system(kind, *params)
    if kind == "box":
        n, h, _ = params
        lg = api.Grid.box(n, n, n, h)
        proj = None
    else:
        spec_r, spec_h = (params[0].radius, params[0].h) if kind == "mol" else (params[2], params[3])
        lg = api.Grid.spheres(atoms, spec_r, spec_h)
        r_c, r_cut = (params[0].r_c, params[0].r_cut) if kind == "mol" else (1.0, 3.0)
        proj = api.Projectors(lg, atoms, E, r_c, r_cut)
    idx = lib_to_oracle_index(g_ora, lg.ijk())
    H = api.Hamiltonian(lg, H_ora.V[idx], proj)
    return lg, H, g_ora, H_ora, idx


def _term_magnitudes(g_ora, H_ora, psi):
    """Oracle term magnitudes (M_loc, M_nl) of H psi at every element (see
    the module docstring): the oracle's own operator with every weight,
    potential value, coupling and projector value replaced by its absolute
    value, applied to |psi|."""
    from oracle import hamiltonian as oh
    a = np.abs(psi)
    zero = np.zeros(g_ora.npts)
    kin = oh.Hamiltonian(g_ora, zero, None, cw=np.abs(H_ora.cw)).apply(a)        # -1/(2h^2) sum |c||psi|
    pr = H_ora.proj
    pabs = oh.Projectors(pr.n_atoms, pr.sph_off, pr.sph_idx, np.abs(pr.gam), np.abs(pr.E))
    full = oh.Hamiltonian(g_ora, zero, pabs, cw=np.abs(H_ora.cw)).apply(a)
    m_loc = -kin + np.abs(H_ora.V)[:, None] * a
    return m_loc, full - kin


def _assert_elementwise_f32(out, ref, m_loc, m_nl):
    u = 2.0 ** -24
    bound = u * (32.0 * m_loc + 512.0 * m_nl)
    ratio = np.abs(out - ref) / bound
    assert np.all(np.isfinite(ratio)) and ratio.max() <= 1.0, f"worst element at {ratio.max():.3f} of the bound"


def _rel_err_per_state(got, ref):
    num = np.linalg.norm(got - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    return num / den


SYSTEMS = {
    "small_mol": ("atoms", (SMALL_ATOMS, SMALL_E, SMALL_RADIUS, SMALL_H)),
    "box17": ("box", (17, 0.3, 1.0)),
}


@pytest.mark.parametrize("system", list(SYSTEMS))
@pytest.mark.parametrize("nb", [1, 2, 4, 8, 16, 32, 64])
def test_hpsi_f64_parity(system, nb):
    kind, params = SYSTEMS[system]
    lg, H, g_ora, H_ora, idx = _lib_system(kind, params)
    psi_ora = wl.random_block(g_ora.npts, nb, 100 + nb)
    ref = H_ora.apply(psi_ora)[idx]
    psi = torch.from_numpy(np.ascontiguousarray(psi_ora[idx])).cuda()
    out = H.apply(psi).cpu().numpy()
    assert np.max(_rel_err_per_state(out, ref)) <= 1e-12


@pytest.mark.parametrize("system", list(SYSTEMS))
@pytest.mark.parametrize("nb", [4, 16, 32, 64])
def test_hpsi_f32_parity(system, nb):
    kind, params = SYSTEMS[system]
    lg, H, g_ora, H_ora, idx = _lib_system(kind, params)
    psi32 = wl.random_block(g_ora.npts, nb, 7).astype(np.float32)
    # the oracle sees the FP32 inputs exactly, the potential and projectors in FP64
    ref = H_ora.apply(psi32.astype(np.float64))[idx]
    psi = torch.from_numpy(np.ascontiguousarray(psi32[idx])).cuda()
    out = H.apply(psi).cpu().numpy().astype(np.float64)
    assert np.max(_rel_err_per_state(out, ref)) <= 2e-6
    smooth = wl.gaussian_sum_block(g_ora.coords, nb, 8).astype(np.float32)
    ref = H_ora.apply(smooth.astype(np.float64))[idx]
    out = H.apply(torch.from_numpy(np.ascontiguousarray(smooth[idx])).cuda()).cpu().numpy()
    assert np.max(_rel_err_per_state(out.astype(np.float64), ref)) <= 3e-5
    assert H.status() == 0


@pytest.mark.parametrize("ld,col0,nb", [(96, 32, 32), (96, 32, 64), (128, 64, 64), (36, 4, 32)])
def test_hpsi_f32_blocks_of_wide_psi(ld, col0, nb):
    """FP32 blocks that are column slices of a wider orbital array (the
    eigensolver's layout), including a slice whose rows start 16 bytes into a
    row; columns outside the block are left untouched."""
    kind, params = SYSTEMS["small_mol"]
    lg, H, g_ora, H_ora, idx = _lib_system(kind, params)
    psi32 = wl.random_block(g_ora.npts, ld, 21).astype(np.float32)
    full = torch.from_numpy(np.ascontiguousarray(psi32[idx])).cuda()
    out = torch.full_like(full, 7.0)
    H.apply(full[:, col0:col0 + nb], out[:, col0:col0 + nb], nb=nb)
    ref = H_ora.apply(psi32[:, col0:col0 + nb].astype(np.float64))[idx]
    o = out.cpu().numpy().astype(np.float64)
    assert np.max(_rel_err_per_state(o[:, col0:col0 + nb], ref)) <= 2e-6
    assert np.all(o[:, :col0] == 7.0) and np.all(o[:, col0 + nb:] == 7.0)
    assert H.status() == 0


def test_hpsi_f32_mol20_repeated_calls():
    """Repeated calls on one handle, one and two state groups: the kernel's
    work queue restarts cleanly on every call.  (The projection integrals are
    summed with atomics, so repeated results agree to rounding, not bitwise.)"""
    spec = wl.MOL20.system
    lg, H, g_ora, H_ora, idx = _lib_system("mol", (spec,))
    psi32 = wl.random_block(g_ora.npts, 64, 31).astype(np.float32)
    ref = H_ora.apply(psi32.astype(np.float64))[idx]
    psi = torch.from_numpy(np.ascontiguousarray(psi32[idx])).cuda()
    for _ in range(3):
        o = H.apply(psi, nb=32)[:, :32].cpu().numpy().astype(np.float64)
        assert np.max(_rel_err_per_state(o, ref[:, :32])) <= 2e-6
    for _ in range(2):
        o = H.apply(psi, nb=64).cpu().numpy().astype(np.float64)
        assert np.max(_rel_err_per_state(o, ref)) <= 2e-6
    assert H.status() == 0


def test_hpsi_f32_interleaved_handles():
    """Two Hamiltonians whose FP32 kernels need different shared memory
    (a molecule with projectors and a box without), applied alternately:
    the second handle's launch configuration must not break the first's."""
    spec = wl.MOL20.system
    lg_m, H_m, g_m, Ho_m, idx_m = _lib_system("mol", (spec,))
    lg_b, H_b, g_b, Ho_b, idx_b = _lib_system("box", (17, 0.3, 1.0))
    psi_m32 = wl.random_block(g_m.npts, 32, 41).astype(np.float32)
    psi_b32 = wl.random_block(g_b.npts, 32, 42).astype(np.float32)
    ref_m = Ho_m.apply(psi_m32.astype(np.float64))[idx_m]
    ref_b = Ho_b.apply(psi_b32.astype(np.float64))[idx_b]
    pm = torch.from_numpy(np.ascontiguousarray(psi_m32[idx_m])).cuda()
    pb = torch.from_numpy(np.ascontiguousarray(psi_b32[idx_b])).cuda()
    for H, p, ref in ((H_m, pm, ref_m), (H_b, pb, ref_b), (H_m, pm, ref_m), (H_b, pb, ref_b)):
        o = H.apply(p, nb=32).cpu().numpy().astype(np.float64)
        assert np.max(_rel_err_per_state(o, ref)) <= 3e-5
    assert H_m.status() == 0 and H_b.status() == 0


def test_hpsi_strided_block_and_untouched_columns():
    kind, params = SYSTEMS["small_mol"]
    lg, H, g_ora, H_ora, idx = _lib_system(kind, params)
    psi_ora = wl.random_block(g_ora.npts, 48, 3)
    full = torch.from_numpy(np.ascontiguousarray(psi_ora[idx])).cuda()
    out = torch.full_like(full, 7.0)
    H.apply(full[:, 16:32], out[:, 16:32], nb=16)
    ref = H_ora.apply(psi_ora[:, 16:32])[idx]
    o = out.cpu().numpy()
    assert np.max(_rel_err_per_state(o[:, 16:32], ref)) <= 1e-12
    assert np.all(o[:, :16] == 7.0) and np.all(o[:, 32:] == 7.0)


def test_hpsi_bad_arguments():
    from paper_1306_2953_gb300._lib import RsError
    kind, params = SYSTEMS["box17"]
    lg, H, g_ora, _, _ = _lib_system(kind, params)
    psi = torch.zeros((g_ora.npts, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(RsError):
        H.apply(psi, nb=3)
    with pytest.raises(RsError):
        H.apply(psi, psi)          # in place is rejected


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_hpsi_full_size_mol100(dtype):
    """The benchmark's workload (100 atoms, h=0.3, blocks of 32) at full size,
    on one block of 32 states, element by element against the oracle."""
    spec = wl.MOL100.system
    lg, H, g_ora, H_ora, idx = _lib_system("mol", (spec,))
    psi_ora = wl.random_block(g_ora.npts, 32, 55)
    if dtype == "f32":
        psi_ora = psi_ora.astype(np.float32).astype(np.float64)
    ref = H_ora.apply(psi_ora)[idx]
    t = torch.float64 if dtype == "f64" else torch.float32
    psi = torch.from_numpy(np.ascontiguousarray(psi_ora[idx])).to(t).cuda()
    out = H.apply(psi).double().cpu().numpy()
    tol = 1e-12 if dtype == "f64" else 2e-6
    assert np.max(_rel_err_per_state(out, ref)) <= tol
    if dtype == "f32":
        m_loc, m_nl = _term_magnitudes(g_ora, H_ora, psi_ora)
        _assert_elementwise_f32(out, ref, m_loc[idx], m_nl[idx])
    assert H.status() == 0


def test_hpsi_full_size_mol300_f32():
    """The 300-atom molecule (1.8 million points, the largest workload) at
    full size: one FP32 block of 32 states, per state and element by element."""
    spec = wl.MOL300.system
    lg, H, g_ora, H_ora, idx = _lib_system("mol", (spec,))
    psi_ora = wl.random_block(g_ora.npts, 32, 77).astype(np.float32).astype(np.float64)
    ref = H_ora.apply(psi_ora)[idx]
    psi = torch.from_numpy(np.ascontiguousarray(psi_ora[idx])).float().cuda()
    out = H.apply(psi).double().cpu().numpy()
    assert np.max(_rel_err_per_state(out, ref)) <= 2e-6
    m_loc, m_nl = _term_magnitudes(g_ora, H_ora, psi_ora)
    _assert_elementwise_f32(out, ref, m_loc[idx], m_nl[idx])
    assert H.status() == 0


def test_bounds_checked_build_runs_clean():
    """The debugging build (RS_BOUNDS_CHECK=1: every point index the FP32 ring
    kernel copies from or stores to is tested first, an index out of range is
    skipped and recorded in the status word) computes the same H psi with a
    clean status word, in a child process that loads that build."""
    import subprocess
    import sys
    from paper_1306_2953_gb300 import build
    lib = build.build(bounds_check=True)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = """
import numpy as np, torch, workloads as wl
from tests.helpers import lib_to_oracle_index, oracle_system
from paper_1306_2953_gb300 import api
s = wl.MOL20.system
g, Ho, atoms, E = oracle_system("mol", s)
lg = api.Grid.spheres(atoms, s.radius, s.h)
idx = lib_to_oracle_index(g, lg.ijk())
H = api.Hamiltonian(lg, Ho.V[idx], api.Projectors(lg, atoms, E, s.r_c, s.r_cut))
psi = wl.random_block(g.npts, 64, 5).astype(np.float32)
ref = Ho.apply(psi.astype(np.float64))[idx]
out = H.apply(torch.from_numpy(np.ascontiguousarray(psi[idx])).cuda()).double().cpu().numpy()
err = np.max(np.linalg.norm(out - ref, axis=0) / np.linalg.norm(ref, axis=0))
assert err <= 2e-6 and H.status() == 0, (err, H.status())
print("checked build ok", err)
"""
    env = dict(os.environ, RSDFT_LIB=lib, PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "checked build ok" in r.stdout, r.stdout + r.stderr
