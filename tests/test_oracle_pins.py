"""Pins of the FP64 oracle against what the mathematics fixes.

Each test checks the oracle against something other than itself: closed
forms (finite-difference weights, stencil symbols, the Kronecker-sum
spectrum of a separable Hamiltonian, harmonic-oscillator levels), exact
integer enumeration, invariants (Hermiticity, positivity and rank of the
nonlocal term, orthonormality) and library routines applied to the same
mathematical object (dense eigensolvers, Cholesky, linear solves).
"""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

import workloads as wl
from oracle import eigensolver, grid as og, hamiltonian as oh, linalg as ol, precond as op, stencil as os_


# ---------------------------------------------------------------- stencil ---

def closed_form_weights(m):
    """Central 2nd-derivative weights, closed form (Fornberg 1988):
    c_j = 2 (-1)^(j+1) (m!)^2 / (j^2 (m-j)! (m+j)!),  c_0 = -2 sum_j c_j."""
    c = [Fraction(2 * (-1) ** (j + 1) * factorial(m) ** 2, j * j * factorial(m - j) * factorial(m + j))
         for j in range(1, m + 1)]
    return [-2 * sum(c)] + c


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6])
def test_fd_weights_closed_form(m):
    assert os_.fd_weights_exact(m) == closed_form_weights(m)


def test_fd_weights_golden():
    # tests/golden/fd_weights_m4.txt: the 25-point (half-width 4) weights
    lines = [l for l in open(__file__.replace("test_oracle_pins.py", "golden/fd_weights_m4.txt"))
             if l.strip() and not l.startswith("#")]
    gold = [Fraction(l.split()[1]) for l in lines]
    assert os_.fd_weights_exact(4) == gold


# ------------------------------------------------------------------- grid ---

def test_single_sphere_count_exact():
    # atom on a lattice point, dyadic h and R: FP64 arithmetic is exact
    for h, R in [(0.5, 1.0), (0.5, 1.5), (0.25, 1.0), (0.5, 2.0)]:
        g = og.sphere_union_grid(np.zeros((1, 3)), R, h)
        n = int(round(R / h))
        brute = sum(1 for i in range(-n, n + 1) for j in range(-n, n + 1) for k in range(-n, n + 1)
                    if (i * i + j * j + k * k) * h * h <= R * R)
        assert g.npts == brute
    # lattice points of norm^2 <= 1, 2, 4 in Z^3 (sphere of radius h, sqrt2 h, 2h)
    assert og.sphere_union_grid(np.zeros((1, 3)), 0.5, 0.5).npts == 7
    assert og.sphere_union_grid(np.zeros((1, 3)), 1.0, 0.5).npts == 33


def test_union_grid_bruteforce_exact_rationals():
    atoms = np.array([[0.25, 0.5, -0.75], [1.5, 0.0, 0.25], [0.5, 1.25, 1.0]])
    h, R = 0.25, 1.0
    g = og.sphere_union_grid(atoms, R, h)
    A = [[Fraction(v) for v in a] for a in atoms]
    hF, RF = Fraction(h), Fraction(R)
    pts = set()
    for i in range(-10, 12):
        for j in range(-10, 12):
            for k in range(-10, 12):
                r = (i * hF, j * hF, k * hF)
                if any(sum((r[d] - a[d]) ** 2 for d in range(3)) <= RF * RF for a in A):
                    pts.add((i, j, k))
    assert set(map(tuple, g.ijk.tolist())) == pts
    # lexicographic order and a consistent map
    assert np.all(np.diff(g.ijk[:, 0]) >= 0)
    assert np.array_equal(g.lookup(g.ijk), np.arange(g.npts))


def test_box_grid():
    g = og.box_grid(5, 0.3)
    assert g.npts == 125
    assert np.allclose(g.coords.sum(axis=0), 0.0)
    assert np.isclose(g.coords[:, 0].max(), 0.6)


# ---------------------------------------------------------------- kinetic ---

def kinetic_only(grid, m=4):
    return oh.Hamiltonian(grid, np.zeros(grid.npts), None, m=m)


def interior(grid, n, w=4):
    i = grid.ijk
    return np.all((i >= w) & (i < n - w), axis=1)


def test_polynomial_exactness():
    n, h = 20, 0.25
    g = og.box_grid(n, h)
    x, y, z = g.coords.T
    psi = x ** 9 + 3 * x ** 4 * y ** 5 - z ** 8 + x * y * z + 2.0
    lap = 72 * x ** 7 + 3 * (12 * x ** 2 * y ** 5 + 20 * x ** 4 * y ** 3) - 56 * z ** 6
    T = kinetic_only(g).apply(psi)
    m = interior(g, n)
    err = np.abs(T[m] - (-0.5 * lap[m])).max() / np.abs(lap[m]).max()
    assert err < 1e-11
    # degree 10 is not reproduced: the check has teeth
    T10 = kinetic_only(g).apply(x ** 10)
    assert np.abs(T10[m] - (-0.5 * 90 * x[m] ** 8)).max() > 1e-6


def test_plane_wave_symbol_interior():
    n, h = 16, 0.3
    g = og.box_grid(n, h)
    k = np.array([0.7, -1.3, 2.1])
    psi = np.cos(g.coords @ k + 0.4)
    c = closed_form_weights(4)
    lam = -0.5 / h ** 2 * sum(float(c[0]) + 2 * sum(float(c[j]) * np.cos(j * ka * h) for j in range(1, 5))
                              for ka in k)
    T = kinetic_only(g).apply(psi)
    m = interior(g, n)
    assert np.abs(T[m] - lam * psi[m]).max() < 1e-11 * abs(lam)


def test_seven_point_sine_modes_whole_box():
    # half-width 1: sine modes are exact eigenvectors with zero boundaries
    n, h = 9, 0.4
    g = og.box_grid(n, h)
    H = oh.Hamiltonian(g, np.zeros(g.npts), None, m=1)
    for modes in [(1, 1, 1), (2, 1, 3), (4, 5, 2)]:
        psi = np.ones(g.npts)
        lam = 0.0
        for a, na in enumerate(modes):
            psi *= np.sin(np.pi * na * (g.ijk[:, a] + 1) / (n + 1))
            lam += (1 - np.cos(np.pi * na / (n + 1))) / h ** 2
        assert np.abs(H.apply(psi) - lam * psi).max() < 1e-12 * lam


# ------------------------------------------------- separable spectrum (P1) ---

def one_d_levels(n, h, omega):
    c = closed_form_weights(4)
    x = (np.arange(n) - (n - 1) / 2) * h
    T = np.zeros((n, n))
    for i in range(n):
        for j in range(-4, 5):
            if 0 <= i + j < n:
                T[i, i + j] += -0.5 * float(c[abs(j)]) / h ** 2
    w, v = np.linalg.eigh(T + np.diag(0.5 * omega ** 2 * x ** 2))
    return w, v


def test_separable_spectrum_dense():
    n, h, om = 7, 0.45, 1.0
    g = og.box_grid(n, h)
    H = oh.Hamiltonian(g, wl.harmonic_potential(g.coords, om))
    M = H.dense()
    assert np.abs(M - M.T).max() < 1e-12
    e1, _ = one_d_levels(n, h, om)
    expect = np.sort((e1[:, None, None] + e1[None, :, None] + e1[None, None, :]).ravel())
    assert np.abs(np.linalg.eigvalsh(M) - expect).max() < 1e-10
    wj, vj = ol.jacobi_eigh(M)
    assert np.abs(wj - expect).max() < 1e-10
    assert np.abs(M @ vj - vj * wj).max() < 1e-9


def test_harmonic_oscillator_block_cg():
    # the 32^3, h=0.3 oscillator; 16 states, lowest 10 judged
    w = wl.HO32
    g = og.box_grid(w.system.n, w.system.h)
    H = oh.Hamiltonian(g, wl.harmonic_potential(g.coords, w.system.omega))
    psi0 = wl.random_block(g.npts, w.n_states, w.seed)
    solver = eigensolver.BlockCG(H, psi0, w.block, tol=1e-7)
    eps = solver.solve(max_iter=400, judged=w.judged)
    e1, _ = one_d_levels(w.system.n, w.system.h, w.system.omega)
    expect = np.sort((e1[:, None, None] + e1[None, :, None] + e1[None, None, :]).ravel())[:w.judged]
    assert np.abs(eps - expect).max() < 1e-9
    # analytic (n + 3/2) omega with degeneracies 1, 3, 6 within discretisation error
    analytic = np.array([1.5] + [2.5] * 3 + [3.5] * 6)
    assert np.abs(eps - analytic).max() < 1e-4


# ------------------------------------------------------------ projectors ---

def small_molecule(h=0.4, R=3.0):
    atoms = np.array([[0.0, 0.0, 0.0], [1.9, 0.3, -0.2], [0.4, 1.7, 0.8]])
    g = og.sphere_union_grid(atoms, R, h)
    E = np.array([[1.3, 0.7], [0.5, 1.9], [1.1, 1.4]])
    pr = oh.make_projectors(g, atoms, E, 1.0, 3.0)
    V = wl.local_potential(g.coords, atoms)
    return g, oh.Hamiltonian(g, V, pr), atoms, E


def test_hermiticity_with_overlapping_projectors():
    g, H, _, _ = small_molecule()
    rng = np.random.default_rng(5)
    phi = rng.standard_normal((g.npts, 3))
    psi = rng.standard_normal((g.npts, 3))
    a = phi.T @ H.apply(psi)
    b = H.apply(phi).T @ psi
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


def test_projector_normalisation_and_kb_eigen():
    h = 0.3
    g = og.sphere_union_grid(np.zeros((1, 3)), 4.0, h)
    E = np.array([[1.7, 0.6]])
    pr = oh.make_projectors(g, np.zeros((1, 3)), E, 1.0, 3.0)
    gm = pr.gamma(0)
    Gram = g.dV * gm @ gm.T
    assert np.abs(Gram - np.eye(4)).max() < 1e-13     # atom on a lattice point: s, p orthonormal
    H = oh.Hamiltonian(g, np.zeros(g.npts), pr)
    for q in range(4):
        v = np.zeros(g.npts)
        v[pr.points(0)] = gm[q]
        out = H.apply(v) - H.apply(v, local_only=True)
        assert np.abs(out - E[0, 0 if q == 0 else 1] * v).max() < 1e-12


def test_projector_sphere_lists_exact():
    # dyadic atoms, h and r_cut: FP64 distances are exact, so the point list
    # of each projector sphere is the exact lattice set d^2 <= r_cut^2
    atoms = np.array([[0.25, 0.5, -0.75], [1.5, 0.0, 0.25]])
    h, R, r_cut = 0.25, 1.5, 1.0
    g = og.sphere_union_grid(atoms, R, h)
    pr = oh.make_projectors(g, atoms, np.ones((2, 2)), 1.0, r_cut)
    hF, rF = Fraction(h), Fraction(r_cut)
    for A, a in enumerate(atoms):
        aF = [Fraction(v) for v in a]
        want = sorted(p for p, ijk in enumerate(g.ijk.tolist())
                      if sum((ijk[d] * hF - aF[d]) ** 2 for d in range(3)) <= rF * rF)
        assert pr.points(A).tolist() == want
        on_sphere = sum(1 for ijk in g.ijk.tolist()
                        if sum((ijk[d] * hF - aF[d]) ** 2 for d in range(3)) == rF * rF)
        assert on_sphere > 0          # the boundary case is exercised


def test_nonlocal_psd_rank_and_dense_agree():
    g, H, atoms, _ = small_molecule(h=0.5, R=2.5)
    n = g.npts
    eye = np.eye(n)
    Vnl_apply = H.apply(eye) - H.apply(eye, local_only=True)
    Vnl = H.nonlocal_dense()
    assert np.abs(Vnl_apply - Vnl).max() < 1e-12
    w = np.linalg.eigvalsh(Vnl)
    assert w.min() > -1e-12
    assert np.sum(w > 1e-9) <= 4 * len(atoms)


# ---------------------------------------------------------- linear algebra ---

def test_cholesky_triinv_against_library():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 25))
    S = A.T @ A
    U = ol.cholesky_upper(S)
    assert np.abs(U - np.linalg.cholesky(S).T).max() < 1e-12
    Ui = ol.tri_inv_upper(U)
    assert np.abs(Ui - np.linalg.inv(U)).max() < 1e-10
    with pytest.raises(ol.NotPositiveDefinite):
        ol.cholesky_upper(-S)


def test_overlap_is_the_grid_integral():
    # <g|g> = dV sum g^2 for g = exp(-r^2/2) on a fine box is the integral of
    # exp(-r^2), pi^(3/2) (the lattice sum of a Gaussian converges
    # exponentially in 1/h; the box edge at 4.9 Bohr cuts off e^-24)
    g = og.box_grid(40, 0.25)
    r2 = np.sum(g.coords ** 2, axis=1)
    f = np.exp(-0.5 * r2)[:, None]
    assert abs(ol.overlap(f, f, g.dV)[0, 0] - np.pi ** 1.5) < 1e-9
    # and x exp(-r^2/2) is orthogonal to it, with norm pi^(3/2) / 2
    fx = (g.coords[:, 0] * np.exp(-0.5 * r2))[:, None]
    S = ol.overlap(np.hstack([f, fx]), np.hstack([f, fx]), g.dV)
    assert abs(S[0, 1]) < 1e-12 and abs(S[1, 1] - np.pi ** 1.5 / 2) < 1e-9


def test_orthonormalize_invariants():
    g, H, _, _ = small_molecule()
    psi = wl.random_block(g.npts, 12, 3)
    out, Ui = ol.orthonormalize(psi, g.dV)
    assert np.abs(ol.overlap(out, out, g.dV) - np.eye(12)).max() < 1e-13
    # span unchanged: psi is reproduced by its projection on the new set
    proj = out @ ol.overlap(out, psi, g.dV)
    assert np.abs(proj - psi).max() < 1e-12 * np.abs(psi).max()


def test_rayleigh_ritz_on_exact_separable_eigenvectors():
    n, h = 10, 0.35
    g = og.box_grid(n, h)
    H = oh.Hamiltonian(g, wl.harmonic_potential(g.coords, 1.0))
    e1, v1 = one_d_levels(n, h, 1.0)
    idx = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (2, 0, 0)]
    cols = [np.einsum("i,j,k->ijk", v1[:, a], v1[:, b], v1[:, c]).ravel() for a, b, c in idx]
    psi = np.stack(cols, axis=1) / np.sqrt(g.dV)
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    psi = psi @ Q                          # rotate inside the subspace
    eps, _, _, _ = ol.subspace_diag(H.apply, psi, g.dV)
    expect = np.sort([e1[a] + e1[b] + e1[c] for a, b, c in idx])
    assert np.abs(eps - expect).max() < 1e-11


def test_rayleigh_ritz_vectors_are_exact_eigenvectors():
    # a rotated set of exact (non-degenerate) separable eigenvectors: the Ritz
    # vectors must be those eigenvectors again, H phi_k = eps_k phi_k
    n, h = 10, 0.35
    g = og.box_grid(n, h)
    H = oh.Hamiltonian(g, wl.harmonic_potential(g.coords, 1.0) + 0.05 * g.coords[:, 0] ** 2)
    ex, vx = one_d_levels(n, h, np.sqrt(1.1))   # V_x = 1.1 x^2 / 2
    e1, v1 = one_d_levels(n, h, 1.0)
    idx = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (2, 0, 0), (1, 1, 0)]
    cols = [np.einsum("i,j,k->ijk", vx[:, a], v1[:, b], v1[:, c]).ravel() for a, b, c in idx]
    psi = np.stack(cols, axis=1) / np.sqrt(g.dV)
    Q, _ = np.linalg.qr(np.random.default_rng(4).standard_normal((5, 5)))
    eps, phi, hphi, _ = ol.subspace_diag(H.apply, psi @ Q, g.dV)
    expect = np.sort([ex[a] + e1[b] + e1[c] for a, b, c in idx])
    assert np.abs(eps - expect).max() < 1e-11
    Hphi = H.apply(phi)
    assert np.abs(Hphi - phi * eps).max() < 1e-9 * np.abs(Hphi).max()
    assert np.abs(hphi - Hphi).max() < 1e-9 * np.abs(Hphi).max()


def test_tiny_molecule_dense_vs_block_cg():
    atoms = np.array([[0.0, 0.0, 0.0], [1.8, 0.0, 0.0]])
    g = og.sphere_union_grid(atoms, 2.5, 0.6)
    pr = oh.make_projectors(g, atoms, np.array([[1.0, 0.8], [1.5, 0.6]]), 1.0, 3.0)
    H = oh.Hamiltonian(g, wl.local_potential(g.coords, atoms), pr)
    M = H.dense()
    ref = np.linalg.eigvalsh(M)
    wj, _ = ol.jacobi_eigh(M)
    assert np.abs(wj - ref).max() < 1e-10
    solver = eigensolver.BlockCG(H, wl.random_block(g.npts, 8, 2), 4, tol=1e-9)
    eps = solver.solve(max_iter=500)
    assert np.abs(eps - ref[:8]).max() < 1e-9


def test_filter_preconditioner_symmetric():
    g, _, _, _ = small_molecule()
    K = eigensolver.FilterPreconditioner(g)
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal((2, g.npts, 2))
    assert abs(np.sum(a * K(b)) - np.sum(K(a) * b)) < 1e-12 * np.sum(np.abs(a * b))
    # a constant is unchanged where all six face neighbours are grid points
    one = np.ones((g.npts, 1))
    full = np.all(g.neighbours(1).reshape(g.npts, 6) >= 0, axis=1)
    assert np.abs(K(one)[full] - 1).max() < 1e-15


# ------------------------------------------------------ CG and conv net ---

def test_cg_converges_to_direct_solve():
    atoms = np.array([[0.0, 0.0, 0.0]])
    g = og.sphere_union_grid(atoms, 1.5, 0.5)
    r = wl.random_block(g.npts, 2, 9)
    x = op.shifted_poisson_cg(g, r, sigma=1.0, n_iter=200)
    A = oh.Hamiltonian(g, np.full(g.npts, 1.0)).dense()
    assert np.abs(x - np.linalg.solve(A, r)).max() < 1e-10


def test_cg_iterate_is_krylov_minimiser():
    # after k steps CG minimises the A-norm error over the Krylov space K_k(A, r)
    atoms = np.array([[0.0, 0.0, 0.0]])
    g = og.sphere_union_grid(atoms, 2.0, 0.5)
    r = wl.random_block(g.npts, 1, 4)[:, 0]
    A = oh.Hamiltonian(g, np.full(g.npts, 1.0)).dense()
    k = 6
    x = op.shifted_poisson_cg(g, r[:, None], n_iter=k)[:, 0]
    K = np.stack([np.linalg.matrix_power(A, j) @ r for j in range(k)], axis=1)
    Q, _ = np.linalg.qr(K)
    y = np.linalg.solve(Q.T @ A @ Q, Q.T @ r)
    assert np.abs(x - Q @ y).max() < 1e-8 * np.abs(x).max()


def brute_conv(x, w):
    B, ci, X, Y, Z = x.shape
    co = w.shape[0]
    y = np.zeros((B, co, X, Y, Z))
    for b in range(B):
        for o in range(co):
            for i in range(X):
                for j in range(Y):
                    for k in range(Z):
                        s = 0.0
                        for c in range(ci):
                            for a in range(3):
                                for bb in range(3):
                                    for cc in range(3):
                                        ii, jj, kk = i + a - 1, j + bb - 1, k + cc - 1
                                        if 0 <= ii < X and 0 <= jj < Y and 0 <= kk < Z:
                                            s += w[o, c, a, bb, cc] * x[b, c, ii, jj, kk]
                        y[b, o, i, j, k] = s
    return y


def test_conv3_bruteforce():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 2, 4, 5, 3))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    assert np.abs(op.conv3(x, w) - brute_conv(x, w)).max() < 1e-12


def test_net_gradients_finite_difference():
    rng = np.random.default_rng(1)
    ws = [w.astype(np.float64) for w in wl.conv_init(7, channels=3)]
    shape = (2, 6, 6, 6)
    xhat = rng.standard_normal(shape)
    mask = rng.uniform(size=shape) > 0.2
    target = rng.standard_normal(shape)
    valid = np.zeros(shape)
    valid[:, 1:5, 1:5, 1:5] = mask[:, 1:5, 1:5, 1:5]

    def loss(wl_):
        y, _ = op.net_forward(xhat, mask, wl_)
        return op.tile_loss(y, target, valid)[0]

    y, cache = op.net_forward(xhat, mask, ws)
    _, gy = op.tile_loss(y, target, valid)
    grads = op.net_backward(gy, cache, ws)
    for li in range(3):
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in ws[li].shape)
            e = 1e-6
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[li][idx] += e
            wm[li][idx] -= e
            fd = (loss(wp) - loss(wm)) / (2 * e)
            assert abs(fd - grads[li][idx]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9


def linear_stencil_net(K, channels=8):
    """Weights for which the bias-free ReLU net computes the linear stencil K
    (3x3x3 cross-correlation): channel 0 carries relu(x), channel 1
    relu(-x), and relu(x) - relu(-x) = x."""
    w0 = np.zeros((channels, 1, 3, 3, 3))
    w1 = np.zeros((channels, channels, 3, 3, 3))
    w2 = np.zeros((1, channels, 3, 3, 3))
    w0[0, 0, 1, 1, 1], w0[1, 0, 1, 1, 1] = 1.0, -1.0
    w1[0, 0, 1, 1, 1] = w1[1, 1, 1, 1, 1] = 1.0
    w2[0, 0], w2[0, 1] = K, -K
    return [w0, w1, w2]


def test_learned_net_reproduces_linear_stencils():
    # on a sphere-union grid (points off the grid are zero): the filter
    # kernel gives the plain filter preconditioner, a one-point kernel gives
    # the neighbour at that offset from the grid's own neighbour table
    g, _, _, _ = small_molecule()
    R = wl.random_block(g.npts, 3, 12)
    a = 0.5
    Kf = np.zeros((3, 3, 3))
    Kf[1, 1, 1] = a
    for d in range(3):
        for s in (0, 2):
            idx = [1, 1, 1]
            idx[d] = s
            Kf[tuple(idx)] = (1 - a) / 6
    ref = eigensolver.FilterPreconditioner(g, a)(R)
    assert np.abs(op.apply_learned(g, R, linear_stencil_net(Kf)) - ref).max() < 1e-14 * np.abs(ref).max()
    nbr = g.neighbours(1)                      # [np, 3, 2]: offsets -1, +1 per axis
    for axis in range(3):
        for t, off in enumerate((-1, 1)):
            Ks = np.zeros((3, 3, 3))
            idx = [1, 1, 1]
            idx[axis] = 1 + off
            Ks[tuple(idx)] = 1.0
            q = nbr[:, axis, t]
            want = np.where((q >= 0)[:, None], R[np.maximum(q, 0)], 0.0)
            assert np.abs(op.apply_learned(g, R, linear_stencil_net(Ks)) - want).max() < 1e-14


def test_bf16_round_matches_library():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(2).standard_normal(10000).astype(np.float32) * 100
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(op.bf16_round(x), ref)
    # exact ties (low 16 bits 0x8000) round to the even neighbour
    hi = np.array([0x3F80, 0x3F81, 0xBF80, 0xBF81, 0x4049, 0x404A, 0x0001, 0x7F7E], dtype=np.uint32)
    for low in (0x8000, 0x7FFF, 0x8001):
        t = ((hi << 16) | low).view(np.float32)
        ref = torch.from_numpy(t.copy()).to(torch.bfloat16).float().numpy()
        assert np.array_equal(op.bf16_round(t), ref), hex(low)


def test_adam_first_step_is_signed_lr():
    # with bias correction, the first Adam step is lr * g / (|g| + eps')
    p = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -4.0, 1e-3])]
    out = op.Adam(p).step(p, g)[0]
    assert np.allclose(out, p[0] - 1e-3 * g[0] / (np.abs(g[0]) + 1e-8), rtol=0, atol=1e-12)


def test_adam_constant_gradient_closed_form():
    # A constant gradient g makes the bias-corrected moments exact at every
    # step: m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so m_hat = g and
    # v_hat = g^2, and after t steps w_t = w_0 - t lr g / (|g| + eps).
    w0 = np.array([1.0, -2.0, 0.5, 0.0])
    g = np.array([0.3, -4.0, 1e-3, 2.5])
    opt = op.Adam([w0], lr=1e-3)
    p = [w0]
    for t in range(1, 8):
        p = opt.step(p, [g])
        assert np.allclose(p[0], w0 - t * 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12), t


def test_adam_alternating_gradient_closed_form():
    # Gradients g, -g, g, ...: the first moment follows
    #   m_t = b1 m_{t-1} + (1 - b1) (-1)^(t+1) g
    #       = (1 - b1) g (-1)^(t+1) (1 - (-b1)^t) / (1 + b1),
    # the second stays v_t = (1 - b2^t) g^2; each step moves w by
    #   -lr (m_t / (1 - b1^t)) / (|g| + eps).
    b1, b2, lr, eps = 0.9, 0.999, 1e-3, 1e-8
    w0 = np.array([0.7, -1.3, 2.0])
    g = np.array([0.5, -2.0, 3e-2])
    opt = op.Adam([w0], lr=lr, b1=b1, b2=b2, eps=eps)
    p, w = [w0], w0.copy()
    for t in range(1, 9):
        p = opt.step(p, [(-1.0) ** (t + 1) * g])
        m = (1 - b1) * g * (-1.0) ** (t + 1) * (1 - (-b1) ** t) / (1 + b1)
        w = w - lr * (m / (1 - b1 ** t)) / (np.sqrt((1 - b2 ** t) * g * g / (1 - b2 ** t)) + eps)
        assert np.allclose(p[0], w, rtol=0, atol=1e-12), t


# ---------------------------------------------------------------- RMM-DIIS ---

def test_diis_coefficients_minimise_the_residual_quotient():
    # The DIIS combination minimises <rbar|rbar> / <xbar|xbar> over the span
    # of the iterates: its quotient is the lowest eigenvalue of the pencil
    # (A, B) (the library's generalized symmetric eigensolver), normalised
    # to <xbar|xbar> = 1 with a non-negative coefficient sum.
    import scipy.linalg as sla
    rng = np.random.default_rng(3)
    for k in (2, 3, 4):
        X = rng.standard_normal((50, k))
        R = rng.standard_normal((50, k)) * np.array([1.0, 0.3, 0.1, 0.05][:k])
        A, B = R.T @ R, X.T @ X
        a = eigensolver.diis_coefficients(A, B)
        lowest = sla.eigh(A, B, eigvals_only=True)[0]
        assert abs(a @ A @ a / (a @ B @ a) - lowest) <= 1e-12 * max(1.0, abs(lowest))
        assert abs(a @ B @ a - 1.0) <= 1e-12 and a.sum() >= 0
        # no other combination does better
        for _ in range(200):
            c = rng.standard_normal(k)
            assert c @ A @ c / (c @ B @ c) >= lowest - 1e-12


def test_rayleigh_trial_step_minimises_the_quotient():
    # lambda from the 2x2 pencil minimises the Rayleigh quotient of x + lambda p
    rng = np.random.default_rng(4)
    M = rng.standard_normal((30, 30))
    Hm = M + M.T
    for _ in range(5):
        x, p = rng.standard_normal(30), rng.standard_normal(30)
        hx, hp = Hm @ x, Hm @ p
        lam = eigensolver.rayleigh_step(x @ x, x @ p, p @ p, x @ hx, x @ hp, p @ hp)
        rq = lambda t: (x + t * p) @ Hm @ (x + t * p) / ((x + t * p) @ (x + t * p))
        for d in (1e-3, -1e-3, 0.1, -0.1, 1.0, -1.0):
            assert rq(lam) <= rq(lam + d) + 1e-12


def test_harmonic_oscillator_rmm_diis():
    # the paper's eigensolver on the separable oscillator (a 20^3 box with the
    # same spacing, 16 states, lowest 10): the Kronecker-sum spectrum (P1)
    n, h, om = 20, 0.3, 1.0
    g = og.box_grid(n, h)
    H = oh.Hamiltonian(g, wl.harmonic_potential(g.coords, om))
    solver = eigensolver.RMMDIIS(H, wl.random_block(g.npts, 16, 5), 16, tol=1e-8)
    eps = solver.solve(max_iter=300, judged=10)
    e1, _ = one_d_levels(n, h, om)
    expect = np.sort((e1[:, None, None] + e1[None, :, None] + e1[None, None, :]).ravel())[:10]
    assert np.abs(eps - expect).max() < 1e-9


def test_tiny_molecule_dense_vs_rmm_diis():
    # P8 for the paper's eigensolver: dense diagonalisation of a tiny
    # two-atom grid with projectors against RMM-DIIS
    atoms = np.array([[0.0, 0.0, 0.0], [1.8, 0.0, 0.0]])
    g = og.sphere_union_grid(atoms, 2.5, 0.6)
    pr = oh.make_projectors(g, atoms, np.array([[1.0, 0.8], [1.5, 0.6]]), 1.0, 3.0)
    H = oh.Hamiltonian(g, wl.local_potential(g.coords, atoms), pr)
    ref = np.linalg.eigvalsh(H.dense())
    solver = eigensolver.RMMDIIS(H, wl.random_block(g.npts, 8, 2), 4, tol=1e-9)
    eps = solver.solve(max_iter=500)
    assert np.abs(eps - ref[:8]).max() < 1e-9


def test_rmm_diis_two_steps_against_brute_force():
    # One state, identity preconditioner, two RMM-DIIS steps on a tiny
    # oscillator box, rebuilt from the method's definition with brute-force
    # one-dimensional minimisations instead of the oracle's 2x2 and DIIS
    # eigenproblems: lambda minimises the Rayleigh quotient of x0 + t r0;
    # alpha minimises |a0 r0 + a1 r1| / |a0 x0 + a1 x1| over directions
    # (a0, a1) = (cos th, sin th); x2 = xbar + lambda rbar.
    from scipy.optimize import minimize_scalar
    g = og.box_grid(5, 0.5)
    H = oh.Hamiltonian(g, wl.harmonic_potential(g.coords, 1.0))
    Hd = H.dense()
    dV = g.dV
    x0 = wl.random_block(g.npts, 1, 8)[:, 0]
    x0 = x0 / np.sqrt(dV * x0 @ x0)
    dot = lambda a, b: dV * (a @ b)
    rq = lambda v: dot(v, Hd @ v) / dot(v, v)
    r0 = Hd @ x0 - rq(x0) * x0
    ts = np.linspace(-20, 20, 40001)
    t0 = ts[np.argmin([rq(x0 + t * r0) for t in ts])]
    lam = minimize_scalar(lambda t: rq(x0 + t * r0), bracket=(t0 - 1e-3, t0, t0 + 1e-3), tol=1e-14).x
    x1 = x0 + lam * r0
    r1 = Hd @ x1 - rq(x1) * x1
    quot = lambda th: (dot(np.cos(th) * r0 + np.sin(th) * r1, np.cos(th) * r0 + np.sin(th) * r1)
                       / dot(np.cos(th) * x0 + np.sin(th) * x1, np.cos(th) * x0 + np.sin(th) * x1))
    thg = np.linspace(0, np.pi, 20001)
    th0 = thg[np.argmin([quot(t) for t in thg])]
    th = minimize_scalar(quot, bracket=(th0 - 1e-3, th0, th0 + 1e-3), tol=1e-14).x
    a0, a1 = np.cos(th), np.sin(th)
    x2 = (a0 * x0 + a1 * x1) + lam * (a0 * r0 + a1 * r1)
    solver = eigensolver.RMMDIIS(H, x0[:, None], 1, precond=lambda R: R.copy(), tol=0.0, n_steps=2)
    solver.step()
    got = solver.Psi[:, 0]
    cosang = abs(dot(got, x2)) / np.sqrt(dot(got, got) * dot(x2, x2))
    assert 1.0 - cosang < 1e-10


# -------------------------------------------------------- Hartree (FFT) ---

def _gaussian_box(sigma, h, half):
    n = int(round(2 * half / h)) + 1
    g = og.box_grid(n, h)
    r = np.linalg.norm(g.coords, axis=1)
    rho = np.exp(-r * r / (2 * sigma * sigma)) / (2 * np.pi * sigma * sigma) ** 1.5
    return g, r, rho


def test_hartree_gaussian_closed_form():
    # a normalised Gaussian charge of width sigma has the potential
    # erf(r / (sqrt(2) sigma)) / r (sqrt(2/pi) / sigma at r = 0)
    from scipy.special import erf
    from oracle import poisson as op
    sigma, h = 1.0, 0.25
    g, r, rho = _gaussian_box(sigma, h, 6.5)
    V = op.hartree(g, rho)
    with np.errstate(invalid="ignore", divide="ignore"):
        ref = np.where(r > 0, erf(r / (np.sqrt(2) * sigma)) / r, np.sqrt(2 / np.pi) / sigma)
    assert np.abs(V - ref).max() <= 1e-9 * ref.max()


def test_hartree_two_charges_and_symmetry():
    # two Gaussians of opposite sign at +-a along an axis: the potential is
    # the sum of the two closed forms, odd under the mirror x -> -x
    from scipy.special import erf
    from oracle import poisson as op
    sigma, h, a = 0.8, 0.25, 1.5
    n = 53
    g = og.box_grid(n, h)
    x = g.coords
    rp = np.linalg.norm(x - np.array([a, 0, 0]), axis=1)
    rm = np.linalg.norm(x + np.array([a, 0, 0]), axis=1)
    gau = lambda r: np.exp(-r * r / (2 * sigma * sigma)) / (2 * np.pi * sigma * sigma) ** 1.5
    V = op.hartree(g, gau(rp) - gau(rm))
    pot = lambda r: np.where(r > 0, erf(r / (np.sqrt(2) * sigma)) / np.where(r > 0, r, 1), np.sqrt(2 / np.pi) / sigma)
    ref = pot(rp) - pot(rm)
    assert np.abs(V - ref).max() <= 1e-7
    mirror = g.lookup(g.ijk * np.array([-1, 1, 1]) + np.array([n - 1, 0, 0]))
    assert np.abs(V + V[mirror]).max() <= 1e-10


def test_smooth_sizes():
    from oracle import poisson as op
    assert [op.smooth_size(n) for n in (1, 5, 7, 10, 17, 100, 289)] == [1, 6, 8, 12, 18, 108, 324]


# ------------------------------------------------------ SCF, LDA, mixing ---

def test_lda_potential_is_the_density_derivative():
    # v_xc = d(n e_xc)/dn, by central differences, on both branches of the
    # Perdew-Zunger correlation (r_s above and below 1)
    from oracle import scf as osc
    n = np.geomspace(1e-4, 20.0, 400)
    d = 1e-6 * n
    exc_p, _ = osc.lda_xc(n + d)
    exc_m, _ = osc.lda_xc(n - d)
    fd = ((n + d) * exc_p - (n - d) * exc_m) / (2 * d)
    _, vxc = osc.lda_xc(n)
    assert np.abs(fd - vxc).max() <= 1e-6 * np.abs(vxc).max()


def test_lda_exchange_and_correlation_limits():
    from oracle import scf as osc
    # Slater exchange of the uniform gas: e_x r_s = -(3/4)(9/(4 pi^2))^(1/3)
    rs = np.array([0.5, 1.0, 2.0, 5.0])
    n = 3.0 / (4.0 * np.pi * rs ** 3)
    exc, _ = osc.lda_xc(n)
    ex = exc - _pz_ec(rs)
    assert np.allclose(ex * rs, -0.75 * (9.0 / (4.0 * np.pi ** 2)) ** (1.0 / 3.0), rtol=1e-12, atol=0)
    # the two Perdew-Zunger branches meet at r_s = 1 (value and slope)
    e1, e2 = osc.lda_xc(np.array([3.0 / (4.0 * np.pi) * (1 - 1e-9) ** -3, 3.0 / (4.0 * np.pi) * (1 + 1e-9) ** -3]))[0]
    assert abs(e1 - e2) < 5e-5
    assert np.all(osc.lda_xc(np.array([0.0, -1.0]))[0] == 0.0)


def _pz_ec(rs):
    # the published Perdew-Zunger 1981 fit of the Ceperley-Alder correlation
    # energy (unpolarised), written out independently for the exchange check
    return np.where(rs >= 1, -0.1423 / (1 + 1.0529 * np.sqrt(rs) + 0.3334 * rs),
                    0.0311 * np.log(rs) - 0.048 + 0.0020 * rs * np.log(rs) - 0.0116 * rs)


def test_broyden_mixing_solves_a_linear_fixed_point():
    # F(n) = b - A n (A symmetric positive definite, dimension 6): Broyden's
    # second method in Anderson form terminates like GMRES, within d + 2 steps
    from oracle import scf as osc
    rng = np.random.default_rng(7)
    M = rng.standard_normal((6, 6))
    A = M @ M.T / 6 + 0.5 * np.eye(6)
    b = rng.standard_normal(6)
    exact = np.linalg.solve(A, b)
    mix = osc.Broyden(alpha=0.3, history=10)
    n = np.zeros(6)
    first = mix.mix(n, b - A @ n)
    assert np.allclose(first, n + 0.3 * b, rtol=0, atol=1e-15)
    n = first
    for _ in range(8):
        n = mix.mix(n, b - A @ n)
    assert np.abs(n - exact).max() <= 1e-9 * np.abs(exact).max()


def test_fermi_occupations():
    from oracle import scf as osc
    eps = np.array([-1.0, -0.5, 0.1, 0.1, 0.4, 0.9])
    f, mu = osc.occupations(eps, 6.0, 0.01)
    assert abs(f.sum() - 6.0) < 1e-12 and np.all(np.diff(f) <= 1e-15) and f.max() <= 2.0
    assert abs(f[2] - f[3]) < 1e-15 and abs(f[2] - 1.0) < 1e-9     # the degenerate pair shares two electrons
    f0, _ = osc.occupations(eps, 4.0, 1e-5)
    assert np.allclose(f0, [2, 2, 0, 0, 0, 0], atol=1e-9)


def test_scf_fixed_point_against_dense_diagonalisation():
    # the SCF fixed point of a tiny two-atom molecule reached by the oracle's
    # block CG with a few sweeps per step equals the one reached with dense
    # diagonalisation of H[n] (every eigenpair) at every step
    from oracle import poisson as op, scf as osc
    atoms = np.array([[0.0, 0, 0], [2.2, 0.3, -0.4]])
    g = og.sphere_union_grid(atoms, 3.2, 0.55)
    pr = oh.make_projectors(g, atoms, np.array([[1.0, 0.8], [1.5, 0.6]]), 1.0, 3.0)
    vext = wl.local_potential(g.coords, atoms)
    n0 = wl.atomic_density_guess(g.coords, atoms, 8, g.dV)
    S = eigensolver.BlockCG(oh.Hamiltonian(g, vext, pr), wl.random_block(g.npts, 12, 3), 4, tol=1e-11)
    scf = osc.SCF(S, g, vext, n0, 8, sweeps=5)
    for _ in range(80):
        if scf.step()[0] < 1e-10:
            break
    assert scf.residual < 1e-10 and scf.f[-1] < 1e-8
    # dense path: H[n] assembled column by column, all eigenpairs, same mixing
    Hd = oh.Hamiltonian(g, vext, pr)
    mix = osc.Broyden(0.3, 8, g.dV)
    n = n0.copy()
    for _ in range(80):
        exc, vxc = osc.lda_xc(n)
        Hd.V = vext + op.hartree(g, n) + vxc
        w, V = np.linalg.eigh(Hd.dense())
        V = V / np.sqrt(g.dV)
        f, _ = osc.occupations(w, 8.0, 0.01)
        F = (V * V) @ f - n          # Eq. 1b: sum_k f_k |phi_k|^2
        if np.sqrt(g.dV * np.sum(F * F)) < 1e-10:
            break
        n = mix.mix(n, F)
    assert np.abs(w[:12] - S.eps).max() < 1e-8
    assert np.sqrt(g.dV * np.sum((n - scf.n_in) ** 2)) < 1e-8


# ------------------------------------------------ certificate (no paper eq.) ---

def _ho_pair(n=10, h=0.35):
    """Two exact separable eigenvectors (ground state and the x-excited
    state) of the harmonic oscillator on a box, normalised <phi|phi> = 1."""
    from oracle import certificate as oc  # noqa: F401
    g = og.box_grid(n, h)
    H = oh.Hamiltonian(g, wl.harmonic_potential(g.coords, 1.0))
    e1, v1 = one_d_levels(n, h, 1.0)
    phi = [np.einsum("i,j,k->ijk", v1[:, a], v1[:, 0], v1[:, 0]).ravel() / np.sqrt(g.dV) for a in (0, 1)]
    mu = [e1[a] + 2 * e1[0] for a in (0, 1)]
    return g, H, phi, mu


def test_ritz_certificate_two_level_closed_form():
    # x = phi_a + t phi_b: Ritz value (mu_a + t^2 mu_b) / (1 + t^2) and
    # residual norm t |mu_b - mu_a| / (1 + t^2)
    from oracle import certificate as oc
    g, H, (pa, pb), (ma, mb) = _ho_pair()
    for t in (1e-3, 0.2, 0.7):
        eps, res, xr = oc.ritz_certificate(H.apply, (pa + t * pb)[:, None], g.dV)
        assert abs(eps[0] - (ma + t * t * mb) / (1 + t * t)) < 1e-12
        assert abs(res[0] - t * abs(mb - ma) / (1 + t * t)) < 1e-10 * max(t, 1e-2)
        assert abs(g.dV * xr[:, 0] @ xr[:, 0] - 1) < 1e-12


def test_ritz_certificate_invariant_subspace_exact():
    # a skewed (non-orthonormal) basis of an exact invariant subspace: Ritz
    # values are the exact eigenvalues and every residual vanishes
    from oracle import certificate as oc
    g, H, (pa, pb), (ma, mb) = _ho_pair()
    X = np.stack([pa + 0.3 * pb, 2.0 * pb - 0.5 * pa], axis=1)
    eps, res, _ = oc.ritz_certificate(H.apply, X, g.dV)
    assert np.abs(eps - np.sort([ma, mb])).max() < 1e-11
    assert res.max() < 1e-9


def test_richardson_step_damping_closed_form():
    # one column phi_a + c phi_b with theta = mu_a: after n steps the phi_a
    # part is unchanged and the phi_b part is c (1 - (mu_b - mu_a)/(lam - mu_a))^n
    from oracle import certificate as oc
    g, H, (pa, pb), (ma, mb) = _ho_pair()
    lam, c = 40.0, 0.25
    for n in (1, 3):
        X = oc.richardson_smooth(H.apply, (pa + c * pb)[:, None], np.array([ma]), lam, n)[:, 0]
        assert abs(g.dV * pa @ X - 1.0) < 1e-11
        assert abs(g.dV * pb @ X - c * (1 - (mb - ma) / (lam - ma)) ** n) < 1e-11


def test_smoothing_removes_high_energy_noise():
    # rounding-like white noise on exact eigenvectors: the smoothed
    # certificate's residuals are several times smaller and its Ritz values
    # stay on the exact eigenvalues
    from oracle import certificate as oc
    g, H, (pa, pb), (ma, mb) = _ho_pair()
    lam = oc.largest_eigenvalue(H.apply, g.npts)
    rng = np.random.default_rng(3)
    X = np.stack([pa, pb], axis=1)
    X = X * (1 + 1e-7 * rng.uniform(-1, 1, X.shape))
    e0, r0, _ = oc.ritz_certificate(H.apply, X, g.dV)
    e4, r4, _ = oc.smoothed_certificate(H.apply, X, np.array([ma, mb]), lam, 4, g.dV)
    assert r4.max() < r0.max() / 4
    assert np.abs(e4 - [ma, mb]).max() < 1e-12


def test_largest_eigenvalue_against_dense():
    from oracle import certificate as oc
    atoms = np.array([[0.0, 0.0, 0.0], [1.8, 0.0, 0.0]])
    g = og.sphere_union_grid(atoms, 2.5, 0.6)
    pr = oh.make_projectors(g, atoms, np.array([[1.0, 0.8], [1.5, 0.6]]), 1.0, 3.0)
    H = oh.Hamiltonian(g, wl.local_potential(g.coords, atoms), pr)
    assert abs(oc.largest_eigenvalue(H.apply, g.npts) - np.linalg.eigvalsh(H.dense())[-1]) < 1e-9
