"""The oracle's pins have teeth: each plausible mistake planted in a copy of
the oracle (a dropped term, a wrong sign, index or operand, a transposed
result) makes at least one pin of test_oracle_pins.py fail.

Every mutant is a single textual edit of one oracle source file.  The edit
is applied to a copy of ``oracle/`` in a temporary directory, next to
copies of the pin tests and the seeded input generators; the pins named
for that mutant then run there in a child process.  The repository's own
oracle is never modified.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@dataclass(frozen=True)
class Mutant:
    name: str
    file: str        # path under oracle/
    old: str         # must occur exactly once in the file
    new: str
    pins: str        # pytest -k expression: the pins expected to catch it


MUTANTS = [
    # kinetic term, Sec. V.A
    Mutant("stencil_centre_weight", "ora_core.c",
           "double acc = 3.0 * cw[0] * psi[p * nst + s];",
           "double acc = 2.0 * cw[0] * psi[p * nst + s];",
           "polynomial_exactness or plane_wave"),
    Mutant("kinetic_sign", "ora_core.c",
           "const double kin = -0.5 / (h * h);",
           "const double kin = 0.5 / (h * h);",
           "polynomial_exactness or plane_wave"),
    Mutant("stencil_offset_off_by_one", "ora_core.c",
           "int j = t < m ? t - m : t - m + 1;",
           "int j = t < m ? t - m : t - m + 2;",
           "polynomial_exactness or plane_wave"),
    Mutant("stencil_axis_mixup", "ora_core.c",
           "int32_t q = nbr[(p * 3 + a) * nn + t];",
           "int32_t q = nbr[(p * 3 + (a == 2 ? 1 : a)) * nn + t];",
           "polynomial_exactness or plane_wave"),
    Mutant("stencil_weight_index", "ora_core.c",
           "acc += cw[j < 0 ? -j : j] * psi",
           "acc += cw[j < 0 ? -j - 1 : j] * psi",
           "polynomial_exactness or plane_wave"),
    # local potential, Sec. V.B
    Mutant("local_potential_dropped", "ora_core.c",
           "hpsi[p * nst + s] = kin * acc + V[p] * psi[p * nst + s];",
           "hpsi[p * nst + s] = kin * acc;",
           "separable_spectrum"),
    Mutant("local_potential_wrong_state", "ora_core.c",
           "hpsi[p * nst + s] = kin * acc + V[p] * psi[p * nst + s];",
           "hpsi[p * nst + s] = kin * acc + V[p] * psi[p * nst];",
           "separable_spectrum"),
    # nonlocal term, Eq. (4)
    Mutant("projection_without_volume_element", "ora_core.c",
           "= E[A * 4 + q] * dV * acc;",
           "= E[A * 4 + q] * acc;",
           "kb_eigen"),
    Mutant("projection_without_coupling", "ora_core.c",
           "= E[A * 4 + q] * dV * acc;",
           "= dV * acc;",
           "kb_eigen"),
    Mutant("scatter_with_s_projector_only", "ora_core.c",
           "double g = gam[4 * o + q * len + i];",
           "double g = gam[4 * o + i];",
           "hermiticity or kb_eigen"),
    Mutant("projection_wrong_state", "ora_core.c",
           "acc += g[i] * psi[(int64_t)sph_idx[o + i] * nst + s];",
           "acc += g[i] * psi[(int64_t)sph_idx[o + i] * nst];",
           "hermiticity or nonlocal_psd"),
    Mutant("projector_normalised_without_dV", "hamiltonian.py",
           "norm = np.sqrt(grid.dV * (rows * rows).sum(axis=1))",
           "norm = np.sqrt((rows * rows).sum(axis=1))",
           "kb_eigen"),
    Mutant("p_projector_wrong_axis", "hamiltonian.py",
           "rows = np.stack([g, dx[sel] * g, dy[sel] * g, dz[sel] * g])",
           "rows = np.stack([g, dx[sel] * g, dx[sel] * g, dz[sel] * g])",
           "kb_eigen"),
    Mutant("couplings_repeated_wrongly", "hamiltonian.py",
           "[1, 3], axis=1",
           "[3, 1], axis=1",
           "kb_eigen"),
    Mutant("projector_sphere_strict", "hamiltonian.py",
           "sel = np.nonzero(d2 <= r_cut * r_cut)[0]",
           "sel = np.nonzero(d2 < r_cut * r_cut)[0]",
           "projector_sphere"),
    # grid, Sec. II
    Mutant("sphere_strict_inequality", "grid.py",
           "inside |= (dx * dx + dy * dy) + dz * dz <= r2",
           "inside |= (dx * dx + dy * dy) + dz * dz < r2",
           "sphere_count or union_grid"),
    Mutant("box_not_centred", "grid.py",
           "coords = (ijk.astype(np.float64) - (n - 1) / 2.0) * h",
           "coords = (ijk.astype(np.float64) - n / 2.0) * h",
           "box_grid or separable_spectrum"),
    # finite-difference weights
    Mutant("fd_rhs_halved", "stencil.py",
           "b = [Fraction(2) if k == 2 else Fraction(0) for k in range(n)]",
           "b = [Fraction(1) if k == 2 else Fraction(0) for k in range(n)]",
           "fd_weights"),
    # Cholesky, triangular inverse, Jacobi, Sec. VI
    Mutant("cholesky_short_update", "ora_core.c",
           "for (int k = 0; k < j; ++k) t -= U[(int64_t)k * n + j] * U[(int64_t)k * n + i];",
           "for (int k = 0; k + 1 < j; ++k) t -= U[(int64_t)k * n + j] * U[(int64_t)k * n + i];",
           "cholesky"),
    Mutant("triangular_inverse_transposed_operand", "ora_core.c",
           "t -= U[(int64_t)i * n + k] * X[(int64_t)k * n + col];",
           "t -= U[(int64_t)k * n + i] * X[(int64_t)k * n + col];",
           "cholesky"),
    Mutant("jacobi_rotation_sign", "ora_core.c",
           "A[(int64_t)k * n + q] = s * akp + c * akq;",
           "A[(int64_t)k * n + q] = -s * akp + c * akq;",
           "separable_spectrum"),
    Mutant("jacobi_vectors_transposed", "ora_core.c",
           "Vec[(int64_t)i * n + k] = Vt[(int64_t)ord[k] * n + i];",
           "Vec[(int64_t)k * n + i] = Vt[(int64_t)ord[k] * n + i];",
           "separable_spectrum"),
    Mutant("jacobi_sorted_descending", "ora_core.c",
           "A[(int64_t)i * n + i] < A[(int64_t)best * n + best]",
           "A[(int64_t)i * n + i] > A[(int64_t)best * n + best]",
           "separable_spectrum"),
    Mutant("overlap_without_volume_element", "linalg.py",
           "return dV * (X.T @ Y)",
           "return X.T @ Y",
           "grid_integral"),
    Mutant("orthonormalize_transposed_factor", "linalg.py",
           "return Psi @ Ui, Ui",
           "return Psi @ Ui.T, Ui",
           "orthonormalize"),
    Mutant("ritz_vectors_transposed", "linalg.py",
           "return eps, Psi @ xi, HPsi @ xi, xi",
           "return eps, Psi @ xi.T, HPsi @ xi.T, xi",
           "vectors_are_exact_eigenvectors"),
    # block eigensolver
    Mutant("residual_sign", "eigensolver.py",
           "R = HX - X * lam",
           "R = HX + X * lam",
           "tiny_molecule"),
    Mutant("block_stops_on_any_state", "eigensolver.py",
           "self.resnorm[sl] = res\n        if np.all(res <= self.tol):\n            return\n        W = ",
           "self.resnorm[sl] = res\n        if np.any(res <= self.tol):\n            return\n        W = ",
           "tiny_molecule"),
    Mutant("ritz_picks_highest", "eigensolver.py",
           "C = Ui @ Yv[:, :nb]",
           "C = Ui @ Yv[:, -nb:]",
           "tiny_molecule"),
    # filter preconditioner, shifted-Poisson CG
    Mutant("filter_weight", "eigensolver.py",
           "(1.0 - self.alpha) / 6.0 * acc",
           "(1.0 - self.alpha) / 3.0 * acc",
           "filter"),
    Mutant("cg_residual_update_sign", "precond.py",
           "Rr -= alpha * Ap",
           "Rr += alpha * Ap",
           "cg_"),
    Mutant("cg_direction_without_beta", "precond.py",
           "Pp = Rr + beta * Pp",
           "Pp = Rr + 0.0 * beta * Pp",
           "cg_"),
    # conv net, its gradients, BF16 rounding, Adam
    Mutant("conv_kernel_flipped", "precond.py",
           'y += np.einsum("oi,bixyz->boxyz", w[:, :, a, b, c]',
           'y += np.einsum("oi,bixyz->boxyz", w[:, :, 2 - a, 2 - b, 2 - c]',
           "conv3_bruteforce"),
    Mutant("grad_x_not_transposed", "precond.py",
           "gp[:, :, 2 - a:2 - a + X, 2 - b:2 - b + Y, 2 - c:2 - c + Z]",
           "gp[:, :, a:a + X, b:b + Y, c:c + Z]",
           "net_gradients"),
    Mutant("relu_mask_dropped_in_backward", "precond.py",
           "g2 = ga2 * m * (z2 > 0)",
           "g2 = ga2 * m",
           "net_gradients"),
    Mutant("loss_gradient_halved", "precond.py",
           "return float(np.sum(d * d) / n), 2.0 * d / n",
           "return float(np.sum(d * d) / n), d / n",
           "net_gradients"),
    Mutant("learned_output_not_rescaled", "precond.py",
           "out[grid.map[mask], s] = rms * y[0][mask]",
           "out[grid.map[mask], s] = y[0][mask]",
           "linear_stencils"),
    Mutant("learned_input_unmasked_layer", "precond.py",
           "a1 = np.maximum(z1, 0.0) * m",
           "a1 = np.maximum(z1, 0.0)",
           "linear_stencils or net_gradients"),
    Mutant("bf16_ties_away", "precond.py",
           "u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000",
           "u = (u + 0x8000) & 0xFFFF0000",
           "bf16"),
    Mutant("adam_without_bias_correction", "precond.py",
           "vh = self.v[i] / (1 - self.b2 ** self.t)",
           "vh = self.v[i]",
           "adam"),
    Mutant("adam_momentum_dropped", "precond.py",
           "self.m[i] = self.b1 * self.m[i] + (1 - self.b1) * g",
           "self.m[i] = (1 - self.b1) * g",
           "adam"),
    Mutant("adam_first_moment_bias_correction_dropped", "precond.py",
           "mh = self.m[i] / (1 - self.b1 ** self.t)",
           "mh = self.m[i]",
           "adam"),
    # Hartree potential by FFT (Sec. X)
    Mutant("poisson_periodic_kernel", "poisson.py",
           "v = 4.0 * np.pi * (1.0 - np.cos(G * Rc)) / G2",
           "v = 4.0 * np.pi / G2",
           "hartree"),
    Mutant("poisson_g0_dropped", "poisson.py",
           "v[0, 0, 0] = 2.0 * np.pi * Rc * Rc",
           "v[0, 0, 0] = 0.0",
           "hartree"),
    Mutant("poisson_cube_too_small", "poisson.py",
           "int(ext[a]) + int(math.ceil(Rc / grid.h)) + 1",
           "int(ext[a]) + int(math.ceil(0.5 * Rc / grid.h)) + 1",
           "hartree"),
    Mutant("poisson_frequency_scale", "poisson.py",
           "g = [2.0 * np.pi * np.fft.fftfreq(n, d=h) for n in shape]",
           "g = [np.pi * np.fft.fftfreq(n, d=h) for n in shape]",
           "hartree"),
    # SCF: LDA, occupations, density, Broyden mixing (Sec. III)
    Mutant("lda_exchange_potential_factor", "scf.py",
           "vx = 4.0 / 3.0 * ex",
           "vx = ex",
           "lda"),
    Mutant("pz_low_density_potential", "scf.py",
           "7.0 / 6.0 * PZ_B1",
           "6.0 / 7.0 * PZ_B1",
           "lda"),
    Mutant("pz_high_density_potential", "scf.py",
           "(PZ_B - PZ_A / 3.0)",
           "(PZ_B + PZ_A / 3.0)",
           "lda"),
    Mutant("broyden_correction_sign", "scf.py",
           "out = out - t * (dn + self.alpha * dF)",
           "out = out + t * (dn + self.alpha * dF)",
           "broyden"),
    Mutant("fermi_bisection_direction", "scf.py",
           "if fd(mid).sum() < n_electrons:",
           "if fd(mid).sum() > n_electrons:",
           "fermi"),
    Mutant("density_ignores_occupations", "scf.py",
           "return np.sum(Psi ** 2 * f[None, :], axis=1)",
           "return 2.0 * np.sum(Psi ** 2, axis=1)",
           "scf_fixed_point"),
    Mutant("scf_hartree_sign", "scf.py",
           "return self.v_ext + vh + vxc, vh, exc, vxc",
           "return self.v_ext - vh + vxc, vh, exc, vxc",
           "scf_fixed_point"),
    # RMM-DIIS (the paper's eigensolver, Sec. III)
    Mutant("rmm_trial_step_sign", "eigensolver.py",
           "            x = x + lam * p",
           "            x = x - lam * p",
           "rmm"),
    Mutant("diis_highest_eigenvector", "eigensolver.py",
           "a = Ui @ V[:, int(np.argmin(w))]",
           "a = Ui @ V[:, int(np.argmax(w))]",
           "diis or rmm"),
    Mutant("rayleigh_step_upper_pair", "eigensolver.py",
           "c = Ui @ V[:, int(np.argmin(w))]",
           "c = Ui @ V[:, int(np.argmax(w))]",
           "rayleigh_trial or rmm"),
    Mutant("rmm_residual_not_combined", "eigensolver.py",
           "r = sum(alpha[i] * rs[i] for i in range(k))",
           "r = rs[-1]",
           "rmm"),
    Mutant("rmm_hx_not_updated", "eigensolver.py",
           "            hx = hx + lam * hp",
           "            hx = hx + 0.0 * hp",
           "rmm"),
    # certificate and its smoothing (no paper equation; Rayleigh-Ritz of Sec. VI)
    Mutant("smooth_step_sign", "certificate.py",
           "X = X - (apply_h(X) - X * theta) / (lam - theta)",
           "X = X + (apply_h(X) - X * theta) / (lam - theta)",
           "richardson"),
    Mutant("smooth_theta_dropped", "certificate.py",
           "X = X - (apply_h(X) - X * theta) / (lam - theta)",
           "X = X - apply_h(X) / (lam - theta)",
           "richardson"),
    Mutant("smooth_step_length_unshifted", "certificate.py",
           "X = X - (apply_h(X) - X * theta) / (lam - theta)",
           "X = X - (apply_h(X) - X * theta) / lam",
           "richardson"),
    Mutant("certificate_residual_without_dV", "certificate.py",
           "res = np.sqrt(dV * ((HXr - Xr * eps) ** 2).sum(axis=0))",
           "res = np.sqrt(((HXr - Xr * eps) ** 2).sum(axis=0))",
           "ritz_certificate"),
    Mutant("certificate_overlap_ignored", "certificate.py",
           "eps, Y = scipy.linalg.eigh(h, 0.5 * (S + S.T))",
           "eps, Y = scipy.linalg.eigh(h)",
           "ritz_certificate"),
    Mutant("certificate_residual_sign", "certificate.py",
           "res = np.sqrt(dV * ((HXr - Xr * eps) ** 2).sum(axis=0))",
           "res = np.sqrt(dV * ((HXr + Xr * eps) ** 2).sum(axis=0))",
           "ritz_certificate"),
    Mutant("adam_second_moment_uses_gradient", "precond.py",
           "self.v[i] = self.b2 * self.v[i] + (1 - self.b2) * g * g",
           "self.v[i] = self.b2 * self.v[i] + (1 - self.b2) * np.abs(g)",
           "adam"),
]


def _copy_tree(dst: str, m: Mutant) -> None:
    ign = shutil.ignore_patterns("__pycache__", "_build", "*.so")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ign)
    shutil.copytree(os.path.join(ROOT, "workloads"), os.path.join(dst, "workloads"), ignore=ign)
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("__init__.py", "conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"), ignore=ign)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), os.path.join(dst, "pytest.ini"))
    path = os.path.join(dst, "oracle", m.file)
    src = open(path).read()
    assert src.count(m.old) == 1, f"{m.name}: the planted edit no longer matches oracle/{m.file}"
    open(path, "w").write(src.replace(m.old, m.new))


def _run(dst: str, m: Mutant, timeout: float = 240.0):
    env = dict(os.environ, OMP_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
    env.pop("PYTHONPATH", None)
    # the mutated C part must still compile: a build error is not a caught mistake
    b = subprocess.run([sys.executable, "-c", "from oracle import _native; _native.lib()"],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=timeout)
    if b.returncode != 0:
        return "build", b.stderr[-1500:]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "tests/test_oracle_pins.py", "-k", m.pins],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=timeout)
    return r.returncode, r.stdout[-3000:]


def test_every_mutant_edit_applies():
    for m in MUTANTS:
        src = open(os.path.join(ROOT, "oracle", m.file)).read()
        assert src.count(m.old) == 1, m.name


def test_pins_pass_on_the_unmodified_copy(tmp_path):
    # the harness itself: the same copy with a no-op edit passes the pins
    m = Mutant("none", "stencil.py", "def fd_weights(m: int = 4)", "def fd_weights(m: int = 4)",
               "fd_weights or polynomial_exactness or kb_eigen or cholesky")
    _copy_tree(str(tmp_path / "copy"), m)
    rc, out = _run(str(tmp_path / "copy"), m)
    assert rc == 0, out


def test_every_planted_mistake_fails_a_pin(tmp_path):
    def one(i_m):
        i, m = i_m
        dst = str(tmp_path / f"m{i:02d}")
        _copy_tree(dst, m)
        return m, _run(dst, m)

    workers = max(1, min(8, len(os.sched_getaffinity(0))))
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(one, enumerate(MUTANTS)))
    survivors = []
    for m, (rc, out) in results:
        if rc == "build":
            survivors.append(f"{m.name}: mutated oracle does not build\n{out}")
        elif rc != 1 or " failed" not in out:
            survivors.append(f"{m.name}: pins '{m.pins}' exit {rc}\n{out[-600:]}")
    assert not survivors, "\n\n".join(survivors)
