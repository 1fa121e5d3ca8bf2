"""Oracle: the self-consistent field loop of Sec. III (Fig. 2) with an LDA
exchange-correlation potential and Broyden density mixing.

TEST INFRASTRUCTURE.  Readings (the paper names the steps, not their
parameters):

* Density (Eq. 1b) of a spin-unpolarised system of N_e electrons:
  n = sum_k f_k |phi_k|^2 (Eq. 1b's spin-orbital sum over both spins),
  orbitals normalised with <a|b> = dV sum a b, occupations
  f_k = 2 / (1 + exp((eps_k - mu) / sigma)) with mu fixed by sum f_k = N_e
  (Fermi-Dirac smearing of width sigma, 0.01 Ha by default, so that states
  degenerate at the Fermi level share their electrons and the density has a
  fixed point; sigma -> 0 gives the closed-shell occupations 2, 0).
* Kohn-Sham potential (Eq. 3): v_ext + v_H[n] + v_xc[n], with v_H from the
  FFT Poisson solver (poisson.py) and v_xc the local density approximation:
  Slater exchange e_x = -(3/4) (3 n / pi)^(1/3) and the Perdew-Zunger (1981)
  parametrisation of the Ceperley-Alder correlation energy of the
  unpolarised electron gas, r_s = (3 / (4 pi n))^(1/3):
      r_s >= 1:  e_c = g / (1 + b1 sqrt(r_s) + b2 r_s),
      r_s <  1:  e_c = A ln r_s + B + C r_s ln r_s + D r_s,
  g = -0.1423, b1 = 1.0529, b2 = 0.3334, A = 0.0311, B = -0.048,
  C = 0.0020, D = -0.0116; v_xc = d(n e_xc)/dn.
* Each SCF step: the Kohn-Sham potential of the input density, a fixed
  number of eigensolver sweeps (the paper does not converge the
  eigenproblem inside each step), the output density, and Broyden mixing.
* Broyden mixing (Broyden 1965, Srivastava 1984): Broyden's second
  (inverse-Jacobian) update with uniform weights, in the form that equals
  Anderson mixing: with F = n_out - n_in, the history dn_i, dF_i of the last
  steps and theta minimising |F - sum theta_i dF_i|,
      n_in' = n_in + alpha F - sum theta_i (dn_i + alpha dF_i).
* Energy (Hartree), the Mermin free energy of the smeared occupations:
  E = sum f_k eps_k - E_H - int n v_xc + E_xc - sigma S with
  E_H = 1/2 int n v_H, E_xc = int n e_xc and the entropy
  S = -sum_k 2 (x ln x + (1 - x) ln(1 - x)), x = f_k / 2 (ion-ion
  repulsion omitted).
"""
from __future__ import annotations

import numpy as np

from . import poisson

PZ_G, PZ_B1, PZ_B2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def lda_xc(n: np.ndarray):
    """(e_xc, v_xc) per point: energy per electron and potential (Ha); zero
    where the density is not positive."""
    n = np.asarray(n, dtype=np.float64)
    pos = n > 1e-30
    nn = np.where(pos, n, 1.0)
    ex = -0.75 * (3.0 * nn / np.pi) ** (1.0 / 3.0)
    vx = 4.0 / 3.0 * ex
    rs = (3.0 / (4.0 * np.pi * nn)) ** (1.0 / 3.0)
    sq = np.sqrt(rs)
    den = 1.0 + PZ_B1 * sq + PZ_B2 * rs
    ec_lo = PZ_G / den
    vc_lo = ec_lo * (1.0 + 7.0 / 6.0 * PZ_B1 * sq + 4.0 / 3.0 * PZ_B2 * rs) / den
    lr = np.log(rs)
    ec_hi = PZ_A * lr + PZ_B + PZ_C * rs * lr + PZ_D * rs
    vc_hi = PZ_A * lr + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * rs * lr + (2.0 * PZ_D - PZ_C) / 3.0 * rs
    ec = np.where(rs >= 1.0, ec_lo, ec_hi)
    vc = np.where(rs >= 1.0, vc_lo, vc_hi)
    return np.where(pos, ex + ec, 0.0), np.where(pos, vx + vc, 0.0)


def occupations(eps: np.ndarray, n_electrons: float, sigma: float):
    """(f, mu): Fermi-Dirac occupations (at most 2 per state) summing to
    n_electrons, mu by bisection."""
    eps = np.asarray(eps, dtype=np.float64)
    fd = lambda mu: 2.0 / (1.0 + np.exp(np.clip((eps - mu) / sigma, -700, 700)))
    lo, hi = eps.min() - 50 * sigma, eps.max() + 50 * sigma
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if fd(mid).sum() < n_electrons:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    return fd(mu), mu


def entropy(f: np.ndarray) -> float:
    x = np.clip(np.asarray(f) / 2.0, 1e-300, 1.0 - 1e-16)
    return float(-2.0 * np.sum(x * np.log(x) + (1.0 - x) * np.log1p(-x)))


def density(Psi: np.ndarray, f: np.ndarray) -> np.ndarray:
    """n = sum_k f_k |psi_k|^2."""
    return np.sum(Psi ** 2 * f[None, :], axis=1)


class Broyden:
    """Broyden mixing in its Anderson form (see the module docstring)."""

    def __init__(self, alpha: float = 0.3, history: int = 8, dV: float = 1.0):
        self.alpha, self.history, self.dV = alpha, history, dV
        self.dn, self.dF = [], []
        self.prev = None

    def mix(self, n_in: np.ndarray, F: np.ndarray) -> np.ndarray:
        if self.prev is not None:
            self.dn.append(n_in - self.prev[0])
            self.dF.append(F - self.prev[1])
            if len(self.dn) > self.history:
                self.dn.pop(0)
                self.dF.pop(0)
        self.prev = (n_in.copy(), F.copy())
        out = n_in + self.alpha * F
        if self.dn:
            G = np.array([[self.dV * np.sum(a * b) for b in self.dF] for a in self.dF])
            rhs = np.array([self.dV * np.sum(a * F) for a in self.dF])
            theta = np.linalg.solve(G, rhs)
            for t, dn, dF in zip(theta, self.dn, self.dF):
                out = out - t * (dn + self.alpha * dF)
        return out


class SCF:
    """The SCF loop around an eigensolver object (BlockCG or RMMDIIS) whose
    Hamiltonian's local potential is replaced every step."""

    def __init__(self, solver, grid, v_ext: np.ndarray, n0: np.ndarray, n_electrons: float, sweeps: int = 3,
                 alpha: float = 0.3, history: int = 8, sigma: float = 0.01):
        self.solver, self.grid, self.v_ext = solver, grid, np.asarray(v_ext, dtype=np.float64)
        self.n_in = np.asarray(n0, dtype=np.float64).copy()
        self.n_electrons, self.sigma = n_electrons, sigma
        self.sweeps = sweeps
        self.mixer = Broyden(alpha, history, grid.dV)
        self.iterations = 0
        self.residual = np.inf

    def potential(self, n: np.ndarray):
        vh = poisson.hartree(self.grid, n)
        exc, vxc = lda_xc(n)
        return self.v_ext + vh + vxc, vh, exc, vxc

    def step(self):
        """One SCF step; returns (residual |n_out - n_in|, energy)."""
        v, vh, exc, vxc = self.potential(self.n_in)
        self.solver.set_potential(v)
        for _ in range(self.sweeps):
            self.solver.step()
        f, self.mu = occupations(self.solver.eps, self.n_electrons, self.sigma)
        self.f = f
        n_out = density(self.solver.Psi, f)
        F = n_out - self.n_in
        self.residual = float(np.sqrt(self.grid.dV * np.sum(F * F)))
        dV = self.grid.dV
        self.energy = float(np.sum(f * self.solver.eps) - 0.5 * dV * np.sum(self.n_in * vh)
                            - dV * np.sum(self.n_in * vxc) + dV * np.sum(self.n_in * exc) - self.sigma * entropy(f))
        self.n_in = self.mixer.mix(self.n_in, F)
        self.iterations += 1
        return self.residual, self.energy
