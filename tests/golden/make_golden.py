"""Writes the oracle's reference eigenvalues used by the GPU eigensolver tests
and the benchmark's time-to-accuracy measurement.

    python tests/golden/make_golden.py ho32_h0.3 mol20_h0.35 [mol100_h0.3 ...]
    python tests/golden/make_golden.py --annotate <workload> ...   (margins only)

Calls only the FP64 CPU oracle (``oracle/``) on the seeded synthetic
workloads of ``workloads``: block CG from the workload's random start
vectors, converged until every judged state's residual norm is below 1e-9
(molecules of 100 or more atoms: 1e-6), so that the eigenvalue error, of
order residual^2 / gap, is far below the 1e-8 Ha / 1e-6 Ha targets, plus,
for the harmonic oscillator, the separable closed form.  Output:
tests/golden/eigs_<workload>.json.

Margin of a file: the smallest gap between adjacent stored eigenvalues and
the eigenvalue error bound residual^2 / gap it gives (a Ritz value whose
residual norm is r lies within r^2 / gap of an eigenvalue when gap separates
it from the rest of the spectrum).  ``--annotate`` adds these two figures to
existing files from their own stored values, without solving again.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import eigensolver, grid as og, hamiltonian as oh  # noqa: E402
from oracle.stencil import fd_weights  # noqa: E402


def build(w: wl.Workload):
    s = w.system
    if isinstance(s, wl.BoxSpec):
        g = og.box_grid(s.n, s.h)
        return g, oh.Hamiltonian(g, wl.harmonic_potential(g.coords, s.omega))
    atoms = wl.atom_positions(s)
    g = og.sphere_union_grid(atoms, s.radius, s.h)
    pr = oh.make_projectors(g, atoms, wl.kb_couplings(s), s.r_c, s.r_cut)
    return g, oh.Hamiltonian(g, wl.local_potential(g.coords, atoms), pr)


def separable_levels(s: wl.BoxSpec, k: int) -> list[float]:
    c = fd_weights(4)
    x = (np.arange(s.n) - (s.n - 1) / 2) * s.h
    T = np.zeros((s.n, s.n))
    for i in range(s.n):
        for j in range(-4, 5):
            if 0 <= i + j < s.n:
                T[i, i + j] += -0.5 * c[abs(j)] / s.h ** 2
    e = np.linalg.eigvalsh(T + np.diag(0.5 * s.omega ** 2 * x ** 2))
    return sorted((e[:, None, None] + e[None, :, None] + e[None, None, :]).ravel())[:k]


def margins(out: dict) -> dict:
    """Smallest adjacent gap among the stored eigenvalues and the error
    bound max_residual^2 / gap (degenerate levels, gap below 1e-8 Ha, are
    treated as one cluster and skipped)."""
    e = np.sort(np.array(out["eigenvalues"]))
    gaps = np.diff(e)
    gaps = gaps[gaps > 1e-8]
    if len(gaps) == 0:
        return out
    g = float(gaps.min())
    out["min_gap_ha"] = g
    out["error_bound_ha"] = float(out["max_residual"]) ** 2 / g
    out["margin_note"] = ("min_gap_ha: smallest gap between adjacent judged eigenvalues (levels closer than 1e-8 Ha "
                          "counted as one cluster); error_bound_ha = max_residual^2 / min_gap_ha; the gap to the "
                          "first state above the judged ones is not stored")
    return out


def annotate(names):
    for name in names:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"eigs_{name}.json")
        with open(path) as f:
            out = json.load(f)
        with open(path, "w") as f:
            json.dump(margins(out), f, indent=1)
        print(name, out.get("min_gap_ha"), out.get("error_bound_ha"))


def scf_golden(spec: wl.ScfSpec):
    """The oracle's SCF run (block CG, spec.sweeps sweeps per step) from the
    atomic-Gaussian density guess and the workload's random start vectors,
    until the density residual is below spec.tol; writes
    tests/golden/scf_<name>.json with the eigenvalues, occupations, energy
    and the residual history."""
    from oracle import scf as osc
    w = spec.base
    g, H = build(w)
    atoms = wl.atom_positions(w.system)
    vext = H.V.copy()
    n0 = wl.atomic_density_guess(g.coords, atoms, spec.n_electrons, g.dV)
    t0 = time.time()
    S = eigensolver.BlockCG(H, wl.random_block(g.npts, spec.n_states, w.seed), spec.block, tol=1e-10)
    scf = osc.SCF(S, g, vext, n0, spec.n_electrons, sweeps=spec.sweeps, alpha=spec.alpha, history=spec.history,
                  sigma=spec.sigma)
    hist = []
    for it in range(300):
        r, e = scf.step()
        hist.append(r)
        print(f"  scf {it} residual {r:.3e} energy {e:.10f} {time.time() - t0:.0f}s", flush=True)
        if r < spec.tol:
            break
    out = {"workload": spec.name, "npts": g.npts, "n_states": spec.n_states, "n_electrons": spec.n_electrons,
           "eigenvalues": [float(v) for v in S.eps], "occupations": [float(v) for v in scf.f],
           "energy": scf.energy, "mu": scf.mu, "residual": scf.residual, "iterations": scf.iterations,
           "residual_history": hist, "cpu_seconds": time.time() - t0,
           "source": "oracle/scf.py SCF around oracle/eigensolver.py BlockCG (FP64), written by "
                     "tests/golden/make_golden.py"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"scf_{spec.name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(spec.name, scf.iterations, f"{time.time() - t0:.1f}s", scf.residual, scf.energy)


def main(names):
    for name in names:
        w = wl.WORKLOADS[name]
        g, H = build(w)
        t0 = time.time()
        psi0 = wl.random_block(g.npts, w.n_states, w.seed)
        log = []
        # the 100+ atom molecules converge in far fewer sweeps with the kinetic
        # preconditioner; it changes the path, not the eigenvalues
        big = isinstance(w.system, wl.MoleculeSpec) and w.system.n_atoms >= 100
        pc = eigensolver.KineticPreconditioner(g, 1.0, 10) if big else None

        def progress(s):
            log.append(float(np.max(s.resnorm[:w.judged])))
            if big:
                print(f"  sweep {s.iterations} max residual {log[-1]:.3e} eps0 {s.eps[0]:.10f} "
                      f"{time.time() - t0:.0f}s", flush=True)

        tol = 1e-6 if big else 1e-9
        solver = eigensolver.BlockCG(H, psi0, w.block, precond=pc, tol=tol)
        eps = solver.solve(max_iter=3000, judged=w.judged, callback=progress)
        out = {"workload": name, "npts": g.npts, "n_states": w.n_states, "judged": w.judged,
               "eigenvalues": [float(v) for v in eps], "residual_tol": tol, "iterations": solver.iterations,
               "max_residual": float(np.max(solver.resnorm[:w.judged])), "cpu_seconds": time.time() - t0,
               "preconditioner": "kinetic CG(10), sigma=1" if big else "filter alpha=0.5",
               "source": "oracle/eigensolver.py BlockCG (FP64), written by tests/golden/make_golden.py"}
        if isinstance(w.system, wl.BoxSpec):
            out["separable_closed_form"] = [float(v) for v in separable_levels(w.system, w.judged)]
        out = margins(out)
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"eigs_{name}.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(name, g.npts, solver.iterations, f"{time.time() - t0:.1f}s", out["max_residual"])


if __name__ == "__main__":
    if sys.argv[1:2] == ["--annotate"]:
        annotate(sys.argv[2:])
    elif sys.argv[1:2] == ["--scf"]:
        for n in sys.argv[2:]:
            scf_golden({s.name: s for s in (wl.SCF_MOL20,)}[n])
    else:
        main(sys.argv[1:])
