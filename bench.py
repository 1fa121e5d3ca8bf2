"""Benchmark of the real-space Kohn-Sham hot path on GB300.

Default workload: the 100-atom synthetic molecule (22 Bohr cube, union of
5 Bohr spheres at h = 0.3 Bohr), 256 states stored [npts][256] FP32, H psi
applied block by block (8 blocks of 32 states) -- one step is H applied to
every state.  Metric: H psi GB/s of algorithmic traffic (psi read once,
H psi written once, potential, point map and projector tables), reported
against the measured HBM copy bandwidth.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the path runs as independent replicas (one per rank, no
collective on the data path); value = work of all ranks / max time.
"""
from __future__ import annotations

import argparse
import contextlib
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "H·ψ GB/s & % HBM roofline; eigensolve s to 1e-6 Ha, mixed+learned vs FP64"
NB = 32


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"rsdft_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_system(workload):
    """Library grid + Hamiltonian of a synthetic molecule (no oracle)."""
    from paper_1306_2953_gb300 import api
    spec = workload.system
    atoms = wl.atom_positions(spec)
    E = wl.kb_couplings(spec)
    g = api.Grid.spheres(atoms, spec.radius, spec.h)
    pr = api.Projectors(g, atoms, E, spec.r_c, spec.r_cut)
    V = wl.local_potential(g.coords(), atoms)
    return g, api.Hamiltonian(g, V, pr)


def omp_threads() -> int:
    """Threads the oracle's OpenMP loops run on: OMP_NUM_THREADS when set,
    else the CPUs this process may run on (libgomp sizes its team from the
    affinity mask, which a container's cpuset can make smaller than the
    machine)."""
    env = os.environ.get("OMP_NUM_THREADS", "").split(",")[0].strip()
    if env.isdigit() and int(env) > 0:
        return int(env)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name on x86; implementer
    and part codes on Arm, which names no model there)."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if fields.get("model name"):
        return fields["model name"]
    if fields.get("CPU implementer"):
        return f"{platform.machine()} (implementer {fields['CPU implementer']}, part {fields.get('CPU part', '?')})"
    return platform.machine() or "unknown"


@contextlib.contextmanager
def oracle_threads(n: int):
    """Runs the oracle's OpenMP loops on n threads inside the block (the
    team size of libgomp, which the oracle's library links), restoring the
    previous size afterwards."""
    from oracle import _native
    L = _native.lib()
    L.omp_get_max_threads.restype = ctypes.c_int
    prev = L.omp_get_max_threads()
    L.omp_set_num_threads(ctypes.c_int(n))
    try:
        yield
    finally:
        L.omp_set_num_threads(ctypes.c_int(prev))


def cpu_baseline(workload, nb_sample: int, budget_s: float = 20.0):
    """The FP64 oracle's H psi (plain C loops, OpenMP on all host cores) on a
    bounded sample: one block of nb_sample states of the same molecule."""
    from oracle import grid as og, hamiltonian as oh
    spec = workload.system
    atoms = wl.atom_positions(spec)
    E = wl.kb_couplings(spec)
    g = og.sphere_union_grid(atoms, spec.radius, spec.h)
    H = oh.Hamiltonian(g, wl.local_potential(g.coords, atoms), oh.make_projectors(g, atoms, E, spec.r_c, spec.r_cut))
    psi = wl.random_block(g.npts, nb_sample, 1)
    H.apply(psi)  # warm
    t0 = time.perf_counter()
    n = 0
    while True:
        H.apply(psi)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 50:
            break
    dt = (time.perf_counter() - t0) / n
    cores = omp_threads()
    # the same block on one thread: a few applications, a few seconds
    dt1 = None
    try:
        with oracle_threads(1):
            t0 = time.perf_counter()
            n1 = 0
            while n1 < 3 and (n1 == 0 or time.perf_counter() - t0 < budget_s / 2):
                H.apply(psi)
                n1 += 1
            dt1 = (time.perf_counter() - t0) / n1
    except (OSError, AttributeError):
        dt1 = None
    return g, dt, cores, dt1


def algorithmic_bytes_f32(npts, n_entries, n_atoms, nst, nb=NB):
    """Same byte model as rs_ham_apply_bytes for FP32, for nst states: psi
    read once, H psi written once, V and the point map, one copy of the
    projector tables and the coefficients."""
    s = 4
    per_block = (npts * nb * 2 * s + npts * s + npts * 4 + n_entries * (4 + 4 * s) + (npts + 1) * 4
                 + n_atoms * 4 * nb * s)
    return per_block * (nst // nb)


def run_reference(args, workload):
    """The CPU oracle as the reference arm: its FP64 H psi on the host cores,
    one block of 8 states of the same molecule per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import grid as og, hamiltonian as oh
    spec = workload.system
    atoms = wl.atom_positions(spec)
    g = og.sphere_union_grid(atoms, spec.radius, spec.h)
    pr = oh.make_projectors(g, atoms, wl.kb_couplings(spec), spec.r_c, spec.r_cut)
    H = oh.Hamiltonian(g, wl.local_potential(g.coords, atoms), pr)
    nb = 8
    psi = wl.random_block(g.npts, nb, 1)
    for _ in range(args.warmup):
        H.apply(psi)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        H.apply(psi)
    dt = (time.perf_counter() - t0) / args.steps
    cores = omp_threads()
    by = algorithmic_bytes_f32(g.npts, int(pr.sph_off[-1]), spec.n_atoms, nb, nb=nb)
    v = by / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload.name, "npts": g.npts, "states_per_step": nb, "block": nb},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": f"FP64 oracle H psi on one block of {nb} states of {workload.name} per step"},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def profiled_traffic(workload_name):
    """DRAM bytes (read + write) per launch of the H psi kernel from the
    committed ncu summary of the 100-atom workload, or None for another
    workload or when the kernel source has changed since that capture (the
    summary records the source's SHA-1)."""
    if workload_name != wl.MOL100.name:
        return None
    import hashlib
    prof = os.path.join(ROOT, "profiles", "k_hpsi_ring_mol100.md")
    src = os.path.join(ROOT, "paper_1306_2953_gb300", "csrc", "stencil_ring.cu")
    if not (os.path.exists(prof) and os.path.exists(src)):
        return None
    with open(src, "rb") as f:
        sha = hashlib.sha1(f.read()).hexdigest()
    fields = {}
    with open(prof) as f:
        for line in f:
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
    if fields.get("stencil_ring.cu sha1") != sha:
        return None
    try:
        return int(fields["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


def load_golden(name):
    p = os.path.join(ROOT, "tests", "golden", f"eigs_{name}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


def build_any(workload):
    """Library grid + Hamiltonian of a workload (molecule or oscillator box)."""
    from paper_1306_2953_gb300 import api
    s = workload.system
    if isinstance(s, wl.BoxSpec):
        g = api.Grid.box(s.n, s.n, s.n, s.h)
        return g, api.Hamiltonian(g, wl.harmonic_potential(g.coords(), s.omega))
    return build_system(workload)


def initial_weights(seed=11):
    """The seeded starting weights of the network (FP32 [2160], device)."""
    import torch
    return torch.from_numpy(np.concatenate([a.reshape(a.shape[0], a.shape[1], 27).ravel()
                                            for a in wl.conv_init(seed)]).astype(np.float32)).cuda()


# the solver's schedules (rs_solver_cfg): the learned preconditioner gives way
# to the filter after 3 sweeps without a 10 % drop of the largest wanted
# residual; FP32 solvers take the closing FP64 Rayleigh-Ritz every 10 sweeps
# once that residual is <= 3e-3 and at every sweep once it is <= 1e-4
SCHEDULE = {"stall_sweeps": 3, "stall_ratio": 0.9, "rr64_every": 10, "rr64_below": 3e-3, "rr64_always": 1e-4}
LEARN = {"n_res": 40, "cg_iters": 200, "sigma": 1.0, "n_tiles": 10000, "epochs": 5, "batch": 64, "seed": 11}


def eigensolve_bench(workload, modes, max_seconds=600.0, tol=1e-6):
    """Seconds until every judged eigenvalue is within tol Ha of the oracle's
    reference (tests/golden), for each precision / preconditioner mode.  Each
    mode is a sequence of library calls: solver creation, (learned mode)
    rs_precond_train, then rs_eigensolver_step until the eigenvalues it
    reports -- from the closing FP64 Rayleigh-Ritz in FP32 mode -- match."""
    import torch
    from paper_1306_2953_gb300 import api, _lib
    gold = load_golden(workload.name)
    if gold is None:
        return {"workload": workload.name, "unavailable": "no oracle reference eigenvalues for this workload"}
    ref = np.array(gold["eigenvalues"])
    judged = len(ref)
    g, H = build_any(workload)
    out = {"workload": workload.name, "npts": g.npts, "states": workload.n_states, "judged": judged,
           "tolerance_ha": tol, "reference": "oracle block CG (tests/golden)", "schedule": SCHEDULE, "modes": {}}
    psi0 = wl.random_block(g.npts, workload.n_states, workload.seed)
    w0 = initial_weights(LEARN["seed"])
    for mode in modes:
        dt = torch.float64 if mode.startswith("f64") else torch.float32
        pc = _lib.RS_PRECOND_LEARNED if mode.endswith("learned") else _lib.RS_PRECOND_FILTER
        method = _lib.RS_EIG_RMMDIIS if mode.endswith("_rmm") else _lib.RS_EIG_BLOCK_CG
        psi0_d = torch.from_numpy(psi0).to(dt).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = api.Solver(H, psi0_d, workload.block, 1e-4, precond=pc, n_wanted=judged, method=method, **SCHEDULE)
        losses = None
        if mode.endswith("_cg"):
            # five CG iterations on (-1/2 Lap + 2) W = R (kept alive by S)
            S.set_precond_cg(api.Hamiltonian(g, np.full(g.npts, 2.0)), 5)
        if pc == _lib.RS_PRECOND_LEARNED:
            losses = S.train_precond(g, w0, **LEARN)
        err = float("inf")
        while True:
            eps, _, _ = S.step()
            st = S.stats()
            err = float(np.abs(eps.cpu().numpy()[:judged] - ref).max()) if st["eps_f64"] else float("inf")
            el = time.perf_counter() - t0
            if err <= tol or el > max_seconds:
                break
        out["modes"][mode] = {"seconds": el, "sweeps": st["sweeps"], "max_error_ha": err, "converged": err <= tol,
                              "train_seconds": st["train_target_seconds"] + st["train_fit_seconds"],
                              "train_target_seconds": st["train_target_seconds"],
                              "train_fit_seconds": st["train_fit_seconds"], "train_losses": losses}
        if pc == _lib.RS_PRECOND_LEARNED:
            out["modes"][mode]["filter_fallback_after_sweep"] = st["fallback_sweep"] or None
        del S, psi0_d
    return out


ORDER_NAMES = {4: "brick4", 1: "lexicographic", 2: "brick2", 8: "brick8", -1: "morton", -2: "tile_column"}


def certificate_bound(eps, res):
    """Per-state eigenvalue error bounds from FP64 Ritz values and residual
    norms (rs_solver_certify).  Ritz values closer than ten times their
    combined residual are grouped into clusters; for a cluster C with
    residual ||R_C||^2 = sum r_i^2 and gap delta_C to the nearest Ritz value
    outside it, every eigenvalue it approximates lies within
    ||R_C||^2 / delta_C (Kato-Temple for an invariant subspace) when
    delta_C > ||R_C||, else within ||R_C||.  The gaps are those between
    Ritz values, so the bound assumes no eigenvalue is missing between them
    or below the lowest; above the highest Ritz value the spectrum is not
    known, so the top cluster takes ||R_C|| (and so do the judged states
    only if they reach the top)."""
    e = np.asarray(eps, dtype=np.float64)
    r = np.asarray(res, dtype=np.float64)
    order = np.argsort(e)
    es, rs = e[order], r[order]
    clusters = [[0]]
    for i in range(1, len(es)):
        prev = clusters[-1]
        if es[i] - es[prev[-1]] < 10.0 * np.sqrt(rs[i] ** 2 + rs[prev[-1]] ** 2):
            prev.append(i)
        else:
            clusters.append([i])
    b = np.empty(len(es))
    for c in clusters:
        R = np.sqrt(np.sum(rs[c] ** 2))
        if c[-1] + 1 == len(es):
            b[c] = R   # no gap known above the highest Ritz value
            continue
        lo = es[c[0]] - es[c[0] - 1] if c[0] > 0 else np.inf
        hi = es[c[-1] + 1] - es[c[-1]]
        d = min(lo, hi)
        b[c] = R * R / d if d > R else R
    out = np.empty(len(es))
    out[order] = b
    return out


def certified_solve(workload, modes, r_stop=1e-5, tol=1e-6, max_seconds=720.0, f64_sweeps=2, cert_below=3e-4,
                    cert_every=100, n_smooth=4, emit=True):
    """Time to a certified tol Ha for a workload without an oracle reference
    (the 300-atom molecule): sweeps, with r_stop as the solver's tolerance
    (a block whose residuals are all below it is left alone), until the
    largest FP32-measured residual of the judged states is below r_stop,
    then rs_solver_certify_smoothed (n_smooth damped FP64 Richardson steps
    on the orbitals, which remove their FP32 rounding noise, then the FP64
    Rayleigh-Ritz and FP64 residual norms of the Ritz vectors; n_smooth = 0
    is the plain rs_solver_certify); the bound of certificate_bound for every judged state
    must be <= tol, otherwise cert_every more sweeps and a new certificate;
    certificates are also taken every cert_every sweeps once the residual is
    below cert_below, and at the time cap a last one is taken and reported.  The plain FP64 path
    is timed for f64_sweeps sweeps and extrapolated to the sweep count of
    the mixed solve of the same method."""
    import torch
    from paper_1306_2953_gb300 import api, _lib
    g, H = build_any(workload)
    judged = workload.judged
    out = {"workload": workload.name, "npts": g.npts, "states": workload.n_states, "judged": judged,
           "tolerance_ha": tol, "r_stop": r_stop, "smoothing_steps": n_smooth,
           "reference": "FP64 certificate (rs_solver_certify_smoothed): max over judged states of r^2/gap "
           "(r where gap <= r)", "modes": {}}
    psi0 = wl.random_block(g.npts, workload.n_states, workload.seed)
    w0 = initial_weights(LEARN["seed"])
    for mode in modes:
        dt = torch.float64 if mode.startswith("f64") else torch.float32
        pc = _lib.RS_PRECOND_LEARNED if "learned" in mode else _lib.RS_PRECOND_FILTER
        method = _lib.RS_EIG_RMMDIIS if "_rmm" in mode else _lib.RS_EIG_BLOCK_CG
        psi0_d = torch.from_numpy(psi0).to(dt).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = api.Solver(H, psi0_d, workload.block, r_stop, precond=pc, n_wanted=judged, stall_sweeps=3,
                       stall_ratio=0.9, method=method)
        t_create = time.perf_counter() - t0
        if mode.endswith("_cg"):
            S.set_precond_cg(api.Hamiltonian(g, np.full(g.npts, 2.0)), 5)
        if pc == _lib.RS_PRECOND_LEARNED:
            S.train_precond(g, w0, **LEARN)
        if mode.startswith("f64"):
            ts = []
            for _ in range(f64_sweeps):
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                S.step()
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t1)
            out["modes"][mode] = {"solver_create_seconds": t_create, "seconds_per_sweep": float(np.mean(ts[1:] or ts)),
                                  "sweeps_timed": f64_sweeps}
            del S, psi0_d
            continue
        certs, bound, nxt, traj = [], float("inf"), None, []
        while True:
            _, res, _ = S.step()
            st = S.stats()
            el = time.perf_counter() - t0
            rmax = float(res[:judged].max())
            if st["sweeps"] % 10 == 0:
                traj.append([st["sweeps"], round(el, 2), rmax])
            final = el > max_seconds
            # certificates: once the largest residual is below r_stop, and
            # every cert_every sweeps once it is below cert_below (the FP32
            # residuals of a large system can stall above r_stop while the
            # FP64 certificate already meets tol)
            periodic = nxt is None and rmax <= cert_below and st["sweeps"] % cert_every == 0
            if final or periodic or (nxt is None and rmax <= r_stop) or (nxt is not None and st["sweeps"] >= nxt):
                tc = time.perf_counter()
                try:
                    eps, r64 = S.certify_smoothed(n_smooth)
                except _lib.RsError as exc:
                    certs.append({"sweep": st["sweeps"], "error": str(exc)})
                    break
                e, r = eps.cpu().numpy(), r64.cpu().numpy()
                b = certificate_bound(e, r)[:judged]
                bound = float(b.max())
                certs.append({"sweep": st["sweeps"], "seconds": time.perf_counter() - t0,
                              "certify_seconds": time.perf_counter() - tc, "max_r64": float(r[:judged].max()),
                              "worst_state": int(np.argmax(b)), "worst_fp32_state": int(np.argmax(res[:judged].cpu().numpy())),
                              "bound_ha": bound, "fp32_max_residual": rmax})
                nxt = st["sweeps"] + cert_every
                if bound <= tol or final:
                    break
        el = time.perf_counter() - t0
        out["modes"][mode] = {"seconds": el, "sweeps": st["sweeps"], "certified": bound <= tol, "bound_ha": bound,
                              "solver_create_seconds": t_create, "certificates": certs, "trajectory": traj,
                              "train_seconds": st["train_target_seconds"] + st["train_fit_seconds"],
                              "filter_fallback_after_sweep": st["fallback_sweep"] or None,
                              "lambda_max_estimate": S.stats()["lambda_max"] or None,
                              "eigenvalues_head": [float(x) for x in e[:8]] if certs else None}
        if certs and n_smooth > 0 and "error" not in certs[-1]:
            # outside the timed region: the same subspace certified without
            # smoothing, and the largest change of a judged Ritz value
            e0, r0 = (t.cpu().numpy() for t in S.certify())
            out["modes"][mode]["unsmoothed"] = {"max_r64": float(r0[:judged].max()),
                                                "bound_ha": float(certificate_bound(e0, r0)[:judged].max()),
                                                "max_ritz_shift_ha": float(np.abs(e0[:judged] - e[:judged]).max())}
        del S, psi0_d
    for mixed, f64name in (("mixed_filter", "f64_filter"), ("mixed_rmm", "f64_rmm")):
        f, f64 = out["modes"].get(mixed), out["modes"].get(f64name)
        if f and f64:
            f64["extrapolated_seconds"] = f64["solver_create_seconds"] + f64["seconds_per_sweep"] * f["sweeps"]
            f64["extrapolation"] = (f"measured FP64 seconds per sweep x the sweeps of the {mixed} solve (same "
                                    "start, same method)")
    if emit:
        print(json.dumps(out), flush=True)
    return out


def scf_bench(spec, precisions=("f64", "f32"), max_steps=300):
    """Seconds until the SCF density residual is below spec.tol (the 20-atom
    molecule made self-consistent: FFT Hartree, LDA, Fermi occupations,
    Broyden mixing around block CG), FP64 and mixed precision, against the
    oracle's self-consistent reference (tests/golden) where it exists."""
    import torch
    from paper_1306_2953_gb300 import api
    s = spec.base.system
    atoms = wl.atom_positions(s)
    g = api.Grid.spheres(atoms, s.radius, s.h)
    coords = g.coords()
    vext = wl.local_potential(coords, atoms)
    pr = api.Projectors(g, atoms, wl.kb_couplings(s), s.r_c, s.r_cut)
    H = api.Hamiltonian(g, vext, pr)
    n0 = wl.atomic_density_guess(coords, atoms, spec.n_electrons, g.dV)
    psi0 = wl.random_block(g.npts, spec.n_states, spec.base.seed)
    gp = os.path.join(ROOT, "tests", "golden", f"scf_{spec.name}.json")
    gold = json.load(open(gp)) if os.path.exists(gp) else None
    out = {"workload": spec.name, "npts": g.npts, "electrons": spec.n_electrons, "states": spec.n_states,
           "tolerance": spec.tol, "modes": {}}
    for prec in precisions:
        dt = torch.float64 if prec == "f64" else torch.float32
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = api.Solver(H, torch.from_numpy(psi0).to(dt).cuda(), spec.block, 1e-10)
        scf = api.SCF(S, g, vext, n0, spec.n_electrons, sigma=spec.sigma, alpha=spec.alpha, history=spec.history,
                      sweeps=spec.sweeps)
        for _ in range(max_steps):
            r, e = scf.step()
            if r < spec.tol:
                break
        el = time.perf_counter() - t0
        _, _, _, steps = scf.state()
        m = {"seconds": el, "steps": steps, "residual": r, "energy_ha": e, "converged": r < spec.tol}
        if gold is not None:
            m["energy_error_vs_oracle_ha"] = abs(e - gold["energy"])
        out["modes"][prec] = m
        del scf, S
    return out


def poisson_timing(workload, n):
    """n FFT Hartree solves (rs_poisson_solve) of a smooth density on the
    workload's grid after three untimed ones; prints the time per solve and
    the algorithmic bytes: six one-dimensional FFT passes reading and
    writing the complex cube, the kernel multiplication (cube read and
    written, the FP64 kernel table read), the cube clear and the grid <->
    cube copies, over CUDA-event time."""
    import torch
    from paper_1306_2953_gb300 import api
    spec = workload.system
    atoms = wl.atom_positions(spec)
    g = api.Grid.spheres(atoms, spec.radius, spec.h)
    P = api.Poisson(g)
    shape, rc, cube_bytes = P.info()
    rho = torch.from_numpy(wl.atomic_density_guess(g.coords(), atoms, 4 * spec.n_atoms, g.dV)).cuda()
    vh = torch.empty_like(rho)
    for _ in range(3):
        P.solve(rho, vh)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n):
        P.solve(rho, vh)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    by = int(cube_bytes * (6 * 2 + 2.5 + 1)) + g.npts * (8 + 4 + 16) * 2
    peak, kind = measured_peaks()
    print(json.dumps({"workload": workload.name, "npts": g.npts, "cube": shape, "r_cut_bohr": rc,
                      "ms_per_solve": ms, "algorithmic_bytes": by, "gbs": by / (ms * 1e-3) / 1e9,
                      "frac_of_peak": by / (ms * 1e-3) / 1e9 / peak, "peak_source": kind}))
    return 0


def nb_sweep(workload, orders=(4,)):
    """H psi throughput against the block size and the grid's point order
    (the analogue of the paper's block-size and ordering study, Sec. V.A):
    for every order, nb = 1..64 states and FP32 / FP64, the algorithmic
    bytes of one block application (rs_ham_apply_bytes) over its CUDA-event
    time, psi [npts][64] resident.  Every order runs the generic fused kernel
    (neighbours through the point map); the default brick order also runs the
    automatic selection, whose FP32 blocks of 32 and 64 take the ring kernel."""
    import torch
    from paper_1306_2953_gb300 import _lib, api
    spec = workload.system
    atoms = wl.atom_positions(spec)
    E = wl.kb_couplings(spec)
    peak, kind = measured_peaks()
    out = {"workload": workload.name, "peak_gbs": peak, "peak_source": kind, "rows": []}
    for order in orders:
        g = api.Grid.spheres(atoms, spec.radius, spec.h, order=order)
        H = api.Hamiltonian(g, wl.local_potential(g.coords(), atoms), api.Projectors(g, atoms, E, spec.r_c, spec.r_cut))
        out["npts"] = g.npts
        kernels = [_lib.RS_KERNEL_GENERIC] + ([_lib.RS_KERNEL_AUTO] if order == 4 else [])
        for kern in kernels:
            H.select_kernel(kern)
            for dt, code in ((torch.float32, _lib.RS_F32), (torch.float64, _lib.RS_F64)):
                if kern == _lib.RS_KERNEL_AUTO and code == _lib.RS_F64:
                    continue   # FP64 blocks always take the generic kernel
                psi = torch.from_numpy(wl.random_block(g.npts, 64, 5)).to(dt).cuda()
                hpsi = torch.empty_like(psi)
                for nb in (1, 2, 4, 8, 16, 32, 64):
                    if kern == _lib.RS_KERNEL_AUTO and nb < 32:
                        continue
                    reps = max(3, min(200, int(2e9 / max(H.apply_bytes(nb, code), 1))))
                    for _ in range(3):
                        H.apply(psi[:, :nb], hpsi[:, :nb], nb=nb)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(reps):
                        H.apply(psi[:, :nb], hpsi[:, :nb], nb=nb)
                    e1.record()
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / reps
                    gbs = H.apply_bytes(nb, code) / (ms * 1e-3) / 1e9
                    out["rows"].append({"order": ORDER_NAMES[order],
                                        "kernel": "generic" if kern == _lib.RS_KERNEL_GENERIC else "auto (ring)",
                                        "dtype": "f32" if code == _lib.RS_F32 else "f64", "nb": nb,
                                        "us_per_apply": ms * 1e3, "gbs": gbs, "frac_of_peak": gbs / peak})
                del psi, hpsi
        if H.status() != 0:
            raise RuntimeError("an H psi pipeline wait gave up during the sweep")
        del H, g
    print(json.dumps(out))
    return 0


def f64_hpsi(H, workload, nb=NB, steps=10):
    """FP64 H psi, the paper's precision, on the benchmark's workload: all
    states applied block by block (the generic fused kernel), timed with
    CUDA events after three untimed steps.  Reported as algorithmic bytes
    per second (rs_ham_apply_bytes in FP64) against the measured HBM copy
    bandwidth, and as flops per second: per point-state 49 for the 25-point
    stencil and 2 for the potential, plus per projector-sphere entry and
    state 16 for the four projections and the four scatters."""
    import torch
    from paper_1306_2953_gb300 import _lib
    nst = workload.n_states
    psi = torch.from_numpy(wl.random_block(H.npts, nst, workload.seed)).cuda()
    hpsi = torch.empty_like(psi)
    na, ne = ctypes.c_int32(), ctypes.c_int64()
    _lib.call("rs_proj_info", H.proj._h, ctypes.byref(na), ctypes.byref(ne))
    for _ in range(3):
        H.apply_all(psi, hpsi, nb=nb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        H.apply_all(psi, hpsi, nb=nb)
    e1.record()
    torch.cuda.synchronize()
    if H.status() != 0:
        raise RuntimeError("an H psi pipeline wait gave up during the FP64 timing")
    s_per_step = e0.elapsed_time(e1) * 1e-3 / steps
    by = H.apply_bytes(nb, _lib.RS_F64) * (nst // nb)
    fl = nst * (51 * H.npts + 16 * ne.value)
    peak, kind = measured_peaks()
    return {"dtype": "f64", "states": nst, "block": nb, "ms_per_step": s_per_step * 1e3,
            "gbs": by / s_per_step / 1e9, "frac_of_hbm_peak": by / s_per_step / 1e9 / peak, "peak_source": kind,
            "tflops": fl / s_per_step / 1e12, "fp64_nominal_tflops": 1.25,
            "flops_model": "49 (stencil) + 2 (V) per point-state, 16 per sphere entry and state"}


def learned_apply_timing(workload, n):
    """n applications of the learned preconditioner (the 1-8-8-1 network on
    the point map) to one 32-state residual block, after three untimed ones;
    prints the mean time per application."""
    import torch
    from paper_1306_2953_gb300 import api
    g, H = build_system(workload)
    w = torch.from_numpy(np.concatenate([a.reshape(a.shape[0], a.shape[1], 27).ravel()
                                         for a in wl.conv_init(11)]).astype(np.float32)).cuda()
    R = torch.from_numpy(wl.random_block(g.npts, 32, 3)).float().cuda()
    for _ in range(3):
        api.precond_apply(H, w, R)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n):
        api.precond_apply(H, w, R)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"workload": workload.name, "npts": g.npts, "states": 32,
                      "ms_per_apply": e0.elapsed_time(e1) / n}))
    return 0


def max_over_ranks(value, device):
    """The largest of every rank's value (all ranks call it; the job's time
    is its slowest replica's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, bytes_per_step, steps, ms_max):
    """Whole-job GB/s of `world` replicas that each moved bytes_per_step per
    step, timed by the slowest replica."""
    return world * bytes_per_step * steps / (ms_max * 1e-3) / 1e9


def profile_sweeps(workload, n, precision="f32", method="cg"):
    """Solver creation and n eigensolver sweeps (filter preconditioner) in
    FP32 (mixed: FP32 orbitals, FP64 subspace steps) or FP64, block CG or
    RMM-DIIS, one JSON line per sweep with its wall time and largest
    residual."""
    import torch
    from paper_1306_2953_gb300 import api, _lib
    g, H = build_system(workload)
    dt = torch.float64 if precision == "f64" else torch.float32
    psi0 = torch.from_numpy(wl.random_block(g.npts, workload.n_states, workload.seed)).to(dt).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = api.Solver(H, psi0, workload.block, 1e-4,
                   method=_lib.RS_EIG_RMMDIIS if method == "rmm" else _lib.RS_EIG_BLOCK_CG)
    torch.cuda.synchronize()
    print(json.dumps({"workload": workload.name, "precision": precision, "method": method, "npts": g.npts,
                      "states": workload.n_states,
                      "solver_create_seconds": time.perf_counter() - t0}))
    for _ in range(n):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, res, _ = S.step()
        torch.cuda.synchronize()
        print(json.dumps({"sweep_seconds": time.perf_counter() - t0, "max_residual": float(res.max())}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=wl.MOL100.name, choices=[wl.MOL100.name, wl.MOL300.name])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--eigensolve", default="mol20_h0.35,mol100_h0.3",
                    help="workload(s) for the time-to-1e-6 Ha eigensolve, comma separated, or 'none'")
    ap.add_argument("--nb-sweep", action="store_true",
                    help="print H psi GB/s of algorithmic bytes for blocks of 1..64 states (FP32 and FP64) on "
                         "--workload and exit (no benchmark line)")
    ap.add_argument("--orders", default="4",
                    help="point orders of the --nb-sweep, comma separated: 4, 1, 2, 8 (brick edges; 1 = "
                         "lexicographic), -1 (Morton), -2 (tile columns), or 'all'")
    ap.add_argument("--learned-apply", type=int, default=0,
                    help="profiling aid: time this many learned-preconditioner applications to one 32-state "
                         "block of --workload (seeded initial weights) and exit (no benchmark line)")
    ap.add_argument("--sweep-precision", default="f32", choices=["f32", "f64"],
                    help="precision of the --profile-sweeps solver")
    ap.add_argument("--sweep-method", default="cg", choices=["cg", "rmm"],
                    help="eigensolver of the --profile-sweeps solver: block CG or RMM-DIIS")
    ap.add_argument("--poisson-timing", type=int, default=0,
                    help="profiling aid: time this many FFT Hartree solves on --workload's grid and exit")
    ap.add_argument("--certified", default="",
                    help="workload(s) for the certified time to 1e-6 Ha without an oracle reference (e.g. "
                         "mol300_h0.3): prints one JSON object per workload and exits (no benchmark line)")
    ap.add_argument("--certified-modes", default="f64_rmm,mixed_rmm,mixed_rmm_learned")
    ap.add_argument("--certified-max-seconds", type=float, default=720.0)
    ap.add_argument("--with-certified", default="",
                    help="opt-in: after the benchmark line's own measurements, run the certified solve of these "
                         "workload(s) (e.g. mol300_h0.3, --certified-modes) and attach it to the line as "
                         "'certified_eigensolve' (minutes per mode)")
    ap.add_argument("--certified-smooth", type=int, default=4,
                    help="FP64 smoothing steps before each certificate (rs_solver_certify_smoothed; 0: none)")
    ap.add_argument("--profile-sweeps", type=int, default=0,
                    help="profiling aid: run this many mixed-precision eigensolver sweeps on --workload, "
                         "print their times and exit (no benchmark line)")
    args = ap.parse_args()
    workload = wl.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, workload)
    if args.poisson_timing > 0:
        return poisson_timing(workload, args.poisson_timing)
    if args.certified:
        for n in args.certified.split(","):
            certified_solve(wl.WORKLOADS[n], args.certified_modes.split(","),
                            max_seconds=args.certified_max_seconds, n_smooth=args.certified_smooth)
        return 0
    if args.profile_sweeps > 0:
        return profile_sweeps(workload, args.profile_sweeps, args.sweep_precision, args.sweep_method)
    if args.nb_sweep:
        orders = (4, 1, 2, 8, -1, -2) if args.orders == "all" else tuple(int(x) for x in args.orders.split(","))
        return nb_sweep(workload, orders)
    if args.learned_apply > 0:
        return learned_apply_timing(workload, args.learned_apply)

    import torch
    import torch.distributed as dist
    from paper_1306_2953_gb300 import _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    g, H = build_system(workload)
    npts = g.npts
    nst = workload.n_states
    psi_h = torch.from_numpy(wl.random_block(npts, nst, workload.seed).astype(np.float32))
    psi = psi_h.to(dev)
    hpsi = torch.empty_like(psi)
    L = _lib.lib()
    bytes_per_apply = H.apply_bytes(NB, _lib.RS_F32)
    bytes_per_step = bytes_per_apply * (nst // NB)
    import ctypes
    pb, sb = ctypes.c_int64(), ctypes.c_int64()
    _lib.call("rs_ham_launch_bytes", H._h, NB, _lib.RS_F32, ctypes.byref(pb), ctypes.byref(sb))

    def step(src, dst):
        for b in range(0, nst, NB):
            H.apply(src[:, b:b + NB], dst[:, b:b + NB], nb=NB)

    for _ in range(max(args.warmup, 3)):
        step(psi, hpsi)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    _lib.call("rs_ham_timing", H._h, 1)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step(psi, hpsi)
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    _lib.call("rs_ham_timing", H._h, 0)
    if H.status() != 0:
        raise RuntimeError("an H psi pipeline wait gave up during the timed region: the results are incomplete")
    ms = e0.elapsed_time(e1)
    pms, sms, ncalls = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _lib.call("rs_ham_timing_read", H._h, ctypes.byref(pms), ctypes.byref(sms), ctypes.byref(ncalls))
    clk = clocks.stop()
    if world > 1:
        ms = max_over_ranks(ms, dev)

    # end to end through the public API: the orbitals in pinned host memory
    # as 32-state blocks, each block copied in, H applied and the result
    # copied out, the three stages of consecutive blocks overlapped on
    # three streams (two device buffers per direction)
    nblk = nst // NB
    blk_in = [psi_h[:, b * NB:(b + 1) * NB].contiguous().pin_memory() for b in range(nblk)]
    blk_out = [torch.empty_like(x).pin_memory() for x in blk_in]
    d_in = [torch.empty(npts, NB, device=dev) for _ in range(2)]
    d_out = [torch.empty(npts, NB, device=dev) for _ in range(2)]
    s_in, s_h, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_h = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def e2e_step():
        for i in range(nblk):
            k = i % 2
            with torch.cuda.stream(s_in):
                s_in.wait_event(ev_h[k])          # block i - 2 no longer reads d_in[k]
                d_in[k].copy_(blk_in[i], non_blocking=True)
                ev_in[k].record(s_in)
            s_h.wait_event(ev_in[k])
            s_h.wait_event(ev_out[k])             # block i - 2 has left d_out[k]
            H.apply(d_in[k], d_out[k], nb=NB, stream=s_h)
            ev_h[k].record(s_h)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_h[k])
                blk_out[i].copy_(d_out[k], non_blocking=True)
                ev_out[k].record(s_out)

    e2e_steps = max(1, min(args.steps, 10))
    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = psi.numel() * 4
    ref0 = hpsi[:, :NB].cpu()
    e2e_err = float((blk_out[0] - ref0).abs().max() / ref0.abs().max().clamp_min(1e-30))

    value = replica_throughput(world, bytes_per_step, args.steps, ms)
    peak, peak_kind = measured_peaks()
    stencil_gbs = sb.value * ncalls.value / (sms.value * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload.name, "npts": npts, "states": nst, "block": NB,
                       "psi_bytes": psi.numel() * 4,
                       "bytes_model": "per 32-state block: psi read once and H psi written once (2 x 4 B per "
                                      "point-state), V and the point map (8 B per point), one copy of the projector "
                                      "tables (20 B per sphere entry), projection coefficients",
                       "l2": f"inputs (psi, {psi.numel() * 4 / 1e9:.2f} GB) larger than L2 (129 MB)",
                       "parallelism": f"replicas{world}"},
            "roofline": {"bound": "hbm", "kernel": "k_hpsi_ring (fused stencil + V + nonlocal gather)",
                         "achieved": stencil_gbs, "peak": peak, "unit": "GB/s", "frac": stencil_gbs / peak,
                         "peak_source": peak_kind, "traffic": profiled_traffic(workload.name),
                         "algorithmic_bytes_per_launch": sb.value,
                         "stencil_ms_per_launch": sms.value / max(ncalls.value, 1),
                         "project_ms_per_launch": pms.value / max(ncalls.value, 1)},
            "e2e": {"value": world * bytes_per_step / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": h2d, "ms_per_step": e2e_s * 1e3,
                    "pipeline": "32-state blocks from pinned host memory; copy in, H psi, copy out overlapped on 3 streams",
                    "max_rel_diff_vs_device_result": e2e_err},
            "gpu_launches": int(2 * (nst // NB) * args.steps), "clocks": clk}
    if rank == 0 and world == 1:
        del hpsi
        line["f64_hpsi"] = f64_hpsi(H, workload)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gcpu, dt, cores, dt1 = cpu_baseline(workload, NB)
        by = bytes_per_apply  # the same FP32 block bytes, computed by the oracle in FP64
        line["cpu_baseline"] = {"value": by / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
                                "cpu": cpu_model(),
                                "sample": f"FP64 oracle H psi on one block of {NB} states of {workload.name} "
                                          f"({dt:.2f} s per block)"}
        if dt1 is not None:
            line["cpu_baseline"]["single_thread"] = {"value": by / dt1 / 1e9, "unit": "GB/s", "cores": 1,
                                                     "seconds_per_block": dt1}
    if rank == 0 and world == 1 and args.eigensolve != "none":
        line["eigensolve"] = [eigensolve_bench(wl.WORKLOADS[n], ["mixed_learned", "mixed_cg", "mixed_filter", "mixed_rmm",
                                                                 "f64_filter", "f64_rmm"])
                              for n in args.eigensolve.split(",")]
    if rank == 0 and world == 1 and args.eigensolve != "none":
        line["scf"] = scf_bench(wl.SCF_MOL20)
    if rank == 0 and world == 1 and args.with_certified:
        line["certified_eigensolve"] = [
            certified_solve(wl.WORKLOADS[n], args.certified_modes.split(","), max_seconds=args.certified_max_seconds,
                            n_smooth=args.certified_smooth, emit=False)
            for n in args.with_certified.split(",")]
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
