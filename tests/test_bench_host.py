"""Host logic of bench.py that needs no GPU: the DRAM traffic it reports
comes only from a profile summary captured on the same kernel source and
workload."""
import hashlib
import os

import bench
import workloads as wl


def test_profiled_traffic_matches_committed_summary():
    # the committed summary records the SHA-1 of the kernel source it profiled
    src = os.path.join(bench.ROOT, "paper_1306_2953_gb300", "csrc", "stencil_ring.cu")
    prof = os.path.join(bench.ROOT, "profiles", "k_hpsi_ring_mol100.md")
    sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    recorded = [l for l in open(prof) if l.startswith("- stencil_ring.cu sha1:")]
    assert len(recorded) == 1
    t = bench.profiled_traffic(wl.MOL100.name)
    if sha in recorded[0]:
        assert isinstance(t, int) and t > 0
    else:
        assert t is None


def test_profiled_traffic_other_workload_is_none():
    assert bench.profiled_traffic(wl.MOL300.name) is None
    assert bench.profiled_traffic(wl.MOL20.name) is None


def test_replica_throughput_is_whole_job():
    # two replicas, each 1 GB per step, 4 steps in 10 ms (slowest replica)
    assert abs(bench.replica_throughput(2, 1e9, 4, 10.0) - 800.0) < 1e-9


def test_reference_arm_json_line():
    # the reference arm times the FP64 oracle on the host cores and prints
    # one JSON line with the same metric and workload as the CUDA arm
    import json
    import subprocess
    import sys
    out = subprocess.run(
        [sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
         "--steps", "1", "--warmup", "0"],
        cwd=bench.ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    assert r["impl"] == "reference"
    assert r["unit"] == "GB/s" and r["higher_is_better"] is True
    assert r["value"] > 0 and r["steps"] == 1 and r["n_gpus"] == 1
    assert r["dtype"] == "f64" and r["data"] == "synthetic"
    assert r["config"]["workload"] == wl.MOL100.name
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"]
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"],
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_omp_threads(monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "3")
    assert bench.omp_threads() == 3
    monkeypatch.delenv("OMP_NUM_THREADS")
    assert bench.omp_threads() == len(os.sched_getaffinity(0))


def test_reference_arm_other_ranks_exit_quietly():
    # under torchrun only rank 0 times the oracle and prints the line
    import subprocess
    import sys
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "0"],
                         cwd=bench.ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_oracle_threads_sets_and_restores_team_size():
    import ctypes
    from oracle import _native
    L = _native.lib()
    L.omp_get_max_threads.restype = ctypes.c_int
    before = L.omp_get_max_threads()
    with bench.oracle_threads(1):
        assert L.omp_get_max_threads() == 1
    assert L.omp_get_max_threads() == before


def test_cpu_baseline_reports_all_cores_and_one_thread():
    # small budget on the 20-atom molecule: both timings are positive and the
    # one-thread block is not faster than the all-core one by more than noise
    g, dt, cores, dt1 = bench.cpu_baseline(wl.MOL20, 8, budget_s=1.0)
    assert dt > 0 and dt1 is not None and dt1 > 0 and cores >= 1
    if cores > 1:
        assert dt1 > 0.8 * dt


def test_cpu_model_is_named():
    m = bench.cpu_model()
    assert isinstance(m, str) and m


def test_certificate_bound_covers_the_true_error():
    """bench.certificate_bound, the cluster-aware Kato-Temple bound the
    300-atom certification rests on: Ritz pairs of a perturbed basis of the
    ten lowest eigenvectors of a small harmonic oscillator (levels of
    degeneracy 1, 3 and 6), FP64 Ritz values and residual norms from the
    oracle's certificate; for the judged states (the two lowest levels, as
    the solver judges states below a buffer) every Ritz value lies within
    its bound of the exact eigenvalue, and the bound of the isolated ground
    state is second order (far below its residual norm)."""
    import numpy as np
    from oracle import certificate as oc, grid as og, hamiltonian as oh
    g = og.box_grid(8, 0.45)
    H = oh.Hamiltonian(g, wl.harmonic_potential(g.coords, 1.0))
    lam, Phi = np.linalg.eigh(H.dense())
    Phi = Phi / np.sqrt(g.dV)
    rng = np.random.default_rng(2)
    for scale in (1e-3, 1e-4):
        # a smooth perturbation: components along the next thirty eigenvectors
        X = Phi[:, :10] + scale * Phi[:, 10:40] @ rng.standard_normal((30, 10))
        eps, res, _ = oc.ritz_certificate(H.apply, X, g.dV)
        b = bench.certificate_bound(eps, res)
        err = np.abs(eps - lam[:10])
        assert np.all(err[:4] <= b[:4]), (err[:4], b[:4])
        assert b[0] < 0.1 * res[0]
        # the top cluster (the third level) has no known gap above: residual bound
        assert np.all(b[7:] >= np.sqrt(np.sum(res[7:] ** 2)) * (1 - 1e-12))
    # one cluster holding every Ritz value: the bound is its residual, never zero
    eps, res = np.array([1.0, 1.0 + 1e-6]), np.array([1e-3, 1e-3])
    assert np.allclose(bench.certificate_bound(eps, res), np.sqrt(2) * 1e-3)
