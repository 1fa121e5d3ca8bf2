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
