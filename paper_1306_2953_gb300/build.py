"""Builds ``librsdft.so`` (the C-ABI library) in-tree for sm_103a.

    python -m paper_1306_2953_gb300.build [--force]

Every translation unit is compiled in parallel with nvcc (CUDA sources) or
g++ (host sources) and linked into ``paper_1306_2953_gb300/librsdft.so``.
Host code is compiled without floating-point contraction so that the grid's
integer decisions are identical on x86-64 and AArch64.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librsdft.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


# translation units of librsdft.so
SOURCES = ["grid.cpp", "ham.cu", "linalg.cu", "subspace.cu", "precond.cu", "solver.cu", "learned.cu", "umma.cu", "noalloc.cu", "stencil_ring.cu", "device.cu", "poisson.cu", "scf.cu"]


def _sources():
    return list(SOURCES)


def _digest() -> str:
    h = hashlib.sha1()
    for d, files in ((CSRC, sorted(os.listdir(CSRC))), (INCLUDE, sorted(os.listdir(INCLUDE)))):
        files = [f for f in files if f.endswith((".cu", ".cpp", ".h"))]
        for f in files:
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    h.update(os.uname().machine.encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, bounds_check: bool = False) -> str:
    """Builds librsdft.so (or, with bounds_check, librsdft_check.so: the
    debugging build whose H psi kernel tests every point index it copies from
    or stores to and records an index out of range in its status word)."""
    out = LIB if not bounds_check else os.path.join(HERE, "librsdft_check.so")
    bdir = BUILD if not bounds_check else BUILD + "_check"
    stamp = os.path.join(bdir, "stamp")
    dig = _digest()
    if not force and os.path.exists(out) and os.path.exists(stamp) and open(stamp).read() == dig:
        return out
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    inc = [f"-I{INCLUDE}", f"-I{CSRC}"]
    extra = ["-DRS_BOUNDS_CHECK=1"] if bounds_check else []
    jobs = []
    for src in _sources():
        obj = os.path.join(bdir, src + ".o")
        path = os.path.join(CSRC, src)
        if src.endswith(".cu"):
            cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                   "--expt-relaxed-constexpr", *extra, *inc, "-c", path, "-o", obj]
        else:
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", *inc,
                   "-I/usr/local/cuda/include", "-c", path, "-o", obj]
        jobs.append((cmd, obj))

    def run(job):
        cmd, obj = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"compilation failed: {os.path.basename(obj)}")
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(run, jobs))
    tmp = out + f".tmp{os.getpid()}"
    link = [nvcc, ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(" ".join(link) + "\n" + r.stdout + r.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, out)
    with open(stamp, "w") as f:
        f.write(dig)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds_check="--bounds-check" in sys.argv))
