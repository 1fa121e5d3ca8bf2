"""Plain FP64 CPU oracle for the real-space Kohn-Sham hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import, call or link anything in
this package.  It shares no code with the CUDA library: the two meet only
in the seeded input generators of ``workloads``.

Modules, each following the passage named in its docstring:
  grid        union-of-spheres and box grids (Sec. II)
  stencil     finite-difference weights of the 25-point Laplacian (Sec. V.A)
  hamiltonian kinetic + local + nonlocal Hamiltonian (Sec. V, Eqs. 3-4)
  linalg      overlap, Cholesky orthogonalisation, Rayleigh-Ritz (Sec. VI)
  eigensolver block CG (LOBPCG) and the filter preconditioner (Sec. III)
  precond     shifted-Poisson CG targets and the learned conv preconditioner
"""
from . import eigensolver, grid, hamiltonian, linalg, precond, stencil  # noqa: F401
