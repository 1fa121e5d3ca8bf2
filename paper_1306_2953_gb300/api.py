"""Thin torch-facing wrappers over the C ABI (argument marshalling only).

Host arrays are numpy; device arrays are torch CUDA tensors whose
``data_ptr()`` is passed straight to the library together with the current
torch stream.  Nothing here computes.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import RS_F32, RS_F64, call

_c = ctypes.c_void_p


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return RS_F64
    if t.dtype == torch.float32:
        return RS_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


class Grid:
    """Union-of-spheres or box grid (host tables; rs_grid_*)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @classmethod
    def spheres(cls, xyz, radius: float, h: float, order: int = 0) -> "Grid":
        """order: 0/4 bricks of 4^3 (default), 1/2/8 other bricks,
        _lib.RS_ORDER_MORTON or _lib.RS_ORDER_TILECOL."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        out = ctypes.c_void_p()
        call("rs_grid_create_spheres", _ptr(xyz), len(xyz), float(radius), float(h), int(order), ctypes.byref(out))
        return cls(out)

    @classmethod
    def box(cls, n0: int, n1: int, n2: int, h: float, order: int = 0) -> "Grid":
        out = ctypes.c_void_p()
        call("rs_grid_create_box", n0, n1, n2, float(h), int(order), ctypes.byref(out))
        return cls(out)

    def info(self):
        npts = ctypes.c_int64()
        origin = (ctypes.c_int32 * 3)()
        dims = (ctypes.c_int32 * 3)()
        h = ctypes.c_double()
        call("rs_grid_info", self._h, ctypes.byref(npts), origin, dims, ctypes.byref(h))
        return npts.value, tuple(origin), tuple(dims), h.value

    @property
    def npts(self) -> int:
        return self.info()[0]

    @property
    def h(self) -> float:
        return self.info()[3]

    @property
    def dV(self) -> float:
        return self.h ** 3

    def ijk(self) -> np.ndarray:
        out = np.empty((self.npts, 3), dtype=np.int32)
        call("rs_grid_ijk", self._h, _ptr(out))
        return out

    def coords(self) -> np.ndarray:
        out = np.empty((self.npts, 3), dtype=np.float64)
        call("rs_grid_coords", self._h, _ptr(out))
        return out

    def point_map(self) -> np.ndarray:
        _, _, dims, _ = self.info()
        out = np.empty(dims, dtype=np.int32)
        call("rs_grid_point_map", self._h, _ptr(out))
        return out

    def close(self):
        if self._h:
            _lib.lib().rs_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Projectors:
    """Kleinman-Bylander projector tables (rs_proj_*)."""

    def __init__(self, grid: Grid, xyz, E, r_c: float = 1.0, r_cut: float = 3.0):
        self._xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self._E = np.ascontiguousarray(E, dtype=np.float64)
        spec = _lib.ProjectorSpec(len(self._xyz), _ptr(self._xyz), _ptr(self._E), float(r_c), float(r_cut))
        out = ctypes.c_void_p()
        call("rs_proj_create", grid._h, ctypes.byref(spec), ctypes.byref(out))
        self._h = out
        self.grid = grid

    def tables(self):
        na = ctypes.c_int32()
        ne = ctypes.c_int64()
        call("rs_proj_info", self._h, ctypes.byref(na), ctypes.byref(ne))
        off = np.empty(na.value + 1, dtype=np.int64)
        idx = np.empty(ne.value, dtype=np.int32)
        gam = np.empty((ne.value, 4), dtype=np.float64)
        call("rs_proj_tables", self._h, _ptr(off), _ptr(idx), _ptr(gam))
        return off, idx, gam

    def close(self):
        if self._h:
            _lib.lib().rs_proj_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hamiltonian:
    """H = -1/2 Lap + V + V_nl on the current CUDA device (rs_ham_*)."""

    def __init__(self, grid: Grid, V, proj: Projectors | None = None, order: int = 4):
        V = np.ascontiguousarray(V, dtype=np.float64)
        out = ctypes.c_void_p()
        call("rs_ham_create", grid._h, _ptr(V), proj._h if proj is not None else None, order, ctypes.byref(out))
        self._h = out
        self.grid = grid
        self.proj = proj
        self.npts = grid.npts

    def apply(self, psi, hpsi=None, nb: int | None = None, stream=None):
        """hpsi[:, :nb] = H psi[:, :nb] for device tensors [npts, ld]."""
        import torch
        if hpsi is None:
            hpsi = torch.empty_like(psi)
        nb = psi.shape[1] if nb is None else nb
        assert psi.stride(1) == 1 and hpsi.stride(1) == 1
        call("rs_ham_apply_block", self._h, _c(psi.data_ptr()), psi.stride(0), _c(hpsi.data_ptr()), hpsi.stride(0),
             nb, dtype_code(psi), _stream(stream))
        return hpsi

    def apply_all(self, psi, hpsi=None, nb: int = 32, stream=None):
        """H applied to every state of psi [npts, nst], nb states per call."""
        import torch
        if hpsi is None:
            hpsi = torch.empty_like(psi)
        nst = psi.shape[1]
        for b in range(0, nst, nb):
            self.apply(psi[:, b:b + nb], hpsi[:, b:b + nb], nb=min(nb, nst - b), stream=stream)
        return hpsi

    def apply_bytes(self, nb: int, dtype: int) -> int:
        return int(_lib.lib().rs_ham_apply_bytes(self._h, nb, dtype))

    def status(self) -> int:
        """rs_ham_status: 0 unless a bounded pipeline wait gave up (blocking)."""
        f = ctypes.c_int32()
        call("rs_ham_status", self._h, ctypes.byref(f))
        return int(f.value)

    def select_kernel(self, which: int):
        """rs_ham_select_kernel: _lib.RS_KERNEL_AUTO or RS_KERNEL_GENERIC."""
        call("rs_ham_select_kernel", self._h, int(which))

    def reset_status(self):
        """rs_ham_reset_status: clears the status word (blocking)."""
        call("rs_ham_reset_status", self._h)

    def set_wait_limit(self, tests: int):
        """rs_ham_set_wait_limit (failure-detection test hook): barrier tests
        before a pipeline wait gives up; < 0 restores the default."""
        call("rs_ham_set_wait_limit", self._h, int(tests))

    def close(self):
        if self._h:
            _lib.lib().rs_ham_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def linalg_workspace(nst: int, device=None):
    import torch
    nbytes = int(_lib.lib().rs_linalg_workspace_bytes(nst))
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def overlap(grid: Grid, X, Y, stream=None):
    """S = dV X^T Y (FP64, device) for device tensors X [npts, nx], Y [npts, ny]."""
    import torch
    S = torch.empty((X.shape[1], Y.shape[1]), dtype=torch.float64, device=X.device)
    call("rs_overlap_block", grid._h, _c(X.data_ptr()), X.stride(0), X.shape[1], _c(Y.data_ptr()), Y.stride(0),
         Y.shape[1], _c(S.data_ptr()), S.stride(0), dtype_code(X), _stream(stream))
    return S


def orthonormalize(grid: Grid, Psi, work=None, stream=None):
    """Psi <- Psi U^-1 in place (Cholesky, Sec. VI); returns U^-1 (FP64)."""
    import torch
    nst = Psi.shape[1]
    work = linalg_workspace(nst, Psi.device) if work is None else work
    Ui = torch.empty((nst, nst), dtype=torch.float64, device=Psi.device)
    call("rs_orthonormalize", grid._h, _c(Psi.data_ptr()), Psi.stride(0), nst, dtype_code(Psi), _c(work.data_ptr()),
         _c(Ui.data_ptr()), _stream(stream))
    return Ui


def subspace_diag(ham: Hamiltonian, Psi, HPsi=None, nb: int = 32, work=None, stream=None):
    """Rayleigh-Ritz in place (Sec. VI); returns (eps, xi, HPsi)."""
    import torch
    nst = Psi.shape[1]
    HPsi = torch.empty_like(Psi) if HPsi is None else HPsi
    work = linalg_workspace(nst, Psi.device) if work is None else work
    eps = torch.empty(nst, dtype=torch.float64, device=Psi.device)
    xi = torch.empty((nst, nst), dtype=torch.float64, device=Psi.device)
    call("rs_subspace_diag", ham._h, _c(Psi.data_ptr()), _c(HPsi.data_ptr()), Psi.stride(0), nst, dtype_code(Psi),
         min(nb, nst), _c(eps.data_ptr()), _c(xi.data_ptr()), _c(work.data_ptr()), _stream(stream))
    return eps, xi, HPsi


class Solver:
    """Block CG (LOBPCG) eigensolver (rs_solver_*)."""

    def __init__(self, ham: Hamiltonian, Psi0, nb: int, tol: float, precond: int = _lib.RS_PRECOND_FILTER,
                 filter_alpha: float = 0.5, n_wanted: int = 0, stall_sweeps: int = 0, stall_ratio: float = 0.9,
                 rr64_every: int = 0, rr64_below: float = 0.0, rr64_always: float = 0.0,
                 method: int = _lib.RS_EIG_BLOCK_CG, rmm_steps: int = 0, stream=None):
        cfg = _lib.SolverCfg(Psi0.shape[1], nb, dtype_code(Psi0), precond, float(tol), float(filter_alpha),
                             int(n_wanted), int(stall_sweeps), float(stall_ratio), int(rr64_every), float(rr64_below),
                             float(rr64_always), int(method), int(rmm_steps))
        assert Psi0.is_contiguous()
        out = ctypes.c_void_p()
        call("rs_solver_create", ham._h, ctypes.byref(cfg), _c(Psi0.data_ptr()), _stream(stream), ctypes.byref(out))
        self._h = out
        self.ham = ham
        self.nst = Psi0.shape[1]
        self.dtype = Psi0.dtype
        self.device = Psi0.device

    def step(self, stream=None):
        """One sweep; returns (eps, resnorm, n_converged) with device FP64 tensors."""
        import torch
        eps = torch.empty(self.nst, dtype=torch.float64, device=self.device)
        res = torch.empty(self.nst, dtype=torch.float64, device=self.device)
        nconv = ctypes.c_int()
        call("rs_eigensolver_step", self._h, _c(eps.data_ptr()), _c(res.data_ptr()), ctypes.byref(nconv),
             _stream(stream))
        return eps, res, nconv.value

    def stats(self) -> dict:
        """rs_solver_stats as a dict."""
        st = _lib.SolverStats()
        call("rs_solver_stats", self._h, ctypes.byref(st))
        return {k: getattr(st, k) for k, _ in _lib.SolverStats._fields_}

    def train_precond(self, grid: Grid, w_init=None, n_res: int = 40, cg_iters: int = 200, sigma: float = 1.0,
                      n_tiles: int = 10000, epochs: int = 5, batch: int = 64, lr: float = 1e-3, seed: int = 11,
                      tile: int = 16, stream=None):
        """rs_precond_train: residuals, CG targets, training and the weights,
        all in the library; returns the per-epoch mean losses."""
        cfg = _lib.LearnCfg(n_res, cg_iters, float(sigma), _lib.TrainCfg(n_tiles, tile, epochs, batch, lr, seed))
        losses = (ctypes.c_float * max(epochs, 1))()
        call("rs_precond_train", self._h, grid._h, ctypes.byref(cfg),
             _c(w_init.data_ptr()) if w_init is not None else None, losses, _stream(stream))
        return list(losses)[:epochs]

    def checkpoint_save(self, path: str):
        """rs_solver_checkpoint_save: the iteration state to a file."""
        call("rs_solver_checkpoint_save", self._h, str(path).encode())

    def checkpoint_load(self, path: str):
        """rs_solver_checkpoint_load: continue from a saved iteration state."""
        call("rs_solver_checkpoint_load", self._h, str(path).encode())

    def save_precond(self, path: str):
        call("rs_precond_save", self._h, str(path).encode())

    def load_precond(self, path: str):
        call("rs_precond_load", self._h, str(path).encode())

    def psi(self):
        """The solver's orbitals as a torch tensor view [npts, nst] (no copy)."""
        import torch
        p = ctypes.c_void_p()
        call("rs_solver_psi", self._h, ctypes.byref(p))
        return _device_view(p.value, (self.ham.npts, self.nst), self.dtype, self.device)

    def set_precond(self, kind: int):
        """rs_solver_set_precond: switch the preconditioner for later sweeps."""
        call("rs_solver_set_precond", self._h, int(kind))

    def set_precond_cg(self, shifted: "Hamiltonian", n_iter: int):
        """rs_solver_set_precond_cg: n_iter CG iterations on the shifted
        Poisson operator ``shifted`` (V = sigma, no projectors) as the
        preconditioner of later sweeps; ``shifted`` must outlive the solver."""
        call("rs_solver_set_precond_cg", self._h, shifted._h, int(n_iter))
        self._shifted = shifted

    def set_precond_weights(self, w):
        """Learned-preconditioner weights: FP32 device tensor of 2160 values."""
        call("rs_solver_set_precond_weights", self._h, _c(w.data_ptr()))

    def rayleigh_ritz_f64(self, stream=None):
        """FP64 eigenvalues of the current subspace (closing step of FP32 mode)."""
        import torch
        eps = torch.empty(self.nst, dtype=torch.float64, device=self.device)
        call("rs_solver_rayleigh_ritz_f64", self._h, _c(eps.data_ptr()), _stream(stream))
        return eps

    def certify(self, stream=None):
        """rs_solver_certify: FP64 Ritz values and FP64 residual norms of the
        current subspace's Ritz vectors, as device tensors (eps, res)."""
        import torch
        eps = torch.empty(self.nst, dtype=torch.float64, device=self.device)
        res = torch.empty(self.nst, dtype=torch.float64, device=self.device)
        call("rs_solver_certify", self._h, _c(eps.data_ptr()), _c(res.data_ptr()), _stream(stream))
        return eps, res

    def certify_smoothed(self, n_smooth: int, lambda_max: float = 0.0, stream=None):
        """rs_solver_certify_smoothed: the certificate after n_smooth damped
        FP64 Richardson steps on the orbitals (lambda_max <= 0: the library's
        estimate of the largest eigenvalue of H), as device tensors (eps, res)."""
        import torch
        eps = torch.empty(self.nst, dtype=torch.float64, device=self.device)
        res = torch.empty(self.nst, dtype=torch.float64, device=self.device)
        call("rs_solver_certify_smoothed", self._h, int(n_smooth), float(lambda_max), _c(eps.data_ptr()),
             _c(res.data_ptr()), _stream(stream))
        return eps, res

    def residual(self, first: int, ncols: int, stream=None):
        """Ritz residuals of states first..first+ncols-1 as a device tensor."""
        import torch
        R = torch.empty((self.ham.npts, ncols), dtype=self.dtype, device=self.device)
        call("rs_solver_residual", self._h, first, ncols, _c(R.data_ptr()), R.stride(0), _stream(stream))
        return R

    def close(self):
        if self._h:
            _lib.lib().rs_solver_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _device_view(ptr: int, shape, dtype, device):
    """A torch tensor aliasing library-owned device memory (copy it before
    the owner is destroyed)."""
    import torch

    class _Holder:
        def __init__(self, p, shape, typestr, strides):
            self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (p, False),
                                             "version": 2, "strides": strides}

    es = torch.tensor([], dtype=dtype).element_size()
    typestr = "<f8" if es == 8 else "<f4"
    strides = (shape[1] * es, es)
    return torch.as_tensor(_Holder(ptr, shape, typestr, strides), device=device)


def shifted_poisson_cg(ham_sigma: Hamiltonian, B, n_iter: int = 200, stream=None):
    """n_iter CG iterations on (-1/2 Lap + sigma) X = B per column (ham_sigma
    built with V = sigma and no projectors); returns X."""
    import torch
    X = torch.empty_like(B)
    nb = B.shape[1]
    nbytes = int(_lib.lib().rs_cg_workspace_bytes(B.shape[0], nb, dtype_code(B)))
    work = torch.empty(nbytes, dtype=torch.uint8, device=B.device)
    call("rs_shifted_poisson_cg", ham_sigma._h, _c(B.data_ptr()), _c(X.data_ptr()), B.stride(0), nb, n_iter,
         dtype_code(B), _c(work.data_ptr()), _stream(stream))
    return X


def convnet_tiles(w, x, mask, target=None, valid=None, grad=True, stream=None):
    """The conv net on dense tiles [ntiles, D, D, D]; returns (y, grad, loss)."""
    import torch
    ntiles, D = x.shape[0], x.shape[1]
    y = torch.empty_like(x)
    g = torch.empty(2160, dtype=torch.float32, device=x.device) if grad else None
    loss = ctypes.c_double(0.0)
    want_loss = target is not None
    call("rs_convnet_tiles", _c(w.data_ptr()), _c(x.data_ptr()), _c(mask.data_ptr()),
         _c(target.data_ptr()) if target is not None else None, _c(valid.data_ptr()) if valid is not None else None,
         ntiles, D, _c(y.data_ptr()), _c(g.data_ptr()) if g is not None else None,
         ctypes.byref(loss) if want_loss else None, _stream(stream))
    return y, g, (loss.value if want_loss else None)


def precond_apply(ham: Hamiltonian, w, R, stream=None):
    """Learned preconditioner W = K R for FP32 residual columns R [npts, nb]."""
    import torch
    W = torch.empty_like(R)
    call("rs_precond_apply", ham._h, _c(w.data_ptr()), _c(R.data_ptr()), R.stride(0), _c(W.data_ptr()), W.stride(0),
         R.shape[1], _stream(stream))
    return W


def precond_train(ham: Hamiltonian, R, X, w, n_tiles: int, epochs: int, batch: int = 64, lr: float = 1e-3,
                  seed: int = 1, tile: int = 16, stream=None):
    """Trains the network weights w (FP32 [2160], updated in place) on tiles
    of (R, X) column pairs; returns the per-epoch mean losses."""
    cfg = _lib.TrainCfg(n_tiles, tile, epochs, batch, lr, seed)
    losses = (ctypes.c_float * max(epochs, 1))()
    call("rs_precond_train_pairs", ham._h, ham.grid._h, _c(R.data_ptr()), _c(X.data_ptr()), R.stride(0), R.shape[1],
         ctypes.byref(cfg), _c(w.data_ptr()), losses, _stream(stream))
    return list(losses)[:epochs]


def precond_train_tiles(w, x, mask, target, valid, batch: int, epochs: int, lr: float = 1e-3, stream=None):
    """Adam on dense tiles [ntiles, D, D, D] (rs_precond_train_tiles); w (FP32
    [2160]) is updated in place; returns the per-epoch mean losses."""
    losses = (ctypes.c_float * max(epochs, 1))()
    call("rs_precond_train_tiles", _c(w.data_ptr()), _c(x.data_ptr()), _c(mask.data_ptr()), _c(target.data_ptr()),
         _c(valid.data_ptr()), x.shape[0], x.shape[1], batch, epochs, float(lr), losses, _stream(stream))
    return list(losses)[:epochs]


def tc_workspace(rows_a: int, rows_b: int, K: int, device=None):
    import torch
    nbytes = int(_lib.lib().rs_tc_workspace_bytes(rows_a, rows_b, K))
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def overlap_tc(grid: Grid, X, Y, work=None, stream=None):
    """Tensor-core S = dV X^T Y for FP32 device tensors (FP32-level accuracy)."""
    import torch
    nx, ny = X.shape[1], Y.shape[1]
    work = tc_workspace(nx, ny, X.shape[0], X.device) if work is None else work
    S = torch.empty((nx, ny), dtype=torch.float64, device=X.device)
    call("rs_overlap_block_tc", grid._h, _c(X.data_ptr()), X.stride(0), nx, _c(Y.data_ptr()), Y.stride(0), ny,
         _c(S.data_ptr()), S.stride(0), _c(work.data_ptr()), _stream(stream))
    return S


def rotate(X, C, Y=None, work=None, stream=None):
    """Tensor-core Y = X C for FP32 X [npts, n] and FP64 C [n, m]."""
    import torch
    npts, n = X.shape
    m = C.shape[1]
    Y = torch.empty((npts, m), dtype=torch.float32, device=X.device) if Y is None else Y
    work = tc_workspace(npts, m, n, X.device) if work is None else work
    call("rs_rotate_block", _c(X.data_ptr()), X.stride(0), n, _c(C.data_ptr()), C.stride(0), m, _c(Y.data_ptr()),
         Y.stride(0), npts, _c(work.data_ptr()), _stream(stream))
    return Y


def eigh(A, refine: int = 2, stream=None):
    """Dense symmetric eigensolver on the device: A [n, n] FP64 -> (w, V)."""
    import torch
    n = A.shape[0]
    work = torch.empty(int(_lib.lib().rs_eigh_workspace_bytes(n)), dtype=torch.uint8, device=A.device)
    w = torch.empty(n, dtype=torch.float64, device=A.device)
    V = torch.empty((n, n), dtype=torch.float64, device=A.device)
    A = A.contiguous()
    call("rs_eigh", _c(A.data_ptr()), n, _c(w.data_ptr()), _c(V.data_ptr()), refine, _c(work.data_ptr()), _stream(stream))
    return w, V


class Poisson:
    """FFT Hartree solver on a grid (rs_poisson_*)."""

    def __init__(self, grid: Grid):
        out = ctypes.c_void_p()
        call("rs_poisson_create", grid._h, ctypes.byref(out))
        self._h = out
        self.grid = grid

    def info(self):
        shape = (ctypes.c_int32 * 3)()
        rc = ctypes.c_double()
        nbytes = ctypes.c_int64()
        call("rs_poisson_info", self._h, shape, ctypes.byref(rc), ctypes.byref(nbytes))
        return tuple(shape), rc.value, nbytes.value

    def solve(self, n, vh=None, stream=None):
        """V_H for the density n (FP64 device tensor [npts]); returns vh."""
        import torch
        vh = torch.empty_like(n) if vh is None else vh
        assert n.dtype == torch.float64 and n.is_contiguous()
        call("rs_poisson_solve", self._h, _c(n.data_ptr()), _c(vh.data_ptr()), _stream(stream))
        return vh

    def close(self):
        if self._h:
            _lib.lib().rs_poisson_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SCF:
    """Self-consistent field loop around a solver (rs_scf_*)."""

    def __init__(self, solver: Solver, grid: Grid, v_ext, n0, n_electrons: float, sigma: float = 0.01,
                 alpha: float = 0.3, history: int = 8, sweeps: int = 3):
        v_ext = np.ascontiguousarray(v_ext, dtype=np.float64)
        n0 = np.ascontiguousarray(n0, dtype=np.float64)
        cfg = _lib.ScfCfg(float(n_electrons), float(sigma), float(alpha), int(history), int(sweeps))
        out = ctypes.c_void_p()
        call("rs_scf_create", solver._h, grid._h, _ptr(v_ext), _ptr(n0), ctypes.byref(cfg), ctypes.byref(out))
        self._h = out
        self.solver = solver
        self.npts = grid.npts

    def step(self, stream=None):
        """One SCF step; returns (residual, energy)."""
        r, e = ctypes.c_double(), ctypes.c_double()
        call("rs_scf_step", self._h, ctypes.byref(r), ctypes.byref(e), _stream(stream))
        return r.value, e.value

    def state(self):
        """(input density as a device tensor, occupations, mu, steps)."""
        import torch
        n = torch.empty(self.npts, dtype=torch.float64, device=self.solver.device)
        occ = np.empty(self.solver.nst)
        mu = ctypes.c_double()
        it = ctypes.c_int()
        call("rs_scf_state", self._h, _c(n.data_ptr()), _ptr(occ), ctypes.byref(mu), ctypes.byref(it))
        return n, occ, mu.value, it.value

    def close(self):
        if self._h:
            _lib.lib().rs_scf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
