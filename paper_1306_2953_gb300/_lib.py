"""ctypes binding of ``librsdft.so`` (declarations in include/rsdft.h).

Argument marshalling only: every computation runs in the library.  The
library must have been built (``python -m paper_1306_2953_gb300.build``);
loading fails loudly otherwise -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# RSDFT_LIB selects another build of the library, e.g. the bounds-checked
# debugging build librsdft_check.so (python -m paper_1306_2953_gb300.build --bounds-check)
LIB_PATH = os.environ.get("RSDFT_LIB") or os.path.join(_HERE, "librsdft.so")

RS_OK, RS_EINVAL, RS_ENOMEM, RS_ECUDA, RS_ENOTSPD, RS_ENOCONV, RS_ENAN, RS_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
RS_F64, RS_F32 = 0, 1
RS_PRECOND_NONE, RS_PRECOND_FILTER, RS_PRECOND_LEARNED, RS_PRECOND_CG = 0, 1, 2, 3
RS_ORDER_MORTON, RS_ORDER_TILECOL = -1, -2
RS_KERNEL_AUTO, RS_KERNEL_GENERIC = 0, 1
RS_EIG_BLOCK_CG, RS_EIG_RMMDIIS = 0, 1
_NAMES = {RS_EINVAL: "RS_EINVAL", RS_ENOMEM: "RS_ENOMEM", RS_ECUDA: "RS_ECUDA", RS_ENOTSPD: "RS_ENOTSPD",
          RS_ENOCONV: "RS_ENOCONV", RS_ENAN: "RS_ENAN", RS_ETIMEOUT: "RS_ETIMEOUT"}


class RsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class ProjectorSpec(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("xyz", ctypes.c_void_p), ("E", ctypes.c_void_p),
                ("r_c", ctypes.c_double), ("r_cut", ctypes.c_double)]


class TrainCfg(ctypes.Structure):
    _fields_ = [("n_tiles", ctypes.c_int), ("tile", ctypes.c_int), ("epochs", ctypes.c_int), ("batch", ctypes.c_int),
                ("lr", ctypes.c_float), ("seed", ctypes.c_uint64)]


class SolverCfg(ctypes.Structure):
    _fields_ = [("nst", ctypes.c_int), ("nb", ctypes.c_int), ("dtype", ctypes.c_int), ("precond", ctypes.c_int),
                ("tol", ctypes.c_double), ("filter_alpha", ctypes.c_double), ("n_wanted", ctypes.c_int),
                ("stall_sweeps", ctypes.c_int), ("stall_ratio", ctypes.c_double), ("rr64_every", ctypes.c_int),
                ("rr64_below", ctypes.c_double), ("rr64_always", ctypes.c_double), ("method", ctypes.c_int),
                ("rmm_steps", ctypes.c_int)]


class SolverStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("eps_f64", ctypes.c_int), ("precond", ctypes.c_int),
                ("fallback_sweep", ctypes.c_int), ("max_residual", ctypes.c_double),
                ("train_target_seconds", ctypes.c_double), ("train_fit_seconds", ctypes.c_double),
                ("lambda_max", ctypes.c_double)]


class ScfCfg(ctypes.Structure):
    _fields_ = [("n_electrons", ctypes.c_double), ("sigma", ctypes.c_double), ("alpha", ctypes.c_double),
                ("history", ctypes.c_int), ("sweeps", ctypes.c_int)]


class LearnCfg(ctypes.Structure):
    _fields_ = [("n_res", ctypes.c_int), ("cg_iters", ctypes.c_int), ("sigma", ctypes.c_double), ("train", TrainCfg)]


P = ctypes.c_void_p
I32, I64, F64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
PP = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes); restype None means "int status, checked"
SIGNATURES = {
    "rs_last_error": (I32, [ctypes.c_char_p, ctypes.c_size_t]),
    "rs_version": (ctypes.c_char_p, []),
    "rs_grid_create_spheres": (None, [P, I32, F64, F64, I32, PP]),
    "rs_grid_create_box": (None, [I32, I32, I32, F64, I32, PP]),
    "rs_grid_info": (None, [P, P, P, P, P]),
    "rs_grid_ijk": (None, [P, P]),
    "rs_grid_coords": (None, [P, P]),
    "rs_grid_point_map": (None, [P, P]),
    "rs_grid_destroy": (None, [P]),
    "rs_proj_create": (None, [P, ctypes.POINTER(ProjectorSpec), PP]),
    "rs_proj_info": (None, [P, P, P]),
    "rs_proj_tables": (None, [P, P, P, P]),
    "rs_proj_destroy": (None, [P]),
    "rs_ham_create": (None, [P, P, P, I32, PP]),
    "rs_ham_destroy": (None, [P]),
    "rs_ham_apply_block": (None, [P, P, I64, P, I64, I32, I32, P]),
    "rs_ham_apply_bytes": (I64, [P, I32, I32]),
    "rs_ham_status": (None, [P, P]),
    "rs_ham_reset_status": (None, [P]),
    "rs_ham_select_kernel": (None, [P, I32]),
    "rs_ham_set_wait_limit": (None, [P, I32]),
    "rs_ham_timing": (None, [P, I32]),
    "rs_ham_timing_read": (None, [P, P, P, P]),
    "rs_ham_launch_bytes": (None, [P, I32, I32, P, P]),
    "rs_overlap_block": (None, [P, P, I64, I32, P, I64, I32, P, I64, I32, P]),
    "rs_linalg_workspace_bytes": (I64, [I32]),
    "rs_tc_workspace_bytes": (I64, [I64, I64, I64]),
    "rs_eigh_workspace_bytes": (I64, [I32]),
    "rs_eigh": (None, [P, I32, P, P, I32, P, P]),
    "rs_overlap_block_tc": (None, [P, P, I64, I32, P, I64, I32, P, I64, P, P]),
    "rs_rotate_block": (None, [P, I64, I32, P, I64, I32, P, I64, I64, P, P]),
    "rs_orthonormalize": (None, [P, P, I64, I32, I32, P, P, P]),
    "rs_orthonormalize_noalloc": (None, [P, P, I64, I32, I32, P]),
    "rs_subspace_diag": (None, [P, P, P, I64, I32, I32, I32, P, P, P, P]),
    "rs_solver_create": (None, [P, ctypes.POINTER(SolverCfg), P, P, PP]),
    "rs_eigensolver_step": (None, [P, P, P, P, P]),
    "rs_solver_stats": (None, [P, ctypes.POINTER(SolverStats)]),
    "rs_solver_psi": (None, [P, PP]),
    "rs_solver_residual": (None, [P, I32, I32, P, I64, P]),
    "rs_solver_rayleigh_ritz_f64": (None, [P, P, P]),
    "rs_solver_certify": (None, [P, P, P, P]),
    "rs_solver_certify_smoothed": (None, [P, I32, F64, P, P, P]),
    "rs_solver_set_precond_weights": (None, [P, P]),
    "rs_solver_set_precond": (None, [P, I32]),
    "rs_solver_set_precond_cg": (None, [P, P, I32]),
    "rs_cg_workspace_bytes": (I64, [I64, I32, I32]),
    "rs_shifted_poisson_cg": (None, [P, P, P, I64, I32, I32, I32, P, P]),
    "rs_precond_apply": (None, [P, P, P, I64, P, I64, I32, P]),
    "rs_convnet_tiles": (None, [P, P, P, P, P, I32, I32, P, P, P, P]),
    "rs_precond_train_pairs": (None, [P, P, P, P, I64, I32, ctypes.POINTER(TrainCfg), P, P, P]),
    "rs_precond_train_tiles": (None, [P, P, P, P, P, I32, I32, I32, I32, ctypes.c_float, P, P]),
    "rs_precond_train": (None, [P, P, ctypes.POINTER(LearnCfg), P, P, P]),
    "rs_precond_save": (None, [P, ctypes.c_char_p]),
    "rs_precond_load": (None, [P, ctypes.c_char_p]),
    "rs_solver_destroy": (None, [P]),
    "rs_poisson_create": (None, [P, PP]),
    "rs_poisson_info": (None, [P, P, P, P]),
    "rs_poisson_solve": (None, [P, P, P, P]),
    "rs_poisson_destroy": (None, [P]),
    "rs_ham_set_potential": (None, [P, P, P]),
    "rs_solver_set_potential": (None, [P, P, P]),
    "rs_solver_checkpoint_save": (None, [P, ctypes.c_char_p]),
    "rs_solver_checkpoint_load": (None, [P, ctypes.c_char_p]),
    "rs_scf_create": (None, [P, P, P, P, ctypes.POINTER(ScfCfg), PP]),
    "rs_scf_step": (None, [P, P, P, P]),
    "rs_scf_state": (None, [P, P, P, P, P]),
    "rs_scf_destroy": (None, [P]),
}

_lock = threading.Lock()
_lib = None


def exported_names() -> list[str]:
    return list(SIGNATURES)


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1306_2953_gb300.build` "
                                   "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.restype = I32 if res is None else res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().rs_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


def call(name: str, *args) -> int:
    """Calls an int-status entry point and raises RsError on failure."""
    rc = getattr(lib(), name)(*args)
    if SIGNATURES[name][0] is None and rc != RS_OK:
        raise RsError(rc, f"{name}: {last_error()}")
    return rc
