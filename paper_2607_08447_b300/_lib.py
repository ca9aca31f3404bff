"""ctypes binding of the C ABI declared in include/khp.h (argument marshalling only).

Every function of the header is bound under its own name.  The library is
the in-tree ``libkhp.so`` built by ``paper_2607_08447_b300.build``; there is
no fallback: importing this module on a machine without the built library
raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkhp.so")

KHP_OK = 0
KHP_BATCH_GRAPH = 1
KHP_BATCH_AUTOTUNE = 2
KHP_BATCH_GROUPED = 4
STATUS_NAMES = {0: "KHP_OK", 1: "KHP_ERR_INVALID_ARG", 2: "KHP_ERR_CUDA", 3: "KHP_ERR_OOM",
                4: "KHP_ERR_NOT_CONVERGED", 5: "KHP_ERR_BREAKDOWN", 6: "KHP_ERR_STATE",
                7: "KHP_ERR_DEGENERATE"}

EXPORTED = ["khp_create_grid", "khp_project_rows", "khp_pair_densities", "khp_position_moments", "khp_create_grid_h0", "khp_poisson_create", "khp_poisson_solve", "khp_poisson_solve_many", "khp_poisson_set_preconditioner", "khp_sp_update",
            "khp_poisson_destroy", "khp_set_potential_strain_field", "khp_apply", "khp_project", "khp_rotate",
            "khp_eigensolve",
            "khp_eigensolve_batched",
            "khp_density", "khp_eigs_backward", "khp_eigs_backward_noalloc", "khp_destroy",
            "khp_last_error", "khp_version", "khp_sp_anderson", "khp_sp_anderson_reset",
            "khp_fermi_level", "khp_filter_step", "khp_state_densities", "khp_sp_relax_occupations"]


class Material(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("gamma1", "gamma2", "gamma3", "delta_so", "kappa", "a_v", "b", "d")]


class SolverOpts(ctypes.Structure):
    _fields_ = [("n_states", ctypes.c_int), ("block_m", ctypes.c_int), ("degree", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("refine_sweeps", ctypes.c_int), ("tol_ev", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("warm_start_dev", ctypes.c_void_p),
                ("warm_cols", ctypes.c_int), ("projections", ctypes.c_int), ("start", ctypes.c_int),
                ("block_out_dev", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("iterations_fp32", ctypes.c_int),
                ("converged", ctypes.c_int), ("shifted_cholesky", ctypes.c_int),
                ("filter_applies", ctypes.c_longlong), ("max_residual", ctypes.c_double),
                ("lambda_upper", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_filter_fp64", ctypes.c_double), ("ms_filter_fp32", ctypes.c_double),
                ("launches_fp64", ctypes.c_longlong), ("launches_fp32", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("point_vectors", ctypes.c_double),
                ("pv_fp64", ctypes.c_double), ("pv_fp32", ctypes.c_double),
                ("flops_per_pv", ctypes.c_double), ("bytes_per_pv_fp64", ctypes.c_double),
                ("bytes_per_pv_fp32", ctypes.c_double), ("block_m", ctypes.c_int),
                ("batch_rounds", ctypes.c_int), ("batch_graphs", ctypes.c_int),
                ("autotune_ms", ctypes.c_double),
                ("ms_gram", ctypes.c_double), ("ms_small", ctypes.c_double), ("ms_rotate", ctypes.c_double),
                ("ms_between", ctypes.c_double), ("bytes_rr", ctypes.c_double), ("n_history", ctypes.c_int),
                ("res_history", ctypes.c_double * 64), ("ms_start", ctypes.c_double),
                ("start_iterations", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "res_history"}
        d["res_history"] = [self.res_history[i] for i in range(min(self.n_history, 64))]
        return d


class KHPError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libkhp.so and declare the signatures of every exported function."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libkhp.so not built at {path}; run `python -m paper_2607_08447_b300.build`")
    lib = ctypes.CDLL(path)
    vp, i, d, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
    lib.khp_create_grid.argtypes = [ctypes.POINTER(vp), i, i, i, d, ctypes.POINTER(Material), dp, vp, vp]
    lib.khp_create_grid_h0.argtypes = [ctypes.POINTER(vp), i, i, i, d, ctypes.POINTER(Material), dp, vp, vp]
    lib.khp_poisson_create.argtypes = [ctypes.POINTER(vp), i, i, i, d, d, vp, vp, vp]
    lib.khp_poisson_solve.argtypes = [vp, vp, vp, d, i, ctypes.POINTER(i), dp]
    lib.khp_poisson_set_preconditioner.argtypes = [vp, i, ctypes.POINTER(i)]
    lib.khp_poisson_solve_many.argtypes = [vp, vp, vp, i, i, d, i, ctypes.POINTER(i), dp]
    lib.khp_sp_update.argtypes = [vp, vp, vp, d, vp, dp]
    lib.khp_sp_anderson.argtypes = [vp, vp, vp, d, i, vp, dp]
    lib.khp_sp_anderson_reset.argtypes = [vp]
    lib.khp_fermi_level.argtypes = [dp, i, d, d, dp, dp]
    lib.khp_state_densities.argtypes = [vp, vp, i, vp]
    lib.khp_sp_relax_occupations.argtypes = [vp, vp, dp, i, d, d, vp, vp, vp, d, dp, dp]
    lib.khp_poisson_destroy.argtypes = [vp]
    lib.khp_project.argtypes = [vp, vp, vp, i, i, vp, vp]
    lib.khp_project_rows.argtypes = [vp, vp, vp, ctypes.c_longlong, i, i, vp, vp]
    lib.khp_rotate.argtypes = [vp, vp, vp, vp, i, i, vp, vp]
    lib.khp_set_potential_strain_field.argtypes = [vp, vp, vp, vp, dp, i, dp, i]
    lib.khp_apply.argtypes = [vp, vp, vp, i, i]
    lib.khp_filter_step.argtypes = [vp, vp, vp, vp, dp, vp, i, i, i, d, d, d, i]
    lib.khp_eigensolve.argtypes = [vp, ctypes.POINTER(SolverOpts), dp, vp, dp, ctypes.POINTER(Stats)]
    lib.khp_eigensolve_batched.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(SolverOpts), dp,
                                           ctypes.POINTER(vp), dp, ctypes.POINTER(Stats), i]
    lib.khp_density.argtypes = [vp, vp, i, dp, vp]
    lib.khp_pair_densities.argtypes = [vp, vp, i, vp]
    lib.khp_position_moments.argtypes = [vp, vp, i, vp]
    lib.khp_eigs_backward.argtypes = [vp, vp, dp, i, dp, vp, vp, vp, i, dp]
    lib.khp_eigs_backward_noalloc.argtypes = [vp, vp, dp, i, dp, vp, vp, vp, i, dp]
    lib.khp_destroy.argtypes = [vp]
    lib.khp_last_error.argtypes = []
    lib.khp_last_error.restype = ctypes.c_char_p
    lib.khp_version.argtypes = []
    lib.khp_version.restype = ctypes.c_int
    for name in EXPORTED:
        if name not in ("khp_last_error", "khp_version"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def check(status: int, allow=()):
    if status != KHP_OK and status not in allow:
        raise KHPError(status, load().khp_last_error().decode())
    return status


def dptr(arr):
    """ctypes double* of a contiguous float64 numpy array (or None)."""
    if arr is None:
        return None
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
