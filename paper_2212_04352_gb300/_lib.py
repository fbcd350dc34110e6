"""ctypes declarations of the libftwa C ABI (include/ftwa.h)."""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libftwa.so")

FTWA_OK = 0
FTWA_ERR_INVALID_ARGUMENT = -1
FTWA_ERR_UNSUPPORTED = -2
FTWA_ERR_OUT_OF_MEMORY = -3
FTWA_ERR_CUDA = -4
FTWA_ERR_DEVICE_TIMEOUT = -5
FTWA_ERR_NONFINITE = -6
FTWA_FP64 = 0
FTWA_FP32 = 1
FTWA_GRAM_FP64 = 0
FTWA_GRAM_BF16X3 = 1
FTWA_MAX_SITES = 256
FTWA_MOMENTS_NOALLOC_MAX_TK = 131072

# every symbol include/ftwa.h declares
EXPORTS = ("ftwa_plan", "ftwa_destroy", "ftwa_get_info", "ftwa_sample", "ftwa_set_initial_basis", "ftwa_philox",
           "ftwa_evolve", "ftwa_evolve_at", "ftwa_set_drive", "ftwa_set_hopping_drive", "ftwa_set_interaction",
           "ftwa_ed_plan", "ftwa_ed_destroy", "ftwa_ed_info", "ftwa_ed_evolve",
           "ftwa_moments", "ftwa_moments_noalloc", "ftwa_adjoint", "ftwa_adjoint_corr", "ftwa_autotune", "ftwa_batch_create",
           "ftwa_batch_create_persistent",
           "ftwa_batch_launch", "ftwa_batch_destroy", "ftwa_status", "ftwa_debug_force_timeout",
           "ftwa_debug_tile_check", "ftwa_measure_peak", "ftwa_error_string",
           "ftwa_version")


class Lattice(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int32), ("n_bonds", ctypes.c_int32),
                ("bonds", ctypes.c_void_p), ("t_bond", ctypes.c_void_p)]


class InitState(ctypes.Structure):
    _fields_ = [("n_up", ctypes.c_void_p), ("n_dn", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("dt", ctypes.c_double), ("out_every", ctypes.c_int32),
                ("cluster_override", ctypes.c_int32), ("threads_override", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("timeout_us", ctypes.c_uint64), ("variant", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("n_sites", "n_bonds", "precision", "cluster", "threads", "samples_per_cta", "smem_bytes",
                 "tmem_cols", "grid_clusters", "units_per_warp", "variant")]


class FtwaError(RuntimeError):
    def __init__(self, code, where, text):
        super().__init__(f"{where} failed: {text} ({code})")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libftwa.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libftwa.so not found at {path}: build it with __graft_entry__.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    lib.ftwa_plan.argtypes = [ctypes.POINTER(Lattice), f64, f64, f64, ctypes.POINTER(InitState),
                              ctypes.POINTER(Options), ctypes.POINTER(P)]
    lib.ftwa_destroy.argtypes = [P]
    lib.ftwa_destroy.restype = None
    lib.ftwa_get_info.argtypes = [P, ctypes.POINTER(PlanInfo)]
    lib.ftwa_sample.argtypes = [P, u64, i64, i64, P, P]
    lib.ftwa_set_initial_basis.argtypes = [P, P, P, P]
    lib.ftwa_philox.argtypes = [u64, i64, i32, i64, i64, P, P]
    lib.ftwa_evolve.argtypes = [P, P, i64, i64, P, P]
    lib.ftwa_evolve_at.argtypes = [P, P, i64, i64, f64, P, P]
    lib.ftwa_set_drive.argtypes = [P, P, f64, f64, f64, f64]
    lib.ftwa_set_interaction.argtypes = [P, P]
    lib.ftwa_set_hopping_drive.argtypes = [P, f64, f64, f64, f64, f64]
    lib.ftwa_ed_plan.argtypes = [ctypes.POINTER(Lattice), f64, i32, i32, ctypes.POINTER(P)]
    lib.ftwa_ed_destroy.argtypes = [P]
    lib.ftwa_ed_destroy.restype = None
    lib.ftwa_ed_info.argtypes = [P, ctypes.POINTER(ctypes.c_int64), P, P]
    lib.ftwa_ed_evolve.argtypes = [P, P, P, f64, i32, P, P, P]
    lib.ftwa_moments.argtypes = [P, P, i64, i32, P, P, P, i32, P]
    lib.ftwa_moments_noalloc.argtypes = [P, i32, i32, i64, i32, P, P, P, P]
    lib.ftwa_adjoint.argtypes = [P, u64, i64, i64, i32, P, P, P, P, P]
    lib.ftwa_adjoint_corr.argtypes = [P, u64, i64, i64, i32, P, P, P, P, P, P, P]
    lib.ftwa_autotune.argtypes = [P, i64, i32, P]
    lib.ftwa_batch_create.argtypes = [P, i32, P, P, i64, P, ctypes.POINTER(P)]
    lib.ftwa_batch_create_persistent.argtypes = [P, i32, P, P, i64, P, i32, ctypes.POINTER(P)]
    lib.ftwa_batch_launch.argtypes = [P, P]
    lib.ftwa_batch_destroy.argtypes = [P]
    lib.ftwa_batch_destroy.restype = None
    lib.ftwa_status.argtypes = [P, P]
    lib.ftwa_debug_force_timeout.argtypes = [P, i32]
    lib.ftwa_measure_peak.argtypes = [i32, ctypes.POINTER(ctypes.c_double), P]
    lib.ftwa_debug_tile_check.argtypes = [i32, i32, P, P, i32, i32, ctypes.POINTER(ctypes.c_int64), ctypes.c_char_p,
                                          i32]
    lib.ftwa_error_string.argtypes = [ctypes.c_int]
    lib.ftwa_error_string.restype = ctypes.c_char_p
    lib.ftwa_version.restype = ctypes.c_int
    for name in ("ftwa_plan", "ftwa_get_info", "ftwa_sample", "ftwa_philox", "ftwa_evolve", "ftwa_moments",
                 "ftwa_moments_noalloc", "ftwa_autotune", "ftwa_batch_create", "ftwa_batch_create_persistent",
                 "ftwa_batch_launch",
                 "ftwa_adjoint", "ftwa_adjoint_corr", "ftwa_status", "ftwa_debug_force_timeout",
                 "ftwa_debug_tile_check", "ftwa_measure_peak"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def check(code: int, where: str):
    if code != FTWA_OK:
        raise FtwaError(code, where, load().ftwa_error_string(code).decode())
