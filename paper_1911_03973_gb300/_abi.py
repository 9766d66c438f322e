"""ctypes declarations of include/ebe.h (argument marshalling only).

The shared library is built in-tree (``paper_1911_03973_gb300/libebe.so``).
If it is missing this module raises at load time: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libebe.so")

# status codes (ebe_status)
EBE_OK = 0
EBE_INVALID_ARG = 1
EBE_INDEX_RANGE = 2
EBE_DEGENERATE_ELEMENT = 3
EBE_SINGULAR = 4
EBE_CUDA_ERROR = 5
EBE_OOM = 6
EBE_MAXIT = 7
EBE_BREAKDOWN = 8
EBE_STALL = 9
EBE_NOT_READY = 10

EBE_F64 = 0
EBE_F32 = 1
EBE_F64_DW = 2
EBE_STORE_FP64 = 0
EBE_STORE_MIXED = 1
EBE_PREC_FP64 = 0
EBE_PREC_MIXED = 1
EBE_PREC_MIXED_TEXTBOOK = 2
EBE_SCATTER_PATCH = 0
EBE_SCATTER_COLOUR = 1
EBE_SCATTER_NODE = 2
EBE_SCATTER_ATOMIC = 3


class ebe_mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_b", ctypes.c_int32), ("n_n", ctypes.c_int64),
                ("n_e", ctypes.c_int64), ("coords", ctypes.POINTER(ctypes.c_double)),
                ("elems", ctypes.POINTER(ctypes.c_int32))]


class ebe_create_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("patch_elems", ctypes.c_int32)]


class ebe_solve_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("delta", ctypes.c_double), ("stall_updates", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("race_iters", ctypes.c_int32)]


class ebe_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int64), ("true_residuals", ctypes.c_int64),
                ("rel_residual", ctypes.c_double), ("r0_norm", ctypes.c_double), ("solve_ms", ctypes.c_double)]


class ebe_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("n_patches", ctypes.c_int64), ("patch_elems", ctypes.c_int64),
                ("n_shared_nodes", ctypes.c_int64), ("n_halo", ctypes.c_int64), ("max_colours", ctypes.c_int64),
                ("n_global_colours", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("device_error", ctypes.c_int64)]


class ebe_partition_sizes(ctypes.Structure):
    _fields_ = [("n_patches", ctypes.c_int64), ("n_slots", ctypes.c_int64), ("n_pnode", ctypes.c_int64),
                ("n_colptr", ctypes.c_int64), ("n_shared", ctypes.c_int64), ("n_halo", ctypes.c_int64),
                ("max_nodes", ctypes.c_int32), ("max_colours", ctypes.c_int32), ("patch_elems", ctypes.c_int32)]


class ebe_batch_config(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("tile_nodes", ctypes.c_int32), ("barrier_ns", ctypes.c_int64)]


class ebe_batch_info(ctypes.Structure):
    _fields_ = [("loops", ctypes.c_int64), ("launches", ctypes.c_int32), ("n_converged", ctypes.c_int32),
                ("solve_ms", ctypes.c_double), ("config", ebe_batch_config), ("phase_ms", ctypes.c_double * 4)]


_H = ctypes.c_void_p
_VP = ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)
_F64P = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)

# (name, restype, argtypes) of every entry point declared in include/ebe.h
SIGNATURES = [
    ("ebe_create", ctypes.c_int, [ctypes.POINTER(_H), ctypes.POINTER(ebe_mesh), ctypes.POINTER(ebe_create_opts), _VP]),
    ("ebe_destroy", None, [_H]),
    ("ebe_last_error", ctypes.c_char_p, [_H]),
    ("ebe_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("ebe_solve_opts_default", None, [ctypes.POINTER(ebe_solve_opts)]),
    ("ebe_set_problem", ctypes.c_int, [_H, ctypes.c_double, _F64P, _I32P, ctypes.c_int64, _F64P, _I32P,
                                       ctypes.c_int64]),
    ("ebe_assemble", ctypes.c_int, [_H, ctypes.c_int32]),
    ("ebe_element_matrices", ctypes.c_int, [_H, _VP, _VP]),
    ("ebe_get_local_matrices", ctypes.c_int, [_H, _VP, ctypes.c_int32]),
    ("ebe_get_rhs", ctypes.c_int, [_H, _VP]),
    ("ebe_jacobi_diag", ctypes.c_int, [_H, _VP]),
    ("ebe_residual", ctypes.c_int, [_H, _VP, _VP, ctypes.c_int32]),
    ("ebe_apply", ctypes.c_int, [_H, _VP, _VP, ctypes.c_int32]),
    ("ebe_time_operator", ctypes.c_int, [_H, _VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _F64P]),
    ("ebe_residual_variant", ctypes.c_int, [_H, _VP, _VP, ctypes.c_int32]),
    ("ebe_solve", ctypes.c_int, [_H, _VP, ctypes.POINTER(ebe_solve_opts), ctypes.POINTER(ebe_solve_info)]),
    ("ebe_solve_host", ctypes.c_int, [_H, _F64P, ctypes.POINTER(ebe_solve_opts), ctypes.POINTER(ebe_solve_info)]),
    ("ebe_create_batch", ctypes.c_int, [ctypes.POINTER(_H), ctypes.POINTER(ebe_mesh), ctypes.c_int32,
                                        ctypes.POINTER(ebe_create_opts), _VP]),
    ("ebe_batch_layout", ctypes.c_int, [_H, _I32P, _I64P, _I64P]),
    ("ebe_set_problem_batch", ctypes.c_int, [_H, _F64P, _F64P, _I32P, ctypes.c_int64, _F64P, _I32P,
                                             ctypes.c_int64]),
    ("ebe_solve_batch", ctypes.c_int, [_H, _VP, ctypes.POINTER(ebe_solve_opts), ctypes.POINTER(ebe_solve_info),
                                       ctypes.POINTER(ebe_batch_info)]),
    ("ebe_solve_batch_host", ctypes.c_int, [_H, _F64P, ctypes.POINTER(ebe_solve_opts),
                                            ctypes.POINTER(ebe_solve_info), ctypes.POINTER(ebe_batch_info)]),
    ("ebe_set_batch_config", ctypes.c_int, [_H, ctypes.POINTER(ebe_batch_config)]),
    ("ebe_batch_tune", ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ebe_batch_config),
                                      ctypes.POINTER(ebe_batch_config), _F64P, ctypes.c_int32, _I32P]),
    ("ebe_mpnn_n_params", ctypes.c_int64, []),
    ("ebe_mpnn_create", ctypes.c_int, [ctypes.POINTER(_H), ctypes.c_int32, _F64P]),
    ("ebe_mpnn_destroy", None, [_H]),
    ("ebe_mpnn_last_error", ctypes.c_char_p, [_H]),
    ("ebe_mpnn_set_params", ctypes.c_int, [_H, _F64P]),
    ("ebe_mpnn_get_params", ctypes.c_int, [_H, _F64P]),
    ("ebe_mpnn_apply", ctypes.c_int, [_H, _H, _VP, _VP]),
    ("ebe_mpnn_grad", ctypes.c_int, [_H, _H, _VP, _VP, _VP, _F64P]),
    ("ebe_mpnn_train_step", ctypes.c_int, [_H, _H, _VP, _VP, ctypes.c_double, _F64P]),
    ("ebe_solve_learned", ctypes.c_int, [_H, _H, _VP, ctypes.POINTER(ebe_solve_opts), ctypes.POINTER(ebe_solve_info),
                                         _I32P]),
    ("ebe_residual_noalloc", ctypes.c_int, [_H, _VP, _VP]),
    ("ebe_richardson", ctypes.c_int, [_H, _VP, ctypes.c_int64, ctypes.c_double]),
    ("ebe_chebyshev2", ctypes.c_int, [_H, _VP, ctypes.c_int64, _F64P, ctypes.c_int64]),
    ("ebe_time_cg_pass", ctypes.c_int, [_H, ctypes.c_int32, _F64P]),
    ("ebe_chebyshev2_bounds", ctypes.c_int, [_H, _VP, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int64]),
    ("ebe_chebyshev3", ctypes.c_int, [_H, _VP, ctypes.c_int64, ctypes.c_double, ctypes.c_double]),
    ("ebe_get_stats", ctypes.c_int, [_H, ctypes.POINTER(ebe_stats)]),
    ("ebe_partition_export", ctypes.c_int, [ctypes.POINTER(ebe_mesh), ctypes.POINTER(ebe_partition_sizes),
                                            _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("ebe_partition_export_batch", ctypes.c_int, [ctypes.POINTER(ebe_mesh), ctypes.c_int32,
                                                  ctypes.POINTER(ebe_partition_sizes), _VP, _VP, _VP, _VP, _VP,
                                                  _VP, _VP, _VP, _VP]),
]

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libebe.so and declare its signatures.  Raises if it is not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"libebe.so is not built ({path}); run "
                                  "`python -m paper_1911_03973_gb300.build` (nvcc, sm_103a)")
            lib = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib
