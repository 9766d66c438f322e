"""All-core timing build of the FP64 CPU oracle -- test infrastructure.

Only the benchmark's CPU-baseline leg and the tests that compare it with the
single-thread oracle use this module.  ``ebe_oracle_par.c`` compiles the
oracle's C source together with OpenMP versions of the parts the baseline
times (element matrices, the element-based residual of Sec. 2, Eq. residual,
and Jacobi-PCG), into ``liboracle_par.so`` next to it.  It is not a checker.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import (_F64P, _HERE, _I32P, _I64, _I64P, _SRC, OracleError, _f64, _i32, _lock, _p)

_PAR_SRC = os.path.join(_HERE, "ebe_oracle_par.c")
_PAR_LIB = os.path.join(_HERE, "liboracle_par.so")
_par_lib = None


def build_parallel(force: bool = False):
    """Compile ``ebe_oracle_par.c`` (the oracle plus OpenMP versions of its
    timed parts) into ``liboracle_par.so``; returns its path, or None where
    gcc has no OpenMP."""
    newest = max(os.path.getmtime(_PAR_SRC), os.path.getmtime(_SRC))
    if force or not os.path.exists(_PAR_LIB) or os.path.getmtime(_PAR_LIB) < newest:
        tmp = _PAR_LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-fopenmp", "-I", _HERE, _PAR_SRC,
               "-o", tmp, "-lm"]
        if subprocess.run(cmd, capture_output=True).returncode != 0:
            return None
        os.replace(tmp, _PAR_LIB)
    return _PAR_LIB


def _load_parallel():
    global _par_lib
    with _lock:
        if _par_lib is None:
            path = build_parallel()
            if path is None:
                return None
            lib = ctypes.CDLL(path)
            lib.orcp_threads.restype = ctypes.c_int
            lib.orcp_colour.restype = ctypes.c_int
            lib.orcp_colour.argtypes = [ctypes.c_int, _I64, _I64, _I32P, _I32P, _I64P, ctypes.c_int]
            lib.orcp_element_matrices.restype = ctypes.c_int
            lib.orcp_element_matrices.argtypes = [ctypes.c_int, _I64, _I64, _F64P, _I32P, _F64P, _F64P]
            lib.orcp_local_system.restype = None
            lib.orcp_local_system.argtypes = [ctypes.c_int, _I64, ctypes.c_double, _F64P, _F64P, _I32P, _F64P, _F64P,
                                              _F64P]
            lib.orcp_residual.restype = None
            lib.orcp_residual.argtypes = [ctypes.c_int, _I64, _I32P, _F64P, _F64P, _F64P, _I32P, _I64, _I32P, _I64P,
                                          ctypes.c_int, _F64P]
            lib.orcp_pcg.restype = ctypes.c_int
            lib.orcp_pcg.argtypes = [ctypes.c_int, _I64, _I64, _I32P, _F64P, _F64P, _I32P, _I64, _F64P, _I32P, _I64P,
                                     ctypes.c_int, _F64P, ctypes.c_double, _I64, _F64P]
            _par_lib = lib
    return _par_lib


class ParallelTiming:
    """The oracle's element matrices, element-based residual and Jacobi-PCG on
    every host core (OpenMP, colour-parallel element loop), for the CPU
    baseline only: the tests judge with the single-thread Problem.  The
    colouring is computed once here, outside any timed region."""

    def __init__(self, prob: dict):
        self.lib = _load_parallel()
        if self.lib is None:
            raise OracleError("gcc without OpenMP: no all-core timing build")
        self.coords = _f64(prob["coords"])
        self.elems = _i32(prob["elems"])
        self.nu = float(prob["nu"])
        self.f = _f64(prob["f"])
        self.nd = _i32(prob["dirichlet"])
        self.g = _f64(prob["g"]) if prob.get("g") is not None else np.zeros(self.nd.shape[0])
        self.n_n, self.dim = self.coords.shape
        self.n_e, self.nb = self.elems.shape
        self.order = np.empty(self.n_e, dtype=np.int32)
        self.col_ptr = np.zeros(65, dtype=np.int64)
        self.n_col = self.lib.orcp_colour(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(self.order, _I32P),
                                          _p(self.col_ptr, _I64P), 64)
        if self.n_col < 0:
            raise OracleError("more than 64 colours")
        self.threads = self.lib.orcp_threads()

    def element_arrays(self):
        """(A, b_e) of Sec. 2 in the paper's layout (flat), from the coordinates."""
        sz = self.n_e * self.nb * self.nb
        K, M = np.empty(sz), np.empty(sz)
        rc = self.lib.orcp_element_matrices(self.dim, self.n_n, self.n_e, _p(self.coords, _F64P),
                                            _p(self.elems, _I32P), _p(K, _F64P), _p(M, _F64P))
        if rc != 0:
            raise OracleError(f"element matrices failed rc={rc}")
        A, be = np.empty(sz), np.empty(self.n_e * self.nb)
        self.lib.orcp_local_system(self.nb, self.n_e, self.nu, _p(K, _F64P), _p(M, _F64P), _p(self.elems, _I32P),
                                   _p(self.f, _F64P), _p(A, _F64P), _p(be, _F64P))
        return A, be

    def residual(self, A, be, x):
        x = _f64(x)
        r = np.empty(self.n_n)
        self.lib.orcp_residual(self.nb, self.n_n, _p(self.elems, _I32P), _p(A, _F64P), _p(be, _F64P),
                               _p(x, _F64P), _p(self.nd, _I32P), self.nd.shape[0], _p(self.order, _I32P),
                               _p(self.col_ptr, _I64P), self.n_col, _p(r, _F64P))
        return r

    def pcg(self, A, be, rtol=1e-8, maxit=100000):
        x = np.zeros(self.n_n)
        info = np.zeros(3)
        rc = self.lib.orcp_pcg(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(A, _F64P), _p(be, _F64P),
                               _p(self.nd, _I32P), self.nd.shape[0], _p(self.g, _F64P), _p(self.order, _I32P),
                               _p(self.col_ptr, _I64P), self.n_col, _p(x, _F64P), rtol, maxit, _p(info, _F64P))
        status = "converged" if rc == 0 else "maxit" if rc == 1 else "breakdown" if rc == 2 else f"error{rc}"
        return x, {"status": status, "iterations": int(info[0]), "rel_residual": float(info[1]),
                   "residual_evals": int(info[2])}
