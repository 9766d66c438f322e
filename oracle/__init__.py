"""FP64 CPU oracle for the element-by-element (EbE) path -- test infrastructure.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``ebe_oracle.c`` (plain C, FP64,
single-threaded), compiled on demand with gcc into ``liboracle.so`` next to it.

Each wrapper cites the passage of Marcinkowski & Valdman, "MATLAB
Implementation of Element-based Solvers", that its C function follows.
Element arrays use the paper's n_b x n_b x n_e layout (Fig. 2), returned here
as numpy arrays of shape (n_e, n_b, n_b) holding entry (i, j) at [e, i, j].
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ebe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# A prebuilt copy of the library may be named here instead (the oracle's own
# tests load copies of ebe_oracle.c with planted mistakes this way).
_LIB_OVERRIDE = os.environ.get("EBE_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

_I64 = ctypes.c_int64
_I32P = ctypes.POINTER(ctypes.c_int32)
_F64P = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile ``ebe_oracle.c`` into ``liboracle.so`` (plain gcc, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(_LIB_OVERRIDE or build())
            lib.orc_element_matrices.restype = ctypes.c_int
            lib.orc_element_matrices.argtypes = [ctypes.c_int, _I64, _I64, _F64P, _I32P, _F64P, _F64P, _F64P, _I64P]
            lib.orc_local_system.restype = None
            lib.orc_local_system.argtypes = [ctypes.c_int, _I64, ctypes.c_double, _F64P, _F64P, _I32P, _F64P, _F64P, _F64P]
            for name in ("orc_residual",):
                getattr(lib, name).restype = None
                getattr(lib, name).argtypes = [ctypes.c_int, _I64, _I64, _I32P, _F64P, _F64P, _F64P, _I32P, _I64, _F64P]
            lib.orc_apply.restype = None
            lib.orc_apply.argtypes = [ctypes.c_int, _I64, _I64, _I32P, _F64P, _F64P, _I32P, _I64, _F64P]
            lib.orc_assemble_vector.restype = None
            lib.orc_assemble_vector.argtypes = [ctypes.c_int, _I64, _I64, _I32P, _F64P, _F64P]
            lib.orc_jacobi_diag.restype = None
            lib.orc_jacobi_diag.argtypes = [ctypes.c_int, _I64, _I64, _I32P, _F64P, _F64P]
            lib.orc_assemble_dense.restype = None
            lib.orc_assemble_dense.argtypes = [ctypes.c_int, _I64, _I64, _I32P, _F64P, _F64P]
            lib.orc_pcg.restype = ctypes.c_int
            lib.orc_pcg.argtypes = [ctypes.c_int, _I64, _I64, _I32P, _F64P, _F64P, _I32P, _I64, _F64P, _F64P,
                                    ctypes.c_double, _I64, _F64P]
            lib.orc_rel_residual.restype = ctypes.c_double
            lib.orc_rel_residual.argtypes = [ctypes.c_int, _I64, _I64, _I32P, _F64P, _F64P, _I32P, _I64, _F64P, _F64P]
            lib.orc_richardson.restype = None
            lib.orc_richardson.argtypes = [ctypes.c_int, _I64, _I64, _I32P, _F64P, _F64P, _I32P, _I64, _F64P, _I64,
                                           ctypes.c_double]
            lib.orc_chebyshev2.restype = None
            lib.orc_chebyshev2.argtypes = [ctypes.c_int, _I64, _I64, _I32P, _F64P, _F64P, _I32P, _I64, _F64P, _I64,
                                           _F64P, _I64]
            lib.orc_chebyshev3.restype = None
            lib.orc_chebyshev3.argtypes = [ctypes.c_int, _I64, _I64, _I32P, _F64P, _F64P, _I32P, _I64, _F64P, _I64,
                                           ctypes.c_double, ctypes.c_double]
            lib.orc_mass_norm.restype = ctypes.c_double
            lib.orc_mass_norm.argtypes = [ctypes.c_int, _I64, _I32P, _F64P, _F64P]
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a, typ):
    return a.ctypes.data_as(typ)


class OracleError(RuntimeError):
    pass


def element_matrices(coords, elems):
    """Local K_e, M_e of Eq. matrices_K_M for every element (Sec. 1, Fig. 2).

    Returns (K, M, meas), K and M of shape (n_e, n_b, n_b), meas the element
    areas/volumes.
    """
    lib = _load()
    coords, elems = _f64(coords), _i32(elems)
    n_n, dim = coords.shape
    n_e, nb = elems.shape
    if nb != dim + 1:
        raise OracleError("n_b must be dim + 1 for P1 simplices")
    K = np.empty(n_e * nb * nb)
    M = np.empty(n_e * nb * nb)
    meas = np.empty(n_e)
    bad = ctypes.c_int64(-1)
    rc = lib.orc_element_matrices(dim, n_n, n_e, _p(coords, _F64P), _p(elems, _I32P), _p(K, _F64P),
                                  _p(M, _F64P), _p(meas, _F64P), ctypes.byref(bad))
    if rc != 0:
        raise OracleError(f"element_matrices failed rc={rc} at element {bad.value}")
    # memory order [e][j][i] (column-major blocks) -> view as [e, i, j]
    K = K.reshape(n_e, nb, nb).transpose(0, 2, 1)
    M = M.reshape(n_e, nb, nb).transpose(0, 2, 1)
    return K, M, meas


def _blocks(a):
    """(n_e, n_b, n_b) [e, i, j] array back to the paper's column-major blocks."""
    return np.ascontiguousarray(np.asarray(a).transpose(0, 2, 1), dtype=np.float64)


class Problem:
    """One discrete problem: mesh, nu, nodal f, Dirichlet/Neumann sets (Sec. 1).

    Holds the paper's element arrays K_e, M_e, A_e = K_e + nu M_e and the local
    load vectors b_e (Sec. 2), all in FP64.  ``A_override`` replaces A_e (used
    to evaluate the oracle on FP32-rounded element matrices).
    """

    def __init__(self, prob: dict, A_override=None):
        self.lib = _load()
        self.coords = _f64(prob["coords"])
        self.elems = _i32(prob["elems"])
        self.nu = float(prob["nu"])
        self.f = _f64(prob["f"])
        self.nd = _i32(prob["dirichlet"])
        self.g = _f64(prob["g"]) if prob.get("g") is not None else np.zeros(self.nd.shape[0])
        self.n_n, self.dim = self.coords.shape
        self.n_e, self.nb = self.elems.shape
        K, M, meas = element_matrices(self.coords, self.elems)
        self.K, self.M, self.meas = K, M, meas
        self._Kb, self._Mb = _blocks(K), _blocks(M)
        self._Ab = np.empty_like(self._Kb)
        self._be = np.empty(self.n_e * self.nb)
        self.lib.orc_local_system(self.nb, self.n_e, self.nu, _p(self._Kb, _F64P), _p(self._Mb, _F64P),
                                  _p(self.elems, _I32P), _p(self.f, _F64P), _p(self._Ab, _F64P),
                                  _p(self._be, _F64P))
        if A_override is not None:
            self._Ab = _blocks(A_override)

    # -- element-level data -------------------------------------------------
    @property
    def A(self):
        """A_e = K_e + nu M_e, shape (n_e, n_b, n_b) (Sec. 2)."""
        return self._Ab.reshape(self.n_e, self.nb, self.nb).transpose(0, 2, 1)

    @property
    def be(self):
        """Local load vectors b_e = M_e f_e, shape (n_e, n_b)."""
        return self._be.reshape(self.n_e, self.nb)

    def with_dirichlet(self, x):
        """Copy of x with x(nd) = g."""
        x = _f64(x).copy()
        x[self.nd] = self.g
        return x

    # -- Algorithm 1 and friends -------------------------------------------
    def residual(self, x):
        """r = mask(b - A x) by Algorithm 1 (looped version), then r(nd) = 0."""
        x = _f64(x)
        r = np.empty(self.n_n)
        self.lib.orc_residual(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(self._Ab, _F64P),
                              _p(self._be, _F64P), _p(x, _F64P), _p(self.nd, _I32P), self.nd.shape[0],
                              _p(r, _F64P))
        return r

    def apply(self, x):
        """y = mask(A x) = mask(sum_e C_e^T A_e C_e x)."""
        x = _f64(x)
        y = np.empty(self.n_n)
        self.lib.orc_apply(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(self._Ab, _F64P),
                           _p(x, _F64P), _p(self.nd, _I32P), self.nd.shape[0], _p(y, _F64P))
        return y

    def rhs(self):
        """Assembled b = sum_e C_e^T b_e (Dirichlet rows not masked)."""
        b = np.empty(self.n_n)
        self.lib.orc_assemble_vector(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(self._be, _F64P),
                                     _p(b, _F64P))
        return b

    def jacobi_diag(self):
        """d = sum_e C_e^T diag(A_e) (Dirichlet rows not masked)."""
        d = np.empty(self.n_n)
        self.lib.orc_jacobi_diag(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(self._Ab, _F64P),
                                 _p(d, _F64P))
        return d

    def dense(self, which="A"):
        """Dense sum_e C_e^T X_e C_e for X in {A, K, M} (Sec. 1); tiny meshes only."""
        if self.n_n > 5000:
            raise OracleError("dense assembly is for tiny meshes")
        src = {"A": self._Ab, "K": self._Kb, "M": self._Mb}[which]
        D = np.empty(self.n_n * self.n_n)
        self.lib.orc_assemble_dense(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(src, _F64P),
                                    _p(D, _F64P))
        return D.reshape(self.n_n, self.n_n)

    def rel_residual(self, x, x0=None):
        """|mask(b - A x)| / |mask(b - A x0)|, x0 = zero iterate carrying g by default."""
        x = _f64(x)
        if x0 is None:
            x0 = self.with_dirichlet(np.zeros(self.n_n))
        x0 = _f64(x0)
        return self.lib.orc_rel_residual(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(self._Ab, _F64P),
                                         _p(self._be, _F64P), _p(self.nd, _I32P), self.nd.shape[0],
                                         _p(x, _F64P), _p(x0, _F64P))

    def pcg(self, x0=None, rtol=1e-8, maxit=100000):
        """Jacobi-PCG to true relative residual rtol.  Returns (x, info dict)."""
        x = self.with_dirichlet(np.zeros(self.n_n) if x0 is None else x0)
        info = np.zeros(3)
        rc = self.lib.orc_pcg(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(self._Ab, _F64P),
                              _p(self._be, _F64P), _p(self.nd, _I32P), self.nd.shape[0], _p(self.g, _F64P),
                              _p(x, _F64P), rtol, maxit, _p(info, _F64P))
        return x, {"status": {0: "converged", 1: "maxit", 2: "breakdown"}.get(rc, f"error{rc}"),
                   "iterations": int(info[0]), "rel_residual": float(info[1]),
                   "residual_evals": int(info[2])}

    def richardson(self, x0, iters, omega):
        """Eq. richardson with r(nd) = 0 after each residual."""
        x = _f64(x0).copy()
        self.lib.orc_richardson(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(self._Ab, _F64P),
                                _p(self._be, _F64P), _p(self.nd, _I32P), self.nd.shape[0], _p(x, _F64P),
                                iters, omega)
        return x

    def chebyshev2(self, x0, iters, alphas):
        """Eq. Czebyshev2lev with the given cyclic root sequence alphas."""
        x = _f64(x0).copy()
        alphas = _f64(alphas)
        self.lib.orc_chebyshev2(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(self._Ab, _F64P),
                                _p(self._be, _F64P), _p(self.nd, _I32P), self.nd.shape[0], _p(x, _F64P),
                                iters, _p(alphas, _F64P), alphas.shape[0])
        return x

    def chebyshev2_bounds(self, x0, iters, lam1, lam2, N):
        """Eq. Czebyshev2lev with the roots of P_N for the bounds lam1 < lam2,
        taken in the order of chebyshev_roots (the paper's listing)."""
        return self.chebyshev2(x0, iters, chebyshev_roots(lam1, lam2, N))

    def chebyshev3(self, x0, iters, lam1, lam2):
        """Eq. Czebyshev3lev with the scaling factors of Eq. recrCk."""
        x = _f64(x0).copy()
        self.lib.orc_chebyshev3(self.nb, self.n_n, self.n_e, _p(self.elems, _I32P), _p(self._Ab, _F64P),
                                _p(self._be, _F64P), _p(self.nd, _I32P), self.nd.shape[0], _p(x, _F64P),
                                iters, lam1, lam2)
        return x

    def mass_norm(self, v):
        """sqrt(v^T M v) with M = sum_e C_e^T M_e C_e, never assembled."""
        v = _f64(v)
        return self.lib.orc_mass_norm(self.nb, self.n_e, _p(self.elems, _I32P), _p(self._Mb, _F64P), _p(v, _F64P))


def chebyshev_roots(lam1: float, lam2: float, N: int):
    """Roots alpha_k of the shifted, scaled Chebyshev polynomial P_N (Sec. 2.2),
    in the order (l1+l2)/2 + (l2-l1)/2 cos(pi (k+1/2)/N), k = 0..N-1."""
    d, c = 0.5 * (lam1 + lam2), 0.5 * (lam2 - lam1)
    return np.array([d + c * math.cos(math.pi * (k + 0.5) / N) for k in range(N)])


