"""GB300 element-by-element (EbE) finite-element residual and Jacobi-PCG.

Python binding of ``libebe.so`` (C ABI in ``include/ebe.h``) with the same
function names.  It only marshals arguments: every step of the residual, the
element matrices and the solver runs in the library's CUDA kernels.  Host
arrays are numpy arrays; device buffers are CUDA tensors (anything with
``data_ptr()``, ``dtype``, ``is_cuda`` and ``numel()``).

The library is loaded on first use; when it is missing the call raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import (EBE_BREAKDOWN, EBE_CUDA_ERROR, EBE_DEGENERATE_ELEMENT, EBE_F32, EBE_F64, EBE_F64_DW,  # noqa: F401
                   EBE_INDEX_RANGE, EBE_INVALID_ARG, EBE_MAXIT, EBE_NOT_READY, EBE_OK, EBE_OOM, EBE_PREC_FP64,
                   EBE_PREC_MIXED, EBE_PREC_MIXED_TEXTBOOK, EBE_SCATTER_ATOMIC, EBE_SCATTER_COLOUR, EBE_SCATTER_NODE, EBE_SCATTER_PATCH,
                   EBE_SINGULAR, EBE_STALL, EBE_STORE_FP64, EBE_STORE_MIXED)

SOLVER_OUTCOMES = (_abi.EBE_OK, _abi.EBE_MAXIT, _abi.EBE_BREAKDOWN, _abi.EBE_STALL)


class EbeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{ebe_status_string(status)}: {message}")
        self.status = status


class Handle:
    """Owner of an ``ebe_handle*``; keeps the mesh sizes for argument checks."""

    def __init__(self, ptr, dim, n_b, n_n, n_e):
        self.ptr = ptr
        self.dim, self.n_b, self.n_n, self.n_e = dim, n_b, n_n, n_e

    def __del__(self):
        try:
            ebe_destroy(self)
        except Exception:
            pass


def _lib():
    return _abi.load()


def ebe_status_string(status: int) -> str:
    return _lib().ebe_status_string(int(status)).decode()


def ebe_last_error(h: Handle | None) -> str:
    return _lib().ebe_last_error(h.ptr if h is not None else None).decode()


def _check(h, status):
    if status != _abi.EBE_OK:
        raise EbeError(status, ebe_last_error(h))


def _dev(t, dtype_code=None, n=None, name="buffer"):
    """Device pointer of a CUDA tensor (contiguous), with optional checks."""
    if t is None:
        return None
    if not getattr(t, "is_cuda", False):
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} entries, has {t.numel()}")
    if dtype_code is not None:
        want = "torch.float64" if dtype_code == EBE_F64 else "torch.float32"
        if str(t.dtype) != want:
            raise TypeError(f"{name} must be {want}, is {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _dtype_code(t):
    s = str(t.dtype)
    if s == "torch.float64":
        return EBE_F64
    if s == "torch.float32":
        return EBE_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _host_f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _host_i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def ebe_create(coords, elems, device: int = 0, stream: int | None = None) -> Handle:
    """ebe_create: coords host [n_n][dim] float64, elems host [n_e][n_b] int32.

    ``stream``: a ``cudaStream_t`` value (e.g. ``torch.cuda.current_stream().cuda_stream``);
    None / 0 means the legacy default stream.
    """
    coords = _host_f64(coords)
    elems = _host_i32(elems)
    if coords.ndim != 2 or elems.ndim != 2:
        raise ValueError("coords and elems must be 2-D")
    mesh = _abi.ebe_mesh(coords.shape[1], elems.shape[1], coords.shape[0], elems.shape[0],
                         coords.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         elems.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    opts = _abi.ebe_create_opts(device, 0)
    ptr = ctypes.c_void_p()
    st = _lib().ebe_create(ctypes.byref(ptr), ctypes.byref(mesh), ctypes.byref(opts),
                           ctypes.c_void_p(stream or 0))
    if st != _abi.EBE_OK:
        raise EbeError(st, ebe_last_error(None))
    return Handle(ptr, coords.shape[1], elems.shape[1], coords.shape[0], elems.shape[0])


def ebe_destroy(h: Handle) -> None:
    if h is not None and h.ptr is not None and h.ptr.value:
        _lib().ebe_destroy(h.ptr)
        h.ptr = ctypes.c_void_p()


def ebe_set_problem(h: Handle, nu: float, f_nodal, dirichlet, g=None, neumann=None) -> None:
    f = _host_f64(f_nodal)
    if f.shape != (h.n_n,):
        raise ValueError("f_nodal must have n_n entries")
    nd = _host_i32(dirichlet if dirichlet is not None else np.zeros(0))
    gv = None if g is None else _host_f64(g)
    if gv is not None and gv.shape != nd.shape:
        raise ValueError("g must match the Dirichlet set")
    nn = _host_i32(neumann if neumann is not None else np.zeros(0))
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t)) if a is not None and a.size else None  # noqa: E731
    _check(h, _lib().ebe_set_problem(h.ptr, float(nu), P(f, ctypes.c_double), P(nd, ctypes.c_int32), nd.size,
                                     P(gv, ctypes.c_double), P(nn, ctypes.c_int32), nn.size))


def ebe_assemble(h: Handle, store: int = EBE_STORE_FP64) -> None:
    _check(h, _lib().ebe_assemble(h.ptr, int(store)))


def ebe_element_matrices(h: Handle, K=None, M=None) -> None:
    n = h.n_e * h.n_b * h.n_b
    _check(h, _lib().ebe_element_matrices(h.ptr, _dev(K, EBE_F64, n, "K"), _dev(M, EBE_F64, n, "M")))


def ebe_get_local_matrices(h: Handle, A) -> None:
    code = _dtype_code(A)
    _check(h, _lib().ebe_get_local_matrices(h.ptr, _dev(A, code, h.n_e * h.n_b * h.n_b, "A"), code))


def ebe_get_rhs(h: Handle, b) -> None:
    _check(h, _lib().ebe_get_rhs(h.ptr, _dev(b, EBE_F64, h.n_n, "b")))


def ebe_jacobi_diag(h: Handle, d) -> None:
    _check(h, _lib().ebe_jacobi_diag(h.ptr, _dev(d, EBE_F64, h.n_n, "d")))


def _op_code(x, double_word):
    code = _dtype_code(x)
    if not double_word:
        return code, code
    if code != EBE_F64:
        raise TypeError("the double-word form takes float64 vectors")
    return EBE_F64_DW, EBE_F64


def ebe_residual(h: Handle, x, r, double_word: bool = False) -> None:
    """r = mask(b - A x); double_word=True runs the FP64 arithmetic as FP32 pairs (EBE_F64_DW)."""
    code, vt = _op_code(x, double_word)
    _check(h, _lib().ebe_residual(h.ptr, _dev(x, vt, h.n_n, "x"), _dev(r, vt, h.n_n, "r"), code))


def ebe_apply(h: Handle, x, y, double_word: bool = False) -> None:
    code, vt = _op_code(x, double_word)
    _check(h, _lib().ebe_apply(h.ptr, _dev(x, vt, h.n_n, "x"), _dev(y, vt, h.n_n, "y"), code))


def ebe_time_operator(h: Handle, x, y, apply: bool = True, reps: int = 20, double_word: bool = False) -> tuple:
    """Mean ms per launch of (patch kernel, fix-up kernel), CUDA events on the handle's stream."""
    code, vt = _op_code(x, double_word)
    ms = (ctypes.c_double * 2)()
    _check(h, _lib().ebe_time_operator(h.ptr, _dev(x, vt, h.n_n, "x"), _dev(y, vt, h.n_n, "y"), code,
                                       int(bool(apply)), int(reps), ms))
    return float(ms[0]), float(ms[1])


def ebe_time_cg_pass(h: Handle, reps: int = 20) -> tuple:
    """Mean ms per launch of (patch kernel, fix-up kernel) of one single-sync
    mixed-precision CG iteration, CUDA events on the handle's stream."""
    ms = (ctypes.c_double * 2)()
    _check(h, _lib().ebe_time_cg_pass(h.ptr, int(reps), ms))
    return float(ms[0]), float(ms[1])


def ebe_residual_variant(h: Handle, x, r, scatter: int) -> None:
    _check(h, _lib().ebe_residual_variant(h.ptr, _dev(x, EBE_F64, h.n_n, "x"), _dev(r, EBE_F64, h.n_n, "r"),
                                          int(scatter)))


def ebe_solve_opts_default() -> dict:
    """Defaults of ebe_solve_opts as a dict."""
    o = _abi.ebe_solve_opts()
    _lib().ebe_solve_opts_default(ctypes.byref(o))
    return {k: getattr(o, k) for k, _ in _abi.ebe_solve_opts._fields_}


def _opts(rtol, maxit, precision, chunk, delta, stall_updates, use_graph):
    o = _abi.ebe_solve_opts()
    _lib().ebe_solve_opts_default(ctypes.byref(o))
    if rtol is not None:
        o.rtol = rtol
    if maxit is not None:
        o.maxit = maxit
    if precision is not None:
        o.precision = precision
    if chunk is not None:
        o.chunk = chunk
    if delta is not None:
        o.delta = delta
    if stall_updates is not None:
        o.stall_updates = stall_updates
    if use_graph is not None:
        o.use_graph = int(use_graph)
    return o


def _info_dict(info):
    return {"status": ebe_status_string(info.status), "status_code": info.status, "iterations": info.iterations,
            "true_residuals": info.true_residuals, "rel_residual": info.rel_residual, "r0_norm": info.r0_norm,
            "solve_ms": info.solve_ms}


def ebe_solve(h: Handle, x, rtol=None, maxit=None, precision=None, chunk=None, delta=None, stall_updates=None,
              use_graph=None) -> dict:
    """ebe_solve on a device x (float64 CUDA tensor, in: x0, out: solution).

    Returns the ebe_solve_info fields; raises only for errors, not for the
    solver outcomes EBE_MAXIT / EBE_BREAKDOWN / EBE_STALL (see ``status``).
    """
    o = _opts(rtol, maxit, precision, chunk, delta, stall_updates, use_graph)
    info = _abi.ebe_solve_info()
    st = _lib().ebe_solve(h.ptr, _dev(x, EBE_F64, h.n_n, "x"), ctypes.byref(o), ctypes.byref(info))
    if st not in SOLVER_OUTCOMES:
        _check(h, st)
    return _info_dict(info)


def ebe_solve_host(h: Handle, x, rtol=None, maxit=None, precision=None, chunk=None, delta=None,
                   stall_updates=None, use_graph=None) -> dict:
    """ebe_solve_host on a host float64 numpy array x (updated in place)."""
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous and x.size == h.n_n):
        raise TypeError("x must be a contiguous float64 numpy array of n_n entries")
    o = _opts(rtol, maxit, precision, chunk, delta, stall_updates, use_graph)
    info = _abi.ebe_solve_info()
    st = _lib().ebe_solve_host(h.ptr, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(o),
                               ctypes.byref(info))
    if st not in SOLVER_OUTCOMES:
        _check(h, st)
    return _info_dict(info)


def ebe_create_batch(meshes, device: int = 0, stream: int | None = None) -> Handle:
    """ebe_create_batch: meshes = [(coords, elems), ...] host arrays, one pair per problem.

    The handle's node / element numbering is the concatenation in the given
    order; ``h.node_off`` / ``h.elem_off`` hold the offsets (ebe_batch_layout).
    """
    if len(meshes) < 1:
        raise ValueError("a batch needs at least one mesh")
    arr, keep = _mesh_array(meshes)
    opts = _abi.ebe_create_opts(device, 0)
    ptr = ctypes.c_void_p()
    st = _lib().ebe_create_batch(ctypes.byref(ptr), arr, len(meshes), ctypes.byref(opts),
                                 ctypes.c_void_p(stream or 0))
    if st != _abi.EBE_OK:
        raise EbeError(st, ebe_last_error(None))
    h = Handle(ptr, keep[0].shape[1], keep[1].shape[1], sum(a.shape[0] for a in keep[0::2]),
               sum(a.shape[0] for a in keep[1::2]))
    h.n_problems, h.node_off, h.elem_off = ebe_batch_layout(h)
    return h


def ebe_batch_layout(h: Handle):
    """(n_problems, node_off[n_problems + 1], elem_off[n_problems + 1]) of the union numbering."""
    n = ctypes.c_int32()
    _check(h, _lib().ebe_batch_layout(h.ptr, ctypes.byref(n), None, None))
    no = np.empty(n.value + 1, np.int64)
    eo = np.empty(n.value + 1, np.int64)
    _check(h, _lib().ebe_batch_layout(h.ptr, ctypes.byref(n), no.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      eo.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return n.value, no, eo


def ebe_set_problem_batch(h: Handle, nu, f_nodal, dirichlet, g=None, neumann=None) -> None:
    """ebe_set_problem_batch: nu host [n_problems]; the rest as ebe_set_problem (union numbering)."""
    nuv = _host_f64(nu)
    f = _host_f64(f_nodal)
    if f.shape != (h.n_n,):
        raise ValueError("f_nodal must have n_n entries")
    nd = _host_i32(dirichlet if dirichlet is not None else np.zeros(0))
    gv = None if g is None else _host_f64(g)
    if gv is not None and gv.shape != nd.shape:
        raise ValueError("g must match the Dirichlet set")
    nn = _host_i32(neumann if neumann is not None else np.zeros(0))
    n_prob = ebe_batch_layout(h)[0]
    if nuv.shape != (n_prob,):
        raise ValueError(f"nu must have one value per problem ({n_prob})")
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t)) if a is not None and a.size else None  # noqa: E731
    _check(h, _lib().ebe_set_problem_batch(h.ptr, P(nuv, ctypes.c_double), P(f, ctypes.c_double),
                                           P(nd, ctypes.c_int32), nd.size, P(gv, ctypes.c_double),
                                           P(nn, ctypes.c_int32), nn.size))


def _batch_result(h, infos, summary):
    return ([_info_dict(i) for i in infos],
            {"loops": summary.loops, "launches": summary.launches, "n_converged": summary.n_converged,
             "solve_ms": summary.solve_ms, "ctas_per_sm": summary.config.ctas_per_sm,
             "tile_nodes": summary.config.tile_nodes,
             "phase_ms": dict(zip(("patch", "fixup", "update", "direction"), list(summary.phase_ms)))})


def ebe_solve_batch(h: Handle, x, rtol=None, maxit=None, precision=None, delta=None, stall_updates=None,
                    use_graph=None):
    """ebe_solve_batch on a device x (float64 CUDA tensor, union numbering).

    Returns (per-problem ebe_solve_info dicts, ebe_batch_info dict); raises
    only for errors, not for the solver outcomes of single problems.
    """
    o = _opts(rtol, maxit, precision, None, delta, stall_updates, use_graph)
    n_prob = ebe_batch_layout(h)[0]
    infos = (_abi.ebe_solve_info * n_prob)()
    summary = _abi.ebe_batch_info()
    st = _lib().ebe_solve_batch(h.ptr, _dev(x, EBE_F64, h.n_n, "x"), ctypes.byref(o), infos, ctypes.byref(summary))
    if st not in SOLVER_OUTCOMES:
        _check(h, st)
    return _batch_result(h, infos, summary)


def ebe_solve_batch_host(h: Handle, x, rtol=None, maxit=None, precision=None, delta=None, stall_updates=None,
                         use_graph=None):
    """ebe_solve_batch_host on a host float64 numpy array x (updated in place)."""
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous and x.size == h.n_n):
        raise TypeError("x must be a contiguous float64 numpy array of n_n entries")
    o = _opts(rtol, maxit, precision, None, delta, stall_updates, use_graph)
    n_prob = ebe_batch_layout(h)[0]
    infos = (_abi.ebe_solve_info * n_prob)()
    summary = _abi.ebe_batch_info()
    st = _lib().ebe_solve_batch_host(h.ptr, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(o),
                                     infos, ctypes.byref(summary))
    if st not in SOLVER_OUTCOMES:
        _check(h, st)
    return _batch_result(h, infos, summary)


def ebe_set_batch_config(h: Handle, ctas_per_sm: int = 0, tile_nodes: int = 0, barrier_ns: int = 0) -> None:
    """Launch shape of ebe_solve_batch and the bound of its grid-barrier waits
    (0 = default for every field)."""
    c = _abi.ebe_batch_config(int(ctas_per_sm), int(tile_nodes), int(barrier_ns))
    _check(h, _lib().ebe_set_batch_config(h.ptr, ctypes.byref(c)))


def ebe_batch_tune(h: Handle, precision: int = EBE_PREC_MIXED, loops: int = 0) -> dict:
    """Autotune the batched solver's launch shape (kept by the handle).

    Returns {"best": (ctas_per_sm, tile_nodes), "candidates": [(ctas, tile, ms), ...]}.
    """
    cap = 64
    shapes = (_abi.ebe_batch_config * cap)()
    ms = (ctypes.c_double * cap)()
    best = _abi.ebe_batch_config()
    n = ctypes.c_int32()
    _check(h, _lib().ebe_batch_tune(h.ptr, int(precision), int(loops), ctypes.byref(best), shapes, ms, cap,
                                    ctypes.byref(n)))
    return {"best": (best.ctas_per_sm, best.tile_nodes),
            "candidates": [(shapes[i].ctas_per_sm, shapes[i].tile_nodes, ms[i]) for i in range(n.value)]}


class Mpnn:
    """Owner of an ``ebe_mpnn*`` (learned preconditioner: weights, optimiser state)."""

    def __init__(self, ptr, device):
        self.ptr = ptr
        self.device = device

    def __del__(self):
        try:
            ebe_mpnn_destroy(self)
        except Exception:
            pass


def ebe_mpnn_last_error(net: Mpnn | None) -> str:
    return _lib().ebe_mpnn_last_error(net.ptr if net is not None else None).decode()


def _net_check(net, status):
    if status != _abi.EBE_OK:
        raise EbeError(status, ebe_mpnn_last_error(net))


def ebe_mpnn_n_params() -> int:
    return int(_lib().ebe_mpnn_n_params())


def ebe_mpnn_create(device: int = 0, theta=None) -> Mpnn:
    """ebe_mpnn_create: theta host [n_params] or None (seeded initial weights, zero decoder)."""
    t = None if theta is None else _host_f64(theta)
    if t is not None and t.shape != (ebe_mpnn_n_params(),):
        raise ValueError("theta must have ebe_mpnn_n_params() entries")
    ptr = ctypes.c_void_p()
    st = _lib().ebe_mpnn_create(ctypes.byref(ptr), int(device),
                                t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if t is not None else None)
    if st != _abi.EBE_OK:
        raise EbeError(st, _lib().ebe_mpnn_last_error(None).decode())
    return Mpnn(ptr, device)


def ebe_mpnn_destroy(net: Mpnn) -> None:
    if net is not None and net.ptr is not None and net.ptr.value:
        _lib().ebe_mpnn_destroy(net.ptr)
        net.ptr = ctypes.c_void_p()


def ebe_mpnn_set_params(net: Mpnn, theta=None) -> None:
    t = None if theta is None else _host_f64(theta)
    _net_check(net, _lib().ebe_mpnn_set_params(
        net.ptr, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if t is not None else None))


def ebe_mpnn_get_params(net: Mpnn) -> np.ndarray:
    t = np.empty(ebe_mpnn_n_params())
    _net_check(net, _lib().ebe_mpnn_get_params(net.ptr, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return t


def ebe_mpnn_apply(net: Mpnn, h: Handle, r, z) -> None:
    """z = B(r) (float64 CUDA tensors of n_n entries) on the mesh of h."""
    _check(h, _lib().ebe_mpnn_apply(net.ptr, h.ptr, _dev(r, EBE_F64, h.n_n, "r"), _dev(z, EBE_F64, h.n_n, "z")))


def ebe_mpnn_grad(net: Mpnn, h: Handle, r, gz, z=None) -> np.ndarray:
    """Parameter gradient for dL/dz = gz (device); returns a host array, writes z if given."""
    g = np.empty(ebe_mpnn_n_params())
    _check(h, _lib().ebe_mpnn_grad(net.ptr, h.ptr, _dev(r, EBE_F64, h.n_n, "r"), _dev(gz, EBE_F64, h.n_n, "gz"),
                                   _dev(z, EBE_F64, h.n_n, "z") if z is not None else None,
                                   g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return g


def ebe_mpnn_train_step(net: Mpnn, h: Handle, r, e, lr: float) -> float:
    """One Adam step on the energy-norm loss of sample (r, e); returns the loss before the step."""
    loss = ctypes.c_double()
    _check(h, _lib().ebe_mpnn_train_step(net.ptr, h.ptr, _dev(r, EBE_F64, h.n_n, "r"), _dev(e, EBE_F64, h.n_n, "e"),
                                         float(lr), ctypes.byref(loss)))
    return loss.value


def ebe_solve_learned(h: Handle, net, x, rtol=None, maxit=None, chunk=None, stall_updates=None,
                      race_iters=None) -> dict:
    """Flexible CG with the network (or Jacobi with net=None) on a device x; adds "fell_back"."""
    o = _opts(rtol, maxit, None, chunk, None, stall_updates, None)
    if race_iters is not None:
        o.race_iters = int(race_iters)
    info = _abi.ebe_solve_info()
    fb = ctypes.c_int32()
    st = _lib().ebe_solve_learned(h.ptr, net.ptr if net is not None else None, _dev(x, EBE_F64, h.n_n, "x"),
                                  ctypes.byref(o), ctypes.byref(info), ctypes.byref(fb))
    if st not in SOLVER_OUTCOMES:
        _check(h, st)
    out = _info_dict(info)
    out["fell_back"] = bool(fb.value)
    return out


def ebe_residual_noalloc(h: Handle, x, r) -> None:
    """ebe_residual_noalloc: FP64 residual without any device allocation in the
    call (scratch from a fixed device array in the library), for callers that
    cannot call cudaMalloc (device memory owned by another allocator, or a
    loop that must not take the allocator's locks)."""
    _check(h, _lib().ebe_residual_noalloc(h.ptr, _dev(x, EBE_F64, h.n_n, "x"), _dev(r, EBE_F64, h.n_n, "r")))


def ebe_richardson(h: Handle, x, iters: int, omega: float) -> None:
    """Eq. richardson on a device x (float64 CUDA tensor), exactly `iters` steps."""
    _check(h, _lib().ebe_richardson(h.ptr, _dev(x, EBE_F64, h.n_n, "x"), int(iters), float(omega)))


def ebe_chebyshev2(h: Handle, x, iters: int, alphas) -> None:
    """Eq. Czebyshev2lev with the cyclic root sequence alphas (host array)."""
    a = _host_f64(alphas)
    _check(h, _lib().ebe_chebyshev2(h.ptr, _dev(x, EBE_F64, h.n_n, "x"), int(iters),
                                    a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.size))


def ebe_chebyshev2_bounds(h: Handle, x, iters: int, lam1: float, lam2: float, N: int) -> None:
    """Eq. Czebyshev2lev with the N roots of P_N built by the library from the
    spectrum bounds lam1 < lam2, in the order of the paper's listing."""
    _check(h, _lib().ebe_chebyshev2_bounds(h.ptr, _dev(x, EBE_F64, h.n_n, "x"), int(iters), float(lam1), float(lam2),
                                           int(N)))


def ebe_chebyshev3(h: Handle, x, iters: int, lam1: float, lam2: float) -> None:
    """Eq. Czebyshev3lev for spectrum bounds lam1 < lam2."""
    _check(h, _lib().ebe_chebyshev3(h.ptr, _dev(x, EBE_F64, h.n_n, "x"), int(iters), float(lam1), float(lam2)))


def _mesh_array(meshes):
    keep = []
    arr = (_abi.ebe_mesh * len(meshes))()
    for k, (c, e) in enumerate(meshes):
        c = _host_f64(c)
        e = _host_i32(e)
        if c.ndim != 2 or e.ndim != 2:
            raise ValueError("coords and elems must be 2-D")
        keep += [c, e]
        arr[k] = _abi.ebe_mesh(c.shape[1], e.shape[1], c.shape[0], e.shape[0],
                               c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return arr, keep


_PARTITION_ARRAYS = ("slot_elem", "lconn", "patch_meta", "pnode", "col_ptr", "sh_node", "sh_ptr", "sh_slot")


def _partition_out(sz, nb):
    return {
        "slot_elem": np.empty(sz.n_slots, np.int32), "lconn": np.empty((nb, sz.n_slots), np.uint16),
        "patch_meta": np.empty((sz.n_patches, 8), np.int32), "pnode": np.empty(sz.n_pnode, np.int32),
        "col_ptr": np.empty(sz.n_colptr, np.int32), "sh_node": np.empty(sz.n_shared, np.int32),
        "sh_ptr": np.empty(sz.n_shared + 1, np.int32), "sh_slot": np.empty(sz.n_halo, np.int32),
    }


def ebe_partition_export(coords, elems) -> dict:
    """Host-only element partition (no device needed) as numpy arrays."""
    arr, keep = _mesh_array([(coords, elems)])
    sz = _abi.ebe_partition_sizes()
    lib = _lib()
    st = lib.ebe_partition_export(arr, ctypes.byref(sz), *([None] * 8))
    if st != _abi.EBE_OK:
        raise EbeError(st, ebe_last_error(None))
    out = _partition_out(sz, keep[1].shape[1])
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    st = lib.ebe_partition_export(arr, ctypes.byref(sz), *[ptr(out[k]) for k in _PARTITION_ARRAYS])
    if st != _abi.EBE_OK:
        raise EbeError(st, ebe_last_error(None))
    out.update({k: getattr(sz, k) for k, _ in _abi.ebe_partition_sizes._fields_})
    return out


def ebe_partition_export_batch(meshes) -> dict:
    """Host-only partition of a batch's union (as ebe_create_batch builds it), plus ``patch_off``."""
    arr, keep = _mesh_array(meshes)
    sz = _abi.ebe_partition_sizes()
    lib = _lib()
    st = lib.ebe_partition_export_batch(arr, len(meshes), ctypes.byref(sz), *([None] * 9))
    if st != _abi.EBE_OK:
        raise EbeError(st, ebe_last_error(None))
    out = _partition_out(sz, keep[1].shape[1])
    out["patch_off"] = np.empty(len(meshes) + 1, np.int32)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    st = lib.ebe_partition_export_batch(arr, len(meshes), ctypes.byref(sz), ptr(out["patch_off"]),
                                        *[ptr(out[k]) for k in _PARTITION_ARRAYS])
    if st != _abi.EBE_OK:
        raise EbeError(st, ebe_last_error(None))
    out.update({k: getattr(sz, k) for k, _ in _abi.ebe_partition_sizes._fields_})
    return out


def ebe_get_stats(h: Handle) -> dict:
    s = _abi.ebe_stats()
    _check(h, _lib().ebe_get_stats(h.ptr, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in _abi.ebe_stats._fields_}
