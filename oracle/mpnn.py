"""FP64 CPU oracle of the learned message-passing preconditioner -- test infrastructure.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs
may import this module; it shares no code with the CUDA library.

The paper has no learned component: its solver loops leave the
preconditioner slot open (the listings apply z = r where a preconditioner
would act, Sec. 2).  This module writes out, plainly and in FP64, the network
that the library places in that slot of a flexible CG (its definition is the
library's own, stated here and in include/ebe.h):

  inputs   s  = rms(r), zj = dinv * r, sz = rms(zj), rms over free nodes
           x_i = [r_i / s, zj_i / sz]                               (2 features)
  encoder  h_i = W_in x_i + b_in                                    (32)
  layers   l = 1..4:  a_i = mean_{j in N(i)} h_j - h_i,  u_i = [h_i; a_i],
           v_i = W_l u_i + b_l,  h_i <- h_i + relu(v_i)             (64 -> 32)
  decoder  o_i = w_out . h_i + b_out
  output   z_i = zj_i + sz * o_i on free nodes, 0 on Dirichlet nodes

N(i) are the mesh neighbours of node i (nodes sharing an element with it).
The map is homogeneous of degree one in r, and with a zero decoder it is the
Jacobi preconditioner.  The GPU keeps weights and hidden features in BF16
(round to nearest even) and accumulates in FP32; ``forward(..., exact=False)``
rounds at the same places so that the two agree to FP32 accumulation error,
``exact=True`` rounds nowhere (used for the finite-difference pins).

Parameter vector order (shared with the C ABI): W_in [32][2], b_in [32],
then per layer W_l [32][64], b_l [32], then w_out [32], b_out [1].
"""
from __future__ import annotations

import numpy as np

H = 32
LAYERS = 4
F_IN = 2


def n_params() -> int:
    return H * F_IN + H + LAYERS * (H * 2 * H + H) + H + 1


def unpack(theta):
    """Views of the flat parameter vector."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (n_params(),)
    o = 0

    def take(shape):
        nonlocal o
        size = int(np.prod(shape))
        v = theta[o:o + size].reshape(shape)
        o += size
        return v

    p = {"W_in": take((H, F_IN)), "b_in": take((H,)), "W": [], "b": []}
    for _ in range(LAYERS):
        p["W"].append(take((H, 2 * H)))
        p["b"].append(take((H,)))
    p["w_out"] = take((H,))
    p["b_out"] = take((1,))
    return p


def init_params(seed: int) -> np.ndarray:
    """Seeded initial weights: uniform +-1/sqrt(fan_in), zero decoder (start at Jacobi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.uniform(-1, 1, (H, F_IN)) / np.sqrt(F_IN), np.zeros(H)]
    for _ in range(LAYERS):
        parts += [rng.uniform(-1, 1, (H, 2 * H)) / np.sqrt(2 * H), np.zeros(H)]
    parts += [np.zeros(H), np.zeros(1)]
    return np.concatenate([q.ravel() for q in parts])


def bf16(x):
    """Round to bfloat16 (through FP32, both round to nearest even), as float64."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    bits = x32.view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((bits >> 16) & 1)
    out = ((bits + bias) & 0xFFFF0000).astype(np.uint32)
    return out.view(np.float32).astype(np.float64)


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def mesh_graph(n_n: int, elems):
    """Neighbour lists (CSR, ascending, no self loops) of the mesh graph."""
    elems = np.asarray(elems, dtype=np.int64)
    nb = elems.shape[1]
    a = np.repeat(elems, nb, axis=1).ravel()
    b = np.tile(elems, (1, nb)).ravel()
    keep = a != b
    pairs = np.unique(np.stack([a[keep], b[keep]], 1), axis=0)
    indptr = np.zeros(n_n + 1, np.int64)
    np.add.at(indptr, pairs[:, 0] + 1, 1)
    indptr = np.cumsum(indptr)
    return indptr, pairs[:, 1].copy()


def _mean_nbr(graph, h):
    indptr, idx = graph
    deg = np.diff(indptr)
    sums = np.add.reduceat(h[idx], indptr[:-1], axis=0)
    return sums / deg[:, None]


def _mean_nbr_T(graph, g):
    """Transpose of _mean_nbr: out_j = sum over i with j in N(i) of g_i / deg_i."""
    indptr, idx = graph
    deg = np.diff(indptr)
    rows = np.repeat(np.arange(len(deg)), deg)
    out = np.zeros_like(g)
    np.add.at(out, idx, g[rows] / deg[rows, None])
    return out


def forward(theta, r, dinv, graph, exact: bool = False):
    """z = B(r) and the cache for backward()."""
    rd = (lambda v: v) if exact else bf16
    r = np.asarray(r, dtype=np.float64)
    dinv = np.asarray(dinv, dtype=np.float64)
    p = unpack(theta)
    free = dinv != 0.0
    nf = max(int(free.sum()), 1)
    s = np.sqrt(np.sum(r[free] ** 2) / nf)
    zj = dinv * r
    sz = np.sqrt(np.sum(zj[free] ** 2) / nf)
    if not (s > 0.0 and sz > 0.0):
        return np.zeros_like(r), None
    x = np.stack([r / s, zj / sz], 1)
    if not exact:
        x = f32(x)
    h = rd(x @ rd(p["W_in"]).T + rd(p["b_in"]))
    cache = {"x": x, "hs": [h], "us": [], "vs": [], "s": s, "sz": sz, "free": free, "graph": graph, "exact": exact}
    for l in range(LAYERS):
        a = _mean_nbr(graph, h) - h
        u = np.concatenate([h, rd(a)], 1)
        v = u @ rd(p["W"][l]).T + rd(p["b"][l])
        h = rd(h + np.maximum(v, 0.0))
        cache["us"].append(u)
        cache["vs"].append(v)
        cache["hs"].append(h)
    o = h @ rd(p["w_out"]) + rd(p["b_out"])[0]
    z = np.where(free, zj + sz * o, 0.0)
    return z, cache


def backward(theta, cache, gz):
    """Gradient of a loss L(z) with respect to theta, given gz = dL/dz.

    Rounding to BF16 is treated as the identity (straight-through); the
    weights enter with the values forward() used."""
    rd = (lambda v: v) if cache["exact"] else bf16
    p = unpack(theta)
    graph = cache["graph"]
    go = np.where(cache["free"], np.asarray(gz, dtype=np.float64) * cache["sz"], 0.0)
    h4 = cache["hs"][-1]
    g = {"w_out": h4.T @ go, "b_out": np.array([go.sum()]), "W": [None] * LAYERS, "b": [None] * LAYERS}
    gh = np.outer(go, rd(p["w_out"]))
    for l in reversed(range(LAYERS)):
        gv = gh * (cache["vs"][l] > 0.0)
        g["W"][l] = gv.T @ cache["us"][l]
        g["b"][l] = gv.sum(0)
        gu = gv @ rd(p["W"][l])
        ga = gu[:, H:]
        gh = gh + gu[:, :H] - ga + _mean_nbr_T(graph, ga)
    g["W_in"] = gh.T @ cache["x"]
    g["b_in"] = gh.sum(0)
    parts = [g["W_in"], g["b_in"]]
    for l in range(LAYERS):
        parts += [g["W"][l], g["b"][l]]
    parts += [g["w_out"], g["b_out"]]
    return np.concatenate([q.ravel() for q in parts])


def energy_loss(apply_A, z, e):
    """L = (e - z)' A (e - z) / e' A e and dL/dz (A: the masked FP64 operator)."""
    w = e - z
    Aw = apply_A(w)
    eAe = float(e @ apply_A(e))
    return float(w @ Aw) / eAe, -2.0 * Aw / eAe


def fcg(apply_A, b_masked, x0, precond, rtol=1e-8, maxit=100000):
    """Flexible CG with one stored direction (p_k = z_k - (z_k.q_{k-1} / p_{k-1}.q_{k-1}) p_{k-1},
    alpha_k = p_k.r_k / p_k.q_k), on the masked system; stops when |r| <= rtol |r0|.

    apply_A(v) = mask(A v); b_masked = mask(b - A x0) is the initial residual.
    Returns (x, iterations)."""
    x = np.array(x0, dtype=np.float64)
    r = np.array(b_masked, dtype=np.float64)
    r0 = np.linalg.norm(r)
    if r0 == 0.0:
        return x, 0
    p = q = None
    for k in range(maxit):
        z = precond(r)
        if p is None:
            p = z.copy()
        else:
            p = z - (z @ q) / (p @ q) * p
        q = apply_A(p)
        al = (p @ r) / (p @ q)
        x += al * p
        r -= al * q
        if np.linalg.norm(r) <= rtol * r0:
            return x, k + 1
    return x, maxit
