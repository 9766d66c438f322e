"""Seeded synthetic inputs: meshes, load data and boundary node sets.

This module is the only code shared by the CUDA path and the FP64 oracle.  It
produces *inputs* (node coordinates, element connectivity, nodal values of f,
Dirichlet/Neumann node sets) and holds none of the method's arithmetic: no
element matrices, no residuals, no solver steps.

Workloads follow the paper's model problem (Sec. 1: -Lap u + nu u = f on the
unit square, P1 triangles with n_b = 3, P1 tetrahedra with n_b = 4) and its
experiment (Sec. 3: uniformly refined triangular meshes with n^2 nodes).

Conventions
-----------
* Nodes are numbered row-major from the origin: node (i, j) of an n x n grid
  has id ``j*n + i`` and coordinates ``(i*h, j*h)``, ``h = 1/(n-1)``; in 3D
  node (i, j, k) has id ``(k*n + j)*n + i``.
* Every square cell is split by its SW-NE diagonal into the triangles
  (SW, SE, NE) and (SW, NE, NW); both are counter-clockwise.  With n = 2 this
  is the 2-element / 4-node mesh of Fig. 1 (left), with n = 3 the 8-element /
  9-node mesh of Fig. 1 (right).  The figure itself is not available, so the
  numbering and the diagonal direction are a chosen reading.
* Every cube is split into the 6 Kuhn tetrahedra
  ``v0, v0+e_s0, v0+e_s0+e_s1, v0+(1,1,1)`` over the permutations s of the
  three axes, reordered so that each has positive volume.
* Random numbers come from numpy's PCG64 generator seeded explicitly.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "square_tri", "cube_tet", "jitter_interior", "square_boundary_nodes",
    "cube_face_nodes", "permute_nodes", "config_square_f1", "config_square_jitter",
    "config_cube_noise", "manufactured_square", "fourier_square",
]


def square_tri(n: int):
    """Structured P1 triangulation of (0,1)^2 with n x n nodes (n >= 2).

    Returns ``coords`` (float64, [n*n, 2]) and ``elems`` (int32, [2(n-1)^2, 3]),
    cells in row-major order, two triangles per cell.
    """
    if n < 2:
        raise ValueError("n must be >= 2")
    h = 1.0 / (n - 1)
    i = np.arange(n)
    X, Y = np.meshgrid(i * h, i * h, indexing="xy")  # X[j, i] = i*h
    coords = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)
    ci, cj = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="xy")
    sw = (cj * n + ci).ravel()
    se = sw + 1
    nw = sw + n
    ne = sw + n + 1
    t1 = np.stack([sw, se, ne], axis=1)
    t2 = np.stack([sw, ne, nw], axis=1)
    elems = np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)
    return coords, elems


def cube_tet(n: int):
    """Kuhn (Freudenthal) tetrahedralisation of (0,1)^3 with n^3 nodes (n >= 2).

    Returns ``coords`` (float64, [n^3, 3]) and ``elems`` (int32, [6(n-1)^3, 4]),
    cubes in row-major (x fastest) order, six tetrahedra per cube.
    """
    if n < 2:
        raise ValueError("n must be >= 2")
    h = 1.0 / (n - 1)
    g = np.arange(n) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")  # X[k, j, i] = i*h
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    m = n - 1
    ck, cj, ci = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    v0 = ((ck * n + cj) * n + ci).ravel().astype(np.int64)
    step = (1, n, n * n)  # node-id increment along x, y, z
    tets = []
    for perm in itertools.permutations(range(3)):
        a = v0
        b = a + step[perm[0]]
        c = b + step[perm[1]]
        d = c + step[perm[2]]
        # orientation: sign of the permutation decides the sign of the volume
        # of (v0, v0+e_s0, v0+e_s0+e_s1, v0+1); swap the last two when odd.
        inversions = sum(1 for x, y in itertools.combinations(perm, 2) if x > y)
        if inversions % 2 == 0:
            tets.append(np.stack([a, b, c, d], axis=1))
        else:
            tets.append(np.stack([a, b, d, c], axis=1))
    elems = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return coords, elems


def _boundary_mask(coords: np.ndarray, tol: float = 1e-12) -> np.ndarray:
    return np.any((coords <= tol) | (coords >= 1.0 - tol), axis=1)


def jitter_interior(coords: np.ndarray, h: float, amount: float, seed: int) -> np.ndarray:
    """Move every interior node, each coordinate independently, by U[-amount*h, amount*h].

    Boundary nodes stay fixed so the domain remains the unit square/cube.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = coords.copy()
    interior = ~_boundary_mask(coords)
    d = rng.uniform(-amount * h, amount * h, size=(int(interior.sum()), coords.shape[1]))
    out[interior] += d
    return out


def square_boundary_nodes(n: int, sides=("x0", "x1", "y0", "y1")) -> np.ndarray:
    """Sorted node ids of the n x n grid lying on the named sides of the square."""
    i = np.arange(n)
    ids = []
    if "x0" in sides:
        ids.append(i * n)
    if "x1" in sides:
        ids.append(i * n + n - 1)
    if "y0" in sides:
        ids.append(i)
    if "y1" in sides:
        ids.append((n - 1) * n + i)
    return np.unique(np.concatenate(ids)).astype(np.int32)


def cube_face_nodes(n: int, faces=("z0",)) -> np.ndarray:
    """Sorted node ids of the n^3 grid lying on the named faces of the cube."""
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ids = ((k * n + j) * n + i).ravel()
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    sel = np.zeros(ids.shape, dtype=bool)
    for f in faces:
        axis = {"x": i, "y": j, "z": k}[f[0]]
        sel |= axis == (0 if f[1] == "0" else n - 1)
    return np.sort(ids[sel]).astype(np.int32)


def permute_nodes(coords, elems, node_sets, seed: int):
    """Renumber nodes by a random permutation (same mesh, scattered ids).

    Returns (coords', elems', [sets'], perm) with ``coords'[perm[k]] = coords[k]``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_n = coords.shape[0]
    perm = rng.permutation(n_n).astype(np.int64)
    c2 = np.empty_like(coords)
    c2[perm] = coords
    e2 = perm[elems].astype(np.int32)
    sets2 = [np.sort(perm[s]).astype(np.int32) for s in node_sets]
    return c2, e2, sets2, perm


def _square_problem_dict(coords, elems, nu, f, dirichlet, g, neumann, name):
    return {
        "name": name, "dim": coords.shape[1], "coords": np.ascontiguousarray(coords),
        "elems": np.ascontiguousarray(elems), "nu": float(nu),
        "f": np.ascontiguousarray(f, dtype=np.float64),
        "dirichlet": np.ascontiguousarray(dirichlet, dtype=np.int32),
        "g": np.ascontiguousarray(g, dtype=np.float64),
        "neumann": np.ascontiguousarray(neumann, dtype=np.int32),
    }


def config_square_f1(n: int = 33, nu: float = 1.0, g_value: float = 0.0):
    """Structured square, f = 1, Dirichlet u = g_value on the whole boundary.

    n = 33, nu = 1, g = 0 is the small Jacobi-PCG workload; nu = 0 with g = 1
    is the paper's experiment (Sec. 3).
    """
    coords, elems = square_tri(n)
    dirichlet = square_boundary_nodes(n)
    f = np.ones(coords.shape[0])
    g = np.full(dirichlet.shape[0], g_value)
    return _square_problem_dict(coords, elems, nu, f, dirichlet, g, np.zeros(0, np.int32),
                                f"square{n}_f1_nu{nu:g}")


def config_square_jitter(n: int = 2049, nu: float = 1.0, seed: int = 2, jitter: float = 0.2):
    """Jittered square, f = (2 pi^2 + nu) sin(pi x) sin(pi y) at the nodes.

    Dirichlet u = x*y (identically 0) on x = 0 and y = 0, homogeneous Neumann on
    x = 1 and y = 1.
    """
    coords, elems = square_tri(n)
    coords = jitter_interior(coords, 1.0 / (n - 1), jitter, seed)
    x, y = coords[:, 0], coords[:, 1]
    f = (2.0 * math.pi ** 2 + nu) * np.sin(math.pi * x) * np.sin(math.pi * y)
    dirichlet = square_boundary_nodes(n, ("x0", "y0"))
    g = coords[dirichlet, 0] * coords[dirichlet, 1]
    neumann = np.setdiff1d(square_boundary_nodes(n, ("x1", "y1")), dirichlet).astype(np.int32)
    return _square_problem_dict(coords, elems, nu, f, dirichlet, g, neumann,
                                f"square{n}_jitter{jitter:g}_nu{nu:g}")


def config_cube_noise(n: int = 129, nu: float = 0.5, seed: int = 3, sigma: float = 0.1):
    """Kuhn cube, f = 1 + sigma*N(0,1) per node, Dirichlet 0 on z = 0, Neumann elsewhere."""
    coords, elems = cube_tet(n)
    rng = np.random.Generator(np.random.PCG64(seed))
    f = 1.0 + sigma * rng.standard_normal(coords.shape[0])
    dirichlet = cube_face_nodes(n, ("z0",))
    bnd = cube_face_nodes(n, ("x0", "x1", "y0", "y1", "z1"))
    neumann = np.setdiff1d(bnd, dirichlet).astype(np.int32)
    g = np.zeros(dirichlet.shape[0])
    return _square_problem_dict(coords, elems, nu, f, dirichlet, g, neumann,
                                f"cube{n}_noise{sigma:g}_nu{nu:g}")


def manufactured_square(n: int, nu: float, kind: str = "dirichlet"):
    """Problems with a known smooth solution u, for the O(h^2) check.

    kind = "dirichlet": u = sin(pi x) sin(pi y), u = 0 on the whole boundary,
    f = (2 pi^2 + nu) u.  kind = "mixed": u = sin(pi x/2) sin(pi y/2), Dirichlet
    0 on x = 0 and y = 0, homogeneous Neumann on x = 1 and y = 1 (du/dn = 0
    there), f = (pi^2/2 + nu) u.  Returns the problem dict and u at the nodes.
    """
    coords, elems = square_tri(n)
    x, y = coords[:, 0], coords[:, 1]
    if kind == "dirichlet":
        u = np.sin(math.pi * x) * np.sin(math.pi * y)
        f = (2.0 * math.pi ** 2 + nu) * u
        dirichlet = square_boundary_nodes(n)
        neumann = np.zeros(0, np.int32)
    elif kind == "mixed":
        u = np.sin(0.5 * math.pi * x) * np.sin(0.5 * math.pi * y)
        f = (0.5 * math.pi ** 2 + nu) * u
        dirichlet = square_boundary_nodes(n, ("x0", "y0"))
        neumann = np.setdiff1d(square_boundary_nodes(n, ("x1", "y1")), dirichlet).astype(np.int32)
    else:
        raise ValueError(kind)
    g = np.zeros(dirichlet.shape[0])
    prob = _square_problem_dict(coords, elems, nu, f, dirichlet, g, neumann,
                                f"manufactured_{kind}{n}_nu{nu:g}")
    return prob, u


def fourier_square(n: int, nu: float, seed: int, modes: int = 8, kmax: int = 8):
    """Structured square with f = sum_m a_m sin(k_m pi x) sin(l_m pi y), full Dirichlet 0.

    a_m ~ N(0,1), k_m, l_m uniform integers in [1, kmax].
    """
    coords, elems = square_tri(n)
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal(modes)
    k = rng.integers(1, kmax + 1, size=modes)
    l = rng.integers(1, kmax + 1, size=modes)
    x, y = coords[:, 0], coords[:, 1]
    f = np.zeros(coords.shape[0])
    for m in range(modes):
        f += a[m] * np.sin(k[m] * math.pi * x) * np.sin(l[m] * math.pi * y)
    dirichlet = square_boundary_nodes(n)
    g = np.zeros(dirichlet.shape[0])
    return _square_problem_dict(coords, elems, nu, f, dirichlet, g, np.zeros(0, np.int32),
                                f"fourier{n}_nu{nu:g}_s{seed}")


def config_batch(n_problems: int = 256, side_lo: int = 17, side_hi: int = 513, nu_lo: float = 1e-2,
                 nu_hi: float = 10.0, seed: int = 4):
    """Batch of independent structured squares (full Dirichlet 0, Fourier f).

    Side lengths s = round(exp(U[ln side_lo, ln side_hi])) nodes, nu =
    exp(U[ln nu_lo, ln nu_hi]), f a sum of 8 Fourier modes (fourier_square)
    with its own seed per problem.  Returns a list of problem dicts.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = np.rint(np.exp(rng.uniform(math.log(side_lo), math.log(side_hi), size=n_problems))).astype(int)
    nus = np.exp(rng.uniform(math.log(nu_lo), math.log(nu_hi), size=n_problems))
    seeds = rng.integers(0, 2 ** 31 - 1, size=n_problems)
    return [fourier_square(int(s), float(nu), int(sd)) for s, nu, sd in zip(sides, nus, seeds)]


def batch_union(problems):
    """Concatenate problem dicts into the union numbering of a batch.

    Returns a dict with node_off / elem_off offsets, the per-problem meshes
    [(coords, elems)], nu [n_problems], and f, dirichlet, g, neumann in the
    union numbering.
    """
    node_off = np.zeros(len(problems) + 1, np.int64)
    elem_off = np.zeros(len(problems) + 1, np.int64)
    for k, pr in enumerate(problems):
        node_off[k + 1] = node_off[k] + pr["coords"].shape[0]
        elem_off[k + 1] = elem_off[k] + pr["elems"].shape[0]
    return {
        "node_off": node_off, "elem_off": elem_off,
        "meshes": [(pr["coords"], pr["elems"]) for pr in problems],
        "nu": np.array([pr["nu"] for pr in problems], np.float64),
        "f": np.concatenate([pr["f"] for pr in problems]),
        "dirichlet": np.concatenate([pr["dirichlet"] + node_off[k] for k, pr in enumerate(problems)]).astype(np.int32),
        "g": np.concatenate([pr["g"] for pr in problems]),
        "neumann": np.concatenate([pr["neumann"] + node_off[k] for k, pr in enumerate(problems)]).astype(np.int32),
    }


def seeded_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """A reproducible U[lo, hi] vector (test iterates x)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=n)
