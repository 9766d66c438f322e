"""Pins of the learned-preconditioner oracle (oracle/mpnn.py), no GPU.

The network is the library's own definition (the paper leaves the
preconditioner slot of its solver loops open, Sec. 2); these tests pin the
oracle to things other than itself: central finite differences of its loss
(a dropped term, wrong sign or transposed operand in backward() fails them),
the homogeneity in r, the scaling with the Jacobi diagonal and the Jacobi
limit that the definition implies, the mesh graph
of the two-element mesh of Fig. 1 by hand, hand-computed BF16 roundings, and
flexible CG with a fixed SPD preconditioner reducing to textbook PCG.
"""
import numpy as np
import pytest

import oracle
from oracle import mpnn
from paper_1911_03973_gb300 import meshgen


def _small(n=9, seed=3, nu=2.0):
    prob = meshgen.config_square_jitter(n, nu=nu, seed=seed)
    orc = oracle.Problem(prob)
    dinv = 1.0 / orc.jacobi_diag()
    dinv[prob["dirichlet"]] = 0.0
    graph = mpnn.mesh_graph(orc.n_n, prob["elems"])
    return prob, orc, dinv, graph


def test_graph_of_the_two_element_mesh():
    # Fig. 1 (reading 11): nodes 0=(0,0), 1=(1,0), 2=(0,1), 3=(1,1); triangles (0,1,3), (0,3,2)
    indptr, idx = mpnn.mesh_graph(4, np.array([[0, 1, 3], [0, 3, 2]]))
    nbrs = [list(idx[indptr[i]:indptr[i + 1]]) for i in range(4)]
    assert nbrs == [[1, 2, 3], [0, 3], [0, 3], [0, 1, 2]]


def test_bf16_rounding_by_hand():
    one = 1.0
    assert mpnn.bf16(one) == 1.0
    assert mpnn.bf16(1.0 + 2.0 ** -8) == 1.0                 # halfway, ties to even (1.0)
    assert mpnn.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # halfway, ties to even mantissa
    assert mpnn.bf16(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7   # above halfway: up
    assert mpnn.bf16(-3.0) == -3.0
    assert mpnn.bf16(1e-30) > 0.0


def test_zero_decoder_is_jacobi_and_dirichlet_rows_are_zero():
    prob, orc, dinv, graph = _small()
    theta = mpnn.init_params(5)                 # zero decoder by construction
    r = orc.residual(orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 1)))
    for exact in (True, False):
        z, _ = mpnn.forward(theta, r, dinv, graph, exact=exact)
        np.testing.assert_allclose(z, dinv * r, rtol=0, atol=1e-15 * np.abs(dinv * r).max())
    theta[-1] = 0.3
    z, _ = mpnn.forward(theta, r, dinv, graph, exact=True)
    assert np.all(z[prob["dirichlet"]] == 0.0)
    assert np.abs(z - dinv * r).max() > 0.0


def test_homogeneous_of_degree_one():
    prob, orc, dinv, graph = _small()
    rng = np.random.Generator(np.random.PCG64(7))
    theta = rng.normal(0, 0.3, mpnn.n_params())
    r = orc.residual(orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 2)))
    z1, _ = mpnn.forward(theta, r, dinv, graph, exact=True)
    for a in (1e-6, 3.0, 1e5):
        za, _ = mpnn.forward(theta, a * r, dinv, graph, exact=True)
        np.testing.assert_allclose(za, a * z1, rtol=1e-12, atol=1e-300)


def test_scales_with_the_jacobi_diagonal():
    """Both input features are scale-free and the output is zj + rms(zj) o, so
    B(r; c dinv) = c B(r; dinv) for every c > 0."""
    prob, orc, dinv, graph = _small()
    rng = np.random.Generator(np.random.PCG64(8))
    theta = rng.normal(0, 0.3, mpnn.n_params())
    r = orc.residual(orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 5)))
    z1, _ = mpnn.forward(theta, r, dinv, graph, exact=True)
    for c in (1e-4, 0.37, 50.0):
        zc, _ = mpnn.forward(theta, r, c * dinv, graph, exact=True)
        np.testing.assert_allclose(zc, c * z1, rtol=1e-12, atol=1e-300)


def test_backward_matches_finite_differences():
    prob, orc, dinv, graph = _small(n=11)
    rng = np.random.Generator(np.random.PCG64(11))
    theta = rng.normal(0, 0.3, mpnn.n_params())
    x = orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 3))
    r = orc.residual(x)
    e = rng.normal(0, 1, orc.n_n)
    e[prob["dirichlet"]] = 0.0

    def loss(th):
        z, _ = mpnn.forward(th, r, dinv, graph, exact=True)
        return mpnn.energy_loss(orc.apply, z, e)[0]

    z, cache = mpnn.forward(theta, r, dinv, graph, exact=True)
    L, gz = mpnn.energy_loss(orc.apply, z, e)
    g = mpnn.backward(theta, cache, gz)
    # every parameter block, several entries each (including relu-gated ones)
    sizes = [2 * 32, 32] + [32 * 64, 32] * 4 + [32, 1]
    starts = np.concatenate([[0], np.cumsum(sizes)])
    picks = []
    for b0, b1 in zip(starts[:-1], starts[1:]):
        picks += list(rng.choice(np.arange(b0, b1), size=min(4, b1 - b0), replace=False))
    for i in picks:
        hstep = 1e-6 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += hstep
        tm[i] -= hstep
        fd = (loss(tp) - loss(tm)) / (2 * hstep)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_rounded_forward_stays_close_to_exact():
    prob, orc, dinv, graph = _small(n=17)
    rng = np.random.Generator(np.random.PCG64(12))
    theta = rng.normal(0, 0.2, mpnn.n_params())
    r = orc.residual(orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 4)))
    ze, _ = mpnn.forward(theta, r, dinv, graph, exact=True)
    zr, _ = mpnn.forward(theta, r, dinv, graph, exact=False)
    assert np.linalg.norm(zr - ze) <= 5e-2 * np.linalg.norm(ze)


def test_fcg_with_jacobi_is_textbook_pcg():
    prob = meshgen.config_square_f1(33, nu=1.0)
    orc = oracle.Problem(prob)
    dinv = 1.0 / orc.jacobi_diag()
    dinv[prob["dirichlet"]] = 0.0
    x0 = orc.with_dirichlet(np.zeros(orc.n_n))
    x, it = mpnn.fcg(orc.apply, orc.residual(x0), x0, lambda r: dinv * r, rtol=1e-8)
    _, info = orc.pcg(rtol=1e-8)
    assert abs(it - info["iterations"]) <= 1, (it, info)
    assert orc.rel_residual(x) <= 1.5e-8
