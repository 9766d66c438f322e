"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a closed form, a
hand-derived fixture (tests/golden/), an invariant or a textbook/library
routine.  CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1911_03973_gb300 import meshgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def _prob(coords, elems, nu=0.0, f=None, dirichlet=None, g=None):
    n_n = coords.shape[0]
    nd = np.zeros(0, np.int32) if dirichlet is None else np.asarray(dirichlet, np.int32)
    return oracle.Problem(dict(coords=coords, elems=elems, nu=nu,
                               f=np.ones(n_n) if f is None else f, dirichlet=nd,
                               g=np.zeros(nd.shape[0]) if g is None else g))


# ---------------------------------------------------------------- element level
@pytest.mark.parametrize("h", [1.0, 0.25, 1.0 / 2048])
def test_right_triangle_closed_form(h):
    """Eq. matrices_K_M on one right triangle equals the hand-derived closed form."""
    gold = _golden("right_triangle.txt")
    coords = np.array([[0.0, 0.0], [h, 0.0], [0.0, h]])
    K, M, meas = oracle.element_matrices(coords, np.array([[0, 1, 2]], np.int32))
    np.testing.assert_allclose(K[0], gold[:3], rtol=0, atol=1e-14)
    np.testing.assert_allclose(M[0] * 24.0 / h ** 2, gold[3:], rtol=1e-13)
    assert meas[0] == pytest.approx(h * h / 2, rel=1e-14)


def test_right_triangle_vertex_order_invariance():
    """Relabelling the vertices permutes rows and columns of K_e, M_e consistently."""
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    K0, M0, _ = oracle.element_matrices(coords, np.array([[0, 1, 2]], np.int32))
    perm = [2, 0, 1]
    K1, M1, _ = oracle.element_matrices(coords, np.array([perm], np.int32))
    np.testing.assert_allclose(K1[0], K0[0][np.ix_(perm, perm)], atol=1e-15)
    np.testing.assert_allclose(M1[0], M0[0][np.ix_(perm, perm)], atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_element_invariants_jittered(dim):
    """K_e: symmetric PSD with zero row sums (constants have no gradient) and
    exactly one zero eigenvalue; M_e: SPD; |T| matches the shoelace/triple
    product; sum of all M entries = |Omega| = 1 (int of 1*1)."""
    if dim == 2:
        c, e = meshgen.square_tri(9)
        c = meshgen.jitter_interior(c, 1 / 8, 0.2, seed=11)
    else:
        c, e = meshgen.cube_tet(5)
        c = meshgen.jitter_interior(c, 1 / 4, 0.2, seed=12)
    K, M, meas = oracle.element_matrices(c, e)
    scale = np.abs(K).max(axis=(1, 2))
    assert np.abs(K.sum(axis=2)).max() <= 1e-13 * scale.max()
    np.testing.assert_allclose(K, K.transpose(0, 2, 1), atol=1e-14 * scale.max())
    np.testing.assert_allclose(M, M.transpose(0, 2, 1), atol=1e-18)
    wK = np.linalg.eigvalsh(K)
    assert (wK[:, 0] >= -1e-12 * scale).all()
    assert (wK[:, 1] > 1e-6 * scale).all()          # only the constant mode is in the kernel
    assert (np.linalg.eigvalsh(M)[:, 0] > 0).all()
    # independent measure: shoelace (2D) / triple product (3D)
    v = c[e]
    if dim == 2:
        a = v[:, 1] - v[:, 0]
        b = v[:, 2] - v[:, 0]
        ref = 0.5 * np.abs(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    else:
        ref = np.abs(np.linalg.det(v[:, 1:] - v[:, :1])) / 6.0
    np.testing.assert_allclose(meas, ref, rtol=1e-12)
    assert M.sum() == pytest.approx(1.0, rel=1e-13)
    assert meas.sum() == pytest.approx(1.0, rel=1e-13)


def test_mass_integrates_products_exactly():
    """M_ij = int lambda_i lambda_j on a random simplex equals the textbook
    moment formula |T| (1 + delta_ij) / 12 (2D) and / 20 (3D), while the
    oracle integrates it with a quadrature rule."""
    rng = np.random.Generator(np.random.PCG64(5))
    for dim, den in ((2, 12.0), (3, 20.0)):
        v = rng.uniform(0, 1, size=(dim + 1, dim))
        K, M, meas = oracle.element_matrices(v, np.arange(dim + 1, dtype=np.int32)[None])
        ref = meas[0] * (np.ones((dim + 1, dim + 1)) + np.eye(dim + 1)) / den
        np.testing.assert_allclose(M[0], ref, rtol=1e-13)


def test_stiffness_against_finite_difference_gradients():
    """K_ij = |T| grad(l_i).grad(l_j): gradients checked by finite differences
    of the barycentric coordinates computed with numpy.linalg.solve."""
    rng = np.random.Generator(np.random.PCG64(6))
    v = rng.uniform(0, 1, size=(3, 2))
    K, M, meas = oracle.element_matrices(v, np.array([[0, 1, 2]], np.int32))

    def bary(p):
        T = np.vstack([np.ones(3), v.T])
        return np.linalg.solve(T, np.array([1.0, p[0], p[1]]))

    p0 = v.mean(axis=0)
    eps = 1e-6
    G = np.stack([(bary(p0 + eps * np.eye(2)[d]) - bary(p0 - eps * np.eye(2)[d])) / (2 * eps)
                  for d in range(2)], axis=1)  # [i, d]
    ref = meas[0] * G @ G.T
    np.testing.assert_allclose(K[0], ref, rtol=1e-7, atol=1e-9)


def test_degenerate_and_out_of_range_rejected():
    c = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]])
    with pytest.raises(oracle.OracleError):
        oracle.element_matrices(c, np.array([[0, 1, 2]], np.int32))
    with pytest.raises(oracle.OracleError):
        oracle.element_matrices(c, np.array([[0, 1, 3]], np.int32))


# ---------------------------------------------------------------- Fig. 1 meshes
def test_two_element_mesh_dense():
    """Fig. 1 (left): dense K and M equal the hand-derived matrices."""
    gold = _golden("two_element_mesh.txt")
    c, e = meshgen.square_tri(2)
    p = _prob(c, e)
    np.testing.assert_allclose(p.dense("K"), gold[:4], atol=1e-15)
    np.testing.assert_allclose(24.0 * p.dense("M"), gold[4:], atol=1e-14)


def test_nine_node_mesh_centre_row():
    """Fig. 1 (right): centre row of K and M equals the hand derivation."""
    gold = _golden("nine_node_mesh.txt")
    c, e = meshgen.square_tri(3)
    assert e.shape == (8, 3)
    p = _prob(c, e)
    np.testing.assert_allclose(p.dense("K")[4], gold[0], atol=1e-14)
    np.testing.assert_allclose(96.0 * p.dense("M")[4], gold[1], atol=1e-13)


def test_structured_interior_rows_are_5_point_stencil():
    """Interior rows of K on the SW-NE mesh equal the 5-point stencil; row sums
    of M equal h^2 (so b = h^2 for f = 1)."""
    n = 9
    h = 1.0 / (n - 1)
    c, e = meshgen.square_tri(n)
    p = _prob(c, e)
    K, M = p.dense("K"), p.dense("M")
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            k = j * n + i
            row = np.zeros(n * n)
            row[k] = 4.0
            row[[k - 1, k + 1, k - n, k + n]] = -1.0
            np.testing.assert_allclose(K[k], row, atol=1e-14)
            assert M[k].sum() == pytest.approx(h * h, rel=1e-13)
            assert M[k, k] == pytest.approx(h * h / 2, rel=1e-13)


def test_kuhn_cube_is_7_point_stencil_times_h():
    n = 5
    h = 1.0 / (n - 1)
    c, e = meshgen.cube_tet(n)
    p = _prob(c, e)
    K = p.dense("K")
    for k3 in range(1, n - 1):
        for j in range(1, n - 1):
            for i in range(1, n - 1):
                k = (k3 * n + j) * n + i
                row = np.zeros(n ** 3)
                row[k] = 6.0 * h
                row[[k - 1, k + 1, k - n, k + n, k - n * n, k + n * n]] = -h
                np.testing.assert_allclose(K[k], row, atol=1e-14)


def test_dense_matches_elementwise_sum_with_nu():
    c, e = meshgen.square_tri(5)
    c = meshgen.jitter_interior(c, 0.25, 0.2, seed=3)
    p0 = _prob(c, e, nu=0.0)
    p1 = _prob(c, e, nu=2.5)
    np.testing.assert_allclose(p1.dense("A"), p0.dense("K") + 2.5 * p0.dense("M"), atol=1e-14)


# ---------------------------------------------------------------- Algorithm 1
@pytest.mark.parametrize("case", ["tri", "tri_perm", "tet"])
def test_alg1_residual_equals_dense(case):
    """Algorithm 1's r = sum_e C_e^T (b_e - A_e R_e x), r(nd) = 0, equals
    mask(b - A x) with A and b assembled densely (Sec. 1)."""
    if case.startswith("tri"):
        c, e = meshgen.square_tri(7)
        c = meshgen.jitter_interior(c, 1 / 6, 0.2, seed=4)
        nd = meshgen.square_boundary_nodes(7, ("x0", "y0"))
    else:
        c, e = meshgen.cube_tet(4)
        nd = meshgen.cube_face_nodes(4, ("z0",))
    if case == "tri_perm":
        c, e, (nd,), _ = meshgen.permute_nodes(c, e, [nd], seed=9)
    n_n = c.shape[0]
    f = meshgen.seeded_vector(n_n, 21)
    p = _prob(c, e, nu=0.7, f=f, dirichlet=nd)
    x = meshgen.seeded_vector(n_n, 22)
    A = p.dense("A")
    b = p.dense("M") @ f                     # b = M f_I (nodal interpolant of f)
    ref = b - A @ x
    ref[nd] = 0.0
    np.testing.assert_allclose(p.residual(x), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    np.testing.assert_allclose(p.rhs(), b, atol=1e-15)
    y = A @ x
    y[nd] = 0.0
    np.testing.assert_allclose(p.apply(x), y, atol=1e-13 * np.abs(y).max())
    np.testing.assert_allclose(p.jacobi_diag(), np.diag(A), atol=1e-15)


def test_first_residual_of_small_square_is_h2():
    """33^2 nodes, f = 1, x0 = 0, Dirichlet 0 on the boundary: r0 = M 1 = h^2 on
    all 961 interior nodes, so |r0| = 31/1024."""
    prob = meshgen.config_square_f1(33, nu=1.0)
    p = oracle.Problem(prob)
    r0 = p.residual(np.zeros(p.n_n))
    interior = np.setdiff1d(np.arange(p.n_n), prob["dirichlet"])
    assert interior.shape[0] == 961
    np.testing.assert_allclose(r0[interior], 1.0 / 1024, rtol=1e-12)
    assert np.abs(r0[prob["dirichlet"]]).max() == 0.0
    assert np.linalg.norm(r0) == pytest.approx(31.0 / 1024.0, rel=1e-12)


# ---------------------------------------------------------------- spectrum (Sec. 3)
def _closed_form_spectrum(n):
    s = np.sin(np.arange(1, n - 1) * math.pi / (2 * (n - 1))) ** 2
    return np.sort((4.0 * (s[:, None] + s[None, :])).ravel())


@pytest.mark.parametrize("n", [5, 9, 17])
def test_spectrum_of_masked_stiffness(n):
    """Sec. 3: the (n-2)^2 eigenvalues of A = K (nu = 0) on the free nodes are
    4(sin^2(i pi/(2(n-1))) + sin^2(j pi/(2(n-1))))."""
    c, e = meshgen.square_tri(n)
    p = _prob(c, e)
    K = p.dense("K")
    free = np.setdiff1d(np.arange(n * n), meshgen.square_boundary_nodes(n))
    w = np.linalg.eigvalsh(K[np.ix_(free, free)])
    np.testing.assert_allclose(w, _closed_form_spectrum(n), rtol=1e-12, atol=1e-12)


def test_paper_33_extreme_eigenvalues():
    lam = _closed_form_spectrum(33)
    assert lam[0] == pytest.approx(8 * math.sin(math.pi / 64) ** 2, rel=1e-14)
    assert lam[0] == pytest.approx(0.019261, abs=5e-7)
    assert lam[-1] == pytest.approx(7.98074, abs=5e-6)


# ---------------------------------------------------------------- PCG
@pytest.mark.parametrize("case", ["f1_nu1", "jitter_nu0", "tet_nu05", "lift_g1"])
def test_pcg_matches_dense_solve(case):
    """Jacobi-PCG reaches the dense solution (numpy.linalg.solve on the free
    block, Dirichlet values lifted) within the residual bound."""
    if case == "f1_nu1":
        prob = meshgen.config_square_f1(17, nu=1.0)
    elif case == "jitter_nu0":
        prob = meshgen.config_square_jitter(17, nu=0.0, seed=2)
    elif case == "tet_nu05":
        prob = meshgen.config_cube_noise(6, nu=0.5, seed=3)
    else:
        prob = meshgen.config_square_f1(17, nu=0.0, g_value=1.0)   # Sec. 3: u = 1 on the boundary
    p = oracle.Problem(prob)
    x, info = p.pcg(rtol=1e-13)
    assert info["status"] == "converged"
    assert info["rel_residual"] <= 1e-13
    A = p.dense("A")
    b = p.dense("M") @ prob["f"]
    nd = prob["dirichlet"]
    free = np.setdiff1d(np.arange(p.n_n), nd)
    u = np.zeros(p.n_n)
    u[nd] = prob["g"]
    u[free] = np.linalg.solve(A[np.ix_(free, free)], b[free] - A[np.ix_(free, nd)] @ prob["g"])
    assert np.linalg.norm(x - u) <= 1e-10 * np.linalg.norm(u)


def test_paper_experiment_solution_is_one():
    """Sec. 3 with f = 0 would give u = 1 exactly; with u = 1 on the boundary
    and f = 1 the solution is >= 1 inside (maximum principle, discrete form
    holds for the non-obtuse SW-NE mesh)."""
    prob = meshgen.config_square_f1(17, nu=0.0, g_value=1.0)
    prob0 = dict(prob)
    prob0["f"] = np.zeros_like(prob["f"])
    x, info = oracle.Problem(prob0).pcg(rtol=1e-13)
    np.testing.assert_allclose(x, 1.0, atol=1e-12)
    x1, _ = oracle.Problem(prob).pcg(rtol=1e-13)
    assert x1.min() >= 1.0 - 1e-12


@pytest.mark.parametrize("kind", ["dirichlet", "mixed"])
def test_h2_convergence(kind):
    """O(h^2) in the discrete L2 norm sqrt(e^T M e) for manufactured solutions
    (the P1 rate; ratio >= 3.6 per halving of h)."""
    errs = []
    for n in (17, 33, 65, 129):
        prob, u = meshgen.manufactured_square(n, nu=1.0, kind=kind)
        p = oracle.Problem(prob)
        x, info = p.pcg(rtol=1e-10)
        assert info["status"] == "converged"
        errs.append(p.mass_norm(u - x))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert min(ratios) >= 3.6, ratios


def test_pcg_reports_maxit():
    prob = meshgen.config_square_f1(17, nu=1.0)
    x, info = oracle.Problem(prob).pcg(rtol=1e-13, maxit=3)
    assert info["status"] == "maxit" and info["iterations"] == 3


def test_jacobi_pcg_is_invariant_under_diagonal_scaling():
    """Jacobi-PCG on S A S y = S b (S a positive diagonal) produces the iterates
    y_k = S^-1 x_k of Jacobi-PCG on A x = b: the preconditioner diag(SAS)^-1
    absorbs S.  Plain CG or any other fixed preconditioner does not."""
    prob = meshgen.config_square_jitter(9, nu=0.5, seed=5)
    n_n = prob["coords"].shape[0]
    nd = prob["dirichlet"]
    prob["f"] = np.zeros(n_n)                                     # b = 0: the lifted g drives the solve
    prob["g"] = 1.0 + 0.5 * np.sin(7.0 * np.arange(nd.shape[0]))
    s = np.exp(np.random.default_rng(11).uniform(-1.0, 1.0, n_n))
    p = oracle.Problem(prob)
    e = prob["elems"]
    As = p.A * s[e][:, :, None] * s[e][:, None, :]               # S_e A_e S_e
    probs = dict(prob, g=prob["g"] / s[nd])
    ps = oracle.Problem(probs, A_override=As)
    for k in (1, 2, 5, 12):
        x, info = p.pcg(rtol=1e-300, maxit=k)
        y, infos = ps.pcg(rtol=1e-300, maxit=k)
        assert info["status"] == infos["status"] == "maxit"
        np.testing.assert_allclose(s * y, x, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("case", ["jitter_g0", "lifted_g1"])
def test_relative_residual_along_the_segment_to_the_solution(case):
    """x_t = x0 + t (x* - x0) has b - A x_t = (1 - t)(b - A x0) when A x* = b,
    so its relative residual is |1 - t| (x0: the zero iterate carrying g, the
    default; Sec. 3's u = 1 on the boundary makes g nonzero)."""
    if case == "jitter_g0":
        prob = meshgen.config_square_jitter(9, nu=1.0, seed=6)
    else:
        prob = meshgen.config_square_f1(9, nu=0.0, g_value=1.0)
    p = oracle.Problem(prob)
    A, b = p.dense("A"), p.dense("M") @ prob["f"]
    nd = prob["dirichlet"]
    free = np.setdiff1d(np.arange(p.n_n), nd)
    xs = p.with_dirichlet(np.zeros(p.n_n))                        # x* by a dense solve on the free block
    xs[free] = np.linalg.solve(A[np.ix_(free, free)], b[free] - A[np.ix_(free, nd)] @ xs[nd])
    x0 = p.with_dirichlet(np.zeros(p.n_n))
    for t in (0.0, 0.25, 0.5, 1.5):
        assert p.rel_residual(x0 + t * (xs - x0)) == pytest.approx(abs(1.0 - t), abs=1e-12)


def test_pcg_from_one_eigenvector_away_takes_one_step():
    """On the SW-NE square with nu = 0 and Dirichlet 0 on the whole boundary the
    masked K is the 5-point Laplacian times 1 (diagonal 4), so Jacobi-PCG is CG
    and sin(pi x) sin(2 pi y) at the nodes is an eigenvector: started at
    x* + 0.3 v, one step lands on x*."""
    n = 17
    prob = meshgen.config_square_f1(n, nu=0.0)
    p = oracle.Problem(prob)
    A, b = p.dense("A"), p.dense("M") @ prob["f"]
    nd = prob["dirichlet"]
    free = np.setdiff1d(np.arange(p.n_n), nd)
    xs = np.zeros(p.n_n)
    xs[free] = np.linalg.solve(A[np.ix_(free, free)], b[free])
    xy = prob["coords"]
    v = np.sin(np.pi * xy[:, 0]) * np.sin(2 * np.pi * xy[:, 1])
    v[nd] = 0.0
    x, info = p.pcg(x0=xs + 0.3 * v, rtol=1e-10)
    assert info["status"] == "converged" and info["iterations"] == 1, info
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-12 * np.abs(xs).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_norm_of_a_linear_function_is_its_l2_norm(dim):
    """A linear u is its own P1 interpolant and M integrates products of P1
    functions exactly, so sqrt(u^T M u) = ||u||_L2 over the unit square/cube:
    int (a.x + c)^2 = |a|^2/3 + (sum_{i<j} a_i a_j)/2 + c sum(a) + c^2."""
    if dim == 2:
        c, e = meshgen.square_tri(9)
        c = meshgen.jitter_interior(c, 1.0 / 8, 0.2, seed=7)
        a = np.array([1.0, -0.3])
    else:
        c, e = meshgen.cube_tet(5)
        a = np.array([1.0, -0.3, 0.6])
    c0 = 0.2
    u = c @ a + c0
    pairs = sum(a[i] * a[j] for i in range(dim) for j in range(i + 1, dim))
    exact = a @ a / 3.0 + pairs / 2.0 + c0 * a.sum() + c0 ** 2
    p = _prob(c, e)
    assert p.mass_norm(u) == pytest.approx(math.sqrt(exact), rel=1e-13)


# ---------------------------------------------------------------- Sec. 2 iterations
def _small_paper_problem(n=9):
    prob = meshgen.config_square_f1(n, nu=0.0, g_value=1.0)
    lam = _closed_form_spectrum(n)
    return prob, lam[0], lam[-1]


def test_richardson_is_chebyshev2_with_N1():
    """Sec. 2.2: Richardson is the two-level method with N = 1; its root is
    (l1+l2)/2, i.e. omega = 2/(l1+l2) (the optimum the listing uses)."""
    prob, l1, l2 = _small_paper_problem()
    p = oracle.Problem(prob)
    x0 = p.with_dirichlet(np.zeros(p.n_n))
    xr = p.richardson(x0, 20, 2.0 / (l1 + l2))
    xc = p.chebyshev2(x0, 20, oracle.chebyshev_roots(l1, l2, 1))
    np.testing.assert_allclose(xr, xc, rtol=1e-14, atol=1e-14)


def test_richardson_contraction_bound():
    """Sec. 2.1: with omega_opt the error contracts by (l2-l1)/(l2+l1) per step."""
    prob, l1, l2 = _small_paper_problem()
    p = oracle.Problem(prob)
    u, _ = p.pcg(rtol=1e-13)
    x = p.with_dirichlet(np.zeros(p.n_n))
    q = (l2 - l1) / (l2 + l1)
    for _ in range(10):
        xn = p.richardson(x, 1, 2.0 / (l1 + l2))
        assert np.linalg.norm(xn - u) <= q * np.linalg.norm(x - u) * (1 + 1e-10)
        x = xn


def test_chebyshev2_error_is_P_N():
    """Eq. Cheberror1: after N two-level steps x^N - u = P_N(A)(x^0 - u), with
    P_N(t) = T_N((l1+l2-2t)/(l2-l1)) / T_N((l1+l2)/(l2-l1)) (dense eigen-
    decomposition of the free block)."""
    n, N = 9, 6
    prob, l1, l2 = _small_paper_problem(n)
    p = oracle.Problem(prob)
    u, _ = p.pcg(rtol=1e-13)
    x0 = p.with_dirichlet(np.zeros(p.n_n))
    xN = p.chebyshev2_bounds(x0, N, l1, l2, N)
    free = np.setdiff1d(np.arange(p.n_n), prob["dirichlet"])
    Aff = p.dense("A")[np.ix_(free, free)]
    w, V = np.linalg.eigh(Aff)
    tN = lambda s: np.cosh(N * np.arccosh(s)) if s >= 1 else np.cos(N * np.arccos(s))
    P = np.array([tN((l1 + l2 - 2 * t) / (l2 - l1)) for t in w]) / tN((l1 + l2) / (l2 - l1))
    e0 = (x0 - u)[free]
    ref = V @ (P * (V.T @ e0))
    np.testing.assert_allclose((xN - u)[free], ref, atol=1e-12 * np.linalg.norm(e0))


@pytest.mark.parametrize("N", [1, 2, 5, 8])
def test_chebyshev2_equals_chebyshev3_at_N(N):
    """Sec. 2.2: x^N of the two-level and the three-level iterations agree."""
    prob, l1, l2 = _small_paper_problem(9)
    p = oracle.Problem(prob)
    x0 = p.with_dirichlet(np.zeros(p.n_n))
    x2 = p.chebyshev2_bounds(x0, N, l1, l2, N)
    x3 = p.chebyshev3(x0, N, l1, l2)
    np.testing.assert_allclose(x2, x3, atol=1e-11 * max(1.0, np.abs(x2).max()))


def test_chebyshev3_bound():
    """Sec. 2.2: |x^N - u| <= 2 ((sqrt l2 - sqrt l1)/(sqrt l2 + sqrt l1))^N |x^0 - u|."""
    prob, l1, l2 = _small_paper_problem(17)
    p = oracle.Problem(prob)
    u, _ = p.pcg(rtol=1e-13)
    x0 = p.with_dirichlet(np.zeros(p.n_n))
    q = (math.sqrt(l2) - math.sqrt(l1)) / (math.sqrt(l2) + math.sqrt(l1))
    for N in (5, 20, 40):
        xN = p.chebyshev3(x0, N, l1, l2)
        assert np.linalg.norm(xN - u) <= 2 * q ** N * np.linalg.norm(x0 - u) * (1 + 1e-8)


def test_paper_experiment_qualitative_outcome():
    """Sec. 3: 33^2 nodes, nu = 0, u = 1 on the boundary, f = 1, 124 iterations
    with the spectrum bounds of Sec. 3: only the three-level Chebyshev method
    converges; Richardson needs more steps; the two-level method with N = 32
    (roots in the listing's order) is visibly worse than the three-level one,
    and its iterate at k = N no longer matches the three-level iterate (the
    instability the paper mentions), while for small N they agree."""
    n = 33
    prob = meshgen.config_square_f1(n, nu=0.0, g_value=1.0)
    lam = _closed_form_spectrum(n)
    l1, l2 = lam[0], lam[-1]
    p = oracle.Problem(prob)
    u, _ = p.pcg(rtol=1e-13)
    x0 = p.with_dirichlet(np.zeros(p.n_n))
    e0 = np.abs(x0 - u).max()
    err = lambda x: np.abs(x - u).max() / e0  # noqa: E731
    e_rich = err(p.richardson(x0, 124, 2.0 / (l1 + l2)))
    e_cheb2 = err(p.chebyshev2(x0, 124, oracle.chebyshev_roots(l1, l2, 32)))
    e_cheb3 = err(p.chebyshev3(x0, 124, l1, l2))
    assert e_rich > 0.5
    assert e_cheb3 < 1e-4
    assert e_cheb2 > 10 * e_cheb3
    x2 = p.chebyshev2(x0, 32, oracle.chebyshev_roots(l1, l2, 32))
    x3 = p.chebyshev3(x0, 32, l1, l2)
    assert np.abs(x2 - x3).max() > 1e-6 * np.abs(x3).max()
