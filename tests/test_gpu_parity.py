"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (written here, derived in the design notes):
  * FP64 residual / apply: |r_gpu - r_orc| / |r_orc| <= 1e-12 (the path and the
    oracle differ only in summation order);
  * FP64 element matrices, b, Jacobi diagonal: entrywise <= 1e-13 relative to
    the largest entry of the element (closed form vs quadrature/inversion);
  * FP32 residual: against the oracle evaluated in FP64 on the FP32-rounded
    oracle A_e and FP32 x: relative norm error <= 1e-5;
  * solves: the oracle recomputes |mask(b - A x)| / |mask(b - A x0)| of the
    returned x in FP64 and it must be <= rtol = 1e-8.
"""
import numpy as np
import pytest

import oracle
from paper_1911_03973_gb300 import meshgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ebe():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1911_03973_gb300 as mod
    return mod


DEV = "cuda:0"


def _cases():
    return {
        "tri_ragged": lambda: meshgen.config_square_jitter(100, nu=1.0, seed=2),        # 19602 el: 19 patches + tail
        "tri_f1_small": lambda: meshgen.config_square_f1(33, nu=1.0),                    # 2048 el: exactly 2 patches
        "tri_tiny": lambda: meshgen.config_square_f1(2, nu=1.0),                         # 2 elements, no shared nodes
        "tri_nu0_perm": lambda: _permuted(meshgen.config_square_jitter(40, nu=0.0, seed=5), 9),
        "tet_ragged": lambda: meshgen.config_cube_noise(18, nu=0.5, seed=3),            # 29478 tets
        "tet_small": lambda: meshgen.config_cube_noise(5, nu=0.5, seed=3),              # 384 tets
    }


def _permuted(prob, seed):
    c, e, (nd, nn), perm = meshgen.permute_nodes(prob["coords"], prob["elems"],
                                                  [prob["dirichlet"], prob["neumann"]], seed)
    f = np.empty_like(prob["f"])
    f[perm] = prob["f"]
    order = np.argsort(perm[prob["dirichlet"]])
    out = dict(prob, coords=c, elems=e, dirichlet=nd, neumann=nn, f=f, g=prob["g"][order])
    return out


def _setup(ebe, prob, store=None):
    h = ebe.ebe_create(prob["coords"], prob["elems"], device=0)
    ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED if store is None else store)
    return h


def _t(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


@pytest.mark.parametrize("case", list(_cases()))
def test_element_matrices_match_oracle(ebe, case):
    prob = _cases()[case]()
    orc = oracle.Problem(prob)
    h = _setup(ebe, prob)
    nb, n_e = orc.nb, orc.n_e
    K = torch.empty(n_e * nb * nb, dtype=torch.float64, device=DEV)
    M = torch.empty_like(K)
    A = torch.empty_like(K)
    ebe.ebe_element_matrices(h, K, M)
    ebe.ebe_get_local_matrices(h, A)
    torch.cuda.synchronize()
    # device layout: element e, entry (i, j) at e*nb*nb + j*nb + i (paper's Fig. 2)
    view = lambda t: t.cpu().numpy().reshape(n_e, nb, nb).transpose(0, 2, 1)  # noqa: E731
    for got, ref in ((view(K), orc.K), (view(M), orc.M), (view(A), orc.A)):
        scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
        assert np.abs(got - ref).max() <= 0 or (np.abs(got - ref) / scale).max() <= 1e-13
    b = torch.empty(orc.n_n, dtype=torch.float64, device=DEV)
    d = torch.empty_like(b)
    ebe.ebe_get_rhs(h, b)
    ebe.ebe_jacobi_diag(h, d)
    torch.cuda.synchronize()
    np.testing.assert_allclose(b.cpu().numpy(), orc.rhs(), rtol=1e-13, atol=1e-13 * np.abs(orc.rhs()).max())
    np.testing.assert_allclose(d.cpu().numpy(), orc.jacobi_diag(), rtol=1e-13)


@pytest.mark.parametrize("case", list(_cases()))
def test_residual_fp64_matches_oracle(ebe, case):
    prob = _cases()[case]()
    orc = oracle.Problem(prob)
    h = _setup(ebe, prob)
    x = orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 17))
    xd = _t(x)
    rd = torch.empty_like(xd)
    yd = torch.empty_like(xd)
    ebe.ebe_residual(h, xd, rd)
    ebe.ebe_apply(h, xd, yd)
    torch.cuda.synchronize()
    r_ref = orc.residual(x)
    y_ref = orc.apply(x)
    r = rd.cpu().numpy()
    y = yd.cpu().numpy()
    assert np.linalg.norm(r - r_ref) <= 1e-12 * np.linalg.norm(r_ref)
    assert np.linalg.norm(y - y_ref) <= 1e-12 * np.linalg.norm(y_ref)
    assert np.all(r[prob["dirichlet"]] == 0.0) and np.all(y[prob["dirichlet"]] == 0.0)


@pytest.mark.parametrize("case", list(_cases()))
def test_residual_double_word_matches_oracle(ebe, case):
    """EBE_F64_DW: A_e and x as FP32 pairs, products and sums in double-word
    arithmetic.  Its error is about 2^-48 |A| |x| per node, so the FP64 bound
    1e-12 holds; a dropped low word (2^-24) would exceed it by 10^4."""
    prob = _cases()[case]()
    orc = oracle.Problem(prob)
    h = _setup(ebe, prob)
    x = orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 17))
    xd = _t(x)
    rd, yd, r64 = torch.empty_like(xd), torch.empty_like(xd), torch.empty_like(xd)
    ebe.ebe_residual(h, xd, rd, double_word=True)
    ebe.ebe_apply(h, xd, yd, double_word=True)
    ebe.ebe_residual(h, xd, r64)
    torch.cuda.synchronize()
    r_ref, y_ref = orc.residual(x), orc.apply(x)
    r, y = rd.cpu().numpy(), yd.cpu().numpy()
    assert np.linalg.norm(r - r_ref) <= 1e-12 * np.linalg.norm(r_ref)
    assert np.linalg.norm(y - y_ref) <= 1e-12 * np.linalg.norm(y_ref)
    # per node against the FP64 pass: within 2^-42 of the node's sum_e |A_e| |x_e| + |b|
    # (the oracle's operator on |A_e| and |x|); a dropped low word errs by 2^-24 of it
    scale = oracle.Problem(prob, A_override=np.abs(orc.A)).apply(np.abs(x)) + np.abs(orc.rhs())
    assert np.all(np.abs(r - r64.cpu().numpy()) <= 2.0 ** -42 * scale)
    assert np.all(r[prob["dirichlet"]] == 0.0) and np.all(y[prob["dirichlet"]] == 0.0)
    with pytest.raises(TypeError):
        ebe.ebe_residual(h, xd.float(), rd.float(), double_word=True)
    ebe.ebe_destroy(h)


@pytest.mark.parametrize("case", ["tri_ragged", "tet_ragged"])
def test_residual_double_word_near_the_solution(ebe, case):
    """At a solution to rtol 1e-11, b - A x cancels deeply (|A| |x| is about
    10^4 |b| per node on the 100^2 square), so the error bound scales with
    |A| |x|, not with r: within 2^-42 of the norm of sum_e |A_e| |x_e| + |b|
    (48-bit arithmetic: about 2^-48 of it), and below 1e-10 |r(x0)|, a hundredth
    of the tightest rtol the mixed solver's replacement checks decide."""
    prob = _cases()[case]()
    orc = oracle.Problem(prob)
    h = _setup(ebe, prob)
    xd = torch.zeros(orc.n_n, dtype=torch.float64, device=DEV)
    info = ebe.ebe_solve(h, xd, rtol=1e-11, precision=ebe.EBE_PREC_FP64)
    assert info["status"] == "EBE_OK", info
    rd = torch.empty_like(xd)
    ebe.ebe_residual(h, xd, rd, double_word=True)
    torch.cuda.synchronize()
    x = xd.cpu().numpy()
    r_ref = orc.residual(x)
    r0 = np.linalg.norm(orc.residual(orc.with_dirichlet(np.zeros(orc.n_n))))
    assert np.linalg.norm(r_ref) <= 2e-11 * r0
    scale = oracle.Problem(prob, A_override=np.abs(orc.A)).apply(np.abs(x)) + np.abs(orc.rhs())
    err = np.linalg.norm(rd.cpu().numpy() - r_ref)
    assert err <= 2.0 ** -42 * np.linalg.norm(scale)
    assert err <= 1e-10 * r0
    ebe.ebe_destroy(h)


def fp32_difference_form(A64):
    """The FP32 operator's matrices, built from the oracle's FP64 A_e: off-diagonal
    entries rounded to FP32, row sums rounded to FP32, diagonal = row sum minus
    the rounded off-diagonals (evaluated in FP64)."""
    nb = A64.shape[1]
    off = A64.astype(np.float32).astype(np.float64)
    off[:, np.arange(nb), np.arange(nb)] = 0.0
    s = A64.sum(axis=2).astype(np.float32).astype(np.float64)
    A = off.copy()
    A[:, np.arange(nb), np.arange(nb)] = s - off.sum(axis=2)
    return A


@pytest.mark.parametrize("case", ["tri_ragged", "tet_ragged", "tri_tiny"])
def test_residual_fp32_matches_oracle_on_rounded_matrices(ebe, case):
    prob = _cases()[case]()
    orc64 = oracle.Problem(prob)
    orc = oracle.Problem(prob, A_override=fp32_difference_form(orc64.A))
    h = _setup(ebe, prob)
    x = orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 18)).astype(np.float32)
    xd = _t(x, torch.float32)
    rd = torch.empty_like(xd)
    ebe.ebe_residual(h, xd, rd)
    torch.cuda.synchronize()
    # b is rounded to FP32 on the device; the oracle keeps FP64 b (difference far below 1e-5)
    r_ref = orc.residual(x.astype(np.float64))
    r = rd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(r - r_ref) <= 1e-5 * np.linalg.norm(r_ref)


@pytest.mark.parametrize("case, dtype", [("tri_ragged", torch.float64), ("tri_ragged", torch.float32),
                                         ("tet_ragged", torch.float32)])
def test_residual_is_bitwise_reproducible(ebe, case, dtype):
    # tet_ragged has about 30 colours per patch: the FP32 pass then adds through
    # per-warp copies of the node sums, merged in a fixed order
    prob = _cases()[case]()
    h = _setup(ebe, prob)
    x = _t(meshgen.seeded_vector(prob["coords"].shape[0], 3), dtype)
    outs = []
    for _ in range(3):
        r = torch.empty_like(x)
        ebe.ebe_residual(h, x, r)
        outs.append(r.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


@pytest.mark.parametrize("scatter", ["COLOUR", "NODE", "ATOMIC"])
@pytest.mark.parametrize("case", ["tri_ragged", "tet_ragged"])
def test_comparison_scatters_match_oracle(ebe, case, scatter):
    prob = _cases()[case]()
    orc = oracle.Problem(prob)
    h = _setup(ebe, prob)
    x = orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 19))
    xd = _t(x)
    rd = torch.empty_like(xd)
    ebe.ebe_residual_variant(h, xd, rd, getattr(ebe, f"EBE_SCATTER_{scatter}"))
    torch.cuda.synchronize()
    r_ref = orc.residual(x)
    assert np.linalg.norm(rd.cpu().numpy() - r_ref) <= 1e-12 * np.linalg.norm(r_ref)


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("case", ["tri_f1_small", "tri_ragged", "tet_ragged", "tri_nu0_perm", "tri_tiny"])
def test_solve_reaches_1e8_judged_by_oracle(ebe, case, precision):
    prob = _cases()[case]()
    orc = oracle.Problem(prob)
    h = _setup(ebe, prob)
    x = torch.zeros(orc.n_n, dtype=torch.float64, device=DEV)
    info = ebe.ebe_solve(h, x, rtol=1e-8, precision=getattr(ebe, f"EBE_PREC_{precision}"))
    assert info["status"] == "EBE_OK", info
    rel = orc.rel_residual(x.cpu().numpy())
    assert rel <= 1e-8, (rel, info)
    if precision == "FP64" and orc.n_n > 10:
        _, oinfo = orc.pcg(rtol=1e-8)
        it, oit = info["iterations"], oinfo["iterations"]
        assert abs(it - oit) <= max(2, 0.02 * oit), (it, oit)


def test_solve_paper_experiment_lifted_dirichlet(ebe):
    """Sec. 3 setting: nu = 0, u = 1 on the boundary, f = 1 (nonzero g)."""
    prob = meshgen.config_square_f1(33, nu=0.0, g_value=1.0)
    orc = oracle.Problem(prob)
    h = _setup(ebe, prob)
    x = torch.zeros(orc.n_n, dtype=torch.float64, device=DEV)
    info = ebe.ebe_solve(h, x, rtol=1e-10)
    assert info["status"] == "EBE_OK"
    xh = x.cpu().numpy()
    assert orc.rel_residual(xh) <= 1e-10
    assert np.all(xh[prob["dirichlet"]] == 1.0)
    ref, _ = orc.pcg(rtol=1e-12)
    assert np.abs(xh - ref).max() <= 1e-8


def test_solve_host_buffers(ebe):
    prob = _cases()["tri_ragged"]()
    orc = oracle.Problem(prob)
    h = _setup(ebe, prob)
    x = np.zeros(orc.n_n)
    info = ebe.ebe_solve_host(h, x, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    assert info["status"] == "EBE_OK"
    assert orc.rel_residual(x) <= 1e-8


def test_solver_outcomes(ebe):
    prob = _cases()["tri_ragged"]()
    h = _setup(ebe, prob)
    x = torch.zeros(prob["coords"].shape[0], dtype=torch.float64, device=DEV)
    info = ebe.ebe_solve(h, x, rtol=1e-8, maxit=5, chunk=4)
    assert info["status"] == "EBE_MAXIT" and info["iterations"] == 5


def test_errors_reported_not_raised_on_device(ebe):
    c, e = meshgen.square_tri(5)
    with pytest.raises(ebe.EbeError) as ei:
        ebe.ebe_create(c, np.array([[0, 1, 25]], np.int32))
    assert ei.value.status == 2
    # a degenerate (zero-area) element is found by the element-matrix kernel
    c2 = c.copy()
    c2[6] = [0.125, 0.0]                    # node 6 onto the edge 0-1: triangle (0, 1, 6) has zero area
    h = ebe.ebe_create(c2, e)
    n = c.shape[0]
    ebe.ebe_set_problem(h, 1.0, np.ones(n), meshgen.square_boundary_nodes(5))
    with pytest.raises(ebe.EbeError) as ei:
        ebe.ebe_assemble(h)
    assert ei.value.status == 3
    h2 = ebe.ebe_create(c, e)
    with pytest.raises(ebe.EbeError) as ei:
        ebe.ebe_set_problem(h2, 0.0, np.ones(n), np.zeros(0, np.int32))
    assert ei.value.status == 4
    with pytest.raises(ebe.EbeError) as ei:
        ebe.ebe_residual(h2, torch.zeros(n, dtype=torch.float64, device=DEV),
                         torch.zeros(n, dtype=torch.float64, device=DEV))
    assert ei.value.status == 10


def test_set_problem_rejects_bad_data_on_the_host(ebe):
    # nu < 0 or not finite, f or g not finite, a Dirichlet node listed twice
    # or out of range, a node in both boundary sets: each is refused before any
    # device work, and the handle then takes a valid problem and solves it
    c, e = meshgen.square_tri(5)
    n = c.shape[0]
    nd = meshgen.square_boundary_nodes(5)
    f = np.ones(n)
    h = ebe.ebe_create(c, e)
    cases = [
        (dict(nu=-1.0), 1),
        (dict(nu=float("nan")), 1),
        (dict(f=np.where(np.arange(n) == 7, np.nan, 1.0)), 1),
        (dict(g=np.where(np.arange(nd.size) == 0, np.inf, 0.0)), 1),
        (dict(dirichlet=np.concatenate([nd, nd[:1]])), 1),
        (dict(dirichlet=np.array([0, n], np.int32)), 2),
        (dict(neumann=nd[:2]), 1),
    ]
    for change, status in cases:
        a = dict(nu=1.0, f=f, dirichlet=nd, g=None, neumann=None)
        a.update(change)
        with pytest.raises(ebe.EbeError) as ei:
            ebe.ebe_set_problem(h, a["nu"], a["f"], a["dirichlet"], a["g"], a["neumann"])
        assert ei.value.status == status, (change, str(ei.value))
    ebe.ebe_set_problem(h, 1.0, f, nd)
    ebe.ebe_assemble(h)
    x = torch.zeros(n, dtype=torch.float64, device=DEV)
    info = ebe.ebe_solve(h, x, rtol=1e-8)
    assert info["status"] == "EBE_OK", info
    ebe.ebe_destroy(h)


def test_random_meshes_residuals_match_oracle(ebe):
    # random sizes, jitter, node and element orders; triangles use colour rounds,
    # tetrahedra (many colours per patch) the per-warp node sums in FP32
    rng = np.random.Generator(np.random.PCG64(77))
    for trial in range(6):
        tri = trial % 2 == 0
        n = int(rng.integers(3, 80)) if tri else int(rng.integers(3, 14))
        if tri:
            c, e = meshgen.square_tri(n)
            c = meshgen.jitter_interior(c, 1.0 / (n - 1), 0.2, seed=int(rng.integers(1 << 30)))
        else:
            c, e = meshgen.cube_tet(n)
        c, e, _, _ = meshgen.permute_nodes(c, e, [], seed=int(rng.integers(1 << 30)))
        e = np.ascontiguousarray(e[rng.permutation(e.shape[0])])
        nd = np.unique(rng.integers(0, c.shape[0], size=max(1, c.shape[0] // 20))).astype(np.int32)
        prob = {"coords": c, "elems": e, "nu": float(rng.uniform(0.0, 2.0)), "f": rng.normal(size=c.shape[0]),
                "dirichlet": nd, "g": rng.normal(size=nd.size), "neumann": np.zeros(0, np.int32)}
        orc = oracle.Problem(prob)
        h = _setup(ebe, prob)
        x = orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 100 + trial))
        xd = _t(x)
        rd = torch.empty_like(xd)
        ebe.ebe_residual(h, xd, rd)
        orc32 = oracle.Problem(prob, A_override=fp32_difference_form(orc.A))
        x32 = x.astype(np.float32)
        rd32 = torch.empty(orc.n_n, dtype=torch.float32, device=DEV)
        ebe.ebe_residual(h, _t(x32, torch.float32), rd32)
        torch.cuda.synchronize()
        ref = orc.residual(x)
        assert np.linalg.norm(rd.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref), (trial, n, tri)
        ref32 = orc32.residual(x32.astype(np.float64))
        r32 = rd32.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(r32 - ref32) <= 1e-5 * np.linalg.norm(ref32), (trial, n, tri)
        ebe.ebe_destroy(h)
