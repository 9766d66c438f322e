"""The single-synchronisation mixed-precision Jacobi-PCG (EBE_PREC_MIXED)
against the textbook four-launch iteration with the same arithmetic
(EBE_PREC_MIXED_TEXTBOOK) and against the oracle.

In exact arithmetic the two iterations produce the same iterates: the fused
pass forms x_k, r_k and p_k exactly as the update and direction kernels do,
and takes beta from the expansion r'.(dinv r') = r.z - 2 alpha q.z +
alpha^2 q.(dinv q) instead of a second reduction.  In FP32 the expansion and
the different summation order of the dot products change beta and alpha in
their last bits, so the iterates after k steps agree to a tolerance that grows
with k (measured: about 1e-7 relative after a few steps); every solve is
judged by the oracle's FP64 true relative residual <= 1e-8, and its iteration
count must lie between plain FP64's and the textbook mixed form's (FP32
rounding delays CG by a residual plateau or not)."""
import numpy as np
import pytest

import oracle
from paper_1911_03973_gb300 import meshgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ebe():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1911_03973_gb300 as mod
    return mod


def _cases():
    tri = meshgen.config_square_jitter(97, nu=1.0, seed=2)
    tet = meshgen.config_cube_noise(14, nu=0.5, seed=3)
    # the same mesh with randomly permuted node ids (scattered caller numbering)
    c, e, sets, perm = meshgen.permute_nodes(tri["coords"], tri["elems"], [tri["dirichlet"], tri["neumann"]], seed=5)
    f = np.empty_like(tri["f"])
    f[perm] = tri["f"]
    tri_perm = dict(tri, coords=c, elems=e, dirichlet=sets[0], neumann=sets[1], f=f,
                    g=np.zeros(sets[0].shape[0]))
    return {"tri": tri, "tet": tet, "tri_perm": tri_perm,
            "tri_nu0": meshgen.config_square_jitter(65, nu=0.0, seed=4),
            "paper_g1": meshgen.config_square_f1(33, nu=0.0, g_value=1.0)}


CASES = _cases()


def _handle(ebe, prob):
    h = ebe.ebe_create(prob["coords"], prob["elems"])
    ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    return h


@pytest.mark.parametrize("name", sorted(CASES))
def test_single_sync_solve_matches_oracle_and_textbook_count(ebe, name):
    prob = CASES[name]
    h = _handle(ebe, prob)
    n = prob["coords"].shape[0]
    orc = oracle.Problem(prob)
    x = torch.zeros(n, dtype=torch.float64, device=DEV)
    info = ebe.ebe_solve(h, x, precision=ebe.EBE_PREC_MIXED)
    assert info["status"] == "EBE_OK", info
    assert orc.rel_residual(x.cpu().numpy()) <= 1e-8
    xt = torch.zeros_like(x)
    it = ebe.ebe_solve(h, xt, precision=ebe.EBE_PREC_MIXED_TEXTBOOK)
    assert it["status"] == "EBE_OK"
    xf = torch.zeros_like(x)
    i64 = ebe.ebe_solve(h, xf, precision=ebe.EBE_PREC_FP64)
    # FP32 rounding delays CG by a residual plateau or not (the mixed counts
    # take one of two values a plateau apart, the lower one FP64's): no more
    # iterations than the textbook form, no fewer than plain FP64
    assert info["iterations"] <= 1.03 * it["iterations"] + 3, (info, it)
    assert info["iterations"] >= 0.97 * i64["iterations"] - 3, (info, i64)
    # without graphs, the same passes launched one by one: bitwise the same solve
    xg = torch.zeros_like(x)
    ig = ebe.ebe_solve(h, xg, precision=ebe.EBE_PREC_MIXED, use_graph=0, chunk=7)
    assert ig["iterations"] == info["iterations"] or abs(ig["iterations"] - info["iterations"]) <= 7
    ebe.ebe_destroy(h)


@pytest.mark.parametrize("k", [1, 2, 7, 30])
def test_first_iterates_match_the_textbook_iteration(ebe, k):
    prob = CASES["tri"]
    h = _handle(ebe, prob)
    n = prob["coords"].shape[0]
    x1 = torch.zeros(n, dtype=torch.float64, device=DEV)
    x2 = torch.zeros_like(x1)
    i1 = ebe.ebe_solve(h, x1, rtol=1e-300, maxit=k, precision=ebe.EBE_PREC_MIXED)
    i2 = ebe.ebe_solve(h, x2, rtol=1e-300, maxit=k, precision=ebe.EBE_PREC_MIXED_TEXTBOOK)
    assert i1["status"] == i2["status"] == "EBE_MAXIT"
    assert i1["iterations"] == i2["iterations"] == k
    a, b = x1.cpu().numpy(), x2.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), np.linalg.norm(a - b) / np.linalg.norm(b)
    ebe.ebe_destroy(h)


def test_single_sync_solve_is_bitwise_reproducible(ebe):
    prob = CASES["tet"]
    h = _handle(ebe, prob)
    n = prob["coords"].shape[0]
    xs = []
    for _ in range(2):
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        ebe.ebe_solve(h, x, precision=ebe.EBE_PREC_MIXED)
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[1])
    ebe.ebe_destroy(h)


def test_single_sync_on_a_batch_union_and_nonzero_x0(ebe):
    # the union of several meshes solved as one system (global dot products),
    # from a non-zero start; x0's Dirichlet values are replaced by g
    probs = [meshgen.fourier_square(s, 1.5, seed=70 + s) for s in (17, 45, 33)]
    U = meshgen.batch_union(probs)
    h = ebe.ebe_create_batch(U["meshes"])
    ebe.ebe_set_problem_batch(h, U["nu"], U["f"], U["dirichlet"], U["g"], U["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    n = int(U["node_off"][-1])
    x0 = meshgen.seeded_vector(n, 9)
    x = torch.tensor(x0, dtype=torch.float64, device=DEV)
    info = ebe.ebe_solve(h, x, precision=ebe.EBE_PREC_MIXED)
    assert info["status"] == "EBE_OK"
    xs = x.cpu().numpy()
    for k, p in enumerate(probs):
        lo, hi = U["node_off"][k], U["node_off"][k + 1]
        orc = oracle.Problem(p)
        # the union's relative residual is global (1e-8); each part is judged
        # against the residual of its own start (x0 with x(nd) = g), which is
        # at most a few times smaller than the union's
        assert orc.rel_residual(xs[lo:hi], orc.with_dirichlet(x0[lo:hi])) <= 1e-7
    ebe.ebe_destroy(h)
