"""The one-CTA mixed-precision solver of small meshes (k_cg_small), through
the C ABI: meshes of at most 4 patches take it when ebe_solve runs in
EBE_PREC_MIXED with use_graph = 1; use_graph = 0 keeps the grid-wide
iteration.  Both are judged by the oracle's FP64 true residual (1e-8); the
one-CTA solve runs the textbook mixed iteration, so its iteration count
matches EBE_PREC_MIXED_TEXTBOOK's to a few iterations (the sums are added in
another order)."""
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
    return {
        "tri33_f1": meshgen.config_square_f1(33, nu=1.0),                       # 2 patches
        "tri46_jitter": meshgen.config_square_jitter(46, nu=1.0, seed=2),        # 4050 elements, 4 patches, ragged
        "tri_tiny": meshgen.config_square_f1(2, nu=1.0),                         # 2 elements
        "tet5": meshgen.config_cube_noise(5, nu=0.5, seed=3),                    # 384 tetrahedra
        "paper_g1": meshgen.config_square_f1(33, nu=0.0, g_value=1.0),           # Dirichlet 1, nu = 0
    }


def _solve(ebe, prob, **kw):
    h = ebe.ebe_create(prob["coords"], prob["elems"])
    ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    x = torch.zeros(prob["coords"].shape[0], dtype=torch.float64, device=DEV)
    info = ebe.ebe_solve(h, x, rtol=1e-8, **kw)
    torch.cuda.synchronize()
    launches = ebe.ebe_get_stats(h)["kernel_launches"]
    ebe.ebe_destroy(h)
    return x.cpu().numpy(), info, launches


@pytest.mark.parametrize("name", list(_cases()))
def test_small_solve_matches_oracle_and_textbook(ebe, name):
    prob = _cases()[name]
    orc = oracle.Problem(prob)
    xs, info, launches = _solve(ebe, prob, precision=ebe.EBE_PREC_MIXED)
    assert info["status"] == "EBE_OK", info
    assert orc.rel_residual(xs) <= 1e-8
    xt, it, _ = _solve(ebe, prob, precision=ebe.EBE_PREC_MIXED_TEXTBOOK)
    assert abs(info["iterations"] - it["iterations"]) <= max(3, 0.05 * it["iterations"]), (info, it)
    xg, ig, launches_grid = _solve(ebe, prob, precision=ebe.EBE_PREC_MIXED, use_graph=0)
    assert ig["status"] == "EBE_OK" and orc.rel_residual(xg) <= 1e-8
    # the one-CTA solve is one kernel launch after the set-up; the grid-wide one
    # two per iteration
    assert launches < launches_grid


def test_small_solve_is_bitwise_reproducible(ebe):
    prob = _cases()["tri46_jitter"]
    x1, i1, _ = _solve(ebe, prob, precision=ebe.EBE_PREC_MIXED)
    x2, i2, _ = _solve(ebe, prob, precision=ebe.EBE_PREC_MIXED)
    np.testing.assert_array_equal(x1, x2)
    assert i1["iterations"] == i2["iterations"]


def test_small_solve_outcomes(ebe):
    prob = meshgen.config_square_f1(33, nu=1.0)
    _, info, _ = _solve(ebe, prob, precision=ebe.EBE_PREC_MIXED, maxit=5)
    assert info["status"] == "EBE_MAXIT" and info["iterations"] == 5, info
    # a NaN in x0 at a free node: the initial true residual is not finite
    h = ebe.ebe_create(prob["coords"], prob["elems"])
    ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    free = np.setdiff1d(np.arange(prob["coords"].shape[0]), prob["dirichlet"])
    x = torch.zeros(prob["coords"].shape[0], dtype=torch.float64, device=DEV)
    x[int(free[len(free) // 2])] = float("nan")
    info = ebe.ebe_solve(h, x, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    assert info["status"] == "EBE_BREAKDOWN", info
    x.zero_()
    info = ebe.ebe_solve(h, x, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    assert info["status"] == "EBE_OK"
    ebe.ebe_destroy(h)
