"""Parity at the full workload sizes, in the configuration bench.py times.

2049^2 jittered triangles (8,388,608 elements) and the 129^3 Kuhn cube
(12,582,912 tetrahedra): the oracle evaluates the whole residual (Algorithm 1,
single thread, a few seconds) and recomputes the FP64 true relative residual
of every GPU solve.  Tolerances as in test_gpu_parity.py.
"""
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


@pytest.fixture(scope="module", params=["square2049", "cube129"])
def full(request, ebe):
    if request.param == "square2049":
        prob = meshgen.config_square_jitter(2049, nu=1.0, seed=2)
    else:
        prob = meshgen.config_cube_noise(129, nu=0.5, seed=3)
    stream = torch.cuda.Stream()
    h = ebe.ebe_create(prob["coords"], prob["elems"], stream=stream.cuda_stream)
    ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    torch.cuda.synchronize()
    orc = oracle.Problem(prob)
    yield request.param, prob, h, orc, stream
    ebe.ebe_destroy(h)


def test_full_size_residual_fp64(ebe, full):
    name, prob, h, orc, stream = full
    x = orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 41))
    with torch.cuda.stream(stream):
        xd = torch.tensor(x, dtype=torch.float64, device=DEV)
        rd = torch.empty_like(xd)
        ebe.ebe_residual(h, xd, rd)
    torch.cuda.synchronize()
    ref = orc.residual(x)
    r = rd.cpu().numpy()
    assert np.linalg.norm(r - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.all(r[prob["dirichlet"]] == 0.0)


def test_full_size_residual_double_word(ebe, full):
    name, prob, h, orc, stream = full
    x = orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 41))
    with torch.cuda.stream(stream):
        xd = torch.tensor(x, dtype=torch.float64, device=DEV)
        rd = torch.empty_like(xd)
        ebe.ebe_residual(h, xd, rd, double_word=True)
    torch.cuda.synchronize()
    ref = orc.residual(x)
    r = rd.cpu().numpy()
    assert np.linalg.norm(r - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.all(r[prob["dirichlet"]] == 0.0)


def test_full_size_jacobi_and_rhs(ebe, full):
    name, prob, h, orc, stream = full
    with torch.cuda.stream(stream):
        b = torch.empty(orc.n_n, dtype=torch.float64, device=DEV)
        d = torch.empty_like(b)
        ebe.ebe_get_rhs(h, b)
        ebe.ebe_jacobi_diag(h, d)
    torch.cuda.synchronize()
    np.testing.assert_allclose(d.cpu().numpy(), orc.jacobi_diag(), rtol=1e-13)
    rb = orc.rhs()
    assert np.abs(b.cpu().numpy() - rb).max() <= 1e-13 * np.abs(rb).max()


def test_full_size_mixed_solve_judged_by_oracle(ebe, full):
    name, prob, h, orc, stream = full
    with torch.cuda.stream(stream):
        x = torch.zeros(orc.n_n, dtype=torch.float64, device=DEV)
        info = ebe.ebe_solve(h, x, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    torch.cuda.synchronize()
    assert info["status"] == "EBE_OK", info
    assert orc.rel_residual(x.cpu().numpy()) <= 1e-8


def test_full_size_nu0_mixed_solve_judged_by_oracle(ebe):
    """The 2049^2 workload with nu = 0 (the stiffness matrix alone): the mixed
    solve to 1e-8, judged by the oracle's FP64 true residual."""
    prob = meshgen.config_square_jitter(2049, nu=0.0, seed=2)
    stream = torch.cuda.Stream()
    h = ebe.ebe_create(prob["coords"], prob["elems"], stream=stream.cuda_stream)
    ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    with torch.cuda.stream(stream):
        x = torch.zeros(prob["coords"].shape[0], dtype=torch.float64, device=DEV)
        info = ebe.ebe_solve(h, x, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    torch.cuda.synchronize()
    ebe.ebe_destroy(h)
    assert info["status"] == "EBE_OK", info
    assert oracle.Problem(prob).rel_residual(x.cpu().numpy()) <= 1e-8
