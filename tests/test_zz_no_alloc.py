"""ebe_residual_noalloc: the residual for callers that cannot call cudaMalloc
(a process whose device memory is handed out by another allocator, or a
real-time loop that must not take the allocator's locks).  Its scratch lives
in a fixed device array in the library, so its result must equal
ebe_residual's on two calls in a row (the second call finds the previous
call's data in the shared array).  Collected last so that a failure here
leaves every other test already run."""
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


@pytest.mark.parametrize("case", ["tri", "tet"])
def test_noalloc_residual_matches_residual_twice(ebe, case):
    prob = (meshgen.config_square_jitter(100, nu=1.0, seed=2) if case == "tri"
            else meshgen.config_cube_noise(14, nu=0.5, seed=3))
    h = ebe.ebe_create(prob["coords"], prob["elems"])
    ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
    ebe.ebe_assemble(h)
    n = prob["coords"].shape[0]
    for seed in (31, 32):                     # two calls in a row, different x
        x = torch.tensor(meshgen.seeded_vector(n, seed), dtype=torch.float64, device="cuda:0")
        r_ref = torch.empty_like(x)
        r = torch.full_like(x, float("nan"))
        ebe.ebe_residual(h, x, r_ref)
        ebe.ebe_residual_noalloc(h, x, r)
        torch.cuda.synchronize()
        a, b = r.cpu().numpy(), r_ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
    # and against the oracle once
    orc = oracle.Problem(prob)
    ref = orc.residual(x.cpu().numpy())
    assert np.linalg.norm(a - ref) <= 1e-12 * np.linalg.norm(ref)
