"""The paper's stationary iterations (Sec. 2) on the GPU vs the oracle.

The GPU's three-level Chebyshev iteration uses the direction form
(p = r + beta p, x += alpha p); the oracle uses the three-term recurrence with
the scaling factors C_k of Eq. recrCk: the same iterates in exact arithmetic.
Tolerance: relative max-norm difference <= 1e-10 (contractive iterations; the
two forms round differently)."""
import math

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


def _bounds(n):
    return 8 * math.sin(math.pi / (2 * (n - 1))) ** 2, 8 * math.sin((n - 2) * math.pi / (2 * (n - 1))) ** 2


def _setup(ebe, prob):
    h = ebe.ebe_create(prob["coords"], prob["elems"])
    ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
    ebe.ebe_assemble(h)
    return h


def _close(a, b, tol):
    return np.abs(a - b).max() <= tol * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("method", ["richardson", "cheb2_N8", "cheb3"])
def test_paper_experiment_iterations_match_oracle(ebe, method):
    n = 33
    prob = meshgen.config_square_f1(n, nu=0.0, g_value=1.0)     # Sec. 3 setting
    orc = oracle.Problem(prob)
    l1, l2 = _bounds(n)
    h = _setup(ebe, prob)
    x0 = np.zeros(orc.n_n)
    xd = torch.tensor(x0, dtype=torch.float64, device=DEV)
    if method == "richardson":
        ebe.ebe_richardson(h, xd, 124, 2.0 / (l1 + l2))
        ref = orc.richardson(orc.with_dirichlet(x0), 124, 2.0 / (l1 + l2))
    elif method == "cheb2_N8":
        roots = oracle.chebyshev_roots(l1, l2, 8)
        ebe.ebe_chebyshev2(h, xd, 40, roots)
        ref = orc.chebyshev2(orc.with_dirichlet(x0), 40, roots)
    else:
        ebe.ebe_chebyshev3(h, xd, 124, l1, l2)
        ref = orc.chebyshev3(orc.with_dirichlet(x0), 124, l1, l2)
    assert _close(xd.cpu().numpy(), ref, 1e-10)


def test_iterations_on_jittered_tets(ebe):
    prob = meshgen.config_cube_noise(10, nu=0.5, seed=3)
    orc = oracle.Problem(prob)
    h = _setup(ebe, prob)
    x0 = np.zeros(orc.n_n)
    xd = torch.tensor(x0, dtype=torch.float64, device=DEV)
    omega = 0.5 / orc.jacobi_diag().max()
    ebe.ebe_richardson(h, xd, 30, omega)
    assert _close(xd.cpu().numpy(), orc.richardson(orc.with_dirichlet(x0), 30, omega), 1e-12)


def test_iteration_argument_errors(ebe):
    prob = meshgen.config_square_f1(9, nu=1.0)
    h = _setup(ebe, prob)
    xd = torch.zeros(prob["coords"].shape[0], dtype=torch.float64, device=DEV)
    with pytest.raises(ebe.EbeError):
        ebe.ebe_chebyshev3(h, xd, 5, 2.0, 1.0)
    with pytest.raises(ebe.EbeError):
        ebe.ebe_chebyshev2(h, xd, 5, np.array([1.0, 0.0]))
