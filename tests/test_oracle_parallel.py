"""The all-core timing build of the oracle (OpenMP, colour-parallel element
loop) against the single-thread oracle (no GPU): the same element arrays
bit for bit, the same residual to rounding (only the order of the additions
into a node differs), and Jacobi-PCG with the same iteration count (+-1) and
an oracle-judged solution.  It is used only to time the CPU baseline."""
import numpy as np
import pytest

import oracle
import oracle.parallel as oracle_parallel
from paper_1911_03973_gb300 import meshgen


@pytest.fixture(scope="module")
def par_lib():
    if oracle_parallel.build_parallel() is None:
        pytest.skip("gcc without OpenMP")


@pytest.mark.parametrize("case", ["tri", "tet"])
def test_parallel_oracle_matches_single_thread(par_lib, case, monkeypatch):
    prob = (meshgen.config_square_jitter(60, nu=1.0, seed=2) if case == "tri"
            else meshgen.config_cube_noise(9, nu=0.5, seed=3))
    ref = oracle.Problem(prob)
    par = oracle_parallel.ParallelTiming(prob)
    assert par.threads >= 1 and par.n_col >= (7 if case == "tri" else 20)
    A, be = par.element_arrays()
    np.testing.assert_array_equal(A, ref._Ab.ravel())
    np.testing.assert_array_equal(be, ref._be.ravel())
    x = ref.with_dirichlet(meshgen.seeded_vector(ref.n_n, 3))
    r_ref = ref.residual(x)
    r = par.residual(A, be, x)
    assert np.linalg.norm(r - r_ref) <= 1e-13 * np.linalg.norm(r_ref)
    xs, info = par.pcg(A, be, rtol=1e-8)
    _, info_ref = ref.pcg(rtol=1e-8)
    assert info["status"] == "converged"
    assert abs(info["iterations"] - info_ref["iterations"]) <= 1
    assert ref.rel_residual(xs) <= 1e-8


def test_colouring_is_valid(par_lib):
    prob = meshgen.config_square_jitter(30, nu=1.0, seed=2)
    par = oracle_parallel.ParallelTiming(prob)
    el = prob["elems"]
    seen = np.zeros(par.n_e, bool)
    for c in range(par.n_col):
        members = par.order[par.col_ptr[c]:par.col_ptr[c + 1]]
        seen[members] = True
        nodes = el[members].ravel()
        assert np.unique(nodes).size == nodes.size       # no node twice within a colour
    assert seen.all() and par.col_ptr[par.n_col] == par.n_e
