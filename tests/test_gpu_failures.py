"""The solvers' failure paths on the GPU, each caused on the host side.

* A grid-wide barrier of the persistent batched solver that runs out of time
  (its bound set to 1 ns through ebe_batch_config.barrier_ns, so the waiting
  CTAs give up instead of waiting): ebe_solve_batch reports EBE_CUDA_ERROR,
  every CTA leaves, and the same handle then solves normally.
* A relative residual below the FP64 floor (rtol = 1e-18): in mixed precision
  the true residual, checked at every replacement, stops improving and the
  solve ends with EBE_STALL after stall_updates checks.  Where the recurrence
  residual itself stagnates above the next threshold there is no further
  check and the solve ends at maxit with EBE_MAXIT and the attainable
  accuracy: plain FP64 (which checks only at rtol |r0|) on this problem.
* A NaN in the caller's x0 (data the host does not inspect): the initial true
  residual is not finite and the solve ends with EBE_BREAKDOWN, for the
  single-problem solver in both precisions and for one problem of a batch,
  whose other problems still converge.
No test makes a kernel wait without a bound; every wait here gives up on its
own limit."""
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


def _single(ebe, prob):
    h = ebe.ebe_create(prob["coords"], prob["elems"])
    ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    return h


def _batch(ebe, probs):
    U = meshgen.batch_union(probs)
    h = ebe.ebe_create_batch(U["meshes"])
    ebe.ebe_set_problem_batch(h, U["nu"], U["f"], U["dirichlet"], U["g"], U["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    return U, h


def test_batch_barrier_timeout_is_reported_and_the_handle_recovers(ebe):
    probs = [meshgen.fourier_square(s, 1.0, seed=40 + s) for s in (65, 129, 97, 33, 161, 49)]
    U, h = _batch(ebe, probs)
    n = int(U["node_off"][-1])
    x = torch.zeros(n, dtype=torch.float64, device=DEV)
    ebe.ebe_set_batch_config(h, barrier_ns=1)
    with pytest.raises(ebe.EbeError) as ei:
        ebe.ebe_solve_batch(h, x, precision=ebe.EBE_PREC_MIXED)
    assert ei.value.status == ebe.EBE_CUDA_ERROR and "barrier" in str(ei.value)
    assert ebe.ebe_get_stats(h)["device_error"] == 0          # reported once, then cleared
    ebe.ebe_set_batch_config(h)                               # back to the 2 s bound
    x.zero_()
    infos, summary = ebe.ebe_solve_batch(h, x, precision=ebe.EBE_PREC_MIXED)
    assert summary["n_converged"] == len(probs)
    xs = x.cpu().numpy()
    for k, p in enumerate(probs):
        assert oracle.Problem(p).rel_residual(xs[U["node_off"][k]:U["node_off"][k + 1]]) <= 1e-8
    ebe.ebe_destroy(h)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_rtol_below_the_fp64_floor_stalls(ebe, precision):
    # f scaled by 1e12 so that the squares of residuals at the FP64 floor
    # (about 1e-16 |b|) stay in the normal FP32 range of the mixed solver's dots
    prob = meshgen.config_square_f1(33, nu=1.0)
    prob["f"] = prob["f"] * 1e12
    h = _single(ebe, prob)
    x = torch.zeros(prob["coords"].shape[0], dtype=torch.float64, device=DEV)
    prec = {"fp64": ebe.EBE_PREC_FP64, "mixed": ebe.EBE_PREC_MIXED,
            "mixed_textbook": ebe.EBE_PREC_MIXED_TEXTBOOK}[precision]
    # mixed precision checks the true residual at every replacement, here
    # whenever the recurrence residual has halved (delta = 0.5): the checks take
    # it from 1 to its floor, then stall_updates checks without progress end the
    # solve.  (With the default delta = 0.1 the FP32 recurrence started from a
    # residual at the floor need not fall tenfold again: some rounding paths
    # then run to maxit instead.)
    info = ebe.ebe_solve(h, x, rtol=1e-18, precision=prec, stall_updates=3, delta=0.5,
                         maxit=3000 if precision == "fp64" else 100000)
    assert info["status"] == ("EBE_MAXIT" if precision == "fp64" else "EBE_STALL"), info
    # the iterate is still the solution to the attainable accuracy
    assert oracle.Problem(prob).rel_residual(x.cpu().numpy()) <= 1e-12
    ebe.ebe_destroy(h)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_in_x0_is_a_breakdown(ebe, precision):
    prob = meshgen.config_square_jitter(40, nu=1.0, seed=2)
    h = _single(ebe, prob)
    n = prob["coords"].shape[0]
    free = np.setdiff1d(np.arange(n), prob["dirichlet"])
    x0 = np.zeros(n)
    x0[free[len(free) // 2]] = np.nan
    x = torch.tensor(x0, dtype=torch.float64, device=DEV)
    prec = ebe.EBE_PREC_FP64 if precision == "fp64" else ebe.EBE_PREC_MIXED
    info = ebe.ebe_solve(h, x, precision=prec)
    assert info["status"] == "EBE_BREAKDOWN", info
    # the handle still solves a valid start afterwards
    x.zero_()
    info = ebe.ebe_solve(h, x, precision=prec)
    assert info["status"] == "EBE_OK"
    assert oracle.Problem(prob).rel_residual(x.cpu().numpy()) <= 1e-8
    ebe.ebe_destroy(h)


def test_nan_in_one_problem_of_a_batch(ebe):
    probs = [meshgen.fourier_square(s, 2.0, seed=60 + s) for s in (33, 65, 49)]
    U, h = _batch(ebe, probs)
    x0 = np.zeros(int(U["node_off"][-1]))
    lo, hi = U["node_off"][1], U["node_off"][2]
    x0[(lo + hi) // 2] = np.nan                                # an interior node of problem 1
    x = torch.tensor(x0, dtype=torch.float64, device=DEV)
    infos, summary = ebe.ebe_solve_batch(h, x, precision=ebe.EBE_PREC_MIXED)
    assert [i["status"] for i in infos] == ["EBE_OK", "EBE_BREAKDOWN", "EBE_OK"]
    xs = x.cpu().numpy()
    for k in (0, 2):
        assert oracle.Problem(probs[k]).rel_residual(xs[U["node_off"][k]:U["node_off"][k + 1]]) <= 1e-8
    ebe.ebe_destroy(h)
