"""Parity of batches of independent problems on the GPU (through the C ABI).

A batch handle holds several meshes as one disjoint union.  The union's
residual, load vector and Jacobi diagonal must equal each problem's own
(oracle, Algorithm 1, per-problem nu); the batched persistent solver must
bring every problem to the FP64 true relative residual rtol, judged by the
oracle problem by problem, with about the iterations of a single solve.
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


def _problems():
    out = [meshgen.config_square_jitter(97, nu=1.0, seed=2),      # Dirichlet x*y, Neumann sides
           meshgen.fourier_square(17, 0.05, seed=11),             # a single patch, no shared nodes
           meshgen.fourier_square(2, 3.0, seed=12),               # every node Dirichlet: r0 = 0
           meshgen.fourier_square(61, 7.0, seed=13),
           meshgen.config_square_f1(33, nu=0.0, g_value=1.0),     # the paper's experiment: nu = 0, u = 1 on the boundary
           meshgen.fourier_square(129, 0.3, seed=14)]
    return out


@pytest.fixture(scope="module")
def batch(ebe):
    probs = _problems()
    U = meshgen.batch_union(probs)
    stream = torch.cuda.Stream()
    h = ebe.ebe_create_batch(U["meshes"], stream=stream.cuda_stream)
    ebe.ebe_set_problem_batch(h, U["nu"], U["f"], U["dirichlet"], U["g"], U["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    torch.cuda.synchronize()
    orcs = [oracle.Problem(p) for p in probs]
    yield probs, U, h, orcs, stream
    ebe.ebe_destroy(h)


def _split(v, U):
    return [v[U["node_off"][k]:U["node_off"][k + 1]] for k in range(len(U["node_off"]) - 1)]


def _solve(ebe, h, U, stream, **kw):
    with torch.cuda.stream(stream):
        x = torch.zeros(int(U["node_off"][-1]), dtype=torch.float64, device=DEV)
        infos, summary = ebe.ebe_solve_batch(h, x, **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy(), infos, summary


def test_layout(ebe, batch):
    probs, U, h, orcs, stream = batch
    n, no, eo = ebe.ebe_batch_layout(h)
    assert n == len(probs)
    np.testing.assert_array_equal(no, U["node_off"])
    np.testing.assert_array_equal(eo, U["elem_off"])


def test_union_residual_is_every_problem_residual(ebe, batch):
    probs, U, h, orcs, stream = batch
    xs = [o.with_dirichlet(meshgen.seeded_vector(o.n_n, 30 + k)) for k, o in enumerate(orcs)]
    with torch.cuda.stream(stream):
        xd = torch.tensor(np.concatenate(xs), dtype=torch.float64, device=DEV)
        rd = torch.empty_like(xd)
        ebe.ebe_residual(h, xd, rd)
    torch.cuda.synchronize()
    for k, (r, o, x) in enumerate(zip(_split(rd.cpu().numpy(), U), orcs, xs)):
        ref = o.residual(x)
        if np.linalg.norm(ref) == 0.0:
            assert np.all(r == 0.0), k
        else:
            assert np.linalg.norm(r - ref) <= 1e-12 * np.linalg.norm(ref), k


def test_union_rhs_and_jacobi_use_each_problems_nu(ebe, batch):
    probs, U, h, orcs, stream = batch
    n = int(U["node_off"][-1])
    with torch.cuda.stream(stream):
        b = torch.empty(n, dtype=torch.float64, device=DEV)
        d = torch.empty_like(b)
        ebe.ebe_get_rhs(h, b)
        ebe.ebe_jacobi_diag(h, d)
    torch.cuda.synchronize()
    for k, (bk, dk, o) in enumerate(zip(_split(b.cpu().numpy(), U), _split(d.cpu().numpy(), U), orcs)):
        np.testing.assert_allclose(dk, o.jacobi_diag(), rtol=1e-13, err_msg=str(k))
        rb = o.rhs()
        assert np.abs(bk - rb).max() <= 1e-13 * max(np.abs(rb).max(), 1e-300), k


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batched_solve_judged_by_oracle(ebe, batch, precision):
    probs, U, h, orcs, stream = batch
    prec = ebe.EBE_PREC_MIXED if precision == "mixed" else ebe.EBE_PREC_FP64
    x, infos, summary = _solve(ebe, h, U, stream, rtol=1e-8, precision=prec)
    assert summary["n_converged"] == len(probs), infos
    assert summary["launches"] == 1
    for k, (xk, o, info) in enumerate(zip(_split(x, U), orcs, infos)):
        assert info["status"] == "EBE_OK", (k, info)
        if k == 2:                                   # all-Dirichlet problem: r0 = 0, nothing to do
            assert info["iterations"] == 0 and info["r0_norm"] == 0.0
            np.testing.assert_array_equal(xk, o.with_dirichlet(np.zeros(o.n_n)))
            continue
        assert o.rel_residual(xk) <= 1e-8, (k, info)
        assert np.all(xk[o.nd] == o.g)


def test_batched_iterations_match_single_solves(ebe, batch):
    probs, U, h, orcs, stream = batch
    _, infos, _ = _solve(ebe, h, U, stream, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    for k, p in enumerate(probs):
        if k == 2:
            continue
        hs = ebe.ebe_create(p["coords"], p["elems"], stream=stream.cuda_stream)
        ebe.ebe_set_problem(hs, p["nu"], p["f"], p["dirichlet"], p["g"], p["neumann"])
        ebe.ebe_assemble(hs, ebe.EBE_STORE_MIXED)
        with torch.cuda.stream(stream):
            xs = torch.zeros(p["coords"].shape[0], dtype=torch.float64, device=DEV)
            # the batched solver iterates in the textbook form (update and direction
            # phases), so it is compared with the single solver in that form
            single = ebe.ebe_solve(hs, xs, rtol=1e-8, precision=ebe.EBE_PREC_MIXED_TEXTBOOK)
        torch.cuda.synchronize()
        ebe.ebe_destroy(hs)
        it_b, it_s = infos[k]["iterations"], single["iterations"]
        assert abs(it_b - it_s) <= max(2, 0.03 * it_s), (k, it_b, it_s)


def test_batched_solve_is_deterministic_with_and_without_graph(ebe, batch):
    probs, U, h, orcs, stream = batch
    x1, i1, _ = _solve(ebe, h, U, stream, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    x2, i2, _ = _solve(ebe, h, U, stream, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    x3, i3, _ = _solve(ebe, h, U, stream, rtol=1e-8, precision=ebe.EBE_PREC_MIXED, use_graph=False)
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(x1, x3)
    assert [i["iterations"] for i in i1] == [i["iterations"] for i in i3]
    xh = np.zeros(int(U["node_off"][-1]))
    ih, sh = ebe.ebe_solve_batch_host(h, xh, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    np.testing.assert_array_equal(x1, xh)


def test_batched_maxit_stops_only_the_unfinished(ebe, batch):
    probs, U, h, orcs, stream = batch
    x, infos, summary = _solve(ebe, h, U, stream, rtol=1e-8, precision=ebe.EBE_PREC_MIXED, maxit=40)
    status = [i["status"] for i in infos]
    assert status[2] == "EBE_OK"
    for k, i in enumerate(infos):
        assert i["iterations"] <= 40
        if i["status"] == "EBE_MAXIT":
            # the reported residual is a true residual of the returned iterate
            assert abs(orcs[k].rel_residual(_split(x, U)[k]) - i["rel_residual"]) <= 1e-6 * i["rel_residual"]
    assert status.count("EBE_MAXIT") >= 3 and summary["n_converged"] == status.count("EBE_OK")


def test_batch_tuner_and_config(ebe, batch):
    probs, U, h, orcs, stream = batch
    res = ebe.ebe_batch_tune(h, ebe.EBE_PREC_MIXED, loops=20)
    cands = res["candidates"]
    assert len(cands) >= 3 and all(ms > 0 for _, _, ms in cands)
    assert res["best"] in [(c, t) for c, t, _ in cands]
    assert {t for _, t, _ in cands} == {1024, 2048, 4096}
    x, infos, summary = _solve(ebe, h, U, stream, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    assert (summary["ctas_per_sm"], summary["tile_nodes"]) == res["best"]
    assert summary["n_converged"] == len(probs)
    assert summary["phase_ms"]["patch"] > 0.0 and sum(summary["phase_ms"].values()) < summary["solve_ms"]
    # the shape tuned for mixed precision is not imposed on FP64 solves (fewer CTAs fit)
    x, infos, summary = _solve(ebe, h, U, stream, rtol=1e-8, precision=ebe.EBE_PREC_FP64)
    assert summary["n_converged"] == len(probs)
    by_tile = {}
    for c, t, _ in cands:                            # every shape gives a valid solve
        ebe.ebe_set_batch_config(h, c, t)
        x, infos, summary = _solve(ebe, h, U, stream, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
        assert summary["n_converged"] == len(probs), (c, t)
        assert orcs[5].rel_residual(_split(x, U)[5]) <= 1e-8
        # which CTA runs an item does not change any sum: same tile size, same bits
        if t in by_tile:
            np.testing.assert_array_equal(x, by_tile[t])
        by_tile[t] = x
    with pytest.raises(ebe.EbeError):
        ebe.ebe_set_batch_config(h, 1, 3000)
    with pytest.raises(ebe.EbeError):
        ebe.ebe_set_batch_config(h, 8, 2048)
        _solve(ebe, h, U, stream, rtol=1e-8)
    ebe.ebe_set_batch_config(h, 0, 0)


def test_batched_solve_on_a_single_mesh_handle(ebe):
    prob = meshgen.config_square_jitter(129, nu=0.0, seed=5)
    orc = oracle.Problem(prob)
    h = ebe.ebe_create(prob["coords"], prob["elems"])
    ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    x = torch.zeros(orc.n_n, dtype=torch.float64, device=DEV)
    infos, summary = ebe.ebe_solve_batch(h, x, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    torch.cuda.synchronize()
    assert infos[0]["status"] == "EBE_OK"
    assert orc.rel_residual(x.cpu().numpy()) <= 1e-8
    ebe.ebe_destroy(h)


def test_batch_errors(ebe, batch):
    probs, U, h, orcs, stream = batch
    with pytest.raises(ValueError):                   # one nu per problem (checked by the binding)
        ebe.ebe_set_problem_batch(h, U["nu"][:-1], U["f"], U["dirichlet"], U["g"], U["neumann"])
    nu = U["nu"].copy()
    nu[3] = 0.0
    keep = U["dirichlet"][(U["dirichlet"] < U["node_off"][3]) | (U["dirichlet"] >= U["node_off"][4])]
    hb = ebe.ebe_create_batch(U["meshes"])
    with pytest.raises(ebe.EbeError) as ei:           # problem 3: nu = 0 and no Dirichlet node
        ebe.ebe_set_problem_batch(hb, nu, U["f"], keep, None, None)
    assert "problem 3" in str(ei.value)
    ebe.ebe_destroy(hb)


def test_config4_full_batch(ebe):
    """256 squares, sides log-uniform in [17, 513], nu log-uniform in [1e-2, 10]."""
    probs = meshgen.config_batch(256, seed=4)
    U = meshgen.batch_union(probs)
    stream = torch.cuda.Stream()
    h = ebe.ebe_create_batch(U["meshes"], stream=stream.cuda_stream)
    ebe.ebe_set_problem_batch(h, U["nu"], U["f"], U["dirichlet"], U["g"], U["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    x, infos, summary = _solve(ebe, h, U, stream, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
    ebe.ebe_destroy(h)
    assert summary["n_converged"] == 256, [i for i in infos if i["status"] != "EBE_OK"][:3]
    worst = 0.0
    for k, (xk, p) in enumerate(zip(_split(x, U), probs)):
        rel = oracle.Problem(p).rel_residual(xk)
        worst = max(worst, rel)
        assert rel <= 1e-8, (k, rel, infos[k])
    assert worst > 0.0


@pytest.mark.parametrize("precision", ["EBE_PREC_MIXED", "EBE_PREC_FP64"])
def test_batched_solve_on_tetrahedra(ebe, precision):
    # two Kuhn cubes of different sizes and nu: the tetrahedral paths of the
    # persistent solver (per-warp colour sums, and in mixed precision the
    # double-word true residual with each FP32 pair side by side)
    probs = [meshgen.config_cube_noise(14, nu=0.5, seed=3),     # 13,182 tets
             meshgen.config_cube_noise(18, nu=2.0, seed=4)]     # 29,478 tets
    U = meshgen.batch_union(probs)
    stream = torch.cuda.Stream()
    h = ebe.ebe_create_batch(U["meshes"], stream=stream.cuda_stream)
    ebe.ebe_set_problem_batch(h, U["nu"], U["f"], U["dirichlet"], U["g"], U["neumann"])
    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
    x, infos, _ = _solve(ebe, h, U, stream, rtol=1e-8, precision=getattr(ebe, precision))
    for k, (pr, xk) in enumerate(zip(probs, _split(x, U))):
        assert infos[k]["status"] == "EBE_OK", infos[k]
        assert infos[k]["true_residuals"] >= 2
        assert oracle.Problem(pr).rel_residual(xk) <= 1e-8
    ebe.ebe_destroy(h)
