"""Host logic of batches, no GPU: the union partition of several independent
meshes (ebe_partition_export_batch, the partition ebe_create_batch uploads).

Each problem must be partitioned exactly as on its own, shifted into the
union numbering, and no patch may mix two problems; a numpy replay of the
patch pass over the union must give every problem's Algorithm 1 residual.
"""
import numpy as np
import pytest

import oracle
from paper_1911_03973_gb300 import meshgen
from partition_checks import check_partition, replay_patch_residual


@pytest.fixture(scope="module")
def ebe():
    from paper_1911_03973_gb300 import build
    build.build()
    import paper_1911_03973_gb300 as mod
    return mod


def _problems():
    p0 = meshgen.config_square_jitter(40, nu=1.0, seed=2)
    p1 = meshgen.fourier_square(17, 0.05, seed=11)     # one patch, no shared nodes
    p2 = meshgen.fourier_square(2, 3.0, seed=12)       # two elements
    cp, ep, (dp,), _ = meshgen.permute_nodes(*meshgen.square_tri(29), [meshgen.square_boundary_nodes(29)], seed=4)
    p3 = meshgen.fourier_square(29, 7.0, seed=13)
    p3 = dict(p3, coords=cp, elems=ep, dirichlet=dp, g=np.zeros(dp.size), f=np.ones(cp.shape[0]))
    return [p0, p1, p2, p3]


def test_batch_partition_is_the_shifted_single_partitions(ebe):
    probs = _problems()
    U = meshgen.batch_union(probs)
    B = ebe.ebe_partition_export_batch(U["meshes"])
    coords = np.concatenate([c for c, _ in U["meshes"]])
    elems = np.concatenate([e + U["node_off"][k] for k, (_, e) in enumerate(U["meshes"])]).astype(np.int32)
    check_partition(B, coords, elems)
    K = B["patch_elems"]
    po = B["patch_off"]
    assert po[0] == 0 and po[-1] == B["n_patches"]
    pn_off = hal_off = col_off = sh_off = 0
    for k, (c, e) in enumerate(U["meshes"]):
        S = ebe.ebe_partition_export(c, e)
        n0, e0 = U["node_off"][k], U["elem_off"][k]
        assert po[k + 1] - po[k] == S["n_patches"]
        sl = slice(po[k] * K, po[k + 1] * K)
        se = B["slot_elem"][sl]
        np.testing.assert_array_equal(np.where(se >= 0, se - e0, -1), S["slot_elem"])
        np.testing.assert_array_equal(B["lconn"][:, sl], S["lconn"])
        meta = B["patch_meta"][po[k]:po[k + 1]].copy()
        meta[:, 0] -= pn_off
        meta[:, 3] -= hal_off
        meta[:, 5] -= col_off
        np.testing.assert_array_equal(meta, S["patch_meta"])
        np.testing.assert_array_equal(B["pnode"][pn_off:pn_off + S["n_pnode"]] - n0, S["pnode"])
        np.testing.assert_array_equal(B["col_ptr"][col_off:col_off + S["n_colptr"]], S["col_ptr"])
        shs = slice(sh_off, sh_off + S["n_shared"])
        np.testing.assert_array_equal(B["sh_node"][shs] - n0, S["sh_node"])
        np.testing.assert_array_equal(B["sh_ptr"][sh_off:sh_off + S["n_shared"] + 1] - hal_off, S["sh_ptr"])
        np.testing.assert_array_equal(B["sh_slot"][hal_off:hal_off + S["n_halo"]] - hal_off, S["sh_slot"])
        # no patch of problem k touches another problem's nodes
        for p in range(po[k], po[k + 1]):
            off, nn = B["patch_meta"][p][:2]
            ids = B["pnode"][off:off + nn]
            assert ids.min() >= n0 and ids.max() < U["node_off"][k + 1]
        pn_off += S["n_pnode"]
        hal_off += S["n_halo"]
        col_off += S["n_colptr"]
        sh_off += S["n_shared"]
    assert pn_off == B["n_pnode"] and hal_off == B["n_halo"] and sh_off == B["n_shared"]


def test_batch_replay_gives_every_problem_residual(ebe):
    probs = _problems()
    U = meshgen.batch_union(probs)
    B = ebe.ebe_partition_export_batch(U["meshes"])
    orcs = [oracle.Problem(p) for p in probs]
    elems = np.concatenate([e + U["node_off"][k] for k, (_, e) in enumerate(U["meshes"])]).astype(np.int32)
    A = np.concatenate([o.A for o in orcs])
    b = np.concatenate([o.rhs() for o in orcs])
    xs = [o.with_dirichlet(meshgen.seeded_vector(o.n_n, 20 + k)) for k, o in enumerate(orcs)]
    r = replay_patch_residual(B, elems, A, b, np.concatenate(xs), U["dirichlet"])
    ref = np.concatenate([o.residual(x) for o, x in zip(orcs, xs)])
    assert not np.isnan(r).any()
    assert np.linalg.norm(r - ref) <= 1e-12 * np.linalg.norm(ref)


def test_batch_validation_names_the_problem(ebe):
    c, e = meshgen.square_tri(5)
    bad = e.copy()
    bad[3, 1] = 99
    with pytest.raises(ebe.EbeError) as ei:
        ebe.ebe_partition_export_batch([(c, e), (c, e), (c, bad)])
    assert ei.value.status == 2 and "problem 2" in str(ei.value)
    c3, e3 = meshgen.cube_tet(3)
    with pytest.raises(ebe.EbeError) as ei:            # all problems must have the same dim
        ebe.ebe_partition_export_batch([(c, e), (c3, e3)])
    assert ei.value.status == 1
    with pytest.raises(ebe.EbeError) as ei:            # validated before any device work
        ebe.ebe_create_batch([(c, e), (c, bad)])
    assert ei.value.status == 2 and "problem 1" in str(ei.value)


def test_config_batch_recipe():
    probs = meshgen.config_batch(n_problems=64, seed=4)
    sides = np.array([int(round(p["coords"].shape[0] ** 0.5)) for p in probs])
    nus = np.array([p["nu"] for p in probs])
    assert sides.min() >= 17 and sides.max() <= 513
    assert nus.min() >= 1e-2 and nus.max() <= 10.0
    # log-uniform: about half of the sides below the geometric mean sqrt(17 * 513) ~ 93
    assert 0.25 < np.mean(sides < 93) < 0.75
    for p in probs[:4]:
        s = int(round(p["coords"].shape[0] ** 0.5))
        assert p["dirichlet"].size == 4 * (s - 1)
        assert np.all(p["g"] == 0.0)
    U = meshgen.batch_union(probs[:3])
    assert U["f"].size == U["node_off"][-1] and U["dirichlet"].max() < U["node_off"][-1]
