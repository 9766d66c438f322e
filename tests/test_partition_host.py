"""Host logic of the library, no GPU: mesh validation and the element
partition that replaces the index arrays ind_e / indt (Sec. 2) on the device.

The last test replays, in numpy, exactly what the patch kernels compute from
the partition (colour-ordered per-patch accumulation, halo sums in patch
order) and compares with the oracle's Algorithm 1 residual: a wrong owned /
shared split, colour class or halo list fails it.
"""
import numpy as np
import pytest

import oracle
from paper_1911_03973_gb300 import meshgen


@pytest.fixture(scope="module")
def ebe():
    from paper_1911_03973_gb300 import build
    build.build()
    import paper_1911_03973_gb300 as mod
    return mod


def _meshes():
    c2, e2 = meshgen.square_tri(100)
    c2 = meshgen.jitter_interior(c2, 1 / 99, 0.2, seed=2)
    c3, e3 = meshgen.cube_tet(12)
    cp, ep, _, _ = meshgen.permute_nodes(*meshgen.square_tri(37), [], seed=4)
    return {"tri_ragged": (c2, e2), "tet": (c3, e3), "tri_perm": (cp, ep), "tri_two": meshgen.square_tri(2)}


@pytest.mark.parametrize("name", list(_meshes()))
def test_partition_invariants(ebe, name):
    coords, elems = _meshes()[name]
    P = ebe.ebe_partition_export(coords, elems)
    n_e, nb = elems.shape
    n_n = coords.shape[0]
    K = P["patch_elems"]
    # every element exactly once
    se = P["slot_elem"]
    assert np.array_equal(np.sort(se[se >= 0]), np.arange(n_e))
    inc = np.bincount(elems.ravel(), minlength=n_n)
    shared_seen = {}
    for p, (node_off, n_nodes, n_owned, halo_off, n_el, col_off, n_col, _) in enumerate(P["patch_meta"]):
        slots = np.arange(p * K, p * K + n_el)
        assert np.all(se[slots] >= 0) and np.all(se[p * K + n_el:(p + 1) * K] == -1)
        gid = P["pnode"][node_off:node_off + n_nodes]
        assert len(np.unique(gid)) == n_nodes
        loc = P["lconn"][:, slots].astype(np.int64)          # [nb][n_el]
        assert loc.max() < n_nodes
        # local connectivity maps back to the caller's element
        np.testing.assert_array_equal(gid[loc].T, elems[se[slots]])
        # owned nodes: all incident elements are in this patch; shared: some are not
        cnt = np.bincount(loc.ravel(), minlength=n_nodes)
        assert np.all(cnt[:n_owned] == inc[gid[:n_owned]])
        assert np.all(cnt[n_owned:] < inc[gid[n_owned:]])
        # colour classes: contiguous slot ranges whose elements share no node
        co = P["col_ptr"][col_off:col_off + n_col + 1]
        assert co[0] == 0 and co[-1] == n_el and np.all(np.diff(co) > 0)
        for c in range(n_col):
            nodes = loc[:, co[c]:co[c + 1]].ravel()
            assert len(np.unique(nodes)) == nodes.size
        for k, l in enumerate(range(n_owned, n_nodes)):
            shared_seen.setdefault(int(gid[l]), []).append(halo_off + k)
    # halo CSR: every shared node lists its halo slots in patch order
    assert len(shared_seen) == P["n_shared"]
    for k, g in enumerate(P["sh_node"]):
        slots = P["sh_slot"][P["sh_ptr"][k]:P["sh_ptr"][k + 1]]
        assert list(slots) == shared_seen[int(g)]
        assert len(slots) >= 2


def _replay_patch_residual(P, elems, A, b, x, dirichlet):
    """What the patch pass + fix-up compute, replayed with the partition."""
    K = P["patch_elems"]
    nb = elems.shape[1]
    r = np.full(b.shape, np.nan)
    halo = np.zeros(P["n_halo"])
    dmask = np.zeros(b.shape, bool)
    dmask[dirichlet] = True
    for p, (node_off, n_nodes, n_owned, halo_off, n_el, col_off, n_col, _) in enumerate(P["patch_meta"]):
        gid = P["pnode"][node_off:node_off + n_nodes]
        xs = x[gid]
        acc = np.zeros(n_nodes)
        co = P["col_ptr"][col_off:col_off + n_col + 1]
        for c in range(n_col):
            s = np.arange(co[c], co[c + 1]) + p * K
            loc = P["lconn"][:, s].astype(np.int64)        # [nb][m]
            Ae = A[P["slot_elem"][s]]                       # [m, nb, nb]
            ye = np.einsum("mij,jm->im", Ae, xs[loc])
            np.add.at(acc, loc.ravel(), ye.ravel())         # no repeats within a colour
        own = gid[:n_owned]
        r[own] = np.where(dmask[own], 0.0, b[own] - acc[:n_owned])
        halo[halo_off:halo_off + n_nodes - n_owned] = acc[n_owned:]
    for k, g in enumerate(P["sh_node"]):
        v = halo[P["sh_slot"][P["sh_ptr"][k]:P["sh_ptr"][k + 1]]].sum()
        r[g] = 0.0 if dmask[g] else b[g] - v
    return r


@pytest.mark.parametrize("case", ["tri", "tet"])
def test_patch_replay_equals_algorithm_1(ebe, case):
    prob = meshgen.config_square_jitter(70, nu=1.0, seed=2) if case == "tri" else meshgen.config_cube_noise(11)
    orc = oracle.Problem(prob)
    P = ebe.ebe_partition_export(prob["coords"], prob["elems"])
    x = orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 5))
    r = _replay_patch_residual(P, prob["elems"], orc.A, orc.rhs(), x, prob["dirichlet"])
    ref = orc.residual(x)
    assert not np.isnan(r).any()
    assert np.linalg.norm(r - ref) <= 1e-12 * np.linalg.norm(ref)


def test_validation_errors_without_gpu(ebe):
    c, e = meshgen.square_tri(4)
    for bad, status in (([[0, 1, 16]], 2), ([[0, 1, -1]], 2), ([[0, 1, 1]], 2)):
        with pytest.raises(ebe.EbeError) as ei:
            ebe.ebe_partition_export(c, np.array(bad, np.int32))
        assert ei.value.status in (status, 1)
    with pytest.raises(ebe.EbeError) as ei:       # node 15 unused
        ebe.ebe_partition_export(c, e[:2])
    assert ei.value.status == 1
    with pytest.raises(ebe.EbeError) as ei:       # n_b != dim + 1
        ebe.ebe_partition_export(c, np.zeros((1, 4), np.int32))
    assert ei.value.status == 1
    c_nan = c.copy()
    c_nan[3, 0] = np.nan
    with pytest.raises(ebe.EbeError) as ei:
        ebe.ebe_partition_export(c_nan, e)
    assert ei.value.status == 1
    with pytest.raises(ebe.EbeError) as ei:       # ebe_create validates before touching a device
        ebe.ebe_create(c, np.array([[0, 1, 99]], np.int32))
    assert ei.value.status == 2
