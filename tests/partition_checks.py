"""Checks of an element partition exported by ebe_partition_export[_batch].

Shared by the host tests of single meshes and of batches.
"""
import numpy as np


def check_partition(P, coords, elems):
    """Every invariant the patch kernels rely on (see plan.cpp)."""
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


def replay_patch_residual(P, elems, A, b, x, dirichlet):
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
