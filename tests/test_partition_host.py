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
from partition_checks import check_partition, replay_patch_residual


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
    check_partition(ebe.ebe_partition_export(coords, elems), coords, elems)


@pytest.mark.parametrize("case", ["tri", "tet"])
def test_patch_replay_equals_algorithm_1(ebe, case):
    prob = meshgen.config_square_jitter(70, nu=1.0, seed=2) if case == "tri" else meshgen.config_cube_noise(11)
    orc = oracle.Problem(prob)
    P = ebe.ebe_partition_export(prob["coords"], prob["elems"])
    x = orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, 5))
    r = replay_patch_residual(P, prob["elems"], orc.A, orc.rhs(), x, prob["dirichlet"])
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
    with pytest.raises(ebe.EbeError) as ei:       # an empty mesh has nothing to partition
        ebe.ebe_partition_export(c, np.zeros((0, 3), np.int32))
    assert ei.value.status == 1


def test_single_element_mesh(ebe):
    # one triangle: one patch of one slot, every node owned, no halo
    c = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    e = np.array([[0, 1, 2]], np.int32)
    P = ebe.ebe_partition_export(c, e)
    check_partition(P, c, e)
    assert P["n_patches"] == 1 and P["n_shared"] == 0 and P["patch_meta"][0][2] == 3


def _bank_wavefronts(P, group=32, banks=32):
    """Shared-memory cycles of the colour rounds' node-sum accesses, as the FP32
    patch kernel issues them: 32 consecutive slots per warp, one access per
    element vertex, split by colour; a cycle per distinct address in the most
    loaded bank.  Returns (cycles, the one-cycle-per-access minimum)."""
    K = P["patch_elems"]
    cycles = ideal = 0
    for p, (node_off, n_nodes, n_owned, halo_off, n_el, col_off, n_col, _) in enumerate(P["patch_meta"]):
        co = P["col_ptr"][col_off:col_off + n_col + 1]
        colour = np.repeat(np.arange(n_col), np.diff(co))
        loc = P["lconn"][:, p * K:p * K + n_el].astype(np.int64)
        for g0 in range(0, n_el, group):
            sl = slice(g0, min(g0 + group, n_el))
            for c in np.unique(colour[sl]):
                sel = colour[sl] == c
                for i in range(loc.shape[0]):
                    b = np.bincount(loc[i, sl][sel] % banks, minlength=banks)
                    cycles += int(b.max())
                    ideal += 1
    return cycles, ideal


def test_local_numbering_spreads_banks(ebe):
    # local node ids are chosen per patch so that a warp's accesses fall in
    # distinct shared-memory banks where possible; numbering nodes in first-touch
    # order instead costs about 2.7x the minimum on this mesh
    c, e = meshgen.square_tri(257)
    c = meshgen.jitter_interior(c, 1 / 256, 0.2, seed=2)
    cycles, ideal = _bank_wavefronts(ebe.ebe_partition_export(c, e))
    assert cycles <= 2.1 * ideal, (cycles, ideal)


def test_random_meshes_partition_and_replay(ebe):
    # random sizes (ragged last patches), jitter, node and element orders, in 2D
    # (few colours per patch) and 3D (many colours): every invariant, and the
    # replayed patch pass against the oracle's Algorithm 1
    rng = np.random.Generator(np.random.PCG64(2024))
    for trial in range(12):
        tri = trial % 3 != 2
        n = int(rng.integers(3, 60)) if tri else int(rng.integers(3, 12))
        if tri:
            c, e = meshgen.square_tri(n)
            c = meshgen.jitter_interior(c, 1.0 / (n - 1), 0.2, seed=int(rng.integers(1 << 30)))
        else:
            c, e = meshgen.cube_tet(n)
        c, e, _, _ = meshgen.permute_nodes(c, e, [], seed=int(rng.integers(1 << 30)))
        e = e[rng.permutation(e.shape[0])]
        P = ebe.ebe_partition_export(c, e)
        check_partition(P, c, e)
        prob = {"coords": c, "elems": e, "nu": 0.5, "f": np.ones(c.shape[0]),
                "dirichlet": np.array([0], np.int32), "g": np.zeros(1), "neumann": np.zeros(0, np.int32)}
        orc = oracle.Problem(prob)
        x = orc.with_dirichlet(meshgen.seeded_vector(orc.n_n, trial))
        r = replay_patch_residual(P, e, orc.A, orc.rhs(), x, prob["dirichlet"])
        ref = orc.residual(x)
        assert np.linalg.norm(r - ref) <= 1e-12 * max(np.linalg.norm(ref), 1e-300), (trial, n, tri)


def test_validation_reports_the_first_failure_on_a_large_mesh(ebe):
    # 2 * 400^2 = 320,000 elements: the checks run over several host threads,
    # and each must still name the lowest failing element or node
    c, e = meshgen.square_tri(401)
    n_e = e.shape[0]
    for bad_at, value, word in ((250_000, -5, "outside"), (300_000, None, "repeats")):
        eb = e.copy()
        later = n_e - 7
        for k in (later, bad_at):                  # a later fault too: the earlier one is reported
            if value is None:
                eb[k, 2] = eb[k, 0]
            else:
                eb[k, 1] = value
        with pytest.raises(ebe.EbeError) as ei:
            ebe.ebe_partition_export(c, eb)
        assert ei.value.status == 2 and f"element {bad_at} " in str(ei.value) and word in str(ei.value), str(ei.value)
    cb = c.copy()
    cb[150_000, 1] = np.inf
    cb[20_000, 0] = np.nan
    with pytest.raises(ebe.EbeError) as ei:
        ebe.ebe_partition_export(cb, e)
    assert ei.value.status == 1 and "node 20000" in str(ei.value), str(ei.value)
    # nodes 100,000 and 160,000 in no element: drop every element touching them
    touch = np.isin(e, [100_000, 160_000]).any(axis=1)
    with pytest.raises(ebe.EbeError) as ei:
        ebe.ebe_partition_export(c, e[~touch])
    assert ei.value.status == 1 and "node 100000 " in str(ei.value), str(ei.value)


def test_partition_does_not_depend_on_the_host_thread_count():
    # the same meshes partitioned on 1 and on 8 host threads (EBE_HOST_THREADS),
    # each in a process of its own: every table is byte-identical
    import hashlib
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import hashlib, numpy as np, paper_1911_03973_gb300 as ebe\n"
        "from paper_1911_03973_gb300 import meshgen\n"
        "p = meshgen.config_square_jitter(513, nu=1.0, seed=2)\n"
        "c, e = meshgen.cube_tet(31)\n"
        "c, e, _, _ = meshgen.permute_nodes(c, e, [], seed=6)\n"
        "e = e[np.random.default_rng(7).permutation(e.shape[0])]\n"
        "for cc, ee in ((p['coords'], p['elems']), (c, e)):\n"
        "    P = ebe.ebe_partition_export(cc, ee)\n"
        "    h = hashlib.sha256()\n"
        "    for k in sorted(P):\n"
        "        h.update(k.encode()); h.update(np.ascontiguousarray(np.asarray(P[k])).tobytes())\n"
        "    print(h.hexdigest())\n")
    out = []
    for t in ("1", "8"):
        env = dict(os.environ, EBE_HOST_THREADS=t)
        env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
        res = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                             timeout=600)
        assert res.returncode == 0, res.stderr[-2000:]
        out.append(res.stdout.split())
    assert len(out[0]) == 2 and out[0] == out[1], out


def test_clustered_mesh_partition(ebe):
    # 1.2 M small triangles in a corner of a bounding box stretched by one
    # large triangle: almost every Morton key shares its 12 highest bits, so
    # the key sort takes its fallback (a bucket above 2^20 keys); the
    # partition must still satisfy every invariant
    c, e = meshgen.square_tri(776)
    c = c * 1e-3
    n0 = c.shape[0]
    c = np.vstack([c, [[10.0, 0.0], [0.0, 10.0], [10.0, 10.0]]])
    e = np.vstack([e, [[n0, n0 + 2, n0 + 1]]]).astype(np.int32)
    P = ebe.ebe_partition_export(c, e)
    check_partition(P, c, e)
