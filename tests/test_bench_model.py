"""The benchmark's algorithmic byte model, pinned to hand counts (no GPU).

Per pass, each of the n_b^2 entries of the element arrays, each int32
connectivity index and each node-vector entry read or written counts once.
"""
import bench


def test_square_2049_bytes():
    n_n, n_e = 2049 * 2049, 2 * 2048 * 2048          # 4,198,401 nodes, 8,388,608 triangles
    m = bench.bytes_model(2, n_n, n_e)
    # FP64 residual: 9 x 8 B + 3 x 4 B per triangle; x, b in and r out, 8 B each
    assert m["residual64"] == n_e * (72 + 12) + n_n * 24 == 805_404_696
    # FP32 operator: 9 x 4 B + 3 x 4 B per triangle; p in, q out
    assert m["apply32"] == n_e * (36 + 12) + n_n * 8 == 436_240_392
    stored = bench.bytes_model(2, n_n, n_e, stored=True)
    assert stored["apply32"] == n_e * (24 + 12) + n_n * 8 == 335_577_096
    assert stored["residual64"] == n_e * (48 + 12) + n_n * 24


def test_cube_129_bytes():
    n_n, n_e = 129 ** 3, 6 * 128 ** 3                  # 2,146,689 nodes, 12,582,912 tetrahedra
    m = bench.bytes_model(3, n_n, n_e)
    assert m["residual32"] == n_e * (64 + 16) + n_n * 12   # about 1,032 MB
    assert abs(m["residual32"] / 1e6 - 1032.4) < 0.1
    assert m["residual64"] == n_e * (128 + 16) + n_n * 24
    stored = bench.bytes_model(3, n_n, n_e, stored=True)
    assert stored["apply32"] == n_e * (40 + 16) + n_n * 8


def test_mixed_iteration_node_bytes():
    # one mixed CG iteration's node work: update reads x (8), p, r, q, dinv (4 each)
    # and writes x (8), r (4); direction reads r, dinv, p and writes p (4 each)
    m = bench.bytes_model(2, 1000, 1)
    assert m["vec_mixed"] == 1000 * (8 + 16 + 12 + 12 + 4)


def test_fp64_pipe_model():
    # FP64 residual on 2049^2 triangles: 9 products + 3 node additions per
    # triangle, r = b - sum and r.r per node; 2 FP64 operations per SM and clock
    n_n, n_e = 2049 * 2049, 2 * 2048 * 2048
    a = bench.fp64_alu_model(3, n_n, n_e, 152, 2070.0)
    assert a["ops_per_launch"] == 12 * n_e + 2 * n_n == 109_060_098
    assert a["peak_gops"] == 629.3                       # 2 x 152 x 2.07 GHz
    t = bench.fp64_alu_model(4, 129 ** 3, 6 * 128 ** 3, 152, 2070.0)
    assert t["ops_per_launch"] == 20 * 6 * 128 ** 3 + 2 * 129 ** 3
    assert bench.fp64_alu_model(3, n_n, n_e, 152, None) is None
    assert bench.fp64_alu_model(3, n_n, n_e, 0, 2070.0) is None


def test_single_sync_iteration_bytes():
    # one pass of the single-sync mixed solver on 2049^2 triangles: the
    # operator's 9 x 4 B + 3 x 4 B per triangle, per node r, q, p, dinv (4 B) and
    # x (8 B) in, r, p, q (4 B) and x (8 B) out
    n_n, n_e = 2049 * 2049, 2 * 2048 * 2048
    m = bench.bytes_model(2, n_n, n_e)
    assert m["cg_mixed"] == n_e * (36 + 12) + n_n * 44 == 587_382_828
    stored = bench.bytes_model(2, n_n, n_e, stored=True)
    assert stored["cg_mixed"] == n_e * (24 + 12) + n_n * 44
    # a step: element matrices, one pass per iteration and per start of the
    # recurrence, a true residual and a restart per check
    info = {"iterations": 100, "true_residuals": 3}
    assert bench.step_bytes(m, info, True) == (m["assemble_mixed"] + 103 * m["cg_mixed"]
                                               + 3 * (m["residual64"] + n_n * 16))


def test_textbook_mixed_step_bytes():
    # the textbook mixed iteration (the batched solver's form): FP32 operator,
    # update and direction per iteration; an FP64 true residual per check and
    # a restart (r64, dinv in; r32 out; then a direction step) per replacement
    n_n, n_e = 2049 * 2049, 2 * 2048 * 2048
    m = bench.bytes_model(2, n_n, n_e)
    assert m["apply32"] + m["vec_mixed"] == n_e * 48 + n_n * (8 + 52)
    assert m["restart_mixed"] == n_n * (16 + 16)
    info = {"iterations": 100, "true_residuals": 3}
    assert bench.solve_bytes(m, info, True, textbook=True) == (100 * (m["apply32"] + m["vec_mixed"])
                                                               + 3 * m["residual64"] + 2 * m["restart_mixed"])
