"""The C ABI from a C program (no GPU): tests/c/abi_host.c is compiled with gcc
as C99 against include/ebe.h, linked with libebe.so and run."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_uses_the_abi():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1911_03973_gb300 import build
    lib = build.build()
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "abi_host")
        subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c", "abi_host.c"), lib, "-o", exe,
                        "-Wl,-rpath," + os.path.dirname(lib)], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert out.returncode == 0, out.stderr
        assert out.stdout.strip() == "ok"


@pytest.mark.gpu
def test_c_program_solves_through_the_abi():
    # create / set_problem / assemble / solve_host from C, judged by the oracle
    import numpy as np

    import oracle
    from paper_1911_03973_gb300 import build, meshgen
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lib = build.build()
    oracle.build()
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "solve_host")
        xbin = os.path.join(d, "x.bin")
        subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c", "solve_host.c"), lib, "-o", exe,
                        "-Wl,-rpath," + os.path.dirname(lib)], check=True)
        out = subprocess.run([exe, xbin], capture_output=True, text=True, timeout=600)
        assert out.returncode == 0, out.stdout + out.stderr
        lines = out.stdout.split("\n")
        assert lines[0].startswith("fp64 EBE_OK") and lines[1].startswith("mixed EBE_OK"), out.stdout
        xs = np.fromfile(xbin, dtype=np.float64).reshape(2, -1)
    orc = oracle.Problem(meshgen.config_square_f1(33, nu=1.0))
    for x in xs:
        assert orc.rel_residual(x) <= 1e-8


def test_binding_struct_layouts_match_the_c_compiler():
    # every struct of include/ebe.h: size and field offsets from gcc against ctypes
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1911_03973_gb300 import _abi
    fields = {
        "ebe_mesh": ["dim", "n_b", "n_n", "n_e", "coords", "elems"],
        "ebe_create_opts": ["device", "patch_elems"],
        "ebe_solve_opts": ["rtol", "maxit", "precision", "chunk", "delta", "stall_updates", "use_graph", "race_iters"],
        "ebe_solve_info": ["status", "iterations", "true_residuals", "rel_residual", "r0_norm", "solve_ms"],
        "ebe_stats": ["kernel_launches", "device_error"],
        "ebe_batch_config": ["ctas_per_sm", "tile_nodes", "barrier_ns"],
        "ebe_batch_info": ["loops", "launches", "n_converged", "solve_ms", "config", "phase_ms"],
        "ebe_partition_sizes": ["n_patches", "patch_elems"],
    }
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "layout")
        subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c", "layout.c"), "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=60, check=True).stdout
    seen = set()
    for line in out.strip().split("\n"):
        name, size, *offs = line.split()
        cls = getattr(_abi, name)
        assert ctypes.sizeof(cls) == int(size), name
        for f, off in zip(fields[name], offs):
            assert getattr(cls, f).offset == int(off), (name, f)
        seen.add(name)
    assert seen == set(fields)
