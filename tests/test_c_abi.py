"""The C ABI from a C program (no GPU): tests/c/abi_host.c is compiled with gcc
as C99 against include/ebe.h, linked with libebe.so and run."""
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
