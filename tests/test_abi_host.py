"""Host-side checks of the C ABI (no GPU needed): the library loads and exports
every entry point include/ebe.h declares, and the binding declares them all."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ebe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ebe_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1911_03973_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_api():
    names = _declared()
    for n in ("ebe_create", "ebe_destroy", "ebe_set_problem", "ebe_assemble", "ebe_residual", "ebe_apply",
              "ebe_solve", "ebe_solve_host", "ebe_jacobi_diag", "ebe_get_rhs", "ebe_element_matrices"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(lib):
    from paper_1911_03973_gb300 import _abi
    bound = {s[0] for s in _abi.SIGNATURES}
    assert set(_declared()) <= bound, set(_declared()) - bound
    import paper_1911_03973_gb300 as ebe
    for n in _declared():
        assert hasattr(ebe, n), n


def test_status_strings_and_defaults(lib):
    import paper_1911_03973_gb300 as ebe
    from paper_1911_03973_gb300 import _abi
    assert ebe.ebe_status_string(0) == "EBE_OK"
    assert ebe.ebe_status_string(8) == "EBE_BREAKDOWN"
    o = _abi.ebe_solve_opts()
    _abi.load().ebe_solve_opts_default(ctypes.byref(o))
    assert o.rtol == 1e-8 and o.precision == 0 and o.use_graph == 1
