"""Host-side checks of the C-ABI library (no GPU work is launched here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hg_[a-zA-Z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1311_0089_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hg_create", "hg_create_grid", "hg_set_coeffs", "hg_set_coeffs_phase",
                     "hg_solve_AH", "hg_submit", "hg_poll", "hg_cancel", "hg_apply"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(built_lib):
    import paper_1311_0089_gb300 as hg
    bound = {name for name, _, _ in hg.SIGNATURES}
    assert set(declared_functions()) <= bound
    hg.load(built_lib)


def test_strerror_and_defaults_without_gpu(built_lib):
    import paper_1311_0089_gb300 as hg
    lib = hg.load(built_lib)
    assert lib.hg_strerror(-2).decode().startswith("unsupported grid size")
    o = hg.default_opts()
    assert o.tol == 1e-10 and o.max_iter == 10000 and o.check_every == 8 and o.prec == 0
    assert o.resident == -1


def test_null_arguments_are_rejected_without_gpu(built_lib):
    import paper_1311_0089_gb300 as hg
    lib = hg.load(built_lib)
    assert lib.hg_create(None, 0, 0, None) == -1
    assert lib.hg_create_grid(None, 2, None, None, None) == -1
    assert lib.hg_solve_AH(None, None, None, None) == -1
    assert lib.hg_poll(None, 1, None, 0) == -1
