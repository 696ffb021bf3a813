"""The C-ABI library builds for sm_103a and exports every entry point that
include/heat3d.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "heat3d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1307_7867_gb300 import build
    return build.build()


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("heat3d_init", "mg_vcycle", "sdc_sweep", "pfasst_run", "heat3d_submit",
                     "heat3d_workspace_size", "heat3d_bind_workspace"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_abi():
    from paper_1307_7867_gb300 import heat3d
    assert sorted(heat3d.ABI_FUNCTIONS) == declared_functions()


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_1307_7867_gb300 import heat3d
    with pytest.raises(RuntimeError):
        heat3d.open_library(str(tmp_path / "missing.so"))
