"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/fenc.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "fenc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fe_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2606_16359_b300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = header_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib_path):
    import paper_2606_16359_b300 as fe
    assert sorted(fe.SIGNATURES) == header_functions()
    lib = fe.load()
    assert lib.fe_last_error() is not None


def test_build_targets_sm_103a():
    from paper_2606_16359_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
