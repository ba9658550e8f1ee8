"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads
without a GPU, and exports every function include/lbib.h declares (no compute
call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lbib_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1907_00080_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["lbib_create", "lbib_add_membrane", "lbib_set_receptors", "lbib_step",
                 "lbib_read_fields", "lbib_read_markers", "lbib_read_bonds", "lbib_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1907_00080_gb300 import lbib
    missing = [n for n in declared_functions() if n not in lbib._SIGS]
    assert not missing, missing


def test_library_is_built_for_sm_103a(lib):
    from paper_1907_00080_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1907_00080_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lbib_oracle" not in text, f
