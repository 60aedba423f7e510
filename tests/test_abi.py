"""The C ABI library loads and exports every entry point include/rst.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(rst_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_core_calls():
    names = declared_functions()
    for want in ["rst_build", "rst_cc", "rst_euler_root", "rst_build_batch", "rst_select", "rst_verify",
                 "rst_status_string", "rst_bcc", "rst_insert_edges", "rst_tree_depth", "rst_set_option"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2603_11645_gb300 import LIB_PATH
    assert os.path.exists(LIB_PATH), "librst.so was not built"
    lib = ctypes.CDLL(LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_host_only_entry_points():
    import paper_2603_11645_gb300 as rst
    L = rst.lib()
    assert L.rst_version() >= 100
    for code in range(8):
        assert L.rst_status_string(code)
    # argument errors are caught before any GPU work
    assert L.rst_build(None, 33, None, 10, 0, 0, 2, None, None) == 1
    assert L.rst_build(None, 32, None, -1, 0, 0, 2, None, None) == 1
    assert L.rst_euler_root(10, None, 20, 0, None, None, None) == 1


def test_oracle_is_not_imported_by_the_package():
    pkg = os.path.join(ROOT, "paper_2603_11645_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".c", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "liboracle" not in text, fn
