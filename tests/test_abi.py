"""The C ABI library builds for sm_103a, loads without a GPU and exports every entry point
that include/rbfsl.h declares (no compute calls: this runs on CPU-only machines)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(rbfsl_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rbfsl_trace_rk4", "rbfsl_knn_query", "rbfsl_stencil_weights",
                 "rbfsl_gather_dot", "rbfsl_create", "rbfsl_step", "rbfsl_get_q"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1804_01609_gb300 import rbfsl
    L = rbfsl.load()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert b"sm_103a" in L.rbfsl_version()


def test_binding_covers_every_declared_symbol():
    from paper_1804_01609_gb300 import rbfsl
    assert set(declared_functions()) <= set(rbfsl.SIGNATURES)
