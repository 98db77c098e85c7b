"""The C-ABI library loads and exports every symbol declared in include/t2s2.h (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(t2s2_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["t2s2_build_operator", "t2s2_apply", "t2s2_round", "t2s2_solve", "t2s2_cn_step"]:
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as T
    lib = T.load()
    for n in sorted(_declared()):
        assert hasattr(lib, n), f"missing export {n}"
    assert T.t2s2_strerror(0) == "ok"
    assert "invalid" in T.t2s2_strerror(1)


def test_no_device_reports_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2506_04732_gb300 as T
    assert T.t2s2_device_count() == 0
