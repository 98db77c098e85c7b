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


def test_operator_builders_validate_before_touching_a_device():
    # bad arguments are rejected up front; good ones reach the device check,
    # which fails cleanly here (no device, no CPU fallback).  The C entry
    # points are called directly with a NULL stream.
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2506_04732_gb300 as T
    lib = T.load()
    EINVAL, ENODEV = 1, 7

    def build(d, n, beta, eps, n_t=None, t_len=None):
        prob = T._Problem(d, (ctypes.c_int * d)(*n), (ctypes.c_double * d)(*beta), float(eps), 0)
        h = ctypes.c_void_p()
        if n_t is None:
            return lib.t2s2_build_operator(ctypes.byref(prob), None, ctypes.byref(h))
        return lib.t2s2_build_spacetime_operator(ctypes.byref(prob), int(n_t), float(t_len), None,
                                                 ctypes.byref(h))

    good = dict(d=2, n=[8, 8], beta=[0.6, 0.8], eps=1e-2)
    for kw in [dict(n=[2, 8]), dict(n=[8, 129]), dict(eps=0.0), dict(beta=[1.0, float("nan")])]:
        args = {**good, **kw}
        assert build(**args) == EINVAL, kw
        assert build(**args, n_t=6, t_len=1.0) == EINVAL, kw
    for n_t, t_len in [(2, 1.0), (129, 1.0), (6, 0.0), (6, -1.0), (6, float("inf"))]:
        assert build(**good, n_t=n_t, t_len=t_len) == EINVAL, (n_t, t_len)
    assert build(16, [8] * 16, [0.25] * 16, 1e-2, n_t=6, t_len=1.0) == EINVAL   # 17 dimensions
    assert build(**good) == ENODEV
    assert build(**good, n_t=6, t_len=1.0) == ENODEV


def test_variable_coefficient_builder_validates_before_touching_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2506_04732_gb300 as T
    lib = T.load()
    EINVAL, ENODEV = 1, 7

    def build(n=(8, 8), beta=(0.6, 0.8), eps=1e-2, rho0=0.0, fn=True):
        base = T._Problem(2, (ctypes.c_int * 2)(*n), (ctypes.c_double * 2)(*beta), float(eps), 0)
        f = T._COEF_FN(lambda k, x, c: 1.0) if fn else T._COEF_FN()
        prob = T._ProblemVar(base, f, f, float(rho0), None)
        h = ctypes.c_void_p()
        return lib.t2s2_build_operator_var(ctypes.byref(prob), None, ctypes.byref(h))

    assert build(n=(2, 8)) == EINVAL
    assert build(eps=0.0) == EINVAL
    assert build(rho0=float("nan")) == EINVAL
    assert build() == ENODEV
    assert build(fn=False) == ENODEV
    assert lib.t2s2_build_operator_var(None, None, ctypes.byref(ctypes.c_void_p())) == EINVAL
