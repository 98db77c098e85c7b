"""Host logic of the operator build, natively on CPU: the library's own
build_dimension (host_1d.cpp, compiled here with g++ into a small driver)
against the oracle and against what a complex Schur form must satisfy.  The
Schur form B = Z T Z^H of B = Rt^{-1} Lt feeds the exact Kronecker-sum
preconditioner of the local solves."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import collocation as C

ROOT = os.path.join(os.path.dirname(__file__), os.pardir)


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("host1d") / "host_1d_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", exe,
                    os.path.join(ROOT, "tests", "native", "host_1d_check.cpp"),
                    os.path.join(ROOT, "paper_2506_04732_gb300", "csrc", "host_1d.cpp")], check=True)
    return exe


def _run(exe, n, eps, beta, plain):
    out = subprocess.run([exe, str(n), repr(eps), repr(beta), str(int(plain))], check=True,
                         capture_output=True, text=True).stdout
    return _shape(json.loads(out), n - 2)


def _shape(d, m):
    return {k: (np.array(v) if k in ("x", "eta", "R0", "L0") else np.array(v).reshape(m, m))
            for k, v in d.items()}


def _check_schur(h, m):
    T = h["Tr"] + 1j * h["Ti"]
    Z = h["Zr"] + 1j * h["Zi"]
    assert np.linalg.norm(Z.conj().T @ Z - np.eye(m)) <= 1e-13 * m
    assert np.max(np.abs(np.tril(T, -1))) <= 1e-14 * np.linalg.norm(T)
    assert np.linalg.norm(Z @ T @ Z.conj().T - h["B"]) <= 1e-12 * np.linalg.norm(h["B"])
    lam = np.diag(T)
    assert abs(lam.sum() - np.trace(h["B"])) <= 1e-11 * np.linalg.norm(h["B"]) * m
    assert abs((lam ** 2).sum() - np.trace(h["B"] @ h["B"])) <= 1e-10 * np.linalg.norm(h["B"]) ** 2 * m


@pytest.mark.parametrize("n,eps,beta,plain", [(3, 0.1, 1.0, False), (6, 1e-2, 0.8, False),
                                              (12, 1e-3, -0.6, False), (20, 0.05, 0.3, True),
                                              (33, 1e-4, 0.57, False), (128, 1e-3, 0.7, False)])
def test_dimension_data_and_schur_form(driver, n, eps, beta, plain):
    h = _run(driver, n, eps, beta, plain)
    o = C.op1d(n, eps, beta, plain)
    m = n - 2
    scale = lambda A: max(1.0, np.max(np.abs(A)))
    assert np.max(np.abs(h["Rt"] - o.Rt)) <= 1e-12 * scale(o.Rt)
    assert np.max(np.abs(h["Lt"] - o.Lt)) <= 1e-11 * scale(o.Lt)
    # interpolation inverse and B = Rt^{-1} Lt
    assert np.max(np.abs(h["Rinv"] @ h["Rt"] - np.eye(m))) <= 1e-11
    B_ref = np.linalg.solve(o.Rt, o.Lt)
    assert np.linalg.norm(h["B"] - B_ref) <= 1e-10 * np.linalg.norm(B_ref)
    # complex Schur form: Z unitary, T upper triangular, Z T Z^H = B; the
    # diagonal of T carries B's spectrum (its trace and the trace of B^2 are
    # well conditioned even where single eigenvalues are not)
    _check_schur(h, m)


@pytest.mark.parametrize("n,T_len", [(3, 1.0), (7, 2.0), (16, 0.25), (64, 1.0)])
def test_time_dimension_data_and_schur_form(driver, n, T_len):
    from oracle import spacetime as ST
    out = subprocess.run([driver, "time", str(n), repr(2.0 / T_len)], check=True, capture_output=True,
                         text=True).stdout
    m = n - 1
    h = _shape(json.loads(out), m)
    o = ST.time_op1d(n, T_len)
    scale = lambda A: max(1.0, np.max(np.abs(A)))
    assert np.max(np.abs(h["x"] - o.x)) <= 1e-15 and np.max(np.abs(h["eta"] - o.g)) <= 1e-14
    assert np.max(np.abs(h["Rt"] - o.Rt)) <= 1e-12 * scale(o.Rt)
    assert np.max(np.abs(h["Lt"] - o.Lt)) <= 1e-11 * scale(o.Lt)
    assert np.max(np.abs(h["R0"] - o.r0)) <= 1e-12 * scale(o.r0)
    assert np.max(np.abs(h["L0"] - o.l0)) <= 1e-11 * scale(o.l0)
    B_ref = np.linalg.solve(o.Rt, o.Lt)
    assert np.linalg.norm(h["B"] - B_ref) <= 1e-10 * np.linalg.norm(B_ref)
    _check_schur(h, m)
    # the inflow-constrained transport operator is stable: its spectrum lies
    # in the right half plane
    assert np.min(np.diag(h["Tr"])) > 0.0
