"""Host logic of the small FP64 GEMM on CPU: the tile / split-K plan of the
latency model (gemm.cu, compiled into a driver that launches nothing) keeps
the invariants the kernel relies on, over many shapes."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.join(os.path.dirname(__file__), os.pardir)
SHAPES = {(16, 16), (8, 16), (16, 8), (8, 8), (4, 16), (16, 4), (1, 64), (64, 1), (4, 4)}
SMALL_MAX_FMAS = 16e6


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    import __graft_entry__ as g
    g.build()
    lib = os.path.join(ROOT, "paper_2506_04732_gb300")
    exe = str(tmp_path_factory.mktemp("gemmplan") / "gemm_plan_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=compute_103a", "-O2", "-std=c++17",
                    "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(ROOT, "tests", "native", "gemm_plan_check.cu"), "-L" + lib, "-lt2s2",
                    "-Xlinker", "-rpath", "-Xlinker", os.path.abspath(lib)], check=True)
    return exe


def _plans(exe, shapes):
    inp = "".join(f"s {M} {N} {K} {b}\n" for M, N, K, b in shapes)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    return [tuple(int(v) for v in ln.split()) for ln in out if ln.strip()]


def test_plans_keep_the_kernel_invariants(driver):
    rng = np.random.default_rng(0)
    shapes = [(1, 1, 0, 1), (1, 1, 1, 1), (30, 9, 30, 1), (9, 9, 8000, 1), (270, 9, 9, 1),
              (960, 40, 40, 1), (40, 40, 960, 1), (5, 7, 100000, 3)]
    for _ in range(1500):
        M, N = (int(v) for v in rng.integers(1, 400, 2))
        K = int(rng.integers(0, 20000)) if rng.random() < 0.3 else int(rng.integers(1, 500))
        b = int(rng.integers(1, 64)) if rng.random() < 0.2 else 1
        shapes.append((M, N, K, b))
    plans = _plans(driver, shapes)
    assert len(plans) == len(shapes)
    for (M, N, K, b), (use, bm, bn, splits, kc) in zip(shapes, plans):
        small = M * N * max(K, 1) * b <= SMALL_MAX_FMAS
        assert bool(use) == small, (M, N, K, b)
        if use:
            assert (bm, bn) in SHAPES and 256 % (bm * bn) == 0
            _check_split(K, b, splits, kc)


def _check_split(K, b, splits, kc):
    if K == 0:
        assert splits == 1 and kc == 0
        return
    assert kc >= 8 and kc % 8 == 0
    assert splits == math.ceil(K / kc)          # every split has work ...
    assert (splits - 1) * kc < K <= splits * kc  # ... and together they cover K
    assert 1 <= splits <= 64 and b * splits <= 65535


def test_group_plans_keep_the_kernel_invariants(driver):
    rng = np.random.default_rng(1)
    groups = []
    for _ in range(400):
        n = int(rng.integers(1, 9))
        groups.append([(int(rng.integers(1, 300)), int(rng.integers(1, 300)), int(rng.integers(0, 3000)),
                        1 if rng.random() < 0.8 else int(rng.integers(1, 16))) for _ in range(n)])
    inp = "".join("g %d %s\n" % (len(g), " ".join(f"{M} {N} {K} {b}" for M, N, K, b in g)) for g in groups)
    out = subprocess.run([driver], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [[int(v) for v in ln.split()] for ln in out if ln.strip()]
    assert len(rows) == len(groups)
    for g, row in zip(groups, rows):
        ok, bm, bn = row[:3]
        small = all(M * N * max(K, 1) * b <= SMALL_MAX_FMAS for M, N, K, b in g)
        assert bool(ok) == small
        if not ok:
            continue
        assert (bm, bn) in SHAPES   # one tile shape for the whole launch
        for i, (M, N, K, b) in enumerate(g):
            _check_split(K, b, row[3 + 2 * i], row[4 + 2 * i])
