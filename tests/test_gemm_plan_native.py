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
    inp = "".join(f"{M} {N} {K} {b}\n" for M, N, K, b in shapes)
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
        if not use:
            continue
        assert (bm, bn) in SHAPES and 256 % (bm * bn) == 0
        if K == 0:
            assert splits == 1 and kc == 0
            continue
        assert kc >= 8 and kc % 8 == 0
        assert splits == math.ceil(K / kc)          # every split has work ...
        assert (splits - 1) * kc < K <= splits * kc  # ... and together they cover K
        assert 1 <= splits <= 64 and b * splits <= 65535
