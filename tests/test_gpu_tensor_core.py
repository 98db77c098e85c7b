"""GPU parity of the tcgen05 tensor-core TT apply (BF16 and TF32 operands).

Each output element of the apply is one sum over j of (operator entry) x
(core entry).  With both factors rounded to the operand format (unit
roundoff u: 2^-8 for BF16, 2^-11 for TF32), their products exact in binary32
and K = m terms accumulated in binary32, the error of an element is at most
    (2u + u^2 + 2 K 2^-24) * sum_j |A_ij| |x_j|,
the standard bound for a dot product with rounded inputs (the factor 2 on the
accumulation term allows accumulation by truncation).  The right-hand side
is the oracle's TT-matrix product of the element-wise absolute values.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import operator as O
from oracle import tt as OT

pytestmark = pytest.mark.gpu

U = {"bf16": 2.0 ** -8, "tf32": 2.0 ** -11}


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2506_04732_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg


APPLY = [
    (3, 14, [1, 3, 4, 1]),
    (6, 30, [1, 5, 7, 20, 9, 3, 1]),      # ragged ranks; one 128-row tile per core
    (4, 31, [1, 33, 70, 65, 1]),          # 2310 / 4550 rows: many tiles and a ragged tail
    (5, 46, [1, 16, 16, 16, 16, 1]),      # 2m = 92, K = 46 (not a multiple of 16)
    (3, 62, [1, 40, 40, 1]),              # n = 64: 2m = 124, the largest tile
    (1, 20, [1, 1]),                      # d = 1
    (2, 1, [1, 1, 1]),                    # m = 1: one-element contractions
]


@pytest.mark.parametrize("fmt", ["bf16", "tf32"])
@pytest.mark.parametrize("d,m,r", APPLY)
@pytest.mark.parametrize("cm,co", [(0.0, 1.0), (1.0, -0.05)])
def test_apply_tc_within_rounding_bound(T, fmt, d, m, r, cm, co):
    from paper_2506_04732_gb300 import problem as P
    p = W.config1(d=d, n=m + 2, ratio=3e-3)
    op = P.build_operator(p)
    ops = O.build(p)
    x = W.random_tt(d, m, r, seed=d * 100 + m)
    tx = T.TT.from_cores(x)
    ty = T.TT.empty(tx.m, 2 * max(r))
    prec = T.BF16_REFINE if fmt == "bf16" else T.TF32_REFINE
    T.t2s2_trace(True)
    T.t2s2_apply(op, tx, ty, c_mass=cm, c_op=co, prec=prec)
    tc = T.t2s2_trace_read("apply_tc")
    T.t2s2_trace(False)
    assert tc["launches"] == 1, "the tensor-core kernel did not run"
    assert ty.r == [1] + [2 * v for v in r[1:-1]] + [1]
    A = O.ttm_cores(ops, cm, co)
    ref = OT.matvec(A, x)
    bound = OT.matvec([np.abs(a) for a in A], [np.abs(c) for c in x])
    u = U[fmt]
    gamma = 2 * u + u * u + 2 * m * 2.0 ** -24
    worst = 0.0
    for a, b, s in zip(ty.cores(), ref, bound):
        assert a.shape == b.shape
        err = np.abs(a - b)
        assert np.all(err <= gamma * s * 1.0001 + 1e-300), (fmt, float(np.max(err / (s + 1e-300))), gamma)
        # blocks that are exactly zero in the product stay exactly zero
        assert np.all(a[s == 0] == 0)
        worst = max(worst, float(np.max(err)))
    # rounded operands leave a visible error (the FP64 kernel did not run instead)
    if m > 1:
        assert worst > 0


@pytest.mark.parametrize("fmt", ["bf16", "tf32"])
def test_apply_tc_large_m_takes_fp64_kernel(T, fmt):
    """Cores with m > 64 are outside the tensor-core tile; the FP64 kernel runs."""
    from paper_2506_04732_gb300 import problem as P
    d, m, r = 2, 70, [1, 3, 1]
    p = W.config1(d=d, n=m + 2, ratio=3e-3)
    op = P.build_operator(p)
    ops = O.build(p)
    x = W.random_tt(d, m, r, seed=7)
    tx = T.TT.from_cores(x)
    ty = T.TT.empty(tx.m, 6)
    prec = T.BF16_REFINE if fmt == "bf16" else T.TF32_REFINE
    T.t2s2_apply(op, tx, ty, prec=prec)
    ref = OT.matvec(O.ttm_cores(ops, 0.0, 1.0), x)
    for a, b in zip(ty.cores(), ref):
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.abs(b).max())


GEMMS = [
    # (M, N, K, tA, tB, batch): the sweep's shapes and ragged / degenerate ones
    (600, 24, 24, False, True, 1),     # mode-3 product X x_3 Q
    (24, 600, 24, False, False, 1),    # mode-1 product (swapped onto the MMA's M side)
    (30, 20, 30, False, False, 20),    # batched mode-2 product
    (20, 24, 600, True, False, 1),     # left interface: split K
    (20, 24, 600, False, True, 1),     # right interface: split K
    (300, 300, 70, True, True, 2),     # several column tiles, K not a stage multiple
    (1, 1, 1, False, False, 1),
    (5, 3, 0, False, False, 1),        # empty K: C = beta C
    (129, 257, 65, False, False, 1),   # one past every tile edge
    (2000, 40, 4000, True, True, 1),   # long K, many row tiles
    (17, 9, 700, True, False, 4),      # batched split K added inside the launch
    (8, 8, 33, False, False, 1),       # K one past a slice
]


@pytest.mark.parametrize("fmt", ["fp64", "bf16", "tf32"])
@pytest.mark.parametrize("M,N,K,tA,tB,batch", GEMMS)
def test_gemm_within_rounding_bound(T, fmt, M, N, K, tA, tB, batch):
    from paper_2506_04732_gb300 import problem as P
    op = P.build_operator(W.config0())
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    a = rng.standard_normal((batch, K, M) if tA else (batch, M, K))
    b = rng.standard_normal((batch, N, K) if tB else (batch, K, N))
    c0 = rng.standard_normal((batch, M, N))
    alpha, beta = 0.75, -0.5
    A, B, C = (torch.tensor(v, device="cuda") for v in (a, b, c0))
    prec = {"fp64": T.FP64, "bf16": T.BF16_REFINE, "tf32": T.TF32_REFINE}[fmt]
    T.t2s2_gemm(op, A, B, C, tA=tA, tB=tB, alpha=alpha, beta=beta, prec=prec)
    torch.cuda.synchronize()
    opa = np.transpose(a, (0, 2, 1)) if tA else a
    opb = np.transpose(b, (0, 2, 1)) if tB else b
    ref = alpha * opa @ opb + beta * c0
    got = C.cpu().numpy()
    if fmt == "fp64":
        scale = np.abs(alpha) * np.abs(opa) @ np.abs(opb) + np.abs(beta * c0)
        assert np.all(np.abs(got - ref) <= 1e-14 * (K + 2) * scale + 1e-300)
        return
    u = U[fmt]
    gamma = 2 * u + u * u + 2 * max(K, 1) * 2.0 ** -24
    bound = gamma * abs(alpha) * (np.abs(opa) @ np.abs(opb)) + 1e-15 * np.abs(beta * c0)
    err = np.abs(got - ref)
    assert np.all(err <= bound * 1.0001 + 1e-300), float(np.max(err / (bound + 1e-300)))
    if K > 1:
        assert float(np.max(err)) > 0  # the operands really were rounded


@pytest.mark.parametrize("fmt", ["fp64", "bf16", "tf32"])
def test_grouped_apply_matches_per_instance_products(T, fmt):
    """Many instances of uneven n and ranks in one persistent launch."""
    from paper_2506_04732_gb300 import problem as P
    probs = [W.config3(i) for i in range(12)]
    ops, xs, ys, refs, bounds = [], [], [], [], []
    for i, p in enumerate(probs):
        m = p.n[0] - 2
        r = [1] + [int(v) for v in np.random.default_rng(i).integers(1, 17, p.d - 1)] + [1]
        x = W.random_tt(p.d, m, r, seed=500 + i)
        ops.append(P.build_operator(p))
        xs.append(T.TT.from_cores(x))
        ys.append(T.TT.empty([m] * p.d, 2 * max(r)))
        A = O.ttm_cores(O.build(p), 0.5, 1.0)
        refs.append(OT.matvec(A, x))
        bounds.append(OT.matvec([np.abs(a) for a in A], [np.abs(c) for c in x]))
    prec = {"fp64": T.FP64, "bf16": T.BF16_REFINE, "tf32": T.TF32_REFINE}[fmt]
    T.t2s2_apply_batched(ops, xs, ys, c_mass=0.5, c_op=1.0, prec=prec)
    T.t2s2_apply_batched(ops, xs, ys, c_mass=0.5, c_op=1.0, prec=prec)  # tuned launch shape
    for y, ref, bnd, p in zip(ys, refs, bounds, probs):
        m = p.n[0] - 2
        for a, b, s in zip(y.cores(), ref, bnd):
            assert a.shape == b.shape
            if fmt == "fp64":
                assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.abs(b).max())
            else:
                u = U[fmt]
                gamma = 2 * u + u * u + 2 * m * 2.0 ** -24
                assert np.all(np.abs(a - b) <= gamma * s * 1.0001 + 1e-300)
    assert "apply" in T.t2s2_autotune_report()


@pytest.mark.parametrize("variant", ["direct", "staged"])
@pytest.mark.parametrize("fmt", ["bf16", "tf32"])
def test_grouped_apply_each_variant_within_rounding_bound(T, fmt, variant, monkeypatch):
    """Both variants of the grouped tensor-core apply (operand rows loaded
    directly, or staged in shared memory by a bulk TMA copy of the next
    tile's rows) against the FP64 oracle product, at the per-element rounding
    bound; instances of uneven n and ranks, including odd ranks (odd range
    lengths and starts of the staged copies)."""
    from paper_2506_04732_gb300 import problem as P
    monkeypatch.setenv("T2S2_APPLY_VARIANT", variant)
    probs = [W.config3(i) for i in range(10)]
    ops, xs, ys, refs, bounds = [], [], [], [], []
    for i, p in enumerate(probs):
        m = p.n[0] - 2
        r = [1] + [int(v) for v in np.random.default_rng(40 + i).integers(1, 24, p.d - 1)] + [1]
        x = W.random_tt(p.d, m, r, seed=900 + i)
        ops.append(P.build_operator(p))
        xs.append(T.TT.from_cores(x))
        ys.append(T.TT.empty([m] * p.d, 2 * max(r)))
        A = O.ttm_cores(O.build(p), 0.25, 1.0)
        refs.append(OT.matvec(A, x))
        bounds.append(OT.matvec([np.abs(a) for a in A], [np.abs(c) for c in x]))
    prec = {"bf16": T.BF16_REFINE, "tf32": T.TF32_REFINE}[fmt]
    for _ in range(2):   # the second launch rewrites the same values
        T.t2s2_apply_batched(ops, xs, ys, c_mass=0.25, c_op=1.0, prec=prec)
    for y, ref, bnd, p in zip(ys, refs, bounds, probs):
        m = p.n[0] - 2
        for a, b, s in zip(y.cores(), ref, bnd):
            assert a.shape == b.shape
            u = U[fmt]
            gamma = 2 * u + u * u + 2 * m * 2.0 ** -24
            assert np.all(np.abs(a - b) <= gamma * s * 1.0001 + 1e-300)
