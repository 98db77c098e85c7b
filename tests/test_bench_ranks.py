"""The bench's multi-rank host logic on CPU: two gloo ranks on 127.0.0.1.

The solve does not shard (independent replicas, one per GPU), so the only
cross-rank steps are the barrier around the timed region and the max over
ranks of the elapsed time; the whole-job rate counts every rank's solves.
"""
import argparse
import multiprocessing as mp
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        dist.barrier()
        # rank r "took" 10 + r seconds
        q.put((rank, bench.max_over_ranks(10.0 + rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 11.0, 1: 11.0}


def test_max_over_ranks_without_a_group_is_the_identity():
    assert bench.max_over_ranks(3.5) == 3.5


def test_replica_rate_counts_every_rank():
    # 2 replicas x 200 solves in 0.5 s (the slowest rank) = 800 solves/s
    assert bench.replica_rate(2, 200, 0.5) == pytest.approx(800.0)
    assert bench.replica_rate(1, 5, 0.0) == 0.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(steps=5, warmup=3, cpu_budget=20.0, gpus=2, impl="reference")
    assert bench.run_reference(args) == 0


def test_clock_lines_median_max_and_reasons():
    ok = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    cap = "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1300.0, 0x8, Active, Not Active, Not Active, Not Active"
    r = bench.parse_clock_lines([ok, cap, ok])
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    r = bench.parse_clock_lines([ok, hot, "garbage", "0, [N/A], 2070, 1, 0, a, b, c, d"])
    assert r["reasons"] == ["hw_slowdown"] and r["samples"] == 2 and r["sm_mhz"] == 2070.0
    assert bench.parse_clock_lines([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_clock_sampler_flow_with_a_fake_nvidia_smi(tmp_path, monkeypatch):
    # a stand-in nvidia-smi that prints one sample every 20 ms: the sampler
    # drops the sample taken before the region and parses the rest
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\nwhile true; do\n"
                    "echo '0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "sleep 0.02\ndone\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    import time
    s = bench.ClockSampler(0)
    s.start()
    assert s.skip >= 1          # the region starts once the sampler is live
    time.sleep(0.2)
    r = s.stop()
    assert r["sm_mhz"] == 2070.0 and r["reasons"] == [] and r["samples"] >= 3
    assert r["samples_in_region"] >= 3


def test_oracle_solves_are_complete_and_timed_one_by_one():
    # the reference arm's steps: whole oracle solves in a child process, each
    # timed on its own and reaching the workload's tolerance
    recs = bench.oracle_solves("config0()", 2, 120.0)
    assert len(recs) == 2
    for r in recs:
        assert r["res"] <= 1e-12 and r["sweeps"] >= 1 and r["t"] > 0


def test_oracle_solves_stop_at_the_budget():
    # a budget shorter than one solve ends the child with nothing finished
    assert bench.oracle_solves("config1()", 5, 0.5) == []


def test_kernel_names_map_to_trace_families():
    # device-time ranking in bench.py groups kernels by the library's trace
    # families; unknown kernels (torch's own) are "other"
    kf = bench.kernel_family
    assert kf("void t2s2::(anonymous namespace)::cholqr3_kernel<26>(t2s2::CqrArgs)") == "cholqr"
    assert kf("t2s2::(anonymous namespace)::cqr_cluster_kernel(t2s2::(anonymous namespace)::CqrArgs)") == "cholqr"
    assert kf("t2s2::sylv_rb1_kernel(t2s2::SylvProblem)") == "sylvester"
    assert kf("void t2s2::small_group_kernel<8, 16>(t2s2::GroupArgs)") == "gemm"
    assert kf("void t2s2::small_kernel<4, 4>(t2s2::Gemm<double>)") == "gemm"
    assert kf("t2s2::tt_norm2_dd_kernel(t2s2::DdArgs)") == "dots"
    assert kf("void t2s2::apply_kernel<t2s2::ParamWork, 16, 16>(t2s2::ApplyBatch)") == "apply"
    assert kf("void t2s2::apply_tc_kernel<2>(t2s2::TcArgs)") == "apply_tc"
    assert kf("t2s2::(anonymous namespace)::k_sumsq(double const*, unsigned long, double*)") == "elementwise"
    assert kf("void at::native::vectorized_elementwise_kernel<4, at::native::FillFunctor<unsigned char>>") == "other"
    assert set(bench.ALU_FAMILIES) <= set(bench.FAMILIES)


def test_round_counts_of_a_matrix_and_their_scaling():
    """d = 2 is one matrix: one QR of the m1 x r unfolding (Q formed), R
    carried into core 0, then one SVD step of the m0 x r unfolding; bytes
    read and written per pass.  Doubling every rank and mode size multiplies
    the FLOPs by 16 (m r^3 terms) and the bytes by 8 (r m r cores; 4 for the
    two end cores)."""
    m0, m1, r, keep = 10, 12, 6, 3
    fl, by, n_in = bench.round_counts([m0, m1], [1, r, 1], [1, keep, 1])
    qr = 4 * m1 * r * r - 4 * r ** 3 / 3 + 2 * 1 * m0 * r * r
    svd = 4 * m0 * r * r - 4 * r ** 3 / 3 + 12 * r ** 3 + 2 * m0 * r * keep + 2 * keep * r * m1 * 1
    assert fl == pytest.approx(qr + svd)
    assert n_in == m0 * r + r * m1
    assert by == 8 * (3 * (m0 * r + r * m1) + (m0 * keep + keep * m1))
    m, rin, rout = [20] * 5, [1, 8, 8, 8, 8, 1], [1, 4, 4, 4, 4, 1]
    f1, b1, _ = bench.round_counts(m, rin, rout)
    f2, b2, _ = bench.round_counts([2 * v for v in m], [1] + [16] * 4 + [1], [1] + [8] * 4 + [1])
    assert 12 < f2 / f1 < 16.5
    assert 7 < b2 / b1 < 8.01
