#!/usr/bin/env python
"""Benchmark of the T^2S^2 hot path on GB300: solves/sec to relative residual 1e-8.

Workload: the steady d=6, n=32 problem (eps/|beta L| = 1e-3, beta a seeded
unit vector, source manufactured from a rank-4 separable u*, TT rank cap 20,
tolerance 1e-8).  One step = one full TT solve through the C ABI
(t2s2_solve): operator application, rounding, alternating sweeps with local
solves, and the FP64 residual that stops them.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|fp32]
    python bench.py --impl reference ...   # the FP64 CPU oracle, timed on the host

Multi-GPU runs (torchrun, one rank per GPU) are replicas: every rank solves its
own instance; value = all ranks' solves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/sec to rel. residual 1e-8 (d=6,n=32)"
UNIT = "solves/s"
FAMILIES = ["gemm", "apply", "local_solve", "small_factor", "elementwise", "apply_tc", "gemm_tc", "mlp", "cholqr",
            "sylvester", "dots"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 200 for the headline solve, whose timed region then spans "
                         "several clock samples; 5 for the other workloads and the reference arm)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the precision-variant and grouped-contraction measurements")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of oracle CPU work for the cpu_baseline sample")
    ap.add_argument("--workload", default="steady",
                    choices=["steady", "batched", "cn", "warm", "contract", "spacetime", "stability", "round"],
                    help="steady: d=6 n=32 solve (headline); batched: 256 d=5 instances; "
                         "cn: Crank-Nicolson steps at d=7 n=64; warm: learned warm start "
                         "(--instances training solves); contract: grouped core contractions of "
                         "--instances d=5 problems in one launch; spacetime: d=5 space plus time "
                         "(n=32, n_t=24) solved as one collocation system; stability: the Plain-SC / "
                         "superconsistent stability map (d=6) through the batched solve; round: TT rounding of the "
                         "Crank-Nicolson right-hand side (d=7, n=64, rank 80 -> 40) and of the 256 batched "
                         "instances after an apply (rank 32 -> 16), against HBM and the FP64 ALU")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--holdout", type=int, default=1000, help="held-out problems of --workload warm")
    ap.add_argument("--warm-rank", type=int, default=1, help="TT rank of the warm-start network's output")
    ap.add_argument("--train-steps", type=int, default=3000, help="Adam steps of --workload warm")
    ap.add_argument("--workers", type=int, default=8)
    return ap.parse_args()


def max_over_ranks(x: float) -> float:
    """The largest x over the ranks of the default process group (x itself
    when no group is initialised or it has one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(ws: int, steps: int, seconds: float) -> float:
    """Whole-job rate of ws independent replicas that each ran `steps` units,
    timed by the slowest rank's `seconds`."""
    return ws * steps / seconds if seconds > 0 else 0.0


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.skip = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
            return
        # the timed region starts once the sampler is live; the sample taken
        # before it is dropped
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.skip = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        inside = len(self.lines) - self.skip
        if inside <= 0:
            # a region shorter than the interval: take the next sample, which
            # the nvidia-smi loop writes within about 100 ms of its end
            t0 = time.time()
            while len(self.lines) <= self.skip and time.time() - t0 < 1.0 and self.proc.poll() is None:
                time.sleep(0.005)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        out = parse_clock_lines(self.lines[self.skip:])
        out["samples_in_region"] = max(0, inside)
        return out


def parse_clock_lines(lines):
    """Median SM clock, the largest maximum clock and the throttle reasons seen
    in nvidia-smi lines of ClockSampler.QUERY (csv, no header, no units)."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2] if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 ALU peak of GB300: 2 DFMA per clock per SM (4 FLOP) x 152 SMs at the
# 1965 MHz clock this part sustains under FP64 load.
FP64_ALU_PEAK_GFLOPS = 4 * 152 * 1.965


# Kernel families that the FP64 ALU bounds (the rest: memory).
ALU_FAMILIES = ("gemm", "apply", "local_solve", "small_factor", "cholqr", "sylvester", "dots")

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# family's dominant kernel from an ncu capture of the current build, with the
# summary it comes from; a family without a current capture is left out.
KERNEL_DRAM_BYTES = {
    "sylvester": (107008.0, "profiles/sylv_rb1_kernel_steady_d6n32.md"),
}


def kernel_family(name: str) -> str:
    """Trace family of a kernel, by its (demangled) name."""
    table = (("cholqr3_kernel", "cholqr"), ("cqr_cluster_kernel", "cholqr"), ("sylv_rb1_kernel", "sylvester"), ("tt_norm2_dd_kernel", "dots"),
             ("tt_dots_kernel", "dots"), ("small_group_kernel", "gemm"), ("small_kernel", "gemm"),
             ("gemm_tc_kernel", "gemm_tc"), ("gemm_kernel", "gemm"), ("splitk", "gemm"),
             ("apply_tc_kernel", "apply_tc"), ("apply_kernel", "apply"), ("gmres_team_kernel", "local_solve"),
             ("local_eig_kernel", "local_solve"), ("jacobi_svd_kernel", "small_factor"),
             ("chol_inv_kernel", "small_factor"), ("t2s2::", "elementwise"))
    for key, famname in table:
        if key in name:
            return famname
    return "other"


def kernel_device_times(fn, torch):
    """{kernel name: (launches, device microseconds)} of one call of fn, from
    CUPTI activity records through torch.profiler; {} if unavailable.  Used to
    rank kernels by device time only: no reported rate comes from it."""
    try:
        from torch.profiler import ProfilerActivity, profile
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
        out = {}
        for ev in prof.key_averages():
            us = getattr(ev, "device_time_total", None)
            if us is None:
                us = getattr(ev, "cuda_time_total", 0.0)
            if us and us > 0 and "Memcpy" not in ev.key and "Memset" not in ev.key:
                out[ev.key] = (int(ev.count), float(us))
        return out
    except Exception as exc:  # recorded by the caller
        return {"__error__": (0, 0.0, repr(exc))}


_ORACLE_CHILD = r"""
import sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import operator as O
from oracle import solve as S
p = W.{cfg}
ops = O.build(p)
b = O.source_tt(p, ops)
for i in range({count}):
    x0 = [np.ones((1, n - 2, 1)) for n in p.n]
    t0 = time.perf_counter()
    x, res, sweeps = S.solve_collocation(ops, b, x0, p.tol, p.rmax, max_sweeps=p.max_sweeps)
    t = time.perf_counter() - t0
    print(json.dumps({{"i": i, "t": t, "res": res, "sweeps": sweeps}}), flush=True)
"""


def oracle_solves(problem_expr, count, budget_s):
    """Complete FP64 oracle solves of a workload on the host cores.

    A child process builds the oracle's operator and source once and then runs
    up to `count` complete solves from the rank-1 start (oracle.solve.
    solve_collocation: AMEn to the workload's tolerance), each timed on its
    own; it is stopped once `budget_s` seconds have passed.  Returns one
    record per finished solve: {"t": seconds, "res": residual, "sweeps": n}.
    """
    import subprocess as sp
    code = _ORACLE_CHILD.format(root=ROOT, cfg=problem_expr, count=int(count))
    proc = sp.Popen([sys.executable, "-c", code], stdout=sp.PIPE, stderr=sp.DEVNULL, text=True)
    lines = []

    def reader():
        for ln in proc.stdout:
            lines.append(ln)

    th = threading.Thread(target=reader, daemon=True)
    th.start()
    try:
        proc.wait(timeout=budget_s)
    except sp.TimeoutExpired:
        proc.kill()
        proc.wait()
    th.join(timeout=5)
    out = []
    for ln in lines:
        try:
            out.append(json.loads(ln))
        except ValueError:
            pass
    return out


def cpu_baseline_sample(problem_expr, budget_s, tol):
    """The oracle's rate on a bounded sample: complete solves within budget_s
    (the first, which pays the process's warm-up, is left out when others
    finished).  Returns (solves/s or 0, description)."""
    recs = oracle_solves(problem_expr, 1000, budget_s)
    timed = recs[1:] if len(recs) > 1 else recs
    conv = [r for r in timed if r["res"] <= tol]
    tot = sum(r["t"] for r in timed)
    if not conv or tot <= 0:
        return 0.0, f"no complete oracle solve within {budget_s:.0f} s"
    return len(conv) / tot, (f"{len(conv)} complete oracle solves to {tol:g} (AMEn in the node-to-node form, "
                             f"{max(r['sweeps'] for r in conv)} sweep(s), residual <= "
                             f"{max(r['res'] for r in conv):.1e}), {tot / len(timed):.2f} s each, "
                             f"within a {budget_s:.0f} s budget; the process's first solve is untimed")


REF_TOTAL_S = 600.0       # bound on the whole reference run


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import workloads as W
    p = W.config1()
    # one child process runs the warm-up solves and then the K timed ones, each
    # step one complete oracle solve of the headline workload
    recs = oracle_solves("config1()", args.warmup + args.steps, REF_TOTAL_S)
    timed = recs[args.warmup:]
    conv = [r for r in timed if r["res"] <= p.tol]
    tot = sum(r["t"] for r in timed)
    value = len(conv) / tot if tot > 0 else 0.0
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(timed), "warmup": min(args.warmup, len(recs)),
            "ms_per_step": 1e3 * tot / len(timed) if timed else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": p.name, "d": p.d, "n": p.n[0], "tol": p.tol,
                                             "rmax": p.rmax, "steps_requested": args.steps,
                                             "sweeps": [r["sweeps"] for r in timed],
                                             "residuals": [r["res"] for r in timed]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{len(timed)} timed complete oracle solves (FP64 numpy, AMEn in the "
                                       f"node-to-node form to {p.tol:g}) after {args.warmup} untimed ones"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batched(args, T, P, W, torch):
    """256 independent d=5 instances (n in {16,24,32,48}) solved by one batched call."""
    import numpy as np
    probs = [W.config3(i) for i in range(args.instances)]
    ops, bs, xs0 = [], [], []
    for p in probs:
        op = P.build_operator(p)
        ops.append(op)
        bs.append(T.TT.from_cores(P.source_cores(p, op)))
        xs0.append([np.ones((1, n - 2, 1)) for n in p.n])

    def fresh():
        return [T.TT.from_cores(c, rcap=16 + T.RANK_KICK) for c in xs0]

    for _ in range(max(1, args.warmup)):
        T.t2s2_solve_batched(ops, bs, fresh(), 1e-8, 16, 50, workers=args.workers, allow_noconv=True)
    torch.cuda.synchronize()
    times, infos, solved = [], None, 0
    for _ in range(args.steps):
        xs = fresh()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = T.t2s2_solve_batched(ops, bs, xs, 1e-8, 16, 50, workers=args.workers, allow_noconv=True)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        solved += sum(1 for inf in infos if inf.residual <= 1e-8)
    # only solves that reached the tolerance count towards the rate
    batched = solved / sum(times)
    # sequential plain solves of a subset, one instance after the other
    nseq = min(32, args.instances)
    xs = fresh()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(nseq):
        T.t2s2_solve(ops[i], bs[i], xs[i], 1e-8, 16, 50, allow_noconv=True)
    torch.cuda.synchronize()
    seq = nseq / (time.perf_counter() - t0)
    conv = sum(1 for inf in infos if inf.residual <= 1e-8)
    line = {"metric": "solves/sec to rel. residual 1e-8 (256 batched d=5 instances)", "value": batched,
            "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.instances} instances d=5 n in {{16,24,32,48}}",
                       "workers": args.workers, "converged": conv, "instances": args.instances,
                       "unconverged": [i for i, inf in enumerate(infos) if inf.residual > 1e-8],
                       "max_sweeps": max(inf.sweeps for inf in infos),
                       "sequential_solves_per_s": seq, "sequential_sample": nseq}}
    print(json.dumps(line))
    return 0


_ORACLE_CN_CHILD = r"""
import sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import operator as O
from oracle import solve as S
p = W.config2()
ops = O.build(p)
u = O.solution_tt(p, ops)
for i in range({count}):
    t0 = time.perf_counter()
    u, res, sweeps = S.cn_step(ops, u, p.dt, p.tol, p.rmax)
    print(json.dumps({{"i": i, "t": time.perf_counter() - t0, "res": res, "sweeps": sweeps}}), flush=True)
"""


def oracle_cn_steps(budget_s):
    """Crank-Nicolson steps of the FP64 oracle on the d=7, n=64 workload in a
    child process, each timed on its own, until budget_s has passed."""
    import subprocess as sp
    code = _ORACLE_CN_CHILD.format(root=ROOT, count=100)
    proc = sp.Popen([sys.executable, "-c", code], stdout=sp.PIPE, stderr=sp.DEVNULL, text=True)
    lines = []
    th = threading.Thread(target=lambda: lines.extend(proc.stdout), daemon=True)
    th.start()
    try:
        proc.wait(timeout=budget_s)
    except sp.TimeoutExpired:
        proc.kill()
        proc.wait()
    th.join(timeout=5)
    out = []
    for ln in lines:
        try:
            out.append(json.loads(ln))
        except ValueError:
            pass
    return out


def run_cn(args, T, P, W, torch):
    """Crank-Nicolson run of the d=7, n=64 Gaussian pulse: the workload's 100
    steps of dt = 1e-3 (rmax 40, tol 1e-8), FP64, timed with device events;
    then the same trajectory with TF32 / BF16 tensor-core contractions under
    FP64 refinement, with their distance to the FP64 states after 10 and 100
    steps (t2s2_diff_norm)."""
    p = W.config2()
    nsteps = args.steps
    op = P.build_operator(p)
    u0 = P.solution_cores(p, op)
    rcap = p.rmax + T.RANK_KICK
    stream = torch.cuda.current_stream()
    # warm-up steps on a scratch copy: the measured trajectory starts at u0
    uw = T.TT.from_cores(u0, rcap=rcap)
    for _ in range(args.warmup):
        T.t2s2_cn_step(op, uw, p.dt, p.tol, p.rmax)
    torch.cuda.synchronize()

    def trajectory(prec):
        u = T.TT.from_cores(u0, rcap=rcap)
        infos, keep = [], {}
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for k in range(1, nsteps + 1):
            e0.record(stream)
            infos.append(T.t2s2_cn_step(op, u, p.dt, p.tol, p.rmax, prec=prec))
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            if k in (10, nsteps):   # states kept outside the timed spans
                keep[k] = T.TT(u.m, list(u.r), [b.clone() for b in u.buffers], u.loc)
        return u, infos, keep, ms

    clocks = ClockSampler(0)
    clocks.start()
    u, infos, keep64, ms = trajectory(T.FP64)
    clk = clocks.stop()
    variants = {}
    for name, prec in (("tf32_refine", T.TF32_REFINE), ("bf16_refine", T.BF16_REFINE)):
        try:
            uv, iv, keepv, msv = trajectory(prec)
            variants[name] = {"steps_per_s": 1e3 * nsteps / msv,
                              "max_step_residual": max(i.residual for i in iv),
                              "rel_diff_vs_fp64": {str(k): T.t2s2_diff_norm(op, keepv[k], keep64[k]) /
                                                   T.t2s2_norm(op, keep64[k]) for k in keep64}}
        except Exception as exc:  # recorded, never hides the FP64 number
            variants[name] = {"error": repr(exc)}
    cpu = None
    if args.cpu_budget > 0:
        recs = oracle_cn_steps(max(60.0, args.cpu_budget))
        if recs:
            tot = sum(r["t"] for r in recs)
            cpu = {"value": len(recs) / tot, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"the oracle's first {len(recs)} Crank-Nicolson steps of the same trajectory "
                             f"(FP64 numpy, {tot / len(recs):.1f} s each)"}
    line = {"metric": "Crank-Nicolson steps/sec (d=7, n=64, dt=1e-3, tol 1e-8)", "value": 1e3 * nsteps / ms,
            "unit": "steps/s", "n_gpus": 1, "steps": nsteps, "warmup": args.warmup, "ms_per_step": ms / nsteps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": p.name, "rmax": p.rmax, "final_ranks": u.r,
                       "step_residuals_max": max(i.residual for i in infos),
                       "all_steps_converged": all(i.residual <= p.tol for i in infos),
                       "sweeps_per_step": [i.sweeps for i in infos],
                       "max_rank": max(i.max_rank for i in infos)},
            "precision_variants": variants, "cpu_baseline": cpu, "clocks": clk}
    print(json.dumps(line))
    return 0


def run_spacetime(args, T, P, W, torch):
    """Unified space-time solve: d=5 spatial dimensions plus time as one
    collocated dimension (n=32, n_t=24), the initial condition lifted into the
    right-hand side by the library, solved to 1e-8 from a rank-1 start."""
    import numpy as np
    st = W.config_spacetime()
    sp = st.space
    op = T.t2s2_build_spacetime_operator(sp.d, sp.n, sp.beta, sp.eps, st.n_t, st.T, sp.plain_sc)
    dims = P.spacetime_dims(st)
    b = T.TT.from_cores(P.spacetime_source_cores(st, dims))
    u0 = T.TT.from_cores(P.spacetime_initial_cores(st, dims))
    rcap_rhs = 4 * max(b.r) + 4 * max(u0.r) + 8
    rhs = T.TT.empty(list(op.m), rcap_rhs)
    T.t2s2_spacetime_rhs(op, b, u0, rhs, 1e-2 * sp.tol, rcap_rhs)
    x = T.TT.from_cores([np.ones((1, m, 1)) for m in op.m], rcap=sp.rmax + T.RANK_KICK)
    x_init = [buf.clone() for buf in x.buffers]

    def reset_x():
        for dst, src in zip(x.buffers, x_init):
            dst.copy_(src)
        x.r = [1] * (op.d + 1)

    infos = []
    for _ in range(args.warmup):
        reset_x()
        infos.append(T.t2s2_solve(op, rhs, x, sp.tol, sp.rmax, sp.max_sweeps, allow_noconv=True))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    clocks.start()
    total = 0.0
    infos = []
    for _ in range(args.steps):
        reset_x()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos.append(T.t2s2_solve(op, rhs, x, sp.tol, sp.rmax, sp.max_sweeps, allow_noconv=True))
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    clk = clocks.stop()
    ms = total / args.steps
    last = infos[-1]
    # only timed solves that reached the tolerance count towards the rate
    solved = sum(1 for inf in infos if inf.residual <= sp.tol)
    line = {"metric": "space-time solves/sec to rel. residual 1e-8 (d=5+t, n=32, n_t=24)",
            "value": 1e3 * solved / total if total > 0 else 0.0, "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": sp.name, "converged": solved, "timed_solves": len(infos),
                       "residual": last.residual, "sweeps": last.sweeps,
                       "max_rank": last.max_rank, "status": last.status, "rhs_ranks": rhs.r},
            "clocks": clk}
    print(json.dumps(line))
    return 0


def run_warm(args, T, P, W, torch):
    """Learned warm start on the d=6, n=32 parameter family (ratio log-uniform
    in [1e-4, 1e-2], rank-4 source from 8 parameters, tol 1e-8, rmax 20):
    generate --instances training solutions with the solver itself (seeds
    10000+i), train the network on the GPU (the library's forward, backward
    and Adam kernels), then solve --holdout held-out problems (seeds 90000+i)
    cold and warm to the same tolerance.  The network outputs TT cores of
    rank --warm-rank (1 by default: a rank-1 guess keeps the first sweep's
    rank-1 right interfaces, the path on which a cold solve of this family
    converges in one sweep)."""
    import numpy as np
    ntrain, nhold, rw = args.instances, args.holdout, args.warm_rank
    d, n, rmax, tol = 6, 32, 20, 1e-8
    m = n - 2

    def solve(p, net=None, r0=None):
        op = P.build_operator(p)
        b = T.TT.from_cores(P.source_cores(p, op))
        x = T.TT.from_cores([np.ones((1, m, 1))] * d, rcap=rmax + T.RANK_KICK)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t_inf = 0.0
        if net is not None:
            net.predict(W.warm_features(p), x)
            t_inf = time.perf_counter() - t0
        if r0 is not None:  # initial residual, outside the solve's timing
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            r0.append(T.t2s2_residual(op, b, x))
            t0 += time.perf_counter() - t1
        info = T.t2s2_solve(op, b, x, tol, rmax, 50, allow_noconv=True)
        torch.cuda.synchronize()
        return op, x, info, time.perf_counter() - t0, t_inf

    t0 = time.perf_counter()
    train = [W.config4(10000 + i, d=d, n=n) for i in range(ntrain)]
    net = T.WarmStartNet(W.WARM_IN_DIM, 256, [m] * d, rw, rmax + T.RANK_KICK, seed=1)
    per = net.d * net.ru * net.mmax * net.ru
    tg = torch.zeros(ntrain * per, dtype=torch.float32, device="cuda")
    uu = torch.zeros(ntrain, dtype=torch.float32, device="cuda")
    train_sweeps, op0, x0 = [], None, None
    for i, p in enumerate(train):
        op, x, info, _, _ = solve(p)
        train_sweeps.append(info.sweeps)
        # each solution goes straight into its packed slot; one operator and
        # solution are kept for the output initialisation
        net.pack_target_into(op, x, tg, uu, i)
        if i == 0:
            op0, x0 = op, x
        else:
            op.destroy()
    t_data = time.perf_counter() - t0
    train_sweeps = np.bincount(train_sweeps).tolist()
    Pf = torch.tensor(np.stack([W.warm_features(p) for p in train]), device="cuda")
    steps, batch = args.train_steps, min(64, ntrain)
    net.init_output_bias(op0, x0)
    sigma_shift = net.calibrate_scale(Pf, tg, uu, 0, min(256, ntrain))
    T.t2s2_trace(True)
    t0 = time.perf_counter()
    losses = []
    for it in range(steps):
        lo = (it * batch) % max(1, ntrain - batch + 1)
        lr = 2e-3 if it < int(0.7 * steps) else 4e-4
        losses.append(net.train_step(Pf, tg, uu, lr, lo=lo, hi=lo + batch))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    mlp = T.t2s2_trace_read("mlp")
    gemm = T.t2s2_trace_read("gemm_tc")
    T.t2s2_trace(False)
    del tg, uu
    hold = [W.config4(90000 + i, d=d, n=n) for i in range(nhold)]
    for p in hold[:2]:  # warm-up
        solve(p)
        solve(p, net)
    cold_t = warm_t = inf_t = 0.0
    sw_c, sw_w = [], []
    conv_c = conv_w = 0
    diffs, r0c, r0w = [], [], []
    for p in hold:
        op, xc, ic, tc, _ = solve(p, r0=r0c)
        _, xw, iw, tw, ti = solve(p, net, r0=r0w)
        cold_t += tc
        warm_t += tw
        inf_t += ti
        sw_c.append(ic.sweeps)
        sw_w.append(iw.sweeps)
        conv_c += ic.residual <= tol
        conv_w += iw.residual <= tol
        diffs.append(T.t2s2_diff_norm(op, xc, xw) / T.t2s2_norm(op, xc))
        op.destroy()
    sw_c, sw_w = np.array(sw_c), np.array(sw_w)
    line = {"metric": "solves/sec to rel. residual 1e-8 with the learned warm start (d=6,n=32 family)",
            "value": conv_w / warm_t, "unit": "solves/s", "n_gpus": 1, "steps": nhold, "warmup": 2,
            "ms_per_step": 1e3 * warm_t / nhold, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 solve, bf16/fp32 network", "data": "synthetic",
            "config": {"workload": f"config-4 family d={d} n={n}: {ntrain} training solves, {nhold} held-out",
                       "cold_solves_per_s": conv_c / cold_t, "warm_rank": rw,
                       "cold_sweeps": int(sw_c.sum()), "warm_sweeps": int(sw_w.sum()),
                       "cold_sweep_histogram": np.bincount(sw_c).tolist(),
                       "warm_sweep_histogram": np.bincount(sw_w).tolist(),
                       "instances_warm_fewer_sweeps": int((sw_w < sw_c).sum()),
                       "instances_warm_more_sweeps": int((sw_w > sw_c).sum()),
                       "inference_ms_per_solve": 1e3 * inf_t / nhold,
                       "cold_converged": conv_c, "warm_converged": conv_w,
                       "initial_residual_median_cold": float(np.median(r0c)),
                       "initial_residual_median_warm": float(np.median(r0w)),
                       "max_rel_diff_cold_vs_warm": max(diffs), "train_steps": steps, "batch": batch,
                       "training_sweep_histogram": train_sweeps,
                       "loss_first": losses[0], "loss_last": float(np.mean(losses[-20:])),
                       "log_scale_calibration": sigma_shift,
                       "data_generation_s": t_data, "training_s": t_train,
                       "mlp_kernels": mlp, "mlp_gemm_tc": gemm,
                       "network": f"15 -> 256 -> 256 -> TT cores rank {rw}, ReLU, Adam"}}
    print(json.dumps(line))
    return 0


def run_stability(args, T, P, W, torch):
    """Stability map of the paper's figure (d=6, beta of ones, b = 1, zero
    data): degrees 8..40 by ratios 1e-1..1e-5, each pixel solved with Plain-SC
    and with superconsistent collocation, all 50 solves in one batched call;
    each pixel classified on its mid-axis line (derivative sign changes,
    total-variation excess)."""
    from paper_2506_04732_gb300 import stability as S
    d, degrees, ratios = 6, (8, 16, 24, 32, 40), (1e-1, 1e-2, 1e-3, 1e-4, 1e-5)
    S.solve_map(T, d, (8,), (1e-1,), workers=args.workers)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pixels, infos = S.solve_map(T, d, degrees, ratios, workers=args.workers)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rows = {}
    for plain in (True, False):
        name = "plain_sc" if plain else "superconsistent"
        rows[name] = {f"N={N}": [f"{pixels[(N, r, plain)]['sign_changes']}:{pixels[(N, r, plain)]['tv_excess']:.2f}"
                                 for r in ratios] for N in degrees}
    macro = {("plain_sc" if pl else "superconsistent"): sum(1 for (N, r, p_), px in pixels.items()
                                                               if p_ == pl and px["tv_excess"] > 0.1)
             for pl in (True, False)}
    conv = sum(1 for inf in infos if inf.residual <= 1e-8)
    line = {"metric": "stability-map pixels/sec (d=6, 25 (degree, ratio) pixels x 2 schemes, one batched call)",
            "value": len(pixels) / dt, "unit": "pixels/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": 1e3 * dt, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "beta=(1,..,1), b=1, zero Dirichlet data, tol 1e-8, rmax 30",
                       "ratios": list(ratios), "degrees": list(degrees),
                       "map_sign_changes_tv_excess": rows, "macroscopic_pixels": macro,
                       "converged": conv, "solves": len(infos)}}
    print(json.dumps(line))
    return 0


def run_contract(args, T, P, W, torch):
    """Grouped core contractions alone: BF16 / TF32 tensor-core and FP64 applies
    of every core of --instances d=5 problems, one persistent launch each."""
    c = measure_contraction(T, P, W, torch, instances=args.instances, reps=max(1, args.steps))
    line = {"metric": "core-contraction TFLOP/s (grouped TT apply, BF16 tensor cores)",
            "value": c["bf16"]["tflops"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": c["bf16"]["ms_per_launch"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 operands, fp32 accumulate, fp64 storage",
            "data": "synthetic", "config": {"workload": c["workload"]}, "contraction": c}
    print(json.dumps(line))
    return 0


def round_counts(m, r_in, r_out):
    """Algorithmic cost of one TT rounding (Methods, TT rounding: right-to-left
    QR orthogonalisation, then left-to-right truncated SVDs), counted for
    Householder QR with the factor Q formed (4 M N^2 - 4 N^3 / 3 for an M x N
    unfolding), an N x N SVD with vectors (12 N^3), and the products that
    carry R, resp. S V^T, into the neighbouring core.  Bytes: the
    orthogonalisation reads and writes every core, the truncation reads it
    again and writes the rounded core: 8 (3 N_in + N_out)."""
    d = len(m)
    fl = 0.0
    r = list(r_in)
    for k in range(d - 1, 0, -1):            # right-to-left QR of core k^T
        M, N = m[k] * r[k + 1], r[k]
        fl += 4 * M * N * N - 4 * N ** 3 / 3
        fl += 2 * r[k - 1] * m[k - 1] * r[k] * r[k]
    ro = list(r_out)
    for k in range(d - 1):                   # left-to-right truncated SVD
        M, N, keep = ro[k] * m[k], r[k + 1], ro[k + 1]
        fl += 4 * M * N * N - 4 * N ** 3 / 3 + 12 * N ** 3 + 2 * M * N * keep
        fl += 2 * keep * N * m[k + 1] * r[k + 2]
    n_in = sum(r_in[k] * m[k] * r_in[k + 1] for k in range(d))
    n_out = sum(r_out[k] * m[k] * r_out[k + 1] for k in range(d))
    return fl, 8.0 * (3 * n_in + n_out), n_in


def run_round(args, T, P, W, torch):
    """TT rounding alone, on the two working sets larger than one core's worth
    of L2 reuse: (a) the Crank-Nicolson right-hand side (M - dt/2 A) u of a
    rank-40 state at d=7, n=64 (rank 80, ~23 MB), rounded to tol 1e-8 and
    rank 40; (b) the 256 batched d=5 instances after an apply of rank-16
    trains (rank 32, ~0.3 GB together), each rounded to tol 1e-8 and rank 16,
    one after another on one stream.  Each timed rounding starts from a fresh
    copy of its input with L2 flushed (256 MB write), both untimed; CUDA
    events on the launching stream bracket the rounding calls."""
    import numpy as np
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    pk, src = peaks()

    def copy_into(dst, src_tt):
        for a, b in zip(dst.buffers, src_tt.buffers):
            a.copy_(b)
        dst.r = list(src_tt.r)

    def timed(pairs):
        """pairs: [(op, y, z, rmax)]: z <- y, flush, then round every z; returns ms."""
        for op, y, z, _ in pairs:
            copy_into(z, y)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for op, y, z, rmax in pairs:
            T.t2s2_round(op, z, 1e-8, rmax)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def measure(name, pairs, workload):
        for _ in range(args.warmup):
            timed(pairs)
        ms = [timed(pairs) for _ in range(args.steps)]
        ms_mean = sum(ms) / len(ms)
        fl = by = n_in = 0.0
        for op, y, z, _ in pairs:
            f, b, n = round_counts(z.m, y.r, z.r)
            fl, by, n_in = fl + f, by + b, n_in + n
        gbs = by / (ms_mean * 1e-3) / 1e9
        gfl = fl / (ms_mean * 1e-3) / 1e9
        t_hbm = by / (pk["hbm_gbs"] * 1e9) * 1e3
        t_alu = fl / (FP64_ALU_PEAK_GFLOPS * 1e9) * 1e3
        return {"workload": workload, "roundings": len(pairs), "ms": ms_mean, "ms_runs": ms,
                "input_bytes": 8 * n_in, "algorithmic_bytes": by, "fp64_flops": fl,
                "hbm_gbs": gbs, "hbm_frac": gbs / pk["hbm_gbs"], "fp64_gflops": gfl,
                "fp64_frac": gfl / FP64_ALU_PEAK_GFLOPS,
                "roofline_ms": max(t_hbm, t_alu), "bound": "fp64 alu" if t_alu > t_hbm else "hbm",
                "roofline_frac": max(t_hbm, t_alu) / ms_mean,
                "ranks_in": list(pairs[0][1].r), "ranks_out": list(pairs[0][2].r)}

    out = {}
    # (a) the Crank-Nicolson right-hand side of a rank-40 state
    p2 = W.config2()
    op2 = P.build_operator(p2)
    m2 = [n - 2 for n in p2.n]
    r40 = [1] + [p2.rmax] * (p2.d - 1) + [1]
    u = T.TT.from_cores(W.random_tt(p2.d, m2[0], r40, seed=911), rcap=p2.rmax)
    y2 = T.TT.empty(m2, 2 * p2.rmax)
    T.t2s2_apply(op2, u, y2, 1.0, -0.5 * p2.dt)
    z2 = T.TT.empty(m2, 2 * p2.rmax)
    out["cn_rhs"] = measure("cn_rhs", [(op2, y2, z2, p2.rmax)],
                            f"(M - dt/2 A) u, d={p2.d} n={p2.n[0]}, u random rank {p2.rmax}: rank "
                            f"{2 * p2.rmax} -> {p2.rmax}")
    del op2, u, y2, z2
    # (b) the 256 batched instances after an apply
    ops, pairs = [], []
    for i in range(args.instances):
        p = W.config3(i)
        m = [n - 2 for n in p.n]
        op = P.build_operator(p)
        r = [1] + [16] * (p.d - 1) + [1]
        x = T.TT.from_cores(W.random_tt(p.d, m[0], r, seed=700 + i))
        y = T.TT.empty(m, 32)
        T.t2s2_apply(op, x, y, 0.0, 1.0)
        z = T.TT.empty(m, 32)
        ops.append(op)
        pairs.append((op, y, z, 16))
    if pairs:
        out["batched"] = measure("batched", pairs, f"{args.instances} instances d=5 n in {{16,24,32,48}}, "
                                                   "A x of random rank-16 x: rank 32 -> 16, one stream")
    a = out["cn_rhs"]
    line = {"metric": "TT roundings/sec (Crank-Nicolson right-hand side, d=7, n=64, rank 80 -> 40)",
            "value": 1e3 / a["ms"], "unit": "roundings/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": a["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": a["workload"], "l2": "flushed before every timed rounding (256 MB write)"},
            "rounding": out, "hbm_peak_gbs": pk["hbm_gbs"], "peak_source": src,
            "fp64_peak_gflops": FP64_ALU_PEAK_GFLOPS,
            "fp64_peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 1.965 GHz"}
    print(json.dumps(line))
    return 0


def measure_contraction(T, P, W, torch, instances=256, reps=10):
    """Grouped core contractions (t2s2_apply_batched): every core of `instances`
    d=5 problems (n in {16,24,32,48}, TT ranks 16) in one persistent launch.
    Kernel time from the library's per-launch CUDA events; algorithmic FLOPs
    4 m^2 r_a r_b and bytes 8 (r_a m r_b (1 + blocks written) + 2 m^2) per core."""
    import numpy as np
    probs = [W.config3(i) for i in range(instances)]
    ops, xs, ys = [], [], []
    for i, p in enumerate(probs):
        m = p.n[0] - 2
        r = [1] + [16] * (p.d - 1) + [1]
        ops.append(P.build_operator(p))
        xs.append(T.TT.from_cores(W.random_tt(p.d, m, r, seed=700 + i)))
        ys.append(T.TT.empty([m] * p.d, 32))
    pk, src = peaks()
    out = {"workload": f"{instances} instances d=5 n in {{16,24,32,48}}, ranks 16, one launch per apply",
           "data_bytes": int(sum(8 * sum(c.numel() for c in x.buffers) for x in xs)
                             + sum(8 * sum(c.numel() for c in y.buffers) for y in ys))}
    for name, prec in (("bf16", T.BF16_REFINE), ("tf32", T.TF32_REFINE), ("fp64", T.FP64)):
        T.t2s2_apply_batched(ops, xs, ys, 0.0, 1.0, prec)  # tunes the launch shape
        T.t2s2_apply_batched(ops, xs, ys, 0.0, 1.0, prec)
        torch.cuda.synchronize()
        T.t2s2_trace(True)
        for _ in range(reps):
            T.t2s2_apply_batched(ops, xs, ys, 0.0, 1.0, prec)
        fam = T.t2s2_trace_read("apply" if name == "fp64" else "apply_tc")
        T.t2s2_trace(False)
        ms = fam["ms"] / max(1, fam["launches"])
        tf = fam["flops"] / max(1, fam["launches"]) / (ms * 1e-3) / 1e12
        gbs = fam["bytes"] / max(1, fam["launches"]) / (ms * 1e-3) / 1e9
        e = {"ms_per_launch": ms, "tflops": tf, "hbm_gbs": gbs, "hbm_frac": gbs / pk["hbm_gbs"],
             "flops_per_launch": fam["flops"] / max(1, fam["launches"]),
             "bytes_per_launch": fam["bytes"] / max(1, fam["launches"])}
        if name == "bf16":
            e["tensor_peak_tflops"] = pk["bf16_tflops"]
            e["tensor_frac"] = tf / pk["bf16_tflops"]
        elif name == "tf32":
            e["tensor_peak_tflops"] = pk["bf16_tflops"] / 2  # dense TF32 is half the BF16 rate
            e["tensor_frac"] = tf / e["tensor_peak_tflops"]
        out[name] = e
    out["autotune"] = T.t2s2_autotune_report().strip().splitlines()
    out["bound"] = "hbm: arithmetic intensity m/10 flop/byte (<= 4.6 at m = 46) is far below the tensor ridge"
    out["peak_source"] = src
    return out


def measure_precisions(T, P, W, torch, op, b, x_ref, steps=3):
    """Mixed-precision solves (FP64 iterative refinement) of the same problem:
    solves/s, FP64 residual, sweeps, refinements and distance to the FP64
    solution ||x - x_fp64|| / ||x_fp64|| (t2s2_diff_norm)."""
    import numpy as np
    p = W.config1()
    m = [n - 2 for n in p.n]
    ref_norm = T.t2s2_norm(op, x_ref)
    out = {}
    for name, prec in (("fp32_refine", T.FP32_REFINE), ("tf32_refine", T.TF32_REFINE),
                       ("bf16_refine", T.BF16_REFINE)):
        times, info, x = [], None, None
        for i in range(steps + 1):
            x = T.TT.from_cores([np.ones((1, mm, 1)) for mm in m], rcap=p.rmax + T.RANK_KICK)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = T.t2s2_solve(op, b, x, p.tol, p.rmax, p.max_sweeps, prec=prec, allow_noconv=True)
            torch.cuda.synchronize()
            if i > 0:
                times.append(time.perf_counter() - t0)
        out[name] = {"solves_per_s": len(times) / sum(times), "residual": info.residual,
                     "converged": info.residual <= p.tol, "sweeps": info.sweeps,
                     "refinements": info.refinements, "max_rank": info.max_rank,
                     "rel_diff_vs_fp64_solution": T.t2s2_diff_norm(op, x, x_ref) / ref_norm}
    return out


def main():
    args = parse()
    if args.steps is None:
        if args.impl == "ours" and args.workload == "steady":
            args.steps = 200
        elif args.impl == "ours" and args.workload == "cn":
            args.steps = 100   # the workload's trajectory
        else:
            args.steps = 5
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "steady":
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__ as g
        g.build()
        import paper_2506_04732_gb300 as T
        from paper_2506_04732_gb300 import problem as P
        import workloads as W
        fn = {"batched": run_batched, "cn": run_cn, "warm": run_warm, "contract": run_contract,
              "spacetime": run_spacetime, "stability": run_stability, "round": run_round}[args.workload]
        return fn(args, T, P, W, torch)
    ws, rank, local = dist_env()
    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__ as g
    if rank == 0 or ws == 1:
        g.build()
    if ws > 1:
        torch.distributed.barrier()
        g.build()
    import numpy as np
    import paper_2506_04732_gb300 as T
    from paper_2506_04732_gb300 import problem as P
    import workloads as W

    prec = {"fp64": T.FP64, "fp32": T.FP32_REFINE, "tf32": T.TF32_REFINE, "bf16": T.BF16_REFINE}[args.prec]
    p = W.config1()
    stream = torch.cuda.current_stream()
    op = P.build_operator(p)
    bcores = P.source_cores(p, op)
    b = T.TT.from_cores(bcores)
    m = [n - 2 for n in p.n]
    x0 = [np.ones((1, mm, 1)) for mm in m]
    rcap = p.rmax + T.RANK_KICK
    x = T.TT.from_cores(x0, rcap=rcap)
    x_init = [buf.clone() for buf in x.buffers]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    def reset_x():
        for dst, src in zip(x.buffers, x_init):
            dst.copy_(src)
        x.r = [1] * (p.d + 1)

    infos = []
    for _ in range(args.warmup):
        reset_x()
        infos.append(T.t2s2_solve(op, b, x, p.tol, p.rmax, p.max_sweeps, prec=prec))
    torch.cuda.synchronize()
    lib = T.load()
    launches0 = lib.t2s2_kernel_launches()
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()                      # evict L2 between timed steps (untimed)
        reset_x()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = T.t2s2_solve(op, b, x, p.tol, p.rmax, p.max_sweeps, prec=prec)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        infos.append(info)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = lib.t2s2_kernel_launches() - launches0
    # per-family kernel times come from one more solve, untimed, with a CUDA
    # event pair around every launch (the events would slow the timed steps)
    flush.zero_()
    reset_x()
    torch.cuda.synchronize()
    T.t2s2_trace(True)
    T.t2s2_solve(op, b, x, p.tol, p.rmax, p.max_sweeps, prec=prec)
    torch.cuda.synchronize()
    fam = {name: T.t2s2_trace_read(name) for name in FAMILIES}
    T.t2s2_trace(False)
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms)
    value = replica_rate(ws, args.steps, total_ms / 1e3)
    last = infos[-1]

    # end to end through the C ABI with host buffers (copies inside the call)
    e2e = None
    if not args.no_e2e:
        bh = T.TT.from_cores(bcores, device="cpu")
        xh = T.TT.from_cores(x0, rcap=rcap, device="cpu")
        xh_init = [buf.clone() for buf in xh.buffers]
        h2d = sum(8 * int(np.prod(c.shape)) for c in bcores) + sum(8 * int(np.prod(c.shape)) for c in x0)
        d2h = 0
        tt = 0.0
        for _ in range(args.steps):
            flush.zero_()
            for dst, src in zip(xh.buffers, xh_init):
                dst.copy_(src)
            xh.r = [1] * (p.d + 1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            T.t2s2_solve(op, bh, xh, p.tol, p.rmax, p.max_sweeps, prec=prec)
            torch.cuda.synchronize()
            tt += time.perf_counter() - t0
            d2h = sum(8 * xh.r[k] * xh.m[k] * xh.r[k + 1] for k in range(xh.d))
        tt = max_over_ranks(tt)
        e2e = {"value": replica_rate(ws, args.steps, tt), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    extras = {}
    if rank == 0 and ws == 1 and args.prec == "fp64" and not args.no_extras:
        for key, fn in (("precision_variants", lambda: measure_precisions(T, P, W, torch, op, b, x)),
                        ("contraction", lambda: measure_contraction(T, P, W, torch))):
            try:
                extras[key] = fn()
            except Exception as exc:  # recorded, never hides the headline number
                extras[key] = {"error": repr(exc)}

    # The dominant kernel by device time: per-kernel device durations of one
    # more solve from CUPTI activity records (no events between launches);
    # the event trace above then gives that family's time per launch (events
    # around each launch include its launch gap, so `achieved` is a lower bound)
    flush.zero_()
    reset_x()
    torch.cuda.synchronize()
    dev = kernel_device_times(lambda: T.t2s2_solve(op, b, x, p.tol, p.rmax, p.max_sweeps, prec=prec), torch)
    cupti_error = dev.pop("__error__", (0, 0.0, None))[2] if dev else "no kernel records"
    pk, src = peaks()
    if dev:
        by_fam = {}
        for name, (cnt, us) in dev.items():
            by_fam[kernel_family(name)] = by_fam.get(kernel_family(name), 0.0) + us
        by_fam.pop("other", None)
        dom_src = "device time per kernel family of one solve (CUPTI activity records)"
    else:
        # per-family event time less what the brackets cost a launch (an
        # empty launch measured the same way), so that families of many short
        # launches are not ranked by their launch gaps
        ovh = T.t2s2_trace_overhead(200)
        by_fam = {k: 1e3 * max(0.0, v["ms"] - v["launches"] * ovh) for k, v in fam.items() if v["launches"]}
        dom_src = (f"event-traced time per family less {1e3 * ovh:.2f} us of bracket cost per launch "
                   f"(CUPTI records unavailable: {cupti_error})")
    total_us = sum(by_fam.values())
    dom = max(by_fam, key=by_fam.get)
    share = {k: round(v / total_us, 4) for k, v in sorted(by_fam.items(), key=lambda kv: -kv[1])}
    fd = fam[dom]
    if dom in ALU_FAMILIES:
        bound, peak, unit = "alu", FP64_ALU_PEAK_GFLOPS / 1e3, "TFLOP/s"
        achieved = fd["flops"] / (fd["ms"] / 1e3) / 1e12 if fd["ms"] > 0 else 0.0
        peak_src = "derived: 2 DFMA/clk/SM x 152 SMs x 1.965 GHz (FP64 ALU)"
    else:
        bound, peak, unit = "hbm", pk["hbm_gbs"], "GB/s"
        achieved = fd["bytes"] / (fd["ms"] / 1e3) / 1e9 if fd["ms"] > 0 else 0.0
        peak_src = f"{src} hbm_gbs"
    traffic = KERNEL_DRAM_BYTES.get(dom)
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak if peak else None,
            "traffic": traffic[0] if traffic else None,
            "traffic_source": traffic[1] if traffic else None,
            "kernel": dom, "kernel_choice": dom_src, "device_time_share": share,
            "peak_source": peak_src,
            "flops_per_launch": fd["flops"] / max(1, fd["launches"]),
            "per_launch_ms": fd["ms"] / max(1, fd["launches"]),
            "achieved_note": "event time per launch includes the launch's bracket cost: a lower bound"}

    cpu = None
    if rank == 0 and args.cpu_budget > 0:
        rate, sample = cpu_baseline_sample("config1()", args.cpu_budget, p.tol)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else args.prec,
                "data": "synthetic",
                "config": {"workload": p.name, "d": p.d, "n": p.n[0], "tol": p.tol, "rmax": p.rmax,
                           "precision": args.prec, "parallelism": f"replicas{ws}",
                           "l2": "flushed between timed steps (256 MB write)",
                           "residual": last.residual, "sweeps": last.sweeps, "max_rank": last.max_rank,
                           "local_iters": last.local_iters},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "kernel_families": fam}
        line.update(extras)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
