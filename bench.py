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
FAMILIES = ["gemm", "apply", "local_solve", "small_factor", "elementwise", "apply_tc", "gemm_tc", "mlp"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of oracle CPU work for the cpu_baseline sample")
    ap.add_argument("--workload", default="steady", choices=["steady", "batched", "cn"],
                    help="steady: d=6 n=32 solve (headline); batched: 256 d=5 instances; "
                         "cn: Crank-Nicolson steps at d=7 n=64")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--workers", type=int, default=8)
    return ap.parse_args()


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

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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


_ORACLE_CHILD = r"""
import sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import operator as O
from oracle import solve as S
p = W.{cfg}
ops = O.build(p)
A = O.ttm_cores(ops)
b = O.source_tt(p, ops)
x = [np.ones((1, n - 2, 1)) for n in p.n]
t0 = time.perf_counter()
for k in range(p.max_sweeps):
    x, res, _ = S.amen_solve(A, b, x, p.tol, p.rmax, max_sweeps=1)
    print(json.dumps({{"sweeps": k + 1, "t": time.perf_counter() - t0, "res": res}}), flush=True)
    if res <= p.tol:
        break
"""


def cpu_baseline_sample(problem_expr, budget_s):
    """Time the FP64 oracle's solve on the host cores, bounded by a hard budget.

    The oracle runs sweep by sweep in a child process that is stopped once the
    budget is spent; the sample is the sweeps completed by then.  The rate per
    solve scales completed sweeps by the sweeps a solve needs -- optimistic for
    the oracle, whose later sweeps (higher ranks) are its most expensive.
    Returns (seconds, sweeps done, converged, last residual).
    """
    import subprocess as sp
    code = _ORACLE_CHILD.format(root=ROOT, cfg=problem_expr)
    t0 = time.perf_counter()
    proc = sp.Popen([sys.executable, "-c", code], stdout=sp.PIPE, stderr=sp.DEVNULL, text=True)
    last = None
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
    for ln in lines:
        try:
            last = json.loads(ln)
        except ValueError:
            pass
    if not last:
        return time.perf_counter() - t0, 0, False, None
    return last["t"], last["sweeps"], last["res"] <= 1e-8, last["res"]


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import workloads as W
    p = W.config1()
    times = []
    info = None
    for i in range(args.warmup + args.steps):
        dt, sweeps, conv, res = cpu_baseline_sample("config1()", args.cpu_budget / max(1, args.steps))
        if i >= args.warmup:
            times.append((dt, sweeps, conv, res))
        info = (dt, sweeps, conv, res)
    # rate: solves/sec, a partial solve counted as sweeps_done / sweeps_needed
    need = SWEEPS_NEEDED_HINT
    tot = sum(t[0] for t in times)
    solves = sum(min(1.0, t[1] / need) for t in times)
    value = solves / tot if tot > 0 else 0.0
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value if value else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": p.name, "d": p.d, "n": p.n[0], "tol": p.tol,
                                             "rmax": p.rmax},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"oracle AMEn sweeps within {args.cpu_budget / max(1, args.steps):.0f} s "
                                       f"per step, scaled by {need} sweeps per solve"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# Sweeps the oracle's alternating solver needs on the d=6, n=32 problem to
# reach 1e-8 (measured with the oracle itself; used to scale a partial sample).
SWEEPS_NEEDED_HINT = 7


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
        return [T.TT.from_cores(c, rcap=20) for c in xs0]

    for _ in range(max(1, args.warmup)):
        T.t2s2_solve_batched(ops, bs, fresh(), 1e-8, 16, 50, workers=args.workers, allow_noconv=True)
    torch.cuda.synchronize()
    times, infos = [], None
    for _ in range(args.steps):
        xs = fresh()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = T.t2s2_solve_batched(ops, bs, xs, 1e-8, 16, 50, workers=args.workers, allow_noconv=True)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    batched = args.instances * len(times) / sum(times)
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
                       "workers": args.workers, "converged": conv,
                       "max_sweeps": max(inf.sweeps for inf in infos),
                       "sequential_solves_per_s": seq, "sequential_sample": nseq}}
    print(json.dumps(line))
    return 0


def run_cn(args, T, P, W, torch):
    """Crank-Nicolson steps of the d=7, n=64 Gaussian pulse (dt = 1e-3, rmax 40, tol 1e-8)."""
    p = W.config2()
    op = P.build_operator(p)
    u = T.TT.from_cores(P.solution_cores(p, op), rcap=p.rmax + 4)
    infos = []
    for _ in range(args.warmup):
        infos.append(T.t2s2_cn_step(op, u, p.dt, p.tol, p.rmax))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        infos.append(T.t2s2_cn_step(op, u, p.dt, p.tol, p.rmax))
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    line = {"metric": "Crank-Nicolson steps/sec (d=7, n=64, dt=1e-3, tol 1e-8)", "value": 1e3 / ms,
            "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": p.name, "rmax": p.rmax, "ranks": u.r,
                       "step_residuals": [inf.residual for inf in infos],
                       "sweeps": [inf.sweeps for inf in infos]}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
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
        return (run_batched if args.workload == "batched" else run_cn)(args, T, P, W, torch)
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
    rcap = p.rmax + 4
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
    T.load().t2s2_trace(1)
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
    import ctypes
    fam = {}
    for i, name in enumerate(FAMILIES):
        n_l = ctypes.c_longlong()
        ms = ctypes.c_double()
        fl = ctypes.c_double()
        by = ctypes.c_double()
        lib.t2s2_trace_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]
        lib.t2s2_trace_read(i, ctypes.byref(n_l), ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(by))
        fam[name] = {"launches": n_l.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}
    lib.t2s2_trace(0)
    total_ms = sum(step_ms)
    if ws > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = ws * args.steps / (total_ms / 1e3)
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
        e2e = {"value": ws * args.steps / tt, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # roofline of the dominant kernel family (largest share of traced time)
    pk, src = peaks()
    dom = max(fam, key=lambda k: fam[k]["ms"])
    fd = fam[dom]
    if dom in ("gemm", "apply", "local_solve", "small_factor"):
        bound, peak, unit = "alu", FP64_ALU_PEAK_GFLOPS / 1e3, "TFLOP/s"
        achieved = fd["flops"] / (fd["ms"] / 1e3) / 1e12 if fd["ms"] > 0 else 0.0
        peak_src = "derived: 2 DFMA/clk/SM x 152 SMs x 1.965 GHz"
    else:
        bound, peak, unit = "hbm", pk["hbm_gbs"], "GB/s"
        achieved = fd["bytes"] / (fd["ms"] / 1e3) / 1e9 if fd["ms"] > 0 else 0.0
        peak_src = f"{src} hbm_gbs"
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak if peak else None, "traffic": None, "kernel": dom,
            "peak_source": peak_src,
            "per_launch_ms": fd["ms"] / max(1, fd["launches"])}

    cpu = None
    if rank == 0:
        dt, sweeps, conv, res = cpu_baseline_sample("config1()", args.cpu_budget)
        solves = min(1.0, sweeps / SWEEPS_NEEDED_HINT) if not conv else 1.0
        cpu = {"value": solves / dt if dt > 0 and sweeps else 0.0, "unit": UNIT, "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"{sweeps} oracle AMEn sweeps completed within a {args.cpu_budget:.0f} s budget "
                         f"({dt:.1f} s)"
                         f"{' (converged)' if conv else f'; rate scaled by {SWEEPS_NEEDED_HINT} sweeps per solve'}"}
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
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
