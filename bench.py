#!/usr/bin/env python
"""Benchmark of the batched three-phase Z-bus power flow on GB300.

Metric: converged scenario-solves per second.  A scenario-solve counts when
the solver flags it converged at tol 1e-8 pu and its FP64 power mismatch
(computed by the library with the sparse admittance matrix) is <= 1e-6 pu;
the CPU-baseline leg additionally checks a sample against the FP64 oracle
(max |dV| <= 1e-6 pu, identical flags).

One step = one zbus_solve of the whole scenario batch (run start, then the
device-resident sweep loop: load currents, contraction, update, convergence),
inputs resident in HBM, L2 flushed between steps (a 512 MiB write, outside the
timed events).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank solves its own batch (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "converged scenario-solves/s at |dV|<=1e-6 pu vs plain FP64 GPU; p50/p99 latency"
UNIT = "scenario-solves/s"
FP64_PEAK_TFLOPS = 1.25     # nominal GB300 FP64 (152 SMs x 2 DFMA/clk x 2 flop x ~2.07 GHz)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="feeder128_b4096")
    p.add_argument("--precision", default="fp64")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# the oracle legs (CPU)
# ---------------------------------------------------------------------------
def oracle_setup(f):
    from oracle import zbus_oracle as O
    Y = O.dense_from_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val)
    Y_LL, Y_Ls, _ = O.partition(Y, f.slack_idx)
    Z, w = O.reduced_impedance(Y_LL, Y_Ls, f.v_slack)
    return Z, w


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_baseline(f, Sw, Sd, wl, seconds, V_gpu, it_gpu, cv_gpu):
    """The oracle as it stands, timed on this host on a bounded sample of the batch."""
    import numpy as np
    from oracle import zbus_oracle as O
    Z, w = oracle_setup(f)
    B = Sw.shape[0]
    bs = min(B, 1024)
    reps, solved, t_total = 0, 0, 0.0
    first = None
    while t_total < seconds or reps == 0:
        lo = (reps * bs) % B
        idx = np.arange(lo, min(B, lo + bs))
        t0 = time.perf_counter()
        V, it, cv = O.fixed_point(Z, w, Sw[idx], Sd[idx], wl.tol, wl.max_iter)
        t_total += time.perf_counter() - t0
        solved += int(cv.sum())
        if first is None:
            first = (idx, V, it, cv)
        reps += 1
        if reps * bs >= 4 * B:
            break
    idx, V, it, cv = first
    m = cv == 1
    dv = float(np.abs(V_gpu[idx][m] - V[m]).max()) if m.any() else 0.0
    parity = {"sampled": int(idx.size), "max_dv_vs_oracle": dv,
              "flags_equal": bool(np.array_equal(cv_gpu[idx], cv)),
              "iters_equal": bool(np.array_equal(it_gpu[idx], it))}
    return ({"value": solved / t_total, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
             "sample": f"{reps} x {bs} scenarios of the {B}-scenario batch "
                       f"({solved} solves, {t_total:.1f} s, setup excluded)"}, parity)


def run_reference(args):
    """The oracle (numpy FP64) as the reference arm, on the host cores."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import zbus_oracle as O
    from paper_2605_14103_gb300 import feeders as F
    f, Sw, Sd, wl = F.make_workload(args.workload)
    Z, w = oracle_setup(f)
    bs = min(wl.B, 512)
    for s in range(args.warmup):
        O.fixed_point(Z, w, Sw[:bs], Sd[:bs], wl.tol, wl.max_iter)
    times, solved = [], 0
    for s in range(args.steps):
        lo = (s * bs) % wl.B
        t0 = time.perf_counter()
        V, it, cv = O.fixed_point(Z, w, Sw[lo:lo + bs], Sd[lo:lo + bs], wl.tol, wl.max_iter)
        times.append(time.perf_counter() - t0)
        solved += int(cv.sum())
    total = sum(times)
    value = solved / total
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "feeder_buses": wl.N, "unknowns": 3 * (wl.N - 1),
                      "scenarios_per_step": bs, "tol": wl.tol},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                            "sample": f"{bs} scenarios of the {wl.B}-scenario batch per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_setup()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_14103_gb300 import feeders as F
    from paper_2605_14103_gb300 import zbus

    torch.cuda.set_device(local)
    f, _, _, wl = F.make_workload(args.workload, B=1)
    Sw_h, Sd_h = F.make_scenarios(f, wl.B, wl.mult[0], wl.mult[1], seed=f.seed + 1 + 7919 * rank)
    B, n = Sw_h.shape
    Sw = torch.from_numpy(Sw_h).cuda()
    Sd = torch.from_numpy(Sd_h).cuda()
    net = zbus.Network.from_feeder(f)
    net.reserve(B, args.precision)
    V = torch.empty((B, n), dtype=torch.complex128, device="cuda")
    it = torch.empty((B,), dtype=torch.int32, device="cuda")
    cv = torch.empty((B,), dtype=torch.uint8, device="cuda")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def solve(profile=False):
        net.solve(Sw, Sd, tol=wl.tol, max_iter=wl.max_iter, precision=args.precision,
                  profile=profile, out=(V, it, cv))

    for _ in range(max(3, args.warmup)):
        solve()
    torch.cuda.synchronize()

    # ---- timed region: K solves through the device-resident loop ----
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record()
        solve()
        evs[k][1].record()
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - t0
    clk = clocks.stop() if clocks else None
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_dev = sum(step_ms) / 1e3

    # ---- what was solved ----
    mm = net.power_mismatch(V, Sw, Sd)
    ok = (cv == 1) & (mm <= 1e-6)
    good = int(ok.sum().item())
    max_iters = int(it.max().item())
    sweeps_total = int(it.sum().item())
    t_max = allreduce_max(t_dev, ws)
    good_all = allreduce_sum(good, ws)
    value = good_all * args.steps / t_max
    launches = args.steps * (1 + 3 * max_iters)

    # ---- roofline of the contraction: profiled pass, events around each launch ----
    prof_steps = min(args.steps, 3)
    g_ms, g_flops = 0.0, 0.0
    for _ in range(prof_steps):
        flush.zero_()
        solve(profile=True)
        torch.cuda.synchronize()
        ms, act = net.last_profile(wl.max_iter)
        for k in range(len(act)):
            if act[k] > 0:
                g_ms += float(ms[k, 1])
                g_flops += 8.0 * n * n * float(act[k])
    achieved = g_flops / (g_ms / 1e3) / 1e12 if g_ms > 0 else 0.0
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": None, "kernel": "k_gemm3m_f64",
                "note": "FP64 pipe; algorithmic 8 n^2 flop per scenario-sweep; peak is nominal "
                        "FP64 (DFMA probe measured 1.197 TFLOP/s)"}

    # ---- end to end through the public API, host buffers ----
    Sw_p = torch.from_numpy(Sw_h).pin_memory()
    Sd_p = torch.from_numpy(Sd_h).pin_memory()
    V_p = torch.empty((B, n), dtype=torch.complex128).pin_memory()
    it_p = torch.empty((B,), dtype=torch.int32).pin_memory()
    cv_p = torch.empty((B,), dtype=torch.uint8).pin_memory()
    e2e_steps = args.steps
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(e2e_steps)]
    e2e_good = 0
    for k in range(e2e_steps):
        flush.zero_()
        ev2[k][0].record()
        Sw.copy_(Sw_p, non_blocking=True)
        Sd.copy_(Sd_p, non_blocking=True)
        solve()
        V_p.copy_(V, non_blocking=True)
        it_p.copy_(it, non_blocking=True)
        cv_p.copy_(cv, non_blocking=True)
        ev2[k][1].record()
        torch.cuda.synchronize()
        e2e_good += int(cv_p.numpy().sum())
    e2e_t = allreduce_max(sum(a.elapsed_time(b) for a, b in ev2) / 1e3, ws)
    e2e_val = allreduce_sum(e2e_good, ws) / e2e_t
    h2d = 2 * B * n * 16
    d2h = B * n * 16 + B * 4 + B

    # ---- CPU baseline (rank 0, one GPU) ----
    cpu, parity = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, parity = cpu_baseline(f, Sw_h, Sd_h, wl, args.cpu_seconds, V.cpu().numpy(),
                                   it.cpu().numpy(), cv.cpu().numpy())

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if args.precision == "fp64" else args.precision + "+f64",
               "data": "synthetic",
               "config": {"workload": args.workload, "feeder_buses": wl.N, "unknowns": n,
                          "scenarios_per_gpu": B, "tol": wl.tol, "max_iter": wl.max_iter,
                          "precision": args.precision, "l2": "flushed between steps (512 MiB write)",
                          "parallelism": f"replicas x{ws}"},
               "converged_per_step": good, "max_iters": max_iters,
               "mean_iters": sweeps_total / B,
               "step_ms": {"p50": statistics.median(step_ms), "max": max(step_ms),
                           "wall_s_incl_flush": wall},
               "gpu_launches": launches,
               "roofline": roofline,
               "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h},
               "clocks": clk, "cpu_baseline": cpu, "parity": parity}
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
