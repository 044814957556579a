#!/usr/bin/env python
"""Benchmark of the batched three-phase Z-bus power flow on GB300.

Metric: converged scenario-solves per second.  A scenario-solve counts when
the solver flags it converged at tol 1e-8 pu and its FP64 power mismatch
(computed by the library with the sparse admittance matrix) is <= 1e-6 pu;
the CPU-baseline leg additionally checks a sample against the FP64 oracle
(max |dV| <= 1e-6 pu, identical flags).

One step = one zbus_solve of the whole scenario batch (run start, then the
device-resident sweep loop: residual / load currents, contraction, update,
convergence; then the FP64 mismatch test and correction of the mixed forms),
inputs resident in HBM, L2 flushed between steps (a 512 MiB write, outside the
timed events).

The default run is the 1024-bus feeder (3069 unknowns, dense complex Z) with
16384 scenarios in the FP16 row-scaled tensor-core form; the same line carries
the BF16 hi+lo and tree forms and the plain FP64 method (with each form's
ratio to it and its parity against the oracle on a 512-scenario sample), and
compact results of the other workloads: the 13-bus latency case, the 128-bus
plain-method case, 64 heterogeneous feeders batched, the 16-feeder serving
loop, load gradients and the Newton-Raphson transmission solver.

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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "converged scenario-solves/s at |dV|<=1e-6 pu vs plain FP64 GPU; p50/p99 latency"
UNIT = "scenario-solves/s"
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (152 SMs x 2 DFMA/clk x 2 flop x ~2.07 GHz): context
DEFAULT_WORKLOAD = "feeder1024_b16384"
DEFAULT_PRECISION = "fp16_scaled"
PARITY_SAMPLE = 512          # scenarios of the batch checked against the oracle, every form


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--precision", default=DEFAULT_PRECISION)
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--forms", default="all", choices=["all", "one"])
    p.add_argument("--batch", type=int, default=0, help="override the scenario count")
    p.add_argument("--requests", type=int, default=2000, help="serving: requests per run")
    p.add_argument("--no-extras", action="store_true",
                   help="default workload: leave out the compact results of the other workloads")
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
    from paper_2605_14103_gb300 import dist as D
    return D.reduce_max(x, device="cuda") if ws > 1 else x


def allreduce_sum(x, ws):
    from paper_2605_14103_gb300 import dist as D
    return D.reduce_sum(x, device="cuda") if ws > 1 else x


# ---------------------------------------------------------------------------
# the oracle legs (CPU)
# ---------------------------------------------------------------------------
def oracle_setup(f):
    """(Z, w, bus_phase of the load unknowns or None) of the oracle."""
    import numpy as np
    from oracle import zbus_oracle as O
    Y = O.dense_from_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val)
    Y_LL, Y_Ls, load_idx = O.partition(Y, f.slack_idx)
    Z, w = O.reduced_impedance(Y_LL, Y_Ls, f.v_slack)
    bp = getattr(f, "bus_phase", None)
    return Z, w, (None if bp is None else np.asarray(bp)[load_idx])


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def oracle_sample(f, Sw, Sd, wl, seconds):
    """The oracle as it stands, on this host's cores: the first PARITY_SAMPLE
    scenarios of the batch (the parity sample of every form), then further
    1024-scenario chunks until about `seconds` of CPU work (the CPU baseline).
    Returns ((V, iters, converged) of the parity sample, cpu_baseline)."""
    from oracle import zbus_oracle as O
    Z, w, bp = oracle_setup(f)
    B = Sw.shape[0]
    bs = min(B, PARITY_SAMPLE)
    t0 = time.perf_counter()
    V, it, cv = O.fixed_point(Z, w, Sw[:bs], Sd[:bs], wl.tol, wl.max_iter, bus_phase=bp)
    t_total = time.perf_counter() - t0
    solved, n_sc, chunks = int(cv.sum()), bs, 1
    lo = bs
    while t_total < seconds and lo < B:
        hi = min(B, lo + 1024)
        t0 = time.perf_counter()
        _, _, c = O.fixed_point(Z, w, Sw[lo:hi], Sd[lo:hi], wl.tol, wl.max_iter, bus_phase=bp)
        t_total += time.perf_counter() - t0
        solved += int(c.sum())
        n_sc += hi - lo
        chunks += 1
        lo = hi
    cpu = {"value": solved / t_total, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
           "sample": f"first {n_sc} scenarios of the {B}-scenario batch in {chunks} chunks "
                     f"({solved} converged solves, {t_total:.1f} s, setup excluded)"}
    return (V, it, cv), cpu


def parity_vs_oracle(ref, out, form):
    """Per-scenario comparison of one form's sample with the oracle's: flags
    equal, max |dV| on converged scenarios, iteration counts equal (FP64) or
    within one (defect forms)."""
    Vr, itr, cvr = ref
    V, it, cv = out
    m = cvr == 1
    dv = float(np.abs(V[m] - Vr[m]).max()) if m.any() else 0.0
    dit = int(np.abs(it[m].astype(np.int64) - itr[m]).max()) if m.any() else 0
    return {"sampled": int(cvr.size), "max_dv_vs_oracle": dv,
            "flags_equal": bool(np.array_equal(cv, cvr)),
            "max_iter_diff": dit, "ok": bool(np.array_equal(cv, cvr) and dv <= 1e-6 and
                                             (dit == 0 if form == "fp64" else dit <= 1))}


def feeder_config(workload, wl, n, B, precision, ws, phased=False):
    """The `config` of a feeder workload's line, the same in both arms."""
    cfg = {"workload": workload, "feeder_buses": wl.N, "unknowns": n,
           "scenarios_per_gpu": B, "tol": wl.tol, "max_iter": wl.max_iter,
           "precision": precision, "l2": "flushed between steps (512 MiB write)",
           "parallelism": f"replicas x{ws}"}
    if phased:
        # the device solves the network padded to three phase slots per bus
        cfg["padded_unknowns"] = 3 * (wl.N - 1)
    return cfg


def grid_config(workload, g, wl, B, precision, ws):
    """The `config` of a Newton-Raphson workload's line, the same in both arms."""
    return {"workload": workload, "method": "batched Newton-Raphson, "
            "preconditioned GMRES (Sec. II-A)", "buses": g.N,
            "branches": g.n_branch, "scenarios_per_gpu": B, "tol": wl.tol,
            "max_iter": wl.max_iter, "gmres": "restart 30, tol 1e-6", "precision": precision,
            "l2": "flushed between steps (512 MiB write)",
            "parallelism": f"replicas x{ws}"}


def run_reference(args):
    """The oracle (numpy FP64) as the reference arm, on the host cores."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload.startswith("grid"):
        return run_reference_nr(args, ws)
    from oracle import zbus_oracle as O
    from paper_2605_14103_gb300 import feeders as F
    workload = args.workload if args.workload in F.WORKLOADS else DEFAULT_WORKLOAD
    f, _, _, wl = F.make_workload(workload, B=1)
    # a bounded sample of the workload per step (the oracle takes ~2.5 ms per
    # scenario at 3069 unknowns on 16 cores): the whole run stays within minutes
    bs = min(wl.B, 512 if f.n < 1000 else 128)
    Sw, Sd = F.workload_scenarios(f, (args.steps + 1) * bs, wl.mult[0], wl.mult[1])
    Z, w, bp = oracle_setup(f)
    for s in range(args.warmup):
        O.fixed_point(Z, w, Sw[:16], Sd[:16], wl.tol, wl.max_iter, bus_phase=bp)
    times, solved = [], 0
    for s in range(args.steps):
        lo = s * bs
        t0 = time.perf_counter()
        V, it, cv = O.fixed_point(Z, w, Sw[lo:lo + bs], Sd[lo:lo + bs], wl.tol, wl.max_iter,
                                  bus_phase=bp)
        times.append(time.perf_counter() - t0)
        solved += int(cv.sum())
    total = sum(times)
    value = solved / total
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": feeder_config(workload, wl, int(Sw.shape[1]), wl.B, args.precision, ws,
                                    getattr(f, "bus_phase", None) is not None),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                            "sample": f"{bs} scenarios of the {wl.B}-scenario workload per step "
                                      "(same generator, consecutive slices)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_reference_nr(args, ws):
    """The Newton-Raphson oracle on the host cores, a few scenarios per step."""
    from oracle import nr_oracle as O
    from paper_2605_14103_gb300 import grids as Gr
    g, P, Q, wl = Gr.make_grid_workload(args.workload)
    Y = O.dense_Y(g.N, g.Y_row, g.Y_col, g.Y_val)
    per = max(1, min(wl.B, int(2000 // g.N)))   # scenarios per step (bounded CPU time)
    for s in range(args.warmup):
        O.newton(Y, g.bus_type, g.v_set, P[s % wl.B], Q[s % wl.B], wl.tol, wl.max_iter)
    times, solved = [], 0
    for s in range(args.steps):
        t0 = time.perf_counter()
        for k in range(per):
            b = (s * per + k) % wl.B
            solved += O.newton(Y, g.bus_type, g.v_set, P[b], Q[b], wl.tol, wl.max_iter)[2]
        times.append(time.perf_counter() - t0)
    value = solved / sum(times)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": grid_config(args.workload, g, wl, wl.B,
                                  args.precision if args.precision in ("fp64", "mixed")
                                  else "fp64", ws),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                            "sample": f"{per} scenarios of the {wl.B}-scenario batch per step "
                                      "(dense Newton-Raphson)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
KERNELS = {"fp64": ("k_currents_f64", "k_gemm3m_f64", "k_decide+k_compact"),
           "fp16_scaled": ("k_residual_group", "k_contract_group", "k_decide_group+k_finish_group"),
           "bf16x2": ("k_residual_group", "k_contract_group", "k_decide_group+k_finish_group"),
           "tree": ("k_residual_group", "k_tree_group", "(sweep end inside k_tree_group)")}
# arithmetic of each form: the sweep's, then the final test's
DTYPE = {"fp64": "f64", "fp16_scaled": "fp16_scaled+f64", "bf16x2": "bf16x2+f64",
         "tree": "f32+f64"}
MIXED_OUTSIDE = ("k_group_reset+k_slot_init+k_group_params+k_finish_group(start)+k_slot_merge"
                 "+k_branch_f64+k_check+k_corr_setup+k_corr_select+k_corr_end")
# launches outside the sweep loop per solve (with no scenario to correct; k_branch_f64 runs
# where every line's two blocks are identical, as in every feeder of the workloads), and per
# sweep (the tensor-core forms fold their stop test into the sweep end up to 1024 slots)
OUTSIDE = {"fp64": ("k_init", 1), "tree": (MIXED_OUTSIDE, 10),
           "fp16_scaled": (MIXED_OUTSIDE, 10), "bf16x2": (MIXED_OUTSIDE, 10)}
PER_SWEEP = {"fp64": 4, "fp16_scaled": 4, "bf16x2": 4, "tree": 2}


def kernel_roofline(form, name, n, B_act_sweeps, ms, peaks, K_pad=None, N_pad=None):
    """Roofline entry of one kernel from its summed launch time over active sweeps.

    B_act_sweeps: sum over the profiled sweeps of the active scenario count.
    Algorithmic work per scenario-sweep: contraction 8 n^2 flop (complex n x n
    times n); residual / currents: the bytes they must move (v, loads, output).
    """
    t = ms / 1e3
    if name == "k_gemm3m_f64":
        ach = 8.0 * n * n * B_act_sweeps / t / 1e12
        n_pad = (n + 47) // 48 * 48
        exe = 6.0 * n_pad * n_pad * B_act_sweeps / t / 1e12
        pk = peaks["fp64_tflops"]
        return {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                "executed": exe, "frac_executed": exe / pk,
                "peak_src": peaks["fp64_src"],
                "note": "achieved counts the algorithmic 8 n^2 flop per scenario-sweep; the 3M "
                        "form executes 6 n_pad^2 (executed, frac_executed)"}
    if name == "k_contract_group":
        zp = 2 if form == "bf16x2" else 1
        ach = 8.0 * n * n * B_act_sweeps / t / 1e12
        exe = 2.0 * N_pad * K_pad * zp * B_act_sweeps / t / 1e12
        byts = (B_act_sweeps * (K_pad * 2 + 32.0 * n)) / t / 1e9   # R rows + v read/write
        pk = peaks["bf16_tflops"]
        tf = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
              "frac": ach / pk, "executed": exe, "frac_executed": exe / pk,
              "peak_src": "MEASURED_PEAKS bf16 burst (fp16 same rate), of measured",
              "note": "achieved: algorithmic 8 n^2 flop per active scenario-sweep; executed: "
                      "2 N_pad K_pad per active scenario-sweep and operand part"}
        hb = {"bound": "hbm", "achieved": byts, "peak": peaks["hbm_gbs"], "unit": "GB/s",
              "frac": byts / peaks["hbm_gbs"], "peak_src": "MEASURED_PEAKS hbm copy, of measured"}
        return tf if tf["frac"] >= hb["frac"] else hb
    # residual / load-current / tree kernels: bytes they must move per
    # scenario-sweep: FP64: v (16 n) + two FP64 load arrays (32 n) + 3M operands
    # written (24 n); mixed residual: double-float v (16 n) + two FP32 load
    # arrays (16 n) + R row (4 n), or the FP32 residual (8 n) for the tree;
    # tree sweep: FP32 residual (8 n) + double-float v read and written (32 n)
    if form == "fp64":
        per = 72.0 * n
    elif form == "tree":
        per = 40.0 * n
    else:
        per = 36.0 * n
    byts = B_act_sweeps * per / t / 1e9
    return {"bound": "hbm", "achieved": byts, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": byts / peaks["hbm_gbs"], "peak_src": "MEASURED_PEAKS hbm copy, of measured"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"], "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}


def probe_fp64(peaks):
    """FP64 roofline denominator: the library's DFMA-chain probe on this GPU
    (best of three launches), beside the nominal rate."""
    from paper_2605_14103_gb300 import zbus
    rates = [zbus.zbus_probe_fp64_rate()[0] for _ in range(3)]
    peaks["fp64_tflops"] = max(rates)
    peaks["fp64_src"] = (f"zbus_probe_fp64_rate: DFMA chains, best of 3 = {max(rates):.3f} "
                         f"TFLOP/s, of measured (nominal {FP64_NOMINAL_TFLOPS})")
    return peaks


def measure(net, form, Sw, Sd, wl, n, steps, warmup, flush, ws, peaks, extra_launches=0,
            n_prof=3):
    """Timed solves of one precision form: value, step times, kernel shares, roofline.
    extra_launches: kernels per solve around the form's own (the scatter of
    the loads into, and the gather of the voltages out of, a partial-phase
    network's padded layout)."""
    import torch
    B = Sw.shape[0]
    net.reserve(B, form)
    V = torch.empty((B, n), dtype=torch.complex128, device="cuda")
    it = torch.empty((B,), dtype=torch.int32, device="cuda")
    cv = torch.empty((B,), dtype=torch.uint8, device="cuda")

    def solve(profile=False):
        net.solve(Sw, Sd, tol=wl.tol, max_iter=wl.max_iter, precision=form,
                  profile=profile, out=(V, it, cv))

    for _ in range(warmup):
        solve()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    barrier(ws)
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        evs[k][0].record()
        solve()
        evs[k][1].record()
    torch.cuda.synchronize()
    barrier(ws)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    mm = net.power_mismatch(V, Sw, Sd)
    good = int(((cv == 1) & (mm <= 1e-6)).sum().item())
    max_iters = int(it.max().item())
    t_max = allreduce_max(sum(step_ms) / 1e3, ws)
    value = allreduce_sum(good, ws) * steps / t_max
    ps = min(B, PARITY_SAMPLE)
    sample = (V[:ps].cpu().numpy(), it[:ps].cpu().numpy(), cv[:ps].cpu().numpy())

    # profiled pass: CUDA events around every kernel of every sweep; the rest
    # of a step (admission, merge, FP64 mismatch test) is the timed step
    # minus the sweeps
    k_ms = [0.0, 0.0, 0.0]
    act_sum = 0
    for _ in range(n_prof):
        flush.zero_()
        solve(profile=True)
        torch.cuda.synchronize()
        ms, act = net.last_profile(wl.max_iter)
        for k in range(len(act)):
            if act[k] > 0:
                for q in range(3):
                    k_ms[q] += float(ms[k, q])
                act_sum += int(act[k])
    names = KERNELS[form]
    step_p50 = statistics.median(step_ms)
    sweep_ms = sum(k_ms) / n_prof
    rest_ms = max(0.0, step_p50 - sweep_ms)
    tot = sweep_ms + rest_ms
    K_pad = (2 * n + 63) // 64 * 64
    N_pad = (2 * n + 255) // 256 * 256
    kernels = []
    for q in range(3):
        e = {"kernel": names[q], "share": k_ms[q] / n_prof / tot if tot else 0.0,
             "ms_per_sweep": k_ms[q] / max(1, act_sum) * B}
        if q < 2:
            e["roofline"] = kernel_roofline(form, names[q], n, act_sum, k_ms[q], peaks, K_pad,
                                            N_pad)
        kernels.append(e)
    kernels.append({"kernel": OUTSIDE[form][0], "share": rest_ms / tot if tot else 0.0,
                    "ms_per_step": rest_ms})
    dom = max(kernels[:2], key=lambda e: e["share"])
    roof = dict(dom["roofline"])
    roof["kernel"] = dom["kernel"]
    tr = TRAFFIC.get((wl.name, B, form, dom["kernel"]))
    roof["traffic"] = tr
    if tr is not None:
        roof["traffic_src"] = TRAFFIC_SRC[(wl.name, B, form, dom["kernel"])]
    if form in ("fp16_scaled", "bf16x2"):
        c = kernels[1]["roofline"]
        if c["bound"] != "tensor":
            c = kernel_roofline(form, "k_contract_group", n, act_sum, k_ms[1],
                                dict(peaks, hbm_gbs=float("inf")), K_pad, N_pad)
        roof["contraction"] = {k: c[k] for k in ("achieved", "executed", "peak", "unit", "frac",
                                                 "frac_executed", "peak_src")}
        roof["contraction"]["share"] = kernels[1]["share"]
    return {"value": value, "ms_per_step": 1e3 * t_max / steps,
            "steps": steps, "warmup": warmup,
            "step_ms_p50": statistics.median(step_ms),
            "step_ms_p99": float(np.percentile(step_ms, 99)), "converged_per_step": good,
            "max_iters": max_iters, "mean_iters": float(it.float().mean().item()),
            "gpu_launches": steps * (OUTSIDE[form][1] + extra_launches + max_iters * (
                PER_SWEEP[form] - (1 if form in ("fp16_scaled", "bf16x2") and
                                   (B + 127) // 128 * 128 <= 1024 else 0))),
            "kernels": kernels, "roofline": roof, "sample": sample}, (V, it, cv)


# DRAM bytes per launch from ncu captures of the current kernels (None until captured)
# (workload, scenarios, form, kernel) -> dram__bytes_read.sum + dram__bytes_write.sum per
# launch from one ncu capture of the current kernel, with how it was taken
TRAFFIC = {
    ("feeder128_b4096", 4096, "fp64", "k_gemm3m_f64"): 66.403584e6 + 1.091584e6,
    ("feeder1024_b16384", 16384, "fp16_scaled", "k_residual_group"):
        4.0 * (404.311040e6 + 49.283840e6),
    ("feeder1024_b16384", 16384, "fp16_scaled", "k_contract_group"):
        2.0 * (1047.367168e6 + 368.998144e6),
}
TRAFFIC_SRC = {
    ("feeder128_b4096", 4096, "fp64", "k_gemm3m_f64"):
        "ncu capture of this launch configuration (sweep 3, all scenarios active)",
    ("feeder1024_b16384", 16384, "fp16_scaled", "k_residual_group"):
        "ncu capture of an FP32 start sweep at 4096 scenarios x 4 (bytes scale with the "
        "scenarios: measured 453.6 MB = algorithmic 452.6 MB; a double-float sweep 453.9 MB)",
    ("feeder1024_b16384", 16384, "fp16_scaled", "k_contract_group"):
        "ncu capture (dram__bytes_read/write.sum, one pass) of sweep 3 at 8192 scenarios x 2: "
        "past one group of 128-slot tiles the bytes grow with the scenarios (4096: 681 MB, "
        "8192: 1416 MB); algorithmic 1886 MB per 16384-scenario launch (Z 75 MB, R rows "
        "201 MB, double-float v read and written 1609 MB)",
}


GRAD_TOL = 1e-10


def measure_gradient(net, Sw, Sd, n, args, flush, ws):
    """Load gradient of the converged FP64 solution (zbus_solve_adjoint), both
    forms (dense FP64 Z^T sweeps; tree sweep in FP64 where the feeder is
    radial): scenario-gradients/s for a seeded loss gradient G, device
    buffers, L2 flushed between steps.  The voltages come from one FP64
    solve before the timed region."""
    import torch
    B = Sw.shape[0]
    V, it, cv = net.solve(Sw, Sd, tol=1e-10, max_iter=100, precision="fp64")
    gen = torch.Generator(device="cuda").manual_seed(1234)
    G = torch.randn((B, n), dtype=torch.complex128, device="cuda", generator=gen)
    out = {}
    for form in ("fp64", "tree"):
        def adj():
            return net.solve_adjoint(V, G, Sw, Sd, tol=GRAD_TOL, max_iter=100, precision=form)

        try:
            for _ in range(max(3, args.warmup)):
                adj()
        except Exception as e:   # a meshed network has no tree form
            out[form] = {"unavailable": str(e)}
            continue
        torch.cuda.synchronize()
        steps = max(3, args.steps // 2)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        barrier(ws)
        torch.cuda.synchronize()
        res = None
        for k in range(steps):
            flush.zero_()
            evs[k][0].record()
            res = adj()
            evs[k][1].record()
        torch.cuda.synchronize()
        barrier(ws)
        step_ms = [a.elapsed_time(b) for a, b in evs]
        _, _, ait, acv = res
        good = int(((acv == 1) & (cv == 1)).sum().item())
        t_max = allreduce_max(sum(step_ms) / 1e3, ws)
        out[form] = {"value": allreduce_sum(good, ws) * steps / t_max,
                     "unit": "scenario-gradients/s", "ms_per_step": 1e3 * t_max / steps,
                     "steps": steps, "converged_per_step": good,
                     "mean_iters": float(ait.float().mean().item()),
                     "max_iters": int(ait.max().item()), "tol": GRAD_TOL}
    out["what"] = ("dL/dS_wye and dL/dS_delta of every scenario at its converged FP64 voltages "
                   "(implicit-function adjoint; fp64: Z^T on the 3M contraction; tree: exact "
                   "Y^T residual and transposed tree sweep, one CTA per scenario)")
    return out


def build_once(ws, rank):
    """Build the library on rank 0 while the other ranks wait at a barrier,
    so that N ranks do not compile and replace the same files at once."""
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier(ws)
    if rank != 0:
        __graft_entry__.build()   # up to date: only loads the library


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_setup()
    build_once(ws, rank)
    from paper_2605_14103_gb300 import feeders as F
    from paper_2605_14103_gb300 import zbus

    torch.cuda.set_device(local)
    peaks = load_peaks()
    f, _, _, wl = F.make_workload(args.workload, B=1)
    Bw = args.batch if args.batch > 0 else wl.B
    from paper_2605_14103_gb300 import dist as D
    Sw_h, Sd_h = F.workload_scenarios(f, Bw, wl.mult[0], wl.mult[1],
                                      seed=D.rank_seed(f.seed + 1, rank))
    B, n = Sw_h.shape
    Sw = torch.from_numpy(Sw_h).cuda()
    Sd = torch.from_numpy(Sd_h).cuda()
    net = zbus.Network.from_feeder(f)
    phased = getattr(f, "bus_phase", None) is not None
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    big = n > 1000

    forms = [args.precision] + ([m for m in ("fp16_scaled", "bf16x2", "tree", "fp64")
                                 if m != args.precision] if args.forms == "all" else [])
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    probe_fp64(peaks)
    results = {}
    head_out = None
    for form in forms:
        head = form == args.precision
        if form == "fp64" and not head and big:
            # the plain method takes seconds per step at this size: a short run
            steps, warm, n_prof = 3, 1, 1
        else:
            steps = args.steps if head else max(3, args.steps // 2)
            warm, n_prof = max(3, args.warmup), 3
        r, out = measure(net, form, Sw, Sd, wl, n, steps, warm, flush, ws, peaks,
                         extra_launches=3 if phased else 0, n_prof=n_prof)
        results[form] = r
        if head:
            head_out = out
    # the load gradient of the converged solution on the plain method's workload
    grad = (measure_gradient(net, Sw, Sd, n, args, flush, ws)
            if "fp64" in results and args.workload == "feeder128_b4096" else None)
    clk = clocks.stop() if clocks else None
    head = results[args.precision]

    # ---- end to end through the public API on pinned host buffers: the call
    # copies the loads in and the results out, overlapped with the sweeps ----
    Sw_p = torch.from_numpy(Sw_h).pin_memory()
    Sd_p = torch.from_numpy(Sd_h).pin_memory()
    V_p = torch.empty((B, n), dtype=torch.complex128).pin_memory()
    it_p = torch.empty((B,), dtype=torch.int32).pin_memory()
    cv_p = torch.empty((B,), dtype=torch.uint8).pin_memory()

    def solve_host():
        net.solve(Sw_p, Sd_p, tol=wl.tol, max_iter=wl.max_iter, precision=args.precision,
                  out=(V_p, it_p, cv_p))

    for _ in range(2):
        solve_host()
    torch.cuda.synchronize()
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    e2e_good = 0
    for k in range(args.steps):
        flush.zero_()
        ev2[k][0].record()
        solve_host()
        ev2[k][1].record()
        torch.cuda.synchronize()
        e2e_good += int(cv_p.numpy().sum())
    e2e_t = allreduce_max(sum(a.elapsed_time(b) for a, b in ev2) / 1e3, ws)
    e2e_val = allreduce_sum(e2e_good, ws) / e2e_t
    del Sw_p, Sd_p, V_p, it_p, cv_p

    cpu, parity = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ref, cpu = oracle_sample(f, Sw_h, Sd_h, wl, args.cpu_seconds)
        parity = {form: parity_vs_oracle(ref, r["sample"], form) for form, r in results.items()}
        parity["what"] = ("first %d scenarios of the batch: flags equal, max |dV| on converged "
                          "scenarios, iteration counts (equal for fp64, within one for the "
                          "defect forms)" % ref[0].shape[0])

    extras = {}
    if (rank == 0 and ws == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_extras
            and args.batch <= 0):
        del Sw, Sd, head_out
        net.close()
        torch.cuda.empty_cache()
        extras = run_extras(args, flush, peaks)

    if rank == 0:
        forms_out = {}
        for k, r in results.items():
            forms_out[k] = {x: r[x] for x in ("value", "ms_per_step", "steps", "warmup",
                                               "mean_iters", "max_iters", "converged_per_step")}
            forms_out[k]["vs_plain_fp64"] = r["value"] / results["fp64"]["value"] \
                if "fp64" in results else None
            forms_out[k]["kernels"] = r["kernels"]
            if parity:
                forms_out[k]["parity"] = parity[k]
        out = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": DTYPE[args.precision],
               "data": "synthetic",
               "config": feeder_config(args.workload, wl, n, B, args.precision, ws, phased),
               "converged_per_step": head["converged_per_step"], "max_iters": head["max_iters"],
               "mean_iters": head["mean_iters"], "gpu_launches": head["gpu_launches"],
               "vs_plain_fp64": forms_out[args.precision]["vs_plain_fp64"],
               "roofline": head["roofline"],
               # one step is one solve of the whole batch: its latency on the device
               "latency": {"p50_ms": head["step_ms_p50"], "p99_ms": head["step_ms_p99"],
                           "per": f"solve of {B} scenarios"},
               "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 2 * B * n * 16,
                       "d2h_bytes_per_step": B * n * 16 + B * 4 + B},
               "clocks": clk, "cpu_baseline": cpu,
               "parity": parity[args.precision] if parity else None,
               "peaks": {"src": peaks["src"], "fp64_tflops": peaks["fp64_tflops"],
                         "fp64_src": peaks["fp64_src"]},
               "forms": forms_out}
        if grad is not None:
            for k in ("fp64", "tree"):
                if "ms_per_step" in grad.get(k, {}):
                    grad[k]["vs_forward_fp64_time"] = (grad[k]["ms_per_step"] /
                                                       results["fp64"]["ms_per_step"])
            out["gradient"] = grad
        out.update(extras)
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_extras(args, flush, peaks):
    """Compact results of the other workloads, for the default line: each a
    short timed run of its own (CUDA events, L2 flushed between steps)."""
    import torch
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    out = {}
    out["feeder13_b8"] = bench_latency()
    out["feeder128_b4096"] = bench_small_plain(flush, peaks)
    out["gradient"] = out["feeder128_b4096"].pop("gradient")
    out["hetero64"] = run_hetero(args, compact=True)
    out["serve16"] = run_serve(args, compact=True)
    out["grid2224_b1000"] = bench_nr_compact(flush)
    out["extras_clocks"] = clocks.stop()
    return out


def bench_latency(solves=200):
    """13-bus feeder x 8 scenarios (the latency-bound case): device time of
    one solve, p50 / p99 over many solves, per form."""
    import torch
    from paper_2605_14103_gb300 import feeders as F
    from paper_2605_14103_gb300 import zbus
    f, Sw_h, Sd_h, wl = F.make_workload("feeder13_b8")
    Sw, Sd = torch.from_numpy(Sw_h).cuda(), torch.from_numpy(Sd_h).cuda()
    net = zbus.Network.from_feeder(f)
    res = {"what": "time of one zbus_solve call of 8 scenarios from Python (CUDA events "
                   "around the call, so the host's call overhead is included), "
                   f"{solves} solves after 10 warm-up"}
    for form in ("fp64", "fp16_scaled", "tree"):
        out = (torch.empty((8, f.n), dtype=torch.complex128, device="cuda"),
               torch.empty((8,), dtype=torch.int32, device="cuda"),
               torch.empty((8,), dtype=torch.uint8, device="cuda"))
        for _ in range(10):
            net.solve(Sw, Sd, tol=wl.tol, max_iter=wl.max_iter, precision=form, out=out)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(solves)]
        for a, b in evs:
            a.record()
            net.solve(Sw, Sd, tol=wl.tol, max_iter=wl.max_iter, precision=form, out=out)
            b.record()
        torch.cuda.synchronize()
        us = np.array([a.elapsed_time(b) * 1e3 for a, b in evs])
        cv = out[2].cpu().numpy()
        res[form] = {"p50_us": float(np.percentile(us, 50)), "p99_us": float(np.percentile(us, 99)),
                     "converged": int(cv.sum()), "solves_per_s": 8 * 1e6 / float(np.median(us))}
    net.close()
    return res


def bench_small_plain(flush, peaks, steps=10):
    """128-bus feeder x 4096 scenarios (the plain method's workload): every
    form's value and its ratio to the plain FP64 method; load gradients."""
    import torch
    from paper_2605_14103_gb300 import feeders as F
    from paper_2605_14103_gb300 import zbus
    f, Sw_h, Sd_h, wl = F.make_workload("feeder128_b4096")
    Sw, Sd = torch.from_numpy(Sw_h).cuda(), torch.from_numpy(Sd_h).cuda()
    n = Sw.shape[1]
    net = zbus.Network.from_feeder(f)
    res = {}
    for form in ("fp64", "fp16_scaled", "bf16x2", "tree"):
        r, _ = measure(net, form, Sw, Sd, wl, n, steps, 3, flush, 1, peaks, n_prof=1)
        res[form] = {"value": r["value"], "ms_per_step": r["ms_per_step"],
                     "converged_per_step": r["converged_per_step"],
                     "mean_iters": r["mean_iters"], "roofline": r["roofline"]}
    for form in res:
        res[form]["vs_plain_fp64"] = res[form]["value"] / res["fp64"]["value"]
    grad = measure_gradient(net, Sw, Sd, n, argparse.Namespace(warmup=3, steps=steps), flush, 1)
    for k in ("fp64", "tree"):
        if "ms_per_step" in grad.get(k, {}):
            grad[k]["vs_forward_fp64_time"] = grad[k]["ms_per_step"] / res["fp64"]["ms_per_step"]
    res["gradient"] = grad
    res["what"] = (f"{wl.name}: {n} unknowns x {Sw.shape[0]} scenarios, tol {wl.tol}, "
                   "CUDA events, L2 flushed, steps " + str(steps))
    net.close()
    return res


# ---------------------------------------------------------------------------
# heterogeneous batch and serving workloads
# ---------------------------------------------------------------------------
def _timed(fn, steps, flush):
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        evs[k][0].record()
        fn()
        evs[k][1].record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def run_hetero(args, compact=False):
    """64 feeders of 50-800 buses, 32-2048 scenarios each, 40 % delta loads.
    compact: a short run whose results are returned (for the default line)."""
    import torch
    if not compact:
        import __graft_entry__
        __graft_entry__.build()
    from paper_2605_14103_gb300 import feeders as F
    from paper_2605_14103_gb300 import zbus
    peaks = load_peaks()
    t0 = time.perf_counter()
    fset = F.heterogeneous_set()
    nets, loads, host = [], [], []
    for f, B in fset:
        Sw, Sd = F.make_scenarios(f, B, 0.8, 1.2)
        nets.append(zbus.Network.from_feeder(f))
        loads.append((torch.from_numpy(Sw).cuda(), torch.from_numpy(Sd).cuda()))
        host.append((f, Sw, Sd))
    setup_s = time.perf_counter() - t0
    total_B = sum(B for _, B in fset)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    forms = {}
    steps = 5 if compact else args.steps
    warmup = 3 if compact else max(3, args.warmup)

    def count(outs):
        good = 0
        for (V, it, cv), net, (sw, sd) in zip(outs, nets, loads):
            mm = net.power_mismatch(V, sw, sd)
            good += int(((cv == 1) & (mm <= 1e-6)).sum().item())
        return good

    for prec in ("fp16_scaled", "bf16x2", "tree"):
        for _ in range(warmup):
            outs = zbus.solve_batched(nets, loads, precision=prec)
        ms = _timed(lambda: zbus.solve_batched(nets, loads, precision=prec), steps, flush)
        outs = zbus.solve_batched(nets, loads, precision=prec)
        good = count(outs)
        sweeps = max(int(it.max().item()) for _, it, _ in outs)
        forms["batched_" + prec] = {"value": good / (statistics.median(ms) / 1e3),
                                    "ms_per_step": statistics.median(ms), "converged": good,
                                    "sweeps": sweeps,
                                    # reset, parameters and tile list, per feeder the
                                    # admission and the three collection kernels, per sweep
                                    # the sweep's kernels
                                    "gpu_launches": 3 + 7 * len(nets) +
                                    (2 if prec == "tree" else 4) * sweeps}
        if prec == "fp16_scaled":
            head_outs = outs

    def seq(prec):
        return [net.solve(sw, sd, precision=prec) for net, (sw, sd) in zip(nets, loads)]
    for prec, nst in (("fp16_scaled", max(2, steps // 2)), ("fp64", 1)):
        seq(prec)
        ms = _timed(lambda: seq(prec), nst, flush)
        good = count(seq(prec))
        forms["one_by_one_" + prec] = {"value": good / (statistics.median(ms) / 1e3),
                                       "ms_per_step": statistics.median(ms), "converged": good}
    head = forms["batched_fp16_scaled"]
    plain = forms["one_by_one_fp64"]["value"]
    for k in forms:
        forms[k]["vs_plain_fp64"] = forms[k]["value"] / plain
    # oracle parity on a sample of feeders
    from oracle import zbus_oracle as O
    worst, flags = 0.0, True
    for idx in (0, 17, 40, 63):
        f, Sw, Sd = host[idx]
        ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack,
                          Sw[:64], Sd[:64])
        V, it, cv = head_outs[idx]
        flags &= bool(np.array_equal(cv[:64].cpu().numpy(), ref["converged"]))
        worst = max(worst, float(np.abs(V[:64].cpu().numpy() - ref["V"]).max()))
    for net in nets:
        net.close()
    if compact:
        return {"value": head["value"], "unit": UNIT, "precision": "fp16_scaled (batched)",
                "ms_per_step": head["ms_per_step"], "vs_plain_fp64": head["vs_plain_fp64"],
                "forms": {k: {x: v[x] for x in ("value", "ms_per_step", "vs_plain_fp64")}
                          for k, v in forms.items()},
                "feeders": len(fset), "scenarios_total": total_B, "steps": steps,
                "parity": {"sampled_feeders": 4, "sampled_scenarios_each": 64,
                           "max_dv_vs_oracle": worst, "flags_equal": flags}}
    out = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "fp16_scaled+f64", "data": "synthetic",
           "config": {"workload": "hetero64", "feeders": len(fset),
                      "buses_range": [min(f.N for f, _ in fset), max(f.N for f, _ in fset)],
                      "scenarios_total": total_B, "tol": 1e-8, "setup_s": setup_s,
                      "l2": "flushed between steps (512 MiB write)"},
           "forms": forms, "peaks": peaks["src"],
           "parity": {"sampled_feeders": 4, "sampled_scenarios_each": 64,
                      "max_dv_vs_oracle": worst, "flags_equal": flags},
           "gpu_launches": head["gpu_launches"]}
    print(json.dumps(out), flush=True)


def run_serve(args, compact=False):
    """Pool of 16 feeders (100-2000 buses); Poisson stream of 1-4096-scenario requests.
    compact: fewer requests per run, results returned (for the default line)."""
    import torch
    if not compact:
        import __graft_entry__
        __graft_entry__.build()
    from paper_2605_14103_gb300 import feeders as F
    from paper_2605_14103_gb300 import zbus
    rng = np.random.default_rng(505)
    t0 = time.perf_counter()
    pool = F.heterogeneous_set(n_feeders=16, seed=505, n_lo=100, n_hi=2000, b_lo=4096,
                               b_hi=4096)
    nets, sc = [], []
    for f, _ in pool:
        nets.append(zbus.Network.from_feeder(f))
        Sw, Sd = F.make_scenarios(f, 4096, 0.8, 1.2)
        sc.append((torch.from_numpy(Sw).cuda(), torch.from_numpy(Sd).cuda()))
    setup_s = time.perf_counter() - t0
    n_req = 1000 if compact else args.requests

    def requests(arrivals):
        out = []
        for i, a in enumerate(arrivals):
            k = int(rng.integers(0, len(pool)))
            B = int(np.clip(np.rint(np.exp(rng.uniform(0.0, np.log(4096.0)))), 1, 4096))
            o = int(rng.integers(0, 4096 - B + 1))
            sw, sd = sc[k]
            out.append({"feeder": k, "S_wye": sw[o:o + B], "S_delta": sd[o:o + B],
                        "arrival": float(a)})
        return out

    prec = "fp16_scaled" if compact or args.precision == "fp64" else args.precision

    def run(reqs):
        t = time.perf_counter()
        res = zbus.serve(nets, reqs, hbm_budget_bytes=120 << 30, max_slots=4096,
                         keep_results=False, precision=prec)
        wall = time.perf_counter() - t
        lat = np.array([r["t_done"] - r["t_arrival"] for r in res])
        scen = sum(r["B"] for r in res)
        good = sum(r["n_converged"] for r in res)
        span = max(r["t_done"] for r in res)
        return {"requests": len(res), "scenarios": scen, "converged": good,
                "throughput": good / span, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "wall_s": wall,
                "operands_formed": int(sum(r.get("operands_formed", 0) for r in res)),
                "all_ok": all(r["status"] == 0 for r in res)}

    zbus.serve(nets, requests(np.zeros(32)), keep_results=False, precision=prec)   # warm-up
    sat = run(requests(np.zeros(n_req)))
    mean_B = sat["scenarios"] / sat["requests"]
    runs = {"saturated": sat}
    for load in (0.3, 0.7, 0.9):
        lam = load * sat["throughput"] / mean_B
        arr = np.cumsum(rng.exponential(1.0 / lam, size=n_req))
        runs[f"load_{load}"] = run(requests(arr))
    head = runs["load_0.7"]
    for net in nets:
        net.close()
    if compact:
        return {"value": sat["throughput"], "unit": UNIT, "precision": prec,
                "requests_per_run": n_req, "hbm_budget_gb": 120,
                "latency_ms": {k: {"p50": v["p50_ms"], "p99": v["p99_ms"]}
                               for k, v in runs.items()},
                "throughput": {k: v["throughput"] for k, v in runs.items()},
                "operands_formed": {k: v["operands_formed"] for k, v in runs.items()},
                "all_ok": all(v["all_ok"] for v in runs.values())}
    out = {"metric": METRIC, "value": sat["throughput"], "unit": UNIT, "n_gpus": 1,
           "steps": 1, "warmup": 1, "ms_per_step": sat["wall_s"] * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": DTYPE[prec], "data": "synthetic",
           "config": {"workload": "serve16", "feeders": len(pool), "precision": prec,
                      "buses_range": [min(f.N for f, _ in pool), max(f.N for f, _ in pool)],
                      "requests_per_run": n_req, "hbm_budget_gb": 120, "setup_s": setup_s},
           "latency": {"p50_ms_at_0.7": head["p50_ms"], "p99_ms_at_0.7": head["p99_ms"]},
           "runs": runs}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# transmission grids: batched Newton-Raphson (Sec. II-A)
# ---------------------------------------------------------------------------
NR_MISMATCH_OK = 1e-9


def nr_cpu_mismatch(g, V, P, Q):
    """max |F_b| of every scenario from the GPU voltages, sparse Y on the CPU
    (outside the timed region)."""
    import scipy.sparse as sp
    Y = sp.csr_matrix((g.Y_val, (g.Y_row, g.Y_col)), shape=(g.N, g.N))
    S = V * np.conj((Y @ V.T).T)
    th = np.nonzero(g.bus_type != 2)[0]
    q = np.nonzero(g.bus_type == 0)[0]
    F = np.concatenate([S.real[:, th] - P[:, th], S.imag[:, q] - Q[:, q]], axis=1)
    return np.abs(F).max(axis=1)


def nr_flops(g, info, iters, gmres):
    """Algorithmic FP64 flops of the solves (estimate from the step counts):
    mismatch per Newton step 8 nnz(Y) + 12 N; per GMRES iteration the
    Jacobian-vector product (8 nnz(Y) + 14 N), the preconditioner (2 nnz of
    the factors + 2 nnz(G) + 2 dim), Gram-Schmidt twice over j vectors
    (8 j dim, j = 1 .. the iterations of that Newton step) and a norm."""
    nnzY = int(g.Y_val.size)
    nt, nq, fnnz, _ = info
    dim = nt + nq
    nnzG = nnzY   # bound: G is a sub-block of Re(Y)
    per_gm = 8 * nnzY + 14 * g.N + 2 * fnnz + 2 * nnzG + 2 * dim + 4 * dim
    tot = 0.0
    for k, gm in zip(iters, gmres):
        k = max(int(k), 1)
        j = gm / k
        tot += (k + 1) * (8 * nnzY + 12 * g.N) + gm * per_gm + k * 8 * dim * j * (j + 1) / 2
    return tot


def bench_nr_compact(flush, steps=5):
    """Newton-Raphson on the 2224-bus grid x 1000 scenarios (Sec. II-A), both
    forms of the Newton direction; CPU-recomputed mismatch of the results."""
    import torch
    from paper_2605_14103_gb300 import grids as Gr
    from paper_2605_14103_gb300 import zbus
    g, P_h, Q_h, wl = Gr.make_grid_workload("grid2224_b1000")
    P, Q = torch.from_numpy(P_h).cuda(), torch.from_numpy(Q_h).cuda()
    B = P.shape[0]
    net = zbus.NrNetwork.from_grid(g)
    out = (torch.empty((B, g.N), dtype=torch.complex128, device="cuda"),
           torch.empty((B,), dtype=torch.int32, device="cuda"),
           torch.empty((B,), dtype=torch.uint8, device="cuda"),
           torch.empty((B,), dtype=torch.int32, device="cuda"))
    res = {}
    for p in ("fp64", "mixed"):
        def solve():
            net.solve(P, Q, tol=wl.tol, max_iter=wl.max_iter, precision=p, out=out)
        for _ in range(3):
            solve()
        torch.cuda.synchronize()
        ms = _timed(solve, steps, flush)
        V, it, cv, gm = (x.cpu().numpy() for x in out)
        mm = nr_cpu_mismatch(g, V, P_h, Q_h)
        good = int(((cv == 1) & (mm <= NR_MISMATCH_OK)).sum())
        res[p] = {"value": good / (statistics.median(ms) / 1e3),
                  "ms_per_step": statistics.median(ms), "converged_per_step": good,
                  "newton_steps_mean": float(it.mean()), "gmres_iters_mean": float(gm.mean()),
                  "max_mismatch": float(mm.max())}
    res["mixed"]["vs_fp64"] = res["mixed"]["value"] / res["fp64"]["value"]
    res["unit"] = "scenario-solves/s"
    res["what"] = ("batched Newton-Raphson with preconditioned GMRES (Sec. II-A), 2224-bus "
                   "meshed grid x 1000 scenarios, tol 1e-10; a solve counts when converged "
                   f"with CPU-recomputed mismatch <= {NR_MISMATCH_OK}")
    net.close()
    return res


def run_nr(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_14103_gb300 import grids as Gr
    from paper_2605_14103_gb300 import zbus
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    g, _, _, wl = Gr.make_grid_workload(args.workload, B=1)
    B = args.batch if args.batch > 0 else wl.B
    from paper_2605_14103_gb300 import dist as D
    P_h, Q_h = Gr.make_injections(g, B, seed=D.rank_seed(g.seed + 1, rank))
    P, Q = torch.from_numpy(P_h).cuda(), torch.from_numpy(Q_h).cuda()
    net = zbus.NrNetwork.from_grid(g)
    info = net.info()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    out = (torch.empty((B, g.N), dtype=torch.complex128, device="cuda"),
           torch.empty((B,), dtype=torch.int32, device="cuda"),
           torch.empty((B,), dtype=torch.uint8, device="cuda"),
           torch.empty((B,), dtype=torch.int32, device="cuda"))

    prec = args.precision if args.precision in ("fp64", "mixed") else "fp64"

    def solve(p=None):
        net.solve(P, Q, tol=wl.tol, max_iter=wl.max_iter, precision=p or prec, out=out)

    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    # the other arithmetic form of the Newton direction, for comparison
    forms = {}
    for p in [x for x in ("fp64", "mixed") if x != prec] + [prec]:
        for _ in range(max(3, args.warmup)):
            solve(p)
        torch.cuda.synchronize()
        barrier(ws)
        msp = _timed(lambda: solve(p), args.steps if p == prec else max(3, args.steps // 2), flush)
        barrier(ws)
        Vp, itp, cvp, gmp = (x.cpu().numpy() for x in out)
        mmp = nr_cpu_mismatch(g, Vp, P_h, Q_h)
        goodp = int(((cvp == 1) & (mmp <= NR_MISMATCH_OK)).sum())
        forms[p] = {"value": goodp / (statistics.median(msp) / 1e3),
                    "ms_per_step": statistics.median(msp), "converged_per_step": goodp,
                    "newton_steps_mean": float(itp.mean()), "gmres_iters_mean": float(gmp.mean()),
                    "max_mismatch": float(mmp.max())}
        ms = msp
    clk = clocks.stop() if clocks else None
    for p in forms:
        forms[p]["vs_fp64"] = forms[p]["value"] / forms["fp64"]["value"]
    V, it, cv, gm = (x.cpu().numpy() for x in out)
    mm = nr_cpu_mismatch(g, V, P_h, Q_h)
    good = int(((cv == 1) & (mm <= NR_MISMATCH_OK)).sum())
    t_max = allreduce_max(sum(ms) / 1e3, ws)
    value = allreduce_sum(good, ws) * args.steps / t_max
    t_step = statistics.median(ms) / 1e3
    flops = nr_flops(g, info, it, gm)
    ach = flops / t_step / 1e12
    pk = probe_fp64(load_peaks())
    roof = {"bound": "alu", "achieved": ach, "peak": pk["fp64_tflops"], "unit": "TFLOP/s",
            "frac": ach / pk["fp64_tflops"], "kernel": f"k_nr_solve<{prec}>", "traffic": None,
            "peak_src": pk["fp64_src"],
            "note": "one CTA per scenario; bound by the latency of the level-by-level "
                    "triangular solves and block barriers, not by a pipe"}

    # end to end through the binding: pinned host injections in, voltages,
    # counts and flags out, inside the timed region
    P_p, Q_p = torch.from_numpy(P_h).pin_memory(), torch.from_numpy(Q_h).pin_memory()
    V_p = torch.empty((B, g.N), dtype=torch.complex128).pin_memory()
    it_p = torch.empty((B,), dtype=torch.int32).pin_memory()
    cv_p = torch.empty((B,), dtype=torch.uint8).pin_memory()

    dtype_line = "f64" if prec == "fp64" else "f32+f64"

    def e2e():
        P.copy_(P_p, non_blocking=True)
        Q.copy_(Q_p, non_blocking=True)
        solve()
        V_p.copy_(out[0], non_blocking=True)
        it_p.copy_(out[1], non_blocking=True)
        cv_p.copy_(out[2], non_blocking=True)

    for _ in range(2):
        e2e()
    torch.cuda.synchronize()
    ms2 = _timed(e2e, args.steps, flush)
    e2e_val = allreduce_sum(int(cv_p.numpy().sum()), ws) * args.steps / \
        allreduce_max(sum(ms2) / 1e3, ws)

    cpu, parity = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import nr_oracle as O
        Y = O.dense_Y(g.N, g.Y_row, g.Y_col, g.Y_val)
        t0, k, solved = time.perf_counter(), 0, 0
        dv, flags_eq, it_ok = 0.0, True, True
        while (time.perf_counter() - t0 < args.cpu_seconds or k == 0) and k < B:
            Vo, ito, cvo = O.newton(Y, g.bus_type, g.v_set, P_h[k], Q_h[k], wl.tol, wl.max_iter)
            solved += int(cvo)
            flags_eq &= bool(cvo == cv[k])
            if cvo:
                dv = max(dv, float(np.abs(V[k] - Vo).max()))
                it_ok &= abs(int(ito) - int(it[k])) <= 1
            k += 1
        t_cpu = time.perf_counter() - t0
        cpu = {"value": solved / t_cpu, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"first {k} scenarios of the {B}-scenario batch, one after another "
                         f"(dense Newton-Raphson, numpy BLAS threads; {t_cpu:.1f} s)"}
        parity = {"sampled": k, "max_dv_vs_oracle": dv, "flags_equal": flags_eq,
                  "newton_steps_within_one": it_ok}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": dtype_line, "data": "synthetic",
                "config": grid_config(args.workload, g, wl, B, prec, ws),
                "precision": prec, "forms": forms,
                "converged_per_step": good, "newton_steps_mean": float(it.mean()),
                "gmres_iters_mean": float(gm.mean()), "max_mismatch": float(mm.max()),
                "factor": {"n_theta": info[0], "n_q": info[1], "nnz": info[2],
                           "levels": info[3]},
                "gpu_launches": args.steps, "roofline": roof,
                "latency": {"p50_ms": statistics.median(ms),
                            "p99_ms": float(np.percentile(ms, 99)),
                            "per": f"solve of {B} scenarios"},
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 2 * B * g.N * 8,
                        "d2h_bytes_per_step": B * g.N * 16 + B * 5},
                "clocks": clk, "cpu_baseline": cpu, "parity": parity}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith("grid"):
        run_nr(args)
    elif args.workload == "hetero64":
        run_hetero(args)
    elif args.workload == "serve16":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
