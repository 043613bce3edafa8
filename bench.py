#!/usr/bin/env python
"""Benchmark: converged Brillouin-zone loop integrals per second.

A step is one pass of the whole hot path over one batch: the 93,312-integral
flow-step batch (ph + pp bubbles at T = 0.05, q on a 24 x 24 zone grid, all
81 pairs of the 9 two-shell form factors, rel tol 1e-6, abs tol 1e-10,
<= 1e5 regions per integral), integrated to convergence on the GPU through the
C ABI (setup, every refinement round, outputs).  Inputs are resident in HBM
when the timed region starts; `e2e` repeats the measurement through the
host-buffer entry point with the host<->device copies inside.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl paid|reference]

`--impl reference` times the FP64 CPU oracle (the reference arm of this
project) on a bounded seeded sample of the same workload.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged BZ loop integrals/s at rel tol 1e-6, learned+batched vs plain FP64"
UNIT = "integrals/s"
# FP64 flops per integrand node of the FP64 region-evaluation kernel
# (k_eval_fp64, N = 4, 81 nodes per region): per region 4117 DFMA (2 flops),
# 736 DADD and 1242 DMUL, from the ncu instruction counters of three launches
# divided by their node evaluations (profiles/k_eval_fp64_first_shell.md).
FP64_FLOPS_PER_NODE = (2 * 4117 + 736 + 1242) / 81.0
# DRAM bytes per evaluated region of the same kernel (same capture): eval-list
# entry and key read, Q_2N and err written.
EVAL_DRAM_BYTES_PER_REGION = 18.3
# FP32 flops per region of the float-float evaluation kernel (k_eval_df, N = 4):
# FFMA counted as 2, FADD / FMUL as 1, from ncu instruction counters over all
# launches of a run divided by the regions that kernel evaluated
# (profiles/k_eval_df_first_shell.md).
DF_FP32_FLOPS_PER_REGION = 2 * 7774.8 + 29243.1 + 3018.3   # 47,811
# FP64 flops per region of the shared-partition kernel (k_eval_group, 81 pairs)
# by rule order N: DFMA counted as 2, DADD / DMUL as 1, from ncu instruction
# counters divided by the regions of the launch
# (profiles/k_eval_group_flow_step_q4.md).  N = 12: the current kernel, one
# launch over 6,240 regions of the flow step at T = 0.05 (DFMA 26,843, DADD
# 4,495, DMUL 8,089 per region).  Other N: counts taken when every node still
# evaluated the near-degenerate series of the kernel F, minus that series (11
# flops per node; it now runs only in warps holding a node with |x1 - x2| <=
# 1/16): lower bounds on the work done.
GROUP_NEAR_FLOPS_PER_NODE = 2 * 4 + 3
GROUP_FP64_FLOPS_PER_REGION = {
    n: f - GROUP_NEAR_FLOPS_PER_NODE * (2 * n + 1) ** 2
    for n, f in {4: 2 * 4839 + 663 + 1766, 6: 2 * 8955 + 1285 + 3118,
                 8: 2 * 14367 + 2131 + 4902, 10: 2 * 21075 + 3201 + 7118}.items()}
GROUP_FP64_FLOPS_PER_REGION[12] = 2 * 26843 + 4495 + 8089      # 66,270
# FP32-pipe thread instructions (FADD + FMUL + FFMA, one issue slot each) and
# FP32 flops (FFMA counted as 2) per region of the float-float form of the
# shared-partition kernel (k_eval_group_ff<N, 1>, ph / pp, 81 pairs, moments in
# the Fourier basis, Jacobian in float-float, seven blocks per SM), from the
# ncu instruction counters of one launch over 6,240 regions of the flow step
# at T = 0.05 divided by its regions (profiles/k_eval_group_ff_flow_step_q4.md:
# FADD 151,014, FMUL 23,938, FFMA 50,107 per region).
GROUP_FP32_INSTR_PER_REGION = {12: 151014 + 23938 + 50107}              # 225,059
GROUP_FP32_FLOPS_PER_REGION = {12: 151014 + 23938 + 2 * 50107}          # 275,166
# pipe utilisation of the same launch (ncu, fraction of peak over active
# cycles), and the DRAM bytes of the kernel per region evaluated, from the
# launch list of the default command's timed steps
# (profiles/launches_flow_step_learned.md: dram__bytes_read.sum +
# dram__bytes_write.sum of its 8 launches, 29.1 + 780.8 MB, over their
# 1,120,076 regions)
GROUP_FP32_PIPES_NCU = {"fma": 0.492, "fp64": 0.280, "alu": 0.173, "lsu": 0.098,
                        "xu_mufu": 0.005, "issue_slots": 0.657, "warps_active_per_sm": 22.0,
                        "source": "ncu --set full, one launch of 6,240 regions of the "
                                  "2,592-integral flow step (k_eval_group_ff_flow_step_q4.md)"}
GROUP_FP32_DRAM_BYTES_PER_REGION = (29.1e6 + 780.8e6) / 1120076                  # 723.1
# the same for the Omega-regulated flow kinds (no exponential; same counters)
GROUP_FLOW_FP64_FLOPS_PER_REGION = {4: 2 * 3822 + 527 + 2171, 6: 2 * 6810 + 1006 + 3963,
                                    8: 2 * 10678 + 1659 + 6347, 10: 2 * 15426 + 2486 + 9323,
                                    12: 2 * 21054 + 3487 + 12891}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["paid", "reference"], default="paid")
    ap.add_argument("--temperature", type=float, default=None,
                    help="flow_step: the temperature (default 0.05)")
    ap.add_argument("--rel-tol", type=float, default=None,
                    help="flow_step / heldout: the relative tolerance (default 1e-6)")
    ap.add_argument("--workload", choices=["flow_step", "flow_step_q4", "first_shell", "sweep",
                                           "flow_omega", "heldout"],
                    default="flow_step")
    ap.add_argument("--path", choices=sorted(PATHS), default="learned",
                    help="learned (the headline): learned seeding + one shared partition per "
                         "(kind, q) for all its pairs, FP32-pipe evaluation; group: the same "
                         "from the uniform start; group_fp64: the same in FP64; plain: one "
                         "partition per integral, FP64; fp32: per integral, FP32 / float-float; "
                         "learned_fp32: fp32 with the learned seed")
    ap.add_argument("--rule-n", type=int, choices=[4, 6, 8, 10, 12], default=12,
                    help="N of the nested rule for the reference arm and for group-mode GPU runs "
                         "without the autotuner (the GPU arm's tuner chooses it otherwise; on "
                         "GB300 it picks 12)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="group paths: keep the default cover and evaluation grid")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the comparison blocks (uniform start, FP64 group, plain FP64)")
    ap.add_argument("--no-global", action="store_true",
                    help="group path: skip the global-error group mode (group_mode = 2) block")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-device-loop", action="store_true",
                    help="skip the extra measurement with the refinement loop as one CUDA graph")
    ap.add_argument("--cpu-sample", type=int, default=4096,
                    help="integrals in the oracle's timed sample")
    return ap.parse_args()


def workload(name, temperature=None, rel_tol=None):
    from paper_1610_09991_gb300 import workloads as W
    if name == "first_shell":
        return W.config_first_shell(), 5
    if name == "flow_step_q4":
        return W.config_flow_step(nq=4), 9
    if name == "sweep":
        return W.config_temperature_sweep(), 9
    if name == "flow_omega":
        return W.config_flow_omega(), 9
    if name == "heldout":
        return W.config_heldout(rel_tol=rel_tol or 1e-6), 9
    # the 93,312-integral flow step; --temperature / --rel-tol give the
    # precision study's variants (T = 0.01 at rel tol 1e-5 and 1e-7)
    w = W.config_flow_step(T=temperature or 0.05, rel_tol=rel_tol or 1e-6)
    return w, 9


def metric_name(w):
    """The headline metric, with the workload's relative tolerance."""
    rt = w.batches[0].rel_tol
    return METRIC if rt == 1e-6 else METRIC.replace("1e-6", "%g" % rt)


def workload_config(w, ff, eval_mode, rule_n=4):
    b0 = w.batches[0]
    return {
        "workload": w.name,
        "integrals": w.n,
        "kinds": sorted({{0: "ph", 1: "pp", 2: "monomial", 3: "overlap", 4: "flow ph",
                          5: "flow pp"}[b.kind] for b in w.batches}),
        "T": b0.T if len({b.T for b in w.batches}) == 1 else sorted({b.T for b in w.batches}),
        "q_points": int(b0.q.shape[0]),
        "form_factors": ff,
        "pairs": int(b0.lm.shape[0]),
        "rel_tol": b0.rel_tol,
        "abs_tol": b0.abs_tol,
        "max_regions": b0.max_regions,
        "rule": "nested Clenshaw-Curtis %dx%d in %dx%d (N = %d)" % (rule_n + 1, rule_n + 1,
                                                                    2 * rule_n + 1, 2 * rule_n + 1,
                                                                    rule_n),
        "init_level": 2,
        "eval": eval_mode,
        "lattice": {"t": w.lattice[0], "tp": w.lattice[1], "mu": w.lattice[2]},
        "l2": "256 MiB buffer written before every timed step; the region pool (tens of GB) exceeds L2",
    }


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling every 50 ms, started before the warm-up steps so
    that the tool is running when the timed region begins; only the samples
    stamped inside the marked window (mark_start / mark_stop, wall clock) are
    kept."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None
        self.window = [None, None]

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark_start(self):
        self.window[0] = time.time()

    def mark_stop(self):
        self.window[1] = time.time()

    def stop(self):
        import datetime
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        t0, t1 = self.window
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                mhz, mx = float(f[2]), float(f[3])
            except ValueError:
                continue
            if t0 is not None and not (t0 - 0.05 <= ts <= (t1 or ts) + 0.05):
                continue
            sm.append(mhz)
            smax.append(mx)
            for n, v in zip(names, f[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "sampling": "nvidia-smi every 50 ms, samples inside the timed region"}


# --------------------------------------------------------------------------- peaks
def fp64_peak(device):
    import ctypes
    from paper_1610_09991_gb300 import build as B
    lib = ctypes.CDLL(B.PEAKS_LIB)
    lib.pipe_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    out, sec = ctypes.c_double(), ctypes.c_double()
    peaks = {}
    for which, name in ((0, "fp64_fma_tflops"), (1, "fp32_fma_tflops"), (2, "mufu_ex2_tops")):
        if lib.pipe_peak(which, device, 5, ctypes.byref(out), ctypes.byref(sec)) == 0:
            peaks[name] = out.value / 1e12
    return peaks


# --------------------------------------------------------------------------- oracle
def cpu_baseline(w, sample, seed=1234, rule_n=4, one_core=256):
    """The oracle on a seeded sample of the workload on all host threads, and
    on the first `one_core` integrals of that sample on one thread."""
    import numpy as np
    import oracle
    from paper_1610_09991_gb300 import workloads as W
    flat = W.flatten(w)
    idx = W.sample_indices(w.n, sample, seed)
    b0 = w.batches[0]
    cores = oracle.max_threads()
    args = (w.lattice, b0.rel_tol, b0.abs_tol, b0.max_regions)
    t0 = time.perf_counter()
    v, e, r, s = oracle.integrate_list(flat["kind"][idx], flat["q"][idx], flat["lm"][idx],
                                       flat["T"][idx], *args, rule_n=rule_n)
    dt = time.perf_counter() - t0
    conv = int((s == 0).sum())
    one = None
    if one_core:
        i1 = idx[:one_core]
        t1 = time.perf_counter()
        _, _, _, s1 = oracle.integrate_list(flat["kind"][i1], flat["q"][i1], flat["lm"][i1],
                                            flat["T"][i1], *args, rule_n=rule_n, nthreads=1)
        d1 = time.perf_counter() - t1
        one = {"value": int((s1 == 0).sum()) / d1, "unit": UNIT, "cores": 1,
               "sample": "the first %d integrals of the same sample, one thread, %.1f s"
                         % (len(i1), d1)}
    return {"value": conv / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d seeded integrals (seed %d) of the %d-integral batch, all %d host "
                      "threads, rule N = %d, %.1f s" % (len(idx), seed, w.n, cores, rule_n, dt),
            "seconds": dt, "converged": conv, "regions_mean": float(r.mean()),
            "one_core": one}, (idx, v, s)


def group_global_check(w, gv, gs, rule_n, rows_per_batch=4, seed=2024):
    """The global-error group mode against Algorithm 2 of the oracle on a few
    sampled (kind, q) groups of every batch: per group the summed deviation
    over its pairs in units of the oracle's group tolerance (the parity bound
    is 2)."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    devs, fails, groups, off = [], 0, 0, 0
    t0 = time.perf_counter()
    for b in w.batches:
        P = b.lm.shape[0]
        v = gv[off:off + b.n].reshape(-1, P)
        st = gs[off:off + b.n].reshape(-1, P)
        off += b.n
        rows = np.sort(rng.choice(b.q.shape[0], min(rows_per_batch, b.q.shape[0]), replace=False))
        vo, eo, ro, so = oracle.integrate_group_global(b.kind, b.q[rows], b.lm, b.T, w.lattice,
                                                       b.rel_tol, b.abs_tol, b.max_regions,
                                                       rule_n=rule_n)
        vo, so = vo.reshape(-1, P), so.reshape(-1, P)
        tol = np.maximum(b.abs_tol, b.rel_tol * np.abs(vo).sum(1))
        d = np.abs(v[rows] - vo).sum(1) / tol
        ok = (st[rows] == 0).all(1) & (so == 0).all(1)
        devs.extend(d[ok].tolist())
        fails += int((d[ok] > 2.0 + 1e-12 / tol[ok]).sum()) + int((~ok).sum())
        groups += len(rows)
    return {"against": "FP64 oracle, Algorithm 2 with the global error, %d sampled groups "
                       "(rule N = %d, %.1f s)" % (groups, rule_n, time.perf_counter() - t0),
            "max_dev_over_group_tol": float(max(devs)) if devs else None,
            "parity_failures": fails}


def accuracy(v, s, vo, so, rel, ab, against, ident=None, lattice=None):
    """Error statement: |v - v_ref| in units of the requested tolerance
    max(rel |v_ref|, abs) on integrals both sides converged.  A pair above 2
    (the parity criterion, plus 1e-12 absolute) is decided by the converged
    dense-trapezoid value of the integral (the oracle's brute force): it counts
    as a parity failure only if v is not within 2 tol of that value.  An
    integral the reference converged and v did not (budget, round cap, pool,
    non-finite) is a parity failure as well."""
    import numpy as np
    both = (s == 0) & (so == 0)
    unconv = np.where((so == 0) & (s != 0))[0]
    tol = np.maximum(rel * np.abs(vo), ab)
    r = np.abs(v - vo)[both] / tol[both]
    over = np.where(both & (np.abs(v - vo) > 2 * tol + 1e-12))[0]
    fails, decided = 0, []
    for i in over:
        if ident is None:
            fails += 1
            continue
        import oracle
        kind, q, l, m, T = ident(int(i))
        truth, M = oracle.brute_force(kind, q, l, m, T, lattice)
        t = max(rel * abs(truth), ab)
        ok = bool(np.isfinite(truth) and abs(v[i] - truth) <= 2 * t + 1e-12)
        fails += 0 if ok else 1
        decided.append({"integral": int(i), "value": float(v[i]), "reference": float(vo[i]),
                        "brute_force": float(truth), "value_within_2tol_of_brute_force": ok})
    return {"against": against, "integrals": int(both.sum()),
            "max_err_over_tol": float(r.max()) if r.size else None,
            "median_err_over_tol": float(np.median(r)) if r.size else None,
            "disagreements_decided_by_brute_force": decided,
            "unconverged_where_reference_converged": int(unconv.size),
            "parity_failures": fails + int(unconv.size)}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_1610_09991_gb300 import workloads as W
    oracle.build()
    w, ff = workload(args.workload, args.temperature, args.rel_tol)
    flat = W.flatten(w)
    b0 = w.batches[0]
    per_step = 512
    times, conv = [], 0
    for k in range(args.warmup + args.steps):
        idx = W.sample_indices(w.n, per_step, 5000 + k)
        t0 = time.perf_counter()
        v, e, r, s = oracle.integrate_list(flat["kind"][idx], flat["q"][idx], flat["lm"][idx],
                                           flat["T"][idx], w.lattice, b0.rel_tol, b0.abs_tol,
                                           b0.max_regions, rule_n=args.rule_n)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            conv += int((s == 0).sum())
    total = sum(times)
    value = conv / total
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": metric_name(w), "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, ff, "fp64", args.rule_n),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d seeded integrals per step (seeds 5000+k) of the "
                                       "%d-integral batch, %d host threads, rule N = %d"
                                       % (per_step, w.n, cores, args.rule_n)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm
PATHS = {
    "learned": "learned proposal seeding (trained on traced plain runs) + batched GPU cubature, "
               "one shared partition per (kind, q) serving all 81 (l, m) pairs, each pair to "
               "its own tolerance; kernel F, row sums and moments in float-float on the FP32 "
               "pipe, region values, errors and totals FP64",
    "group": "batched GPU cubature, one shared partition per (kind, q) serving all 81 (l, m) "
             "pairs from the uniform level-2 start; FP32-pipe evaluation as above",
    "group_fp64": "the same shared partitions, everything FP64",
    "plain": "plain FP64 GPU cubature, one partition per integral, uniform level-2 start",
    "fp32": "one partition per integral, FP32 / float-float integrand, FP64 sums",
    "learned_fp32": "learned proposal seeding + one partition per integral, FP32 / float-float "
                    "integrand, FP64 sums",
}


def path_options(path, rule_n):
    """Context options of a bench path."""
    group = path in ("learned", "group", "group_fp64")
    fp32 = path in ("learned", "group", "fp32", "learned_fp32")
    o = dict(eval_fp32=1 if fp32 else 0, group_mode=1 if group else 0)
    if group:
        o["rule_n"] = rule_n
    return o


def roofline_fp32_group(n_regions, eval_s, rule_n, peaks, launches=0):
    """FP32-pipe roofline of the float-float group kernel: thread instructions
    on the FP32 pipe (FADD, FMUL, FFMA: one issue slot of the pipe each) per
    region from its ncu counters, over the summed event time, against the pipe's
    instruction rate (the measured FFMA peak / 2 flops)."""
    ipr = GROUP_FP32_INSTR_PER_REGION.get(rule_n)
    pk = peaks.get("fp32_fma_tflops")
    if not ipr or not pk or eval_s <= 0:
        return None
    achieved = n_regions * ipr / eval_s / 1e12
    peak = pk / 2.0
    f = GROUP_FP32_FLOPS_PER_REGION[rule_n]
    bpr = GROUP_FP32_DRAM_BYTES_PER_REGION if rule_n == 12 else None
    traffic = bpr * n_regions / launches if bpr and launches else None
    return {"bound": "alu", "kernel": "k_eval_group_ff<%d>" % rule_n, "achieved": achieved,
            "peak": peak, "unit": "T FP32-pipe thread instructions/s", "frac": achieved / peak,
            "traffic": traffic,
            "traffic_note": "compute-bound: ~20 B of eval list / key read and 81 x 12 B of pair "
                            "vectors written per region for %d FP32-pipe instructions; traffic = "
                            "DRAM bytes per region of the ncu launch list x regions per launch "
                            "(the pair vectors' write-back partly lands after the kernel)" % ipr,
            "pipes_ncu": GROUP_FP32_PIPES_NCU if rule_n == 12 else None,
            "peak_source": "measured FFMA micro-benchmark in this run (pipe_peaks.cu), "
                           "2 flops per FFMA instruction",
            "instructions_per_region": ipr,
            "flops_per_region": f, "tflops": n_regions * f / eval_s / 1e12,
            "tflops_frac_of_fma_peak": n_regions * f / eval_s / 1e12 / pk,
            "rule_n": rule_n}


def run_paid(args):
    import numpy as np
    import torch
    from paper_1610_09991_gb300 import build as B
    B.build()
    from paper_1610_09991_gb300 import paid as P
    from paper_1610_09991_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w, ff = workload(args.workload, args.temperature, args.rel_tol)
    if args.workload == "flow_omega" and args.path not in ("group", "group_fp64"):
        # the Omega-regulated flow kinds exist in the shared-partition kernel only
        args.path = "group"
    opts = path_options(args.path, args.rule_n)
    group = opts["group_mode"]
    learned = args.path in ("learned", "learned_fp32")
    ctx = P.Context(*w.lattice, ffset=ff, device=local, timing=1, **opts)
    dev = torch.device("cuda", local)
    # N > 1: the temperature sweep is one fixed job split across the ranks by
    # q row (cost-balanced, no exchange; strong scaling); every other workload
    # is one instance per rank (weak scaling)
    scaling = "weak"
    w_job = w
    if world > 1 and args.workload == "sweep":
        from paper_1610_09991_gb300 import shard as S
        mine = [sub for _, sub in S.local_batches(w.batches, S.plan(w.batches, world)[rank])]
        w = W.Workload(w.name, w.lattice, w.ffset, mine)
        scaling = "strong"
    dbs = [dict(kind=b.kind, T=b.T, q=torch.as_tensor(b.q, device=dev),
                lm=torch.as_tensor(b.lm, dtype=torch.int32, device=dev), rel_tol=b.rel_tol,
                abs_tol=b.abs_tol, max_regions=b.max_regions) for b in w.batches]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peaks = fp64_peak(local)
    tune = None
    if not args.no_autotune:
        # autotuner (outside the timed region): rule order, cover, start level
        # and (group mode) the evaluation grid; the shared-partition paths are
        # tuned on the whole batch up to 10^5 integrals (a trial is one
        # integration, milliseconds at N = 12, and the grid's best size depends
        # on the number of regions), everything else on every 6th q point of
        # each batch
        t0 = time.perf_counter()
        n_all = sum(int(d["q"].shape[0]) * int(d["lm"].shape[0]) for d in dbs)
        whole = group and n_all <= 100000
        sample = dbs if whole else [dict(d, q=d["q"][::6].contiguous()) for d in dbs]
        o = ctx.autotune(sample)
        n_s = sum(int(d["q"].shape[0]) * int(d["lm"].shape[0]) for d in sample)
        tune = {"rule_n": o.rule_n, "cover": o.cover, "eval_blocks": o.eval_blocks,
                "init_level": o.init_level,
                "seconds": time.perf_counter() - t0,
                "sample": ("the whole batch (%d integrals)" % n_s) if whole else
                          ("every 6th q point of each batch (%d integrals)" % n_s)}
        ctx.release_workspace()
    tuned = dict(rule_n=ctx.options.rule_n, cover=ctx.options.cover,
                 eval_blocks=ctx.options.eval_blocks, init_level=ctx.options.init_level)
    prop_info, prop, margin = None, None, None
    if learned:
        from paper_1610_09991_gb300 import proposal as PR
        popts = dict(opts, rule_n=tuned["rule_n"], cover=tuned["cover"]) if group else dict(opts)
        prop, hist, t_train = PR.train_default(device=local, **popts)
        t0 = time.perf_counter()
        margin, calib = PR.calibrate_default(prop, device=local, **popts)   # a MarginPolicy
        prop_info = {"train_seconds": t_train, "calibrate_seconds": time.perf_counter() - t0,
                     "targets": "traced level maps of unseeded runs (options.trace): per unit "
                                "the level of the coarsest final region in each level-4 cell",
                     "draws": "seeds 0..191 of t' ~ U[-0.35,0], mu ~ U[-1.4,0], T log-U[0.005,1], "
                              "12x12 q grid, ph+pp; 300 epochs; margin policy calibrated per "
                              "temperature band on seeds 0..95 (8x8 q grid)",
                     "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                     "margin_policy": margin.as_dict(),
                     "calibration_region_evals_rounds": calib}

    def make_step(c, seeded):
        def step():
            flush.fill_(1)
            if not seeded:
                return c.integrate_multi(dbs, stream=stream)
            return PR.integrate(prop, c, dbs, margin, stream=stream)
        return step

    step = make_step(ctx, learned)
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        step()
    # the per-step bookkeeping below uses torch kernels that load on first use
    warm = torch.zeros(4, dtype=torch.int32, device=dev)
    int((torch.cat([warm, warm]) == 0).sum())
    torch.cuda.synchronize()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark_start()
    prop_l0 = prop.launches if prop is not None else 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    agg = dict(conv=0, budget=0, region_evals=0, node_evals=0, launches=0, eval_launches=0,
               eval_ms=0.0, reduce_ms=0.0, scan_ms=0.0, split_ms=0.0, rounds=0, peak_pool=0,
               df_ms=0.0, df_regions=0, escalated=0)
    ev0.record(stream)
    # an NVTX range around the timed steps lets a profiler capture exactly them
    torch.cuda.nvtx.range_push("timed_steps")
    step_outs, step_stats = [], []
    for _ in range(args.steps):
        step_outs.append(step())
        step_stats.append(ctx.last_stats())
    torch.cuda.nvtx.range_pop()
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.mark_stop()
    prop_launches = (prop.launches - prop_l0) if prop is not None else 0
    if dist:
        dist.barrier()
    for outs, st in zip(step_outs, step_stats):
        s = torch.cat([o.status for o in outs])
        agg["conv"] += int((s == 0).sum())
        agg["budget"] += int((s == 1).sum())
        for k in ("region_evals", "node_evals", "launches", "eval_launches", "eval_ms",
                  "reduce_ms", "scan_ms", "split_ms", "rounds", "df_ms", "df_regions",
                  "escalated"):
            agg[k] += st[k]
        agg["peak_pool"] = max(agg["peak_pool"], st["peak_pool"])
    outs = step_outs[-1]
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    if dist:
        t = torch.tensor([elapsed], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
        c = torch.tensor([agg["conv"]], device=dev, dtype=torch.float64)
        dist.all_reduce(c)
        conv_all = float(c.item())
    else:
        conv_all = agg["conv"]
    value = conv_all / elapsed

    # e2e: host numpy inputs -> pinned H2D -> (proposal) -> integrate -> D2H,
    # wall clock over several steps, through a context with the library's
    # default loop (the device loop: what a user's call runs) and the tuned
    # options
    e2e = None
    if not args.no_e2e:
        hb = [dict(kind=b.kind, T=b.T, q=b.q, lm=b.lm, rel_tol=b.rel_tol, abs_tol=b.abs_tol,
                   max_regions=b.max_regions) for b in w.batches]
        ce = P.Context(*w.lattice, ffset=ff, device=local, **dict(opts, **tuned))
        ce.integrate_host(hb, proposal=prop, margin=margin)   # warm-up (graph, pinned pools)
        torch.cuda.synchronize()
        n_e2e = max(5, min(args.steps, 10))
        t0 = time.perf_counter()
        conv_e2e, h2d, d2h = 0, 0, 0
        for _ in range(n_e2e):
            flush.fill_(1)
            res, h2d, d2h = ce.integrate_host(hb, proposal=prop, margin=margin)
            conv_e2e += sum(int((r.status == 0).sum()) for r in res)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": conv_e2e * world / te, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": n_e2e,
               "loop": "device loop (the library default), tuned options"}
        ce.close()
        del ce
        torch.cuda.empty_cache()

    eval_s = agg["eval_ms"] / 1e3
    roof = None
    if group and opts["eval_fp32"]:
        roof = roofline_fp32_group(agg["region_evals"], eval_s, ctx.options.rule_n, peaks,
                                   agg["eval_launches"])
    elif group and eval_s > 0:
        flow = all(b.kind in (W.FLOW_PH, W.FLOW_PP) for b in w.batches)
        fpr = (GROUP_FLOW_FP64_FLOPS_PER_REGION if flow
               else GROUP_FP64_FLOPS_PER_REGION)[ctx.options.rule_n]
        achieved = agg["region_evals"] * fpr / eval_s / 1e12
        pk = peaks.get("fp64_fma_tflops")
        roof = {"bound": "alu", "kernel": "k_eval_group<%d>" % ctx.options.rule_n,
                "achieved": achieved, "peak": pk,
                "unit": "TFLOP/s", "frac": achieved / pk if pk else None, "traffic": None,
                "traffic_note": "compute-bound: ~20 B of eval list / key read and 81 x 12 B of "
                                "pair vectors written per region for %d FP64 flops" % fpr,
                "peak_source": "measured FP64 FMA micro-benchmark in this run (pipe_peaks.cu)",
                "flops_per_region": fpr, "rule_n": ctx.options.rule_n}
    elif FP64_FLOPS_PER_NODE and eval_s > 0 and not opts["eval_fp32"]:
        achieved = agg["node_evals"] * FP64_FLOPS_PER_NODE / eval_s / 1e12
        pk = peaks.get("fp64_fma_tflops")
        per_launch = agg["region_evals"] / max(1, agg["eval_launches"])
        roof = {"bound": "alu", "kernel": "k_eval_fp64", "achieved": achieved, "peak": pk,
                "unit": "TFLOP/s", "frac": achieved / pk if pk else None,
                "traffic": EVAL_DRAM_BYTES_PER_REGION * per_launch,
                "traffic_note": "bytes per average launch, scaled by regions from the ncu "
                                "capture of the 400-integral case (18.3 B/region)",
                "peak_source": "measured FP64 FMA micro-benchmark in this run (pipe_peaks.cu)",
                "flops_per_node": FP64_FLOPS_PER_NODE}
    df_s = agg["df_ms"] / 1e3
    if not group and opts["eval_fp32"] and DF_FP32_FLOPS_PER_REGION and df_s > 0:
        achieved = agg["df_regions"] * DF_FP32_FLOPS_PER_REGION / df_s / 1e12
        pk = peaks.get("fp32_fma_tflops")
        roof = {"bound": "alu", "kernel": "k_eval_df", "achieved": achieved, "peak": pk,
                "unit": "TFLOP/s", "frac": achieved / pk if pk else None, "traffic": None,
                "traffic_note": "compute-bound (a region is 32 bytes of pool traffic for ~10^5 flops)",
                "peak_source": "measured FP32 FMA micro-benchmark in this run (pipe_peaks.cu)",
                "flops_per_region": DF_FP32_FLOPS_PER_REGION,
                "share_of_eval": df_s / max(eval_s, 1e-12)}
    line = {
        "metric": metric_name(w_job), "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": scaling, "vs_baseline": None,
        "dtype": "f32x2+f64" if opts["eval_fp32"] else "f64", "data": "synthetic",
        "config": dict(workload_config(w_job, ff, "fp32 pipe (float-float), fp64 sums"
                                       if opts["eval_fp32"] else "fp64", ctx.options.rule_n),
                       partition="one per (kind, q) group" if group else "one per integral",
                       parallelism="%d ranks, %s" % (world, "q rows split across ranks"
                                                     if scaling == "strong" else
                                                     "one instance per rank")),
        "clocks": clk, "roofline": roof, "gpu_launches": agg["launches"] + prop_launches,
        "gpu_launches_split": {"integrate_calls": agg["launches"],
                               "proposal_inference": prop_launches},
        "e2e": e2e,
        "path": PATHS[args.path],
        "proposal": prop_info,
        "autotune": tune,
        "budget_integrals_per_step": agg["budget"] / args.steps,
        "region_evals_per_s": agg["region_evals"] * world / elapsed,
        "region_evals_per_step": agg["region_evals"] / args.steps,
        "node_evals_per_s": agg["node_evals"] * world / elapsed,
        "rounds_per_step": agg["rounds"] / args.steps,
        "peak_pool_regions": agg["peak_pool"],
        "kernel_ms_per_step": {k: agg[k] / args.steps for k in
                               ("eval_ms", "df_ms", "reduce_ms", "scan_ms", "split_ms")},
        "eval_launches": agg["eval_launches"],
        "pipe_peaks": peaks,
    }
    if not group and opts["eval_fp32"]:
        line["float_float_regions_per_step"] = agg["df_regions"] / args.steps
        line["escalated_integrals_per_step"] = agg["escalated"] / args.steps
    vals = torch.cat([o.values for o in outs]).cpu().numpy()
    stats = torch.cat([o.status for o in outs]).cpu().numpy()
    # each context below sizes its own pool from the free memory
    del step_outs, outs
    ctx.release_workspace()

    def timed(c, seeded, nsteps):
        """nsteps timed steps of context c (after one warm-up): (block, values, status)."""
        st = make_step(c, seeded)
        st()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        os_, sts = [], []
        for _ in range(nsteps):
            os_.append(st())
            sts.append(c.last_stats())
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        conv = sum(int((torch.cat([o.status for o in x]) == 0).sum()) for x in os_)
        v_ = torch.cat([x.values for x in os_[-1]]).cpu().numpy()
        s_ = torch.cat([x.status for x in os_[-1]]).cpu().numpy()
        blk = {"value": conv * world / t, "unit": UNIT, "ms_per_step": 1e3 * t / nsteps,
               "steps": nsteps, "region_evals": sts[-1]["region_evals"],
               "rounds": sts[-1]["rounds"], "kernels_per_step": sts[-1]["launches"],
               "eval_ms": sts[-1]["eval_ms"], "rule_n": c.options.rule_n,
               "cover": c.options.cover}
        del os_
        return blk, v_, s_

    if not args.no_device_loop:
        # the same steps with the refinement loop on the device: one CUDA graph
        # launch per call (conditional WHILE node), no per-round host sync and
        # no per-kernel events
        cg = P.Context(*w.lattice, ffset=ff, device=local, device_loop=1, **dict(opts, **tuned))
        blk, gv, _ = timed(cg, learned, args.steps)
        blk["values_identical_to_host_loop"] = bool(np.array_equal(gv, vals))
        line["device_loop"] = blk
        cg.close()
        torch.cuda.empty_cache()
    if learned and group and not args.no_compare:
        # what the learned seed gains: the same path from the uniform start
        cu = P.Context(*w.lattice, ffset=ff, device=local, timing=1, **dict(opts, **tuned))
        blk, uv, us = timed(cu, False, args.steps)
        blk["path"] = PATHS["group"]
        line["group_uniform_start"] = blk
        line["speedup_of_learned_seed"] = value / blk["value"]
        line["region_evals_saved_by_learned_seed"] = 1.0 - (
            line["region_evals_per_step"] / max(1, blk["region_evals"]))
        cu.close()
        torch.cuda.empty_cache()
    if group and opts["eval_fp32"] and not args.no_compare:
        # the FP64 form of the shared-partition kernel, same partitions' rule
        c64g = P.Context(*w.lattice, ffset=ff, device=local, timing=1, group_mode=1,
                         **tuned)
        blk, v64g, s64g = timed(c64g, False, min(args.steps, 5))
        fpr = GROUP_FP64_FLOPS_PER_REGION[c64g.options.rule_n]
        ev_s = blk["eval_ms"] / 1e3
        pk = peaks.get("fp64_fma_tflops")
        blk["path"] = PATHS["group_fp64"]
        blk["roofline"] = {"bound": "alu", "kernel": "k_eval_group<%d>" % c64g.options.rule_n,
                           "achieved": blk["region_evals"] * fpr / ev_s / 1e12 if ev_s else None,
                           "peak": pk, "unit": "TFLOP/s", "flops_per_region": fpr}
        if pk and ev_s:
            blk["roofline"]["frac"] = blk["roofline"]["achieved"] / pk
        line["group_fp64"] = blk
        c64g.close()
        torch.cuda.empty_cache()
    glob = None
    if group and not args.no_global:
        # the paper's own stopping test (Algorithm 2, global error): one error
        # sum and one tolerance per (kind, q) group, on the same shared
        # partitions, rule and grid
        cgl = P.Context(*w.lattice, ffset=ff, device=local, group_mode=2,
                        eval_fp32=opts["eval_fp32"], **tuned)
        blk, gv, gs = timed(cgl, False, min(args.steps, 5))
        ge = None
        met, ngr, off, agree = 0, 0, 0, 0.0
        # errors of the last step for the group test
        o_ = cgl.integrate_multi(dbs, stream=stream)
        torch.cuda.synchronize()
        ge = torch.cat([x.errors for x in o_]).cpu().numpy()
        for b in w.batches:
            Pn = b.lm.shape[0]
            vv, ee = gv[off:off + b.n].reshape(-1, Pn), ge[off:off + b.n].reshape(-1, Pn)
            vp = vals[off:off + b.n].reshape(-1, Pn)
            off += b.n
            tolg = np.maximum(b.abs_tol, b.rel_tol * np.abs(vv).sum(1))
            met += int((ee.sum(1) <= tolg * (1 + 1e-6)).sum())
            ngr += vv.shape[0]
            agree = max(agree, float((np.abs(vv - vp).sum(1) / tolg).max()))
        glob = (gv, gs)
        blk.update({
            "path": "group mode 2: shared partition per (kind, q), one error sum and one "
                    "tolerance per group (Algorithm 2's global error, rel_tol on sum |V_c|)",
            "speedup_vs_per_pair_group": blk["value"] / value,
            "groups_meeting_group_tol": met, "groups": ngr,
            "max_dev_from_per_pair_results_over_group_tol": agree})
        line["group_global"] = blk
        del o_
        cgl.close()
        torch.cuda.empty_cache()
    if args.path != "plain" and not args.no_compare:
        # the plain FP64 GPU path (one partition per integral) on the same
        # batch: with its own autotuned rule and cover, and with the library
        # defaults; the metric's denominator
        c64 = P.Context(*w.lattice, ffset=ff, device=local, timing=1)
        if not args.no_autotune:
            t0 = time.perf_counter()
            c64.autotune([dict(d, q=d["q"][::6].contiguous()) for d in dbs])
            c64.release_workspace()
            tune64 = time.perf_counter() - t0
        line["plain_fp64"], v64, s64 = timed(c64, False, 1)
        line["plain_fp64"]["path"] = PATHS["plain"]
        c64.close()
        torch.cuda.empty_cache()
        if not args.no_autotune:
            line["plain_fp64"]["autotune_seconds"] = tune64
            cd = P.Context(*w.lattice, ffset=ff, device=local, timing=1)
            line["plain_fp64_default"], _, _ = timed(cd, False, 1)
            cd.close()
            torch.cuda.empty_cache()
            line["speedup_vs_plain_fp64_default"] = value / line["plain_fp64_default"]["value"]
        line["speedup_vs_plain_fp64"] = value / line["plain_fp64"]["value"]
        flat = W.flatten(w)
        ident_all = lambda i: (int(flat["kind"][i]), flat["q"][i], int(flat["lm"][i][0]),
                               int(flat["lm"][i][1]), float(flat["T"][i]))
        line["accuracy_vs_fp64_gpu"] = accuracy(vals, stats, v64, s64, w.batches[0].rel_tol,
                                                w.batches[0].abs_tol, "FP64 GPU path, every integral",
                                                ident_all, w.lattice)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, (idx, vo, so) = cpu_baseline(w, args.cpu_sample, rule_n=ctx.options.rule_n)
        line["cpu_baseline"] = cb
        flat = W.flatten(w)
        ident_s = lambda i: (int(flat["kind"][idx[i]]), flat["q"][idx[i]], int(flat["lm"][idx[i]][0]),
                             int(flat["lm"][idx[i]][1]), float(flat["T"][idx[i]]))
        line["accuracy"] = accuracy(vals[idx], stats[idx], vo, so, w.batches[0].rel_tol,
                                    w.batches[0].abs_tol, "FP64 oracle, the CPU-baseline sample",
                                    ident_s, w.lattice)
        if glob is not None:
            line["group_global"]["accuracy"] = group_global_check(w, glob[0], glob[1],
                                                                  ctx.options.rule_n)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_paid(args)


if __name__ == "__main__":
    sys.exit(main())
