#!/usr/bin/env python
"""Time to relative KKT 1e-5 of the GPU LoRADS solve on the MaxCut SDP of an
Erdos-Renyi graph with n = 10^7 vertices (average degree 4, weights in {-1,+1},
rank r = 24), plus the roofline of its dominant kernel.

A step is one full solve (init + L-BFGS/ALM iterations to rel. KKT <= 1e-5,
err2 by Lanczos included) with the problem already resident in HBM; timed step
k starts from its own seeded unit-row factor (seed 1 + k, drawn on the device
before the timed region), so the steps form a seed sweep of the iteration
count.  Warm-up steps are solves capped at --warmup-iters L-BFGS iterations
(graph capture, caches, clocks).  The timed loop stops early, before starting
a solve that would end past --time-budget seconds; `steps` reports the solves
actually timed.  `e2e` repeats one solve through the public C ABI from host
buffers (upload of C, A, b and R0 inside the timed region, download of R and y
at the end).

The CPU baseline and --impl reference time the FP64 CPU oracle on a bounded
sample: L-BFGS iterations on an Erdos-Renyi graph with n = 10^6 of the same
family (average degree 4, w in {-1,+1}, same rank), whose per-iteration work
is linear in n and in the stored entries, scaled by n_workload / 10^6 and by
the iteration count to tolerance.

Multi-GPU (torchrun): replicas only -- every rank solves its own copy of the
workload (the single-instance path has no exchange step); value is the max
over ranks.

Other workloads: --workload maxcut_er_1e6 / maxcut_er_1e5 / maxcut_torus_1e6
(same line), serving_batch_512 (the batched persistent solve, instances/s);
--spmm-vs-cusparse N prints an informational comparison of the library's SpMM
with cuSPARSE on the ER graph with N vertices instead of a bench line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

# The oracle legs report single-thread CPU times: numpy's BLAS and OpenMP pools
# are held at one thread (set before numpy is first imported).
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))
T_START = time.perf_counter()

METRIC = "time to rel. KKT 1e-5 (MaxCut n=1e7); SpMM+A(RRᵀ) HBM GB/s vs 8 TB/s"
WORKLOADS = {
    "maxcut_er_1e7": dict(n=10_000_000, edges=20_000_000, weights="pm1", r=24, seed=0, admm_switch=3e-4, lbfgs_mem=2,
                          desc="MaxCut SDP, Erdos-Renyi n=1e7, M=2e7 edges (avg degree 4), w in {-1,+1}, r=24"),
    "maxcut_er_4e6": dict(n=4_000_000, edges=8_000_000, weights="pm1", r=24, seed=0,
                          desc="MaxCut SDP, Erdos-Renyi n=4e6, M=8e6 edges (avg degree 4), w in {-1,+1}, r=24"),
    "maxcut_er_2e6": dict(n=2_000_000, edges=4_000_000, weights="pm1", r=24, seed=0,
                          desc="MaxCut SDP, Erdos-Renyi n=2e6, M=4e6 edges (avg degree 4), w in {-1,+1}, r=24"),
    "maxcut_er_1e6": dict(n=1_000_000, edges=2_000_000, weights="pm1", r=20, seed=0,
                          desc="MaxCut SDP, Erdos-Renyi n=1e6, M=2e6 edges (avg degree 4), w in {-1,+1}, r=20"),
    "maxcut_er_1e5": dict(n=100_000, edges=200_000, weights="pm1", r=17, seed=0,
                          desc="MaxCut SDP, Erdos-Renyi n=1e5, M=2e5 edges (avg degree 4), w in {-1,+1}, r=17"),
    "maxcut_torus_1e6": dict(n=1_000_000, edges=2_000_000, weights="pm1", r=20, seed=0, graph="torus", side=1000,
                             desc="MaxCut SDP, 1000x1000 torus (4-regular, wraparound), w in {-1,+1}, r=20"),
    "maxcut_er_1p7e8": dict(n=170_000_000, edges=340_000_000, weights="pm1", r=28, seed=0, admm_switch=3e-4,
                            lbfgs_mem=2, scale=True,
                            desc="MaxCut SDP, Erdos-Renyi n=1.7e8, M=3.4e8 edges (avg degree 4), w in {-1,+1}, "
                                 "r=28 fixed, two stored L-BFGS pairs (the order of the largest MaxCut of Table 4)"),
    "mc_5e4_rank3": dict(kind="mc", side=50_000, rank=3, n=100_000, m=2_704_945, r=22, seed=0, admm_switch=1e-3,
                         desc="matrix-completion SDP: M = U V^T, U, V in R^{50000x3} iid N(0,1), |Omega| = "
                              "ceil(5 n ln n) = 2,704,945 uniform samples, X of order 1e5, C = I, r = 22"),
}
# metric of each workload's line (the benchmark's own metric for the MaxCut workloads)
MC_METRIC = "time to rel. KKT 1e-5 (matrix completion 5e4 x 5e4, |Omega| 2.7e6)"
BATCH_WORKLOADS = {
    "serving_batch_512": dict(count=512, seed=0, admm_switch=1e-3,
                              desc="512 uneven SDPs: ~3/4 MaxCut on ER graphs (n log-uniform in [200, 20000], "
                                   "average degree 3-20, w in {-1,+1}), ~1/4 matrix completion (side 100-5000, "
                                   "rank 2-5, |Omega| = 5 side ln side); r0 = ceil(log2 m)"),
}
BATCH_METRIC = "instances/s to rel. KKT 1e-5, one persistent launch (512 mixed MaxCut / matrix-completion SDPs)"
# iterations to tolerance used to scale the reference arm's per-iteration time when no
# GPU run of the same invocation provides it (L-BFGS iterations of the GPU two-stage solve
# of maxcut_er_1e7 at switch 3e-4 with two stored pairs, mean over start seeds 1-20; its
# one or two ADMM iterations are not counted)
DEFAULT_ITERS_TO_TOL = {"maxcut_er_1e7": 4170, "maxcut_er_1e6": 6381, "maxcut_er_1e5": 5000,
                       "maxcut_torus_1e6": 5271, "mc_5e4_rank3": 236}
# seconds of one solve to tolerance measured on a GB300 (bench default workload and form);
# plan_seconds uses it to check that the default --steps 20 --warmup 5 run ends within RUN_LIMIT_S
MEASURED_SOLVE_S = {"maxcut_er_1e7": 30.0}
# fixed legs of a default run on the GPU host (seconds, upper estimates): interpreter and
# CUDA start, instance generation, upload, per-kernel profile, one e2e solve on top of its
# solve time, CPU-baseline sample
FIXED_LEGS_S = {"start": 40.0, "generate": 30.0, "create": 10.0, "profile": 20.0, "e2e_extra": 20.0,
                "cpu_baseline": 40.0, "fp64_same_run": 420.0}
RUN_LIMIT_S = 1800.0
DEFAULT_TIME_BUDGET_S = 800.0
FP64_SAME_RUN_LIMIT_S = 400.0


def _args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="maxcut_er_1e7", choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS))
    ap.add_argument("--prec", default="mixed", choices=["fp64", "mixed", "df64", "fp32"])
    ap.add_argument("--admm-switch", type=float, default=None,
                    help="two-stage solve: err1/|err3| at which the ALM stage hands over to the ADMM stage "
                         "(0: ALM only; default: the workload's)")
    ap.add_argument("--reopt-level", type=int, default=0, choices=[0, 1, 2],
                    help="re-opt of Sec. 4.1 with the level-1/2 final criteria")
    ap.add_argument("--e2e-steps", type=int, default=1, help="end-to-end steps")
    ap.add_argument("--profile-iters", type=int, default=200,
                    help="L-BFGS iterations of the CUDA-event-timed solve used for per-kernel durations")
    ap.add_argument("--cpu-iters", type=int, default=2,
                    help="oracle L-BFGS iterations of the CPU-baseline sample (reference arm: per step)")
    ap.add_argument("--cpu-sample-n", type=int, default=1_000_000,
                    help="vertices of the same-family graph the oracle is sampled on (0: the workload itself)")
    ap.add_argument("--warmup-iters", type=int, default=60,
                    help="L-BFGS iterations of each (capped) warm-up solve")
    ap.add_argument("--fp64-same-run", type=int, default=None,
                    help="1: after the timed solves, one cold solve of the plain FP64 form from the first timed "
                         "start (bounded by a time limit), reported beside the headline (default: on for "
                         "the n=1e7 MaxCut workload)")
    ap.add_argument("--time-budget", type=float, default=DEFAULT_TIME_BUDGET_S,
                    help="seconds of timed solves: no solve starts that would end past it (at least one runs)")
    ap.add_argument("--iters-to-tol", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--warm-start", choices=["none", "gnn"], default="none",
                    help="starting factor: seeded random rows, or the learned network (trained before timing "
                         "on solved ER graphs; its prediction is inside the timed region)")
    ap.add_argument("--lbfgs-mem", type=int, default=None,
                    help="stored L-BFGS pairs T (default: the workload's, else 4)")
    ap.add_argument("--scale-time-limit", type=float, default=1500.0,
                    help="time limit (s) of the solve of a scale workload")
    ap.add_argument("--train-graphs", type=int, default=96)
    ap.add_argument("--train-max-n", type=int, default=30000,
                    help="training graphs: n log-uniform in [1000, this]")
    ap.add_argument("--train-epochs", type=int, default=40)
    ap.add_argument("--compare-cold", action="store_true",
                    help="with --warm-start gnn: also time one solve from the random start")
    ap.add_argument("--instance-time-limit", type=float, default=60.0,
                    help="batched solve: per-instance time limit (s); instances past it count as unsolved")
    ap.add_argument("--tune-iters", type=int, default=20, help="batched solve: iterations per autotuner probe")
    ap.add_argument("--kernel-probe", type=int, default=0, metavar="ITERS",
                    help="print the CUDA-event time of every kernel family over the first ITERS L-BFGS iterations "
                         "of a host-stepped solve of the workload (twice) and exit: the target of ncu captures")
    ap.add_argument("--l2-fetch-limit", type=int, default=0, metavar="BYTES",
                    help="with --kernel-probe: set the context's L2 fetch granularity limit (a hint, 0-128 bytes; "
                         "it lasts until the process exits) before timing, and report the limit in force")
    ap.add_argument("--gather-locality", type=int, default=0, metavar="N",
                    help="informational, CPU only: L2 reuse of the SpMM's neighbour gathers on the ER graph with "
                         "N vertices, natural vs reverse Cuthill-McKee order, and exit")
    ap.add_argument("--spmm-vs-cusparse", type=int, default=0, metavar="N",
                    help="informational: time C D of the library's SpMM and of cuSPARSE (torch CSR @ dense) "
                         "on the ER graph with N vertices (degree 4, r = 24, FP32) and exit")
    args = ap.parse_args(argv)
    if args.fp64_same_run is None:
        args.fp64_same_run = 1 if (args.workload == "maxcut_er_1e7" and args.prec != "fp64") else 0
    if args.admm_switch is None:
        args.admm_switch = {**WORKLOADS, **BATCH_WORKLOADS}.get(args.workload, {}).get("admm_switch", 0.0)
    if args.lbfgs_mem is None:
        args.lbfgs_mem = WORKLOADS.get(args.workload, {}).get("lbfgs_mem", 4)
    return args


# ----------------------------------------------------------------------------- helpers

def build_instance(name, with_start: bool = True):
    import workloads as W
    cfg = WORKLOADS[name]
    t = time.perf_counter()
    if cfg.get("kind") == "mc":
        inst, _ = W.config_instance(name, cfg["seed"])
        R0 = W.initial_factor(inst, cfg["r"], cfg["seed"] + 1)
        return inst, R0, time.perf_counter() - t
    if cfg.get("graph") == "torus":
        edges = W.torus_graph(cfg["side"], cfg["seed"], cfg["weights"])
    else:
        edges = W.er_graph(cfg["n"], cfg["edges"], cfg["seed"], cfg["weights"])
    inst = W.maxcut_instance(cfg["n"], edges)
    R0 = W.initial_factor(inst, cfg["r"], cfg["seed"] + 1) if with_start else None
    return inst, R0, time.perf_counter() - t


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        loaded = [s for s, p in zip(sm, power) if p > 0.5 * max(power)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


def kernel_bytes(fam: str, n: int, ld: int, nnz: int, m: int, wR: int, wD: int, T: int, m_off: int = 0) -> float:
    """Algorithmic bytes of one launch (each operand read or written once).  m_off:
    off-diagonal constraints (matrix completion: all of them), each a gathered pair of rows."""
    nl = n * ld
    row_meta = 4 + 8 + 8 + 8                      # dk, da, y, b per row
    if m_off > 0:
        if fam == "k_cons(ls)":                   # i, j, coefficient, id, y, cached z; rows of R and D at i, j
            return m_off * (4 + 4 + 8 + 4 + 8 + 8 + 2 * ld * (wR + wD))
        if fam == "k_cons(ytil)":                 # i, j, coefficient, id, y, b; y~ and z written; rows of R
            return m_off * (4 + 4 + 8 + 4 + 8 + 8 + 8 + 8 + 2 * ld * wR)
        if fam == "k_spmm_a":                     # pattern (2 entries per constraint): column, id, coefficient,
            return 8 * (n + 1) + 2 * m_off * (4 + 4 + 8 + 8 + ld * wR) + nl * wD   # y~, gathered row; W out
        if fam == "k_step":                       # R, C R read and written; D, C D read
            return nl * (4 * wR + 2 * wD)
        if fam == "k_update(step)" and m_off == m:    # no diagonal constraint: R, C R read (the step is k_step)
            return nl * (2 * wR + 6 * wD + 2 * (T - 1) * wD)
    if fam == "k_spmm_c(CD,ls)":
        return nnz * (4 + (8 if wD == 8 else 4)) + (n + 1) * 8 + nl * (2 * wD + wR) + n * row_meta
    if fam == "k_spmm_c(CR,obj)":
        return nnz * (4 + (8 if wR == 8 else 4)) + (n + 1) * 8 + nl * 2 * wR
    if fam == "k_dir":
        return nl * wD * (2 + 2 * T)
    if fam == "k_update(step)":
        return nl * (4 * wR + 6 * wD + 2 * (T - 1) * wD) + n * row_meta
    if fam == "k_update(grad)":
        return nl * (2 * wR + wD) + n * row_meta
    if fam == "k_cons(yupd)":
        return nl * wR + m * (4 + 4 + 8 + 4 + 8 + 8 + 8)
    return float("nan")


# sources that define the single-instance streaming kernels (their device code)
KERNEL_SOURCES = ("common.cuh", "dfloat.cuh", "kernels.cuh", "launch.cuh", "launch_decl.h",
                  "kern_mixed.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update((ROOT / "paper_2407_15049_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, prec: str, lbfgs_mem: int = 4, kernel_variant: int | None = None):
    """DRAM bytes of the committed ncu capture, if the kernels are unchanged and the
    capture ran the same precision form, number of stored pairs and kernel forms."""
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text())
    if d.get("source_hash") != kernel_source_hash() or d.get("prec", "mixed") != prec:
        return None
    if d.get("lbfgs_mem", 4) != lbfgs_mem:
        return None
    if kernel_variant is not None and d.get("kernel_variant") not in (None, kernel_variant):
        return None
    return d.get("kernels", {}).get(kernel)


def dram_rate(traffic_rec, n: int, ld: int, avg_ms: float):
    """DRAM bytes of one launch at this workload (the committed capture's bytes per
    element of the n x ld factor, times n * ld) and the rate in GB/s at which a launch
    of avg_ms moves them; (None, None) without a usable record."""
    if not traffic_rec or not traffic_rec.get("measured_units") or not avg_ms or avg_ms <= 0:
        return None, None
    b = traffic_rec["dram_bytes_measured"] / traffic_rec["measured_units"] * n * ld
    return b, b / (avg_ms * 1e-3) / 1e9


# ----------------------------------------------------------------------------- CPU oracle

def host_cpu() -> str:
    """Architecture, logical CPU count and model name of the host (for the CPU-baseline lines)."""
    import platform
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return f"{platform.machine()}, {os.cpu_count()} logical CPUs" + (f", {model}" if model else "")


def plan_seconds(steps: int, warmup: int, per_solve_s: float, budget_s: float, warmup_frac: float = 0.02) -> dict:
    """Wall-time plan of a default run: the fixed legs, `warmup` capped solves
    (a small fraction of a solve each), the timed solves (the loop starts no solve
    that would end past budget_s, so at most floor(budget_s / per_solve_s) and at
    least one run) and one e2e solve."""
    timed_steps = max(1, min(steps, int(budget_s // per_solve_s)))
    timed = timed_steps * per_solve_s
    total = sum(FIXED_LEGS_S.values()) + warmup * warmup_frac * per_solve_s + timed + per_solve_s
    return {"timed_steps": timed_steps, "timed_s": timed, "total_s": total, "limit_s": RUN_LIMIT_S,
            "fits_in_limit": total <= 0.85 * RUN_LIMIT_S}


def sample_instance(name: str, n_sample: int):
    """The oracle's sample: the workload itself (n_sample = 0 or >= its n) or an
    Erdos-Renyi graph of the same family with n_sample vertices (same average
    degree and weights), seed 0, plus its seeded unit-row start of the same rank."""
    import workloads as W
    cfg = WORKLOADS[name]
    if not n_sample or n_sample >= cfg["n"] or cfg.get("graph") == "torus":
        inst, R0, _ = build_instance(name)
        return inst, R0, 1.0
    edges = W.er_graph(n_sample, int(round(cfg["edges"] * n_sample / cfg["n"])), 0, cfg["weights"])
    inst = W.maxcut_instance(n_sample, edges)
    return inst, W.initial_factor(inst, cfg["r"], 1), cfg["n"] / n_sample


def oracle_overhead(P, R0):
    """Seconds of the oracle's solve around its inner loop (start-up products, the
    multiplier step and the error measures): one outer step with no iteration."""
    from oracle import lorads_oracle as O
    t = time.perf_counter()
    O.solve(P, R0, O.Params(max_outer=1, max_inner=0, tol=1e-300))
    return time.perf_counter() - t


def oracle_iteration_seconds(P, R0, iters: int, overhead: float, mem: int = 4):
    """Seconds per L-BFGS iteration of the FP64 oracle (T = mem stored pairs): one outer
    step with `iters` iterations, less the solve's fixed overhead."""
    from oracle import lorads_oracle as O
    t = time.perf_counter()
    O.solve(P, R0, O.Params(max_outer=1, max_inner=iters, tol=1e-300, lbfgs_mem=mem))
    return max(time.perf_counter() - t - overhead, 1e-9) / iters


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import lorads_oracle as O
    inst, R0, scale = sample_instance(args.workload, args.cpu_sample_n)
    P = O.Problem(inst)
    iters_to_tol = args.iters_to_tol or DEFAULT_ITERS_TO_TOL[args.workload]
    overhead = statistics.median([oracle_overhead(P, R0) for _ in range(max(1, args.warmup))])
    per = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        per.append(oracle_iteration_seconds(P, R0, args.cpu_iters, overhead, args.lbfgs_mem))
    wall = time.perf_counter() - t0
    s_iter = statistics.mean(per) * scale
    value = s_iter * iters_to_tol
    line = {
        "impl": "reference", "metric": _metric(args), "value": value, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(args),
        "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": _sample_text(args, inst, scale, s_iter, iters_to_tol, "per step")},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _sample_text(args, inst, scale, s_iter, iters, what) -> str:
    n_w = WORKLOADS[args.workload]["n"]
    where = (f"the n={n_w:,} solve itself" if scale == 1.0 else
             f"an Erdos-Renyi graph of the same family with n={inst.n:,} ({inst.nnz:,} stored entries, same "
             f"rank), scaled by {scale:g} to n={n_w:,} (per-iteration work is linear in n and nnz)")
    return (f"{args.cpu_iters} oracle L-BFGS iterations {what} on {where}, less the solve's fixed overhead: "
            f"{s_iter:.2f} s/iteration at full size, one thread on {host_cpu()}; times {iters} iterations "
            f"to tolerance")


def _l2_policy(cfg) -> str:
    r_bytes = cfg["n"] * cfg["r"] * 8
    if r_bytes > 129e6:
        return f"inputs larger than L2 (R alone is {r_bytes / 1e6:,.0f} MB at FP64)"
    return f"inputs smaller than L2 (R is {r_bytes / 1e6:,.0f} MB at FP64): timings include L2 reuse"


def _mc_recovery(inst, obj: float) -> dict:
    """The matrix-completion SDP's optimum is 2 ||M||_* (w.h.p. at |Omega| = 5 n ln n): the
    nuclear norm of M = U V^T from the singular values of R_u R_v^T (QR of U and of V)."""
    import numpy as np
    U, V = inst.meta["U"], inst.meta["V"]
    ru = np.linalg.qr(U, mode="r")
    rv = np.linalg.qr(V, mode="r")
    nuc = float(np.sum(np.linalg.svd(ru @ rv.T, compute_uv=False)))
    return {"two_nuclear_norm": 2 * nuc, "objective": obj, "rel_gap": (obj - 2 * nuc) / (2 * nuc)}


def _metric(args) -> str:
    return MC_METRIC if WORKLOADS[args.workload].get("kind") == "mc" else METRIC


def _config(args):
    cfg = WORKLOADS[args.workload]
    mc = cfg.get("kind") == "mc"
    if mc:
        start = "cold (seeded Gaussian rows scaled to ||R0||_F^2 = ||b||_1 / 2)"
    elif args.warm_start == "gnn":
        start = "learned warm start (network trained before timing; prediction timed)"
    else:
        start = "cold (seeded unit-norm Gaussian rows)"
    return {"workload": args.workload, "description": cfg["desc"], "n": cfg["n"], "m": cfg["m"] if mc else cfg["n"],
            "nnz_C": cfg["n"] if mc else cfg["n"] + 2 * cfg["edges"], "rank": cfg["r"],
            "solver_precision": args.prec, "start": start, "tolerance": 1e-5, "lbfgs_mem": args.lbfgs_mem,
            "two_stage": ({"admm_switch": args.admm_switch, "cg_rel": 1e-2, "cg_max": 50}
                          if args.admm_switch > 0 else None),
            "reopt_level": args.reopt_level,
            "l2_policy": _l2_policy(cfg),
            "parallelism": f"replicas x{args.gpus}"}


# ----------------------------------------------------------------------------- native

def max_over_ranks(values, world: int, device: str = "cuda"):
    """Element-wise maximum of per-rank timings over every rank (replicas: the job
    takes as long as its slowest rank).  `None` entries count as 0."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor([0.0 if v is None else float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def run_native(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2407_15049_gb300 as L
    from paper_2407_15049_gb300 import _native as N

    L.load()
    prec_code = {"fp64": L.LORADS_FP64, "mixed": L.LORADS_MIXED, "df64": L.LORADS_DF64,
                 "fp32": L.LORADS_FP32}[args.prec]
    inst, R0, gen_s = build_instance(args.workload)
    cfg = WORKLOADS[args.workload]
    stream = torch.cuda.Stream()
    # rel. KKT = max(err1, err2, err3): err2 (Lanczos on C - A*(y)) is evaluated at the
    # end of every timed solve
    params = L.default_params(prec=prec_code, compute_err2=1, admm_switch=args.admm_switch,
                              reopt_level=args.reopt_level, lbfgs_mem=args.lbfgs_mem)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        t = time.perf_counter()
        ctx = L.lorads_create(inst, params, stream=stream.cuda_stream)
        create_s = time.perf_counter() - t
        R0_dev = torch.as_tensor(R0, device="cuda")
        warm = None
        if args.warm_start == "gnn":
            import math as _m
            import numpy as _np
            import workloads as W
            from paper_2407_15049_gb300 import warmstart as WS
            rng = _np.random.default_rng(12345)
            train = []
            for k in range(args.train_graphs):
                nk = int(round(_m.exp(rng.uniform(_m.log(1000), _m.log(args.train_max_n)))))
                train.append(W.maxcut_instance(nk, W.er_graph(nk, 2 * nk, 5000 + k, "pm1")))
            net, warm = WS.train_on_solved(train, cfg["r"], epochs=args.train_epochs)
            graph = WS.device_graph(inst)
            ldw = N.padded_ld(cfg["r"])

            def start(seed):
                return net.predict(graph, feature_seed=seed, ld=ldw)[:, :cfg["r"]].contiguous()
        else:
            start = None

        def cold_start(seed):
            # seeded Gaussian rows drawn on the device, scaled as the workload's start recipe:
            # unit rows (MaxCut) or ||R0||_F^2 = ||b||_1 / 2 (matrix completion)
            g = torch.Generator(device="cuda")
            g.manual_seed(seed)
            Rs = torch.randn((inst.n, cfg["r"]), dtype=torch.float64, device="cuda", generator=g)
            if inst.kind == "mc":
                target = max(0.5 * float(np.abs(inst.b).sum()), 1.0)
                Rs *= math.sqrt(target) / torch.linalg.vector_norm(Rs)
            else:
                Rs /= torch.linalg.vector_norm(Rs, dim=1, keepdim=True)
            return Rs

        if start is None:
            start = cold_start
        # warm-up: solves capped at a few iterations (graph capture, caches, clocks)
        for _ in range(args.warmup):
            L.lorads_solve(ctx, start(0), on_device=True, max_total_inner=args.warmup_iters)
        # starting factors of the timed solves (seeds 1..K): random starts are drawn before the
        # timed region, the network's predictions inside it (part of the warm-started method)
        starts = [start(1 + k) for k in range(args.steps)] if warm is None else None
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        timed, step_s = [], []
        with ClockSampler(local) as clk:
            barrier()
            t_wall = time.perf_counter()
            ev0.record(stream)
            for k in range(args.steps):
                e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e_a.record(stream)
                timed.append(L.lorads_solve(ctx, starts[k] if starts else start(1 + k), on_device=True))
                e_b.record(stream)
                e_b.synchronize()
                step_s.append(e_a.elapsed_time(e_b) / 1e3)
                spent = time.perf_counter() - t_wall
                # start no solve that would end past the budget (the slowest so far as the estimate)
                if k + 1 < args.steps and spent + max(step_s) > args.time_budget:
                    break
            ev1.record(stream)
            barrier()
        elapsed = ev0.elapsed_time(ev1) / 1e3
        steps_timed = len(timed)
        del starts
        cold = None
        if warm is not None and args.compare_cold:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = L.lorads_solve(ctx, R0_dev, on_device=True)
            e1.record(stream)
            torch.cuda.synchronize()
            cold = {"seconds": e0.elapsed_time(e1) / 1e3, "inner_iters": rc["inner_iters"],
                    "outer_iters": rc["outer_iters"], "primal_obj": rc["primal_obj"], "status": rc["status_name"]}
        last = timed[-1]
        launches = sum(r["kernel_launches"] for r in timed)
        # per-kernel durations: a host-stepped run of the same solve (first profile_iters
        # L-BFGS iterations) with a CUDA event pair around every launch on the solve stream
        prof = {}
        if not args.no_profile:
            pctx = L.lorads_create(inst, L.default_params(prec=prec_code, verbose=2, max_outer=10**6,
                                                          max_inner=args.profile_iters, rank_update_threshold=10**6,
                                                          lbfgs_mem=args.lbfgs_mem),
                                   stream=stream.cuda_stream)
            L.lorads_solve(pctx, R0_dev, on_device=True, max_total_inner=args.profile_iters)
            prof = L.lorads_kernel_times(pctx)
            L.lorads_destroy(pctx)
        L.lorads_destroy(ctx)
        # the plain FP64 form on the same workload and start as the first timed solve
        fp64 = None
        if args.fp64_same_run:
            fctx = L.lorads_create(inst, L.default_params(prec=L.LORADS_FP64, compute_err2=1,
                                                          admm_switch=args.admm_switch, reopt_level=args.reopt_level,
                                                          time_limit=FP64_SAME_RUN_LIMIT_S, lbfgs_mem=args.lbfgs_mem),
                                   stream=stream.cuda_stream)
            f0 = cold_start(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rf = L.lorads_solve(fctx, f0, on_device=True)
            e1.record(stream)
            torch.cuda.synchronize()
            L.lorads_destroy(fctx)
            del f0
            first = timed[0]
            fp64 = {"seconds": e0.elapsed_time(e1) / 1e3, "start": "cold, seed 1 (the first timed step's "
                    "start when that is cold)", "time_limit_s": FP64_SAME_RUN_LIMIT_S,
                    **{k: rf[k] for k in ("status_name", "primal_obj", "err1", "err2", "err3", "inner_iters",
                                          "outer_iters", "admm_iters", "cg_steps")},
                    "mixed_same_start": {"seconds": step_s[0], "primal_obj": first["primal_obj"],
                                         "inner_iters": first["inner_iters"]},
                    "rel_obj_diff_mixed_vs_fp64": (first["primal_obj"] - rf["primal_obj"]) / abs(rf["primal_obj"]),
                    "speedup_mixed_vs_fp64": (e0.elapsed_time(e1) / 1e3) / step_s[0]}
        del R0_dev
        # end to end through the C ABI from host buffers
        e2e_steps = args.e2e_steps
        R0_pinned = torch.from_numpy(R0).pin_memory().numpy()
        e2e_times, e2e_parts = [], []
        # the first timed step's start, from pinned host memory: the e2e solve repeats that solve
        if warm is None:
            R0_pinned = cold_start(1).cpu().pin_memory().numpy()
        h2d = (inst.rowptr.nbytes + inst.colind.nbytes + inst.val.nbytes + inst.con.nbytes + inst.row.nbytes
               + inst.col.nbytes + inst.aval.nbytes + inst.b.nbytes + R0_pinned.nbytes)
        d2h = 0
        for _ in range(e2e_steps):
            barrier()
            t = time.perf_counter()
            c2 = L.lorads_create(inst, params, stream=stream.cuda_stream)
            t_c = time.perf_counter()
            if warm is not None:
                g2 = WS.device_graph(inst)
                rr = L.lorads_solve(c2, net.predict(g2, feature_seed=0, ld=ldw)[:, :cfg["r"]].contiguous(),
                                    on_device=True)
                del g2
            else:
                rr = L.lorads_solve(c2, R0_pinned)
            t_s = time.perf_counter()
            Rh, yh = L.lorads_get_solution(c2, inst.n, inst.m)
            L.lorads_destroy(c2)
            barrier()
            e2e_times.append(time.perf_counter() - t)
            e2e_parts.append({"create_s": t_c - t, "solve_s": t_s - t_c, "download_destroy_s": time.perf_counter() - t_s,
                              "inner_iters": rr["inner_iters"]})
            d2h = Rh.nbytes + yh.nbytes

    per_step = elapsed / steps_timed
    e2e_mean = statistics.mean(e2e_times) if e2e_times else None
    if world > 1:
        per_step, e2e_mean = max_over_ranks([per_step, e2e_mean], world)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel (largest total time in the profiled solve)
    wR = 8 if args.prec in ("fp64", "mixed", "df64") else 4
    wD = 8 if args.prec in ("fp64", "df64") else 4
    ld = N.padded_ld(cfg["r"])
    peak, peak_kind = measured_peaks()
    # launches of each family in the timed solve: inner-iteration kernels once per
    # L-BFGS iteration, outer-step kernels once per outer step
    per_inner = {"k_dir", "k_spmm_c(CD,ls)", "k_ctrl_root", "k_update(step)", "k_ctrl_hist", "k_cons(ls)",
                 "k_step", "k_spmm_a", "k_cons(ytil)"}
    kernels = {}
    m_off = int(np.sum(inst.row != inst.col))
    for name, (ms, cnt) in prof.items():
        b = kernel_bytes(name, inst.n, ld, inst.nnz, inst.m, wR, wD, params.lbfgs_mem, m_off)
        solve_launches = last["inner_iters"] if name in per_inner else last["outer_iters"]
        kernels[name] = {"avg_ms": ms, "profiled_launches": cnt, "solve_launches": solve_launches,
                         "share": None, "algorithmic_bytes": None if math.isnan(b) else b,
                         "GBps": None if math.isnan(b) else b / (ms * 1e-3) / 1e9}
    tot = sum(v["avg_ms"] * v["solve_launches"] for v in kernels.values()) or 1.0
    for v in kernels.values():
        v["share"] = v["avg_ms"] * v["solve_launches"] / tot
    roofline = None
    hot = [k for k in kernels if kernels[k]["GBps"] is not None]
    if hot:
        dom = max(hot, key=lambda k: kernels[k]["avg_ms"] * kernels[k]["solve_launches"])
        ach = kernels[dom]["GBps"]
        tr = ncu_traffic(dom, args.prec, args.lbfgs_mem, params.kernel_variant)
        # DRAM bytes per unit from the committed capture, times this workload's units
        # (the streaming passes move every operand once: traffic grows with n * ld)
        traffic, dram_gbps = dram_rate(tr, cfg["n"], ld, kernels[dom]["avg_ms"])
        roofline = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "peak_kind": peak_kind, "frac_of_8TBps": ach / 8000.0,
                    "traffic": traffic, "dram_GBps": dram_gbps,
                    "algorithmic_bytes_per_launch": kernels[dom]["algorithmic_bytes"],
                    "avg_launch_ms": kernels[dom]["avg_ms"]}
        spmm = kernels.get("k_spmm_c(CD,ls)")
        if spmm:
            # the neighbour gathers read each row of D once per stored entry: DRAM bytes
            # (lower bound when scaled from the smaller capture) above the algorithmic ones
            s_tr, s_gbps = dram_rate(ncu_traffic("k_spmm_c(CD,ls)", args.prec, args.lbfgs_mem, params.kernel_variant),
                                     cfg["n"], ld, spmm["avg_ms"])
            roofline["spmm"] = {"achieved": spmm["GBps"], "frac": spmm["GBps"] / peak,
                                "frac_of_8TBps": spmm["GBps"] / 8000.0, "avg_launch_ms": spmm["avg_ms"],
                                "traffic": s_tr, "dram_GBps": s_gbps,
                                "dram_frac": None if s_gbps is None else s_gbps / peak}
    iters_mean = statistics.mean(r["inner_iters"] for r in timed)
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import lorads_oracle as O
        s_inst, s_R0, scale = sample_instance(args.workload, args.cpu_sample_n)
        P = O.Problem(s_inst)
        s_iter = oracle_iteration_seconds(P, s_R0, args.cpu_iters, oracle_overhead(P, s_R0), args.lbfgs_mem) * scale
        cpu = {"value": s_iter * iters_mean, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": _sample_text(args, s_inst, scale, s_iter, round(iters_mean),
                                      "(the mean L-BFGS iteration count of the timed GPU solves)")}
    plan = plan_seconds(args.steps, args.warmup, MEASURED_SOLVE_S.get(args.workload, per_step), args.time_budget)
    line = {
        "metric": _metric(args), "value": per_step, "unit": "s", "n_gpus": world, "steps": steps_timed,
        "steps_requested": args.steps, "warmup": args.warmup, "warmup_iters": args.warmup_iters, "ms_per_step": per_step * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f32 (+double-float R, CR)", "df64": "double-float (2xf32)",
                  "fp32": "f32"}[args.prec],
        "data": "synthetic", "config": {**_config(args), "l2_fetch_limit_bytes": l2_fetch_limit()},
        "e2e": {"value": e2e_mean, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "parts": e2e_parts, "start": "the first timed step's (seed 1), from pinned host memory"},
        "gpu_launches": int(launches),
        "roofline": roofline, "cpu_baseline": cpu, "clocks": clk.summary(),
        "solve": {k: last[k] for k in ("status_name", "primal_obj", "dual_obj", "err1", "err2", "err3", "sigma_min",
                                       "rho", "rank", "outer_iters", "inner_iters", "admm_iters", "cg_steps",
                                       "reopt_rounds", "seconds")},
        "per_step": {"start_seed": list(range(1, steps_timed + 1)), "seconds": step_s,
                     "inner_iters": [r["inner_iters"] for r in timed],
                     "admm_iters": [r["admm_iters"] for r in timed], "cg_steps": [r["cg_steps"] for r in timed],
                     "outer_iters": [r["outer_iters"] for r in timed],
                     "status": [r["status_name"] for r in timed],
                     "primal_obj": [r["primal_obj"] for r in timed],
                     "max_rel_kkt": [max(r["err1"], abs(r["err3"]), max(r["err2"], 0.0)) for r in timed]},
        "spread": {"seconds_min": min(step_s), "seconds_median": statistics.median(step_s),
                   "seconds_max": max(step_s), "iters_mean": iters_mean},
        "consistency": {"timed_wall_s": elapsed, "time_budget_s": args.time_budget,
                        "wall_s_total": time.perf_counter() - T_START, "plan": plan,
                        "fits_in_limit": (time.perf_counter() - T_START) <= RUN_LIMIT_S},
        "sdp_value": last["primal_obj"] if inst.kind == "mc" else -last["primal_obj"],
        "mc_recovery": _mc_recovery(inst, last["primal_obj"]) if inst.kind == "mc" else None,
        "warm_start": None if warm is None else {
            "kind": "learned (3-layer message passing, bf16 activations)", "training": {
                k: v for k, v in warm.items() if k != "batch_stats"}, "cold_start_same_run": cold},
        "fp64_same_run": fp64,
        "kernels": kernels, "setup_s": {"generate": gen_s, "create": create_s},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def batch_bytes(inst, ld: int, wR: int, wD: int, T: int, inner: int, outer: int, cg_steps: int = 0) -> float:
    """Algorithmic bytes of one instance's batched solve: per L-BFGS iteration the
    direction, line-search SpMM / constraint pass and row update (each operand once),
    per outer step the multiplier pass and C R, per CG step of the ADMM stage the
    operator pass (p, r read, p and Q written, V read; slot gathers of p and V) and the
    update pass (X read and written, p, r, Q read, r written)."""
    n, m, nnz = inst.n, inst.m, inst.nnz
    fam = lambda f: kernel_bytes(f, n, ld, nnz, m, wR, wD, T)  # noqa: E731
    per_inner = fam("k_dir") + fam("k_spmm_c(CD,ls)") + fam("k_update(step)")
    m_off = m - (n if inst.kind == "maxcut" else 0)
    if m_off > 0:                       # constraint line-search pass, y~ pass, A*(y~) R
        per_inner += m_off * (4 * 4 + 8 * 3) + 2 * m_off * ld * (wR + wD) + 2 * m_off * ld * wR + n * ld * wD
    per_outer = fam("k_cons(yupd)") + fam("k_spmm_c(CR,obj)") + fam("k_update(grad)")
    per_cg = n * ld * (4 * wD + wR) + n * ld * (2 * wR + 4 * wD) + 2 * m_off * ld * (wD + wR)
    return per_inner * inner + per_outer * outer + per_cg * cg_steps


def _oracle_instance_seconds(inst, r0, admm_switch: float = 0.0):
    from oracle import lorads_oracle as O
    from oracle import admm_oracle as A
    import workloads as W
    R0 = W.initial_factor(inst, r0, 1)
    t = time.perf_counter()
    if admm_switch > 0:
        ref = A.solve_two_stage(O.Problem(inst), R0, O.Params(), A.AdmmParams(switch_err1=admm_switch))
    else:
        ref = O.solve(O.Problem(inst), R0, O.Params())
    return time.perf_counter() - t, ref


def _batch_cpu_sample(B, budget_s: float = 20.0, admm_switch: float = 0.0):
    """The oracle on a seeded sample of the batch's instances, smallest first until
    about budget_s of CPU time: instances per second on that sample."""
    import numpy as np
    import workloads as W
    rng = np.random.default_rng(5)
    idx = sorted(rng.choice(len(B), size=min(16, len(B)), replace=False), key=lambda i: B[i].n)
    done, spent, names = 0, 0.0, []
    for i in idx:
        if spent > budget_s:
            break
        s, _ = _oracle_instance_seconds(B[i], W.rank_log2(B[i].m), admm_switch)
        spent += s
        done += 1
        names.append(f"{B[i].kind} n={B[i].n}")
    return done / spent if spent > 0 else None, spent, names


def run_batch(args):
    import numpy as np
    import torch
    import workloads as W
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = BATCH_WORKLOADS[args.workload]
    t = time.perf_counter()
    B = W.serving_batch(cfg["count"], cfg["seed"])
    gen_s = time.perf_counter() - t
    count = len(B)
    if args.impl == "reference":
        if rank != 0:
            return 0
        per = []
        for _ in range(args.steps):
            v, spent, names = _batch_cpu_sample(B, budget_s=20.0, admm_switch=args.admm_switch)
            per.append((v, spent, names))
        v, spent, names = per[-1]
        line = {"impl": "reference", "metric": BATCH_METRIC, "value": v, "unit": "instances/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": spent * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "description": cfg["desc"]},
                "cpu_baseline": {"value": v, "unit": "instances/s", "cores": 1, "kind": "oracle",
                                 "sample": f"{len(names)} seeded instances of the batch, smallest first, solved to "
                                           f"tolerance by the oracle ({spent:.1f} s, one thread on {host_cpu()}): " + ", ".join(names)},
                "e2e": {"value": v, "unit": "instances/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2407_15049_gb300 as L
    L.load()
    prec_code = {"fp64": L.LORADS_FP64, "mixed": L.LORADS_MIXED, "fp32": L.LORADS_FP32}[args.prec]
    params = L.default_params(prec=prec_code, time_limit=args.instance_time_limit, admm_switch=args.admm_switch)
    t = time.perf_counter()
    b = L.lorads_batch_create(B, params)
    create_s = time.perf_counter() - t
    t = time.perf_counter()
    shape = L.lorads_batch_tune(b, args.tune_iters)
    tune_s = time.perf_counter() - t

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        L.lorads_batch_solve(b, count)
    barrier()
    secs, stats = [], None
    with ClockSampler(local) as clk:
        barrier()
        for _ in range(args.steps):
            res, stats = L.lorads_batch_solve(b, count)
            secs.append(stats["seconds"])
        barrier()
    per_step = max(secs)
    L.lorads_batch_destroy(b)
    # end to end: host arrays -> create -> solve -> every solution back to the host
    barrier()
    t = time.perf_counter()
    b2 = L.lorads_batch_create(B, params)
    L.lorads_batch_set_shape(b2, shape["ctas_per_sm"], shape["rows_per_warp"], shape["order"], shape["threads"],
                             shape["cluster"], shape["team_count"])
    res2, st2 = L.lorads_batch_solve(b2, count)
    d2h = 0
    for i, inst in enumerate(B):
        Rh, yh = L.lorads_batch_get_solution(b2, i, inst.n, inst.m)
        d2h += Rh.nbytes + yh.nbytes
    L.lorads_batch_destroy(b2)
    barrier()
    e2e_s = time.perf_counter() - t
    h2d = sum(x.rowptr.nbytes + x.colind.nbytes + x.val.nbytes + x.con.nbytes + x.row.nbytes + x.col.nbytes
              + x.aval.nbytes + x.b.nbytes for x in B)
    if world > 1:
        per_step, e2e_s = max_over_ranks([per_step, e2e_s], world)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    wR = 8 if args.prec in ("fp64", "mixed") else 4
    wD = 8 if args.prec == "fp64" else 4
    alg = 0.0
    for inst, r in zip(B, res):
        alg += batch_bytes(inst, L.padded_ld(max(r["rank"], 1)), wR, wD, params.lbfgs_mem, r["inner_iters"],
                           r["outer_iters"], r["cg_steps"])
    peak, peak_kind = measured_peaks()
    ach = alg / per_step / 1e9
    kinds = np.array([x.kind for x in B])
    stat = np.array([r["status"] for r in res])
    solved = {k: int(np.sum((kinds == k) & (stat == 0))) for k in ("maxcut", "mc")}
    totals = {k: int(np.sum(kinds == k)) for k in ("maxcut", "mc")}
    cpu = None
    if not args.no_cpu_baseline:
        v, spent, names = _batch_cpu_sample(B, budget_s=20.0, admm_switch=args.admm_switch)
        cpu = {"value": v, "unit": "instances/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(names)} seeded instances of the batch, smallest first, solved to tolerance by "
                         f"the oracle ({spent:.1f} s, one thread on {host_cpu()}): " + ", ".join(names)}
    line = {
        "metric": BATCH_METRIC, "value": count * world / per_step, "unit": "instances/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f32 (+double-float R, CR)", "fp32": "f32"}[args.prec],
        "data": "synthetic",
        "config": {"workload": args.workload, "description": cfg["desc"], "count": count,
                   "solver_precision": args.prec, "instance_time_limit_s": args.instance_time_limit,
                   "two_stage": ({"admm_switch": args.admm_switch, "cg_rel": 1e-2, "cg_max": 50}
                                 if args.admm_switch > 0 else None),
                   "tolerance": 1e-5, "shape": shape, "l2_policy": "state of all instances 1.1x L2 and up; "
                   "each launch restarts every instance from its start", "parallelism": f"replicas x{world}"},
        "e2e": {"value": count / e2e_s, "unit": "instances/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": args.steps,
        "latency_ms": {"p50": stats["latency_p50_ms"], "p99": stats["latency_p99_ms"],
                       "max": stats["latency_max_ms"]},
        "solved": solved, "instances": totals, "inner_iters": stats["inner_iters"],
        "admm": {"instances_with_stage": int(sum(1 for r in res if r["admm_iters"] > 0)),
                 "admm_iters": int(sum(r["admm_iters"] for r in res)),
                 "cg_steps": int(sum(r["cg_steps"] for r in res))},
        "status_counts": {nm: int(sum(1 for r in res if r["status_name"] == nm))
                          for nm in sorted({r["status_name"] for r in res})},
        "roofline": {"kernel": "k_batch_solve", "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak, "peak_kind": peak_kind, "traffic": None,
                     "algorithmic_bytes_per_launch": alg, "avg_launch_ms": per_step * 1e3},
        "cpu_baseline": cpu, "clocks": clk.summary(),
        "setup_s": {"generate": gen_s, "create": create_s, "tune": tune_s},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def gather_reuse(indptr, indices, windows, row_bytes: int = 96, chunk: int = 64) -> dict:
    """Fraction of the SpMM's neighbour-row fetches that an L2 holding the last W
    processed rows' traffic could serve: rows are processed in index order (time =
    row), each stored entry (i, j) fetches the `chunk`-byte pieces of row j of the
    gathered operand (row_bytes each), and a fetch counts as reused when the same
    piece was fetched at most W rows earlier.  Returns {W: fraction} and the number
    of fetches."""
    import numpy as np
    indptr = np.asarray(indptr, dtype=np.int64)
    col = np.asarray(indices, dtype=np.int64)
    t = np.repeat(np.arange(len(indptr) - 1, dtype=np.int64), np.diff(indptr))
    first = col * row_bytes // chunk
    last = (col * row_bytes + row_bytes - 1) // chunk
    span = last - first
    pieces, times = [first], [t]
    for k in range(1, int(span.max(initial=0)) + 1):
        sel = span >= k
        pieces.append(first[sel] + k)
        times.append(t[sel])
    pc, tm = np.concatenate(pieces), np.concatenate(times)
    order = np.lexsort((tm, pc))
    pc, tm = pc[order], tm[order]
    same = np.r_[False, pc[1:] == pc[:-1]]
    gap = np.r_[np.inf, (tm[1:] - tm[:-1]).astype(float)]
    gap[~same] = np.inf
    return {"reuse": {int(w): float(np.mean(gap <= w)) for w in windows}, "fetches": int(len(pc))}


def gather_locality(n: int) -> int:
    """Informational (CPU only): how much a one-time vertex relabelling would let L2
    serve the line-search SpMM's neighbour gathers on the benchmark's graph family
    (Erdos-Renyi, average degree 4): reuse fractions of gather_reuse for the natural
    order and for reverse Cuthill-McKee (scipy), D rows of 96 bytes (ld 24, FP32),
    64-byte fetches."""
    import numpy as np
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    import workloads as W
    i, j, _ = W.er_graph(n, 2 * n, 0, "pm1")
    A = sp.coo_matrix((np.ones(len(i)), (i, j)), shape=(n, n))
    A = (A + A.T).tocsr()
    windows = [20_000, 50_000, 100_000, 200_000]
    out = {}
    for name in ("natural", "rcm"):
        t = time.perf_counter()
        B = A
        if name == "rcm":
            perm = reverse_cuthill_mckee(A, symmetric_mode=True)
            B = A[perm][:, perm].tocsr()
        out[name] = {**gather_reuse(B.indptr, B.indices, windows), "seconds": time.perf_counter() - t}
    print(json.dumps({"analysis": "gather_locality", "n": n, "edges": 2 * n, "row_bytes": 96, "fetch_bytes": 64,
                      "window_unit": "rows processed", **out}), flush=True)
    return 0


def spmm_vs_cusparse(n: int) -> int:
    """C D with the library's SpMM entry point and with cuSPARSE (torch's CSR
    matmul) on the same CSR and D: CUDA events over 20 calls after 3, outputs
    compared.  Informational comparator, not a bench line."""
    import torch
    import workloads as W
    import paper_2407_15049_gb300 as L
    L.load()
    r = 24
    inst = W.maxcut_instance(n, W.er_graph(n, 2 * n, 0, "pm1"))
    s = torch.cuda.current_stream()
    ctx = L.lorads_create(inst, stream=s.cuda_stream)
    try:
        ld = L.padded_ld(r)
        g = torch.Generator(device="cuda")
        g.manual_seed(0)
        D = torch.randn(n, ld, dtype=torch.float32, device="cuda", generator=g)
        out = torch.empty_like(D)
        Cs = torch.sparse_csr_tensor(torch.as_tensor(inst.rowptr, device="cuda").to(torch.int32),
                                     torch.as_tensor(inst.colind, device="cuda").to(torch.int32),
                                     torch.as_tensor(inst.val, device="cuda").to(torch.float32), size=(n, n))
        nnz = int(inst.rowptr[-1])
        alg = nnz * 8 + 4 * (n + 1) + 2 * n * ld * 4

        def timeit(fn, reps=20):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        t_lib = timeit(lambda: L.lorads_spmm(ctx, D, None, out, r=r))
        ref = Cs @ D
        t_cus = timeit(lambda: torch.mm(Cs, D))
        diff = (out - ref).abs().max().item() / ref.abs().max().item()
    finally:
        L.lorads_destroy(ctx)
    print(json.dumps({"comparator": "spmm_vs_cusparse", "n": n, "r": r, "nnz": nnz, "library_ms": t_lib,
                      "cusparse_ms": t_cus, "library_GBps": alg / t_lib / 1e6, "cusparse_GBps": alg / t_cus / 1e6,
                      "max_rel_diff": diff}), flush=True)
    return 0


def l2_fetch_limit(set_bytes: int = 0) -> int | None:
    """The current context's L2 fetch granularity limit in bytes (the driver API's
    CU_LIMIT_MAX_L2_FETCH_GRANULARITY), after setting it to set_bytes when that is
    nonzero; None when the driver library cannot be queried."""
    import ctypes
    import torch
    torch.zeros(1, device="cuda")                 # the primary context, current on this thread
    torch.cuda.synchronize()
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError:
        return None
    limit_id = ctypes.c_int(5)                    # CU_LIMIT_MAX_L2_FETCH_GRANULARITY
    if set_bytes:
        rc = cu.cuCtxSetLimit(limit_id, ctypes.c_size_t(set_bytes))
        if rc != 0:
            raise RuntimeError(f"cuCtxSetLimit(L2 fetch granularity, {set_bytes}) failed: CUresult {rc}")
    v = ctypes.c_size_t(0)
    return int(v.value) if cu.cuCtxGetLimit(ctypes.byref(v), limit_id) == 0 else None


def kernel_probe(args) -> int:
    """Per-kernel CUDA-event times of the first ITERS iterations of a host-stepped solve
    (the same kernels and decisions as the graph path), twice; one JSON line each."""
    import torch
    import paper_2407_15049_gb300 as L
    L.load()
    code = {"fp64": L.LORADS_FP64, "mixed": L.LORADS_MIXED, "df64": L.LORADS_DF64, "fp32": L.LORADS_FP32}[args.prec]
    inst, R0, _ = build_instance(args.workload)
    R0d = torch.as_tensor(R0, device="cuda")
    limit = l2_fetch_limit(args.l2_fetch_limit)
    for rep in range(2):
        ctx = L.lorads_create(inst, L.default_params(prec=code, verbose=2, max_outer=10**6, max_inner=args.kernel_probe,
                                                     rank_update_threshold=10**6, lbfgs_mem=args.lbfgs_mem))
        res = L.lorads_solve(ctx, R0d, on_device=True, max_total_inner=args.kernel_probe)
        t = L.lorads_kernel_times(ctx)
        L.lorads_destroy(ctx)
        print(json.dumps({"workload": args.workload, "prec": args.prec, "lbfgs_mem": args.lbfgs_mem, "rep": rep,
                          "iters": res["inner_iters"], "l2_fetch_limit": limit,
                          "kernels_ms": {k: v[0] for k, v in t.items()}}), flush=True)
    return 0


SCALE_HOST_NEED_GB = 100.0      # generation (~45 GB at 1.7e8) plus the host mirrors of lorads_create


def _host_available_gb() -> float:
    """Memory this process may still take: MemAvailable, capped by a cgroup v2 limit."""
    avail = float("inf")
    try:
        for line in Path("/proc/meminfo").read_text().splitlines():
            if line.startswith("MemAvailable:"):
                avail = float(line.split()[1]) * 1024 / 1e9
    except OSError:
        pass
    try:
        lim = Path("/sys/fs/cgroup/memory.max").read_text().strip()
        if lim != "max":
            cur = float(Path("/sys/fs/cgroup/memory.current").read_text().strip())
            avail = min(avail, (float(lim) - cur) / 1e9)
    except (OSError, ValueError):
        pass
    return avail


def scale_device_bytes(n: int, nnz: int, ld: int, T: int) -> float:
    """Device bytes of a mixed-form solve of a MaxCut instance (one diagonal constraint per
    row): the solver state (R, C R double-float; D, C D, G and 2T history slots FP32),
    C (row pointers, columns, FP64 / FP32 / double-float values), the per-row constraint
    arrays and their state, and the err2 Lanczos vectors (three n x 4 FP64 blocks)."""
    nl = n * ld
    state = nl * (2 * 8 + 3 * 4 + 2 * T * 4)
    c = (n + 1) * 8 + nnz * (4 + 8 + 4 + 8)
    rows = n * (4 + 8 + 4 + 8 + 8 + 4 + 4 + 8 + 4 + 8 + 8) + n * (8 + 8 + 8 + 4)
    lanczos = 3 * n * 4 * 8
    return float(state + c + rows + lanczos)


def run_scale(args) -> int:
    """One timed solve of a workload at the size of the largest MaxCut of Table 4: the
    mixed form, the rank fixed at the workload's r and two stored L-BFGS pairs (the state
    then fills most of HBM), the start drawn on the device.  Checks host and device memory
    before it starts and prints an ``unavailable`` line when either is short."""
    import torch
    import paper_2407_15049_gb300 as L
    cfg = WORKLOADS[args.workload]
    n, r, T = cfg["n"], cfg["r"], cfg["lbfgs_mem"]
    nnz = n + 2 * cfg["edges"]
    ld = L.padded_ld(r)
    head = {"metric": f"time to rel. KKT 1e-5 (MaxCut ER n={n:.2g}, r={r})", "workload": args.workload}
    host = _host_available_gb()
    need = scale_device_bytes(n, nnz, ld, T)
    if host < SCALE_HOST_NEED_GB:
        print(json.dumps({**head, "unavailable": f"host memory: {host:.0f} GB available, "
                          f"{SCALE_HOST_NEED_GB:.0f} GB needed"}), flush=True)
        return 0
    free_b, total_b = torch.cuda.mem_get_info()
    if free_b < need + 4e9:
        print(json.dumps({**head, "unavailable": f"device memory: {free_b / 1e9:.0f} GB free, "
                          f"{need / 1e9:.0f} + 4 GB needed"}), flush=True)
        return 0
    L.load()
    inst, _, gen_s = build_instance(args.workload, with_start=False)
    stream = torch.cuda.Stream()
    params = L.default_params(prec=L.LORADS_MIXED, compute_err2=1, admm_switch=args.admm_switch,
                              lbfgs_mem=T, rank_update_threshold=10**6, time_limit=args.scale_time_limit, seed=1)
    with torch.cuda.stream(stream):
        t = time.perf_counter()
        ctx = L.lorads_create(inst, params, stream=stream.cuda_stream)
        create_s = time.perf_counter() - t
        # warm-up: a capped solve (graph capture, first launches)
        L.lorads_solve(ctx, None, r0=r, max_total_inner=args.warmup_iters)
        torch.cuda.synchronize()
        used_b = total_b - torch.cuda.mem_get_info()[0]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            torch.cuda.synchronize()
            ev0.record(stream)
            res = L.lorads_solve(ctx, None, r0=r)
            ev1.record(stream)
            torch.cuda.synchronize()
        L.lorads_destroy(ctx)
    secs = ev0.elapsed_time(ev1) / 1e3
    it_bytes = sum(kernel_bytes(f, n, ld, nnz, n, 8, 4, T) for f in ("k_dir", "k_spmm_c(CD,ls)", "k_update(step)"))
    peak, kind = measured_peaks()
    per_it = secs / max(res["inner_iters"], 1)
    print(json.dumps({
        **head, "value": secs, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 1, "warmup_iters": args.warmup_iters,
        "higher_is_better": False, "dtype": "mixed (double-float R and C R, f32 work arrays)", "data": "synthetic",
        "config": {"workload": args.workload, "description": cfg["desc"], "n": n, "m": n, "nnz_C": nnz, "rank": r,
                   "lbfgs_mem": T, "rank_rule": "off (rank fixed)", "two_stage": {"admm_switch": args.admm_switch},
                   "start": "cold (unit rows drawn on the device, seed 1)", "tolerance": 1e-5},
        "solve": {k: res[k] for k in ("status_name", "inner_iters", "outer_iters", "admm_iters", "cg_steps",
                                      "primal_obj", "err1", "err2", "err3", "rank")},
        "per_iteration": {"ms_upper_bound": per_it * 1e3, "algorithmic_bytes": it_bytes,
                          "algorithmic_gbs_lower_bound": it_bytes / per_it / 1e9,
                          "frac_of_peak_lower_bound": it_bytes / per_it / 1e9 / peak, "peak_gbs": peak,
                          "peak_kind": kind,
                          "note": "solve time over L-BFGS iterations: the outer steps, the ADMM stage and the "
                                  "final err2 are charged to the iterations too"},
        "memory": {"device_used_gb": used_b / 1e9, "device_estimate_gb": need / 1e9,
                   "device_total_gb": total_b / 1e9, "host_available_gb_at_start": host},
        "setup_s": {"generate": gen_s, "create": create_s},
        "clocks": clk.summary(),
        "context": "Table 4 reports 158 s on an H100 for the k-mer graph kmer_A2a (n = 170,728,175); "
                   "a different graph, machine and precision",
    }), flush=True)
    return 0


def main():
    args = _args()
    if args.kernel_probe:
        return kernel_probe(args)
    if WORKLOADS.get(args.workload, {}).get("scale"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle is not run at this size "
                              "(hours per iteration)"}), flush=True)
            return 0
        return run_scale(args)
    if args.spmm_vs_cusparse:
        return spmm_vs_cusparse(args.spmm_vs_cusparse)
    if args.gather_locality:
        return gather_locality(args.gather_locality)
    if args.workload in BATCH_WORKLOADS:
        return run_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
