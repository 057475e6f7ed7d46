#!/usr/bin/env python
"""Throughput of the CPWL evaluation path on GB300.

Workload (one "step", the whole path over one batch of synthetic input): the
Gaussian exp(-x^2/2) on [-4, 4], the Lorentzian 1/(1+x^2) on [-10, 10] and
J0 on [0, 50], each with N = 256, 1024 and 4096 intervals; for every
(function, N): design of the nearly optimal partition (FP64 density, scan,
inversion), vertex values of both pi_T and P_T (FP64), in-place rebuild of
both tables, and evaluation of two query sets of 2^28 FP32 points each
(uniform on the domain, seed 1; normal(0, 1.5) clipped to the domain,
seed 2) through both tables.  Query sets are 1 GiB each (larger than L2), so
no L2 flush is needed between launches.

Metric: G PWL evaluations per second (whole job), next to the achieved HBM
bandwidth of the evaluation kernel (8 bytes per query) against the measured
copy bandwidth, the max error vs FP64 f, and fwd+bwd evaluations per second.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm of this build).  Under torchrun every rank runs
the same workload on its own GPU (independent replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G PWL evals/s + HBM GB/s at stated max err vs FP64 f; fwd+bwd evals/s"
FUNC_NAMES = ("gaussian", "lorentzian", "bessel_j0")
NS = (256, 1024, 4096)
FORMS = ("interp", "project")
BYTES_FWD = 8   # 4 B of x in, 4 B of y out per query
BYTES_BWD = 12  # x, gy in, gx out
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "eval_kernel_traffic.txt")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2m", type=int, default=28, help="queries per set (log2)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-log2", type=int, default=24,
                    help="queries per function of the single-thread oracle timing (log2)")
    ap.add_argument("--fwd-bwd-steps", type=int, default=3)
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the precision, Table I, channel-wise and batched measurements of the default line")
    ap.add_argument("--report", default=None,
                    choices=[None, "variants", "channels", "batched", "backward", "table1"],
                    help="variants: per-table throughput of every evaluation path and the error of each "
                         "vertex-table precision (one JSON line)")
    ap.add_argument("--k-cells", type=int, default=0, help="cell count of the tables in --report variants")
    ap.add_argument("--rows", type=int, default=65536, help="rows of x in --report channels")
    ap.add_argument("--batch-funcs", type=int, default=4096, help="functions in --report batched")
    ap.add_argument("--batch-m", type=int, default=16, help="density cells per interval in --report batched")
    ap.add_argument("--batch-cpk", type=int, default=0,
                    help="--report batched: index cells per knot (0: the library's default)")
    ap.add_argument("--no-per-function", action="store_true",
                    help="--report batched: skip the one-table-per-function comparison")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# distributed plumbing (independent replicas; barrier + max over ranks)
# ----------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def replica_throughput(dist, ms: float, evals_per_step: int, steps: int):
    """Whole-job throughput of independent replicas (weak scaling): every rank
    ran evals_per_step x steps evaluations and the job took the slowest rank's
    time.  Returns (G evals/s over all ranks, that time in ms)."""
    ms_max = dist.max(ms)
    return dist.world * evals_per_step * steps / (ms_max / 1e3) / 1e9, ms_max


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": float(max(power))}


# ----------------------------------------------------------------------------
# FP64 reference f for the error report (numpy / scipy, not the oracle)
# ----------------------------------------------------------------------------
def f64(name, x):
    if name == "gaussian":
        return np.exp(-0.5 * x * x)
    if name == "lorentzian":
        return 1.0 / (1.0 + x * x)
    from scipy.special import j0
    return j0(x)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


EVAL_SOURCES = ("pwl_eval.cu", "pwl_stream.cuh", "pwl_common.cuh", "pwl_table.cuh")


def eval_source_hash() -> str:
    """First 16 hex digits of the SHA-256 of the evaluation kernel's sources
    (the .cu and the headers its kernel code comes from), concatenated, with
    comments and whitespace removed: an edit of a comment keeps the record."""
    import re
    h = hashlib.sha256()
    for name in EVAL_SOURCES:
        with open(os.path.join(ROOT, "paper_1510_02975_gb300", "csrc", name), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(re.sub(r"\s+", "", text).encode())
    return h.hexdigest()[:16]


def recorded_traffic():
    """Per-launch DRAM bytes of the evaluation kernel from the last ncu
    capture, or None if the kernel source changed since."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    vals = {}
    for ln in open(TRAFFIC_FILE):
        if "=" in ln and not ln.startswith("#"):
            k, v = ln.split("=", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256_16") != eval_source_hash():
        return None
    try:
        return float(vals["bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
class Workload:
    def __init__(self, log2m: int):
        import torch

        import paper_1510_02975_gb300 as pwl
        from paper_1510_02975_gb300 import workloads as W
        self.torch, self.pwl, self.W = torch, pwl, W
        self.m = 1 << log2m
        self.funcs = [W.PAPER_FUNCTIONS[n] for n in FUNC_NAMES]
        self.x = {}
        for fi, f in enumerate(self.funcs):
            self.x[(fi, "uniform")] = W.uniform_queries(f, self.m, seed=1)
            self.x[(fi, "normal")] = W.normal_queries(f, self.m, seed=2)
        self.y = torch.empty(self.m, dtype=torch.float32, device="cuda")
        self.items = []  # (fi, N, knots, vi, vp, ws_d, ws_p, table_i, table_p)
        self.wsp2 = []   # a second projection workspace per item (the two forms run side by side)
        lib = pwl._capi.load()
        for fi, f in enumerate(self.funcs):
            for N in NS:
                kn = pwl.pwl_design(f, N)
                vi = pwl.pwl_project(f, kn, "interp")
                vp = pwl.pwl_project(f, kn, "project")
                wsd = torch.empty(lib.pwl_design_workspace_size(N, 0), dtype=torch.uint8, device="cuda")
                wsp = torch.empty(lib.pwl_project_workspace_size(N), dtype=torch.uint8, device="cuda")
                ti = pwl.Table(kn, vi)
                tp = pwl.Table(kn, vp)
                self.items.append((fi, N, kn, vi, vp, wsd, wsp, ti, tp))
                self.wsp2.append(torch.empty_like(wsp))
        torch.cuda.synchronize()
        self.capture_design()
        self.evals_per_step = len(self.items) * len(FORMS) * 2 * self.m

    def _design_item(self, k, st, side):
        """Item k on stream st: the design, then the interpolant's values and
        its table rebuild on st and, side by side on `side`, the projection's
        values and its table rebuild (both need only the knots)."""
        torch, pwl = self.torch, self.pwl
        fi, N, kn, vi, vp, wsd, wsp, ti, tp = self.items[k]
        f = self.funcs[fi]
        with torch.cuda.stream(st):
            pwl.pwl_design(f, N, 0, "fp64", knots=kn, workspace=wsd)
        side.wait_stream(st)
        with torch.cuda.stream(st):
            pwl.pwl_project(f, kn, "interp", values=vi, workspace=wsp)
            ti.update(kn, vi)
        with torch.cuda.stream(side):
            pwl.pwl_project(f, kn, "project", values=vp, workspace=self.wsp2[k])
            tp.update(kn, vp)
        st.wait_stream(side)

    def capture_design(self):
        """Design, both projections and both table rebuilds of every
        (function, N) captured once into a CUDA graph: a branch per
        (function, N), forked after the design into one branch per form; a
        step replays it."""
        torch = self.torch
        cur = torch.cuda.current_stream()
        for k in range(len(self.items)):  # eager pass: sets kernel attributes outside capture
            self._design_item(k, cur, cur)
        torch.cuda.synchronize()
        self.streams = [(torch.cuda.Stream(), torch.cuda.Stream()) for _ in self.items]
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
            main = torch.cuda.current_stream()
            for k, (st, side) in enumerate(self.streams):
                st.wait_stream(main)
                self._design_item(k, st, side)
            for st, _ in self.streams:
                main.wait_stream(st)
        torch.cuda.synchronize()

    def design_and_tables(self):
        self.graph.replay()

    def step(self, events=None):
        self.design_and_tables()
        pwl = self.pwl
        for fi, N, kn, vi, vp, wsd, wsp, ti, tp in self.items:
            for t in (ti, tp):
                for qs in ("uniform", "normal"):
                    if events is not None:
                        e0 = self.torch.cuda.Event(enable_timing=True)
                        e1 = self.torch.cuda.Event(enable_timing=True)
                        e0.record()
                        pwl.pwl_eval(t.handle, self.x[(fi, qs)], self.y)
                        e1.record()
                        events.append((e0, e1))
                    else:
                        pwl.pwl_eval(t.handle, self.x[(fi, qs)], self.y)

    def launch_keys(self):
        """Names of a step's evaluation launches, in launch order."""
        keys = []
        for fi, N, kn, vi, vp, wsd, wsp, ti, tp in self.items:
            for form in FORMS:
                for qs in ("uniform", "normal"):
                    keys.append(f"{FUNC_NAMES[fi]}/{form}/N{N}/{qs}")
        return keys

    def error_report(self, sample=1 << 20):
        """max |y - f| (FP64 f) and max |y - v64| (FP64 PWL) on a sample of
        each query set, per function and form, at N = 4096."""
        torch = self.torch
        out = {}
        for fi, N, kn, vi, vp, wsd, wsp, ti, tp in self.items:
            if N != NS[-1]:
                continue
            name = FUNC_NAMES[fi]
            k64 = kn.cpu().numpy()
            for form, t, v in (("interp", ti, vi), ("project", tp, vp)):
                v64 = v.cpu().numpy()
                ef, ep = 0.0, 0.0
                for qs in ("uniform", "normal"):
                    xs = self.x[(fi, qs)][:sample]
                    y = self.pwl.pwl_eval(t.handle, xs).cpu().numpy().astype(np.float64)
                    xd = xs.cpu().numpy().astype(np.float64)
                    ef = max(ef, float(np.abs(y - f64(name, xd)).max()))
                    ep = max(ep, float(np.abs(y - np.interp(xd, k64, v64)).max()))
                out[f"{name}/{form}/N{N}"] = {"max_err_vs_f64_f": ef, "max_err_vs_f64_pwl": ep}
        torch.cuda.synchronize()
        return out


def run_ours(args):
    import torch
    dist = Dist()
    torch.cuda.set_device(dist.local)
    dist.init("nccl")
    from paper_1510_02975_gb300 import _build
    _build.build()
    wl = Workload(args.log2m)
    for _ in range(max(args.warmup, 3)):
        wl.step()
    torch.cuda.synchronize()
    dist.barrier()
    clocks = ClockSampler(dist.local)
    clocks.start()
    time.sleep(0.3)
    events = []
    torch.cuda.synchronize()
    dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        wl.step(events)
    t1.record()
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    value, ms_max = replica_throughput(dist, ms, wl.evals_per_step, args.steps)
    launch_ms = [a.elapsed_time(b) for a, b in events]
    avg_launch_s = float(np.mean(launch_ms)) / 1e3
    per_table = {}
    for k, ms_k in zip(wl.launch_keys() * args.steps, launch_ms):
        per_table.setdefault(k, []).append(ms_k)
    per_table_gbs = {k: round(BYTES_FWD * wl.m / (float(np.mean(v)) / 1e3) / 1e9, 1) for k, v in per_table.items()}
    peak, peak_kind = measured_peaks()
    achieved = BYTES_FWD * wl.m / avg_launch_s / 1e9

    # time of the design / projection / table rebuild part of a step
    torch.cuda.synchronize()
    d0 = torch.cuda.Event(enable_timing=True)
    d1 = torch.cuda.Event(enable_timing=True)
    d0.record()
    for _ in range(3):
        wl.design_and_tables()
    d1.record()
    torch.cuda.synchronize()
    design_ms = d0.elapsed_time(d1) / 3

    # fwd + bwd on the same tables and query sets
    fb = fwd_bwd(wl, args.fwd_bwd_steps)
    errors = wl.error_report()
    ceiling = compute_ceiling(wl)
    small = small_case(wl)
    extra = {}
    if not args.no_configs:
        extra["precision"] = precision_measure(wl)
        extra["table_I"] = table_one_measure(wl)
        extra["channels"] = channels_measure()
        extra["batched"] = batched_measure(steps=3)
    e2e = None if args.no_e2e else run_e2e(wl, args.e2e_steps)
    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_sample_log2)
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "G evals/s",
        "n_gpus": dist.world,
        "steps": args.steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": round(ms_max / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic: seeded uniform and clipped-normal FP32 queries; analytic functions",
        "config": {
            "workload": "3 functions (Gaussian [-4,4], Lorentzian [-10,10], J0 [0,50]) x N in {256,1024,4096} "
                        "intervals x {pi_T, P_T}; per step FP64 design + projection + table rebuild, then "
                        f"2 query sets of 2^{args.log2m} FP32 (uniform, normal(0,1.5) clipped) per table",
            "evals_per_step": wl.evals_per_step,
            "queries_per_set": wl.m,
            "l2": "inputs larger than L2 (1 GiB per query set); no flush",
            "parallelism": f"replicas x{dist.world}",
        },
        "roofline": {
            "bound": "hbm",
            "kernel": "eval_kernel<float>",
            "achieved": round(achieved, 1),
            "peak": peak,
            "peak_kind": f"{peak_kind} copy bandwidth",
            "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": recorded_traffic(),
            "bytes_per_launch_algorithmic": BYTES_FWD * wl.m,
            "avg_launch_ms": round(avg_launch_s * 1e3, 4),
            "launches_timed": len(launch_ms),
        },
        "design_ms_per_step": round(design_ms, 3),
        "per_table_forward_gbs": per_table_gbs,
        "fwd_bwd": fb,
        "errors_N4096": errors,
        "compute_ceiling": ceiling,
        "small_case": small,
        "gpu_launches": gpu_launches_per_step(wl) * args.steps,
        "clocks": clk,
        **extra,
    }
    if e2e is not None:
        line["e2e"] = e2e
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()


def compute_ceiling(wl, m: int = 1 << 28, reps: int = 5):
    """Algorithm 1 on 2^28 queries generated in registers (no query loads,
    no result stores): the compute ceiling in ps per evaluation, on the
    Gaussian N = 256 P_T table and the N = 4096 one."""
    torch, pwl = wl.torch, wl.pwl
    out = {}
    acc = torch.zeros(1, dtype=torch.float64, device="cuda")
    for fi, N, kn, vi, vp, wsd, wsp, ti, tp in wl.items:
        if fi != 0 or N not in (256, 4096):
            continue
        sec = time_launches(lambda: pwl.pwl_eval_synthetic(tp.handle, m, 7, acc), reps)
        out[f"gaussian/project/N{N}"] = {"ps_per_eval": round(sec / m * 1e12, 3),
                                         "G_evals_per_s": round(m / sec / 1e9, 1)}
    return out


def precision_measure(wl, N: int = 1024, reps: int = 3, sample: int = 1 << 20) -> dict:
    """Vertex tables in FP32 / BF16 / FP16 with the FP32 FMA lerp (pwl_eval)
    and with the texture filter (fixed-point weight; FP32 texels, FP16 for
    FP16 tables), at N = 1024 on the 2^28 uniform query set of each function
    (P_T values): throughput and fraction of the measured copy bandwidth,
    and max / RMS error against FP64 f and against the FP64 CPWL function
    (on the first 2^20 queries)."""
    torch, pwl = wl.torch, wl.pwl
    peak, _ = measured_peaks()
    out = {}
    for fi, n, kn, vi, vp, wsd, wsp, ti, tp in wl.items:
        if n != N:
            continue
        name = FUNC_NAMES[fi]
        x = wl.x[(fi, "uniform")]
        xs = x[:sample]
        xh = xs.cpu().numpy().astype(np.float64)
        fx = f64(name, xh)
        k64, v64 = kn.cpu().numpy(), vp.cpu().numpy()
        pw = np.interp(xh, k64, v64)
        for dt in ("fp32", "bf16", "fp16"):
            t = pwl.Table(kn, vp, dt)
            for lerp, mode_fn in (("fma", lambda xx, yy: pwl.pwl_eval(t.handle, xx, yy)),
                                  ("texture", lambda xx, yy: pwl.pwl_eval_variant(t.handle, 1, xx, yy))):
                sec = time_launches(lambda: mode_fn(x, wl.y), reps)
                gbs = BYTES_FWD * wl.m / sec / 1e9
                yv = mode_fn(xs, torch.empty_like(xs)).cpu().numpy().astype(np.float64)
                ef, ep = yv - fx, yv - pw
                out[f"{name}/{dt}/{lerp}"] = {
                    "gbs": round(gbs, 1), "frac_of_peak": round(gbs / peak, 4),
                    "max_err_vs_f64_f": float(np.abs(ef).max()), "rms_err_vs_f64_f": float(np.sqrt(np.mean(ef * ef))),
                    "max_err_vs_f64_pwl": float(np.abs(ep).max()),
                    "rms_err_vs_f64_pwl": float(np.sqrt(np.mean(ep * ep)))}
            t.close()
    return {"N": N, "form": "project", "queries": wl.m, "error_sample": sample, "results": out}


# The paper's Table I (GTX 580, ps per evaluation, Gaussian), for context
PAPER_TABLE_I_PS = {
    "expf": 33.3, "__expf": 14.2, "uniform_manual": 19.75, "uniform_texture": 7.85,
    "optimized_manual": {"32": 142.0, "64": 161.9, "128": 181.8, "256": 203.1, "512": 224.1},
    "optimized_texture": {"32": 122.7, "64": 142.9, "128": 163.2, "256": 188.3, "512": 211.1},
    "lorentzian_division": 19.5, "lorentzian_fast_division": 9.2, "j0_cuda": 78.0, "j0_asymptotic_sfu": 42.0,
}


def table_one_measure(wl, m: int = 1 << 28, reps: int = 3) -> dict:
    """Table I on this GPU: ps per evaluation with queries generated in
    registers (no memory traffic; the paper's synthetic benchmark) for every
    row: the direct Gaussian with expf and __expf, the uniform partition
    (cell lookup with the FMA lerp; texture coordinate straight from x), the
    nearly optimal partition with the paper's unrolled binary search (FMA
    lerp; texture filter) and with this library's cell index (FMA; texture),
    at N + 1 = 32 .. 512 knots of the Gaussian on [-4, 4] (P_T values); plus
    the direct Lorentzian (IEEE and fast division) and J0 (j0f; the one-term
    asymptotic form with SFU cos and rsqrt).  Then the same direct kernels
    streaming 2^28 FP32 queries from HBM (GB/s, 8 bytes per query)."""
    torch, pwl, W = wl.torch, wl.pwl, wl.W
    acc = torch.zeros(1, dtype=torch.float64, device="cuda")
    ps = lambda sec: round(sec / m * 1e12, 3)
    gauss, lor = W.PAPER_FUNCTIONS["gaussian"], W.PAPER_FUNCTIONS["lorentzian"]
    j0 = W.PAPER_FUNCTIONS["bessel_j0"]
    rows = {}
    for key, f, meth in (("expf", gauss, "library"), ("__expf", gauss, "fast"),
                         ("lorentzian_division", lor, "library"), ("lorentzian_fast_division", lor, "fast"),
                         ("j0_cuda", j0, "library"), ("j0_asymptotic_sfu", j0, "fast")):
        rows[key] = ps(time_launches(lambda: pwl.pwl_direct_synthetic(f, meth, m, 11, acc), reps))
    cols = {k: {} for k in ("uniform_manual", "uniform_texture", "optimized_search_manual",
                            "optimized_search_texture", "optimized_cells_manual", "optimized_cells_texture")}
    a, b = gauss["a"], gauss["b"]
    for knots in (32, 64, 128, 256, 512):
        n = knots - 1
        ku = torch.tensor(a + (b - a) * np.arange(n + 1) / n, dtype=torch.float64, device="cuda")
        ku[-1] = b
        tu = pwl.Table(ku, pwl.pwl_project(gauss, ku, "project"), "fp32", 2 * n)
        ko = pwl.pwl_design(gauss, n)
        to = pwl.Table(ko, pwl.pwl_project(gauss, ko, "project"))
        for key, t, mode in (("uniform_manual", tu, None), ("uniform_texture", tu, 5),
                             ("optimized_search_manual", to, 0), ("optimized_search_texture", to, 4),
                             ("optimized_cells_manual", to, None), ("optimized_cells_texture", to, 1)):
            if mode is None:
                fn = lambda: pwl.pwl_eval_synthetic(t.handle, m, 11, acc)
            else:
                fn = lambda: pwl.pwl_eval_synthetic_variant(t.handle, mode, m, 11, acc)
            cols[key][str(knots)] = ps(time_launches(fn, reps))
        tu.close()
        to.close()
    rows.update(cols)
    peak, _ = measured_peaks()
    stream = {}
    for key, fi, meth in (("expf", 0, "library"), ("__expf", 0, "fast"), ("lorentzian_division", 1, "library"),
                          ("lorentzian_fast_division", 1, "fast"), ("j0_cuda", 2, "library"),
                          ("j0_asymptotic_sfu", 2, "fast")):
        f = W.PAPER_FUNCTIONS[FUNC_NAMES[fi]]
        x = wl.x[(fi, "uniform")]
        sec = time_launches(lambda: pwl.pwl_direct_eval(f, meth, x, wl.y), reps)
        gbs = BYTES_FWD * wl.m / sec / 1e9
        stream[key] = {"gbs": round(gbs, 1), "frac_of_peak": round(gbs / peak, 4),
                       "G_evals_per_s": round(wl.m / sec / 1e9, 1)}
    return {"queries": m, "ps_per_eval_register_generated": rows, "direct_streaming_2e28": stream,
            "paper_gtx580_ps": PAPER_TABLE_I_PS}


def small_case(wl, reps: int = 50):
    """The small configuration: exp(-x^2/2) on [-4, 4] with 63 intervals (64
    knots), 10^6 uniform FP32 queries (seed 0), both forms: time per
    evaluation launch and the max error against FP64 f."""
    torch, pwl, W = wl.torch, wl.pwl, wl.W
    sc = W.SMALL
    f = sc["func"]
    x = W.uniform_queries(f, sc["m"], seed=sc["seed"])
    y = torch.empty_like(x)
    kn = pwl.pwl_design(f, sc["n_intervals"])
    out = {"n_intervals": sc["n_intervals"], "queries": sc["m"]}
    xd = x.cpu().numpy().astype(np.float64)
    for form in FORMS:
        t = pwl.Table(kn, pwl.pwl_project(f, kn, form))
        sec = time_launches(lambda: pwl.pwl_eval(t.handle, x, y), reps)
        err = float(np.abs(y.cpu().numpy().astype(np.float64) - f64("gaussian", xd)).max())
        # the same launches replayed from a CUDA graph: device time per launch
        # without the per-call host work (argument checks, ctypes, launch)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(reps):
                pwl.pwl_eval(t.handle, x, y)
        graph.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        gsec = e0.elapsed_time(e1) / reps / 1e3
        out[form] = {"us_per_launch": round(sec * 1e6, 2), "G_evals_per_s": round(sc["m"] / sec / 1e9, 1),
                     "us_per_launch_graph": round(gsec * 1e6, 2),
                     "G_evals_per_s_graph": round(sc["m"] / gsec / 1e9, 1), "max_err_vs_f64_f": err}
        del graph
        t.close()
    return out


def gpu_launches_per_step(wl) -> int:
    # per (function, N): design 5 (descriptor setup + density, chunk scan,
    # cumulative, inversion), interpolant values 2, projection 3, two table
    # rebuilds of 3 kernels, four evaluations
    per_item = 5 + 2 + 3 + 6 + 4
    return per_item * len(wl.items)


def fwd_bwd(wl, steps):
    torch, pwl = wl.torch, wl.pwl
    gy = wl.W.upstream_grad((wl.m,), seed=5)
    gx = torch.empty_like(gy)
    bufs = []
    for fi, N, kn, vi, vp, wsd, wsp, ti, tp in wl.items:
        for t in (ti, tp):
            gv = torch.zeros(N + 1, device="cuda")
            gk = torch.zeros(N + 1, device="cuda")
            ws = torch.empty(pwl._capi.load().pwl_eval_backward_workspace_size(t.handle), dtype=torch.uint8,
                             device="cuda")
            bufs.append((fi, t, gv, gk, ws))

    def one():
        for fi, t, gv, gk, ws in bufs:
            for qs in ("uniform", "normal"):
                x = wl.x[(fi, qs)]
                pwl.pwl_eval(t.handle, x, wl.y)
                pwl.pwl_eval_backward(t.handle, x, gy, gx, gv, gk, ws)

    one()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        one()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    evals = len(bufs) * 2 * wl.m * steps
    # the backward calls alone, per table size and query set (CUDA events
    # around each call: the backward kernel and its row reduction)
    bwd = {}
    for fi, t, gv, gk, ws in bufs:
        N = int(t.info["n_intervals"])
        for qs in ("uniform", "normal"):
            x = wl.x[(fi, qs)]
            sec = time_launches(lambda: pwl.pwl_eval_backward(t.handle, x, gy, gx, gv, gk, ws), 2)
            bwd.setdefault(f"N{N}/{qs}", []).append(sec)
    peak, _ = measured_peaks()
    by_n = {k: {"gbs": round(BYTES_BWD * wl.m / float(np.mean(v)) / 1e9, 1),
                "frac_of_peak": round(BYTES_BWD * wl.m / float(np.mean(v)) / 1e9 / peak, 4)} for k, v in bwd.items()}
    gbs = evals * (BYTES_FWD + BYTES_BWD) / (ms / 1e3) / 1e9
    return {"value": round(evals / (ms / 1e3) / 1e9, 3), "unit": "G evals/s (forward + backward)",
            "bytes_per_eval": BYTES_FWD + BYTES_BWD, "gbs": round(gbs, 1), "frac_of_peak": round(gbs / peak, 4),
            "backward_alone": by_n}


def run_e2e(wl, steps):
    """Same metric through the public API with host buffers: every step copies
    its query sets from pinned host memory and reads every result back.  The
    inputs are double-buffered on the device: while a step's evaluations and
    read-backs run, the next step's query sets go up on their own stream (a
    bank is refilled once the evaluations that read it are done), so the host
    link carries both directions at once.  The read-backs run on a third
    stream; two result buffers alternate, each reused only after its previous
    read-back.  The timed region starts with the first step's own uploads and
    holds exactly `steps` steps of uploads and of read-backs."""
    torch, pwl = wl.torch, wl.pwl
    hx = {k: v.cpu().pin_memory() for k, v in wl.x.items()}
    hy = torch.empty(wl.m, dtype=torch.float32).pin_memory()
    banks = [{k: torch.empty(wl.m, dtype=torch.float32, device="cuda") for k in wl.x} for _ in range(2)]
    ys = [torch.empty(wl.m, dtype=torch.float32, device="cuda") for _ in range(2)]
    comp = torch.cuda.current_stream()
    h2d_s, d2h_s = torch.cuda.Stream(), torch.cuda.Stream()
    uploaded = [{k: torch.cuda.Event() for k in wl.x} for _ in range(2)]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]  # the evaluations reading a bank are done
    read = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    for e in consumed:
        e.record(comp)
    for e in read:
        e.record(d2h_s)

    def upload(bank):
        h2d_s.wait_event(consumed[bank])
        with torch.cuda.stream(h2d_s):
            for k in wl.x:
                banks[bank][k].copy_(hx[k], non_blocking=True)
                uploaded[bank][k].record(h2d_s)
        return wl.m * 4 * len(wl.x)

    def step(bank):
        d2h = 0
        dx = banks[bank]
        wl.design_and_tables()
        j = 0
        for fi, N, kn, vi, vp, wsd, wsp, ti, tp in wl.items:
            for t in (ti, tp):
                for qs in ("uniform", "normal"):
                    b = j & 1
                    comp.wait_event(uploaded[bank][(fi, qs)])
                    comp.wait_event(read[b])  # the buffer's previous result has been read
                    pwl.pwl_eval(t.handle, dx[(fi, qs)], ys[b])
                    done[b].record(comp)
                    d2h_s.wait_event(done[b])
                    with torch.cuda.stream(d2h_s):
                        hy.copy_(ys[b], non_blocking=True)
                        read[b].record(d2h_s)
                    d2h += wl.m * 4
                    j += 1
        consumed[bank].record(comp)
        return d2h

    def run(k):
        h2d_s.wait_stream(comp)  # no upload starts before the timed region does
        h2d = upload(0)
        d2h = 0
        for s in range(k):
            if s + 1 < k:
                h2d += upload((s + 1) % 2)  # the next step's inputs, under this step's work
            d2h += step(s % 2)
        comp.wait_stream(d2h_s)  # the run ends when its last result is on the host
        return h2d, d2h

    run(2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    h2d, d2h = run(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": round(wl.evals_per_step * steps / (ms / 1e3) / 1e9, 3), "unit": "G evals/s",
            "h2d_bytes_per_step": h2d // steps, "d2h_bytes_per_step": d2h // steps, "steps": steps,
            "overlap": "inputs double-buffered (the next step's uploads under this step's work), "
                       "read-backs on their own stream, two result buffers"}


# ----------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------
def host_threads() -> int:
    """Host CPU threads this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def oracle_eval_threads(k, v, x, threads: int) -> np.ndarray:
    """The oracle's Algorithm 1 over x, split into `threads` contiguous
    ranges evaluated by as many host threads (the C call releases the GIL)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    y = np.empty_like(x)
    bounds = np.linspace(0, x.size, threads + 1).astype(np.int64)

    def work(i):
        y[bounds[i]:bounds[i + 1]] = oracle.evaluate(k, v, x[bounds[i]:bounds[i + 1]])

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(work, range(threads)))
    return y


def oracle_step(sample_log2: int, seed_offset: int = 0, threads: int = 1):
    """One bounded sample of the workload on the FP64 CPU oracle: design and
    both vertex-value forms for all 9 (function, N) (one thread), then
    2^sample_log2 queries of each set through each table (over `threads`
    host threads).  Returns (evals, seconds)."""
    import oracle
    from paper_1510_02975_gb300 import workloads as W
    rng = np.random.default_rng(1234 + seed_offset)
    n = 1 << sample_log2
    evals = 0
    t0 = time.perf_counter()
    for name in FUNC_NAMES:
        f = W.PAPER_FUNCTIONS[name]
        xu = rng.uniform(f["a"], f["b"], n).astype(np.float32).astype(np.float64)
        xn = np.clip(rng.normal(0.0, 1.5, n), f["a"], f["b"]).astype(np.float32).astype(np.float64)
        for N in NS:
            k = oracle.design(f, N)
            for form in FORMS:
                v = oracle.values(f, k, form)
                for xs in (xu, xn):
                    if threads > 1:
                        oracle_eval_threads(k, v, xs, threads)
                    else:
                        oracle.evaluate(k, v, xs)
                    evals += n
    return evals, time.perf_counter() - t0


def cpu_baseline(wl, single_log2: int = 24, n_table: int = 1024):
    """The FP64 C oracle on this host's CPU cores, on the bench's own query
    sets (the 2^28 uniform set of each function, copied to the host):
      - design: the oracle's knots and both vertex-value forms for every
        (function, N) of the workload, one thread, timed apart;
      - single thread: Algorithm 1 (binary search + lerp) through the
        N = 1024 P_T table on the first 2^24 queries of each set;
      - all cores: the same tables on the full 2^28 queries of each set,
        split into contiguous ranges, one per host thread.
    `value` is the all-core evaluation rate."""
    import oracle
    from paper_1510_02975_gb300 import workloads as W
    oracle.build()
    threads = host_threads()
    design = {}
    tables = {}
    for name in FUNC_NAMES:
        f = W.PAPER_FUNCTIONS[name]
        for N in NS:
            t0 = time.perf_counter()
            k = oracle.design(f, N)
            t1 = time.perf_counter()
            oracle.values(f, k, "interp")
            t2 = time.perf_counter()
            v = oracle.values(f, k, "project")
            t3 = time.perf_counter()
            design[f"{name}/N{N}"] = {"design_ms": round((t1 - t0) * 1e3, 2), "interp_ms": round((t2 - t1) * 1e3, 2),
                                      "project_ms": round((t3 - t2) * 1e3, 2)}
            if N == n_table:
                tables[name] = (k, v)
    st_evals = st_sec = mc_evals = mc_sec = 0.0
    for fi, name in enumerate(FUNC_NAMES):
        x = wl.x[(fi, "uniform")].cpu().numpy().astype(np.float64)
        k, v = tables[name]
        t0 = time.perf_counter()
        oracle.evaluate(k, v, x[: 1 << single_log2])
        st_sec += time.perf_counter() - t0
        st_evals += 1 << single_log2
        t0 = time.perf_counter()
        oracle_eval_threads(k, v, x, threads)
        mc_sec += time.perf_counter() - t0
        mc_evals += x.size
        del x
    total_design_ms = sum(d["design_ms"] + d["interp_ms"] + d["project_ms"] for d in design.values())
    return {"value": round(mc_evals / mc_sec / 1e9, 6), "unit": "G evals/s", "cores": threads, "kind": "oracle",
            "sample": f"FP64 C oracle (binary search + lerp) through the N = {n_table} P_T table of each of the 3 "
                      f"functions: all {threads} host threads on the full 2^{int(np.log2(wl.m))} uniform set of "
                      f"each function ({int(mc_evals)} evaluations in {mc_sec:.1f} s, contiguous ranges per thread)",
            "single_thread": {"value": round(st_evals / st_sec / 1e9, 6), "unit": "G evals/s", "cores": 1,
                              "sample": f"first 2^{single_log2} queries of each set ({int(st_evals)} evaluations in "
                                        f"{st_sec:.1f} s)"},
            "design_one_thread": {"total_ms": round(total_design_ms, 1), "per_table": design,
                                  "what": "oracle design (density, cumulative, inversion) and both vertex-value "
                                          "forms per (function, N), M = 64 N, Q = 8"}}


def run_reference(args):
    dist = Dist()
    if dist.rank != 0:
        return
    import oracle
    oracle.build()
    sample = 20
    threads = host_threads()
    for w in range(args.warmup):
        oracle_step(sample, w, threads)
    total_e, total_s = 0, 0.0
    for s in range(args.steps):
        e, sec = oracle_step(sample, 100 + s, threads)
        total_e += e
        total_s += sec
    value = total_e / total_s / 1e9
    line = {
        "metric": METRIC, "value": round(value, 6), "unit": "G evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_s / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded uniform and clipped-normal queries; analytic functions",
        "impl": "reference",
        "config": {"workload": "3 functions x N in {256,1024,4096} x {pi_T, P_T}; design + values on the "
                               f"oracle (one thread), then 2^{sample} queries per (table, query set) per step "
                               f"over {threads} host threads",
                   "evals_per_step": total_e // max(args.steps, 1)},
        "cpu_baseline": {"value": round(value, 6), "unit": "G evals/s", "cores": threads, "kind": "oracle",
                         "sample": f"2^{sample} queries per (table, query set) per step, design included"},
        "e2e": {"value": round(value, 6), "unit": "G evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_launches(fn, reps: int = 5) -> float:
    """Average device time of fn() in seconds (CUDA events, after one warm-up)."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


def run_variants(args):
    """Per-table throughput of the evaluation paths (main cell-index path, the
    paper's binary search, the texture filter) for the three functions and
    N in {256, 1024, 4096}, and, at N = 1024, the error of FP32 / BF16 / FP16
    vertex tables (max and RMS vs FP64 f and vs the FP64 CPWL); then the N
    each function needs for a target L2 error on the nearly optimal and on
    the uniform partition (Results 4-6)."""
    import torch

    import paper_1510_02975_gb300 as pwl
    from paper_1510_02975_gb300 import _build
    from paper_1510_02975_gb300 import workloads as W
    _build.build()
    m = 1 << args.log2m
    y = torch.empty(m, dtype=torch.float32, device="cuda")
    rows = []
    errors = []
    for name in FUNC_NAMES:
        f = W.PAPER_FUNCTIONS[name]
        xs = {"uniform": W.uniform_queries(f, m, seed=1), "normal": W.normal_queries(f, m, seed=2)}
        for N in NS:
            kn = pwl.pwl_design(f, N)
            vp = pwl.pwl_project(f, kn, "project")
            for dt in (("fp32", "bf16", "fp16") if N == 1024 else ("fp32",)):
                t = pwl.Table(kn, vp, dt, args.k_cells)
                for qs, x in xs.items():
                    row = {"func": name, "N": N, "values": dt, "queries": qs, "K": int(t.info["k_cells"]),
                           "n_chain": int(t.info["n_chain"]), "smem_kb": round(t.info["eval_smem_bytes"] / 1024, 1)}
                    row["layout"] = int(t.info["layout"])
                    for label, fn in (("main", lambda: pwl.pwl_eval(t.handle, x, y)),
                                      ("cells8", lambda: pwl.pwl_eval_variant(t.handle, 2, x, y)),
                                      ("cells8_one_side_record", lambda: pwl.pwl_eval_variant(t.handle, 6, x, y)),
                                      ("cells16", lambda: pwl.pwl_eval_variant(t.handle, 3, x, y)),
                                      ("search", lambda: pwl.pwl_eval_variant(t.handle, 0, x, y)),
                                      ("texture", lambda: pwl.pwl_eval_variant(t.handle, 1, x, y))):
                        if dt != "fp32" and label in ("search", "cells8", "cells8_one_side_record", "cells16"):
                            continue
                        sec = time_launches(fn)
                        row[label + "_gbs"] = round(BYTES_FWD * m / sec / 1e9, 1)
                    rows.append(row)
                if N == 1024:
                    k64 = kn.cpu().numpy()
                    v64 = vp.cpu().numpy()
                    xd = xs["uniform"][: 1 << 20]
                    xh = xd.cpu().numpy().astype(np.float64)
                    for label, fn in (("fma", lambda: pwl.pwl_eval(t.handle, xd)),
                                      ("texture", lambda: pwl.pwl_eval_variant(t.handle, 1, xd))):
                        yv = fn().cpu().numpy().astype(np.float64)
                        ef = yv - f64(name, xh)
                        ep = yv - np.interp(xh, k64, v64)
                        errors.append({"func": name, "N": N, "values": dt, "lerp": label,
                                       "max_vs_f64_f": float(np.abs(ef).max()),
                                       "rms_vs_f64_f": float(np.sqrt(np.mean(ef * ef))),
                                       "max_vs_f64_pwl": float(np.abs(ep).max()),
                                       "rms_vs_f64_pwl": float(np.sqrt(np.mean(ep * ep)))})
                t.close()
    # N for a target L2 error on the nearly optimal and on the uniform
    # partition (Results 4-6): the memory the optimised partition saves
    sizing = []
    for name in FUNC_NAMES:
        f = W.PAPER_FUNCTIONS[name]
        i25, isq = (float(v) for v in pwl.pwl_error_constants(f).cpu())
        for target in (1e-4, 1e-6, 1e-8):
            for form in ("interp", "project"):
                n_opt = pwl.pwl_n_for_error(i25, isq, f["a"], f["b"], target, form, False)
                n_uni = pwl.pwl_n_for_error(i25, isq, f["a"], f["b"], target, form, True)
                sizing.append({"func": name, "target_l2": target, "form": form, "N_optimised": n_opt,
                               "N_uniform": n_uni, "uniform_over_optimised": round(n_uni / n_opt, 3)})
    peak, kind = measured_peaks()
    print(json.dumps({"report": "variants", "queries_per_launch": m, "peak_gbs": peak, "peak_kind": kind,
                      "throughput": rows, "errors": errors, "n_for_error": sizing,
                      "uniform_vs_optimised": uniform_vs_optimised(pwl, W, m, y, sizing)}), flush=True)


def uniform_vs_optimised(pwl, W, m, y, sizing):
    """The uniform partition's fast path against the nearly optimal partition
    at equal predicted L2 error (Results 4-6): each table built at the N that
    pwl_n_for_error gives for it; the uniform one with two cells per interval,
    which pwl_eval serves from the 16-byte index (a cell holds at most one
    knot: one record load, a compare and an FMA per query, the direct lookup
    of Section IV made exact at the knots).  Throughput on uniform queries, the index's shared memory,
    and the measured L2 error (midpoint sums of (y - f)^2 on 2^20 points, f in
    FP64 by numpy / scipy) and max error against FP64 f."""
    import torch
    out = []
    for row in sizing:
        if row["target_l2"] not in (1e-4, 1e-6):
            continue
        name, form = row["func"], row["form"]
        f = W.PAPER_FUNCTIONS[name]
        a, b = f["a"], f["b"]
        x = W.uniform_queries(f, m, seed=1)
        n_pts = 1 << 20
        xm = torch.tensor(a + (b - a) * (np.arange(n_pts) + 0.5) / n_pts, dtype=torch.float32, device="cuda")
        xh = xm.cpu().numpy().astype(np.float64)
        fx = f64(name, xh)
        entry = {"func": name, "form": form, "target_l2": row["target_l2"]}
        for label, n in (("optimised", row["N_optimised"]), ("uniform", row["N_uniform"])):
            if label == "optimised":
                kn = pwl.pwl_design(f, n)
                t = pwl.Table(kn, pwl.pwl_project(f, kn, form))
            else:
                kn = a + (b - a) * torch.arange(n + 1, dtype=torch.float64, device="cuda") / n
                kn[-1] = b
                # two cells per interval: a knot sits on a cell boundary, and
                # whichever way FP32 rounding moves it, no cell gets two
                t = pwl.Table(kn, pwl.pwl_project(f, kn, form), "fp32", 2 * n)
            sec = time_launches(lambda: pwl.pwl_eval(t.handle, x, y))
            d = pwl.pwl_eval(t.handle, xm).cpu().numpy().astype(np.float64) - fx
            entry[label] = {"N": n, "gbs": round(BYTES_FWD * m / sec / 1e9, 1),
                            "layout": int(t.info["layout"]), "k_cells": int(t.info["k_cells"]),
                            "n_chain": int(t.info["n_chain"]),
                            "index_kb": round(t.info["eval_smem_bytes"] / 1024, 1),
                            "l2_err": float(np.sqrt(np.sum(d * d) * (b - a) / n_pts)),
                            "max_err": float(np.abs(d).max())}
            t.close()
        out.append(entry)
    return out


class _Queries:
    """The uniform query sets of the bench workload only (what table_one_measure reads)."""

    def __init__(self, log2m: int):
        import torch

        import paper_1510_02975_gb300 as pwl
        from paper_1510_02975_gb300 import workloads as W
        self.torch, self.pwl, self.W = torch, pwl, W
        self.m = 1 << log2m
        self.x = {(fi, "uniform"): W.uniform_queries(W.PAPER_FUNCTIONS[n], self.m, seed=1)
                  for fi, n in enumerate(FUNC_NAMES)}
        self.y = torch.empty(self.m, dtype=torch.float32, device="cuda")


def run_table1(args):
    """Table I on this GPU alone (the `table_I` key of the default line),
    with 2^log2m queries."""
    from paper_1510_02975_gb300 import _build
    _build.build()
    out = table_one_measure(_Queries(args.log2m), m=1 << args.log2m)
    print(json.dumps({"report": "table1", **out}), flush=True)


def run_backward(args):
    """pwl_eval_backward (x, values, knots) per call on the Gaussian tables at
    N in {256, 1024, 4096} (P_T values), 2^log2m queries, for query sets that
    take different scatter paths: uniform (per-lane atomics), sorted
    (warp-aggregated), normal(0, 1.5) clipped to the domain, and uniform with
    half the queries at x = 0 (the hot interval).  CUDA events over 10 calls
    after one warm-up call, each call the backward and its row reduction."""
    import torch

    import paper_1510_02975_gb300 as pwl
    from paper_1510_02975_gb300 import _build
    from paper_1510_02975_gb300 import workloads as W
    _build.build()
    f = W.GAUSSIAN
    m = 1 << args.log2m
    xu = W.uniform_queries(f, m, seed=1)
    g = torch.Generator(device="cuda").manual_seed(7)
    xp = xu.clone()
    xp[torch.rand(m, generator=g, device="cuda") < 0.5] = 0.0
    sets = {"uniform": xu, "sorted": torch.sort(xu).values, "normal_clipped": W.normal_queries(f, m, seed=2),
            "half_at_zero": xp}
    gy = W.upstream_grad((m,), seed=5)
    gx = torch.empty_like(gy)
    lib = pwl._capi.load()
    out = []
    for N in NS:
        kn = pwl.pwl_design(f, N)
        t = pwl.Table(kn, pwl.pwl_project(f, kn, "project"))
        ws = torch.empty(lib.pwl_eval_backward_workspace_size(t.handle), dtype=torch.uint8, device="cuda")
        gv = torch.zeros(N + 1, device="cuda")
        gk = torch.zeros(N + 1, device="cuda")
        row = {"N": N, "backward_smem_kb": round(t.info["backward_smem_bytes"] / 1024, 1)}
        for name, x in sets.items():
            sec = time_launches(lambda: pwl.pwl_eval_backward(t.handle, x, gy, gx, gv, gk, ws), reps=10)
            row[name] = {"us": round(sec * 1e6, 1), "gbs": round(BYTES_BWD * m / sec / 1e9, 1)}
        out.append(row)
        t.close()
    peak, kind = measured_peaks()
    print(json.dumps({"report": "backward", "queries": m, "bytes_per_query": BYTES_BWD, "peak_gbs": peak,
                      "peak_kind": kind, "tables": out}), flush=True)


def channels_measure(rows: int = 65536, reps: int = 5) -> dict:
    """Channel-wise learnable map: x[rows, 4096] ~ N(0, 2^2) (FP32 and BF16),
    4096 channels of 257 knots on [-8, 8] from the Gaussian design and P_T
    values, perturbed per channel; forward, backward (x, values, knots) and
    fwd+bwd throughput (CUDA events, mean of `reps` calls after a warm-up)."""
    import torch

    import paper_1510_02975_gb300 as pwl
    from paper_1510_02975_gb300 import workloads as W
    R, C, N = rows, 4096, 256
    f = {"kind": "gaussian", "a": -8.0, "b": 8.0, "p": [1.0, 0.0, 1.0]}
    k64 = pwl.pwl_design(f, N)
    v64 = pwl.pwl_project(f, k64, "project")
    g = torch.Generator(device="cuda").manual_seed(4)
    h = float(torch.diff(k64).min())
    knots = k64.float().repeat(C, 1)
    knots[:, 1:-1] += (torch.rand(C, N - 1, generator=g, device="cuda") - 0.5) * 0.4 * h
    values = v64.float().repeat(C, 1) + torch.randn(C, N + 1, generator=g, device="cuda") * 1e-3
    x = W.channel_inputs(R, C, seed=4)
    gy = W.upstream_grad((R, C), seed=5)
    y = torch.empty_like(x)
    gx = torch.empty_like(x)
    gv = torch.zeros_like(values)
    gk = torch.zeros_like(knots)
    xb = x.to(torch.bfloat16)
    yb = torch.empty_like(xb)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    m = R * C
    peak, kind = measured_peaks()
    out = {"shape": [R, C], "knots_per_channel": N + 1, "peak_gbs": peak, "peak_kind": kind}
    for label, fn, nbytes in (
            ("forward_fp32", lambda: pwl.pwl_channels_forward(knots, values, x, y, status=st), 8),
            ("forward_bf16", lambda: pwl.pwl_channels_forward(knots, values, xb, yb, status=st), 4),
            ("backward_fp32", lambda: pwl.pwl_channels_backward(knots, values, x, gy, gx, gv, gk, status=st), 12),
            ("fwd_bwd_fp32", lambda: (pwl.pwl_channels_forward(knots, values, x, y, status=st),
                                      pwl.pwl_channels_backward(knots, values, x, gy, gx, gv, gk, status=st)), 20)):
        sec = time_launches(fn, reps)
        gbs = nbytes * m / sec / 1e9
        out[label] = {"G_evals_per_s": round(m / sec / 1e9, 2), "gbs": round(gbs, 1),
                      "frac_of_peak": round(gbs / peak, 4), "ms": round(sec * 1e3, 4), "bytes_per_eval": nbytes}
    out["status"] = int(st.item())
    del x, gy, y, gx, xb, yb
    torch.cuda.empty_cache()
    return out


def run_channels(args):
    from paper_1510_02975_gb300 import _build
    _build.build()
    out = channels_measure(args.rows)
    print(json.dumps({"report": "channels", **out}), flush=True)


def f64_desc(desc, x):
    """FP64 f for a function descriptor (numpy / scipy, not the oracle)."""
    p = desc["p"]
    if desc["kind"] == "gaussian":
        u = (x - p[1]) / p[2]
        return p[0] * np.exp(-0.5 * u * u)
    if desc["kind"] == "lorentzian":
        u = (x - p[1]) / p[2]
        return p[0] / (1.0 + u * u)
    from scipy.special import j0
    return p[0] * j0(p[1] * x)


def batched_measure(n_funcs: int = 4096, m_per_interval: int = 16, cells_per_knot: int = 0, steps: int = 5,
                    per_function: bool = False) -> dict:
    """Batches of independent functions: 4096 functions (Gaussians, sigma
    log-uniform on [0.1, 10]; Lorentzians, gamma log-uniform on [0.1, 10];
    J0(alpha x), alpha uniform on [0.5, 5]), N_f + 1 uniform on 16..4096
    knots, log-uniform 10^3..10^6 FP32 queries per function uniform on its
    domain.  A step is design (FP32 density, FP64 scan and inversion),
    P_T values (FP32 integrand, FP64 sums and solve), index build and
    evaluation of every query, captured in one CUDA graph."""
    import torch

    import paper_1510_02975_gb300 as pwl
    from paper_1510_02975_gb300 import workloads as W
    funcs, n_int, n_q = W.batch_functions(n_funcs, seed=3)
    x, qo = W.batch_queries(funcs, n_q, seed=6)
    y = torch.empty_like(x)
    nq = int(qo[-1])
    b = pwl.Batch(funcs, n_int, m_per_interval=m_per_interval, cells_per_knot=cells_per_knot)
    prec = "fp32"

    def pipeline(stream=None):
        b.design(prec, stream)
        b.project("project", 8, prec, stream)
        b.build(stream)

    pipeline()
    b.check()
    b.plan(qo)
    b.eval(x, y)
    tune = b.autotune(x, y, reps=2)
    info = b.info()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
            pipeline(s)
            b.eval(x, y, s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    phases = {
        "design": time_launches(lambda: b.design(prec)),
        "project": time_launches(lambda: b.project("project", 8, prec)),
        "build": time_launches(lambda: b.build()),
        "eval": time_launches(lambda: b.eval(x, y)),
    }
    step = time_launches(graph.replay, reps=max(steps, 3))
    peak, kind = measured_peaks()
    ev_gbs = BYTES_FWD * nq / phases["eval"] / 1e9
    out = {
        "n_funcs": len(funcs), "total_knots": int(info["total_knots"]),
        "total_queries": nq, "m_per_interval": m_per_interval, "cells_per_knot": cells_per_knot or 3,
        "step_ms": round(step * 1e3, 4),
        "step_G_evals_per_s": round(nq / step / 1e9, 2),
        "phase_ms": {k: round(v * 1e3, 4) for k, v in phases.items()},
        "eval": {"G_evals_per_s": round(nq / phases["eval"] / 1e9, 2), "gbs": round(ev_gbs, 1),
                 "frac_of_peak": round(ev_gbs / peak, 4), "peak_gbs": peak, "peak_kind": kind,
                 "grid": int(info["eval_grid"]), "threads": int(info["eval_threads"]),
                 "shape": int(info["eval_shape"]), "stage_min": int(info["stage_min"]),
                 "pieces": int(info["n_items"]), "staged_pieces": int(info["n_staged"]),
                 "smem_bytes": int(info["smem_bytes"]), "index_bytes": int(info["index_bytes"]),
                 "autotune_ms": {f"shape{k[0]}/stage{k[1]}": round(v, 4) for k, v in tune.items()}},
    }
    # error against FP64 f on the first 64 functions (4096 queries each)
    yh_all = y[: min(nq, qo[64] if len(qo) > 64 else nq)].cpu().numpy().astype(np.float64)
    xh_all = x[: yh_all.size].cpu().numpy().astype(np.float64)
    err = {}
    for fi in range(min(64, len(funcs))):
        q0, q1 = qo[fi], min(qo[fi + 1], qo[fi] + 4096)
        if q1 <= q0:
            continue
        e = float(np.abs(yh_all[q0:q1] - f64_desc(funcs[fi], xh_all[q0:q1])).max())
        k = funcs[fi]["kind"]
        err[k] = max(err.get(k, 0.0), e)
    out["max_err_vs_f64_f_first64"] = err
    if per_function:
        # the same evaluation as one pwl_eval launch per function (4096
        # tables built from the batch's FP64 knots and values), the launches
        # captured in one CUDA graph
        kn = b.knots()
        vv = b.values()
        off = b.offsets()
        tables = [pwl.Table(kn[off[f]:off[f + 1]], vv[off[f]:off[f + 1]]) for f in range(len(funcs))]
        y2 = torch.empty_like(x)
        g2 = torch.cuda.CUDAGraph()
        s2 = torch.cuda.Stream()
        for f, t in enumerate(tables):  # eager pass: kernel attributes set outside capture
            if qo[f + 1] > qo[f]:
                pwl.pwl_eval(t.handle, x[qo[f]:qo[f + 1]], y2[qo[f]:qo[f + 1]])
        torch.cuda.synchronize()
        s2.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s2):
            with torch.cuda.graph(g2, stream=s2, capture_error_mode="thread_local"):
                for f, t in enumerate(tables):
                    if qo[f + 1] > qo[f]:
                        pwl.pwl_eval(t.handle, x[qo[f]:qo[f + 1]], y2[qo[f]:qo[f + 1]], stream=s2)
        torch.cuda.current_stream().wait_stream(s2)
        sec = time_launches(g2.replay)
        out["per_function_launches"] = {"G_evals_per_s": round(nq / sec / 1e9, 2),
                                        "gbs": round(BYTES_FWD * nq / sec / 1e9, 1), "ms": round(sec * 1e3, 4),
                                        "launches": sum(1 for f in range(len(funcs)) if qo[f + 1] > qo[f])}
        # the two index different cell grids: equal up to FP32 rounding
        out["per_function_launches"]["max_abs_diff_vs_batched"] = float((y - y2).abs().max())
        for t in tables:
            t.close()
    b.close()
    del graph, x, y
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    from paper_1510_02975_gb300 import _build
    _build.build()
    out = batched_measure(args.batch_funcs, args.batch_m, args.batch_cpk, args.steps, not args.no_per_function)
    print(json.dumps({"report": "batched", **out}), flush=True)


def main():
    args = parse_args()
    if args.report == "variants":
        run_variants(args)
        return
    if args.report == "channels":
        run_channels(args)
        return
    if args.report == "batched":
        run_batched(args)
        return
    if args.report == "backward":
        run_backward(args)
        return
    if args.report == "table1":
        run_table1(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
