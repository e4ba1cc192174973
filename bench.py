#!/usr/bin/env python
"""Throughput benchmark of the Boys-function evaluation on one GB300.

One step = one evaluation of F_0..F_{n_max} for the whole synthetic argument
array (the scale workload: x = p R^2, p log-uniform on [0.05, 1e4], R
uniform on [0, 12], 2^26 arguments, n_max = 8, FP64) through the library's C
ABI.  Prints one JSON line (rank 0).  Metric: G F_m values/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload scale_f64_n8|...] [--no-cpu-baseline]

Under torchrun (N > 1) every rank evaluates its own 2^26 arguments (weak
scaling: the path shards with no exchange) and rank 0 reports the total.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "scale_f64_n8": dict(count=1 << 26, n_max=8, dtype="f64"),
    "scale_f64_n0": dict(count=1 << 26, n_max=0, dtype="f64"),
    "scale_f64_n4": dict(count=1 << 26, n_max=4, dtype="f64"),
    "scale_f64_n16": dict(count=1 << 26, n_max=16, dtype="f64"),
    "scale_f64_n36": dict(count=1 << 24, n_max=36, dtype="f64"),
    # two-point evaluation (Trick B): second closed form at n_max/2
    "two_point_f64_n36": dict(count=1 << 24, n_max=36, dtype="f64", two_point=True),
    # the float path on the same arguments rounded to float
    "scale_f32_n8": dict(count=1 << 26, n_max=8, dtype="f32"),
    "scale_f32_n16": dict(count=1 << 26, n_max=16, dtype="f32"),
    "scale_f32_n36": dict(count=1 << 24, n_max=36, dtype="f32"),
    "scale_f32_n36_small": dict(count=1 << 22, n_max=36, dtype="f32"),
    # 4096 ragged requests (counts log-uniform on [64, 65536], n_max uniform on 0..16), graph replays
    "ragged_f64": dict(count=0, n_max=16, dtype="f64", kind="ragged"),
    # differentiation: 2^24 arguments, forward to n_max = 9, backward of sum_{m<=8} w_m F_m
    "grad_f64": dict(count=1 << 24, n_max=8, dtype="f64", kind="grad"),
    # small cases of the same kernels for detailed profiling (outputs still larger than L2)
    "scale_f64_n0_small": dict(count=1 << 22, n_max=0, dtype="f64"),
    "scale_f64_n4_small": dict(count=1 << 22, n_max=4, dtype="f64"),
    "scale_f64_n8_small": dict(count=1 << 22, n_max=8, dtype="f64"),
    "scale_f32_n8_small": dict(count=1 << 24, n_max=8, dtype="f32"),
    "scale_f64_n16_small": dict(count=1 << 22, n_max=16, dtype="f64"),
    "scale_f64_n36_small": dict(count=1 << 21, n_max=36, dtype="f64"),
    "two_point_f64_n36_small": dict(count=1 << 21, n_max=36, dtype="f64", two_point=True),
    # fused consumer: sum_m w_m F_m(x) per argument, rows kept in registers
    "contract_f64_n8": dict(count=1 << 26, n_max=8, dtype="f64", kind="contract"),
    "contract_f32_n8": dict(count=1 << 26, n_max=8, dtype="f32", kind="contract"),
    "contract_f32_n8_small": dict(count=1 << 25, n_max=8, dtype="f32", kind="contract"),
    "ragged_f64_small": dict(count=0, n_max=16, dtype="f64", kind="ragged", requests=256),
}
METRIC = "G F_m values/s at stated max rel err (FP64, FP32); % of ALU/HBM roofline"
TOL = {"f64": 2e-14, "f32": 2e-6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale_f64_n8", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip microbenchmarks and e2e (for profiling)")
    ap.add_argument("--peak-sweep", action="store_true",
                    help="print the DFMA rate over chains per thread x blocks per SM, then the library's "
                    "microbenchmark once, and exit")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    QUERY = (
        "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
            )
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.reader.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": mx,
            "reasons": sorted(reasons),
            "samples": len(sm),
        }


# ---------------------------------------------------------------------------


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate(x_all, n_max: int, target_cpu_s: float = 15.0, budget_s: float = 30.0, rows=None, dtype="f64"):
    """Time the CPU oracle on a bounded sample on all host cores.

    With rows (the benchmark's own output on the device, [count, n_max+1]),
    the oracle's values for the sample also measure the error of those rows:
    returns (baseline, accuracy)."""
    import numpy as np

    import oracle

    oracle.build()
    cores = cpu_cores()
    probe = x_all[:256]
    t0 = time.perf_counter()
    oracle.boys(probe, n_max)
    per = max((time.perf_counter() - t0) / probe.size, 1e-9)
    sample = int(min(x_all.size, max(1024, target_cpu_s / per)))
    sample = int(min(sample, budget_s * cores / per))
    xs = np.ascontiguousarray(x_all[:sample])
    t0 = time.perf_counter()
    ref = oracle.boys_threaded(xs, n_max, cores)
    dt = time.perf_counter() - t0
    base = {
        "value": round(sample * (n_max + 1) / dt / 1e9, 6),
        "unit": "G F_m values/s",
        "cores": cores,
        "kind": "oracle",
        "sample": f"first {sample} arguments of the same workload, n_max={n_max}, long double, "
        f"{cores} host threads, {dt:.2f} s wall",
    }
    if rows is None:
        return base, None
    return base, row_errors(rows[:sample].cpu().numpy().astype(np.float64), ref, dtype, sample)


def row_errors(got, ref, dtype, sample):
    """Maximum relative error per m of the rows against the oracle, with the
    tolerance of the path (FP64 2e-14, FP32 2e-6 for every m).  Where the
    exact value is below the smallest normal number of the output type the
    test is absolute (2 subnormal units for double; 2e-6 |F| + 2^-149 for
    float)."""
    import numpy as np

    tiny, sub = (np.finfo(np.float32).tiny, 2.0 ** -149) if dtype == "f32" else (np.finfo(np.float64).tiny, 2.0 ** -1073)
    normal = np.abs(ref) >= tiny
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.where(normal, np.abs(got - ref) / np.where(normal, np.abs(ref), 1.0), 0.0)
    small_ok = bool(np.all(normal | (np.abs(got - ref) <= TOL[dtype] * np.abs(ref) + sub)))
    finite = bool(np.all(np.isfinite(got)))
    per_m = [float(v) for v in rel.max(axis=0)]
    worst = max(per_m) if per_m else 0.0
    return {
        "max_rel_err_per_m": [float(f"{v:.3g}") for v in per_m],
        "max_rel_err": float(f"{worst:.3g}"),
        "tolerance": TOL[dtype],
        "pass": bool(worst <= TOL[dtype] and small_ok and finite),
        "how": f"the benchmark's own output rows for its first {sample} arguments against the CPU oracle "
        f"(long double), every m",
    }


def run_reference(args, wl):
    """The oracle as the reference arm: each step times it on a bounded sample."""
    import numpy as np

    from paper_2504_07637_gb300 import workloads

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    x = workloads.scale(1 << 20)
    n_max = wl["n_max"]
    import oracle

    oracle.build()
    cores = cpu_cores()
    probe = x[:256]
    t0 = time.perf_counter()
    oracle.boys(probe, n_max)
    per = max((time.perf_counter() - t0) / probe.size, 1e-9)
    # each step: about 10 s of CPU work, so K + W steps stay within minutes
    sample = int(min(x.size, max(1024, 10.0 / per)))
    xs = np.ascontiguousarray(x[:sample])
    for _ in range(args.warmup):
        oracle.boys_threaded(xs[: max(1024, sample // 8)], n_max, cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.boys_threaded(xs, n_max, cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = sample * (n_max + 1) * args.steps / tot / 1e9
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 6),
        "unit": "G F_m values/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "long double",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} (oracle sample of {sample} arguments per step)", "n_max": n_max},
        "cpu_baseline": {
            "value": round(value, 6),
            "unit": "G F_m values/s",
            "cores": cores,
            "kind": "oracle",
            "sample": f"{sample} arguments of the scale workload per step, {cores} host threads",
        },
        "e2e": {"value": round(value, 6), "unit": "G F_m values/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def microbench(capi, device):
    """Measured throughput (ops/s) of the FP64 operations the method uses."""
    import torch

    lib = capi.load()
    sink = torch.zeros(1, dtype=torch.float64, device=device)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    chains = lib.boys_microbench_ops_per_thread_iter()
    blocks = sms * 8
    rates = {}
    stream = torch.cuda.current_stream(device)
    for name, op, iters in (("fma", 0, 4096), ("exp_cuda", 1, 256), ("exp", 10, 256), ("sqrt", 2, 512),
                            ("rsqrt", 3, 512), ("div", 4, 512)):
        capi.call("boys_microbench_launch", op, 16, sink.data_ptr(), blocks, stream.cuda_stream)
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            capi.call("boys_microbench_launch", op, iters, sink.data_ptr(), blocks, stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            dt = e0.elapsed_time(e1) / 1e3
            best = dt if best is None else min(best, dt)
        rates[name] = blocks * 256 * iters * chains / best
    # exp/sqrt/rsqrt/div were each timed with one extra add: remove it
    t_fma = 1.0 / rates["fma"]
    for k in ("exp_cuda", "exp", "sqrt", "rsqrt", "div"):
        rates[k] = 1.0 / max(1.0 / rates[k] - t_fma, 1e-30)
    # integer pipes, in warp instructions per second: the 32-bit multiply-add
    # chain (fmaheavy pipe) and the 64-bit shift chain (ALU pipe); how many
    # instructions of that pipe one chain step issues was counted by ncu
    micro = pipes_micro()
    warps = blocks * 256 // 32
    for name, kind, iters in (("imad", 1, 4096), ("alu", 3, 4096)):
        per_step = micro.get(name, {}).get("inst_per_chain_step")
        if not per_step:
            continue
        capi.call("boys_microbench_int", kind, 16, sink.data_ptr(), blocks, stream.cuda_stream)
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            capi.call("boys_microbench_int", kind, iters, sink.data_ptr(), blocks, stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            dt = e0.elapsed_time(e1) / 1e3
            best = dt if best is None else min(best, dt)
        rates[name + "_warp"] = warps * iters * chains * per_step / best
    rates["sms"] = sms
    return rates


# FP64 nominal rate of GB300: 1.25 TFLOP/s, i.e. 0.625 T fused multiply-adds per second
F64_NOMINAL_TFMA = 0.625


def traffic_record(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it still matches the sources."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        recs = json.load(fh)
    rec = recs.get(kernel_key)
    if not rec:
        return None
    h = hashlib.sha256()
    for fn in rec.get("sources", []):
        with open(os.path.join(ROOT, fn), "rb") as fh:
            h.update(fh.read())
    return rec.get("bytes_per_launch") if h.hexdigest() == rec.get("sha256") else None


def instruction_record(kernel_key: str):
    """Warp instructions per argument from the committed ncu summary, if it still matches the sources."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "instructions.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh).get(kernel_key)
    if not rec:
        return None
    h = hashlib.sha256()
    for fn in rec.get("sources", []):
        with open(os.path.join(ROOT, fn), "rb") as fh:
            h.update(fh.read())
    return rec.get("warp_inst_per_arg") if h.hexdigest() == rec.get("sha256") else None


def _pipes():
    path = os.path.join(ROOT, "profiles", "pipes.json")
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


def _sources_sha(files):
    import hashlib

    h = hashlib.sha256()
    for fn in files:
        with open(os.path.join(ROOT, fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def pipes_micro():
    """The microbenchmarks' instructions per chain step on each pipe (ncu),
    if the record still matches the microbenchmark's source."""
    rec = _pipes().get("micro")
    if not rec or _sources_sha(rec.get("sources", [])) != rec.get("sha256"):
        return {}
    return rec


def pipe_ceiling(kernel_key, count, seconds, rates, sm_hz):
    """The ceiling of a kernel over the pipes it uses.

    Per argument, the kernel's work on each pipe comes from one small ncu
    capture (profiles/pipes.json, valid while its sources are unchanged):
    FP64-pipe cycles in DFMA warp instructions, ALU-pipe cycles in the ALU
    microbenchmark's instructions, fmaheavy-pipe cycles in 32-bit
    multiply-adds, and every issued warp instruction.  Each is divided by
    its rate measured in this run (the DFMA, ALU and multiply-add chains;
    issue at one warp instruction per clock per scheduler, 4 per SM, at the
    sampled SM clock).  The slowest pipe bounds the kernel; frac is that
    time over the measured one."""
    rec = _pipes().get(kernel_key)
    if not rec or _sources_sha(rec.get("sources", [])) != rec.get("sha256"):
        return None
    need = ("fma", "alu_warp", "imad_warp", "sms")
    if rates is None or any(k not in rates for k in need) or not sm_hz:
        return None
    w = rec["per_arg"]
    t = {
        "fp64": w["fp64_dfma"] * count / (rates["fma"] / 32.0),
        "alu": w["alu"] * count / rates["alu_warp"],
        "fmaheavy": w["fmaheavy_imad"] * count / rates["imad_warp"],
        "issue": w["inst"] * count / (ISSUE_PER_SM_CLOCK * rates["sms"] * sm_hz),
    }
    pipe = max(t, key=t.get)
    rate_g = {"fp64": rates["fma"] / 32e9, "alu": rates["alu_warp"] / 1e9, "fmaheavy": rates["imad_warp"] / 1e9,
              "issue": ISSUE_PER_SM_CLOCK * rates["sms"] * sm_hz / 1e9}
    return {
        "bound_pipe": pipe,
        "rate_g": {k: round(v, 3) for k, v in rate_g.items()},
        "frac": round(t[pipe] / seconds, 4),
        "pipe_ms": {k: round(v * 1e3, 4) for k, v in t.items()},
        "measured_ms": round(seconds * 1e3, 4),
        "per_arg": w,
        "source": rec.get("how", ""),
    }


def apply_ceiling(roof, ceiling):
    """Make the pipe ceiling the roofline's headline figures, keeping the
    FP64 op-count model beside it under "fp64_model"."""
    roof["fp64_model"] = {k: roof[k] for k in ("achieved", "peak", "unit", "frac", "note")}
    if ceiling is None:
        roof["ceiling"] = None
        roof["note"] = ("no current per-pipe profile of this kernel (profiles/pipes.json): headline figures are "
                        "the FP64 op-count model's; " + roof["note"])
        return
    pipe = ceiling["bound_pipe"]
    t_pipe = ceiling["pipe_ms"][pipe] / 1e3
    t_meas = ceiling["measured_ms"] / 1e3
    # the bounding pipe's measured rate, in G warp instructions per second
    peak = {"fp64": "dfma", "alu": "alu", "fmaheavy": "imad", "issue": "issue"}[pipe]
    roof["achieved"] = round(t_pipe / t_meas * ceiling["rate_g"][pipe], 3)
    roof["peak"] = round(ceiling["rate_g"][pipe], 3)
    roof["unit"] = f"G warp instructions/s on the {pipe} pipe ({peak} rate measured in this run)"
    roof["frac"] = ceiling["frac"]
    roof["ceiling"] = ceiling
    roof["note"] = ("combined ceiling: the kernel's per-argument work on the FP64, ALU and fmaheavy pipes and its "
                    "issued instructions (ncu, small case), each at its rate measured in this run; the slowest "
                    f"pipe ({pipe}) bounds the kernel. The FP64 op-count model is under fp64_model.")


# GB300 issue rate: 4 warp schedulers per SM, one warp instruction per clock
# each, at the maximum SM clock of 2,070 MHz
ISSUE_PER_SM_CLOCK, SM_CLOCK_MAX_HZ = 4, 2.07e9


def measured_peaks():
    """Measured HBM bandwidth if present, else the earlier GB300 figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _events_ms(fn, stream, reps):
    """Per-call milliseconds of fn() over reps calls (CUDA events, one pair per call)."""
    import torch

    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def _pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, int(round(q / 100 * (len(v) - 1))))]


def _f64_alu_model(capi, rates, x_host, n_max):
    """Seconds of FP64-pipe work per argument set under the op-count model."""
    import numpy as np

    from paper_2504_07637_gb300 import roofline

    lib = capi.load()
    n_top = lib.boys_top_order_f64(n_max)
    z = lib.boys_cutoff(n_top, 53)
    fb = float(np.mean(x_host <= z)) if x_host.size else 0.0
    below, above = roofline.f64_counts(n_max, n_top)
    t = sum((fb * below[k] + (1 - fb) * above[k]) / rates[k] for k in ("fma", "div", "sqrt", "exp", "rsqrt"))
    return t * x_host.size


def run_ragged(args, wl, emit=True):
    """Config: 4096 ragged requests in one graph-captured call vs one plain
    launch per request (also graph-captured), with the autotuned variant."""
    import numpy as np
    import torch

    import paper_2504_07637_gb300 as boys
    from paper_2504_07637_gb300 import _capi, autotune, workloads

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    x_host, offsets, n_max = workloads.ragged(wl.get("requests", 4096), 16, seed=workloads.SEED_BASE + 3 + rank)
    counts = np.diff(offsets)
    values = int(np.sum(counts * (n_max.astype(np.int64) + 1)))
    batch = boys.RaggedBatch(offsets, n_max, device)
    x = torch.from_numpy(x_host).to(device)
    out = torch.empty(batch.out_size, dtype=torch.float64, device=device)
    lean = getattr(args, "no_extras", False)  # profiling: no tuning, latency trials or per-request baseline
    if lean:
        tune = {"variant": 0, "all": [{"block": b, "tile": t, "ms": None} for b, t in boys.ragged_variants()]}
    else:
        tune = autotune.tune_ragged(batch, x, out, use_cache=False, reps=3)
    variant = tune["variant"]
    g = batch.capture(x, out, variant)
    stream = torch.cuda.current_stream(device)
    for _ in range(max(args.warmup, 3)):
        g.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if lean:
        print(json.dumps({"workload": "ragged (profiling run)", "ms_per_step": round(ms, 4)}), flush=True)
        return None
    lat = _events_ms(g.replay, stream, 200)
    # baseline: one plain launch per request, captured in one graph too
    views = [(x[offsets[r]:offsets[r + 1]], out[batch.out_offsets_host[r]:batch.out_offsets_host[r + 1]], int(n_max[r]))
             for r in range(n_max.size)]
    sptr_holder = {}

    def plain_all():
        sp = torch.cuda.current_stream(device).cuda_stream
        for xv, ov, n in views:
            if xv.numel():
                _capi.call("boys_eval_f64", xv.data_ptr(), xv.numel(), n, ov.data_ptr(), sp)

    plain_all()
    torch.cuda.synchronize()
    gp = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gp):
        plain_all()
    for _ in range(3):
        gp.replay()
    torch.cuda.synchronize()
    lat_plain = _events_ms(gp.replay, stream, 50)
    rates = microbench(_capi, device)
    t_alu = sum(_f64_alu_model(_capi, rates, x_host[offsets[r]:offsets[r + 1]], int(n_max[r])) for r in range(n_max.size))
    achieved = t_alu * rates["fma"] / (ms / 1e3) / 1e12
    peak = rates["fma"] / 1e12
    line = {
        "metric": METRIC,
        "value": round(values / (ms / 1e3) / 1e9, 4),
        "unit": "G F_m values/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": f"ragged_f64: 4096 requests, {int(offsets[-1])} arguments, {values} values, n_max uniform 0..16",
            "variant": {"index": variant, "block": tune["all"][variant]["block"], "tile": tune["all"][variant]["tile"]},
            "autotune_ms": {f"b{d['block']}_t{d['tile']}": d["ms"] for d in tune["all"]},
            "l2": "output (2.7 GB) larger than L2",
        },
        "latency_ms": {"p50": round(_pct(lat, 50), 4), "p99": round(_pct(lat, 99), 4), "trials": len(lat)},
        "plain_launches": {
            "p50_ms": round(_pct(lat_plain, 50), 4),
            "p99_ms": round(_pct(lat_plain, 99), 4),
            "speedup_p50": round(_pct(lat_plain, 50) / _pct(lat, 50), 3),
            "how": "4096 boys_eval_f64 calls captured in one CUDA graph",
        },
        "clocks": clk,
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "alu", "achieved": round(achieved, 5), "peak": round(peak, 5), "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "note": "FP64-pipe instruction equivalents (per-request op-count model) vs the measured DFMA rate"},
    }
    apply_ceiling(line["roofline"], pipe_ceiling("ragged<0..16>/plain", int(offsets[-1]), ms / 1e3, rates,
                                                 ((clk or {}).get("sm_mhz") or SM_CLOCK_MAX_HZ / 1e6) * 1e6))
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_grad(args, wl, emit=True):
    """Config: forward (n_max = 9) plus hand-written backward of
    sum_{m<=8} w_m sum_i F_m(x_i) through torch.autograd."""
    import numpy as np
    import torch

    import paper_2504_07637_gb300 as boys
    from paper_2504_07637_gb300 import _capi, workloads

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    count, n_max = wl["count"], wl["n_max"]
    x_host = workloads.plain(count, 53, seed=workloads.SEED_BASE + 4 + rank)
    w = torch.from_numpy(workloads.gradient_weights(n_max)).to(device)
    x = torch.from_numpy(x_host).to(device).requires_grad_(True)
    stream = torch.cuda.current_stream(device)
    gw = w.expand(count, n_max + 1)

    def step():
        F = boys.boys_autograd(x, n_max)
        torch.autograd.backward(F, gw)

    for _ in range(max(args.warmup, 3)):
        x.grad = None
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        x.grad = None
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # the pieces: forward alone (n_max + 1 = 9) and the backward kernel alone
    xd = x.detach()
    F = boys.boys(xd, n_max + 1)
    fwd = _events_ms(lambda: boys.boys(xd, n_max + 1, out=F), stream, 10)
    bwd = _events_ms(lambda: boys.boys_backward(xd, gw, n_max, F), stream, 10)
    # the backward's device time: calls queued back to back, so the host's
    # ~30 us per call (wrapper, checks, launch) overlaps the previous kernel
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    for _ in range(20):
        boys.boys_backward(xd, gw, n_max, F)
    q1.record(stream)
    q1.synchronize()
    bwd_queued_ms = q0.elapsed_time(q1) / 20
    # the backward without saved rows (recomputed in the kernel), device time;
    # one untimed call first (the kernel's first launch loads and sets it up)
    boys.boys_backward(xd, gw, n_max, None)
    torch.cuda.synchronize()
    q0.record(stream)
    for _ in range(5):
        boys.boys_backward(xd, gw, n_max, None)
    q1.record(stream)
    q1.synchronize()
    bwd_recompute_ms = q0.elapsed_time(q1) / 5
    # central differences would need two forwards of n_max (the method's own alternative)
    fwd8 = _events_ms(lambda: boys.boys(xd, n_max), stream, 10)
    bwd_ms = statistics.median(bwd)
    hbm_peak, src = measured_peaks()
    rates = microbench(_capi, device)
    bwd_bytes = count * 8 * (n_max + 1 + 1)  # F_1..F_{n_max+1} read, grad written (w broadcast)
    line = {
        "metric": METRIC,
        "value": round(count * (n_max + 2) / (ms / 1e3) / 1e9, 4),
        "unit": "G F_m values/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"grad_f64: 2^24 arguments, forward n_max={n_max + 1}, backward of sum_m w_m F_m, "
                               "value counts the forward's F_m values per forward+backward step",
                   "max_rel_err_grad": 1e-12},
        "forward_ms": round(statistics.median(fwd), 4),
        "backward_ms": round(bwd_ms, 4),
        "backward_ms_queued": round(bwd_queued_ms, 4),
        "backward_recompute_ms_queued": round(bwd_recompute_ms, 4),
        "central_difference_ms": round(2 * statistics.median(fwd8), 4),
        "backward_speedup_vs_central_difference": round(2 * statistics.median(fwd8) / bwd_ms, 2),
        "clocks": clk,
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "alu", "achieved": round(count * (n_max + 1) / (bwd_queued_ms / 1e3) / 1e12, 5),
                     "peak": round(rates["fma"] / 1e12, 5), "unit": "TFLOP/s",
                     "frac": round(count * (n_max + 1) / (bwd_queued_ms / 1e3) / rates["fma"], 4),
                     "traffic": traffic_record("grad_saved_kernel<8>/differentiation_2^24"),
                     "note": f"backward kernel (device time, calls queued): n_max+1 FP64 fma per argument vs the "
                     f"measured DFMA rate; HBM side {bwd_bytes / (bwd_queued_ms / 1e3) / 1e9:.0f} GB/s of "
                     f"{hbm_peak:.0f} ({src}) for {8 * (n_max + 2)} algorithmic bytes per argument"},
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


def measure_scale(wl, steps, warmup, device, seed, rates=None, e2e=False, clocks_index=None, keep_rows=False):
    """Time one scale-workload configuration; returns its figures.

    The timed region is exactly `steps` evaluation calls on the current
    stream, bracketed by CUDA events; the arguments (2^26 of them, 256 or
    512 MB) and the output exceed the L2, so no flush is needed."""
    import numpy as np
    import torch

    from paper_2504_07637_gb300 import _capi, roofline, workloads

    n_max, count = wl["n_max"], wl["count"]
    f32 = wl["dtype"] == "f32"
    np_t, th_t, esz = (np.float32, torch.float32, 4) if f32 else (np.float64, torch.float64, 8)
    fn = "boys_eval_f32" if f32 else ("boys_eval_f64_two_point" if wl.get("two_point") else "boys_eval_f64")
    x_host = workloads.scale(count, seed=seed).astype(np_t)
    x = torch.from_numpy(x_host).to(device)
    out = torch.empty((count, n_max + 1), dtype=th_t, device=device)
    stream = torch.cuda.current_stream(device)
    sptr = stream.cuda_stream

    def step():
        _capi.call(fn, x.data_ptr(), count, n_max, out.data_ptr(), sptr)

    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(clocks_index) if clocks_index is not None else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1) / steps
    res = {"ms": ms, "values": count * (n_max + 1), "clocks": clk, "x_host": x_host}
    if keep_rows:
        res["rows"] = out
    hbm_peak, hbm_src = measured_peaks()
    hbm_gbs = roofline.bytes_per_arg(n_max, esz) * count / (ms / 1e3) / 1e9
    if not f32 and rates is not None:
        lib = _capi.load()
        n_top = lib.boys_top_order_f64(n_max)
        z = lib.boys_cutoff(n_top, 53)
        fb = float(np.mean(x_host <= z))
        def t_per_arg(int_chain):
            if wl.get("two_point"):  # Trick B: n_bar = n_max / 2, closed forms at n_top and n_top(n_bar)
                n_bar = n_max // 2
                below, above = roofline.f64_counts_two_point(n_max, n_top, n_bar, lib.boys_top_order_f64(n_bar),
                                                             int_chain)
            else:
                below, above = roofline.f64_counts(n_max, n_top, int_chain)
            return sum((fb * below[k] + (1 - fb) * above[k]) / rates[k] for k in ("fma", "div", "sqrt", "exp", "rsqrt"))

        t_arg = t_per_arg(True)
        if wl.get("two_point"):
            n_bar = n_max // 2
            int_rec = roofline.int_recursion(n_top - n_bar - 1 + lib.boys_top_order_f64(n_bar))
        else:
            int_rec = roofline.int_recursion(n_top, n_max)
        rec_note = ("and the downward recursion run on the integer pipes and are not counted" if int_rec else
                    "runs on the integer pipes and is not counted; the downward recursion stays in FP64")
        two = bool(wl.get("two_point"))
        if roofline.int_rsqrt(n_max, two):
            rec_note += "; so do F_0 = c_0/sqrt(x), 1/x and the closed form after Q (Newton steps)"
        else:
            rec_note += "; so do F_0 = c_0/sqrt(x) and 1/x (Newton steps)"
        if roofline.int_exp(n_max, two):
            rec_note += " and e^{-x} (64-bit fixed point)"
        achieved = t_arg * rates["fma"] * count / (ms / 1e3) / 1e12
        achieved64 = t_per_arg(False) * rates["fma"] * count / (ms / 1e3) / 1e12
        peak = rates["fma"] / 1e12
        sm_hz = (clk or {}).get("sm_mhz") or SM_CLOCK_MAX_HZ / 1e6
        key = f"{'f64_two_point' if wl.get('two_point') else 'f64_rows'}<{n_max}>/scale"
        ceiling = pipe_ceiling(key, count, ms / 1e3, rates, sm_hz * 1e6)
        res["roofline"] = {
            "bound": "alu",
            "achieved": round(achieved, 5),
            "peak": round(peak, 5),
            "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4),
            "traffic": None if wl.get("two_point") else traffic_record(f"f64_rows<{n_max}>/scale_2^26"),
            "note": "FP64-pipe instruction equivalents per second (1 per add/mul/fma; exp, sqrt, rsqrt and div "
            "weighted by their measured cost) vs the DFMA rate measured in this run; the asymptote's upward "
            f"product chain ({roofline.int_chain_orders(n_max)} orders) {rec_note}; "
            f"{fb:.3f} of arguments below z_{{{n_top},53}}",
            "all_fp64": {"achieved": round(achieved64, 5), "frac": round(achieved64 / peak, 4),
                         "note": "the same evaluation with the recursion and the asymptote's chain as two FP64 "
                         "operations per order: the bound of an all-FP64 kernel (above 1: faster than that "
                         "bound)"},
            "hbm": {"achieved_gbs": round(hbm_gbs, 1), "peak_gbs": hbm_peak, "frac": round(hbm_gbs / hbm_peak, 4),
                    "peak_source": hbm_src},
            "nominal": {"peak": F64_NOMINAL_TFMA, "frac": round(achieved / F64_NOMINAL_TFMA, 4),
                        "source": "GB300 FP64 1.25 TFLOP/s nominal = 0.625 T FMA/s (2 DFMA per clock per SM at "
                        "152 SMs x 2.07 GHz)"},
            "measured_rates_gops": {k: round(v / 1e9, 2) for k, v in rates.items() if k != "sms"},
        }
        apply_ceiling(res["roofline"], ceiling)
    elif f32:
        n_top = _capi.load().boys_top_order_f32(n_max)
        z = _capi.load().boys_cutoff(n_top, 24)
        res["roofline"] = {
            "bound": "hbm",
            "achieved": round(hbm_gbs, 1),
            "peak": hbm_peak,
            "unit": "GB/s",
            "frac": round(hbm_gbs / hbm_peak, 4),
            "traffic": traffic_record(f"f32_split_kernel<{n_max}>/scale_2^26"),
            "note": f"{roofline.bytes_per_arg(n_max, esz)} algorithmic bytes per argument (x in, n_max+1 floats out) "
            f"vs the {hbm_src} copy bandwidth; {float(np.mean(x_host <= z)):.3f} of arguments below z_{{{n_top},24}}",
        }
    if e2e:
        # end to end through the C ABI with host buffers: pinned host arrays are
        # streamed through a device workspace in chunks whose copies overlap
        # the neighbouring chunk's kernel
        xp = torch.from_numpy(x_host).pin_memory()
        op = torch.empty((count, n_max + 1), dtype=th_t, pin_memory=True)
        # 256 MiB: chunks small enough that filling and draining the
        # pipeline costs little (measured on GB300 at n_max = 8: 64 MiB 23.4,
        # 256 MiB 23.5, 1 GiB 23.0, 4 GiB 20.9 G values/s)
        ws_bytes = 1 << 28
        wsp = torch.empty(ws_bytes, dtype=torch.uint8, device=device)

        def e2e_step():
            _capi.call(fn + "_host", xp.data_ptr(), count, n_max, op.data_ptr(), wsp.data_ptr(), ws_bytes, sptr)

        e2e_step()
        torch.cuda.synchronize()
        k2 = max(2, min(steps, 5))
        t0 = time.perf_counter()
        for _ in range(k2):
            e2e_step()
            stream.synchronize()
        dt = (time.perf_counter() - t0) / k2
        h2d_b, d2h_b = esz * count, esz * count * (n_max + 1)
        link = link_rates(xp, op, device)
        t_h2d, t_d2h = h2d_b / (link["h2d_gbs"] * 1e9), d2h_b / (link["d2h_gbs"] * 1e9)
        res["e2e"] = {
            "value": round(count * (n_max + 1) / dt / 1e9, 4),
            "unit": "G F_m values/s",
            "h2d_bytes_per_step": h2d_b,
            "d2h_bytes_per_step": d2h_b,
            "how": f"{fn}_host: pinned host in/out, 256 MiB device workspace, chunked copies overlapped with "
            "compute; host wall clock",
            # the host link bounds this number: plain pinned copies of the
            # same buffers, timed in the same run
            "link_gbs": {"h2d": link["h2d_gbs"], "d2h": link["d2h_gbs"], "both": link["both_gbs"]},
            "link_frac": round((h2d_b + d2h_b) / (link["both_gbs"] * 1e9) / dt, 4),
            "link_frac_serial": round((t_h2d + t_d2h) / dt, 4),
            "link_note": "link_frac: the same bytes copied in both directions at once (plain pinned copies of these "
            "buffers, this run; on GB300 the two directions share the link's rate) over the measured step; "
            "link_frac_serial: the two copies one after the other",
        }
        del xp, op, wsp
    del x, out
    torch.cuda.empty_cache()
    return res


def link_rates(host_in, host_out, device):
    """Plain pinned host <-> device copy rates (GB/s, best of 3 with CUDA
    events) for the buffers of the end-to-end run: host_in -> device and
    device -> host_out."""
    import torch

    stream = torch.cuda.current_stream(device)
    dev_in = torch.empty(host_in.shape, dtype=host_in.dtype, device=device)
    dev_out = torch.empty(host_out.shape, dtype=host_out.dtype, device=device)
    out = {}
    for name, dst, src, nbytes in (("h2d_gbs", dev_in, host_in, host_in.numel() * host_in.element_size()),
                                   ("d2h_gbs", host_out, dev_out, host_out.numel() * host_out.element_size())):
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        out[name] = round(nbytes / best / 1e9, 1)
    # both directions at once (the host pipeline overlaps them): the link's
    # total rate then, measured from the start of both to the end of both
    side = torch.cuda.Stream(device)
    best = None
    for _ in range(3):
        e0, e1, es = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        side.wait_event(e0)
        with torch.cuda.stream(side):
            dev_in.copy_(host_in, non_blocking=True)
            es.record(side)
        host_out.copy_(dev_out, non_blocking=True)
        stream.wait_event(es)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    out["both_gbs"] = round((host_in.numel() * host_in.element_size() + host_out.numel() * host_out.element_size())
                            / best / 1e9, 1)
    del dev_in, dev_out
    return out


def measure_contract(wl, steps, warmup, device, seed, rates=None):
    """The fused consumer on the scale workload: out = sum_m w_m F_m(x)."""
    import numpy as np
    import torch

    from paper_2504_07637_gb300 import _capi, roofline, workloads

    n_max, count = wl["n_max"], wl["count"]
    f32 = wl["dtype"] == "f32"
    np_t, th_t, esz = (np.float32, torch.float32, 4) if f32 else (np.float64, torch.float64, 8)
    x_host = workloads.scale(count, seed=seed).astype(np_t)
    x = torch.from_numpy(x_host).to(device)
    w = torch.from_numpy(workloads.gradient_weights(n_max).astype(np_t)).to(device)
    out = torch.empty(count, dtype=th_t, device=device)
    stream = torch.cuda.current_stream(device)
    fn = "boys_eval_contract_f32" if f32 else "boys_eval_contract_f64"
    f = lambda: _capi.call(fn, x.data_ptr(), count, n_max, w.data_ptr(), 0, 1, out.data_ptr(), stream.cuda_stream)
    for _ in range(max(warmup, 3)):
        f()
    # `steps` calls queued back to back between one pair of events (device time per call)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        f()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    res = {"value": round(count * (n_max + 1) / (ms / 1e3) / 1e9, 4), "unit": "G F_m values/s (consumed)",
           "ms_per_step": round(ms, 4), "bytes_per_arg": 2 * esz}
    if not f32 and rates is not None:
        n_top = _capi.load().boys_top_order_f64(n_max)
        fb = float(np.mean(x_host <= _capi.load().boys_cutoff(n_top, 53)))
        # the weights are the same for every argument (row stride 0)
        below, above = roofline.f64_counts_contract(n_max, n_top, uniform=True)
        t_arg = sum((fb * below[k] + (1 - fb) * above[k]) / rates[k] for k in ("fma", "div", "sqrt", "exp", "rsqrt"))
        res["roofline_bound"] = "alu"
        res["roofline_frac"] = round(t_arg * count / (ms / 1e3), 4)
    else:
        # 8 bytes per argument: the fused float path is bound by instruction
        # issue (ncu: ~80% of issue slots active, top stall "not selected")
        hbm_peak, _ = measured_peaks()
        hbm_frac = round(2 * esz * count / (ms / 1e3) / 1e9 / hbm_peak, 4)
        ipa = instruction_record(f"f32_split_kernel<{n_max}, 1>/contract_scale")
        if ipa is not None:
            sms = torch.cuda.get_device_properties(device).multi_processor_count
            peak = ISSUE_PER_SM_CLOCK * sms * SM_CLOCK_MAX_HZ
            achieved = ipa * count / (ms / 1e3)
            res["roofline_bound"] = "alu"
            res["roofline_frac"] = round(achieved / peak, 4)
            res["roofline"] = {"bound": "alu", "achieved": round(achieved / 1e12, 4), "peak": round(peak / 1e12, 4),
                               "unit": "T warp instructions/s", "frac": round(achieved / peak, 4),
                               "note": f"instruction issue: {ipa} warp instructions per argument (ncu) vs 4 per clock "
                               f"per SM at 2.07 GHz; HBM side {hbm_frac} of the copy bandwidth"}
        else:
            res["roofline_bound"] = "hbm"
            res["roofline_frac"] = hbm_frac
            res["note"] = "8 bytes per argument: the fused float path is bound by instruction issue, not HBM"
    del x, out
    torch.cuda.empty_cache()
    return res


def measure_plain(device, rates):
    """The plain 65,536-argument FP64 workload (n_max = 8): one launch, median of 50."""
    import torch

    from paper_2504_07637_gb300 import _capi, workloads

    x = torch.from_numpy(workloads.plain(65536, 53)).to(device)
    out = torch.empty((65536, 9), dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    f = lambda: _capi.call("boys_eval_f64", x.data_ptr(), 65536, 8, out.data_ptr(), stream.cuda_stream)
    for _ in range(5):
        f()
    ms = statistics.median(_events_ms(f, stream, 50))
    # the same call 200 times back to back: the host's ~10 us per call then
    # overlaps the kernels, leaving the device time per call
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(200):
        f()
    e1.record(stream)
    e1.synchronize()
    ms_q = e0.elapsed_time(e1) / 200
    return {"value": round(65536 * 9 / (ms / 1e3) / 1e9, 3), "ms_per_launch": round(ms, 5),
            "ms_per_launch_queued": round(ms_q, 5),
            "note": "one call over 65,536 arguments (256-argument tiles), events around each call (median of 50); "
            "queued: 200 calls back to back"}


def peak_sweep():
    """DFMA rate (G/s) over chains per thread x blocks of 256 threads per SM:
    whether the roofline's measured peak is the GPU's ceiling."""
    import torch

    from paper_2504_07637_gb300 import _capi

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.current_stream(dev)
    iters, table = 2048, {}
    for chains in (1, 2, 4, 8, 16):
        for per_sm in (1, 2, 4, 8):
            blocks = sms * per_sm
            _capi.call("boys_microbench_dfma", chains, 64, sink.data_ptr(), blocks, stream.cuda_stream)
            best = None
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _capi.call("boys_microbench_dfma", chains, iters, sink.data_ptr(), blocks, stream.cuda_stream)
                e1.record(stream)
                e1.synchronize()
                dt = e0.elapsed_time(e1) / 1e3
                best = dt if best is None else min(best, dt)
            table[f"{chains}x{per_sm}"] = round(blocks * 256 * iters * chains / best / 1e9, 1)
    rates = microbench(_capi, dev)
    print(json.dumps({"dfma_gops_chains_x_blocks_per_sm": table, "microbench_fma_gops": round(rates["fma"] / 1e9, 1)}),
          flush=True)


def main():
    args = parse()
    if args.peak_sweep:
        peak_sweep()
        return
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
        return
    if wl.get("kind") == "ragged":
        run_ragged(args, wl)
        return
    if wl.get("kind") == "grad":
        run_grad(args, wl)
        return
    if wl.get("kind") == "contract":
        import torch

        from paper_2504_07637_gb300 import _capi, workloads

        torch.cuda.set_device(0)
        dev = torch.device("cuda", 0)
        rates = None if wl["dtype"] == "f32" else microbench(_capi, dev)
        print(json.dumps({"workload": args.workload, **measure_contract(wl, args.steps, args.warmup, dev,
                                                                        workloads.SEED_BASE + 1, rates)}), flush=True)
        return
    import torch
    import torch.distributed as dist

    from paper_2504_07637_gb300 import _capi, shard, workloads

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    _capi.load()
    n_max, count = wl["n_max"], wl["count"]
    seed = shard.shard_seed(workloads.SEED_BASE + 1, rank)
    if ws > 1:
        dist.barrier()
    rates = None if args.no_extras or wl["dtype"] == "f32" else microbench(_capi, device)
    main_res = measure_scale(wl, args.steps, args.warmup, device, seed, rates=rates, e2e=not args.no_extras,
                             clocks_index=local, keep_rows=rank == 0 and not args.no_cpu_baseline)
    ms = main_res["ms"]
    ms_max = shard.max_over_ranks(ms, device)
    value = main_res["values"] * ws / (ms_max / 1e3) / 1e9
    extras = {}
    if "roofline" in main_res:
        extras["roofline"] = main_res["roofline"]
    if "e2e" in main_res:
        e = dict(main_res["e2e"])
        e["value"] = round(e["value"] * ws, 4)
        extras["e2e"] = e
    # the other configurations, summarised in the same line (single GPU, default run only)
    if ws == 1 and not args.no_extras and args.workload == "scale_f64_n8":
        suite = {"plain_f64_n8_65536": measure_plain(device, rates)}
        for name in ("scale_f64_n0", "scale_f64_n4", "scale_f64_n16", "scale_f64_n36", "two_point_f64_n36",
                     "scale_f32_n8", "scale_f32_n16", "scale_f32_n36"):
            r = measure_scale(WORKLOADS[name], 10, 3, device, seed, rates=rates)
            suite[name] = {"value": round(r["values"] / (r["ms"] / 1e3) / 1e9, 4), "unit": "G F_m values/s",
                           "ms_per_step": round(r["ms"], 4)}
            if "roofline" in r:
                suite[name]["roofline_bound"] = r["roofline"]["bound"]
                suite[name]["roofline_frac"] = r["roofline"]["frac"]
                if "all_fp64" in r["roofline"]:
                    suite[name]["all_fp64_frac"] = r["roofline"]["all_fp64"]["frac"]
                if "fp64_model" in r["roofline"]:
                    suite[name]["fp64_model_frac"] = r["roofline"]["fp64_model"]["frac"]
                    c = r["roofline"].get("ceiling")
                    suite[name]["ceiling_pipe"] = c["bound_pipe"] if c else None
        # the float path against the double one on the same arguments and order (n_max = 8)
        suite["scale_f32_n8"]["speedup_vs_f64_n8"] = round(suite["scale_f32_n8"]["value"] / value, 2)
        for name in ("contract_f64_n8", "contract_f32_n8"):
            suite[name] = measure_contract(WORKLOADS[name], 10, 3, device, seed, rates=rates)
        sub = argparse.Namespace(steps=10, warmup=3, gpus=1)
        rg = run_ragged(sub, WORKLOADS["ragged_f64"], emit=False)
        suite["ragged_f64"] = {k: rg[k] for k in ("value", "unit", "ms_per_step", "latency_ms", "plain_launches")}
        suite["ragged_f64"]["roofline_frac"] = rg["roofline"]["frac"]
        suite["ragged_f64"]["fp64_model_frac"] = rg["roofline"]["fp64_model"]["frac"]
        c = rg["roofline"].get("ceiling")
        suite["ragged_f64"]["ceiling_pipe"] = c["bound_pipe"] if c else None
        suite["ragged_f64"]["variant"] = rg["config"]["variant"]
        gr = run_grad(sub, WORKLOADS["grad_f64"], emit=False)
        suite["grad_f64"] = {k: gr[k] for k in ("value", "unit", "ms_per_step", "forward_ms", "backward_ms",
                                                "backward_ms_queued", "backward_recompute_ms_queued",
                                                "backward_speedup_vs_central_difference")}
        suite["grad_f64"]["backward_roofline"] = gr["roofline"]
        extras["workloads"] = suite
    accuracy = None
    if rank == 0 and not args.no_cpu_baseline:
        import numpy as np

        extras["cpu_baseline"], accuracy = oracle_rate(main_res["x_host"].astype(np.float64), n_max,
                                                        rows=main_res.get("rows"), dtype=wl["dtype"])
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": round(value, 4),
            "unit": "G F_m values/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms_max, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": wl["dtype"],
            "data": "synthetic",
            "config": {
                "workload": f"{args.workload}: {count} arguments x = p R^2 per GPU ({wl['dtype']}), n_max={n_max}",
                "global_batch": count * ws,
                "n_max": n_max,
                "max_rel_err": accuracy["max_rel_err"] if accuracy else "not measured (--no-cpu-baseline)",
                "accuracy": accuracy,
                "l2": "inputs and outputs larger than the 129 MB L2; no flush needed",
                "parallelism": f"dp{ws} (independent shards, no collective)",
            },
            "clocks": main_res["clocks"],
            "gpu_launches": args.steps,
            **extras,
        }
        print(json.dumps(line), flush=True)
    main_res.pop("rows", None)
    if ws > 1:
        dist.destroy_process_group()
    if accuracy is not None and not accuracy["pass"]:
        # the metric is values/s at the stated error: a run above it has no value
        sys.exit(f"bench: measured max relative error {accuracy['max_rel_err']:g} above {accuracy['tolerance']:g}")


if __name__ == "__main__":
    main()
