#!/usr/bin/env python3
"""Throughput benchmark of the FHT2DT forward transform on GB300.

Workload (default): one 4095 x 4095 float32 image, pixels i.i.d. N(0, 1)
(seed 2), all four slope quadrants, EXTENDED boundary (output 4 x 4095 x 8189
float32).  A step is one complete forward transform of that image.

Prints one JSON line on rank 0.  `value` is input Mpix/s over all ranks with
the image resident in HBM; `e2e` is the same metric through the public API
with host buffers (pinned host -> device copy of the image and device -> host
copy of the whole Hough output inside every step).  `roofline` reports the
dominant kernel's model bytes per launch over its event-timed duration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fht|reference]

`--impl reference` times the CPU oracle (the plain single-threaded C
recursion) on the host cores on a bounded sample of the same workload.
Multi-GPU runs are independent replicas (weak scaling, no data exchange).
"""
from __future__ import annotations

import argparse
import gc
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "c2-extended": dict(h=4095, w=4095, quads=15, boundary="extended",
                        desc="4095x4095 float32 N(0,1) seed 2, 4 quadrants, extended boundary"),
    "c2-cyclic": dict(h=4095, w=4095, quads=15, boundary="cyclic",
                      desc="4095x4095 float32 N(0,1) seed 2, 4 quadrants, cyclic boundary"),
    # the comparison method of the paper (balanced Split_S tree), same image
    "c2-extended-split-s": dict(h=4095, w=4095, quads=15, boundary="extended", split="S",
                                desc="4095x4095 float32 N(0,1) seed 2, 4 quadrants, extended boundary, FHT2DS"),
}
METRIC = "FHT Mpix/s (4 quadrants)"
UNIT = "Mpix/s"
FLUSH_BYTES = 256 << 20  # > 129 MB L2


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# --------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(gpu: int):
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    try:
        p = subprocess.Popen(["nvidia-smi", "-i", str(gpu), f"--query-gpu={CLOCK_FIELDS}",
                              "--format=csv,noheader,nounits", "-lms", "100"], stdout=f, stderr=subprocess.DEVNULL)
    except OSError:
        p = None
    return p, f.name


def clocks_stop(handle) -> dict:
    p, path = handle
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    sm, smax, reasons, power = [], [], set(), []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    with open(path) as f:
        for line in f:
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
    os.unlink(path)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------
def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


FORWARD_SOURCES = ("fht_desc.h", "fht_device.cuh", "fht_block.cuh", "fht_forward.cu", "fht_launch.hpp")


def _source_hash() -> str:
    """Hash of the sources of the forward kernels (the ones the roofline reports)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2411_07351_gb300", "csrc")
    for fn in FORWARD_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("source_hash") != _source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# --------------------------------------------------------------------------
# CPU oracle (reported baseline and the reference arm)
# --------------------------------------------------------------------------
def oracle_sample_seconds(img, wl, rows: int):
    import oracle

    sub = np.ascontiguousarray(img[:rows])
    t = time.perf_counter()
    oracle.fht(sub, 1, oracle.EXTENDED if wl["boundary"] == "extended" else oracle.CYCLIC, _rule(oracle, wl))
    return time.perf_counter() - t


def _rule(oracle, wl):
    return oracle.SPLIT_S if wl.get("split", "T") == "S" else oracle.SPLIT_T


def _oracle_full_image(job):
    """Worker of the all-core oracle baseline: the full 4-quadrant transform of
    the seeded workload image, once (a spawned process: no CUDA state)."""
    h, w, boundary, split = job
    import oracle
    from paper_2411_07351_gb300 import inputs

    img = inputs.c2_image(h=h, w=w)
    t = time.perf_counter()
    oracle.fht(img, 15, oracle.EXTENDED if boundary == "extended" else oracle.CYCLIC, _rule(oracle, {"split": split}))
    return time.perf_counter() - t


def cpu_baselines(img, wl, min_seconds: float = 10.0):
    """The oracle as it stands on the host cores: (1) one core, the full
    4-quadrant transform of the workload image repeated for >= min_seconds;
    (2) all cores, one independent full transform per core in spawned
    processes (the oracle itself is single-threaded)."""
    import multiprocessing as mp

    import oracle

    h, w = img.shape
    b = oracle.EXTENDED if wl["boundary"] == "extended" else oracle.CYCLIC
    runs, t0 = 0, time.perf_counter()
    while runs == 0 or time.perf_counter() - t0 < min_seconds:
        oracle.fht(img, 15, b, _rule(oracle, wl))
        runs += 1
    sec1 = time.perf_counter() - t0
    one = {"value": runs * h * w / sec1 / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"the full {h}x{w} image, 4 quadrants, {runs} runs in {sec1:.1f} s",
           "cpu": _cpu_model(), "nproc": os.cpu_count()}
    n = os.cpu_count() or 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(n) as pool:
        pool.map(_oracle_full_image, [(h, w, wl["boundary"], wl.get("split", "T"))] * n)
    secn = time.perf_counter() - t0
    alln = {"value": n * h * w / secn / 1e6, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} independent full 4-quadrant transforms of the {h}x{w} image, one per core, "
                      f"{secn:.1f} s wall including process start", "cpu": _cpu_model(), "nproc": n}
    return one, alln


def per_height_model_bytes(h: int, w: int, ext: bool, in_size: int = 4, acc: int = 4, F: int = 64) -> int:
    """HBM bytes of the per-height schedule of the Split_T recursion, four
    quadrants: the image read once per quadrant, every subtree of at most F
    rows written once, and every node above them reading its two children and
    writing its own rows (row width L + m - 1 extended, L cyclic)."""

    def split_t(m):
        p = 1
        while 2 * p < m:
            p *= 2
        return p, m - p

    total = 0
    for n, L in ((h, w), (h, w), (w, h), (w, h)):
        def width(m, L=L):
            return L + m - 1 if ext else L

        def rec(m):
            if m <= F:
                return m * width(m) * acc
            a, b = split_t(m)
            return rec(a) + rec(b) + (a * width(a) + b * width(b) + m * width(m)) * acc

        total += n * L * in_size + rec(n)
    return total


def _band_rows(per_step_budget_s: float, w: int, h: int) -> int:
    # cost model of one quadrant of a band of r rows: r (w + r) log2 r, 3 s at r = 4095 (measured)
    def est(r):
        return 3.0 * (r * (w + r) * max(1.0, math.log2(r))) / (4095 * 8190 * 12)

    r = h
    while r > 64 and est(r) > per_step_budget_s:
        r //= 2
    return r


def run_reference(args, wl):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2411_07351_gb300 import inputs

    oracle.build()
    img = inputs.c2_image(h=wl["h"], w=wl["w"])
    rows = _band_rows(150.0 / max(1, args.steps + args.warmup), wl["w"], wl["h"])
    for _ in range(args.warmup):
        oracle_sample_seconds(img, wl, rows)
    times = [oracle_sample_seconds(img, wl, rows) for _ in range(args.steps)]
    sec = statistics.mean(times)
    # one quadrant of `rows` image rows per step: a quarter of the 4-quadrant work per pixel
    value = rows * wl["w"] / 4.0 / sec / 1e6
    sample = f"quadrant Q0 of the first {rows} rows of the image (one quarter of the 4-quadrant work)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "h": wl["h"], "w": wl["w"], "quadrants": 4,
                       "boundary": wl["boundary"], "split": wl.get("split", "T"), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu": _cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_fht(args, wl):
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2411_07351_gb300 as F
    from paper_2411_07351_gb300 import _capi, inputs

    h, w = wl["h"], wl["w"]
    img = inputs.c2_image(h=h, w=w)
    x = torch.from_numpy(img).cuda()
    plan = F.Plan(h, w, torch.float32, wl["quads"], wl["boundary"], wl.get("split", "T"), device=local)
    out = plan.new_output()
    ws = plan.new_workspace()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    lib = _capi.load()
    nl = ctypes.c_int32()
    _capi.check(lib.fht_plan_launches(plan._h, ctypes.byref(nl)), "fht_plan_launches")
    launches = nl.value
    kinds, lbytes = [], []
    for k in range(launches):
        kd, by = ctypes.c_int32(), ctypes.c_int64()
        _capi.check(lib.fht_plan_launch_info(plan._h, k, ctypes.byref(kd), ctypes.byref(by)), "launch_info")
        kinds.append(kd.value)
        lbytes.append(by.value)

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    clk = clocks_start(local)
    for _ in range(max(3, args.warmup)):
        plan.forward(x, out, ws)
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps outside the step events ----
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    barrier()
    torch.cuda.synchronize()
    for i in range(K):
        flush.zero_()
        ev[i][0].record(stream)
        plan.forward(x, out, ws)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(statistics.mean(step_ms))
    value = world * h * w / (ms * 1e-3) / 1e6

    # ---- per-kernel timing (events around every launch) ----
    KP = min(K, 50)
    kev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * launches)]
    for e in kev:
        e.record(stream)  # materialise the handles
    handles = (ctypes.c_void_p * (2 * launches))(*[e.cuda_event for e in kev])
    per_launch = np.zeros(launches)
    torch.cuda.synchronize()
    for _ in range(KP):
        flush.zero_()
        _capi.check(lib.fht_forward_timed(plan._h, x.data_ptr(), x.stride(0), out.data_ptr(), ws.data_ptr(),
                                          ws.numel(), stream.cuda_stream, handles, 2 * launches), "fht_forward_timed")
        torch.cuda.synchronize()
        for k in range(launches):
            per_launch[k] += kev[2 * k].elapsed_time(kev[2 * k + 1])
    per_launch /= KP
    kind_names = {0: "fused_kernel", 1: "upper_kernel", 2: "band_kernel", 3: "spine_kernel", 4: "block_kernel"}
    kernels = {}
    for k in range(launches):
        nm = kind_names[kinds[k]]
        d = kernels.setdefault(nm, {"launches": 0, "ms": 0.0, "model_bytes": 0})
        d["launches"] += 1
        d["ms"] += per_launch[k]
        d["model_bytes"] += lbytes[k]
    dom = max(kernels, key=lambda n: kernels[n]["ms"])
    peak, peak_kind = _peaks()
    dk = kernels[dom]
    achieved = dk["model_bytes"] / (dk["ms"] * 1e-3) / 1e9
    for nm, d in kernels.items():
        d["gbs"] = d["model_bytes"] / (d["ms"] * 1e-3) / 1e9
        d["share"] = d["ms"] / float(per_launch.sum())

    # ---- end to end through the C ABI with host buffers (fht_pipe_submit):
    # every step copies its image in from pinned host memory, transforms it
    # and copies the packed output back; consecutive steps overlap ----
    host_in = torch.from_numpy(img).pin_memory()
    host_out = torch.empty(plan.out_elems, dtype=torch.float32).pin_memory()
    pipe = F.HostPipeline(plan, depth=2, copy_streams=1)
    for _ in range(max(3, args.warmup)):
        pipe.submit(host_in, host_out)
    pipe.synchronize()
    legacy = torch.cuda.default_stream()  # the pipe's blocking streams order with it
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(legacy)
    for i in range(K):
        pipe.submit(host_in, host_out)
    e1.record(legacy)
    torch.cuda.synchronize()
    pipe.synchronize()
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / K)
    pipe.close()
    clocks = clocks_stop(clk)
    e2e_value = world * h * w / (e2e_ms * 1e-3) / 1e6

    ph_bytes = per_height_model_bytes(h, w, wl["boundary"] == "extended")
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, cpu_all = cpu_baselines(img, wl)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["desc"], "h": h, "w": w, "quadrants": 4, "boundary": wl["boundary"],
                       "split": wl.get("split", "T"), "fused_rows": int(plan.info.fused_rows),
                       "tile_cols": int(plan.info.tile_cols),
                       "l2": "256 MiB buffer written between timed steps, outside the step events",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": _traffic(dom, "c2-" + wl["boundary"]),
                         "algorithmic_bytes_per_launch": dk["model_bytes"] / dk["launches"]},
            "kernels": kernels,
            "model_bytes_per_step": int(plan.info.model_bytes), "ideal_bytes_per_step": int(plan.info.ideal_bytes),
            "vs_per_height_schedule": {
                "per_height_model_bytes": ph_bytes,
                "speed": ph_bytes / (ms * 1e-3) / 1e9 / peak,
                "note": "speed relative to a per-height schedule (64-row fused subtrees, one HBM pass per upper "
                        "tree height) running at the measured copy bandwidth: that schedule's bytes over this "
                        "step's time, over the peak; not a roofline fraction (this build moves "
                        "model_bytes_per_step)"},
            "step_bandwidth": {"model_bytes": int(plan.info.model_bytes),
                               "achieved": int(plan.info.model_bytes) / (ms * 1e-3) / 1e9, "peak": peak,
                               "unit": "GB/s", "frac": int(plan.info.model_bytes) / (ms * 1e-3) / 1e9 / peak},
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_ms,
                    "api": "fht_pipe_submit, 2 device sets, copies on their own streams",
                    "h2d_bytes_per_step": int(host_in.numel() * host_in.element_size()),
                    "d2h_bytes_per_step": int(host_out.numel() * host_out.element_size())},
            "gpu_launches": launches * K,
            "clocks": clocks,
        }
        if world == 1 and not args.no_extras:
            # the rest of the metric (latency, batched vs plain, served vs plain),
            # measured after the headline's timed region on the same GPU
            # (an extra that fails is reported as such; the headline line still prints)
            def c1_part():
                c1 = measure_c1(args)
                return dict(c1["latency_us"], unit="us", workload=c1["config"]["workload"],
                            launches_per_call=c1["gpu_launches_per_call"])

            def c3_part():
                c3 = measure_c3(args)
                out = {k: c3[k] for k in ("batched_ms", "graph_ms", "plain_ms", "plain_value", "graph_value",
                                          "speedup_vs_plain", "model_gbs_batched", "gpu_launches")}
                out.update(batched_value=c3["value"], unit=UNIT, workload=c3["config"]["workload"])
                return out

            def c5_part():
                c5 = _c5_in_fresh_process(args)
                return {"served": c5["served"], "plain": c5["plain"], "unit": UNIT, "workload": c5["config"]["workload"]}

            for key, part in (("c1_latency", c1_part), ("c3_batching", c3_part), ("c5_serving", c5_part)):
                try:
                    line[key] = part()
                except Exception as exc:  # noqa: BLE001 - recorded in the line
                    line[key] = {"error": f"{type(exc).__name__}: {str(exc)[-400:]}"}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# the other workloads: one JSON line each (not the headline)
# --------------------------------------------------------------------------
def _launches(plan) -> int:
    """Kernel launches one fht_forward of `plan` enqueues (fht_plan_launches)."""
    from paper_2411_07351_gb300 import _capi

    n = ctypes.c_int32()
    _capi.check(_capi.load().fht_plan_launches(plan._h, ctypes.byref(n)), "fht_plan_launches")
    return n.value


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * (len(xs) - 1) + 0.5))] if xs else None


def run_c1(args):
    print(json.dumps(measure_c1(args)), flush=True)


def measure_c1(args) -> dict:
    """257 x 257 uint8, one quadrant, cyclic: per-call latency."""
    import torch

    import paper_2411_07351_gb300 as F
    from paper_2411_07351_gb300 import inputs

    img = inputs.c1_image()
    x = torch.from_numpy(img).cuda()
    plan = F.Plan(257, 257, torch.uint8, F.FHT_Q0, "cyclic", tuning="auto")
    out, ws = plan.new_output(), plan.new_workspace()
    for _ in range(50):
        plan.forward(x, out, ws)
    torch.cuda.synchronize()
    # the same call captured once in a CUDA graph (the three launches without host gaps)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.forward(x, out, ws)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.forward(x, out, ws)
    gdev = []
    for i in range(max(args.steps, 1000) + 50):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        graph.replay()
        b.record()
        b.synchronize()
        if i >= 50:
            gdev.append(a.elapsed_time(b) * 1e3)
    n = max(args.steps, 1000)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    host = []
    for i in range(n):
        t = time.perf_counter()
        ev[i][0].record()
        plan.forward(x, out, ws)
        ev[i][1].record()
        ev[i][1].synchronize()
        host.append((time.perf_counter() - t) * 1e6)
    dev = [a.elapsed_time(b) * 1e3 for a, b in ev]
    mean_us = statistics.mean(dev)
    line = {"metric": METRIC, "value": 257 * 257 / mean_us, "unit": UNIT, "n_gpus": 1, "steps": n,
            "higher_is_better": True, "dtype": "u8->i32", "data": "synthetic",
            "config": {"workload": "c1: 257x257 uint8 U{0..255} seed 1, quadrant Q0, cyclic"},
            "latency_us": {"device_p50": _pct(dev, 0.5), "device_p99": _pct(dev, 0.99),
                           "host_p50": _pct(host, 0.5), "host_p99": _pct(host, 0.99),
                           "graph_device_p50": _pct(gdev, 0.5), "graph_device_p99": _pct(gdev, 0.99)},
            "tile_cols": int(plan.info.tile_cols),
            "gpu_launches_per_call": _launches(plan)}
    return line


def _extra_dist(fn, args):
    """Run an extra workload on this rank's GPU (torchrun: one process per GPU,
    NCCL only for the timing reductions) and print rank 0's line."""
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    line = fn(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_c3(args):
    _extra_dist(measure_c3, args)


def measure_c3(args) -> dict:
    """4096 binary edge maps of 17..511 pixels a side: plain launches per image
    vs one persistent batched launch vs its CUDA-graph replay."""
    import torch

    import paper_2411_07351_gb300 as F
    from paper_2411_07351_gb300 import inputs
    from paper_2411_07351_gb300.batch import BatchQueue

    from paper_2411_07351_gb300 import parallel

    world, _ = parallel.world_rank()
    imgs = inputs.c3_batch()
    mpix = sum(im.size for im in imgs) / 1e6  # the whole batch, over all ranks
    imgs = [imgs[i] for i in parallel.my_shard([im.shape for im in imgs])]  # all of them at world 1
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    # the plans' launch shape chosen by measurement on this batch (autotuned tiles)
    from paper_2411_07351_gb300.tune import tune_batch

    tuned = tune_batch(xs, F.FHT_QALL, "cyclic", "T")
    q = BatchQueue(max_jobs=len(xs), max_units=1 << 23, shape=tuned["shape"])
    plans = [q.plan_for(x, F.FHT_QALL, "cyclic", "T") for x in xs]
    outs = [p.new_output() for p in plans]
    wss = [p.new_workspace() for p in plans]
    model = sum(int(p.info.model_bytes) for p in plans)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    def plain():
        for x, p, o, w in zip(xs, plans, outs, wss):
            p.forward(x, o, w)

    def batched():
        q.submit(xs, F.FHT_QALL, "cyclic", "T", outs=outs, workspaces=wss, plans=plans)

    plain()
    batched()
    torch.cuda.synchronize()
    reps = max(3, min(args.steps, 20))
    t_plain = timed(plain, reps)
    t_batch = timed(batched, reps)
    assert q.status() == 0
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
            q.submit(xs, F.FHT_QALL, "cyclic", "T", outs=outs, workspaces=wss, stream=s, plans=plans)
    torch.cuda.synchronize()
    t_graph = timed(g.replay, reps)
    # the batch's time is its slowest rank's (no exchange on the data path)
    dev = torch.device("cuda", torch.cuda.current_device())
    t_plain, t_batch, t_graph = (parallel.max_over_ranks(t, dev) for t in (t_plain, t_batch, t_graph))
    model = int(parallel.sum_over_ranks(float(model), dev))
    line = {"metric": METRIC, "value": mpix / (t_batch * 1e-3), "unit": UNIT, "n_gpus": world, "steps": reps,
            "scaling": "strong",
            "higher_is_better": True, "dtype": "u8->i32", "data": "synthetic",
            "config": {"workload": "c3: 4096 binary edge maps, h, w ~ U{17..511} seed 3, 4 quadrants, cyclic",
                       "mpix": mpix, "l2": "256 MiB buffer written before every timed run"},
            "batched_ms": t_batch, "graph_ms": t_graph, "plain_ms": t_plain,
            "plain_value": mpix / (t_plain * 1e-3), "graph_value": mpix / (t_graph * 1e-3),
            "speedup_vs_plain": t_plain / t_batch, "model_bytes": model,
            "model_gbs_batched": model / (t_batch * 1e-3) / 1e9,
            "gpu_launches": {"plain": sum(_launches(p) for p in plans), "batched": 1},
            "tuned_shape": {"tile_cols_threads_generic_cols": list(tuned["shape"]),
                            "candidates_ms": tuned["candidates"]},
            "sharding": "size-balanced shard of the batch per rank, slowest rank's time" if world > 1 else None}
    q.close()
    return line


def run_c4(args):
    """64 float32 images of 200..600 pixels a side: forward + adjoint backward of
    0.5 ||FHT(x) - y||^2 over the packed 4-quadrant cyclic output."""
    import torch

    from paper_2411_07351_gb300 import inputs
    from paper_2411_07351_gb300.autograd import fht

    imgs = inputs.c4_batch()
    ys = [torch.from_numpy(y).cuda() for y in inputs.c4_targets(imgs)]
    xs = [torch.from_numpy(im).cuda().requires_grad_(True) for im in imgs]
    mpix = sum(im.size for im in imgs) / 1e6

    # the 64 images are independent: their forward and backward chains run on
    # 8 side streams (autograd replays each op's backward on the op's stream)
    side = [torch.cuda.Stream() for _ in range(8)]

    def step():
        main = torch.cuda.current_stream()
        parts = []
        for k, (x, y) in enumerate(zip(xs, ys)):
            s = side[k % len(side)]
            s.wait_stream(main)
            with torch.cuda.stream(s):
                parts.append(0.5 * ((fht(x, 15, "cyclic") - y) ** 2).sum())
        for s in side:
            main.wait_stream(s)
        loss = torch.stack(parts).sum()
        loss.backward()
        for s in side:
            main.wait_stream(s)
        return loss

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    reps = max(3, min(args.steps, 20))
    ts = []
    for _ in range(reps):
        for x in xs:
            x.grad = None
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    # the same step captured once in a CUDA graph and replayed (no per-launch host cost)
    for x in xs:
        x.grad = None
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # warm the side stream (gradients allocated here are reused by the graph)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        gl = step()
    torch.cuda.synchronize()
    gts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        torch.cuda.synchronize()
        gts.append(a.elapsed_time(b))
    gms = statistics.median(gts)
    line = {"metric": METRIC + " forward+backward", "value": mpix / (gms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": reps, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c4: 64 float32 images, h, w ~ U{200..600}, U[0,1) seed 4, targets N(0,1) seed 5, "
                                   "4 quadrants cyclic, loss 0.5||FHT(x)-y||^2", "mpix": mpix},
            "ms_per_step_graph": gms, "ms_per_step_eager": ms, "eager_value": mpix / (ms * 1e-3)}
    print(json.dumps(line), flush=True)


def run_c5(args):
    _extra_dist(measure_c5, args)


def _records(done) -> list:
    """Per served request: (latency, plan, admit, launch, device) in ms and its
    pixels.  Stages: arrival -> plan built (seen by the serving loop), ->
    admitted under the memory budget, -> launch enqueued, -> completion seen
    by the host."""
    out = []
    for r in done:
        st = None
        if None not in (r.t_ready, r.t_admit, r.t_launch):
            st = ((r.t_ready - r.arrival) * 1e3, (r.t_admit - r.t_ready) * 1e3, (r.t_launch - r.t_admit) * 1e3,
                  (r.done - r.t_launch) * 1e3)
        out.append(((r.done - r.arrival) * 1e3, st, int(r.image.numel())))
    return out


def _gathered(records: list, wall: float) -> tuple[list, float]:
    """Every rank's records and the slowest rank's wall time (one rank: as given)."""
    from paper_2411_07351_gb300 import parallel

    world, rank = parallel.world_rank()
    if world == 1:
        return records, wall
    merged = parallel.gather_by_index({rank: records})
    return [x for k in sorted(merged) for x in merged[k]], parallel.max_over_ranks(wall)


def _summary(records: list, wall: float) -> dict:
    lat = [x[0] for x in records]
    mp = sum(x[2] for x in records) / 1e6
    stages = {}
    for k, name in enumerate(("plan", "admit", "launch", "device")):
        v = [x[1][k] for x in records if x[1] is not None]
        stages[name] = {"p50_ms": _pct(v, 0.5), "p99_ms": _pct(v, 0.99)}
    return {"requests": len(records), "wall_s": wall, "mpix_per_s": mp / wall, "p50_ms": _pct(lat, 0.5),
            "p99_ms": _pct(lat, 0.99), "max_ms": max(lat), "stages": stages}


def _c5_in_fresh_process(args) -> dict:
    """The serving measurement in a process of its own, as a serving process
    starts: the stream's latencies then depend on nothing the other workloads
    left behind (cached device blocks, plans, chunks of the table arena)."""
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", "c5", "--serve-seconds", str(args.serve_seconds)]
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK=os.environ.get("LOCAL_RANK", "0"))
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(f"c5 measurement failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def measure_c5(args) -> dict:
    """Poisson stream of uint8 requests (h, w log-uniform in [64, 4096], 10 %
    non-zero), 4 quadrants cyclic, 16 GB admission budget: continuous batching
    vs plain per-request launches on the same arrival sequence."""
    import torch

    from paper_2411_07351_gb300 import parallel
    from paper_2411_07351_gb300.serve import PlainServer, Request, Server, run_stream

    world, rank = parallel.world_rank()
    rate, dur, lo, hi = 2000.0, args.serve_seconds, 64, 4096
    g = np.random.Generator(np.random.PCG64(6))
    # one seeded 4096 x 4096 noise field; each request is a window of it (10 % non-zero, values U{1..255})
    field = np.where(g.random((hi, hi)) < 0.1, g.integers(1, 256, (hi, hi)), 0).astype(np.uint8)
    dfield = torch.from_numpy(field).cuda()

    def make_requests(seed=60, seconds=None):
        gg = np.random.Generator(np.random.PCG64(seed))
        t, out = 0.0, []
        while True:
            t += gg.exponential(1.0 / rate)
            if t > (dur if seconds is None else seconds):
                return out
            h = int(round(math.exp(gg.uniform(math.log(lo), math.log(hi)))))
            w = int(round(math.exp(gg.uniform(math.log(lo), math.log(hi)))))
            y0, x0 = int(gg.integers(0, hi - h + 1)), int(gg.integers(0, hi - w + 1))
            out.append(Request(len(out), t, dfield[y0:y0 + h, x0:x0 + w]))

    def my_requests(reqs):
        # several GPUs: each arrival is routed to one rank (least work so far;
        # every rank routes the same stream identically, nothing is exchanged)
        if world == 1:
            return reqs
        to = parallel.route([tuple(r.image.shape) for r in reqs], world)
        return [r for r, k in zip(reqs, to) if k == rank]

    res = {}
    makers = (("served", lambda: Server(budget_bytes=16 << 30, streams=4, keep_outputs=False)),
              ("plain", lambda: PlainServer(keep_outputs=False)))
    def warmed(mk):
        # half a second of other requests first: kernels loaded, allocator and
        # streams warm (the measured stream's shapes still need new plans)
        srv = mk()
        run_stream(srv, make_requests(seed=61, seconds=0.5))
        srv.finished, srv.batches = [], 0
        return srv

    def fresh():
        # each measured run starts from the same device state: the previous
        # run's requests, plans and cached blocks released first
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    for name, mk in makers:
        fresh()
        reqs = my_requests(make_requests())
        srv = warmed(mk)
        done, wall = run_stream(srv, reqs)
        res[name] = _summary(*_gathered(_records(done), wall))
        res[name]["launch_groups"] = int(parallel.sum_over_ranks(float(srv.batches)))
        srv.close()
        del done, reqs, srv
    # saturation: the same request mix arriving 10x faster, so that throughput,
    # not the offered load, decides Mpix/s
    nonlocal_rate = rate
    for name, mk in makers:
        fresh()
        reqs = my_requests(make_requests()[: int(nonlocal_rate * min(dur, 2.0))])
        for r in reqs:
            r.arrival /= 10.0
        srv = warmed(mk)
        done, wall = run_stream(srv, reqs)
        sat = _summary(*_gathered(_records(done), wall))
        res[name]["saturated"] = {k: sat[k] for k in ("requests", "wall_s", "mpix_per_s", "p50_ms", "p99_ms")}
        res[name]["saturated"]["offered_req_per_s"] = rate * 10
        srv.close()
    line = {"metric": METRIC + " served", "value": res["served"]["mpix_per_s"], "unit": UNIT, "n_gpus": world,
            "scaling": "strong",
            "higher_is_better": True, "dtype": "u8->i32", "data": "synthetic",
            "config": {"workload": f"c5: Poisson {rate:.0f} req/s for {dur} s, h, w log-uniform [64, 4096], "
                                   "10% non-zero uint8 windows of a seeded field, 4 quadrants cyclic, 16 GB budget",
                       "warm_up": "0.5 s of requests from another seed through each server before its measured run",
                       "routing": "each arrival to the rank with the least work so far" if world > 1 else None},
            "served": res["served"], "plain": res["plain"]}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["fht", "reference"], default="fht")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["c1", "c3", "c4", "c5"], default="c2-extended")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the c1 latency, c3 batching and c5 serving measurements of the default line")
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    args = ap.parse_args()
    extra = {"c1": run_c1, "c3": run_c3, "c4": run_c4, "c5": run_c5}
    if args.workload in extra:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the headline workload only"}))
            return
        extra[args.workload](args)
        return
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_fht(args, wl)


if __name__ == "__main__":
    main()
