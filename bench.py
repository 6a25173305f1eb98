"""Benchmark of the Array-OL repetitive-task library on GB300.

Headline step: the two chained 8->3 FIR downscalers (horizontal then vertical)
on 64 float32 frames of 1080x1920 -> 64 x 405 x 720, one fused kernel launch
through the C ABI.  Metric: tiler elements per second (pattern elements
gathered + elements scattered, both tasks) and the fraction of the measured
HBM copy bandwidth reached by the kernel on its algorithmic bytes (input read
once, output written once).  The same JSON line also reports, with L2
emptied before each timed call:

  * the 64x64 task's latency per call;
  * the batched uneven workload (512 tasks, one graph launch vs one launch
    per task) and 128 batched two-stage chains;
  * the 3x3 stencil on 8192x8192 (a FIR on a 2-D pattern);
  * the backward pass (fwd+bwd over fwd, 16 frames);
  * the tensor-core matmul task (4096^3 bf16 -> f32);
  * the chain with bf16 and with IEEE half storage;
  * the conjugate-gradient solve and its SpMV.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --case batched|chains|chain5to2|config0_scaled|generic|stencil|backward|matmul|config0|cg|bf16|f16

Under torchrun every rank runs its own 64 frames (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

FRAMES, HEIGHT, WIDTH = 64, 1080, 1920
METRIC = "tiler elems/s (fused 2-task FIR downscaler chain)"
UNIT = "elems/s"
WORKLOAD = "downscale chain 64x1080x1920 f32 -> 64x405x720 (8-tap->3 FIR, step 8, both axes)"
L2_BYTES = 126 * 1024 * 1024


# FP32 FMA peak derived from the part's unit counts and clock: 152 SMs x 128
# FP32 lanes x 2 flops x 2.07 GHz (the maximum SM clock).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 peak: the part's nominal dense float64 rate (not measured here)
FP64_PEAK_TFLOPS = 1.25


def chain_units(frames, height=HEIGHT, width=WIDTH):
    """Tiler elements of one pass of the chain: gathered + scattered, both tasks."""
    wr, hr = width // 8, height // 8
    gathered = frames * height * wr * 8 + frames * hr * (wr * 3) * 8
    scattered = frames * height * wr * 3 + frames * hr * 3 * wr * 3
    return gathered + scattered


def chain_bytes(frames, height=HEIGHT, width=WIDTH):
    """Algorithmic bytes of the fused chain: X read once, Y written once."""
    return 4 * frames * height * width + 4 * frames * (height // 8 * 3) * (width // 8 * 3)


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the headline kernel from an ncu capture, with the source version it was
# taken on; reported as null once the kernel source differs.
HEADLINE_TRAFFIC = {"source": "paper_1105_4424_gb300/csrc/k_downscale.cu", "sha256_prefix": "e4613f6adca5c030",
                    "bytes": 530882304 + 63358720}


def headline_traffic():
    import hashlib
    path = os.path.join(ROOT, HEADLINE_TRAFFIC["source"])
    try:
        with open(path, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    return HEADLINE_TRAFFIC["bytes"] if digest.startswith(HEADLINE_TRAFFIC["sha256_prefix"]) else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (read-only queries)
    every ~0.5 ms by a background thread while the timed region runs, so even
    a few-millisecond region gets samples."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_index):
        import ctypes
        import threading
        import torch
        self.ok = False
        self.samples = []
        self._stop = threading.Event()
        self._thread = None
        try:
            L = ctypes.CDLL("libnvidia-ml.so.1")
            if L.nvmlInit_v2() != 0:
                return
            pr = torch.cuda.get_device_properties(torch_index)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
            h = ctypes.c_void_p()
            if L.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(h)) != 0:
                return
            self._reasons_fn = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                L.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint()
            L.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
            self.max_mhz = mx.value
            self.L, self.h, self.ctypes = L, h, ctypes
            self.ok = True
        except (OSError, AttributeError, RuntimeError):
            self.ok = False

    def _run(self):
        c = self.ctypes
        mhz, rs = c.c_uint(), c.c_ulonglong()
        while not self._stop.is_set():
            if self.L.nvmlDeviceGetClockInfo(self.h, 1, c.byref(mhz)) == 0 and \
                    self._reasons_fn(self.h, c.byref(rs)) == 0:
                self.samples.append((mhz.value, rs.value))
            time.sleep(0.0005)

    def __enter__(self):
        import threading
        if self.ok:
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()
            t0 = time.perf_counter()
            while not self.samples and self._thread.is_alive() and time.perf_counter() - t0 < 0.5:
                time.sleep(0.0002)
        return self

    def __exit__(self, *exc):
        if self._thread is not None:
            self._stop.set()
            self._thread.join()

    def summary(self):
        if not self.samples:
            return None
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(m for m, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(self.samples), "source": "nvml"}


# -------------------------------------------------------- rank aggregation

def aggregate(elapsed_ms_per_rank, units_per_rank, steps):
    """Whole-job throughput: the units all ranks processed over the whole timed
    region (all steps), divided by the slowest rank's time for it."""
    t = max(elapsed_ms_per_rank)
    total = sum(units_per_rank)
    return total / (t / 1e3), t / steps


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


def dist_max(value, world):
    """Every rank's value (all-gather), on the device the backend needs."""
    if world == 1:
        return [value]
    import torch
    import torch.distributed as dist
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=device)
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t)
    return [float(o.item()) for o in out]


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------- measurements

def time_loop(fn, steps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


class L2Flush:
    """Empties L2 between timed iterations: a 256 MB write evicts whatever
    the measured kernel touched, then a read of a second 256 MB buffer
    (written once here) pushes the write's dirty lines back to DRAM, so the
    next timed kernel starts on a clean L2 and pays only for its own bytes."""

    def __init__(self, torch):
        n = 256 * 1024 * 1024 // 4
        self.w = torch.empty(n, device="cuda")
        self.r = torch.ones(n, device="cuda")
        self.sink = torch.empty((), device="cuda")
        self.torch = torch

    def __call__(self):
        self.w.zero_()
        self.torch.sum(self.r, 0, out=self.sink)


def time_each_flushed(fn, reps, stream, flush):
    """Per-iteration CUDA-event times with an L2 flush between iterations,
    outside the timed events."""
    import torch
    ts = []
    for _ in range(reps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts


def bench_batched(A, torch, stream, flush, reps, tune=True):
    tasks, xs = W.config3()
    b = A.Batch(tasks)
    ins = [torch.from_numpy(x).cuda() for x in xs]
    outs = b.empty_outputs()
    cfg = b.tune(ins, outs) if tune else b.config
    run, run_per_task = b.prepare(ins, outs)   # pointer arrays marshalled once, outside the timed region
    for _ in range(3):
        run()
        run_per_task()
    batched = time_each_flushed(run, reps, stream, flush)
    per_task = time_each_flushed(run_per_task, reps, stream, flush)
    nbytes = sum(4 * x.size for x in xs) + sum(4 * int(np.prod(t["outputs"][0]["shape"])) for t in tasks)
    units = sum(t["rep"][0] * t["rep"][1] * (t["inputs"][0]["pattern"][0] + t["outputs"][0]["pattern"][0])
                for t in tasks)
    # FIR multiply-adds: repetitions x m x T per task
    fma = sum(t["rep"][0] * t["rep"][1] * t["taps"].size for t in tasks)
    tb, tp = statistics.median(batched), statistics.median(per_task)
    b.sync_status()
    return {"tasks": len(tasks), "unique_bytes": nbytes, "tiler_elems": units,
            "batched_ms": tb, "per_task_ms": tp, "speedup": tp / tb,
            "batched_gbs": nbytes / (tb * 1e-3) / 1e9, "batched_elems_per_s": units / (tb * 1e-3),
            "fma": fma, "fp32_tflops": 2 * fma / (tb * 1e-3) / 1e12,
            "fp32_frac_of_derived_peak": 2 * fma / (tb * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
            "launches_batched": 1, "launches_per_task": len(tasks), "autotuned": cfg}


def bench_batched_chains(A, torch, stream, flush, reps, hbm):
    """128 two-stage 8 -> 3 downscaler chains of uneven frame sizes in one
    batch: one launch of the batched downscaler over every member (the
    intermediates stay on chip), against one launch per member, the batch
    run stage by stage (the row-FIR kernel, then the persistent kernel's
    column tiles, intermediates through HBM; inputs one float off a 16-byte
    boundary route the members there) and one fused chain launch per
    member."""
    chains, xs = W.chain_batch()
    b = A.Batch(chains)
    ins = [torch.from_numpy(x).cuda() for x in xs]
    outs = b.empty_outputs()
    run, run_per_task = b.prepare(ins, outs)
    bs = A.Batch(chains)
    # the same inputs one float past a 16-byte boundary: stage by stage
    bufs = [torch.empty(x.size + 1, device="cuda") for x in xs]
    sins = []
    for buf, x in zip(bufs, ins):
        buf[1:] = x.reshape(-1)
        sins.append(buf[1:].view(x.shape))
    souts = bs.empty_outputs()
    run_staged, _ = bs.prepare(sins, souts)
    fused = [A.Chain(c) for c in chains]
    fouts = [torch.empty_like(o) for o in outs]
    fused_calls = [f.prepare([x], y) for f, x, y in zip(fused, ins, fouts)]

    def run_fused():
        for call in fused_calls:
            call()

    for _ in range(3):
        run()
        run_per_task()
        run_staged()
        run_fused()
    tb = statistics.median(time_each_flushed(run, reps, stream, flush))
    tp = statistics.median(time_each_flushed(run_per_task, reps, stream, flush))
    ts = statistics.median(time_each_flushed(run_staged, reps, stream, flush))
    tf = statistics.median(time_each_flushed(run_fused, reps, stream, flush))
    b.sync_status()
    bs.sync_status()
    mid = sum(4 * int(np.prod(c[0]["outputs"][0]["shape"])) for c in chains)
    nbytes = sum(4 * x.size for x in xs) + sum(4 * int(np.prod(c[-1]["outputs"][0]["shape"])) for c in chains)
    gbs = nbytes / (tb * 1e-3) / 1e9
    return {"chains": len(chains), "unique_bytes": nbytes, "intermediate_bytes": mid,
            "batched_ms": tb, "per_task_ms": tp, "staged_ms": ts, "fused_per_chain_ms": tf,
            "speedup_vs_per_task": tp / tb, "speedup_vs_staged": ts / tb, "speedup_vs_fused_per_chain": tf / tb,
            "batched_gbs_unique": gbs, "frac_of_hbm": gbs / hbm, "kernel": "downscale_batch_kernel",
            "launches": {"batched": 1, "per_task": len(chains), "staged": 2, "fused_per_chain": len(chains)}}


def _task_gbs(A, torch, stream, flush, reps, hbm, tk, xs, kernel_name):
    t = A.Task(tk) if isinstance(tk, dict) else A.Chain(tk)
    ins = [torch.from_numpy(x).cuda() for x in xs]
    last = tk if isinstance(tk, dict) else tk[-1]
    out = torch.empty(tuple(last["outputs"][0]["shape"]), dtype=torch.float32, device="cuda")
    call = t.prepare(ins, out)
    for _ in range(3):
        call()
    ms = statistics.median(time_each_flushed(call, reps, stream, flush))
    t.sync_status()
    nbytes = sum(4 * x.size for x in xs) + 4 * out.numel()
    gbs = nbytes / (ms * 1e-3) / 1e9
    return t, ms, {"ms": ms, "unique_bytes": nbytes, "gbs": gbs, "frac_of_hbm": gbs / hbm, "kernel": kernel_name,
                   "info_kernel": t.info["kernel"], "path": t.info.get("path")}


def bench_chain_5to2(A, torch, stream, flush, reps, hbm):
    """The 5-tap -> 2 step-4 downscaler chain on 64 x 1080 x 1920: the
    streaming row-then-column kernel against the tile kernel (the streaming
    kernel switched off for one chain) and the same chain stage by stage (a
    one-member batch: two launches, the intermediate through HBM)."""
    chain, xs = W.config1_5to2()
    _, ms, out = _task_gbs(A, torch, stream, flush, reps, hbm, chain, xs, "sepstream_kernel")
    prev = os.environ.get("AROL_SEPSTREAM")
    os.environ["AROL_SEPSTREAM"] = "off"
    try:
        _, out["tile_kernel_ms"], _ = _task_gbs(A, torch, stream, flush, reps, hbm, chain, xs, "sepchain_kernel")
    finally:
        if prev is None:
            del os.environ["AROL_SEPSTREAM"]
        else:
            os.environ["AROL_SEPSTREAM"] = prev
    # stage by stage: the chain made with the streaming kernel off, in a
    # one-member batch
    os.environ["AROL_SEPSTREAM"] = "off"
    try:
        b = A.Batch([chain])
    finally:
        if prev is None:
            del os.environ["AROL_SEPSTREAM"]
        else:
            os.environ["AROL_SEPSTREAM"] = prev
    ins = [torch.from_numpy(x).cuda() for x in xs]
    outs = b.empty_outputs()
    run, _ = b.prepare(ins, outs)
    for _ in range(3):
        run()
    out["staged_ms"] = statistics.median(time_each_flushed(run, reps, stream, flush))
    out["fused_speedup"] = out["staged_ms"] / ms
    out["roofline"] = {"bound": "hbm", "achieved": out["gbs"], "peak": hbm, "unit": "GB/s", "frac": out["frac_of_hbm"]}
    # the chain's backward on 16 frames (the intermediate recomputed by the
    # row pass, then one sweep per pass for dX and the tap gradients): loss
    # sum(G * Y)
    chain16, xs16 = W.config1_5to2(frames=16)
    c = A.Chain(chain16)
    x16 = torch.from_numpy(xs16[0]).cuda()
    g16 = torch.from_numpy(W.rng(7).standard_normal(chain16[-1]["outputs"][0]["shape"]).astype(np.float32)).cuda()
    gx = torch.empty_like(x16)
    gt = torch.empty(20, device="cuda")
    y16 = c.run([x16])
    for _ in range(3):
        c.backward(g16, [x16], gx, gt)
    fwd16 = statistics.median(time_each_flushed(lambda: c.run([x16], y16), reps, stream, flush))
    bwd16 = statistics.median(time_each_flushed(lambda: c.backward(g16, [x16], gx, gt), reps, stream, flush))
    c.sync_status()
    bbytes = 4 * (2 * x16.numel() + g16.numel())   # reads X and dY, writes dX
    out["backward_16_frames"] = {"fwd_ms": fwd16, "bwd_ms": bwd16, "ratio": (fwd16 + bwd16) / fwd16,
                                 "bwd_gbs": bbytes / (bwd16 * 1e-3) / 1e9,
                                 "bwd_frac_of_hbm": bbytes / (bwd16 * 1e-3) / 1e9 / hbm}
    return out


def bench_config0_scaled(A, torch, stream, flush, reps, hbm):
    """The 64 x 64 task's step-4 wrapping 8 -> 3 tiler on 64 x 1080 x 1920 (a
    row-FIR task: the library's choice, the row FIR in 16-word regions), and
    the same task as a one-member batch (the row-FIR tile kernel)."""
    tk, xs = W.config0_scaled()
    _, _, out = _task_gbs(A, torch, stream, flush, reps, hbm, tk, xs, "rowfir_region_kernel")
    b = A.Batch([tk])
    ins = [torch.from_numpy(x).cuda() for x in xs]
    outs = b.empty_outputs()
    for _ in range(3):
        b.run(ins, outs)
    out["tiles_ms"] = statistics.median(time_each_flushed(lambda: b.run(ins, outs), reps, stream, flush))
    b.sync_status()
    out["tiles_frac_of_hbm"] = out["unique_bytes"] / (out["tiles_ms"] * 1e-3) / 1e9 / hbm
    out["roofline"] = {"bound": "hbm", "achieved": out["gbs"], "peak": hbm, "unit": "GB/s", "frac": out["frac_of_hbm"]}
    return out


def bench_generic(A, torch, stream, flush, reps, hbm):
    """A tiler no specialised kernel takes (diagonal 8-element patterns) on
    64 x 1080 x 1920: the per-repetition walk."""
    tk, xs = W.diagonal_fir()
    return _task_gbs(A, torch, stream, flush, reps, hbm, tk, xs, "tiler_tiled_kernel")[2]


def bench_stencil(A, torch, stream, flush, reps, hbm):
    """A 3x3 stencil as a repetitive task (2-D pattern, identity fitting,
    origin (-1, -1) with wrap) on an 8192 x 8192 float32 image, one call."""
    n = 8192
    g = W.rng(5)
    x = g.random((n, n), dtype=np.float32)
    H = (g.standard_normal((1, 9)) / 9).astype(np.float32)
    inp = W.port((n, n), (-1, -1), ((1, 0), (0, 1)), ((1, 0), (0, 1)), (3, 3))
    out = W.port((n, n), (0, 0), ((1, 0), (0, 1)), ((0,), (0,)), (1,))
    t = A.Task(W.task((n, n), "fir", [inp], [out], H))
    xd = torch.from_numpy(x).cuda()
    y = t.empty_output("cuda")
    run = t.prepare([xd], y)
    for _ in range(3):
        run()
    ms = statistics.median(time_each_flushed(run, reps, stream, flush))
    nbytes = 8 * n * n
    return {"workload": "3x3 stencil, 8192x8192 f32, wrap", "ms": ms, "unique_bytes": nbytes,
            "gbs": nbytes / (ms * 1e-3) / 1e9, "frac_of_hbm": nbytes / (ms * 1e-3) / 1e9 / hbm}


def bench_backward(A, torch, stream, flush, reps):
    chain, (x,), w = W.config4()
    c = A.Chain(chain)
    xd = torch.from_numpy(x).cuda()
    wd = torch.from_numpy(w).cuda()
    y = c.run([xd])
    gx = torch.empty_like(xd)
    gt = torch.empty(48, device="cuda")
    for _ in range(3):
        c.run([xd], y)
        c.backward(wd, [xd], gx, gt)
        c.fwd_bwd([xd], wd, y, gx, gt)
    fwd = statistics.median(time_each_flushed(lambda: c.run([xd], y), reps, stream, flush))
    bwd = statistics.median(time_each_flushed(lambda: c.backward(wd, [xd], gx, gt), reps, stream, flush))

    def both():
        c.run([xd], y)
        c.backward(wd, [xd], gx, gt)
    fb = statistics.median(time_each_flushed(both, reps, stream, flush))
    fused = statistics.median(time_each_flushed(lambda: c.fwd_bwd([xd], wd, y, gx, gt), reps, stream, flush))
    fb_bytes = 4 * (x.size + w.size) + 4 * x.size   # bwd reads X and dY, writes dX
    out = {"frames": 16, "fwd_ms": fwd, "bwd_ms": bwd, "fwd_plus_bwd_ms": fb, "ratio": fb / fwd,
           "fused_fwd_bwd_ms": fused, "fused_ratio": fused / fwd,
           "fwd_gbs": chain_bytes(16) / (fwd * 1e-3) / 1e9, "bwd_gbs": fb_bytes / (bwd * 1e-3) / 1e9,
           # the backward moves (X + dY + dX) / (X + Y) = 1.88x the forward's bytes, so
           # separate calls at equal bandwidth take 2.88x the forward
           "bytes_ratio_bwd_over_fwd": fb_bytes / chain_bytes(16)}
    # the same at 64 frames, where the fixed costs of a launch weigh less
    del xd, wd, gx, y
    chain, (x,), w = W.config4(frames=64)
    c = A.Chain(chain)
    xd = torch.from_numpy(x).cuda()
    wd = torch.from_numpy(w).cuda()
    y = c.run([xd])
    gx = torch.empty_like(xd)
    for _ in range(3):
        c.run([xd], y)
        c.backward(wd, [xd], gx, gt)
        c.fwd_bwd([xd], wd, y, gx, gt)
    f64 = statistics.median(time_each_flushed(lambda: c.run([xd], y), reps, stream, flush))
    b64 = statistics.median(time_each_flushed(lambda: c.backward(wd, [xd], gx, gt), reps, stream, flush))

    def both64():
        c.run([xd], y)
        c.backward(wd, [xd], gx, gt)
    fb64 = statistics.median(time_each_flushed(both64, reps, stream, flush))
    fu64 = statistics.median(time_each_flushed(lambda: c.fwd_bwd([xd], wd, y, gx, gt), reps, stream, flush))
    c.sync_status()
    out["frames64"] = {"fwd_ms": f64, "bwd_ms": b64, "fwd_plus_bwd_ms": fb64, "ratio": fb64 / f64,
                       "fused_fwd_bwd_ms": fu64, "fused_ratio": fu64 / f64,
                       "bwd_gbs": (8 * x.size + 4 * w.size) / (b64 * 1e-3) / 1e9}
    return out


def bench_matmul(A, torch, stream, flush, reps, peak_tf):
    tk, (a, b) = W.config2()
    t = A.Task(tk)
    ad = torch.from_numpy(a.view(np.int16)).cuda().view(torch.bfloat16)
    bd = torch.from_numpy(b.view(np.int16)).cuda().view(torch.bfloat16)
    c = t.run([ad, bd])
    for _ in range(3):
        t.run([ad, bd], c)
    t.sync_status()
    ms = statistics.median(time_each_flushed(lambda: t.run([ad, bd], c), reps, stream, flush))
    ref = statistics.median(time_each_flushed(lambda: torch.matmul(ad, bd), reps, stream, flush))
    flops = 2.0 * 4096 ** 3
    out = {"mnk": [4096, 4096, 4096], "ms": ms, "tflops": flops / (ms * 1e-3) / 1e12,
           "frac_of_bf16_peak": flops / (ms * 1e-3) / 1e12 / peak_tf,
           "torch_matmul_bf16_out_ms": ref, "torch_tflops": flops / (ref * 1e-3) / 1e12}
    # like for like: cuBLAS with a float32 C, as this task writes it
    c32 = torch.empty((4096, 4096), dtype=torch.float32, device="cuda")
    try:
        torch.mm(ad, bd, out_dtype=torch.float32, out=c32)
        ref32 = statistics.median(time_each_flushed(lambda: torch.mm(ad, bd, out_dtype=torch.float32, out=c32),
                                                    reps, stream, flush))
        out.update(torch_mm_f32_out_ms=ref32, torch_mm_f32_out_tflops=flops / (ref32 * 1e-3) / 1e12,
                   ratio_vs_cublas_f32_out=ref32 / ms)
    except (TypeError, RuntimeError) as e:
        out["torch_mm_f32_out"] = f"unavailable: {type(e).__name__}"
    return out


def bench_bf16(A, torch, stream, flush, reps, hbm):
    """The same 64x1080x1920 chain with bfloat16 frames and output (f32
    arithmetic and intermediate): half the bytes per tiler element."""
    chain, (x,) = W.config1_bf16(seed=2)
    c = A.Chain(chain)
    xd = torch.from_numpy(x.view(np.int16)).cuda().view(torch.bfloat16)
    y = c.run([xd])
    for _ in range(3):
        c.run([xd], y)
    ms = statistics.median(time_each_flushed(lambda: c.run([xd], y), reps, stream, flush))
    nbytes = 2 * FRAMES * HEIGHT * WIDTH + 2 * FRAMES * (HEIGHT // 8 * 3) * (WIDTH // 8 * 3)
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"workload": "64x1080x1920 bf16 -> 64x405x720 bf16", "ms": ms, "elems_per_s": chain_units(FRAMES) / (ms * 1e-3),
            "unique_bytes": nbytes, "gbs": gbs, "frac_of_hbm": gbs / hbm}


def bench_f16(A, torch, stream, flush, reps, hbm):
    """The same 64x1080x1920 chain with IEEE half frames and output (f32
    arithmetic and intermediate)."""
    chain, (x,) = W.config1_f16(seed=3)
    c = A.Chain(chain)
    xd = torch.from_numpy(x).cuda()
    y = c.run([xd])
    for _ in range(3):
        c.run([xd], y)
    ms = statistics.median(time_each_flushed(lambda: c.run([xd], y), reps, stream, flush))
    nbytes = 2 * FRAMES * HEIGHT * WIDTH + 2 * FRAMES * (HEIGHT // 8 * 3) * (WIDTH // 8 * 3)
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"workload": "64x1080x1920 f16 -> 64x405x720 f16", "ms": ms, "elems_per_s": chain_units(FRAMES) / (ms * 1e-3),
            "unique_bytes": nbytes, "gbs": gbs, "frac_of_hbm": gbs / hbm}


def bench_cg(A, torch, stream, flush, reps, hbm):
    """Conjugate gradient of the case study on a synthetic SPD matrix with the
    paper's N and NNZ (27-point stencil on 51^3), tol 1e-10, float64."""
    from oracle import cg as CG
    row_ptr, col, vals, b = W.stencil27_csr(51)
    rp, cd, vd = (torch.from_numpy(a).cuda() for a in (row_ptr, col, vals))
    solver = A.ConjugateGradient(rp, cd, vd)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    solver.solve(bd, x, 1e-10, 1000)
    ts = []
    for _ in range(max(3, min(reps, 10))):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        iters, rel = solver.solve(bd, x, 1e-10, 1000)[1:]
        ts.append(time.perf_counter() - t0)
    solve_s = statistics.median(ts)
    y = torch.empty_like(bd)
    spmv_hbm = statistics.median(time_each_flushed(lambda: solver.spmv(bd, y), reps, stream, flush))
    spmv_l2 = time_loop(lambda: solver.spmv(bd, y), 20, stream) / 20
    n, nnz = len(b), int(row_ptr[-1])
    nbytes = 12 * nnz + 8 * (n + 1) + 16 * n
    t0 = time.perf_counter()
    _, k_cpu, _ = CG.cg(row_ptr, col, vals, b, tol=1e-10)
    cpu_s = time.perf_counter() - t0
    return {"n": n, "nnz": nnz, "tol": 1e-10, "iterations": iters, "rel_residual": rel, "solve_ms": solve_s * 1e3,
            "ms_per_iteration": solve_s * 1e3 / max(iters, 1), "spmv_us_after_l2_flush": spmv_hbm * 1e3,
            "spmv_gbs_after_l2_flush": nbytes / (spmv_hbm * 1e-3) / 1e9, "spmv_frac_of_hbm": nbytes / (spmv_hbm * 1e-3) / 1e9 / hbm,
            "spmv_us_l2_resident": spmv_l2 * 1e3,
            # the float64 side of the SpMV roofline: one multiply-add per nonzero
            "spmv_fp64": {"bound": "fp64", "achieved": 2 * nnz / (spmv_hbm * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                          "unit": "TFLOP/s", "frac": 2 * nnz / (spmv_hbm * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                          "frac_l2_resident": 2 * nnz / (spmv_l2 * 1e-3) / 1e12 / FP64_PEAK_TFLOPS},
            "oracle_cpu_s": cpu_s, "oracle_iterations": k_cpu,
            "paper_table1_context": {"hardware": "Tesla T10 (OpenCL, 1 GPU) / Core 2 Duo (Matlab pcg), FP64",
                                     "opencl_1gpu_s": 0.659, "matlab_pcg_s": 3.17, "iterations": 116}}


def bench_config0(A, torch, stream, reps):
    tk, (x,) = W.config0()
    t = A.Task(tk)
    xd = torch.from_numpy(x).cuda()
    y = t.run([xd])
    for _ in range(10):
        t.run([xd], y)
    ms = time_loop(lambda: t.run([xd], y), reps, stream) / reps
    return {"us_per_call": ms * 1e3}


def cpu_baseline_chain(max_seconds=12.0):
    """The C oracle, as it stands, on a bounded sample of the chain workload
    (whole frames of 1080x1920), on all host cores."""
    from oracle import cpu_ref as C
    frames = 1
    g = W.rng(1)
    while True:
        chain, (x,) = W.config1(seed=1, frames=frames)
        t0 = time.perf_counter()
        C.run_chain(chain, [x])
        dt = time.perf_counter() - t0
        if dt * 2 > max_seconds or frames >= FRAMES:
            break
        frames = min(FRAMES, max(frames * 2, int(frames * max_seconds / max(dt, 1e-3) / 2)))
    del g
    # the same oracle on one core, one frame
    cores = C.threads()
    chain1, (x1,) = W.config1(seed=1, frames=1)
    C.set_threads(1)
    try:
        t0 = time.perf_counter()
        C.run_chain(chain1, [x1])
        dt1 = time.perf_counter() - t0
    finally:
        C.set_threads(cores)
    return {"value": chain_units(frames) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{frames} of 64 frames (1080x1920), full chain, float64 accumulation",
            "seconds": dt, "single_core": {"value": chain_units(1) / dt1, "sample": "1 frame", "seconds": dt1}}


# -------------------------------------------------------------- main arms

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import cpu_ref as C
    frames = 2
    chain, (x,) = W.config1(seed=1, frames=frames)
    for _ in range(args.warmup):
        C.run_chain(chain, [x])
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        C.run_chain(chain, [x])
        ts.append(time.perf_counter() - t0)
    total = sum(ts)
    value = chain_units(frames) * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_frames": frames},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": C.threads(), "kind": "oracle",
                             "sample": f"{frames} of 64 frames per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    import paper_1105_4424_gb300 as A
    hbm, bf16, bf16_sus, peak_kind = measured_peaks()
    stream = torch.cuda.current_stream()

    # equal partition (Sec. 7): the job is FRAMES * world frames with the
    # 64-frame workload's taps (seed 0); this rank's chain is its part from
    # arol_task_shard_frames (FRAMES frames), its frames drawn from seed `rank`
    chain0, (x,) = W.config1(seed=rank)
    taps = [t["taps"] for t in (chain0 if rank == 0 else W.config1(seed=0)[0])]
    job = W.downscale_chain(FRAMES * world, HEIGHT, WIDTH, *taps)
    from paper_1105_4424_gb300 import shard
    chain, first = shard.shard_chain(job, world, rank)
    assert chain[0]["inputs"][0]["shape"] == x.shape and first == rank * FRAMES
    c = A.Chain(chain)
    xd = torch.from_numpy(x).cuda()
    y = c.run([xd])
    units = chain_units(FRAMES)
    nbytes = chain_bytes(FRAMES)

    nvml = NvmlSampler(local)
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            c.run([xd], y)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        with nvml:
            ms = time_loop(lambda: c.run([xd], y), args.steps, stream)
        torch.cuda.synchronize()
        barrier(world)
    all_ms = dist_max(ms, world)
    value, ms_per_step = aggregate(all_ms, [units * args.steps] * world, args.steps)
    # one step moves `units` tiler elements per rank: value * time per step must give them back
    assert abs(value * ms_per_step * 1e-3 - units * world) <= 1e-6 * units * world
    kernel_ms = ms / args.steps                      # one kernel launch per step
    achieved = nbytes / (kernel_ms * 1e-3) / 1e9

    # end to end through the C ABI with page-locked host buffers
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty(tuple(chain[-1]["outputs"][0]["shape"]), dtype=torch.float32).pin_memory()
    for _ in range(2):
        c.run_host([xh], yh)
    e2e_steps = max(3, min(args.steps, 20))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        c.run_host([xh], yh)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    all_e2e = dist_max(e2e_s * 1e3, world)
    e2e_value = units * world / (max(all_e2e) * 1e-3)
    # ceiling for the host-buffer path: one plain pinned copy of the input
    xdev = torch.empty_like(xd)
    for _ in range(2):
        xdev.copy_(xh, non_blocking=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        xdev.copy_(xh, non_blocking=True)
    torch.cuda.synchronize()
    h2d_gbs = x.nbytes * e2e_steps / (time.perf_counter() - t0) / 1e9
    del xdev

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_gpu": FRAMES, "tiler_elems_per_step_per_gpu": units,
                       "unique_bytes_per_step_per_gpu": nbytes,
                       "l2": "inputs (531 MB per step) exceed L2 (126 MB): no flush; extras flush L2 with a 256 MB write then a 256 MB read of a clean buffer",
                       "parallelism": f"frames split equally over {world} GPUs (no exchange)" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "kernel": "downscale_bulk_kernel<0>", "achieved": achieved, "peak": hbm,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": headline_traffic(), "algorithmic_bytes": nbytes},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(x.nbytes),
                    "d2h_bytes_per_step": int(yh.numel() * 4), "ms_per_step": e2e_s * 1e3,
                    "path": "arol_task_run_host, 8 frame chunks pipelined over 3 streams",
                    "pinned_h2d_copy_gbs": h2d_gbs},
            "gpu_launches": args.steps,
            "clocks": nvml.summary() or dict(clk.summary(), source="nvidia-smi")}
    if rank == 0 and world == 1 and not args.no_extras:
        flush = L2Flush(torch)
        reps = max(5, min(args.steps, 20))
        line["config0"] = bench_config0(A, torch, stream, 200)
        line["batched"] = bench_batched(A, torch, stream, flush, reps)
        line["batched_chains"] = bench_batched_chains(A, torch, stream, flush, reps, hbm)
        line["stencil"] = bench_stencil(A, torch, stream, flush, reps, hbm)
        line["chain_5to2"] = bench_chain_5to2(A, torch, stream, flush, reps, hbm)
        line["config0_scaled"] = bench_config0_scaled(A, torch, stream, flush, reps, hbm)
        line["generic_diagonal"] = bench_generic(A, torch, stream, flush, reps, hbm)
        line["fwd_bwd"] = bench_backward(A, torch, stream, flush, reps)
        line["matmul"] = bench_matmul(A, torch, stream, flush, reps, bf16)
        line["bf16_storage"] = bench_bf16(A, torch, stream, flush, reps, hbm)
        line["f16_storage"] = bench_f16(A, torch, stream, flush, reps, hbm)
        line["cg"] = bench_cg(A, torch, stream, flush, reps, hbm)
        del flush
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_chain()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def warm_clocks(torch, buf, seconds=0.3):
    """Keep the GPU busy for a moment so its clocks leave the idle state."""
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for _ in range(20):
            buf.zero_()
        torch.cuda.synchronize()


def run_case(args):
    """One measurement alone (for profiling): prints its JSON object."""
    import torch
    import paper_1105_4424_gb300 as A
    hbm, bf16, _, _ = measured_peaks()
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch)
    reps = max(1, args.steps)
    warm_clocks(torch, flush.w)
    if args.case == "batched":
        out = bench_batched(A, torch, stream, flush, reps, tune=not args.no_tune)
    elif args.case == "stencil":
        out = bench_stencil(A, torch, stream, flush, reps, hbm)
    elif args.case == "chains":
        out = bench_batched_chains(A, torch, stream, flush, reps, hbm)
    elif args.case == "chain5to2":
        out = bench_chain_5to2(A, torch, stream, flush, reps, hbm)
    elif args.case == "config0_scaled":
        out = bench_config0_scaled(A, torch, stream, flush, reps, hbm)
    elif args.case == "generic":
        out = bench_generic(A, torch, stream, flush, reps, hbm)
    elif args.case == "backward":
        out = bench_backward(A, torch, stream, flush, reps)
    elif args.case == "matmul":
        out = bench_matmul(A, torch, stream, flush, reps, bf16)
    elif args.case == "cg":
        out = bench_cg(A, torch, stream, flush, reps, hbm)
    elif args.case == "bf16":
        out = bench_bf16(A, torch, stream, flush, reps, hbm)
    elif args.case == "f16":
        out = bench_f16(A, torch, stream, flush, reps, hbm)
    else:
        out = bench_config0(A, torch, stream, reps)
    print(json.dumps({"case": args.case, **out}))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="headline only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", choices=["batched", "chains", "chain5to2", "config0_scaled", "generic", "stencil", "backward",
                                       "matmul", "config0", "cg", "bf16", "f16"],
                    help="run one extra measurement alone (profiling)")
    ap.add_argument("--no-tune", action="store_true", help="batched case: keep the default launch shape")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
