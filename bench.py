#!/usr/bin/env python3
"""Throughput of the RSST finite-volume step on GB300.

Metric: cell-updates per second per RK stage (cells x 2 stages per step /
time).  Default workload: the 2D periodic 512 x 512 float64 shear layer at
Mach 0.01 (density ratio 10, tanh width 0.02, xi = 30, semi-conservative
PVS form), adaptive CFL dt.  One step = one SSP-RK2 step = two fused stage
kernels.  The state (8 MB per field set) fits in L2, so a 256 MiB buffer is
written between timed steps (outside the timed events) to flush it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (test
infrastructure, run here only as the reference arm) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "cell-updates/s per RK stage"
UNIT = "cell-updates/s"
L2_FLUSH_BYTES = 256 << 20

# float64 operations per cell per stage of the fused kernel, counted from the
# algorithm: 2D, per face 122 (+2 div, 4 sqrt), divergence 8, correction +
# force + RK ~40 (+3 div, 2 sqrt); div and sqrt counted as one operation each.
FP64_FLOPS_PER_CELL_STAGE_2D = 2 * (122 + 6) + 8 + 45
FP64_FLOP_COUNT = ("algorithmic float64 operations per 2D cell-stage, counted from the algorithm "
                   "(bench.py FP64_FLOPS_PER_CELL_STAGE_2D: per face 122 + 2 divisions + 4 square roots, "
                   "divergence 8, correction + force + RK 45)")

# float64 operations of the discrete adjoint per primal cell-stage (2D, PVS,
# constant xi), counted the same way from the reverse-mode code: the forward
# record and the segment recompute are one forward stage each (309); the
# stage VJP is 2 faces x 334 (face states 48, two c_tot evaluations 32, LLF
# reverse 36, two flux reverses 148, MC reverse 64, phi 8, xi 2) + the
# reduced-tendency reverse 133 + the mu scaling, gather and combines 52.
ADJ_FLOPS_PER_CELL_STAGE_2D = 309 + 309 + (2 * 334 + 133 + 52)


def _sources_sha(files):
    """Hash of the kernel sources' code (comments and blank lines removed),
    so that the stored DRAM traffic of a kernel goes stale when its code
    changes but not when only its comments do."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_1812_04135_gb300", "csrc", f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code = "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())
        h.update(code.encode())
    return h.hexdigest()[:16]


def _traffic_key(key):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary (profiles/traffic.json), only if its sources are unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        table = json.load(f)
    e = table.get(key)
    if not e or _sources_sha(e["sources"]) != e["sources_sha"]:
        return None
    return e["dram_bytes_per_launch"]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """SM clock and clock-event reasons DURING the timed region.

    NVML (the library nvidia-smi reads; queries only, nothing is set) is
    opened once at start-up, then read when the region opens and when it
    closes (so a region of a few milliseconds still has its clock on both
    sides), and every 100 ms in between from a thread.  A query takes under
    0.1 ms, but a Python thread polling every 5 ms slowed the launching loop
    tenfold (the two contend for the interpreter lock), which starved the GPU
    of work and lowered the very clock being read.  Without
    NVML, nvidia-smi -lms 200 is started and its first line awaited before
    the region opens."""
    INTERVAL_S = 0.1

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # clock-event reason bits of the NVML API
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40, "hw_power_brake_slowdown": 0x80}
    NVML_CLOCK_SM = 1

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.samples = []      # (sm_mhz, reason_bits) from NVML
        self.max_mhz = None
        self.nvml = None
        self.source = None

    # -- NVML ---------------------------------------------------------------
    _handles = {}  # device index -> (lib, handle, reasons query, ctypes, max MHz), opened once per process

    @classmethod
    def open_nvml(cls, index: int) -> bool:
        """Initialise NVML and find the device once (it takes a few hundred
        milliseconds: done before warm-up, never between warm-up and the
        timed region, where the idle GPU would lower its clock)."""
        if index in cls._handles:
            return cls._handles[index] is not None
        cls._handles[index] = None
        import ctypes as C
        try:
            lib = C.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return False
            dev = C.c_void_p()
            ok = False
            try:
                pr = torch.cuda.get_device_properties(index)
                bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
                ok = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), C.byref(dev)) == 0
            except Exception:
                ok = False
            if not ok and lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(dev)) != 0:
                return False
            reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = C.c_uint()
            max_mhz = float(mx.value) if lib.nvmlDeviceGetMaxClockInfo(dev, cls.NVML_CLOCK_SM, C.byref(mx)) == 0 else None
            cls._handles[index] = (lib, dev, reasons, C, max_mhz)
            return True
        except Exception:
            return False

    def _nvml_open(self):
        if not self.open_nvml(self.index):
            return False
        lib, dev, reasons, C, self.max_mhz = self._handles[self.index]
        self.nvml = (lib, dev, reasons, C)
        return True

    def _nvml_sample(self):
        lib, dev, reasons, C = self.nvml
        clk, bits = C.c_uint(), C.c_ulonglong()
        if lib.nvmlDeviceGetClockInfo(dev, self.NVML_CLOCK_SM, C.byref(clk)) == 0 and \
                reasons(dev, C.byref(bits)) == 0:
            self.samples.append((float(clk.value), int(bits.value)))

    def _nvml_loop(self):
        while not self.stop.wait(self.INTERVAL_S):
            self._nvml_sample()

    # -- nvidia-smi fallback --------------------------------------------------
    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.first.set()

    def __enter__(self):
        self.stop = threading.Event()
        if self._nvml_open():
            self.source = "nvml: region open and close, every 100 ms between"
            self._nvml_sample()
            self.t = threading.Thread(target=self._nvml_loop, daemon=True)
            self.t.start()
            return self
        try:
            self.first = threading.Event()
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self.first.wait(5.0)
            self.lines.clear()  # keep only samples taken once the region has opened
            self.source = "nvidia-smi, every 200 ms"
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.nvml:
            self.stop.set()
            self.t.join(timeout=1.0)
            self._nvml_sample()
            return
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], self.max_mhz, set()
        if self.nvml:
            for mhz, bits in self.samples:
                sm.append(mhz)
                reasons |= {nm for nm, b in self.BITS.items() if bits & b}
        else:
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for ln in self.lines:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm), "source": self.source}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("RSST_DIST_BACKEND") or ("nccl" if torch.cuda.is_available() else "gloo")
        dist.init_process_group(backend)
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    on_gpu = dist.get_backend() == "nccl"
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if on_gpu else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(args):
    from paper_1812_04135_gb300 import inputs
    if args.workload == "polytrope3d":
        return inputs.polytrope_3d(variant=args.variant)
    return inputs.shear_layer_2d(args.n, args.n, xi=30.0, variant=args.variant, ratio=10.0)


def bytes_per_cell_stage(w, precision):
    """Algorithmic HBM bytes per cell per stage: stage 1 reads and writes one
    state, stage 2 reads two and writes one: 2.5 * nvar * bytes per scalar
    (8 for float64 and double-float, 4 for float32)."""
    nvar = w["ndim"] + 2
    return 2.5 * nvar * (4 if precision == "fp32_pert" else 8)


_FP64_PEAK = {}


def fp64_peak_measured(dev):
    """Float64 FMA throughput of this GPU (TFLOP/s) from the library's probe
    kernel (rsst_fp64_fma_peak: independent FMA chains on every SM, CUDA
    events), measured once per process, with the SM clock read during it."""
    if dev.index not in _FP64_PEAK:
        from paper_1812_04135_gb300 import rsst
        with ClockSampler(dev.index) as clk:
            tf, ms = rsst.rsst_fp64_fma_peak(8000)
        _FP64_PEAK[dev.index] = (tf, ms, clk.summary().get("sm_mhz"))
    return _FP64_PEAK[dev.index]


def _roof_hbm(w, precision, cells, launch_s, peaks, src, traffic_key):
    alg = bytes_per_cell_stage(w, precision) * cells
    gbs = alg / launch_s / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / peaks["hbm_gbs"], "traffic": _traffic_key(traffic_key) if traffic_key else None,
            "algorithmic_bytes_per_launch": alg, "peak_source": src}


def _roof_alu(flops_per_cell_stage, cells, launch_s, dev, what):
    tf_peak, _, mhz = fp64_peak_measured(dev)
    tf = flops_per_cell_stage * cells / launch_s / 1e12
    return {"bound": "alu", "achieved": tf, "peak": tf_peak, "unit": "TFLOP/s", "frac": tf / tf_peak,
            "traffic": None, "flops_per_cell_stage": flops_per_cell_stage, "flop_count": what,
            "peak_source": f"measured: rsst_fp64_fma_peak probe (float64 FMA chains on every SM) at {mhz} MHz"}


def measure_single(w, precision, steps, warmup, dev, peaks, src, *, flush_l2=True, traffic_key=None,
                   alu_flops=None, e2e_steps=None, bound=None, extra=None):
    """One single-run configuration as a full bench entry: `steps` SSP-RK2
    steps timed one by one with CUDA events on the launching stream (after
    `warmup` untimed steps; with flush_l2 a 256 MiB buffer is written between
    steps, outside the events), SM clocks sampled during the timed region,
    the HBM roofline of the stage kernel (and the float64 arithmetic roofline
    when alu_flops is given), and the same steps end to end through the C
    ABI with the state copied in from and out to pinned host memory."""
    from paper_1812_04135_gb300 import rsst
    stream = torch.cuda.current_stream(dev)
    s = rsst.Solver(w, precision, stream=stream)
    U0 = torch.from_numpy(w["U"]).to(dev)
    s.set_state(U0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev) if flush_l2 else None
    for _ in range(warmup):
        s.step(1)
    s.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    l0 = s.launches()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        for k in range(steps):
            if flush is not None:
                flush.fill_(float(k))
            ev[k][0].record(stream)
            s.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = s.launches() - l0
    s.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t = sum(step_ms) / 1e3
    # end to end: host state in, step, host state out, every step
    ne = e2e_steps or steps
    host_in = torch.from_numpy(w["U"]).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    rsst.rsst_set_state(s.h, host_in, on_host=True)
    s.step(1)
    rsst.rsst_get_state(s.h, host_out, on_host=True)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(ne):
        rsst.rsst_set_state(s.h, host_in, on_host=True)
        s.step(1)
        rsst.rsst_get_state(s.h, host_out, on_host=True)
    torch.cuda.synchronize()
    e_el = time.perf_counter() - e0
    s.close()
    del flush
    cells = int(np.prod(w["n"]))
    launch_s = t / (2 * steps)
    hbm = _roof_hbm(w, precision, cells, launch_s, peaks, src, traffic_key)
    d = {"value": cells * 2 * steps / t, "unit": UNIT, "steps": steps, "warmup": warmup,
         "ms_per_step": t / steps * 1e3, "step_ms_median": statistics.median(step_ms), "cells": cells,
         "roofline": hbm, "clocks": clk.summary(), "gpu_launches": launches,
         "l2": "256 MiB buffer written between timed steps" if flush_l2 else "state larger than L2",
         "e2e": {"value": cells * 2 * ne / e_el, "unit": UNIT, "steps": ne,
                 "h2d_bytes_per_step": host_in.numel() * 8, "d2h_bytes_per_step": host_out.numel() * 8}}
    if alu_flops:
        d["roofline"] = _roof_alu(alu_flops[0], cells, launch_s, dev, alu_flops[1])
        d["roofline"]["hbm"] = {k: hbm[k] for k in ("achieved", "peak", "frac", "traffic", "unit")}
    if bound:
        d["bound"] = bound
    if extra:
        d.update(extra)
    return d


def measure_batched(dev, peaks, src, steps=20, warmup=3, world=1):
    """64 independent float32-perturbation shear layers of uneven size, xi and
    density ratio (2.5e7 cells, 0.8 GB of state: inputs larger than L2): one
    persistent kernel per stage over all runs' tiles (graph-captured) against
    one launch pair per run per step, tile shape from the autotuner."""
    from paper_1812_04135_gb300 import inputs, rsst
    ws = inputs.batched_runs(count=64, seed=4)
    cells = sum(int(np.prod(w["n"])) for w in ws)
    b = rsst.BatchSolver(ws)
    for i, w in enumerate(ws):
        b.set_state(i, torch.from_numpy(w["U"]).to(dev))
    choice, tune_ms = b.autotune(3)
    shape = b.tile_shape()
    stream = b.stream

    def timed(fn):
        for _ in range(warmup):
            fn(1)
        b.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        _barrier(world)
        torch.cuda.synchronize()
        for k in range(steps):
            ev[k][0].record(stream)
            fn(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        _barrier(world)
        return sum(a.elapsed_time(c) for a, c in ev) / 1e3

    l0 = b.launches()
    with ClockSampler(dev.index) as clk:
        t_persist = timed(b.step)
    launches = b.launches() - l0 - 2 * warmup
    with ClockSampler(dev.index) as clk_loop:
        t_loop = timed(b.step_looped)
    b.sync()
    # end to end through the C ABI with host buffers, every run, every step
    hosts = [torch.from_numpy(w["U"]).pin_memory() for w in ws]
    outs = [torch.empty_like(h).pin_memory() for h in hosts]
    ne = max(2, steps // 4)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(ne):
        for i in range(len(ws)):
            rsst.rsst_batch_set_state(b.b, i, hosts[i], on_host=True)
        b.step(1)
        for i in range(len(ws)):
            rsst.rsst_batch_get_state(b.b, i, outs[i], on_host=True)
    torch.cuda.synchronize()
    e_el = time.perf_counter() - e0
    nbytes = sum(h.numel() * 8 for h in hosts)
    b.close()
    launch_s = t_persist / (2 * steps)
    alg = 40 * cells
    hbm = alg / launch_s / 1e9
    return {"value": cells * 2 * steps / t_persist, "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": t_persist / steps * 1e3, "cells": cells, "runs": len(ws),
            "tile_shape": shape, "autotune_choice": choice, "autotune_ms_per_step": tune_ms,
            "roofline": {"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": hbm / peaks["hbm_gbs"], "traffic": _traffic_key(f"batched:fp32_pert:{len(ws)}"),
                         "algorithmic_bytes_per_launch": alg, "peak_source": src},
            "looped_single_run": {"value": cells * 2 * steps / t_loop, "ms_per_step": t_loop / steps * 1e3,
                                  "clocks": clk_loop.summary()},
            "persistent_over_looped": t_loop / t_persist,
            "e2e": {"value": cells * 2 * ne / e_el, "unit": UNIT, "steps": ne,
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "gpu_launches": launches, "clocks": clk.summary(), "l2": "inputs larger than L2 (0.8 GB of state)"}


def measure_adjoint(dev, steps=3, warmup=1):
    """Discrete adjoint of the 2D 256^2 float64 stratified box (contrast 20,
    xi = 20): forward record of 400 steps with a checkpoint every 20, then the
    reverse sweep for dJ/dU0 and dJ/dxi of the final kinetic energy; one
    bench step is one full gradient, timed with CUDA events.  The value counts
    the primal cell-stages (cells x 2 x 400) per second of forward + reverse."""
    from paper_1812_04135_gb300 import inputs, rsst
    w = inputs.polytrope_2d(256, 256, xi=20.0, contrast=20.0, amp=1e-3)
    cells, nsteps, every = 256 * 256, 400, 20
    stream = torch.cuda.current_stream(dev)
    s = rsst.Solver(w, "fp64", stream=stream)
    U0 = torch.from_numpy(w["U"]).to(dev)
    s.set_state(U0)
    dt = s.dt()
    g = torch.empty(tuple(U0.shape), dtype=torch.float64, device=dev)

    def gradient(src, on_host=False):
        rsst.rsst_set_state(s.h, src, on_host=on_host)
        rsst.rsst_adjoint_record(s.h, dt, nsteps, every)
        rsst.rsst_kinetic_energy(s.h, g)
        dxi = 0.0
        for seg in reversed(range(rsst.rsst_adjoint_segments(s.h))):
            dxi += rsst.rsst_adjoint_step(s.h, seg, g)
        return dxi

    for _ in range(warmup):
        gradient(U0)
    torch.cuda.synchronize()
    l0 = s.launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(dev.index) as clk:
        for k in range(steps):
            ev[k][0].record(stream)
            dxi = gradient(U0)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = s.launches() - l0
    t = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    host_in = torch.from_numpy(w["U"]).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(steps):
        gradient(host_in, on_host=True)
        host_out.copy_(g, non_blocking=True)
        torch.cuda.synchronize()
    e_el = time.perf_counter() - w0
    s.close()
    primal = cells * 2 * nsteps
    launch_s = t / steps  # one gradient
    roof = _roof_alu(ADJ_FLOPS_PER_CELL_STAGE_2D, primal, launch_s, dev,
                     "algorithmic float64 operations per primal cell-stage of forward record, segment recompute "
                     "and reverse sweep (bench.py ADJ_FLOPS_PER_CELL_STAGE_2D); whole gradient, all kernels")
    return {"value": primal * steps / t, "unit": UNIT + " (primal cell-stages of forward record + reverse sweep)",
            "steps": steps, "warmup": warmup, "ms_per_step": t / steps * 1e3, "cells": cells,
            "steps_per_gradient": nsteps, "checkpoint_every": every, "roofline": roof, "clocks": clk.summary(),
            "gpu_launches": launches, "dJ_dxi": dxi,
            "e2e": {"value": primal * steps / e_el, "unit": UNIT, "steps": steps,
                    "h2d_bytes_per_step": host_in.numel() * 8, "d2h_bytes_per_step": host_out.numel() * 8}}


def run_modes(dev, peaks, src):
    """The other configurations the metric covers, each as a full entry
    (CUDA events, clocks, roofline, e2e), for the same JSON line."""
    from paper_1812_04135_gb300 import inputs, rsst
    out = {}
    hbm_fp32 = "hbm (instruction-issue limited)"
    w = inputs.shear_layer_2d(512, 512, xi=30.0, variant="pvs")
    out["fp32_pert_shear_512"] = measure_single(w, "fp32_pert", 20, 3, dev, peaks, src, bound=hbm_fp32,
                                                traffic_key="shear2d:fp32_pert:512")
    w = inputs.shear_layer_2d(2048, 2048, xi=30.0, variant="pvs")
    out["fp32_pert_shear_2048"] = measure_single(w, "fp32_pert", 20, 3, dev, peaks, src, flush_l2=False,
                                                 bound=hbm_fp32, traffic_key="shear2d:fp32_pert:2048", e2e_steps=5)
    w = inputs.shear_layer_2d(4096, 4096, xi=30.0, variant="pvs")
    out["fp32_pert_shear_4096"] = measure_single(w, "fp32_pert", 20, 3, dev, peaks, src, flush_l2=False,
                                                 bound=hbm_fp32, traffic_key="shear2d:fp32_pert:4096", e2e_steps=3)
    out["fp64_shear_4096"] = measure_single(w, "fp64", 20, 3, dev, peaks, src, flush_l2=False,
                                            traffic_key="shear2d:fp64:4096", e2e_steps=3,
                                            alu_flops=(FP64_FLOPS_PER_CELL_STAGE_2D, FP64_FLOP_COUNT))
    del w
    w = inputs.polytrope_3d(variant="pvs")
    out["fp64_polytrope_3d"] = measure_single(w, "fp64", 20, 3, dev, peaks, src, flush_l2=False,
                                              traffic_key="polytrope3d:fp64:256", e2e_steps=5,
                                              bound="alu (float64 pipe); HBM roofline of the primary 3D configuration")
    out["fp32_pert_polytrope_3d"] = measure_single(w, "fp32_pert", 20, 3, dev, peaks, src, flush_l2=False,
                                                   bound=hbm_fp32, traffic_key="polytrope3d:fp32_pert:256",
                                                   e2e_steps=5)
    df = {"dtype": "f32x2 double-float (48-bit significand), parity 1e-10 vs f64"}
    out["fp64_df_polytrope_3d"] = measure_single(w, "fp64_df", 10, 2, dev, peaks, src, flush_l2=False,
                                                 bound="alu (float32 pipe, double-float arithmetic)", extra=df,
                                                 e2e_steps=2)
    w = inputs.shear_layer_2d(512, 512, xi=30.0, variant="pvs")
    out["fp64_df_shear_512"] = measure_single(w, "fp64_df", 20, 3, dev, peaks, src,
                                              bound="alu (float32 pipe, double-float arithmetic)", extra=df)
    del w
    out["batched_fp32_pert_64runs"] = measure_batched(dev, peaks, src)
    out["adjoint_fp64_polytrope_256"] = measure_adjoint(dev)
    # 1D N=256 sound wave, 2000 steps: launch-bound; CUDA-graph blocks vs plain launches
    w = inputs.sound_wave_1d(256, xi=10.0, variant="pvs")
    for k, name in ((16, "fp64_sound1d_256_graph"), (0, "fp64_sound1d_256_plain")):
        stream = torch.cuda.current_stream(dev)
        s = rsst.Solver(w, "fp64", stream=stream)
        s.set_graph_steps(k)
        s.set_state(torch.from_numpy(w["U"]).to(dev))
        s.step(64)
        s.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev.index) as clk:
            e0.record(stream)
            s.step(2000)
            e1.record(stream)
            torch.cuda.synchronize()
        s.sync()
        s.close()
        t = e0.elapsed_time(e1) / 1e3
        out[name] = {"value": 256 * 2 * 2000 / t, "unit": UNIT, "steps_per_s": 2000 / t, "steps": 2000,
                     "graph_steps": k, "bound": "launch latency", "clocks": clk.summary()}
    return out


def run_batched(args, world, rank, local):
    """The batched workload as the bench's main line (--workload batched)."""
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, src = _peaks()
    d = measure_batched(dev, peaks, src, steps=args.steps, warmup=args.warmup, world=world)
    t_max = _max_over_ranks(d["ms_per_step"] * args.steps / 1e3, world)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": d["cells"] * 2 * args.steps * world / t_max, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (perturbation about an f64 background)", "data": "synthetic",
            "config": {"workload": "batched: 64 independent 2D shear layers, N in {128..1024}^2, xi in {1,3,10,30}, "
                                   "density ratio in {1,3,10,100}, FP32 perturbation, PVS, adaptive CFL per run",
                       "cells": d["cells"], "tile_shape": d["tile_shape"], "autotune_choice": d["autotune_choice"],
                       "l2": d["l2"], "parallelism": f"replicas x{args.gpus}"},
            "roofline": d["roofline"], "looped_single_run": d["looped_single_run"],
            "e2e": d["e2e"], "gpu_launches": d["gpu_launches"], "clocks": d["clocks"]}
    print(json.dumps(line), flush=True)


def run_adjoint(args, world, rank, local):
    """The adjoint workload as the bench's main line (--workload adjoint)."""
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    d = measure_adjoint(dev, steps=args.steps, warmup=args.warmup)
    t_max = _max_over_ranks(d["ms_per_step"] * args.steps / 1e3, world)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": d["cells"] * 2 * 400 * args.steps * world / t_max, "unit": d["unit"],
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "adjoint: 2D 256x256 stratified box, contrast 20, xi=20, FP64 PVS, 400 steps, "
                                   "checkpoint every 20, gradient of the final kinetic energy w.r.t. U0 and xi",
                       "cells": d["cells"], "steps_per_gradient": 400, "checkpoint_every": 20,
                       "l2": "working set (checkpoints, recompute storage) larger than L2",
                       "parallelism": f"replicas x{args.gpus}"},
            "roofline": d["roofline"], "e2e": d["e2e"], "gpu_launches": d["gpu_launches"], "clocks": d["clocks"],
            "dJ_dxi": d["dJ_dxi"]}
    print(json.dumps(line), flush=True)


def _oracle_rate(w, seconds: float):
    from oracle import rsst_oracle as ro
    from oracle.workload import problem_from
    prob, U = problem_from(w)
    cells = int(np.prod(w["n"]))
    t0 = time.perf_counter()
    steps = 0
    while True:
        dt = ro.cfl_dt(U, prob)
        U = ro.ssp_rk2_step(U, dt, prob)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return cells * 2 * steps / el, steps, el


def cpu_baseline(w, seconds: float):
    """The oracle as it stands on the host cores: full-grid steps until
    ~``seconds``; then a shorter sample on one core."""
    v, steps, el = _oracle_rate(w, seconds)
    threads = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        v1, steps1, el1 = _oracle_rate(w, max(2.0, seconds / 4))
    finally:
        torch.set_num_threads(threads)
    return {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{steps} full-grid SSP-RK2 steps of the {w['n'][0]}x{w['n'][1]} workload "
                      f"({el:.1f} s, torch CPU float64)",
            "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": f"{steps1} full-grid steps ({el1:.1f} s, one thread)"}}


def run_reference_adjoint(args):
    """The oracle's discrete adjoint (torch autograd of the oracle step) on
    the 256^2 adjoint workload: each step is a 2-step gradient with a
    checkpoint every step, a bounded sample of the 400-step gradient."""
    from oracle import adjoint as adj
    from oracle import rsst_oracle as ro
    from oracle.workload import problem_from
    from paper_1812_04135_gb300 import inputs
    w = inputs.polytrope_2d(256, 256, xi=20.0, contrast=20.0, amp=1e-3)
    prob, U = problem_from(w)
    dt = ro.cfl_dt(U, prob)
    cells, k = 256 * 256, 2
    for _ in range(args.warmup):
        adj.adjoint_run(U, prob, k, dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        adj.adjoint_run(U, prob, k, dt, 1)
    el = time.perf_counter() - t0
    v = cells * 2 * k * args.steps / el
    cfg = {"workload": "adjoint: 2D 256x256 stratified box, contrast 20, xi=20, FP64 PVS; oracle sample of "
                       f"{k}-step gradients", "cells": cells}
    return v, el, cfg, f"{args.steps} gradients of {k} steps (checkpoint every step) after {args.warmup} warm-up"


def run_reference_batched(args):
    """The oracle on the batched workload: each step advances 4 of the 64 runs
    by one SSP-RK2 step (rotating through the list), a bounded sample."""
    from oracle import rsst_oracle as ro
    from oracle.workload import problem_from
    from paper_1812_04135_gb300 import inputs
    ws = inputs.batched_runs(count=64, seed=4)
    probs = [problem_from(w) for w in ws]
    state = [U for _, U in probs]
    done = 0

    def one(i):
        prob = probs[i][0]
        state[i] = ro.ssp_rk2_step(state[i], ro.cfl_dt(state[i], prob), prob)
        return int(np.prod(ws[i]["n"]))

    for j in range(args.warmup):
        one(j % 64)
    t0 = time.perf_counter()
    for j in range(args.steps):
        for r in range(4):
            done += one((4 * j + r) % 64)
    el = time.perf_counter() - t0
    v = done * 2 / el
    cfg = {"workload": "batched: 64 independent 2D shear layers, N in {128..1024}^2; oracle sample of 4 runs per step",
           "cells": sum(int(np.prod(w["n"])) for w in ws)}
    return v, el, cfg, f"{args.steps} steps of 4 runs each (rotating through the 64) after {args.warmup} warm-up"


def run_reference(args, world, rank):
    if rank != 0:
        return
    if args.workload in ("adjoint", "batched"):
        v, el, cfg, sample = (run_reference_adjoint if args.workload == "adjoint" else run_reference_batched)(args)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg,
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    w = workload(args)
    from oracle import rsst_oracle as ro
    from oracle.workload import problem_from
    prob, U = problem_from(w)
    cells = int(np.prod(w["n"]))
    for _ in range(args.warmup):
        U = ro.ssp_rk2_step(U, ro.cfl_dt(U, prob), prob)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = ro.ssp_rk2_step(U, ro.cfl_dt(U, prob), prob)
    el = time.perf_counter() - t0
    v = cells * 2 * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(args, w),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": f"{args.steps} timed full-grid steps after {args.warmup} warm-up steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(args, w):
    if args.workload == "polytrope3d":
        desc = (f"3D polytropic stratified box 256x128x128 {args.precision.upper()}, contrast 100, gravity -z, "
                f"reflecting z walls, xi=50, {args.variant.upper()} form, adaptive CFL 0.4")
    else:
        desc = (f"2D periodic shear layer {w['n'][0]}x{w['n'][1]} {args.precision.upper()}, Mach 0.01, "
                f"density ratio 10, xi=30, {args.variant.upper()} form, adaptive CFL 0.4")
    return {"workload": desc, "cells": int(np.prod(w["n"])), "variant": args.variant, "precision": args.precision,
            "l2": "256 MiB buffer written between timed steps",
            "parallelism": f"replicas x{args.gpus}"}


def run_gpu(args, world, rank, local):
    from paper_1812_04135_gb300 import rsst
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args)
    cells = int(np.prod(w["n"]))
    stream = torch.cuda.current_stream(dev)
    s = rsst.Solver(w, args.precision, stream=stream)
    U0 = torch.from_numpy(w["U"]).to(dev)
    s.set_state(U0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        s.step(1)
    s.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = s.launches()
    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        w0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            s.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    _barrier(world)
    launches = s.launches() - l0
    s.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = sum(step_ms) / 1e3
    t_max = _max_over_ranks(t_dev, world)
    value = cells * 2 * args.steps * world / t_max

    # end to end through the C ABI with host buffers: H2D state, step, D2H state
    host_in = torch.from_numpy(w["U"]).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    rsst.rsst_set_state(s.h, host_in, on_host=True)
    s.step(1)
    s.sync()
    _barrier(world)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        rsst.rsst_set_state(s.h, host_in, on_host=True)
        s.step(1)
        rsst.rsst_get_state(s.h, host_out, on_host=True)
    torch.cuda.synchronize()
    e_el = _max_over_ranks(time.perf_counter() - e0, world)
    e2e = cells * 2 * args.steps * world / e_el
    nbytes = host_in.numel() * 8
    s.close()

    peaks, src = _peaks()
    c = clk.summary()
    launch_s = t_dev / (2 * args.steps)
    hbm = _roof_hbm(w, args.precision, cells, launch_s, peaks, src, f"{args.workload}:{args.precision}:{w['n'][0]}")
    if args.precision == "fp64" and w["ndim"] == 2:
        roof = _roof_alu(FP64_FLOPS_PER_CELL_STAGE_2D, cells, launch_s, dev, FP64_FLOP_COUNT)
        roof["hbm"] = {k: hbm[k] for k in ("achieved", "peak", "frac", "traffic", "unit")}
    else:
        roof = hbm
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32_pert": "f32 (perturbation about an f64 background)",
                      "fp64_df": "f32x2 double-float (48-bit significand)"}[args.precision],
            "data": "synthetic", "config": _config(args, w),
            "roofline": roof,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "gpu_launches": launches, "clocks": c, "wall_s": wall,
            "step_ms_min": min(step_ms), "step_ms_median": statistics.median(step_ms)}
    if world == 1 and not args.no_modes and args.workload == "shear2d" and args.precision == "fp64" and args.n == 512:
        line["modes"] = run_modes(dev, peaks, src)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--variant", default="pvs")
    ap.add_argument("--workload", default="shear2d", choices=["shear2d", "polytrope3d", "batched", "adjoint"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_pert", "fp64_df"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-modes", action="store_true", help="only the headline configuration")
    args = ap.parse_args()
    world, rank, local = _dist()
    if args.impl != "reference" and torch.cuda.is_available():
        ClockSampler.open_nvml(local)  # before any warm-up
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batched":
        run_batched(args, world, rank, local)
    elif args.workload == "adjoint":
        run_adjoint(args, world, rank, local)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
