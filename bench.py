"""Benchmark of the FP64 iterative-stencil library on one GB300 (or N replicas).

One "step" is one full sweep of the headline workload: the 3D 7-point heat
stencil (u' = u + 0.1*(sum of the 6 face neighbours - 6u), periodic) on a
512^3 grid for T = 1000 time steps, starting from a uniform [0,1) field plus
the sine mode k = (3,5,7).  The metric is the paper's Eq. 5: cell updates per
second (N_x N_y N_z T / time), in GStencil/s.  The other workloads (2D 9-point
box 16384^2, 3D 27-point box 384^3, 2D 5-point heat 256^2, the 96-grid batched
form and the adjoint of the 256^3 variable-coefficient sweep) are reported
under "forms", each with its own rate and roofline fraction.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank advances its own replica (weak scaling); rank 0
prints one JSON line.
"""
import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "GStencil/s FP64 and roofline fraction at 1 GB300; batched/adjoint vs plain sweep"
HEADLINE = dict(name="heat3d-7pt", shape=(512, 512, 512), T=1000, alpha=0.1, boundary=1,
                sine=(3, 5, 7))
# algorithmic FP64 flops per cell update: K-tap weighted sum = K multiplies
# and K-1 adds; variable-coefficient step after hoisting the step-invariant
# face coefficients = 7 products and 6 sums; adjoint step = the transposed
# update (13) plus 3 faces x (2 differences, 1 product, 1 sum) = 25.
FLOPS = {"heat3d-7pt": 13, "box2d-9pt": 17, "box3d-27pt": 53, "heat2d-5pt": 9,
         "varcoef-7pt": 13, "adjoint-7pt": 13 + 25, "star2d-9pt": 17, "box2d-25pt": 49,
         "heat1d-3pt": 5, "star1d-5pt": 9}
NOMINAL_FP64_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12   # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz x 2 flop
# FP64 instructions the kernels issue per cell update (one pipe slot each):
# K for a K-tap chain; 4.25 for the equal-weight 9-point box with shared
# partial sums (17 warp instructions per 2 rows x 64 columns, strip edges
# included); adjoint: forward 7 + recompute 7 + transposed step 7 + 3 faces x 3.
INSTR = {"heat3d-7pt": 7, "box3d-27pt": 27, "box2d-9pt": 4.25, "heat2d-5pt": 5,
         "varcoef-7pt": 7, "adjoint-7pt": 7 + 7 + 7 + 9, "star2d-9pt": 9, "box2d-25pt": 25,
         "heat1d-3pt": 3 * (2048 + 8) / 2048, "star1d-5pt": 5 * (2048 + 16) / 2048}


# ------------------------------------------------------------------ helpers

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.first = threading.Event()
        self.start_line = 0

    def mark(self):
        """Count only the samples taken from now on (the timed region)."""
        self.start_line = len(self.lines)

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd.insert(1, f"--id={self.uuid}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi's start-up holds the driver for a while (launches and
        # copies from this process wait): time nothing until its first sample
        self.first.wait(timeout=10.0)

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())
            self.first.set()
        self.first.set()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.start_line:]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(ngpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank


def barrier_max(world, value):
    """Barrier, then the max of `value` over ranks."""
    if world == 1:
        return value
    from paper_2303_08365_gb300 import shard
    return shard.max_over_ranks(value)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cuda_time(fn, stream):
    """Milliseconds of fn() on `stream`, CUDA events on that stream."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


KERNEL_SOURCES = {"stream3d": ["stream.cu", "ptx.cuh", "taps.cuh"],
                  "stream2d": ["stream2d.cu", "ptx.cuh", "taps.cuh"],
                  "temporal": ["temporal.cu", "taps.cuh"],
                  "exchange": ["exchange.cu", "ptx.cuh", "taps.cuh"],
                  "direct": ["direct.cu", "taps.cuh"],
                  "batched": ["batched.cu"],
                  "persistent": ["batched.cu"],
                  "varcoef": ["varcoef.cu", "taps.cuh"],
                  "adjoint": ["varcoef.cu", "taps.cuh"]}


def _code_only(text):
    """C++/CUDA source without its comments and blank lines (a comment edit
    leaves the recorded counters valid)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_2303_08365_gb300", "csrc")
    for f in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(cs, f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the kernel's current sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None
    cur = kernel_source_hash(kernel)
    for ln in open(path):
        parts = ln.split()
        if len(parts) >= 4 and not ln.startswith("#") and parts[0] == kernel and parts[1] == workload:
            if parts[3] == cur:
                return float(parts[2])
    return None


def recorded_instr(kernel, workload):
    """FP64 instructions per cell update counted by ncu (profiles/fp64_instr.txt),
    if counted on the kernel's current sources (else None)."""
    return recorded_instr_state(kernel, workload)[0]


def recorded_instr_state(kernel, workload):
    """(count, state): state is "current", "stale" (counted on older sources)
    or "none" (never counted)."""
    path = os.path.join(ROOT, "profiles", "fp64_instr.txt")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None, "none"
    cur = kernel_source_hash(kernel)
    state = "none"
    for ln in open(path):
        parts = ln.split()
        if len(parts) >= 4 and not ln.startswith("#") and parts[0] == kernel and parts[1] == workload:
            if parts[3] == cur:
                return float(parts[2]), "current"
            state = "stale"
    return None, state


def variant_kernel(variant, ndim):
    """The kernel family a variant name runs (for the traffic record)."""
    if variant == "stream":
        return "stream3d" if ndim == 3 else "stream2d"
    return variant


def _measured_hbm_gbs(default=6681.8):
    """HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json beside this script
    when present (a STREAM-style copy measured on GB300), else `default`,
    the value that file held when this script was written."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError, TypeError):
        return default


HBM_GBS = _measured_hbm_gbs()


def roofline(name, cells, T, ms, launches, peak_tflops, kernel, Tb=1, bytes_per_cell=16,
             instr=None, flops=None, traffic_key=None):
    """The stated roofline: min(FP64 peak / F, HBM bandwidth * Tb / bytes per
    cell) in cell updates per second; `frac` = achieved FP64 flops / peak
    (the FP64 term binds for every workload here).  `traffic_key` names the
    DRAM-traffic record when it is not the workload name (plus "@tb<Tb>")."""
    F = FLOPS[name] if flops is None else flops
    achieved = F * cells * T / (ms * 1e-3) / 1e12
    per_launch = F * cells * T / max(launches, 1)
    instr_source = "given by the caller"
    if instr is None:
        # a Tb-fused kernel's count (halo recompute included) is keyed "<name>@tb<Tb>"
        counted, state = recorded_instr_state(kernel, f"{name}@tb{Tb}") if Tb > 1 else (None, "none")
        if counted is None:
            counted, state0 = recorded_instr_state(kernel, name)
            state = state0 if state == "none" else state
        instr = INSTR[name] if counted is None else counted
        instr_source = "ncu count, profiles/fp64_instr.txt" if counted is not None else \
            "table (kernel changed since the ncu count)" if state == "stale" else \
            "table (no ncu count recorded)"
    instr_rate = instr * cells * T / (ms * 1e-3)             # FP64 instructions per second
    fp64_ceiling = peak_tflops * 1e12 / F / 1e9
    hbm_ceiling = HBM_GBS * 1e9 * Tb / bytes_per_cell / 1e9
    rate = cells * T / (ms * 1e-3) / 1e9
    pipe_frac = instr_rate / (peak_tflops * 1e12 / 2)
    if fp64_ceiling <= hbm_ceiling:
        # the FP64 pipe binds; when the kernel issues fewer FP64 instructions
        # per cell than the K taps the metric's F credits (shared partial sums
        # of an equal-weight box), flops / peak overstates its efficiency and
        # `frac` is the executed-instruction fraction instead
        credited = (F + 1) / 2
        if instr < credited - 1e-9:
            out = {"bound": "alu", "achieved": round(instr_rate * 2 / 1e12, 4), "peak": round(peak_tflops, 4),
                   "unit": "TFLOP/s", "frac": round(pipe_frac, 4),
                   "frac_basis": f"executed FP64 instructions ({instr:g} per cell, x2 flop) / peak: the kernel "
                                 f"shares partial sums, so the metric's F = {F} flop/cell over-counts "
                                 f"its work (flops-credited fraction {achieved / peak_tflops:.3f})"}
        else:
            out = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak_tflops, 4),
                   "unit": "TFLOP/s", "frac": round(achieved / peak_tflops, 4),
                   "frac_basis": f"algorithmic flops (F = {F:g} per cell) / measured FP64 peak"}
    else:
        gbs = bytes_per_cell * cells * T / Tb / (ms * 1e-3) / 1e9
        out = {"bound": "hbm", "achieved": round(gbs, 2), "peak": round(HBM_GBS, 1), "unit": "GB/s",
               "frac": round(gbs / HBM_GBS, 4),
               "frac_basis": f"algorithmic bytes ({bytes_per_cell} per cell per Tb block) / measured HBM copy"}
    stated = rate / min(fp64_ceiling, hbm_ceiling)
    out.update({
            "fp64_ceiling_gstencil_per_s": round(fp64_ceiling, 3),
            "hbm_ceiling_gstencil_per_s": round(hbm_ceiling, 3),
            "frac_of_stated_roofline": round(min(stated, pipe_frac) if stated > 1.0 else stated, 4),
            "fp64_instr_per_cell": round(instr, 4),
            "fp64_instr_source": instr_source,
            "fp64_pipe_frac": round(pipe_frac, 4),
            "traffic": recorded_traffic(kernel, traffic_key or (name if Tb == 1 else f"{name}@tb{Tb}")),
            "algorithmic_flops_per_launch": per_launch,
            "algorithmic_bytes_per_launch": bytes_per_cell * cells * T / Tb / max(launches, 1),
            "peak_source": "FP64 DFMA microbenchmark measured in this run, best of 3 (x2 flop/FMA); "
                           f"nominal {NOMINAL_FP64_TFLOPS:.3f} TFLOP/s"})
    if stated > 1.0:
        out["stated_roofline_note"] = (f"rate / min(FP64 ceiling, HBM ceiling) = {stated:.3f}: above 1 because the "
                                       "kernel executes fewer FP64 instructions than F credits; "
                                       "frac_of_stated_roofline reports the executed-instruction fraction")
    return out


# ------------------------------------------------------------ our workloads

def headline(st, steps, warmup, world, stream):
    import torch
    shape, T = HEADLINE["shape"], HEADLINE["T"]
    u0 = synth.uniform(synth.SEED_HEAT3D, shape) + synth.sine_mode(shape, HEADLINE["sine"])
    grid = torch.from_numpy(u0).cuda()
    plan = st.Plan(shape, 1, synth.heat_weights(3, HEADLINE["alpha"]), st.PERIODIC)
    tb, variant = plan.get_tuning()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    # the clock sampler starts before the warm-ups (nvidia-smi's start-up
    # idles the GPU for a moment); only the timed region's samples count
    sampler = ClockSampler(uuid)
    sampler.start()
    for _ in range(warmup):
        plan.run(grid, T, stream=stream)
    torch.cuda.synchronize()
    barrier(world)
    sampler.mark()
    l0 = st.stencil_launch_count()
    ms = cuda_time(lambda: [plan.run(grid, T, stream=stream) for _ in range(steps)], stream)
    launches = st.stencil_launch_count() - l0
    clocks = sampler.stop()
    ms = barrier_max(world, ms)
    # properties the result keeps at any size (periodic, weights >= 0 summing to 1):
    # the mean is conserved and every value stays within the initial range
    m0 = float(np.mean(u0))
    checks = {"steps_applied": (warmup + steps) * T,
              "mean_drift_rel": abs(float(grid.mean()) - m0) / abs(m0),
              "within_initial_range": bool(float(grid.min()) >= float(u0.min()) and
                                           float(grid.max()) <= float(u0.max()))}
    # end to end through the host-buffer entry point (pinned memory): the
    # clock sampler first (the GPU idles while nvidia-smi starts, and a GPU
    # that has idled runs the next seconds slower), then two untimed calls
    # (the plan's staging buffer is allocated in the first) that bring it
    # back to its steady state, then `steps` timed calls, each copying the
    # grid in, sweeping T steps and copying the result out
    host = torch.from_numpy(u0).pin_memory()
    h2d = host.numel() * 8
    e2e_sampler = ClockSampler(uuid)
    e2e_sampler.start()
    for _ in range(2):
        plan.run_host(host, T, stream=stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_sampler.mark()
    t0 = time.perf_counter()
    e2e_calls = []
    for _ in range(steps):
        t1 = time.perf_counter()
        plan.run_host(host, T, stream=stream)
        e2e_calls.append(round((time.perf_counter() - t1) * 1e3, 2))
    e2e_ms = (time.perf_counter() - t0) * 1e3 / steps
    e2e_clocks = e2e_sampler.stop()
    e2e_ms = barrier_max(world, e2e_ms)
    # the copies alone, for the record: the same pinned buffer to and from
    # the device (CUDA events on the stream), GB/s each way
    copy_ms = {"h2d": cuda_time(lambda: grid.copy_(host, non_blocking=True), stream),
               "d2h": cuda_time(lambda: host.copy_(grid, non_blocking=True), stream)}
    copy_gbs = {k: round(h2d / (v * 1e-3) / 1e9, 1) for k, v in copy_ms.items()}
    plan.close()
    del grid
    torch.cuda.empty_cache()
    return dict(ms=ms / steps, launches=launches, clocks=clocks, e2e_ms=e2e_ms, e2e_clocks=e2e_clocks,
                h2d=h2d, d2h=h2d, copy_gbs=copy_gbs, e2e_calls=e2e_calls,
                Tb=tb, variant=st.stencil_variant_name(variant), u0=u0, checks=checks)


def time_plan(st, plan, grid, T, reps, stream, warm=1):
    for _ in range(warm):
        plan.run(grid, T, stream=stream)
    l0 = st.stencil_launch_count()
    ms = cuda_time(lambda: [plan.run(grid, T, stream=stream) for _ in range(reps)], stream)
    return ms / reps, (st.stencil_launch_count() - l0) // reps


def form_const(st, name, shape, radius, weights, boundary, T, u0, stream, peak, reps=2,
               tb_sweep=None, autotune_steps=0):
    """One constant-weight workload with the plan's own choice of kernel and Tb
    (or, with `autotune_steps`, the plan autotuner's choice, timed on a scratch
    copy first); `tb_sweep` ([(Tb, variant), ...]) also times each listed Tb
    (GStencil/s)."""
    import torch
    grid = torch.from_numpy(u0).cuda()
    plan = st.Plan(shape, radius, weights, boundary)
    if autotune_steps:
        scratch = grid.clone()
        plan.autotune(scratch, autotune_steps, stream=stream)
        del scratch
    ms, launches = time_plan(st, plan, grid, T, reps, stream)
    cells = int(np.prod(shape))
    tb, v = plan.get_tuning()
    tile = plan.get_tile()
    sweep = None
    if tb_sweep:
        sweep = {}
        fp64_ceiling = peak * 1e12 / FLOPS[name] / 1e9
        for tbs, vs in tb_sweep:
            plan.set_tuning(tbs, vs)
            ms_s, _ = time_plan(st, plan, grid, T, 1, stream)
            rate = cells * T / (ms_s * 1e-3) / 1e9
            ceiling = min(fp64_ceiling, HBM_GBS * tbs / 16)
            entry = {"gstencil_per_s": round(rate, 3), "frac_of_stated_roofline": round(rate / ceiling, 4)}
            instr = shared_sum_instr(name, st.stencil_variant_name(vs), tbs)
            if instr is not None and rate / ceiling > 1.0:
                # shared partial sums: F over-counts the work, report the executed fraction
                entry["frac_of_stated_roofline"] = round(rate * 1e9 * instr / (peak * 1e12 / 2), 4)
                entry["frac_basis"] = f"executed FP64 instructions ({instr:.3f} per cell) / peak"
            sweep[f"Tb={tbs} {st.stencil_variant_name(vs)}"] = entry
        plan.set_tuning(0, 0)
    plan.close()
    del grid
    torch.cuda.empty_cache()
    out = {"workload": f"{name} {'x'.join(map(str, shape))} T={T} "
                       f"{'periodic' if boundary else 'dirichlet0'}",
           "gstencil_per_s": round(cells * T / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 3),
           "Tb": tb, "variant": st.stencil_variant_name(v), "autotuned": bool(autotune_steps),
           "tile": list(tile) if tile[0] else None,
           "launches": launches,
           "roofline": roofline(name, cells, T, ms, launches, peak,
                                variant_kernel(st.stencil_variant_name(v), len(shape)), Tb=tb)}
    if sweep is not None:
        out["tb_sweep_gstencil_per_s"] = sweep
    return out


def shared_sum_instr(name, variant, Tb):
    """FP64 instructions per cell of the kernels that share partial sums (the
    equal-weight 2D 9-point box; None for every other workload): the streaming
    kernel's 4.25, and the temporal kernel's 6 per cell times its row segment's
    halo recompute ((TX + Tb - 1) / TX, TX = 254, 252, 248 for Tb = 2, 4, 8)."""
    if name != "box2d-9pt":
        return None
    if variant == "stream":
        return recorded_instr("stream2d", name) or INSTR[name]
    if variant == "temporal":
        tx = {2: 254, 4: 252, 8: 248}.get(Tb)
        return None if tx is None else 6.0 * (tx + Tb - 1) / tx
    return None


def form_forced(st, name, shape, radius, weights, boundary, T, u0, stream, peak, Tb, variant, reps=1,
                traffic_key=None):
    """One constant-weight workload on a forced (Tb, variant), with its roofline:
    FP64 instructions per cell include what the exchange kernel computes
    twice (the periodic z-halo, (Tb-1)/nz of the planes, and the margin rows
    of a plane cut into bands).  `u0`: the initial grid, or a seed for a
    uniform grid drawn on the device."""
    import torch
    if isinstance(u0, np.ndarray):
        grid = torch.from_numpy(u0).cuda()
    else:  # a seed: the grid is drawn on the device (large grids)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(int(u0))
        grid = torch.rand(shape, dtype=torch.float64, device="cuda", generator=gen)
    plan = st.Plan(shape, radius, weights, boundary)
    plan.set_tuning(Tb, variant)
    ms, launches = time_plan(st, plan, grid, T, reps, stream)
    assert plan.status() == 0
    vname = st.stencil_variant_name(variant)
    bands = plan.exchange_layout(Tb) if vname == "exchange" else None
    plan.close()
    del grid
    torch.cuda.empty_cache()
    cells = int(np.prod(shape))
    counted = recorded_instr(variant_kernel(vname, len(shape)), name)
    instr = INSTR[name] if counted is None else counted
    if vname == "exchange":
        if boundary == 1:
            instr *= 1 + (Tb - 1) / shape[0]  # the stage skew's extra planes
        instr *= bands[1] / shape[1]          # margin rows that two bands both compute
    out = {"workload": f"{name} {'x'.join(map(str, shape))} T={T} {'periodic' if boundary else 'dirichlet0'}",
           "gstencil_per_s": round(cells * T / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 3), "Tb": Tb,
           "variant": vname, "launches": launches,
           "roofline": roofline(name, cells, T, ms, launches, peak, variant_kernel(vname, len(shape)), Tb=Tb,
                                instr=instr, traffic_key=traffic_key)}
    if bands is not None:
        out["bands"] = {"count": bands[0], "rows_computed": bands[1], "rows": shape[1]}
    return out


# The paper's eight benchmark stencils at its own problem sizes (Table 1),
# each for a bounded number of steps (the rate per step does not depend on T).
# Weights: Eq. 3 heat weights for the Heat shapes, seeded random weights
# summing to 1 for the others; Dirichlet zero (Table 1 states no boundary).
TABLE1 = [
    ("Heat-1D", "heat1d-3pt", (10_000_000,), 1, "heat", 1000),
    ("Star-1D5P", "star1d-5pt", (10_000_000,), 2, "star", 1000),
    ("Heat-2D", "heat2d-5pt", (10_000, 10_000), 1, "heat", 100),
    ("Star-2D9P", "star2d-9pt", (10_000, 10_000), 2, "star", 50),
    ("Box-2D9P", "box2d-9pt", (10_000, 10_000), 1, "box", 50),
    ("Box-2D25P", "box2d-25pt", (10_000, 10_000), 2, "box", 20),
    ("Heat-3D", "heat3d-7pt", (1024, 1024, 1024), 1, "heat", 10),
    ("Box-3D27P", "box3d-27pt", (1024, 1024, 1024), 1, "box", 3),
]


def table1_weights(ndim, radius, kind, seed):
    if kind == "heat":
        return synth.heat_weights(ndim, 0.1 if ndim > 1 else 0.25)
    side = 2 * radius + 1
    v = synth.uniform(seed, (side,) * ndim)
    if kind == "star":
        c = (radius,) * ndim
        mask = np.zeros_like(v, dtype=bool)
        for d in range(ndim):
            idx = list(c)
            for o in range(side):
                idx[d] = o
                mask[tuple(idx)] = True
        v = np.where(mask, v, 0.0)
    return v / v.sum()


def radius2_weights():
    """The radius-2 2D workloads' weights (Star-2D9P, Box-2D25P): seeded
    uniform weights summing to 1, the star keeping the box's centre row and
    column."""
    v = synth.uniform(synth.SEED_BOX2D + 10, (5, 5))
    box25 = v / v.sum()
    star9 = np.zeros((5, 5))
    star9[2, :] = box25[2, :]
    star9[:, 2] = box25[:, 2]
    return star9 / star9.sum(), box25


def onedim_weights():
    """The 1D workloads' weights: Heat-1D (alpha = 0.25) and Star-1D5P
    (seeded, summing to 1)."""
    v5 = synth.uniform(synth.SEED_HEAT2D + 21, (5,))
    return np.array([0.25, 0.5, 0.25]), v5 / v5.sum()


def form_table1(st, stream, peak):
    """GStencil/s of each Table 1 stencil at Table 1's grid size.  The input
    is drawn on the device from a seeded generator (a 1024^3 grid is 8 GiB)."""
    import torch
    out = {}
    gen = torch.Generator(device="cuda")
    for i, (label, name, shape, radius, kind, T) in enumerate(TABLE1):
        gen.manual_seed(synth.SEED_HEAT3D + 100 + i)
        grid = torch.rand(shape, dtype=torch.float64, device="cuda", generator=gen)
        w = table1_weights(len(shape), radius, kind, synth.SEED_HEAT3D + 200 + i)
        plan = st.Plan(shape, radius, w, st.DIRICHLET_ZERO)
        ms, launches = time_plan(st, plan, grid, T, 1, stream)
        tb, v = plan.get_tuning()
        cells = int(np.prod(shape))
        # the shared-partial-sum count of INSTR holds only for equal box weights
        instr = 9 if name == "box2d-9pt" and not np.all(w == w.flat[0]) else None
        r = roofline(name, cells, T, ms, max(launches, 1), peak,
                     variant_kernel(st.stencil_variant_name(v), len(shape)), Tb=tb, instr=instr)
        out[label] = {"shape": list(shape), "T": T, "variant": st.stencil_variant_name(v), "Tb": tb,
                      "gstencil_per_s": round(cells * T / (ms * 1e-3) / 1e9, 3),
                      "frac": r["frac"], "fp64_pipe_frac": r["fp64_pipe_frac"]}
        plan.close()
        del grid
        torch.cuda.empty_cache()
    return out


def form_batched(st, stream, peak, rank=0, world=1):
    """The 96-grid batch; with N ranks each advances its own shard (greedy
    packing on cells x T) and the rate is all updates / the slowest rank."""
    import torch
    from paper_2303_08365_gb300 import shard
    all_items = synth.batch_items(synth.SEED_BATCH)
    mine = shard.rank_items(all_items, rank, world)
    items = [all_items[i] for i in mine]
    total_updates = sum(ny * nx * T for ny, nx, _, T in all_items)
    grids0 = [synth.uniform(synth.SEED_BATCH + 1000 + i, all_items[i][:2]) for i in mine]
    dev = [torch.from_numpy(g).cuda() for g in grids0]
    alphas = [a for _, _, a, _ in items]
    steps = [T for *_, T in items]
    updates = sum(ny * nx * T for ny, nx, _, T in items)
    b = st.Batch(dev, alphas, steps)
    # the batch autotuner picks the kernel configuration (on scratch copies)
    tuned_rate = b.autotune(probe_steps=50, stream=stream)
    tb, cpt, per_sm = b.get_tuning()
    b.run(stream)
    assert b.status() == 0
    l0 = st.stencil_launch_count()
    reps = 3
    ms = cuda_time(lambda: [b.run(stream) for _ in range(reps)], stream) / reps
    launches = (st.stencil_launch_count() - l0) // reps
    assert b.status() == 0
    b.close()
    ms = shard.max_over_ranks(ms)
    updates = total_updates
    # the plain single-grid sweep over the same grids, one after another
    plans = [st.Plan((ny, nx), 1, synth.heat_weights(2, a), st.DIRICHLET_ZERO) for ny, nx, a, _ in items]

    def plain():
        for p, d, T in zip(plans, dev, steps):
            p.run(d, T, stream=stream)
    plain()
    ms_plain = shard.max_over_ranks(cuda_time(plain, stream))
    for p in plans:
        p.close()
    del dev
    torch.cuda.empty_cache()
    rate = updates / (ms * 1e-3) / 1e9
    return {"workload": f"batched 96 x heat2d-5pt, sides log-uniform [128,4096], T in [50,500], "
                        f"{updates:.3e} updates" + (f", sharded over {world} ranks" if world > 1 else ""),
            "gstencil_per_s": round(rate, 3), "ms": round(ms, 3), "launches": launches,
            "autotuned": {"Tb": tb, "cells_per_thread": cpt, "blocks_per_sm": per_sm,
                          "probe_gstencil_per_s": round(tuned_rate, 3)},
            "plain_sweep_ms": round(ms_plain, 3),
            "plain_sweep_gstencil_per_s": round(updates / (ms_plain * 1e-3) / 1e9, 3),
            "speedup_vs_plain": round(ms_plain / ms, 3),
            "roofline": roofline("heat2d-5pt", updates, 1, ms, max(launches, 1), peak, "batched")}


def form_adjoint(st, stream, peak):
    import torch
    shape, T, ck = (256, 256, 256), 1000, 32
    seed = synth.SEED_ADJOINT
    u0 = torch.from_numpy(synth.uniform(seed, shape)).cuda()
    kappa_h = synth.lognormal(seed + 1, shape, 0.5)
    kappa = torch.from_numpy(kappa_h).cuda()
    target = torch.from_numpy(synth.normal(seed + 2, shape)).cuda()
    dt = 0.1 / float(kappa_h.max())
    plan = st.Plan.varcoef(shape, st.PERIODIC)
    cells = int(np.prod(shape))
    # FP64 instructions per cell-step: forward 7, transposed step 7 + 3 faces x 3, and the
    # recompute of every segment but the last (the forward sweep keeps that one's states)
    nseg = -(-T // ck)
    recomputed = (nseg - 1) * (ck - 1)
    fwd = recorded_instr("varcoef", "varcoef-7pt") or 7.0     # ncu counts when current
    adj = recorded_instr("adjoint", "adjoint-step") or 16.0
    instr = fwd + fwd * recomputed / T + adj
    plan.adjoint(u0, kappa, dt, target, T, ckpt_every=ck, stream=stream)  # warm-up
    l0 = st.stencil_launch_count()
    ms = cuda_time(lambda: plan.adjoint(u0, kappa, dt, target, T, ckpt_every=ck, stream=stream), stream)
    launches = st.stencil_launch_count() - l0
    grid = u0.clone()
    plan.run(grid, T, kappa, dt, stream=stream)
    ms_fwd = cuda_time(lambda: plan.run(grid, T, kappa, dt, stream=stream), stream)
    plan.close()
    # the same gradients with every forward state kept (ckpt_every = 1: no
    # recompute; T + 10 grids of scratch, 126 GiB here) when HBM holds it
    store_all = None
    need = (T + 10) * cells * 8
    if torch.cuda.mem_get_info()[0] > 1.1 * need:
        plan = st.Plan.varcoef(shape, st.PERIODIC)
        plan.adjoint(u0, kappa, dt, target, T, ckpt_every=1, stream=stream)  # warm-up
        ms_all = cuda_time(lambda: plan.adjoint(u0, kappa, dt, target, T, ckpt_every=1,
                                                stream=stream), stream)
        plan.close()
        store_all = {"ms": round(ms_all, 3),
                     "gstencil_per_s": round(cells * T / (ms_all * 1e-3) / 1e9, 3),
                     "ratio_vs_forward": round(ms_all / ms_fwd, 3),
                     "scratch_gib": round(need / 2**30, 1),
                     "roofline": roofline("adjoint-7pt", cells, T, ms_all, 2 * T, peak, "adjoint",
                                          bytes_per_cell=48 + 104, instr=fwd + adj,
                                          traffic_key="adjoint-step")}
    del u0, kappa, target, grid
    torch.cuda.empty_cache()
    return {"workload": "adjoint varcoef-7pt 256^3 T=1000 periodic, checkpoints every 32",
            "ms": round(ms, 3), "gstencil_per_s": round(cells * T / (ms * 1e-3) / 1e9, 3),
            "forward_ms": round(ms_fwd, 3),
            "forward_gstencil_per_s": round(cells * T / (ms_fwd * 1e-3) / 1e9, 3),
            "ratio_vs_forward": round(ms / ms_fwd, 3), "launches": launches,
            # bytes per cell-step: forward and recompute read u, c0, cx, cy, cz and write u'
            # (48 each); the transposed step reads lambda, u, c0..cz, reads and writes the
            # three face-gradient accumulators and writes lambda' (104; periodic grids have no
            # ghost faces, so the fourth accumulator is untouched)
            # F per cell-step: forward 13, transposed step 13 + 3 faces x (2 differences, a
            # product, a sum) = 25, and the forward recompute that checkpointing every 32 steps
            # makes part of the method (13 per recomputed step); frac_without_recompute_credit
            # counts only the 38 of a run that stores every state
            # traffic: DRAM bytes of one k_adjoint launch (the dominant kernel), against
            # its algorithmic 104 B per cell
            "roofline": dict(roofline("adjoint-7pt", cells, T, ms, launches, peak, "adjoint",
                                      bytes_per_cell=48 + 48 * recomputed / T + 104, instr=instr,
                                      flops=FLOPS["adjoint-7pt"] + 13 * recomputed / T,
                                      traffic_key="adjoint-step"),
                             frac_without_recompute_credit=round(
                                 FLOPS["adjoint-7pt"] * cells * T / (ms * 1e-3) / 1e12 / peak, 4),
                             traffic_kernel="k_adjoint, per launch",
                             traffic_algorithmic_bytes=104 * cells),
            "forward_roofline": roofline("varcoef-7pt", cells, T, ms_fwd, T, peak, "varcoef",
                                         bytes_per_cell=48),
            "every_state_kept": store_all}


# ------------------------------------------------------------ CPU baseline

def cpu_baseline(u0, budget_s=12.0, gpu_run=None):
    """The oracle as it stands, on all host cores, on a bounded number of
    steps of the headline grid; GStencil/s.  With `gpu_run(u0, steps)` (the
    library's sweep of the same grid) the oracle's sample is also compared
    with the GPU result, element by element over the whole 512^3 grid."""
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    w = synth.heat_weights(3, HEADLINE["alpha"])
    t0 = time.perf_counter()
    oracle.run(u0, w, 1, 1, 1, nthreads=cores)
    one = time.perf_counter() - t0
    steps = max(1, min(200, int(budget_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    ref = oracle.run(u0, w, 1, 1, steps, nthreads=cores)
    el = time.perf_counter() - t0
    cells = u0.size
    parity = None
    if gpu_run is not None:
        got = gpu_run(u0, steps)
        parity = {"steps": steps, "cells": int(cells),
                  "normwise_rel_err": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
                  "bar": 1e-12}
    del ref
    # one core: the 2D 5-point 256^2 case in full, and the 27-point box with the 384^3
    # case's weights and boundary on a 128^3 grid for 2 steps (a bounded sample)
    single = []
    for label, shp, w, bnd, T, u in (
            ("heat2d-5pt 256^2 T=100 dirichlet0 (all steps)", (256, 256),
             synth.heat_weights(2, 0.1), 0, 100, synth.uniform(synth.SEED_HEAT2D, (256, 256))),
            ("box3d-27pt dirichlet0, 128^3 sample, 2 steps", (128, 128, 128),
             synth.box_weights(3, seed=synth.SEED_BOX3D), 0, 2,
             synth.normal(synth.SEED_BOX3D, (128, 128, 128)))):
        t1 = time.perf_counter()
        oracle.run(u, w, 1, bnd, T, nthreads=1)
        e1 = time.perf_counter() - t1
        single.append({"workload": label, "value": round(int(np.prod(shp)) * T / e1 / 1e9, 5),
                       "unit": "GStencil/s", "seconds": round(e1, 3)})
    return {"value": round(cells * steps / el / 1e9, 5), "unit": "GStencil/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{HEADLINE['name']} 512^3 periodic, {steps} of the 1000 steps "
                      f"({el:.1f} s), plain C loop nest, OpenMP over rows",
            "single_core": single, "parity_vs_gpu": parity}


# ------------------------------------------------------------------ main

def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.lib()
    shape = HEADLINE["shape"]
    u0 = synth.uniform(synth.SEED_HEAT3D, shape) + synth.sine_mode(shape, HEADLINE["sine"])
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    w = synth.heat_weights(3, HEADLINE["alpha"])
    sample_steps = 2
    for _ in range(args.warmup):
        oracle.run(u0, w, 1, 1, 1, nthreads=cores)
    times = []
    u = u0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u = oracle.run(u, w, 1, 1, sample_steps, nthreads=cores)
        times.append(time.perf_counter() - t0)
    el = sum(times)
    cells = u0.size
    value = cells * sample_steps * args.steps / el / 1e9
    line = {"metric": METRIC, "value": round(value, 5), "unit": "GStencil/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "heat3d-7pt 512^3 periodic (each step: 2 of the 1000 time steps)",
                       "shape": list(HEADLINE["shape"]), "T": HEADLINE["T"], "grids": 1,
                       "parallelism": "none (host cores)",
                       "l2_flush": "input 1 GiB > L2"},
            "cpu_baseline": {"value": round(value, 5), "unit": "GStencil/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{sample_steps} time steps of the 512^3 grid per step"},
            "e2e": {"value": round(value, 5), "unit": "GStencil/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


THERMAL = dict(mu=0.23, n=9600, T_full=3_800_000,
               table3={"naive_s": 124448.5, "tetris_cpu_s": 27709.1, "tetris_gpu_s": 5597.4,
                       "tetris_s": 4270.9, "tetris_gpu_gst": 63.3, "tetris_gst": 82.9,
                       "hardware": "AMD EPYC 7V13 (24 cores) + NVIDIA A100-80GB, FP64"})


def thermal_case(st, n, T, stream, fp32=True, peak=None):
    """The paper's copper-plate case study (Sec. 5.5) on an n x n grid: heat
    stencil with mu = 0.23 (Eq. 3 weights 0.08 / 0.23), Dirichlet 0 at the
    edges, Gaussian initial field peaked at 100 degrees.  FP64 production
    sweep timed; optionally the FP32 twin for the Table 4 deviation counts."""
    import torch
    w = synth.heat_weights(2, THERMAL["mu"])
    u0 = synth.gaussian_plate((n, n))
    g = torch.from_numpy(u0).cuda()
    plan = st.Plan((n, n), 1, w, st.DIRICHLET_ZERO)
    plan.run(g, min(T, 10), stream=stream)          # warm-up (and plan set-up)
    g.copy_(torch.from_numpy(u0))
    ms = cuda_time(lambda: plan.run(g, T, stream=stream), stream)
    tb, v = plan.get_tuning()
    out = {"workload": f"thermal plate {n}x{n}, mu=0.23, Dirichlet 0, Gaussian 100 C (sigma "
                       f"{1376.0 * n / 9600:.0f} cells), T={T}",
           "variant": st.stencil_variant_name(v), "Tb": tb,
           "gstencil_per_s": round(n * n * T / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 3),
           "centre_C": round(float(g[n // 2, n // 2]), 4)}
    rate = n * n * T / (ms * 1e-3)
    if peak:
        out["roofline"] = roofline("heat2d-5pt", n * n, T, ms, T, peak,
                                   variant_kernel(st.stencil_variant_name(v), 2), Tb=tb,
                                   traffic_key=f"heat2d-5pt-{n}sq" if tb == 1 else None)
    if n == THERMAL["n"]:
        full = THERMAL["n"] ** 2 * THERMAL["T_full"] / rate
        out["extrapolated_full_run_s"] = round(full, 1)
        out["paper_table3_context"] = THERMAL["table3"]
    if fp32:
        g32 = torch.from_numpy(u0.astype(np.float32)).cuda()
        work = torch.empty_like(g32)
        st.stencil_run_f32(plan.handle, g32, work, T)
        torch.cuda.synchronize()
        d = (g32.double() - g).abs()
        rel = d / g.abs().clamp_min(1e-300)
        total = d.numel()
        out["fp32_vs_fp64_percent_of_cells"] = {
            "abs>0.1C": round(100.0 * float((d > 0.1).sum()) / total, 3),
            "abs>0.5C": round(100.0 * float((d > 0.5).sum()) / total, 3),
            "abs>1.0C": round(100.0 * float((d > 1.0).sum()) / total, 3),
            "rel>1%": round(100.0 * float((rel > 0.01).sum()) / total, 3),
            "rel>3%": round(100.0 * float((rel > 0.03).sum()) / total, 3),
            "rel>5%": round(100.0 * float((rel > 0.05).sum()) / total, 3),
            "max_abs_C": float(d.max())}
        del g32, work
    plan.close()
    del g
    torch.cuda.empty_cache()
    return out


def run_case(args):
    """One workload at a chosen size for profiling (not the benchmark line):
    W warm-up runs and `steps` timed runs of T time steps each."""
    import torch
    import paper_2303_08365_gb300 as st
    st.lib()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = args.size
    name = args.case
    radius = 2 if name in ("star2d9", "box2d25", "star1d5") else 1
    if name in ("heat3d", "box3d"):
        shape = (args.nz or n, n, n)
        w = synth.heat_weights(3, 0.1) if name == "heat3d" else synth.box_weights(3, seed=synth.SEED_BOX3D)
        bnd = 1 if name == "heat3d" else 0
    elif name in ("heat2d", "box2d"):
        shape = (n, n)
        w = synth.heat_weights(2, 0.1) if name == "heat2d" else synth.box_weights(2, 1.0 / 9.0)
        bnd = 0 if name == "heat2d" else 1
    elif name in ("star2d9", "box2d25"):
        # the radius-2 workloads of the benchmark line (periodic)
        shape = (n, n)
        w = radius2_weights()[0 if name == "star2d9" else 1]
        bnd = 1
    elif name in ("heat1d", "star1d5"):
        # the 1D workloads (Heat-1D Dirichlet, Star-1D5P periodic), --size cells
        shape = (n,)
        w = onedim_weights()[0 if name == "heat1d" else 1]
        bnd = 0 if name == "heat1d" else 1
    elif name in ("varcoef", "adjoint"):
        shape = (n, n, n)
    elif name == "thermal":
        print(json.dumps(thermal_case(st, n, args.T, stream)))
        return 0
    elif name == "batched":
        # --size 0: the benchmark line's 96-grid workload with the kernel
        # configuration --Tb / --cpt / --per-sm (the batch autotuner's pick);
        # else a reduced batch of its kind: sides log-uniform in [64, n]
        if n == 0:
            items = synth.batch_items(synth.SEED_BATCH)
        else:
            items = synth.batch_items(synth.SEED_BATCH, count=24, side_lo=64, side_hi=n, t_lo=args.T,
                                      t_hi=args.T)
        dev = [torch.from_numpy(synth.uniform(synth.SEED_BATCH + 1000 + i, (ny, nx))).cuda()
               for i, (ny, nx, _, _) in enumerate(items)]
        b = st.Batch(dev, [a for _, _, a, _ in items], [T for *_, T in items])
        if n == 0:
            b.set_tuning(args.Tb or 1, args.cpt, args.per_sm)
        for _ in range(args.warmup):
            b.run(stream)
        ms = cuda_time(lambda: [b.run(stream) for _ in range(args.steps)], stream) / args.steps
        assert b.status() == 0
        upd = sum(ny * nx * T for ny, nx, _, T in items)
        print(json.dumps({"case": name, "items": len(items), "updates": upd, "ms": round(ms, 4),
                          "gstencil_per_s": round(upd / (ms * 1e-3) / 1e9, 3)}))
        return 0
    else:
        raise SystemExit(f"unknown case {name}")
    grid = torch.from_numpy(synth.uniform(synth.SEED_HEAT3D, shape)).cuda()
    if name in ("varcoef", "adjoint"):
        kappa = torch.from_numpy(synth.lognormal(synth.SEED_ADJOINT + 1, shape)).cuda()
        dt = 0.1 / float(kappa.max())
        plan = st.Plan.varcoef(shape, st.PERIODIC)
        if name == "varcoef":
            fn = lambda: plan.run(grid, args.T, kappa, dt, stream=stream)
        else:
            target = torch.from_numpy(synth.normal(synth.SEED_ADJOINT + 2, shape)).cuda()
            fn = lambda: plan.adjoint(grid, kappa, dt, target, args.T, ckpt_every=args.ckpt,
                                      stream=stream)
    else:
        plan = st.Plan(shape, radius, w, bnd)
        if args.variant:
            plan.set_tuning(args.Tb or 1, args.variant)
        fn = lambda: plan.run(grid, args.T, stream=stream)
    for _ in range(args.warmup):
        fn()
    ms = cuda_time(lambda: [fn() for _ in range(args.steps)], stream) / args.steps
    cells = int(np.prod(shape))
    print(json.dumps({"case": name, "shape": shape, "T": args.T, "tuning": plan.get_tuning(),
                      "ms": round(ms, 4), "gstencil_per_s": round(cells * args.T / (ms * 1e-3) / 1e9, 3)}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="all", help="all | none | comma list of "
                    "box2d,box3d,heat2d,batched,adjoint,radius2,onedim,thermal,heat3d_tb,temporal,table1")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default=None,
                    help="profiling mode: heat3d | box3d | heat2d | box2d | star2d9 | box2d25 | heat1d | "
                         "star1d5 | varcoef | adjoint | batched | thermal (the case study with the FP32 "
                         "deviation counts)")
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--nz", type=int, default=0, help="3D cases: slowest-axis length (0: --size)")
    ap.add_argument("--T", type=int, default=4)
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--Tb", type=int, default=0)
    ap.add_argument("--cpt", type=int, default=0, help="batched case: cells per thread (0 = default)")
    ap.add_argument("--per-sm", type=int, default=0, help="batched case: blocks per SM (0 = default)")
    ap.add_argument("--ckpt", type=int, default=0, help="adjoint case: checkpoint interval "
                    "(0 = about sqrt(T), 1 = keep every state)")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2303_08365_gb300 as st
    st.lib()
    world, rank = dist_setup(args.gpus)
    stream = torch.cuda.current_stream()
    # the FP64 peak: best of three ~0.3 s measurements (a single one varies by ~1%)
    peak_dfma = max(st.stencil_fp64_peak(300.0) for _ in range(3))
    peak_tflops = 2 * peak_dfma / 1e12

    h = headline(st, args.steps, args.warmup, world, stream)
    shape, T = HEADLINE["shape"], HEADLINE["T"]
    cells = int(np.prod(shape))
    per_rank = cells * T / (h["ms"] * 1e-3) / 1e9
    value = per_rank * world
    e2e_value = cells * T / (h["e2e_ms"] * 1e-3) / 1e9 * world
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "GStencil/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(h["ms"], 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "heat3d-7pt 512^3 T=1000 periodic, u0 = U[0,1) + sin mode (3,5,7)",
                   "shape": list(HEADLINE["shape"]), "T": T, "grids": world,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "Tb": h["Tb"], "variant": h["variant"],
                   "tile": {"stream": "64 x 32 cells of (x, y), streamed along z, 4-plane TMA ring",
                            "temporal": "64 x 32 (Tb 2), 32 x 32 (Tb 4) or 16 x 16 (Tb 8) cells of (x, y) "
                                        "plus a Tb halo, streamed along z",
                            "exchange": "64 columns x 26-27 rows of (x, y) per co-resident CTA, streamed "
                                        "along z, levels handed over through an L2 ring",
                            "direct": "one cell per thread, 32 x 8 threads"}.get(h["variant"], h["variant"]),
                   "l2_flush": "none needed: each launch streams 2 GiB > 129 MB L2"},
        "roofline": roofline("heat3d-7pt", cells, T, h["ms"], h["launches"] // args.steps,
                             peak_tflops, variant_kernel(h["variant"], 3), Tb=h["Tb"]),
        "fp64_peak_tflops_measured": round(peak_tflops, 4),
        "e2e": {"value": round(e2e_value, 4), "unit": "GStencil/s",
                "h2d_bytes_per_step": h["h2d"], "d2h_bytes_per_step": h["d2h"],
                "copy_gbs_pinned": h["copy_gbs"], "ms_per_call": h["e2e_calls"],
                "clocks": h["e2e_clocks"]},
        "gpu_launches": int(h["launches"]),
        "clocks": h["clocks"],
        "result_checks": h["checks"],
    }
    if rank == 0 and not args.no_cpu_baseline:
        def gpu_run(u, steps):
            g = torch.from_numpy(u).cuda()
            p = st.Plan(u.shape, 1, synth.heat_weights(3, HEADLINE["alpha"]), st.PERIODIC)
            p.run(g, steps, stream=stream)
            out = g.cpu().numpy()
            p.close()
            return out
        line["cpu_baseline"] = cpu_baseline(h["u0"], gpu_run=gpu_run)
    forms = {}
    want = set(["box2d", "box3d", "heat2d", "batched", "adjoint", "radius2", "onedim", "thermal",
                "heat3d_tb", "temporal", "table1"]) \
        if args.forms == "all" else \
        set() if args.forms == "none" else set(args.forms.split(","))
    if "batched" in want:
        forms["batched"] = form_batched(st, stream, peak_tflops, rank, world)
    if rank == 0:
        if "heat2d" in want:
            shp = (256, 256)
            forms["heat2d"] = form_const(st, "heat2d-5pt", shp, 1, synth.heat_weights(2, 0.1), 0, 100,
                                         synth.uniform(synth.SEED_HEAT2D, shp), stream, peak_tflops,
                                         reps=20)
        if "heat3d_tb" in want:
            # the headline grid at every Tb the 3D kernels offer, 100 of its 1000 steps each
            shp = HEADLINE["shape"]
            u0 = h["u0"]
            r = form_const(st, "heat3d-7pt", shp, 1, synth.heat_weights(3, HEADLINE["alpha"]), 1, 100, u0,
                           stream, peak_tflops, reps=1,
                           tb_sweep=[(1, st.VARIANT_STREAM), (2, st.VARIANT_TEMPORAL),
                                     (4, st.VARIANT_TEMPORAL), (8, st.VARIANT_TEMPORAL),
                                     (2, st.VARIANT_EXCHANGE), (4, st.VARIANT_EXCHANGE),
                                     (8, st.VARIANT_EXCHANGE)])
            forms["heat3d_tb_sweep"] = {"workload": r["workload"],
                                        "tb_sweep_gstencil_per_s": r["tb_sweep_gstencil_per_s"]}
        if "temporal" in want:
            # the temporal-blocked sweep on the headline workload at full T: the
            # exchange kernel (no recomputed halo), Tb = 4 and 8
            for tb in (4, 8):
                forms[f"temporal_tb{tb}"] = form_forced(st, "heat3d-7pt", HEADLINE["shape"], 1,
                                                        synth.heat_weights(3, HEADLINE["alpha"]), 1, HEADLINE["T"],
                                                        h["u0"], stream, peak_tflops, tb, st.VARIANT_EXCHANGE)
        if "temporal" in want:
            # Table 1's Heat-3D grid size (1024^3; periodic, as the headline):
            # 1024^2 planes are cut into four bands of rows per Tb-block; 40 steps
            shp = (1024, 1024, 1024)
            for tb in (4, 8):
                forms[f"temporal_1024_tb{tb}"] = form_forced(
                    st, "heat3d-7pt", shp, 1, synth.heat_weights(3, HEADLINE["alpha"]), 1, 40,
                    synth.SEED_HEAT3D + 300, stream, peak_tflops, tb, st.VARIANT_EXCHANGE,
                    traffic_key=f"heat3d-7pt-1024cube@tb{tb}")
        if "box2d" in want:
            shp = (16384, 16384)
            forms["box2d"] = form_const(st, "box2d-9pt", shp, 1, synth.box_weights(2, 1.0 / 9.0), 1, 1000,
                                        synth.uniform(synth.SEED_BOX2D, shp), stream, peak_tflops,
                                        tb_sweep=[(1, st.VARIANT_STREAM), (2, st.VARIANT_TEMPORAL),
                                                  (4, st.VARIANT_TEMPORAL), (8, st.VARIANT_TEMPORAL)])
        if "radius2" in want:
            # Table 1's radius-2 shapes (Star-2D9P, Box-2D25P), seeded random weights summing to 1
            shp = (8192, 8192)
            star9, box25 = radius2_weights()
            u0 = synth.uniform(synth.SEED_BOX2D + 11, shp)
            forms["star2d9p"] = form_const(st, "star2d-9pt", shp, 2, star9, 1, 100, u0, stream, peak_tflops)
            forms["box2d25p"] = form_const(st, "box2d-25pt", shp, 2, box25, 1, 100, u0, stream, peak_tflops)
        if "thermal" in want:
            forms["thermal"] = thermal_case(st, THERMAL["n"], 1000, stream, fp32=False, peak=peak_tflops)
        if "table1" in want:
            forms["table1"] = form_table1(st, stream, peak_tflops)
        if "onedim" in want:
            # Table 1's 1D shapes: Heat-1D (alpha = 0.25) and Star-1D5P, 10^7 cells
            n1 = 10_000_000
            u1 = synth.uniform(synth.SEED_HEAT2D + 20, (n1,))
            heat3, star5 = onedim_weights()
            forms["heat1d"] = form_const(st, "heat1d-3pt", (n1,), 1, heat3, 0, 1000, u1, stream, peak_tflops)
            forms["star1d5p"] = form_const(st, "star1d-5pt", (n1,), 2, star5, 1, 1000, u1, stream,
                                           peak_tflops)
        if "box3d" in want:
            shp = (384, 384, 384)
            # Tb picked by the plan autotuner among {1, 2, 4, 8} (and the Tb = 1
            # kernels), then every Tb timed for the record
            forms["box3d"] = form_const(st, "box3d-27pt", shp, 1, synth.box_weights(3, seed=synth.SEED_BOX3D),
                                        0, 500, synth.normal(synth.SEED_BOX3D, shp), stream, peak_tflops,
                                        tb_sweep=[(1, st.VARIANT_STREAM), (2, st.VARIANT_TEMPORAL),
                                                  (4, st.VARIANT_TEMPORAL), (8, st.VARIANT_TEMPORAL),
                                                  (2, st.VARIANT_EXCHANGE), (4, st.VARIANT_EXCHANGE),
                                                  (8, st.VARIANT_EXCHANGE)],
                                        autotune_steps=8)
        if "adjoint" in want:
            forms["adjoint"] = form_adjoint(st, stream, peak_tflops)
        line["forms"] = forms
        print(json.dumps(line))
    barrier(world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
