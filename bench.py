"""Benchmark of the GB300 fire-model step: fire-mesh cell-steps per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

A step is one fire_step (Sect. 5 items 1-6 of the paper) over the whole
fire mesh.  The default workload is the large forward case: an 820x820
atmospheric mesh refined 10x to 8200x8200 fire nodes, seeded wind / hills /
13-class fuel map, 50 point ignitions, FP32 state with FP64 ignition time and
heat reduction, 2000 steps of 0.5 s (the state, 2.2 GB, is larger than L2, so
no flush is needed between steps).  Under torchrun every rank runs its own
replica of the workload (the problems are independent: weak scaling, no
collective on the data path); the time is the max over ranks.

One JSON line is printed by rank 0.  Besides the device-timed value it carries
the end-to-end value through fire_step_host (host wind in, host heat out),
the roofline of the fused step kernel against the measured HBM copy
bandwidth, the FP64 GPU path on the same mesh, and the FP64 CPU oracle timed
on a bounded sample of the same recipe on the host cores.

--impl reference times the oracle itself (on all host cores, through its
OpenMP loops over rows) on a bounded sample of the same workload, one oracle
step per bench step.
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fire-mesh cell-steps/s"
UNIT = "cell-steps/s"
# algorithmic bytes per cell-step of the one-pass FP32 step: psi r/w 4+4,
# F r/w 4+4, ignition time read 8, fuel class 1, terrain gradient 8
BYTES_PER_CELL_STEP = {"fp32": 33, "fp64": 57}
KERNEL_SOURCES = ["paper_1102_1343_gb300/csrc/march_kernel.cuh",
                  "paper_1102_1343_gb300/csrc/pair_math.cuh",
                  "paper_1102_1343_gb300/csrc/warp_kernel.cuh",
                  "paper_1102_1343_gb300/csrc/fire_device.cuh",
                  "paper_1102_1343_gb300/csrc/fire_internal.h",
                  "paper_1102_1343_gb300/csrc/step_f32.cu",
                  "paper_1102_1343_gb300/csrc/warp4_kernel.cuh",
                  "paper_1102_1343_gb300/csrc/step_warp4.cu"]
PROFILE_SUMMARY = "profiles/fire_warp_f32_points8200.md"
KERNEL_VARIANTS = ["tile", "march", "warp", "warp4", "warp_dense"]  # FIRE_KERNEL_* order
KERNEL_NAMES = ["k_fire_step", "k_fire_march", "k_fire_warp", "k_fire_warp4", "k_fire_warp"]


def kernel_hash() -> str:
    """Hash of the step kernel's sources without comments and blank space, so
    that a profile summary stays valid across comment-only edits."""
    import re
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(path=None):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    path = path or os.path.join(ROOT, PROFILE_SUMMARY)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, _, v = line.strip()[2:].partition(":")
            vals[k.strip()] = v.strip()
    if (vals.get("kernel_source_hash") or "-").split()[0] != kernel_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"].split()[0])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax),
                       reasons=sorted(reasons), samples=len(sm))
        return out


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def make_workload(name: str):
    from paper_1102_1343_gb300 import synth
    if name == "points8200":
        return synth.points_fire_8200()
    if name == "line2000":
        return synth.line_fire_2000()
    if name == "circle100":
        return synth.plain_circle()
    if name == "burning8200":
        return synth.burning_fire_8200()
    if name == "points4000":
        # a smaller case of the same recipe (4000x4000 nodes, state 0.53 GB > L2) for
        # profiler captures that the 8200x8200 mesh is too large for
        return synth.random_landscape(400, 400, seed=synth.BASE_SEED, ignition="points",
                                      n_points=12, edge_margin=500.0, steps=2000,
                                      name="points-fire-4000x4000")
    if name == "burning4000":
        # the burning recipe on the same smaller mesh, for profiler captures
        # of the quadrature-heavy regime
        return synth.random_landscape(400, 400, seed=synth.BASE_SEED, ignition="points",
                                      n_points=12, edge_margin=3500.0, ignition_radius=3000.0,
                                      steps=2000, name="burning-fire-4000x4000")
    raise ValueError(name)


def oracle_sample(name: str, budget_cell_steps: float):
    """A bounded sample of the same recipe for the CPU oracle: a smaller
    square mesh with the same generators, sized to the cell-step budget."""
    from paper_1102_1343_gb300 import synth
    if name == "circle100":
        return synth.plain_circle(), 1
    side_atm = int(max(10, min(82, math.sqrt(budget_cell_steps) / 10)))
    ign = "points" if name.startswith("points") else "line"
    w = synth.random_landscape(side_atm, side_atm, seed=synth.BASE_SEED, ignition=ign,
                               n_points=max(1, round(50 * (side_atm / 820) ** 2)),
                               edge_margin=2000.0 * side_atm / 820, steps=1)
    return w, side_atm


def host_cpu_model() -> str:
    """The host CPU model (lscpu's model name, else /proc/cpuinfo, else the
    machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine() or "unknown"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(name: str, seconds: float = 12.0, max_steps: int | None = None,
                threads: int = 1):
    """Oracle cell-steps/s on a sample of the workload with the given number
    of host threads (its OpenMP loops over rows; 1 = the plain serial run)."""
    import oracle
    w, side = oracle_sample(name, budget_cell_steps=0.67e6)
    used = oracle.set_threads(threads)
    try:
        o = oracle.OracleFire.from_workload(w)
        o.step(w.u, w.v, w.dt)  # first-touch
        n = 0
        t0 = time.perf_counter()
        while True:
            o.step(w.u, w.v, w.dt)
            n += 1
            el = time.perf_counter() - t0
            if el >= seconds or (max_steps and n >= max_steps):
                break
    finally:
        oracle.set_threads(1)
    cells = w.nx * w.ny
    how = "single thread" if used == 1 else f"{used} threads (OpenMP over rows)"
    return dict(value=cells * n / el, unit=UNIT, cores=used, kind="oracle",
                cpu=f"{host_cpu_model()}, {host_cores()} cores available",
                sample=f"{w.nx}x{w.ny} fire mesh of the same recipe ({w.name}), "
                       f"{n} FP64 oracle steps, {how}, {el:.1f} s")


# ---------------------------------------------------------------------------
# the reference arm: the oracle, one sample step per bench step
# ---------------------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_1102_1343_gb300 import synth
    total = args.steps + args.warmup
    threads = oracle.set_threads(host_cores())
    # ~100 s of oracle time at ~2.5e6 cell-steps/s per thread (half of it
    # counted: the rows loops do not scale perfectly)
    budget = 100.0 * 2.5e6 * max(1.0, threads / 2) / max(1, total)
    side = int(max(10, min(82, math.sqrt(budget) / 10)))
    w = synth.random_landscape(side, side, seed=synth.BASE_SEED, ignition="points",
                               n_points=max(1, round(50 * (side / 820) ** 2)),
                               edge_margin=2000.0 * side / 820, steps=1)
    o = oracle.OracleFire.from_workload(w)
    for _ in range(args.warmup):
        o.step(w.u, w.v, w.dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(w.u, w.v, w.dt)
    el = time.perf_counter() - t0
    oracle.set_threads(1)
    cells = w.nx * w.ny
    val = cells * args.steps / el
    how = "single host thread" if threads == 1 else f"{threads} host threads (OpenMP over rows)"
    sample = (f"{w.nx}x{w.ny} fire mesh of the {args.workload} recipe, one FP64 oracle step "
              f"per bench step, {how}")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1000 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES[args.workload], "oracle_sample": f"{w.nx}x{w.ny}"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "cpu": f"{host_cpu_model()}, {host_cores()} cores available",
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


WORKLOAD_NAMES = {"points8200": "points-fire-8200x8200 (820x820 atmos x10, 50 point ignitions)",
                  "points4000": "points-fire-4000x4000 (400x400 atmos x10, 12 point ignitions)",
                  "line2000": "line-fire-2000x2000 (200x200 atmos x10, 1 km line ignition)",
                  "circle100": "circle-fp64-100x100 (10x10 atmos x10)",
                  "burning8200": "burning-fire-8200x8200 (820x820 atmos x10, 50 ignitions "
                                 "of radius 3 km)",
                  "burning4000": "burning-fire-4000x4000 (400x400 atmos x10, 12 ignitions "
                                 "of radius 3 km)"}


# ---------------------------------------------------------------------------
# the GB300 arm
# ---------------------------------------------------------------------------

def max_over_ranks(x: float, device, world: int) -> float:
    """The largest value of x over the ranks (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Cell-steps/s of the whole job: every rank advances its own replica."""
    return cells_per_rank * steps * world / seconds


def run_gpu(args, rank, world):
    import torch
    import torch.distributed as dist

    import paper_1102_1343_gb300 as pkg
    from paper_1102_1343_gb300 import build

    build.build()
    pkg.load_library()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.only in ("adjoint", "ensemble"):
        # one section alone (for profiler captures): its own JSON object
        if rank == 0:
            out = bench_adjoint(pkg, dev) if args.only == "adjoint" else bench_ensemble(pkg, dev)
            print(json.dumps({"section": args.only, **out}), flush=True)
        return

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    w = make_workload(args.workload)
    cells = w.nx * w.ny
    prec = args.precision
    m = pkg.FireModel.from_workload(w, precision=prec, device=dev)
    u, v = m.wind(w.u, w.v)
    if args.kernel:
        pkg.fire_set_kernel(m.ctx, *args.kernel)
    elif args.autotune:
        m.autotune(u, v, w.dt, probe_steps=3)  # the library's own tuner, before timing
    kernel = pkg.fire_get_kernel(m.ctx)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        m.step(u, v, w.dt)
    barrier()

    # ---- device-timed region: K fire steps, inputs resident in HBM
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ad_on, counts0, _ = pkg.fire_adaptive_info(m.ctx)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        pkg.fire_step(m.ctx, u, v, w.dt, m.heat_s, m.heat_l)
    e1.record(stream)
    barrier()
    # the adaptive kernel choice counts burnt nodes every 64 steps (one small
    # kernel each, inside the timed region)
    _, counts1, burnt_seen = pkg.fire_adaptive_info(m.ctx)
    kernel_end = pkg.fire_get_kernel(m.ctx)
    clk = clocks.stop() if rank == 0 else {}
    ms = max_over_ranks(e0.elapsed_time(e1), dev, world)
    value = whole_job_rate(cells, args.steps, world, ms / 1000.0)
    status = m.status()

    # ---- kernel duration of the fused step kernel (events on the launching stream)
    kt_steps = min(args.steps, 200)
    pkg.fire_enable_timing(m.ctx, True)
    pkg.fire_kernel_time_ms(m.ctx)
    for _ in range(kt_steps):
        pkg.fire_step(m.ctx, u, v, w.dt, m.heat_s, m.heat_l)
    k_ms, k_n = pkg.fire_kernel_time_ms(m.ctx)
    pkg.fire_enable_timing(m.ctx, False)
    k_avg = k_ms / max(1, k_n)
    peak, peak_kind = measured_peaks()
    alg_bytes = BYTES_PER_CELL_STEP[prec] * cells
    achieved = alg_bytes / (k_avg / 1000.0) / 1e9
    traffic = profiled_traffic() if (args.workload == "points8200" and prec == "fp32") else None

    # ---- end to end through the public host-buffer entry point
    e2e_steps = min(args.steps, args.e2e_steps)
    npdt = np.float32 if prec == "fp32" else np.float64
    uh = torch.from_numpy(np.ascontiguousarray(w.u, npdt)).pin_memory().numpy()
    vh = torch.from_numpy(np.ascontiguousarray(w.v, npdt)).pin_memory().numpy()
    hs_h = torch.zeros((w.nya, w.nxa), dtype=torch.float64).pin_memory().numpy()
    hl_h = torch.zeros((w.nya, w.nxa), dtype=torch.float64).pin_memory().numpy()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pkg.fire_step_host(m.ctx, uh, vh, w.dt, hs_h, hl_h)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev, world)
    e2e_value = whole_job_rate(cells, e2e_steps, world, e2e_s)
    h2d = uh.nbytes + vh.nbytes
    d2h = hs_h.nbytes + hl_h.nbytes
    final_status = m.status()
    m.close()
    del m
    torch.cuda.empty_cache()

    # ---- the plain FP64 GPU path on the same mesh (speedup reference)
    fp64 = None
    if prec == "fp32" and not args.no_fp64:
        m64 = pkg.FireModel.from_workload(w, precision="fp64", device=dev)
        u64, v64 = m64.wind(w.u, w.v)
        n64 = args.fp64_steps
        for _ in range(2):
            m64.step(u64, v64, w.dt)
        barrier()
        e0.record(stream)
        for _ in range(n64):
            pkg.fire_step(m64.ctx, u64, v64, w.dt, m64.heat_s, m64.heat_l)
        e1.record(stream)
        barrier()
        ms64 = e0.elapsed_time(e1)
        v64 = cells * n64 / (ms64 / 1000.0)
        fp64 = {"value": v64, "unit": UNIT, "steps": n64, "ms_per_step": ms64 / n64,
                "speedup_fp32_over_fp64": value / world / v64}
        m64.close()

    burn = None
    if rank == 0 and prec == "fp32" and args.workload == "points8200" and not args.no_burning:
        burn = bench_burning(pkg, dev, args.burning_steps)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = time_oracle(args.workload, seconds=args.cpu_seconds)
        cores = host_cores()
        if cores > 1:
            # the same oracle on every host core (its OpenMP loops over rows)
            allc = time_oracle(args.workload, seconds=max(3.0, args.cpu_seconds / 2),
                               threads=cores)
            if allc["cores"] > 1:
                cpu["all_cores"] = {k: allc[k] for k in ("value", "cores", "sample")}
    adj = ens = None
    if rank == 0 and not args.no_adjoint:
        adj = bench_adjoint(pkg, dev)
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_ensemble:
        ens = bench_ensemble(pkg, dev)
        torch.cuda.empty_cache()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAMES[args.workload], "fire_mesh": [w.nx, w.ny],
                       "refinement": [w.srx, w.sry], "precision": prec,
                       "state_in_hbm": "yes; state 2.2 GB > L2, no flush needed"
                       if args.workload == "points8200" else "yes",
                       "kernel": {"variant": KERNEL_VARIANTS[kernel[0]],
                                  "tile_atmos_cells": list(kernel[1:]),
                                  "chosen_by": "--kernel" if args.kernel else
                                  ("fire_autotune" if args.autotune else "fire_init default"),
                                  "adaptive": {"on": ad_on, "burnt_fraction_seen": burnt_seen,
                                               "counts_in_timed_region": counts1 - counts0,
                                               "variant_at_end": KERNEL_VARIANTS[kernel_end[0]],
                                               "tile_at_end": list(kernel_end[1:])}},
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": args.steps + (counts1 - counts0),
            "e2e": {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": KERNEL_NAMES[kernel[0]] + ("<float>" if prec == "fp32" else "<double>"),
                         "kernel_ms": k_avg,
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "cpu_baseline": cpu,
            "accuracy": accuracy_record(),
            "burning": burn,
            "fp64_plain_gpu": fp64,
            "adjoint": adj,
            "ensemble": ens,
            "clocks": clk,
            "status": pkg.fire_strerror(status if status else final_status),
        }
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# accuracy record and the heavily burning state
# ---------------------------------------------------------------------------

ACCURACY_SUMMARY = "profiles/accuracy_line2000_fp32_fp64.md"


def accuracy_record(path=None):
    """The errors of the FP32 and FP64 paths against the FP64 oracle on the
    2000x2000 line fire over all 1200 steps, as recorded by the full-run GPU
    test (tests/test_fullrun_gpu.py) in the committed summary: the JSON block
    of the summary, with a flag saying whether it was taken on the current
    step-kernel source."""
    path = path or os.path.join(ROOT, ACCURACY_SUMMARY)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    a, b = txt.find("```json"), txt.rfind("```")
    if a < 0 or b <= a:
        return None
    try:
        rec = json.loads(txt[a + len("```json"):b])
    except ValueError:
        return None
    rec["current_kernel_source"] = rec.get("kernel_source_hash") == kernel_hash()
    rec["source"] = ACCURACY_SUMMARY
    return rec


def bench_burning(pkg, dev, steps):
    """The 8200x8200 mesh in a heavily burning state (50 ignitions of radius
    3 km, about 40 % of the domain burnt from the start): cell-steps/s and the
    roofline fraction of the step kernel where most warps run the
    fuel-fraction quadrature and the ignition-time path, with fire_init's
    default (the adaptive choice between the two warp-strip kernels) and
    then with the kernel the autotuner picks there."""
    import torch
    from paper_1102_1343_gb300 import synth
    w = synth.burning_fire_8200()
    cells = w.nx * w.ny
    m = pkg.FireModel.from_workload(w, precision="fp32", device=dev)
    u, v = m.wind(w.u, w.v)
    for _ in range(5):
        m.step(u, v, w.dt)
    psi = m.state()[0]
    burnt = float((psi <= 0).float().mean())
    del psi
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    peak, peak_kind = measured_peaks()

    def timed():
        """steps from the current state: events around the whole loop, then
        the step kernel's own events over up to 100 more steps"""
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            pkg.fire_step(m.ctx, u, v, w.dt, m.heat_s, m.heat_l)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        pkg.fire_enable_timing(m.ctx, True)
        pkg.fire_kernel_time_ms(m.ctx)
        for _ in range(min(steps, 100)):
            pkg.fire_step(m.ctx, u, v, w.dt, m.heat_s, m.heat_l)
        k_ms, k_n = pkg.fire_kernel_time_ms(m.ctx)
        pkg.fire_enable_timing(m.ctx, False)
        k_avg = k_ms / max(1, k_n)
        kernel = pkg.fire_get_kernel(m.ctx)
        achieved = BYTES_PER_CELL_STEP["fp32"] * cells / (k_avg / 1000.0) / 1e9
        return {"value": cells * steps / (ms / 1e3), "unit": UNIT, "steps": steps,
                "ms_per_step": ms / steps, "kernel_ms": k_avg,
                "kernel": KERNEL_NAMES[kernel[0]] + "<float>",
                "variant": KERNEL_VARIANTS[kernel[0]], "tile_atmos_cells": list(kernel[1:]),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs"}}

    out = {"workload": f"{w.name} (820x820 atmos x10, 50 ignitions of radius 3 km)",
           "burnt_fraction_at_start": burnt}
    out.update(timed())
    # the kernel the autotuner picks on this state (timed from where the
    # default kernel's steps left the fire)
    m.autotune(u, v, w.dt)
    out["autotuned"] = timed()
    out["status"] = pkg.fire_strerror(m.status())
    m.close()
    return out


# ---------------------------------------------------------------------------
# the two growth rows: adjoint and batched ensemble
# ---------------------------------------------------------------------------

def _clone_state(st):
    return tuple(x.clone() if hasattr(x, "clone") else x for x in st)


def bench_adjoint(pkg, dev, ckpt=20):
    """fire_adjoint on the 510x510 adjoint workload (400 steps of 0.5 s,
    checkpoints every 20, and every state kept): misfit against the arrival
    times of a perturbed truth run, gradients w.r.t. multiplier, moisture and
    wind; and fire_adjoint_heat against the heat that run released per
    atmospheric cell.  Cell-steps/s of the whole call (forward with
    checkpoints + reverse sweep) and of the plain forward on the same mesh,
    each with its autotuned kernel."""
    import torch
    from paper_1102_1343_gb300 import synth
    w, truth = synth.adjoint_case()
    n = w.nx * w.ny * w.steps
    import dataclasses
    wt = dataclasses.replace(w, mult=truth["mult"], classes=truth["classes"])
    tr = pkg.FireModel.from_workload(wt, precision="fp64", device=dev)
    ut, vt = tr.wind(w.u * truth["wind_scale"], w.v * truth["wind_scale"])
    tr.autotune(ut, vt, w.dt)
    # the truth run, also summing its heat flux for the heat-misfit
    # observations (sensible heat released per atmospheric cell)
    qobs = torch.zeros((w.nya, w.nxa), dtype=torch.float64, device=dev)
    for _ in range(w.steps):
        hs, _ = tr.step(ut, vt, w.dt)
        qobs += hs * w.dt
    tobs = tr.state()[1]
    tobs = torch.where(torch.isfinite(tobs), tobs, torch.full_like(tobs, float("nan")))
    tr.close()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    out = {"workload": f"{w.name} (51x51 atmos x10, centre ignition), {w.steps} steps of "
                       f"{w.dt} s, checkpoints every {ckpt}; t_obs from a truth run with "
                       "multiplier 1+0.2f, moisture +0.02, wind x1.1",
           "unit": UNIT}
    grads = {}
    for prec in ("fp64", "fp32"):
        m = pkg.FireModel.from_workload(w, precision=prec, device=dev)
        u, v = m.wind(w.u, w.v)
        kern = m.autotune(u, v, w.dt)
        st0 = _clone_state(m.state())
        J, gm, gM, gu, gv = m.adjoint(u, v, w.dt, w.steps, tobs, ckpt)  # warm-up
        m.set_state(*st0)
        stream = torch.cuda.current_stream(dev)
        torch.cuda.synchronize()
        e0.record(stream)
        J, gm, gM, gu, gv = m.adjoint(u, v, w.dt, w.steps, tobs, ckpt)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        grads[prec] = (J, gm, gM, gu, gv)
        rec = {"value": n / (ms / 1e3), "ms": ms, "J": J,
               "kernel": {"variant": KERNEL_VARIANTS[kern[0]],
                          "tile_atmos_cells": list(kern[1:])}}
        # every state kept (checkpoint interval 1: no recomputed forward;
        # 401 states of the mesh in HBM)
        m.set_state(*st0)
        m.adjoint(u, v, w.dt, w.steps, tobs, 1)
        m.set_state(*st0)
        torch.cuda.synchronize()
        e0.record(stream)
        J1, *_ = m.adjoint(u, v, w.dt, w.steps, tobs, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms1 = e0.elapsed_time(e1)
        rec["every_state_kept"] = {"value": n / (ms1 / 1e3), "ms": ms1, "J": J1,
                                   "state_bytes": (w.steps + 1) * w.nx * w.ny *
                                   (8 if prec == "fp64" else 4)}
        # the heat-misfit adjoint on the same run (warm-up, then timed)
        m.set_state(*st0)
        m.adjoint_heat(u, v, w.dt, w.steps, qobs, ckpt)
        m.set_state(*st0)
        torch.cuda.synchronize()
        e0.record(stream)
        Jh, *_ = m.adjoint_heat(u, v, w.dt, w.steps, qobs, ckpt)
        e1.record(stream)
        torch.cuda.synchronize()
        hms = e0.elapsed_time(e1)
        rec["heat_misfit"] = {"value": n / (hms / 1e3), "ms": hms, "J": Jh}
        # the plain forward on the same mesh and kernel
        m.set_state(*st0)
        m.run(2, u, v, w.dt)
        m.set_state(*st0)
        torch.cuda.synchronize()
        e0.record(stream)
        m.run(w.steps, u, v, w.dt)
        e1.record(stream)
        torch.cuda.synchronize()
        fms = e0.elapsed_time(e1)
        rec["plain_forward"] = {"value": n / (fms / 1e3), "ms": fms}
        rec["ratio_to_plain_forward"] = {f"ckpt{ckpt}": fms / ms, "ckpt1": fms / ms1}
        # one reverse step: the call with every state kept less its forward
        # (the plain forward's time), per step; algorithmic bytes per node of
        # the FP32 fused step: psi^s, psi^{s+1}, lambda in and out, t_i at
        # the start and end, t_obs, class, multiplier, slope, node wind, and
        # the four compensated parameter sums read and written
        E = 8 if prec == "fp64" else 4
        b_node = 5 * E + 3 * 8 + 1 + (E if w.mult is not None else 0) + 2 * E + 4 * 2 * 8
        us = (ms1 - fms) * 1e3 / w.steps
        peak, peak_kind = measured_peaks()
        gbs = b_node * w.nx * w.ny / (us * 1e-6) / 1e9
        rec["reverse_step"] = {"us": us, "bytes_per_node": b_node, "achieved_gbs": gbs,
                               "frac_of_hbm": gbs / peak, "peak_source": f"{peak_kind} hbm_gbs",
                               "kernel": "k_adj_step<float> (one launch)" if prec == "fp32" else
                               "k_adj_stage1/vjp_star/vjp_n/finish<double> (four launches)",
                               "note": "estimated as (every-state-kept call - plain forward) / "
                                       "steps; the step's working set fits in L2"}
        out[prec] = rec
        m.close()
    base = out["fp64"]["plain_forward"]["value"]
    out["speedup_vs_fp64_plain_forward"] = {p: out[p]["value"] / base for p in ("fp64", "fp32")}
    out["heat_misfit_speedup_vs_fp64_plain_forward"] = {
        p: out[p]["heat_misfit"]["value"] / base for p in ("fp64", "fp32")}

    def rel(a, b):
        return float(torch.linalg.norm((a - b).flatten()) / max(float(torch.linalg.norm(b.flatten())), 1e-300))
    g64, g32 = grads["fp64"], grads["fp32"]
    out["fp32_vs_fp64_gradient_rel"] = {k: rel(g32[i], g64[i]) for i, k in
                                        ((1, "mult"), (2, "moisture"), (3, "u"), (4, "v"))}
    out["fp32_vs_fp64_J_rel"] = abs(g32[0] - g64[0]) / max(abs(g64[0]), 1e-300)
    out["accuracy_note"] = ("GPU FP64 gradients equal the oracle's reference adjoint to ~1e-15 "
                            "relative on this workload (tests/test_adjoint_gpu.py)")
    return out


def bench_ensemble(pkg, dev, steps=600, n_members=64):
    """64 members of uneven size (fire meshes 390^2..2050^2, 96.8 M nodes in
    all), wind x U[0.8, 1.2] and moisture +- 0.03 per member, FP32 with FP64
    ignition time: one fire_ensemble_step call of 600 steps (persistent
    cooperative launch replayed from a CUDA graph, autotuned strips), against
    the same members run one by one (fire_run, FP32 and the plain FP64 step)."""
    import torch
    from paper_1102_1343_gb300 import synth
    sizes = synth.ensemble_sizes(n_members)
    ws = [synth.ensemble_member(k, s, steps=steps) for k, s in enumerate(sizes)]
    cells = sum(w.nx * w.ny for w in ws)
    keep, members, us, vs = [], [], [], []
    for w in ws:
        fuel = torch.as_tensor(w.fuel).to(dev).contiguous()
        zx = torch.as_tensor(w.dzdx).to(dev, torch.float32).contiguous()
        zy = torch.as_tensor(w.dzdy).to(dev, torch.float32).contiguous()
        keep += [fuel, zx, zy]
        members.append(dict(grid=pkg.make_grid(w.nxa, w.nya, w.srx, w.sry, w.dx_atm, w.dy_atm,
                                               pkg.FIRE_FP32, w.band, w.eps),
                            classes=w.classes, fuel_class_dev=fuel, dzdx_dev=zx, dzdy_dev=zy,
                            ignitions=w.ignitions))
        us.append(torch.as_tensor(w.u).to(dev, torch.float32).contiguous())
        vs.append(torch.as_tensor(w.v).to(dev, torch.float32).contiguous())
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    ens = pkg.fire_ensemble_create(members, stream.cuda_stream)
    dt = ws[0].dt
    shape = pkg.fire_ensemble_autotune(ens, 3, dt, us, vs)
    grid, items = pkg.fire_ensemble_get_kernel(ens)
    pkg.fire_ensemble_step(ens, 5, dt, us, vs)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    pkg.fire_ensemble_step(ens, steps, dt, us, vs)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    code, _ = pkg.fire_ensemble_status(ens, n_members)
    pkg.fire_ensemble_destroy(ens)
    value = cells * steps / (ms / 1e3)
    out = {"workload": f"{n_members} members, fire meshes {min(w.nx for w in ws)}^2.."
                       f"{max(w.nx for w in ws)}^2 ({cells / 1e6:.1f} M nodes), {steps} steps "
                       f"of {dt} s, FP32 + FP64 t_i",
           "value": value, "unit": UNIT, "ms": ms, "launch_calls": 1,
           "strip_nodes": list(shape), "grid_ctas": grid, "work_items_per_step": items,
           "status": pkg.fire_strerror(code)}
    # the same members one by one (sample of 20 steps each)
    del keep
    seq = {}
    for prec in ("fp32", "fp64"):
        tot_ms, tot_cs = 0.0, 0
        for w in ws:
            m = pkg.FireModel.from_workload(w, precision=prec, device=dev)
            u, v = m.wind(w.u, w.v)
            m.autotune(u, v, w.dt, probe_steps=2)
            m.run(2, u, v, w.dt)
            torch.cuda.synchronize()
            e0.record(stream)
            m.run(20, u, v, w.dt)
            e1.record(stream)
            torch.cuda.synchronize()
            tot_ms += e0.elapsed_time(e1)
            tot_cs += w.nx * w.ny * 20
            m.close()
        seq[prec] = {"value": tot_cs / (tot_ms / 1e3), "unit": UNIT,
                     "sample": "each member alone (own autotuned kernel), 20 steps"}
    out["one_by_one"] = seq
    out["speedup_vs_fp64_plain_per_run"] = value / seq["fp64"]["value"]
    out["speedup_vs_fp32_per_run"] = value / seq["fp32"]["value"]
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["points8200", "line2000", "circle100", "points4000",
                                           "burning8200", "burning4000"],
                    default="points8200")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--kernel", type=int, nargs=3, default=None,
                    metavar=("VARIANT", "KX", "KY"),
                    help="step kernel (FIRE_KERNEL_*): 0 = 2-D tile, 1 = column march, "
                         "2 = warp strips, 3 = four-column warp strips, 4 = dense warp strips; "
                         "shape in atmos cells")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--only", choices=["adjoint", "ensemble"], default=None,
                    help="run one growth section alone and print its object (profiling)")
    ap.add_argument("--autotune", action="store_true",
                    help="time the shape fire_autotune picks instead of fire_init's default")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-burning", action="store_true")
    ap.add_argument("--burning-steps", type=int, default=200)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if args.impl == "gb300":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_gpu(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            if dist.is_initialized():
                dist.destroy_process_group()


if __name__ == "__main__":
    main()
