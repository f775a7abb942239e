#!/usr/bin/env python3
"""Throughput of the fused two-component D2Q9 step on one GB300.

A step is one pass of the whole hot path over the lattice: pull streaming
with bounce-back, Set-3 boundaries, densities, virtual solid densities,
forces, system relaxation time and velocity, forced collision.  The timed
workload is the 2048x1024 polydisperse (lognormal, mean radius 10, sigma_log
0.4, radii halved downstream) disk medium of seed 99 in FP32, viscosity ratio
10 (tau 1.7 / 0.62), water-wet theta = 50 deg, primary drainage with
rho_in = 1.005 and rho_out = 1.  Its working set (two population buffers:
181 MB in the fluid-only layout, 302 MB dense) exceeds the 129 MB L2, so
consecutive steps stream from HBM without a flush.  The 1024x512
lattice of the same recipe is also timed and reported as L2-resident.

One JSON line on stdout (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (bounded samples of the same workload).
Under torchrun every rank advances its own replica; the job time is the
slowest rank's and the work is summed.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_2111_08666_gb300 import media, replicas  # noqa: E402

METRIC = "2-comp D2Q9 MLUPS (fused step, FP32 storage)"
UNIT = "MLUPS"
FALLBACK_HBM_GBS = 6800.0
# The step kernels: their sources, and the DRAM bytes per launch from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) on the workload below with
# the hash of the sources they were taken with; reported only while the
# sources match.  The fluid-only kernel's figure is the steady state: the
# mean of five consecutive launches captured without cache flushes, so that
# the write-back of each step's output is counted.
_COMMON = ["paper_2111_08666_gb300/csrc/async_copy.cuh",
           "paper_2111_08666_gb300/csrc/lbm_device.cuh",
           "paper_2111_08666_gb300/csrc/lbm.cuh"]
STEP_KERNELS = {
    "sparse_kernel": {"sources": ["paper_2111_08666_gb300/csrc/sparse.cu"] + _COMMON,
                      "ncu_bytes": 183841741, "ncu_sha": "c253f58b1307dfe1"},
    "tma_tile_kernel": {"sources": ["paper_2111_08666_gb300/csrc/tma_tile.cu"] + _COMMON,
                        "ncu_bytes": 268262144, "ncu_sha": "127f58da57dc516e"},
    "fused_step_kernel": {"sources": ["paper_2111_08666_gb300/csrc/step.cu"] + _COMMON,
                          "ncu_bytes": None, "ncu_sha": None},
    "sweep_kernel": {"sources": ["paper_2111_08666_gb300/csrc/sweep.cu"] + _COMMON,
                     "ncu_bytes": None, "ncu_sha": None},
}
FLUID_ONLY_PRECISIONS = ("fp32", "fp16dev", "bf16dev")
# The FP64 step (kernel 1) is bound by the FP64 pipe, not by HBM: FP64
# floating-point operations per fluid-node update counted by ncu on the
# workload below (DADD + DMUL + 2 DFMA thread instructions per launch over
# the fluid nodes), and the GB300's FP64 FMA rate measured by a probe of
# independent FMA chains (1.257 TFLOP/s; nominal 1.25).
FP64_FLOPS_PER_FLUID_NODE = 367.0
FP64_PEAK_GFLOPS = 1257.0


def step_kernel(kernel: str, prec: str) -> str:
    """Name of the kernel a step runs (the library's automatic choice for 'auto')."""
    if kernel == "auto":
        if prec in FLUID_ONLY_PRECISIONS:
            return "sparse_kernel"
        return "fused_step_kernel" if prec == "fp64" else "tma_tile_kernel"
    return {"tile": "fused_step_kernel", "strip": "sweep_kernel", "tma": "tma_tile_kernel",
            "fluid": "sparse_kernel"}[kernel]


def tile_label(kname: str, shape: int, prec: str) -> str:
    """Tile of the step kernel that runs."""
    if kname == "sparse_kernel":
        return "16-row bands, width <= 32, <= 384 fluid" if shape == 1 else "12-row bands, width <= 32, <= 256 fluid"
    if kname == "tma_tile_kernel":
        return "32x8" if shape == 1 else ("32x12" if prec == "fp32dev" else "32x16")
    return "32x16"


def l2_note(c, kname: str, prec: str) -> str:
    """The two population buffers of the timed step against the 129 MB L2:
    the fluid-only layout holds the fluid nodes only, the dense layout every
    node with its ghost rows and columns."""
    nb = PLANES[prec] * {"fp64": 8, "fp32": 4, "fp32dev": 4, "fp16dev": 2, "bf16dev": 2}[prec]
    nodes = int((c["solid"] == 0).sum()) if kname == "sparse_kernel" else (c["nx"] + 8) * (c["ny"] + 6)
    mb = 2 * nodes * nb / 1e6
    return f"working set {mb:.0f} MB (two population buffers) > 129 MB L2, no flush needed"


def kernel_sha(name: str = "sparse_kernel") -> str:
    h = hashlib.sha256()
    for p in STEP_KERNELS[name]["sources"]:
        h.update((ROOT / p).read_bytes())
    return h.hexdigest()[:16]


def workload(nx=2048, ny=1024, seed=99):
    c = media.config_paper_scale(nx, ny, seed)
    c["rho_in1"] = 1.005
    c["rho_out2"] = 1.0
    return c


PLANES = {"fp64": 18, "fp32": 18, "fp32dev": 20, "fp16dev": 20, "bf16dev": 20}


def algorithmic_bytes(c, store_bytes: int, planes: int = 18) -> float:
    """Per launch: each fluid node reads and writes its stored values once
    (2 x 9 populations, plus the two reference densities of the deviation
    storages); every node's 1-byte geometry code is read once."""
    n_fluid = int((c["solid"] == 0).sum())
    n_all = c["nx"] * c["ny"]
    return 2 * planes * store_bytes * n_fluid + n_all


def measured_peaks() -> tuple[float, str]:
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            d = json.loads(p.read_text())
            for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "pci.bus_id")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.rows: list[list[str]] = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self

        def reader():
            for line in self.proc.stdout:
                self.rows.append([s.strip() for s in line.split(",")])
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        return self

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        rows = [r for r in self.rows if len(r) >= 9]
        if self.bus_id:
            mine = [r for r in rows if self.bus_id[-12:] in r[8].lower()]
            rows = mine or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[4 + k].lower() in ("active", "yes", "1")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def run_gpu(args, rank, world):
    import torch
    from paper_2111_08666_gb300 import mclbm
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.Stream()
    prec = mclbm.PRECISIONS[args.prec]
    c = workload()
    kernel = {"auto": 0, "tile": 1, "strip": 2, "tma": 3, "fluid": 4}[args.kernel]
    lat = mclbm.Lattice(c["solid"], c["xi"], prec=prec, nu1=c["nu1"], nu2=c["nu2"],
                        rho_in1=c["rho_in1"], rho_out2=c["rho_out2"], stream=stream,
                        kernel=kernel, tile_shape=args.tile_shape)
    lat.init(c["rho1"], c["rho2"])
    n_all = c["nx"] * c["ny"]
    lat.step(max(args.warmup, 3))
    lat.sync()
    bus = None
    try:
        bus = torch.cuda.get_device_properties(torch.cuda.current_device()).pci_bus_id
    except Exception:
        pass
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    replicas.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(bus).start() if rank == 0 else None
    launches0 = mclbm.mclbm_launch_count()
    # the timed steps: one API call, as a user advances a lattice (one
    # launch per step)
    start.record(stream)
    lat.step(args.steps)
    end.record(stream)
    launches = mclbm.mclbm_launch_count() - launches0
    torch.cuda.synchronize()
    replicas.barrier()
    clocks = sampler.stop() if sampler else None
    sec = start.elapsed_time(end) / 1e3
    diag = lat.diagnostics()
    units, job_sec = replicas.aggregate(n_all * args.steps, sec)
    value = units / job_sec / 1e6
    per_launch = sec / args.steps
    abytes = algorithmic_bytes(c, mclbm.STORE_BYTES[prec], PLANES[args.prec])
    peak, peak_kind = measured_peaks()
    achieved = abytes / per_launch / 1e9
    traffic = None
    kname = step_kernel(args.kernel, args.prec)
    rec = STEP_KERNELS[kname]
    if rec["ncu_bytes"] and rec["ncu_sha"] == kernel_sha(kname):
        traffic = rec["ncu_bytes"]

    # end to end through the public API with host buffers: upload the
    # initial densities, step, read back the water density and diagnostics
    rho1 = np.ascontiguousarray(c["rho1"])
    rho2 = np.ascontiguousarray(c["rho2"])
    pin1 = torch.from_numpy(rho1).pin_memory()
    pin2 = torch.from_numpy(rho2).pin_memory()
    out = torch.empty((c["ny"], c["nx"]), dtype=torch.float64).pin_memory()
    e2e_steps = args.steps
    torch.cuda.synchronize()
    replicas.barrier()
    t0 = time.perf_counter()
    mclbm.mclbm_init_densities(lat.h, pin1, pin2)
    mclbm.mclbm_step(lat.h, e2e_steps)
    mclbm.mclbm_read_density(lat.h, 2, out)
    d_e2e = lat.diagnostics()
    e2e_sec = time.perf_counter() - t0
    replicas.barrier()
    e2e_units, e2e_job = replicas.aggregate(n_all * e2e_steps, e2e_sec)
    h2d = 2 * rho1.nbytes
    d2h = out.numel() * 8 + 8 * 8

    # the 1024x512 lattice of the same recipe: L2-resident, context only
    c2 = workload(1024, 512, 1)
    lat2 = mclbm.Lattice(c2["solid"], c2["xi"], prec=prec, nu1=c2["nu1"], nu2=c2["nu2"],
                         rho_in1=c2["rho_in1"], rho_out2=c2["rho_out2"], stream=stream,
                         kernel=kernel, tile_shape=args.tile_shape)
    lat2.init(c2["rho1"], c2["rho2"])
    lat2.step(20)
    lat2.sync()
    k2 = max(args.steps, 100)
    start.record(stream)
    lat2.step(k2)
    end.record(stream)
    torch.cuda.synchronize()
    l2_mlups = 1024 * 512 * k2 / (start.elapsed_time(end) / 1e3) / 1e6
    lat2.close()

    batched = None
    if args.batch_steps > 0:
        batched = batched_section(args, stream, peak)
    storages = None
    if args.prec == "fp32" and args.storage_steps > 0:
        storages = storage_section(args, stream, c, peak)
    fp64 = None
    if args.prec == "fp32" and args.fp64_steps > 0:
        fp64 = fp64_section(args, stream, c)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": round(job_sec / args.steps * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "fp32dev": "f32",
                  "fp16dev": "f16-storage/f32", "bf16dev": "bf16-storage/f32"}[args.prec],
        "data": "synthetic",
        "config": {"workload": f"{c['name']} seed 99 (drainage, M=10, theta=50 deg, "
                               f"rho_in=1.005, rho_out=1)",
                   "nx": c["nx"], "ny": c["ny"], "porosity": round(c["porosity"], 4),
                   "storage": args.prec, "step_kernel": args.kernel, "tile_shape": args.tile_shape,
                   "tile": tile_label(kname, args.tile_shape, args.prec),
                   "parallelism": f"replicas x{world}",
                   "l2": l2_note(c, kname, args.prec),
                   "mflups": round(value * (c["solid"] == 0).mean(), 1),
                   "l2_resident_1024x512_mlups": round(l2_mlups, 1)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_source": peak_kind, "algorithmic_bytes_per_launch": abytes,
                     "kernel": kname, "launch_us": round(per_launch * 1e6, 3)},
        "e2e": {"value": round(e2e_units / e2e_job / 1e6, 1), "unit": UNIT,
                "h2d_bytes_per_step": round(h2d / e2e_steps, 1),
                "d2h_bytes_per_step": round(d2h / e2e_steps, 1)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cpu_baseline": cpu,
        "batched": batched,
        "storages": storages,
        "fp64": fp64,
        "diag": {k: (None if isinstance(v, float) and math.isnan(v) else v)
                 for k, v in diag.items()},
    }
    lat.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def storage_section(args, stream, c, peak) -> dict:
    """The same workload in the 16-bit deviation storages (FP16 and BF16
    values, FP32 arithmetic): MLUPS and the fraction of the HBM roofline on
    their own algorithmic bytes (20 stored values of 2 bytes per fluid node,
    read and written, plus the geometry byte)."""
    import torch
    from paper_2111_08666_gb300 import mclbm
    out = {}
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name in ("fp16dev", "bf16dev"):
        p = mclbm.PRECISIONS[name]
        lat = mclbm.Lattice(c["solid"], c["xi"], prec=p, nu1=c["nu1"], nu2=c["nu2"],
                            rho_in1=c["rho_in1"], rho_out2=c["rho_out2"], stream=stream)
        lat.init(c["rho1"], c["rho2"])
        lat.step(20)
        lat.sync()
        start.record(stream)
        lat.step(args.storage_steps)
        end.record(stream)
        torch.cuda.synchronize()
        sec = start.elapsed_time(end) / 1e3 / args.storage_steps
        ab = algorithmic_bytes(c, mclbm.STORE_BYTES[p], PLANES[name])
        out[name] = {"mlups": round(c["nx"] * c["ny"] / sec / 1e6, 1), "launch_us": round(sec * 1e6, 3),
                     "algorithmic_bytes_per_launch": ab,
                     "achieved_gbs": round(ab / sec / 1e9, 1), "frac": round(ab / sec / 1e9 / peak, 4),
                     "steps": args.storage_steps}
        lat.close()
    return out


def fp64_section(args, stream, c) -> dict:
    """The same workload in FP64 storage and arithmetic (the parity path):
    MLUPS and the fraction of the FP64 FMA rate its floating-point
    operations reach (the FP64 pipe, not HBM, bounds this step)."""
    import torch
    from paper_2111_08666_gb300 import mclbm
    lat = mclbm.Lattice(c["solid"], c["xi"], prec="fp64", nu1=c["nu1"], nu2=c["nu2"],
                        rho_in1=c["rho_in1"], rho_out2=c["rho_out2"], stream=stream)
    lat.init(c["rho1"], c["rho2"])
    lat.step(3)
    lat.sync()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    lat.step(args.fp64_steps)
    end.record(stream)
    torch.cuda.synchronize()
    sec = start.elapsed_time(end) / 1e3 / args.fp64_steps
    lat.close()
    n_fluid = int((c["solid"] == 0).sum())
    gflops = FP64_FLOPS_PER_FLUID_NODE * n_fluid / sec / 1e9
    return {"mlups": round(c["nx"] * c["ny"] / sec / 1e6, 1), "launch_us": round(sec * 1e6, 1),
            "roofline": {"bound": "alu", "achieved": round(gflops, 1), "peak": FP64_PEAK_GFLOPS,
                         "unit": "GFLOP/s (FP64)", "frac": round(gflops / FP64_PEAK_GFLOPS, 4),
                         "flops_per_fluid_node": FP64_FLOPS_PER_FLUID_NODE},
            "steps": args.fp64_steps}


def batched_section(args, stream, peak) -> dict:
    """24 uneven cases (256x256 .. 1024x512, seeds 10..33, theta 30..150 deg,
    M = 1, 10, 50), FP32: one persistent launch per step under a CUDA graph
    with the autotuned tile, against the same cases stepped one at a time.
    The roofline fraction counts the algorithmic bytes of all cases (144 B
    per fluid node and 1 B per node) per batched step."""
    import torch
    from paper_2111_08666_gb300 import mclbm
    cases = [media.config_batch(k) for k in range(24)]
    nodes = sum(c["nx"] * c["ny"] for c in cases)
    abytes = sum(algorithmic_bytes(c, 4) for c in cases)
    k_steps = args.batch_steps
    b = mclbm.mclbm_batch_create(cases, mclbm.MCLBM_FP32, stream)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        mclbm.mclbm_batch_step(b, 48)          # tuning + graph capture + warm-up
        torch.cuda.synchronize()
        l0 = mclbm.mclbm_launch_count()
        start.record(stream)
        mclbm.mclbm_batch_step(b, k_steps)
        end.record(stream)
        torch.cuda.synchronize()
        launches = mclbm.mclbm_launch_count() - l0
        t_batch = start.elapsed_time(end) / 1e3
        info = mclbm.mclbm_batch_info(b)
        tuning = mclbm.mclbm_batch_tuning(b)
    finally:
        mclbm.mclbm_batch_destroy(b)
    def one_at_a_time(kernel):
        lats = []
        for c in cases:
            lat = mclbm.Lattice(c["solid"], c["xi"], prec="fp32", nu1=c["nu1"], nu2=c["nu2"],
                                rho_in1=c["rho_in1"], rho_out2=c["rho_out2"], stream=stream,
                                kernel=kernel)
            lat.init(c["rho1"], c["rho2"])
            lat.step(3)
            lats.append(lat)
        torch.cuda.synchronize()
        start.record(stream)
        for lat in lats:
            lat.step(k_steps)
        end.record(stream)
        torch.cuda.synchronize()
        t = start.elapsed_time(end) / 1e3
        for lat in lats:
            lat.close()
        return t

    t_seq = one_at_a_time(3)       # the batch's kernel, one launch per lattice
    t_fluid = one_at_a_time(4)     # the fluid-only kernel, one lattice at a time
    return {"workload": "24 disk media 256x256..1024x512, seeds 10-33, theta 30-150 deg, "
                        "M=1/10/50, FP32, drainage rho_in=1.005",
            "nodes": nodes, "steps": k_steps,
            "mlups_batched": round(nodes * k_steps / t_batch / 1e6, 1),
            "algorithmic_bytes_per_step": abytes,
            "frac": round(abytes / (t_batch / k_steps) / 1e9 / peak, 4),
            "mlups_one_at_a_time": round(nodes * k_steps / t_seq / 1e6, 1),
            "mlups_one_at_a_time_fluid_only": round(nodes * k_steps / t_fluid / 1e6, 1),
            "launches": int(launches),
            "step": ["tile 32x16", "tile 32x8", "fluid-only 12-row bands", "fluid-only 16-row bands"][info["shape"]],
            "grid": "persistent" if info["grid"] == 0 else "one CTA per tile",
            "tuner_ms_per_step": [round(x, 4) for x in tuning]}


def cpu_baseline(seconds: float) -> dict:
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload: the same medium recipe over the full 2048-node length and a
    shorter height, stepped for about ``seconds``."""
    import oracle
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    c = workload(2048, 128, 99)
    o = oracle.Oracle(c["solid"], c["xi"], nu1=c["nu1"], nu2=c["nu2"], rho_in1=c["rho_in1"],
                      rho_out2=c["rho_out2"])
    o.init(c["rho1"], c["rho2"])
    o.step(1)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        o.step(2)
        n += 2
    dt = time.perf_counter() - t0
    return {"value": round(c["nx"] * c["ny"] * n / dt / 1e6, 3), "unit": UNIT,
            "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"{c['nx']}x{c['ny']} lattice of the same medium recipe, {n} FP64 steps "
                      f"in {dt:.1f} s"}


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, timed per step on a bounded sample
    of the workload (the same medium recipe at full length, a height chosen
    so the whole run stays within a few minutes)."""
    if rank != 0:
        return
    import oracle
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    total = args.steps + max(args.warmup, 3)
    budget_lups = 1.5e9
    ny = int(max(16, min(1024, budget_lups / total / 2048)))
    c = workload(2048, ny, 99)
    o = oracle.Oracle(c["solid"], c["xi"], nu1=c["nu1"], nu2=c["nu2"], rho_in1=c["rho_in1"],
                      rho_out2=c["rho_out2"])
    o.init(c["rho1"], c["rho2"])
    o.step(max(args.warmup, 3))
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = c["nx"] * c["ny"] * args.steps / dt / 1e6
    sample = f"{c['nx']}x{c['ny']} lattice of the workload's medium recipe per step"
    line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": round(dt / args.steps * 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{c['name']} (bounded sample of the 2048x1024 seed-99 "
                                   f"workload)", "nx": c["nx"], "ny": c["ny"]},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT,
                             "cores": oracle.get_threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["fp64", "fp32", "fp32dev", "fp16dev", "bf16dev"],
                    default="fp32")
    ap.add_argument("--kernel", choices=["auto", "tile", "strip", "tma", "fluid"], default="auto")
    ap.add_argument("--tile-shape", type=int, choices=[0, 1], default=0,
                    help="tile shape: TMA kernel 0 = 32x16 (32x12 fp32dev), 1 = 32x8; "
                         "fluid-only kernel 0 = 12-row bands, 1 = 16-row bands")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batch-steps", type=int, default=400,
                    help="steps of the 24-case batched section (0: skip it)")
    ap.add_argument("--storage-steps", type=int, default=2000,
                    help="steps of each 16-bit deviation storage's timing (0: skip it)")
    ap.add_argument("--fp64-steps", type=int, default=100,
                    help="steps of the FP64 step's timing (0: skip it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank, world, _ = replicas.rank_info()
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_gpu(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
