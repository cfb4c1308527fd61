#!/usr/bin/env python3
"""Benchmark of the semi-Lagrangian level-set iteration on one GB300.

Workload (default): 1,000,000 points on a union of three superquadrics with a
10x density variation, 256^3 grid on [-1,1]^3, φ^0 = sphere of radius 0.9,
narrow band of 6h, WENO interpolation, FP32 storage and arithmetic, p = 2,
δ = 1, Δt = h/4.

One benchmark step is one iteration of Algorithm 1 on the device: band
rebuild + SL update + cut (one fused kernel), the energy quadrature of the
new state, and the record/stop kernel — replayed from a captured CUDA graph.
The metric is SL node-updates per second: band nodes updated in the timed
steps divided by their device time (CUDA events on the job's stream). The L2
cache is flushed (a 256 MB write) between timed steps, outside the events.

Also reported on the same JSON line:
  roofline      the dominant kernel of a step against its bound;
  cpu_baseline  the FP64 oracle on the host cores, a bounded sample;
  e2e           whole jobs through the public API from host buffers (copy in,
                distance grid, init, evolve to the stop test, extract, copy out);
  latency       p50/p99 of the iteration time and of the whole-job solve time;
  variants      node-updates/s of Q1 and of FP64 at the same workload;
  clocks        nvidia-smi samples taken during the timed region.

--impl reference times the oracle (the CPU FP64 implementation written from
the paper) on the same workload instead; see run_reference().
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2410_22205_gb300 import synth  # noqa: E402

METRIC = "SL node-updates/s at 256^3 (WENO, FP32, narrow band 6h)"
UNIT = "node-updates/s"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--n", type=int, default=256, help="nodes per axis")
    ap.add_argument("--points", type=int, default=1_000_000)
    ap.add_argument("--e2e-jobs", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--interp", choices=["weno", "q1"], default="weno",
                    help="interpolator of the timed workload (the headline is WENO)")
    ap.add_argument("--precision", type=int, choices=[32, 64], default=32,
                    help="storage and arithmetic precision of the timed workload (the headline is FP32)")
    ap.add_argument("--fullgrid", action="store_true",
                    help="time the whole-grid step (band off) instead of the narrow band")
    ap.add_argument("--reinit", action="store_true",
                    help="time the iteration with the reinitialisation of §3.7 (Algorithm 1) on")
    ap.add_argument("--batch-jobs", type=int, default=64, help="jobs of the batched mix (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=15.0,
                    help="length of each Poisson serving stream (0: skip)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; no data-path collective)
# ---------------------------------------------------------------------------

class Dist:
    def __init__(self, backend):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def reduce(self, value, op):
        """Reduce a float over ranks: op in {"sum", "max"}."""
        if not self.pg:
            return value
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM if op == "sum" else self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(units, seconds, dist):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    tot = dist.reduce(units, "sum")
    tmax = dist.reduce(seconds, "max")
    return tot / tmax if tmax > 0 else 0.0, tot, tmax


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def workload(args, seed=2):
    grid = synth.cube_grid(3, args.n)
    cloud = synth.superquadric_union_cloud(args.points, 3, seed)
    return grid, cloud


def cfg_kw():
    return dict(p=2.0, delta=1.0)


# the sources each dominant kernel is compiled from (its translation unit and
# the headers it includes): profiles/traffic.json holds DRAM counters only
# for the hash of these files, so any change to the kernel voids them
KERNEL_SOURCES = {
    "k_step_brick": ["slr_brick.cu", "slr_brick.cuh", "slr_compact.cuh", "slr_internal.cuh"],
    "k_step_band": ["slr_step.cu", "slr_step.cuh", "slr_compact.cuh", "slr_internal.cuh"],
    "k_energy": ["slr_energy.cu", "slr_energy.cuh", "slr_compact.cuh", "slr_internal.cuh"],
}


def sha_of_kernel(name):
    """Hash of the sources of kernel `name`: its translation unit and the
    headers its device code uses (every csrc file if the name is unknown)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2410_22205_gb300", "csrc")
    files = KERNEL_SOURCES.get(name.split("<")[0], sorted(os.listdir(csrc)))
    for fn in files:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


# WENO flops per band node and step as the survey counts the paper's
# algorithm (§3.2: 4 feet x 21 one-dimensional WENO evaluations of about 40
# operations with the quadratic forms A_L, A_R and the weights alpha_k =
# C_k / (I_k + eps)^2; 3.4-4.0 kflop): the lower end is the roofline's count
WENO_FLOPS_SURVEY = 3400.0
# the kernel's own count: 4 feet x 21 evaluations of the closed form (24 flops
# with FMA = 2) plus ~140 for gradients, tangents and feet
WENO_FLOPS_EXECUTED = 2156.0


def alu_peaks(peaks, probe):
    """FP32 ALU peaks: derived from the unit counts (SMs x 128 FP32 lanes x 2
    flops per FMA x the maximum SM clock, both read from the device) and
    measured by slr_probe_fma on the device in this run."""
    derived = peaks["sms"] * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    return {"derived_tflops": derived, "derived_from": f"{peaks['sms']} SMs x 128 FP32 lanes x 2 x "
                                                     f"{peaks['sm_max_mhz']:.0f} MHz",
            "measured_tflops": probe.get("fp32_tflops"), "measured_fp64_tflops": probe.get("fp64_tflops")}


def roofline_for(kernel, ms, band_nodes, peaks, kernel_sha, probe):
    """Algorithmic work per launch of the dominant kernel over its measured
    duration. Per band node and step (FP32):
      bytes: read u_j, d_j, the band-list entry, write u_j and the new band
             entry = 20 B (SURVEY's 19-22 B); 12 B on the whole grid (read u_j,
             d_j, write u_j). HBM bound for Q1.
      flops: WENO_FLOPS_SURVEY per node (ALU bound), the kernel's own
             WENO_FLOPS_EXECUTED beside it.
    Energy kernel: per front cell 305 WENO evaluations + 125 trilinear
    d-lookups, reported when it dominates (flops, ALU bound).
    The ALU peak is the measured FP32 FMA rate (slr_probe_fma) when the probe
    ran, else the derived one."""
    ap = alu_peaks(peaks, probe)
    fp32_peak = ap["measured_tflops"] or ap["derived_tflops"]
    peak_src = ("measured: slr_probe_fma (8 FMA chains x 256 threads x 8 blocks per SM)" if ap["measured_tflops"]
                else "derived: " + ap["derived_from"])
    info = {}
    traffic = None
    side = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(side):
        try:
            tr = json.load(open(side))
            if tr.get("src_sha") == kernel_sha and tr.get("kernel") == kernel["name"]:
                traffic = tr.get("dram_bytes_per_launch")
        except (OSError, ValueError):
            traffic = None
    bpn = kernel.get("bytes_per_node", 20.0)
    hbm = bpn * band_nodes / (ms * 1e-3) / 1e9
    if kernel["kind"] == "step_weno":
        achieved = WENO_FLOPS_SURVEY * band_nodes / (ms * 1e-3) / 1e12
        executed = WENO_FLOPS_EXECUTED * band_nodes / (ms * 1e-3) / 1e12
        info = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic, "peak_source": peak_src,
                "flops_per_node": WENO_FLOPS_SURVEY,
                "executed_view": {"flops_per_node": WENO_FLOPS_EXECUTED, "achieved_tflops": executed,
                                  "frac": executed / fp32_peak},
                "alu_peaks": ap,
                "hbm_view": {"bytes_per_node": bpn, "achieved_gbs": hbm, "peak_gbs": peaks["hbm_gbs"],
                             "frac": hbm / peaks["hbm_gbs"]}}
    elif kernel["kind"] == "step_q1":
        info = {"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s", "bytes_per_node": bpn,
                "frac": hbm / peaks["hbm_gbs"], "traffic": traffic, "peak_source": "measured (MEASURED_PEAKS)"}
    else:
        fc = kernel.get("front_cells", 0)
        flops = (305 * 24 + 125 * 20) * fc
        achieved = flops / (ms * 1e-3) / 1e12
        info = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic, "peak_source": peak_src, "alu_peaks": ap}
    info["kernel"] = kernel["name"]
    info["ms_per_launch"] = ms
    return info


def device_peaks(torch):
    """HBM and bf16 peaks from MEASURED_PEAKS.json, the SM count from the
    device and its maximum SM clock (MEASURED_PEAKS, else nvidia-smi)."""
    peaks = {"hbm_gbs": 6794.5, "bf16_tflops": 1921.5, "sm_max_mhz": None}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks.update({k: v for k, v in json.load(open(pk)).items() if isinstance(v, (int, float))})
    peaks["sms"] = int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    if not peaks.get("sm_max_mhz"):
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()), "--query-gpu=clocks.max.sm",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20).stdout
            peaks["sm_max_mhz"] = float(out.strip().splitlines()[0])
        except (OSError, ValueError, IndexError, subprocess.SubprocessError):
            peaks["sm_max_mhz"] = 2070.0
    return peaks


def fma_probe(slr):
    """FP32 and FP64 FMA rates of this device (slr_probe_fma); None on failure."""
    out = {}
    for prec, key in ((32, "fp32_tflops"), (64, "fp64_tflops")):
        try:
            out[key], out[key.replace("tflops", "ms")] = slr.slr_probe_fma(prec)
        except slr.SlrError:
            out[key] = None
    return out


def measure_steps(rec, steps, warmup, flush_buf, torch, profiled=False):
    """Warm-up, then `steps` timed iterations; returns per-step ms, per-phase
    ms (step kernel, front-cell + energy kernels, record kernel; profiled
    runs only: the iteration graph then also records an event between the
    kernels) and the band sizes of the timed steps."""
    rec.set_profiling(profiled)
    st = rec.stream
    for _ in range(warmup):
        rec.step_async(1)
    torch.cuda.synchronize()
    n0 = rec.diagnostics()["iters"]
    step_ms, kern_ms = [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    launches0 = rec.kernel_launches
    for _ in range(steps):
        with torch.cuda.stream(st):
            flush_buf.zero_()  # L2 flush between timed steps, outside the events
        ev0.record(st)
        rec.step_async(1)
        ev1.record(st)
        if profiled:
            kern_ms.append(rec.last_iteration_times())  # synchronises the stream
        else:
            ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
    launches = rec.kernel_launches - launches0
    diag = rec.diagnostics()
    bands = diag["band"][n0:n0 + steps]
    return step_ms, kern_ms, bands, launches


def record_step(rec, label, n, prec, interp, band, seed=11, nodes=2000):
    """The inputs and outputs of one GPU step for the per-result error against
    the FP64 oracle: φ^n and d as stored, E_p of φ^n (given to both sides),
    and φ^{n+1} on a seeded sample of band nodes (any nodes on the whole
    grid). The comparison itself runs in the cpu_baseline leg."""
    u0 = rec.u()
    d = rec.d()
    Ep = float(rec.energy(2.0)[0])
    rec.step(1, energy_override=Ep)
    u1 = rec.u()
    dt = np.float32 if prec == 32 else np.float64
    g = np.float32(6.0 * 2.0 / (n - 1)) if prec == 32 else 6.0 * 2.0 / (n - 1)
    pool = np.flatnonzero(np.abs(u0.astype(dt)) < g) if band else np.arange(u0.size)
    rng = np.random.default_rng(seed)
    sample = np.sort(rng.choice(pool, min(nodes, pool.size), replace=False))
    return {"label": label, "n": n, "prec": prec, "interp": interp, "band": band, "u0": u0.astype(dt),
            "d": d.astype(dt), "Ep": Ep, "sample": sample, "u1": u1[sample]}


def run_gpu(args):
    import torch

    from paper_2410_22205_gb300 import slr

    dist = Dist("nccl")
    torch.cuda.set_device(dist.local_rank)
    peaks = device_peaks(torch)
    probe = fma_probe(slr)
    t_setup = time.time()
    grid, cloud = workload(args)
    cloud_s = time.time() - t_setup
    n = args.n
    interp = 1 if args.interp == "weno" else 0
    band = 0 if args.fullgrid else 1
    prec = args.precision
    rec = slr.Reconstruction(dim=3, n=n, precision=prec, interp=interp, band=band, reinit=int(args.reinit),
                             **cfg_kw())
    st = rec.stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    rec.load_cloud(cloud)
    ev[0].record(st)
    rec.build_distance()
    ev[1].record(st)
    rec.init_sphere(0.9)
    ev[2].record(st)
    ev[2].synchronize()
    dist_ms = ev[0].elapsed_time(ev[1])
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    # the timed steps: the iteration graph without profiling event nodes
    # (they add ~17 us per step)
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dist.local_rank)
    clocks.start()
    step_ms, _, bands, launches = measure_steps(rec, args.steps, args.warmup, flush, torch)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    # the per-kernel durations of the roofline: further steps of the same
    # job with an event recorded between the kernels inside the graph
    kprof = max(3, min(args.steps, 50))
    pstep_ms, kern_ms, _, _ = measure_steps(rec, kprof, 2, flush, torch, profiled=True)

    units = float(np.sum(bands))
    secs = float(np.sum(step_ms)) / 1e3
    value, tot_units, tmax = aggregate(units, secs, dist)
    ms_per_step = tmax * 1e3 / args.steps
    kern = np.array(kern_ms)
    tname = "float" if prec == 32 else "double"
    iname = "WENO" if interp else "Q1"
    # the list step runs with the reinitialisation (its band can leave the bricks of the initial band) and,
    # by the library's rule, for a band run with Q1 on rows that TMA cannot stage; the bricks otherwise
    try:
        brick_info = rec.brick_shape()
    except slr.SlrError:
        brick_info = None
    step_name = (f"k_step_brick<{tname},{iname},{'band' if band else 'whole grid'}>" if brick_info else
                 f"k_step_band<{tname},3,{iname}>")
    names = [step_name,
             f"k_energy<{tname},3,{iname},R=5> (front cells + quadrature)", "k_record"]
    kmean = kern.mean(axis=0)
    dom = int(np.argmax(kmean[:2]))  # the step or the energy pass (the record kernel is a small reduction)
    mean_band = float(np.mean(bands))
    front = 1.5 * 4 * math.pi * 0.81 / ((2.0 / (n - 1)) ** 2)
    kernel = {"name": names[dom], "kind": [("step_weno" if interp else "step_q1"), "energy"][dom],
              "front_cells": front, "bytes_per_node": 20.0 if band else 12.0}
    sha = sha_of_kernel(names[dom])
    roof = roofline_for(kernel, float(kmean[dom]), mean_band, peaks, sha, probe)
    roof["kernel_share_of_step"] = float(kmean[dom] / np.mean(pstep_ms))
    roof["kernels_ms"] = {nm: float(v) for nm, v in zip(names, kmean)}
    roof["kernels_timed"] = (f"{kprof} further steps with an event between the kernels captured in the graph "
                             f"({float(np.mean(pstep_ms)):.4f} ms per step with the events)")
    if brick_info:
        bt, bs, bms = brick_info
        roof["launch_shape"] = {"threads_per_block": bt, "stages": bs, "autotune_trial_ms": bms,
                                "chosen_by": "the brick step's autotuner at init (fastest of 4 shapes on φ^0)"}
    iter_lat = {"p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99))}
    if args.reinit:
        roof["phases_ms"] = {k: float(v) for k, v in
                             zip(("step", "reinit", "energy", "record"), rec.last_iteration_phases())}
    records = []
    want_err = not args.no_cpu_baseline and dist.rank == 0 and dist.world == 1 and not args.reinit
    if want_err:
        records.append(record_step(rec, "headline", n, prec, interp, band))
    rec.close()
    phase_s = {"cloud_generation": cloud_s, "setup_and_timed_steps": time.time() - t_setup - cloud_s}
    t_ph = time.time()

    variants = {}
    if not args.no_variants and dist.rank == 0:
        for prec, interp, band, rei, label in ((32, 0, 1, 0, "q1_fp32_band"), (64, 1, 1, 0, "weno_fp64_band"),
                                               (64, 0, 1, 0, "q1_fp64_band"), (32, 1, 0, 0, "weno_fp32_fullgrid"),
                                               (32, 0, 0, 0, "q1_fp32_fullgrid"),
                                               (32, 1, 1, 1, "weno_fp32_band_reinit"),
                                               (32, 0, 1, 1, "q1_fp32_band_reinit")):
            r2 = slr.Reconstruction(dim=3, n=n, precision=prec, interp=interp, band=band, reinit=rei, **cfg_kw())
            r2.load_cloud(cloud)
            r2.build_distance()
            r2.init_sphere(0.9)
            ks = max(3, min(args.steps // 4, 50))
            sm, _, bd, _ = measure_steps(r2, ks, 2, flush, torch)
            _, km, _, _ = measure_steps(r2, ks, 1, flush, torch, profiled=True)
            variants[label] = {"value": float(np.sum(bd)) / (float(np.sum(sm)) / 1e3), "ms_per_step": float(np.mean(sm)),
                               "nodes_per_step": float(np.mean(bd)), "kernels_ms": [float(x) for x in np.mean(km, 0)]}
            if rei:
                variants[label]["phases_ms"] = {k: float(v) for k, v in
                                                zip(("step", "reinit", "energy", "record"), r2.last_iteration_phases())}
            try:
                bt, bs, bms = r2.brick_shape()
                variants[label]["launch_shape"] = {"threads_per_block": bt, "stages": bs}
            except slr.SlrError:
                variants[label]["step"] = "list step (k_step_band)"
            if want_err and not rei:
                records.append(record_step(r2, label, n, prec, interp, band))
            r2.close()
    phase_s["variants"] = time.time() - t_ph
    t_ph = time.time()

    e2e = e2e_alg1 = e2e_runs = None
    solve_lat = None
    if args.e2e_jobs > 0:
        e2e, solve_lat = run_e2e(args, cloud, slr, torch)
        e2e_alg1, _ = run_e2e(args, cloud, slr, torch, reinit=1)
        e2e_runs = run_multirun(args, cloud, slr, torch)
    phase_s["e2e"] = time.time() - t_ph
    t_ph = time.time()

    batched = serving = None
    if dist.rank == 0 and args.batch_jobs > 0:
        batched = run_batched(args, slr, torch)
    phase_s["batched"] = time.time() - t_ph
    t_ph = time.time()
    if dist.rank == 0 and args.serve_seconds > 0:
        serving = run_serving(args, slr, torch)
    phase_s["serving"] = time.time() - t_ph
    t_ph = time.time()

    cpu = None
    errors = {}
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(grid, cloud, budget_s=20.0, records=records)
        errors = cpu.get("error_vs_oracle", {})
        for lab, e in errors.items():
            if lab in variants:
                variants[lab]["error_vs_oracle"] = e
    phase_s["cpu_baseline"] = time.time() - t_ph

    if dist.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": f"f{prec}", "data": "synthetic (seeded superquadric-union cloud)",
            "config": {"workload": f"sq3union{args.points // 1000}k_{n}cube_{'band6h' if band else 'fullgrid'}"
                                   f"_{args.interp}_fp{prec}" + ("_reinit" if args.reinit else ""),
                       "grid": f"{n}^3", "reinit": bool(args.reinit),
                       "points": args.points, "interp": iname, "band": "6h" if band else "off (whole grid)",
                       "p": 2, "delta": 1,
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{dist.world}",
                       "units_all_ranks": tot_units, "distance_grid_ms": dist_ms},
            "error_vs_oracle": errors.get("headline"),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "e2e_algorithm1_reinit": e2e_alg1,
            "e2e_paper_pipeline": e2e_runs,
            "latency": {"iteration": iter_lat, "solve": solve_lat},
            "variants": variants, "batched": batched, "serving": serving, "gpu_launches": int(launches), "clocks": clk,
            "setup_s": time.time() - t_setup, "phase_s": phase_s,
        }
        print(json.dumps(line), flush=True)
    dist.close()


def run_e2e(args, cloud, slr, torch, reinit=0):
    """Whole jobs through the public API with host buffers: pinned host cloud
    -> load (H2D) -> exact distance grid -> φ^0 -> evolve to the stop test ->
    extract |φ| < 2h (D2H). Timed by the host clock around each job. With
    reinit = 1 every iteration also runs the reinitialisation of Algorithm 1 (§3.7), so the
    band follows the front; the error on the cloud (eq. errCloud) of the
    result is reported next to the rate."""
    pinned = torch.empty(cloud.shape, dtype=torch.float64, pin_memory=True)
    pinned.numpy()[:] = cloud
    host = pinned.numpy()
    h = 2.0 / (args.n - 1)
    times, units, h2d, d2h, iters = [], 0.0, 0, 0, []
    for j in range(args.e2e_jobs + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # Algorithm 1 with the reinitialisation runs the paper's first-run parameters (p = 1,
        # δ = 0: the front moves Δt|∇d| = h/4 per step towards the cloud)
        # and may need more than 100 iterations to cross the gap at 256^3
        kw = dict(p=1.0, delta=0.0, max_iters=400) if reinit else cfg_kw()
        rec = slr.Reconstruction(dim=3, n=args.n, precision=32, interp=1, band=1, reinit=reinit, **kw)
        rec.load_cloud(host)
        rec.build_distance()
        rec.init_sphere(0.9)
        it, conv = rec.evolve()
        idx, val = rec.extract(2 * h)
        t1 = time.perf_counter()
        diag = rec.diagnostics(err_cloud=True)
        rec.close()
        if j == 0:
            continue  # first job warms the allocator and the graph instantiation path
        times.append(t1 - t0)
        err_s = diag["err_cloud"]
        units += float(np.sum(diag["band"]))
        h2d += host.nbytes
        d2h += idx.nbytes + val.nbytes
        iters.append(it)
    jobs = len(times)
    e2e = {"value": units / sum(times), "unit": UNIT, "h2d_bytes_per_step": h2d // jobs, "d2h_bytes_per_step": d2h // jobs,
           "step": "one whole job (H2D cloud, distance grid, init, evolve to the stop test, extract, D2H)"
                   + (", Algorithm 1 with the reinitialisation of §3.7 every iteration, p = 1, δ = 0 (the paper's first "
                      "run)" if reinit else ""),
           "jobs": jobs, "iterations_per_job": iters, "err_cloud_over_h": err_s / h}
    lat = {"p50_ms": 1e3 * float(np.percentile(times, 50)), "p99_ms": 1e3 * float(np.percentile(times, 99)), "jobs": jobs}
    return e2e, lat


def run_multirun(args, cloud, slr, torch):
    """The paper's whole pipeline through slr_reconstruct (§4): h_S from a
    10% sample, the §3.6 initial data, then three runs of Algorithm 1 with the
    reinitialisation, (p, δ) = (1, 0), (2, 0), (2, 1), from a pinned host
    cloud to the extracted level set. The node budget of one run is the bench
    grid's (n^3), so the runs are coarsened to about that size. Reported per
    whole reconstruction, with the per-run table of the paper (grid, E_2,
    Err_S), and once with the §3.4 swept distance grid."""
    pinned = torch.empty(cloud.shape, dtype=torch.float64, pin_memory=True)
    pinned.numpy()[:] = cloud
    host = pinned.numpy()
    out = {}
    u_last = None
    for distance in ("exact", "fsm"):
        times, reps, d2h = [], [], 0
        jobs = max(1, min(2, args.e2e_jobs)) if distance == "exact" else 1
        for j in range(jobs + (1 if distance == "exact" else 0)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rec, rep = slr.reconstruct(host, dim=3, precision=32, interp=1, runs=3, K_s=2.0, sample_frac=0.1, seed=1,
                                       max_nodes=args.n ** 3, max_iters=100, distance=distance)
            idx, val = rec.extract(2 * rep["run_dx"][-1])
            t1 = time.perf_counter()
            if distance == "exact":
                u_last = rec.u()
            rec.close()
            if distance == "exact" and j == 0:
                continue
            times.append(t1 - t0)
            reps.append(rep)
            d2h = idx.nbytes + val.nbytes
        rep = reps[-1]
        iters = [int(x) for x in rep["run_iters"]]
        out[distance] = {
            "reconstructions_per_s": len(times) / sum(times), "seconds_per_reconstruction": sum(times) / len(times),
            "h2d_bytes_per_step": int(host.nbytes), "d2h_bytes_per_step": int(d2h), "h_s": rep["h_s"],
            "coarsened": rep["coarsened"],
            "runs": [{"grid": list(rep["run_n"][r]), "dx": rep["run_dx"][r], "iters": iters[r],
                      "converged": rep["run_converged"][r], "E2": rep["run_energy"][r],
                      "err_cloud_over_dx": rep["run_err_cloud"][r] / rep["run_dx"][r]} for r in range(len(iters))],
        }
    out["step"] = ("one whole reconstruction from the host cloud: sample and h_S, three runs (distance grid, φ^0, "
                   "Algorithm 1 with §3.7 to the stop test), extract |φ| < 2Δx, D2H")
    # the same reconstruction in FP64 on the GPU: how far the FP32 result is
    # from it near the front (the measurement behind keeping d in FP32)
    rec64, rep64 = slr.reconstruct(host, dim=3, precision=64, interp=1, runs=3, K_s=2.0, sample_frac=0.1, seed=1,
                                   max_nodes=args.n ** 3, max_iters=100, distance="exact")
    u64 = rec64.u()
    rec64.close()
    rep32 = out["exact"]
    dx = rep64["run_dx"][-1]
    same_grid = u_last is not None and u_last.size == u64.size
    near = np.abs(u64) < 2 * dx
    out["fp32_vs_fp64"] = {
        "same_iterations": [int(x) for x in rep64["run_iters"]] == [r["iters"] for r in rep32["runs"]],
        "iterations_fp64": [int(x) for x in rep64["run_iters"]],
        "max_abs_diff_within_2dx_over_dx": float(np.abs(u_last - u64)[near].max() / dx) if same_grid else None,
        "nodes_within_2dx": int(near.sum()),
        "err_cloud_over_dx_fp64": rep64["run_err_cloud"][-1] / dx,
        "err_cloud_over_dx_fp32": rep32["runs"][-1]["err_cloud_over_dx"],
        "how": "the exact-distance pipeline run again in FP64 on the GPU; φ compared where |φ_64| < 2Δx"}
    return out


# ---------------------------------------------------------------------------
# batched and served forms
# ---------------------------------------------------------------------------

def _job_cfg(slr, job, **kw):
    g = job["grid"]
    n = tuple(g.n[: g.dim]) + ((1,) if g.dim == 2 else ())
    return slr.slr_config_default(dim=g.dim, n=n, lo=g.lo[: g.dim], hi=g.hi[: g.dim], precision=job.get("precision", 32),
                                  interp=job["interp"], band=job.get("band", 1), **kw)


def _run_job(slr, job, stream=None):
    """One whole reconstruction through the public API; returns (rec, iters)."""
    g = job["grid"]
    n = tuple(g.n[: g.dim]) + ((1,) if g.dim == 2 else ())
    rec = slr.Reconstruction(dim=g.dim, n=n, lo=g.lo[: g.dim], hi=g.hi[: g.dim], precision=job.get("precision", 32),
                             interp=job["interp"], band=job.get("band", 1), stream=stream)
    rec.load_cloud(job["cloud"])
    rec.build_distance()
    rec.init_sphere(job.get("u0_radius", 0.9))
    return rec


def run_batched(args, slr, torch):
    """The 64-job mix (half 2-D, half 3-D, Q1/WENO mixed, FP32): whole jobs
    one after another versus all jobs set up on their own streams from a
    thread pool and evolved together by slr_batch_evolve (one graph launch
    advances every job by 8 iterations; the autotuned chunk costs more in
    graph instantiation than it saves on a batch this short). Reconstructions
    per second over the whole job (distance grid, φ^0, evolve to the stop
    test, extract)."""
    import concurrent.futures as cf

    t0 = time.time()
    jobs = synth.batch_mix(seed=3, n_jobs=args.batch_jobs)
    gen_s = time.time() - t0
    h_of = lambda j: (j["grid"].hi[0] - j["grid"].lo[0]) / (j["grid"].n[0] - 1)
    # one job at a time
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_iters, seq_state = [], []
    for j in jobs:
        rec = _run_job(slr, j)
        it, _ = rec.evolve()
        idx, val = rec.extract(2 * h_of(j))
        seq_iters.append(it)
        seq_state.append((idx.size, float(val.sum())))
        rec.close()
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    # batched: set-up overlapped on per-job streams, one batched evolve
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(8) as ex:
        recs = list(ex.map(lambda j: _run_job(slr, j, stream=torch.cuda.Stream()), jobs))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    its, _ = slr.slr_batch_evolve([r.ctx for r in recs], chunk=8)
    chunk = slr.slr_batch_chunk(recs[0].ctx)
    t_evolve = time.perf_counter() - t0 - t_setup
    bat_state = []
    for j, r in zip(jobs, recs):
        idx, val = r.extract(2 * h_of(j))
        bat_state.append((idx.size, float(val.sum())))
    torch.cuda.synchronize()
    t_bat = time.perf_counter() - t0
    for r in recs:
        r.close()
    same = its == seq_iters and bat_state == seq_state
    # persistent: the same set-up, then one persistent graph-captured kernel
    # advances every job (slr_batch_run, block size autotuned)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(8) as ex:
        recs = list(ex.map(lambda j: _run_job(slr, j, stream=torch.cuda.Stream()), jobs))
    torch.cuda.synchronize()
    t_psetup = time.perf_counter() - t0
    pits, _ = slr.slr_batch_run([r.ctx for r in recs], autotune=True)
    shape = slr.slr_batch_run_info(recs[0].ctx)
    t_pevolve = time.perf_counter() - t0 - t_psetup
    per_state = []
    for j, r in zip(jobs, recs):
        idx, val = r.extract(2 * h_of(j))
        per_state.append((idx.size, float(val.sum())))
    torch.cuda.synchronize()
    t_per = time.perf_counter() - t0
    for r in recs:
        r.close()
    psame = pits == seq_iters and per_state == seq_state
    return {"jobs": len(jobs), "workload": "batch mix: 32 2-D (64^2-512^2) + 32 3-D (64^3-192^3), 1k-200k points, "
                                            "Q1/WENO mixed, FP32, band",
            "one_at_a_time": {"reconstructions_per_s": len(jobs) / t_seq, "seconds": t_seq},
            "batched": {"reconstructions_per_s": len(jobs) / t_bat, "seconds": t_bat, "setup_s": t_setup,
                        "evolve_s": t_evolve, "chunk": chunk},
            "persistent": {"reconstructions_per_s": len(jobs) / t_per, "seconds": t_per, "setup_s": t_psetup,
                           "evolve_s": t_pevolve, "launch_shape": shape, "identical_results": bool(psame)},
            "speedup": t_seq / t_bat, "speedup_persistent": t_seq / t_per, "identical_results": bool(same),
            "iterations": its,
            "input_generation_s": gen_s}


def run_serving(args, slr, torch):
    """Continuous batching: requests of 3-D WENO FP32 reconstructions (grids
    log-uniform 64^3-256^3, clouds log-uniform 5k-2M points on superquadric
    unions, drawn from a pool of pre-generated clouds) are submitted to the
    server. A burst first measures its capacity (one setup thread); then the
    same Poisson stream at 0.8 x that capacity (same seed, same arrivals) runs
    for --serve-seconds with one, two and four setup threads, whose set-ups
    (context, distance grid, φ^0) overlap each other and the iterations. Per
    stream: p50/p99 submit-to-finish latency, its split into queue, setup and
    iteration time, and reconstructions per second."""
    pool_sizes = [int(round(math.exp(x))) for x in np.linspace(math.log(5000), math.log(2_000_000), 6)]
    t0 = time.time()
    pool = [synth.superquadric_union_cloud(nn, 3, 100 + i) for i, nn in enumerate(pool_sizes)]
    gen_s = time.time() - t0

    def draws(seed, count):
        rng = np.random.default_rng(seed)
        out = []
        for _ in range(count):
            n = int(round(math.exp(rng.uniform(math.log(64), math.log(256)))))
            out.append((n, int(rng.integers(0, len(pool))), float(rng.exponential(1.0))))
        return out

    def cfg_of(n):
        return slr.slr_config_default(dim=3, n=(n, n, n), lo=(-1.0,) * 3, hi=(1.0,) * 3, precision=32, interp=1,
                                      band=1)

    def serve(setup_threads, reqs, lam, policy=0):
        """Submit reqs (lam None: all at once) and wait for all; returns the
        finished jobs' (latency, queue, setup, iterate) in ms and the span."""
        srv = slr.slr_server_create(96 << 30, max_active=16, setup_threads=setup_threads, policy=policy)
        done, pending = [], {}
        try:
            t_start = time.perf_counter()
            t_next = t_start
            k = 0
            deadline = t_start + (args.serve_seconds if lam else 600.0)
            while (k < len(reqs) and time.perf_counter() < deadline) or pending:
                now = time.perf_counter()
                while k < len(reqs) and now < deadline and (lam is None or now >= t_next):
                    n, ci, ex = reqs[k]
                    pending[slr.slr_server_submit(srv, cfg_of(n), pool[ci], (0.0, 0.0, 0.0, 0.9))] = k
                    k += 1
                    if lam:
                        t_next += ex / lam
                    now = time.perf_counter()
                for t in list(pending):
                    st, _, lat = slr.slr_server_poll(srv, t)
                    if st == 2:
                        q, su, it = slr.slr_server_timing(srv, t)
                        done.append((lat, q, su, it))
                        slr.slr_server_release(srv, t)
                        del pending[t]
                if time.perf_counter() > deadline + 300:
                    break
                time.sleep(0.001)
            span = (time.perf_counter() - t_start) if lam is None else args.serve_seconds
        finally:
            slr.slr_server_destroy(srv)
        return np.array(done).reshape(-1, 4), span, k

    def pct(x):
        return {"p50": float(np.percentile(x, 50)), "p99": float(np.percentile(x, 99))} if len(x) else None

    burst = draws(4, 24)
    res_b, span_b, _ = serve(1, burst, None)
    cap = len(res_b) / span_b
    lam = 0.8 * cap
    stream = draws(5, int(lam * args.serve_seconds * 2) + 16)
    out = {"workload": "3-D WENO FP32, grids 64^3-256^3, clouds 5k-2M points (superquadric unions)",
           "capacity_burst_per_s": cap, "capacity_setup_threads": 1, "lambda_per_s": lam, "max_active": 16,
           "cloud_pool_generation_s": gen_s}
    # the same arrivals: first come first served with 1, 2 and 4 setup
    # threads, and the least-estimated-set-up-first admission with 1
    settings = [(1, 0), (2, 0), (4, 0), (1, 1)]
    key = lambda th, pol: f"setup_threads_{th}" + ("_shortest_first" if pol else "")
    for th, pol in settings:
        res, span, submitted = serve(th, stream, lam, pol)
        out[key(th, pol)] = {
            "policy": "least estimated set-up first (aged)" if pol else "first come first served",
            "submitted": submitted, "completed": int(len(res)), "reconstructions_per_s": len(res) / span,
            "latency_ms": pct(res[:, 0]), "queue_ms": pct(res[:, 1]), "setup_ms": pct(res[:, 2]),
            "iterate_ms": pct(res[:, 3])}
    best = min(settings, key=lambda tp: out[key(*tp)]["latency_ms"]["p99"])
    out["best_by_p99"] = key(*best)
    out["reconstructions_per_s"] = out[key(*best)]["reconstructions_per_s"]
    out["latency_ms"] = out[key(*best)]["latency_ms"]
    return out


# ---------------------------------------------------------------------------
# CPU: the oracle
# ---------------------------------------------------------------------------

def oracle_setup(grid, cloud):
    """φ^0 (sphere r = 0.9, cut) and d by the oracle's exact k-d tree search on
    the nodes the first iterations read: the band and its 26-neighbourhood."""
    import oracle as O

    P = O.params_for_grid(grid, interp=1, band=1, p=2.0, delta=1.0, prec=32)
    u = synth.sphere_sdf(grid, 0.9).astype(np.float32).astype(np.float64)
    u = O.cut(P, u)
    n = grid.n[0]
    inb = (np.abs(u) < np.float32(P.gamma)).reshape(n, n, n)
    need = inb.copy()
    for ax in range(3):
        for s in (-1, 1):
            need |= np.roll(inb, s, axis=ax)
    nodes = np.flatnonzero(need.reshape(-1))
    d = np.zeros(grid.num_nodes)
    dd, _ = O.distance(P, cloud, nodes, method="kd")
    d[nodes] = dd.astype(np.float32).astype(np.float64)
    return O, P, u, d


def oracle_iteration(O, P, u, d, Ep):
    out, _, _ = O.sl_step(P, u, d, Ep)
    E = O.energy(P, out, d, 2.0)["E"]
    nb = int(np.count_nonzero(np.abs(u) < np.float32(P.gamma)))
    return out, E, nb


def oracle_errors(O, records):
    """Per result: max |u_gpu - u_oracle| over the recorded sample of one step
    from identical inputs (φ^n and d as the GPU stores them, the same E_p),
    in units of h, beside the bar of the parity tests (1e-5 h in FP32, with 4
    units in the last place where the FP32 value is large enough for that to
    exceed it; 1e-12 in FP64). Nodes the oracle flags within 1e-6 of the
    singular-gradient threshold are excluded and counted."""
    out = {}
    for r in records:
        n = r["n"]
        P = O.params(3, (n,) * 3, (-1.0,) * 3, (1.0,) * 3, interp=r["interp"], band=r["band"], prec=r["prec"],
                     p=2.0, delta=1.0)
        ref, flags = O.sl_nodes(P, r["u0"], r["d"], r["Ep"], r["sample"])
        if r["band"]:
            g = np.float32(P.gamma) if r["prec"] == 32 else P.gamma
            ref = np.clip(ref, -g, g)
        ok = (flags & O.FLAG_MARGIN) == 0
        err = np.abs(r["u1"] - ref)[ok]
        if r["prec"] == 32:
            bar = np.maximum(1e-5 * P.h, 4.0 * np.spacing(np.abs(ref[ok]).astype(np.float32)).astype(np.float64))
        else:
            bar = np.full(err.size, 1e-12)
        out[r["label"]] = {"max_abs_over_h": float(err.max() / P.h) if err.size else 0.0,
                           "bar_over_h": (1e-5 if r["prec"] == 32 else 1e-12 / P.h),
                           "within_bar": bool((err <= bar).all()), "nodes": int(err.size),
                           "excluded_near_singular_threshold": int((~ok).sum()),
                           "how": "one GPU step from identical inputs vs the FP64 oracle on seeded sampled nodes"}
    return out


def cpu_baseline(grid, cloud, budget_s=20.0, records=()):
    """The oracle as it stands on the host cores: whole iterations (band scan,
    WENO SL step in FP64 on every band node, cut, energy) from φ^0 until about
    budget_s seconds of work. It also compares the recorded GPU steps with the
    oracle (oracle_errors)."""
    O, P, u, d = oracle_setup(grid, cloud)
    cores = O.set_threads(len(os.sched_getaffinity(0)))
    Ep = O.energy(P, u, d, 2.0)["E"]
    t0 = time.perf_counter()
    units, its = 0, 0
    while True:
        u, Ep, nb = oracle_iteration(O, P, u, d, Ep)
        units += nb
        its += 1
        if time.perf_counter() - t0 > budget_s * 0.5 or its >= 3:
            break
    dt = time.perf_counter() - t0
    out = {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{its} whole oracle iterations (WENO FP64 SL step on {units // its} band nodes + energy) of the "
                     f"{grid.n[0]}^3 workload from φ^0, {dt:.1f} s"}
    out["detail"] = oracle_detail(O, P, u, d, cloud, cores)
    if records:
        out["error_vs_oracle"] = oracle_errors(O, records)
    return out


def cpu_model():
    """The host CPU's name as lscpu, /proc/cpuinfo or the platform gives it."""
    import platform
    import subprocess

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "hardware", "cpu model"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_detail(O, P, u, d, cloud, cores):
    """The oracle's rates on 1 thread and on every core: the SL step (node
    updates/s) of the bench's WENO band, of the 128^3 torus band (Q1 and WENO)
    and of the 64^2 circle (whole grid, FP64 Q1), and the exact distance grid
    (nodes/s, k-d tree). Each a bounded sample of a second or so."""
    rng = np.random.default_rng(0)
    res = {"cpu_model": cpu_model(), "affinity_cores": len(os.sched_getaffinity(0))}

    def rate(fn, units, threads):
        O.set_threads(threads)
        t0 = time.perf_counter()
        fn()
        return units / (time.perf_counter() - t0)

    band = np.flatnonzero(np.abs(u) < np.float32(P.gamma))
    Ep = O.energy(P, u, d, 2.0)["E"]
    s1, sa = rng.choice(band, 4000, replace=False), rng.choice(band, 60000, replace=False)
    nc = int(P.n[0])
    res[f"sl_weno_fp64_{nc}cube"] = {
        "1_thread": rate(lambda: O.sl_nodes(P, u, d, Ep, s1), s1.size, 1),
        "all_cores": rate(lambda: O.sl_nodes(P, u, d, Ep, sa), sa.size, cores)}
    nodes = rng.choice(P.n[0] * P.n[1] * P.n[2], 20000, replace=False)
    res[f"distance_grid_kd_{nc}cube_{len(cloud) // 1000}k_points"] = {
        "1_thread": rate(lambda: O.distance(P, cloud, nodes[:2000], method="kd"), 2000, 1),
        "all_cores": rate(lambda: O.distance(P, cloud, nodes, method="kd"), nodes.size, cores)}
    # the 128^3 torus workload
    g2 = synth.cube_grid(3, 128)
    torus = synth.torus_cloud(20000, 0.5, 0.2, 0.002, 1)
    for interp, name in ((0, "q1"), (1, "weno")):
        P2 = O.params_for_grid(g2, interp=interp, band=1, p=2.0, delta=1.0, prec=64)
        u2 = O.cut(P2, synth.sphere_sdf(g2, 0.9))
        b2 = np.flatnonzero(np.abs(u2) < P2.gamma)
        smp = rng.choice(b2, 20000, replace=False)
        d2 = np.zeros(g2.num_nodes)
        near = np.unique(np.concatenate([smp + o for o in (0, -1, 1, -128, 128, -128 * 128, 128 * 128)]))
        d2[near] = O.distance(P2, torus, near, method="kd")[0]
        res[f"sl_{name}_fp64_torus_128cube"] = {
            "1_thread": rate(lambda: O.sl_nodes(P2, u2, d2, 0.5, smp[:4000]), 4000, 1),
            "all_cores": rate(lambda: O.sl_nodes(P2, u2, d2, 0.5, smp), smp.size, cores)}
    # the 64^2 circle workload, whole grid
    g1 = synth.cube_grid(2, 64)
    P1 = O.params_for_grid(g1, interp=0, band=0, prec=64)
    circ = synth.circle_noisy(200, 0.5, 0.005, 0)
    d1, _ = O.distance(P1, circ, method="kd")
    u1 = synth.sphere_sdf(g1, 0.9)
    res["sl_q1_fp64_circle_64sq_whole_grid"] = {
        "1_thread": rate(lambda: [O.sl_step(P1, u1, d1, 0.5) for _ in range(20)], 20 * g1.num_nodes, 1),
        "all_cores": rate(lambda: [O.sl_step(P1, u1, d1, 0.5) for _ in range(20)], 20 * g1.num_nodes, cores)}
    O.set_threads(cores)
    res["unit"] = "node-updates/s (SL step), nodes/s (distance grid)"
    return res


def run_reference(args):
    """--impl reference: the oracle, as it stands, on the host cores, on the
    same workload; each step is one whole oracle iteration."""
    dist = Dist("gloo")
    if dist.rank != 0:
        dist.barrier()
        dist.close()
        return
    grid, cloud = workload(args)
    O, P, u, d = oracle_setup(grid, cloud)
    cores = O.set_threads(len(os.sched_getaffinity(0)))
    Ep = O.energy(P, u, d, 2.0)["E"]
    for _ in range(args.warmup):
        u, Ep, _ = oracle_iteration(O, P, u, d, Ep)
    times, units = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u, Ep, nb = oracle_iteration(O, P, u, d, Ep)
        times.append(time.perf_counter() - t0)
        units += nb
    secs = sum(times)
    value = units / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded superquadric-union cloud)",
            "config": {"workload": f"sq3union{args.points // 1000}k_{args.n}cube_band6h_weno_fp32", "grid": f"{args.n}^3",
                       "points": args.points, "interp": "WENO", "band": "6h",
                       "note": "FP64 oracle on the host; its inputs are the FP32-rounded φ^0 and d"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed whole oracle iterations after {args.warmup} warm-up"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    dist.barrier()
    dist.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
