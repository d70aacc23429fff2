"""Benchmark: wave-LB GLUPS and radiation forces/s on one GB300.

Default line (--workload sphere512): the 512^3 force-vs-position workload of
Sec. VII (F proportional to sin 2kz): 512^3 D3Q7, FP32 populations,
lambda = 256, R = 24, kappa~ = 0.5, 4096 Fibonacci points, 30 periods (30720
LB steps) with the last 10 averaged.  One step = the whole force evaluation
of one position k z0 = j pi / 15 (setup and initial condition, the unsampled
and the sampled periods, the FP64 force, all on the device); step i takes
position j = i mod 16, so 16 steps cover the sweep.  --workload sphere256 is
the 256^3 sphere (lambda = 128, R = 16 at lambda/8, seeded compressibility
ratio, 2000 points, 15360 steps).  Inputs (two population copies of 3.8 GB at
512^3, 470 MB at 256^3) are far larger than L2, so no flush is needed.

value       GLUPS = cells x LB steps / device time (CUDA events on the
            library's stream, max over ranks), whole job.
roofline    the update kernel: algorithmic bytes per launch (57 B per cell:
            7 + 7 FP32 populations and the class byte) / its average launch
            time, measured over the unsampled periods of the timed steps;
            glups_bound is the GLUPS that one pass over the state per launch
            at the measured copy bandwidth allows.
e2e         the same metric through the public C ABI from host parameters to
            host force: handle creation on a torch workspace, wlb_run, read-back.
cpu_baseline  the FP64 oracle on the host cores, a bounded sample of the same
            lattice (a few LB steps with sampling, setup included), as GLUPS.

--impl reference times the oracle alone (the paper has no code to run).
N > 1 (torchrun): independent replicas, one lattice per rank ("replicas only").
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOADS = {
    "sphere512": "3D sphere 512^3 D3Q7 FP32 force-vs-position sweep, lambda=256, R=24, kappa~=0.5, 4096 Fibonacci "
                 "points, 30 periods avg last 10; step i = position k z0 = (i mod 16) pi/15",
    "sphere256": "3D sphere 256^3 D3Q7 FP32, lambda=128, R=16 at lambda/8, 2000 Fibonacci points, 30 periods avg last 10",
}
METRIC = "wave-LB GLUPS (% HBM roofline); radiation forces/s at <=1% err vs FP64 oracle"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, NVIDIA's figure (context beside the measured copy peak)

def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def _profile_name(steps_per_launch=1, edge=256, precision="f32"):
    """Committed ncu summary of the update kernel on an edge^3 lattice."""
    kernel = "update2_slab" if steps_per_launch == 2 else "update_rows"
    return "%s_d3q7_%s_%dcubed.md" % (kernel, precision, edge)


def _traffic(kernel_src_sha, steps_per_launch=1, edge=256, name=None):
    """Per-launch DRAM bytes of the update kernel from the committed ncu summary
    (by default the FP32 update kernel's on an edge^3 lattice), if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", name or _profile_name(steps_per_launch, edge))
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            v = v.strip()
            vals[k.strip()] = v.split("`")[1] if v.startswith("`") else (v.split() or [""])[0]
    if vals.get("kernel_source_sha256") != kernel_src_sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


HOST_MARKER = b"// ---------------------------------------------------------------- host side: plans and launches"


def _kernel_sha(steps_per_launch=1, two_step_src="wlb_two_step.cu"):
    """sha256 over the update kernel's device code and the device header it
    includes: wlb_step.cu whole, or the two-step source (wlb_two_step.cu, or
    wlb_two_step_2d.cu for the 2D batches) up to its host-side part (plans and
    launches, which a profile's counters do not depend on)."""
    csrc = os.path.join(ROOT, "paper_2404_02346_gb300", "csrc")
    h = hashlib.sha256()
    if steps_per_launch == 2:
        text = open(os.path.join(csrc, two_step_src), "rb").read()
        cut = text.find(HOST_MARKER)
        h.update(text if cut < 0 else text[:cut])
    else:
        h.update(open(os.path.join(csrc, "wlb_step.cu"), "rb").read())
    h.update(open(os.path.join(csrc, "wlb_kernels.cuh"), "rb").read())
    return h.hexdigest()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def job_totals(local_ms, local_units, world, device=None):
    """Whole-job figures for N independent replicas: the slowest rank's time and
    the units all ranks processed (max / sum all-reduce; gloo or NCCL)."""
    if world <= 1:
        return float(local_ms), float(local_units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def cpu_baseline(prob, target_s=15.0, steps=None, max_steps=60):
    """Time the FP64 oracle, as it stands, on a bounded sample of the workload:
    the full lattice for a few LB steps (about target_s seconds, at most
    max_steps), a third of them sampled."""
    import oracle
    oracle.build.build()
    if steps is None:
        probe = dict(prob, n_steps=3, n_window=1)
        t0 = time.perf_counter()
        oracle.run(probe)
        t_probe = time.perf_counter() - t0
        steps = max(3, min(max_steps, int(3 * target_s / max(t_probe, 1e-3))))
        steps -= steps % 3
    sample = dict(prob, n_steps=steps, n_window=steps // 3)
    t0 = time.perf_counter()
    oracle.run(sample)
    dt = time.perf_counter() - t0
    cells = prob["n"][0] * prob["n"][1] * prob["n"][2]
    return {"value": cells * steps / dt / 1e9, "unit": "GLUPS", "cores": oracle.threads(),
            "kind": "oracle",
            "sample": "%d LB steps (%d sampled) of the %dx%dx%d lattice incl. setup, %.1f s"
                      % (steps, steps // 3, *prob["n"], dt)}


def cpu_baseline_mlp(sur, q, n=65536):
    """Time the FP64 oracle network, as it stands, on a bounded sample of the
    queries (the first n), with the surrogate's weights."""
    import numpy as np

    from oracle import mlp as ref
    x = q[:n].cpu().numpy().astype(np.float64)
    theta = ref.bf16(sur.net.get_weights().astype(np.float64))
    xn = ref.bf16(ref.normalise(x, sur.lo.astype(np.float64), sur.hi.astype(np.float64)))
    t0 = time.perf_counter()
    ref.forward(theta, xn)
    dt = time.perf_counter() - t0
    return {"value": len(x) / dt, "unit": "forces/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d queries through the FP64 numpy network (BLAS threads: all host cores), %.2f s"
                      % (len(x), dt)}


def step_problems(args):
    """The problems of the timed workload, one per bench step in turn: the 16
    positions of the 512^3 sweep, or the single 256^3 sphere."""
    if args.workload == "sphere512":
        return [workloads.sphere_3d_large(position=j, precision=args.precision) for j in range(16)]
    return [workloads.sphere_3d(seed=args.seed, precision=args.precision)]


def run_reference(args, probs):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build.build()
    prob = probs[0]
    cells = prob["n"][0] * prob["n"][1] * prob["n"][2]
    # LB steps per bench step (a third sampled, setup included): bounded so
    # that K + W steps take minutes
    per_step = 3 if cells > 256 ** 3 else 6
    t_all = 0.0
    for i in range(args.warmup + args.steps):
        p = probs[i % len(probs)]
        sample = dict(p, n_steps=per_step, n_window=per_step // 3)
        t0 = time.perf_counter()
        oracle.run(sample)
        if i >= args.warmup:
            t_all += time.perf_counter() - t0
    value = cells * per_step * args.steps / t_all / 1e9
    sample_txt = "%d LB steps (%d sampled) of the %dx%dx%d lattice per step, setup included" % (
        per_step, per_step // 3, *prob["n"])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_all / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] + " (oracle: %d LB steps per step)" % per_step,
                   "l2": "inputs larger than L2"},
        "cpu_baseline": {"kind": "oracle", "cores": oracle.threads(), "value": value, "unit": "GLUPS",
                         "sample": sample_txt},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, probs):
    import ctypes

    import torch

    import paper_2404_02346_gb300 as wlb
    from paper_2404_02346_gb300 import build as B

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.build()
    stream = torch.cuda.Stream()
    prob0 = probs[0]
    cells = prob0["n"][0] * prob0["n"][1] * prob0["n"][2]
    edge = prob0["n"][0]

    def make(prob):
        s = wlb.Solver(prob, stream=stream)
        if args.single_step:
            s.set_two_step(False)
            return s
        if args.tiles:
            s.set_two_step_tiles(args.tiles)
        if args.slab_rows:
            s.set_two_step(True, args.slab_rows)
        return s

    # one handle for a fixed problem; a new one per position otherwise (the
    # setup differs; creating it is part of the position's force evaluation)
    fixed = make(prob0) if len(probs) == 1 else None
    if fixed is not None:
        info = fixed.info()
    else:
        with make(prob0) as s:
            info = s.info()
    n_steps, n_window = info.n_steps, info.n_window
    n_free = n_steps - n_window
    n_avg = n_window // info.period

    def one_step(i, ev=None):
        solver = fixed or make(probs[i % len(probs)])
        solver.init()
        if ev is not None:
            ev[0].record(stream)
        solver.step(n_free, sample=False)
        if ev is not None:
            ev[1].record(stream)
        solver.step(n_window, sample=True)
        F = solver.force()
        if fixed is None:
            solver.close()
        return F

    for i in range(args.warmup):
        one_step(i)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    k1 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    forces = []
    start.record(stream)
    for i in range(args.steps):
        forces.append(one_step(i, k1[i]))
    end.record(stream)
    barrier()
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    # average duration of one update launch in the unsampled phase (one or two
    # steps per launch)
    spl = info.steps_per_launch
    k1_ms = sum(a.elapsed_time(b) for a, b in k1) / (args.steps * n_free) * spl
    ms, lu = job_totals(ms, cells * n_steps * args.steps, world, device="cuda")
    glups = lu / (ms * 1e-3) / 1e9
    forces_per_s = lu / (cells * n_steps) / (ms * 1e-3)
    if fixed is not None:
        fixed.close()

    # end to end through the public API: host parameters in, host force out
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        Fe = wlb.compute_force(probs[i % len(probs)])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": cells * n_steps * e2e_steps * world / e2e_s / 1e9, "unit": "GLUPS",
           "h2d_bytes_per_step": ctypes.sizeof(wlb.Params), "d2h_bytes_per_step": 4 * 8 + 4,
           "forces_per_s": e2e_steps / e2e_s, "force": [float(v) for v in Fe]}

    peaks = _peaks()
    # algorithmic HBM bytes per cell of one update launch: every population
    # read and written once, plus the class byte (also with two steps per
    # launch: the state between them stays on chip; c^2 of the few
    # interface-band rows is not counted)
    bpu = info.bytes_per_update
    achieved = bpu * cells / (k1_ms * 1e-3) / 1e9
    if peaks and "hbm_gbs" in peaks:
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    traffic = (_traffic(_kernel_sha(spl), spl, edge, name=_profile_name(spl, edge, args.precision))
               if args.precision in ("f32", "f16") else None)
    # lattice updates per second if every launch moved exactly its algorithmic
    # bytes at the measured copy bandwidth (one pass over the state per launch)
    glups_bound = peak / (bpu / spl)
    # per force: 3 setup kernels, one update launch per step pair (sampled
    # launches add their sampling kernel; one per step on the row-vectorised
    # one-step path is fused), per averaged period a fold and the two launches
    # that record its force in the history, the force
    if spl == 2:
        per_step = 3 + n_free // 2 + 2 * (n_window // 2) + 3 * n_avg + 1
    else:
        per_step = 3 + n_window + n_free + (0 if info.vector_path else n_window) + 3 * n_avg + 1
    launches = args.steps * per_step
    if rank == 0:
        positions = sorted({i % len(probs) for i in range(args.steps)})
        line = {
            "metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "f64": "f64", "f16": "f16 storage, f32 arithmetic"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "cells": cells, "lb_steps_per_force": n_steps,
                       "window_steps": n_window, "kappa_ratio": prob0.get("kappa"),
                       "positions_timed": len(positions) if len(probs) > 1 else 1,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs (2 x %.2f GB populations) larger than L2; no flush"
                             % (7 * cells * {"f32": 4, "f16": 2, "f64": 8}[args.precision] / 1e9)},
            "forces_per_s": forces_per_s,
            "force": [float(v) for v in forces[0]],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                         "kernel": ("update2_slab, 2 steps/launch, %d-row slabs, %d x-tile%s per row"
                                    % (info.two_step_rows, info.two_step_tiles, "" if info.two_step_tiles == 1 else "s")
                                    if spl == 2 else "update_rows")
                                   + " (%s storage)" % args.precision, "bytes_per_cell_per_launch": bpu,
                         "steps_per_launch": spl, "avg_launch_us": k1_ms * 1e3,
                         "glups_bound": glups_bound, "glups_frac_of_bound": glups / (world * glups_bound),
                         "peak_source": peak_src + " hbm_gbs"},
            "cpu_baseline": None, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        }
        if len(probs) > 1:
            line["forces_by_position"] = {str(i % len(probs)): float(F[2]) for i, F in enumerate(forces)}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(prob0, steps=12 if cells > 256 ** 3 else None)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_ensemble(args):
    """Batched ensemble: forces/s of one batched launch sequence over all
    lattices, against the same lattices run one at a time through the
    single-lattice path (a sample of them, timed on the same GPU)."""
    import numpy as np
    import torch

    import paper_2404_02346_gb300 as wlb
    from paper_2404_02346_gb300 import build as B

    B.build()
    if args.workload == "ensemble3d":
        count = args.count or 64
        probs = workloads.ensemble_3d(seed=args.seed, count=count, precision=args.precision)
        desc = "%d x 3D D3Q7 lattices, edge U{96,128,160}, lambda=edge/2, R~U[4,12], 1000 points, 25 periods" % count
    else:
        count = args.count or 512
        probs = workloads.ensemble_2d(seed=args.seed, count=count, precision=args.precision)
        desc = "%d x 2D D2Q5 192^2 lattices, lambda=96, R~U[4,12], 1000 points, 25 periods" % count
    stream = torch.cuda.Stream()
    batch = wlb.Batch(probs, stream=stream)
    tune = batch.autotune(steps_per_trial=16)
    info = batch.info()
    for _ in range(args.warmup):
        F = batch.run()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    start.record(stream)
    for _ in range(args.steps):
        F = batch.run()
    end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = start.elapsed_time(end) / args.steps
    batch.close()
    # the same lattices through the single-lattice path, one after another
    n_single = min(len(probs), 16 if args.workload == "ensemble3d" else 32)
    idx = list(range(0, len(probs), max(1, len(probs) // n_single)))[:n_single]
    singles, lu_single = [], 0
    solvers = [wlb.Solver(probs[i], stream=stream) for i in idx]
    solvers[0].run()  # graph capture outside the timed region
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in solvers:
        singles.append(s.run())
        lu_single += s.cells * s.info().n_steps
    t1.record(stream)
    torch.cuda.synchronize()
    ms_single = t0.elapsed_time(t1)
    for s in solvers:
        s.close()
    ax = probs[0]["wave_axis"]
    rel = max(abs(F[i, ax] - singles[k][ax]) / max(abs(singles[k][ax]), 1e-300) for k, i in enumerate(idx))
    # roofline of the batched update: algorithmic bytes of one launch over every
    # lattice (each population read and written once per launch, plus the class
    # byte) / its duration, from the library's own event timing of update-only
    # steps (autotune: all lattices before their windows; the sampling launch
    # between updates exits at once)
    q = 2 * probs[0]["dim"] + 1
    size = {"f32": 4, "f16": 2, "f64": 8}[args.precision]
    bpu = 2 * q * size + 1
    cells_all = sum(int(np.prod(p["n"][:p["dim"]])) for p in probs)
    spl = info.steps_per_launch if info.steps_per_launch > 0 else 1
    launch_ms = tune["ms_per_step"] * spl
    achieved = bpu * cells_all / (launch_ms * 1e-3) / 1e9
    peaks = _peaks()
    peak = float(peaks["hbm_gbs"]) if peaks and "hbm_gbs" in peaks else 6800.0
    # the oracle on a bounded sample of the first lattice, as forces/s at the
    # ensemble's mean lattice updates per force
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(probs[0], target_s=10.0, max_steps=30000)
        lu_per_force = info.lattice_updates / len(probs)
        cpu = dict(cpu, glups=cpu["value"], value=cpu["value"] * 1e9 / lu_per_force, unit="forces/s",
                   sample=cpu["sample"] + "; forces/s at the ensemble's mean %.3g LU per force" % lu_per_force)
    # DRAM bytes of one two-step pass from the committed ncu summaries (the
    # 64-lattice 3D and 512-lattice 2D FP32 ensembles only)
    traffic = None
    if args.workload == "ensemble3d" and args.precision == "f32" and len(probs) == 64 and spl == 2:
        traffic = _traffic(_kernel_sha(2), name="batch_update2_d3q7_f32_ensemble64.md")
    elif args.workload == "ensemble2d" and args.precision == "f32" and len(probs) == 512 and spl == 2:
        traffic = _traffic(_kernel_sha(2, "wlb_two_step_2d.cu"), name="batch2d_update2_d2q5_f32_ensemble512.md")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": ("batched two-step update" if spl == 2 else "batched update")
                                          + " (%s storage), all lattices" % args.precision,
                "bytes_per_cell_per_launch": bpu, "avg_launch_us": launch_ms * 1e3,
                "peak_source": ("measured" if peaks and "hbm_gbs" in peaks else "fallback") + " hbm_gbs"}
    line = {
        "metric": "radiation forces/s, batched ensemble", "value": len(probs) / (ms * 1e-3), "unit": "forces/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
        "data": "synthetic",
        "config": {"workload": desc, "lattices": len(probs), "lattice_updates": info.lattice_updates,
                   "tuning": tune, "l2": "inputs larger than L2"},
        "glups": info.lattice_updates / (ms * 1e-3) / 1e9,
        "single_instance": {"forces_per_s": len(idx) / (ms_single * 1e-3), "sampled_lattices": len(idx),
                            "glups": lu_single / (ms_single * 1e-3) / 1e9,
                            "max_rel_force_diff_vs_batch": rel},
        "speedup_vs_single": (len(probs) / (ms * 1e-3)) / (len(idx) / (ms_single * 1e-3)),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def _time_predict(sur, q, args):
    """Seconds per predict call (host clock) and the roofline of the fused
    forward (CUDA events on the current stream; each call is one kernel
    launch plus a 4-byte status read)."""
    import torch

    for _ in range(args.warmup):
        sur.predict(q)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    t0 = time.perf_counter()
    for s in range(args.steps):
        ev[2 * s].record()
        sur.predict(q)
        ev[2 * s + 1].record()
    torch.cuda.synchronize()
    q_s = (time.perf_counter() - t0) / args.steps
    k_s = sum(ev[2 * s].elapsed_time(ev[2 * s + 1]) for s in range(args.steps)) / args.steps * 1e-3
    # algorithmic products: 2 (4*256 + 2*256*256 + 256) flops per query
    flops = 2.0 * (4 * 256 + 2 * 256 * 256 + 256) * int(q.shape[0])
    peaks = _peaks()
    peak = peaks.get("bf16_tflops") if peaks else None
    achieved = flops / k_s / 1e12
    return q_s, {"bound": "tensor", "kernel": "mlp_forward_fused", "achieved": achieved, "peak": peak,
                 "unit": "TFLOP/s", "frac": achieved / peak if peak else None, "traffic": None,
                 "peak_source": "measured bf16_tflops (burst)" if peak else None, "kernel_ms": k_s * 1e3}


def run_surrogate_infer(args):
    """Inference of the surrogate network alone: the fused tensor-core forward
    on seeded queries with seeded initial weights (trained weights do the same
    work)."""
    import numpy as np
    import torch

    from paper_2404_02346_gb300 import build as B
    from paper_2404_02346_gb300 import surrogate as S

    B.build()
    sur = S.Surrogate(workloads.SURROGATE_BOX)
    sur.net.init_weights(args.seed)
    q = torch.tensor(np.array(workloads.surrogate_queries(args.queries, seed=args.seed + 2000), dtype=np.float32),
                     device="cuda")
    q_s, roofline = _time_predict(sur, q, args)
    cpu = None if args.no_cpu_baseline else cpu_baseline_mlp(sur, q)
    sur.close()
    line = {
        "metric": "radiation forces/s, learned surrogate (inference)", "value": args.queries / q_s,
        "unit": "forces/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": q_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 weights/activations, fp32 accumulate (tcgen05)", "data": "synthetic",
        "config": {"workload": "MLP 4-256-256-256-1 GELU, seeded initial weights; %d seeded queries" % args.queries},
        "roofline": roofline, "gpu_launches": args.steps, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def run_surrogate(args):
    """Learned surrogate: 20k training and 2k held-out forces from the batched
    2D lattice runs (512-lattice chunks of 192^2 D2Q5, 25 periods), training on
    the tensor-core network, validation error, and 1M seeded queries."""
    import numpy as np
    import torch

    from paper_2404_02346_gb300 import build as B
    from paper_2404_02346_gb300 import surrogate as S

    B.build()
    train = workloads.surrogate_problems(20000, seed=args.seed)
    val = workloads.surrogate_problems(2000, seed=args.seed + 1000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_train = S.lattice_targets(train)
    t_val = S.lattice_targets(val)
    torch.cuda.synchronize()
    lb_s = time.perf_counter() - t0
    sur = S.Surrogate(workloads.SURROGATE_BOX, batch_max=1 << 17)
    t0 = time.perf_counter()
    hist = sur.fit([p["features"] for p in train], t_train, epochs=args.epochs, batch=512)
    train_s = time.perf_counter() - t0
    y, _ = sur.predict([p["features"] for p in val])
    err = y.cpu().numpy() - t_val
    scale = float(np.abs(t_val).max())
    q = torch.tensor(np.array(workloads.surrogate_queries(args.queries, seed=args.seed + 2000), dtype=np.float32),
                     device="cuda")
    q_s, roofline = _time_predict(sur, q, args)
    cpu = None if args.no_cpu_baseline else cpu_baseline_mlp(sur, q)
    sur.close()
    lb_rate = (len(train) + len(val)) / lb_s
    line = {
        "metric": "radiation forces/s, learned surrogate", "value": args.queries / q_s, "unit": "forces/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": q_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 weights/activations, fp32 accumulate (tcgen05)", "data": "synthetic",
        "config": {"workload": "MLP 4-256-256-256-1 GELU; 20k train / 2k held-out 2D lattice forces "
                               "(192^2 D2Q5, 25 periods); %d seeded queries" % args.queries,
                   "epochs": args.epochs, "batch": 512},
        "roofline": roofline,
        "gpu_launches": args.steps,
        "cpu_baseline": cpu,
        "lattice_forces_per_s_batched": lb_rate,
        "speedup_vs_batched_lattice": (1 << 20) / q_s / lb_rate,
        "train_s": train_s, "final_train_loss": float(hist[-1]),
        "val_error": {"rms": float(np.sqrt(np.mean(err ** 2))), "max_abs": float(np.abs(err).max()),
                      "target_scale_max_abs": scale,
                      "rms_over_scale": float(np.sqrt(np.mean(err ** 2))) / scale,
                      "frac_within_1pct_of_scale": float(np.mean(np.abs(err) <= 0.01 * scale))},
    }
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """512^3 D3Q7 force-vs-position sweep: 16 positions k z0 = j pi / 15, run one
    after another, for each requested storage precision; F(kz) against the
    sin(2 k z0) law and the FP16 - FP32 difference per position."""
    import math

    import torch

    import paper_2404_02346_gb300 as wlb
    from paper_2404_02346_gb300 import build as B

    B.build()
    stream = torch.cuda.Stream()
    precs = ["f32", "f16"] if args.precision == "f32" else [args.precision]
    positions = list(range(16))[: max(1, min(16, args.positions))]
    res = {}
    lu = 0
    t_all = {}
    cells = 512 ** 3
    peaks = _peaks()
    peak = float(peaks["hbm_gbs"]) if peaks and "hbm_gbs" in peaks else 6800.0
    roofline = {}
    for prec in precs:
        # the update kernel alone: 64 unsampled steps of position 0, CUDA events
        with wlb.Solver(workloads.sphere_3d_large(position=0, precision=prec), stream=stream) as s0:
            info = s0.info()
            s0.init()
            s0.step(64)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s0.step(64)
            b.record(stream)
            torch.cuda.synchronize()
            launch_ms = a.elapsed_time(b) / 64 * info.steps_per_launch
            achieved = info.bytes_per_update * cells / (launch_ms * 1e-3) / 1e9
            roofline[prec] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                              "frac": achieved / peak,
                              "traffic": (_traffic(_kernel_sha(2), 2, 512, name=_profile_name(2, 512, prec))
                                          if info.steps_per_launch == 2 else None),
                              "kernel": "update2_slab, %d steps/launch, %d-row slabs (%s storage)"
                                        % (info.steps_per_launch, info.two_step_rows, prec),
                              "bytes_per_cell_per_launch": info.bytes_per_update,
                              "avg_launch_us": launch_ms * 1e3}
    for prec in precs:
        forces = []
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for j in positions:
            prob = workloads.sphere_3d_large(position=j, precision=prec)
            with wlb.Solver(prob, stream=stream) as sj:
                forces.append(float(sj.run()[2]))
                steps = sj.info().n_steps
        end.record(stream)
        torch.cuda.synchronize()
        t_all[prec] = start.elapsed_time(end) * 1e-3
        res[prec] = forces
        lu = cells * steps * len(positions)
    f32 = res.get("f32")
    fit = None
    if f32 and len(f32) == 16:
        amp = max(abs(v) for v in f32)
        kz = [j * math.pi / 15 for j in range(16)]
        # least-squares amplitude of the sin(2 k z0) law and the residual
        a = sum(f * math.sin(2 * k) for f, k in zip(f32, kz)) / sum(math.sin(2 * k) ** 2 for k in kz)
        resid = max(abs(f - a * math.sin(2 * k)) for f, k in zip(f32, kz)) / amp
        fit = {"amplitude": a, "max_residual_over_amplitude": resid}
    line = {
        "metric": "512^3 force-vs-position sweep", "value": lu / t_all[precs[0]] / 1e9, "unit": "GLUPS",
        "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": t_all[precs[0]] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": precs[0], "data": "synthetic",
        "config": {"workload": "512^3 D3Q7, lambda=256, R=24, 4096 points, kappa~=0.5, %d of the 16 positions "
                               "x 30 periods" % len(positions)},
        "roofline": roofline[precs[0]], "roofline_by_precision": roofline,
        "cpu_baseline": (None if args.no_cpu_baseline
                         else cpu_baseline(workloads.sphere_3d_large(position=0), steps=6)),
        "forces": res, "sin2kz_fit_f32": fit,
        "seconds": t_all,
        "glups": {p: lu / t_all[p] / 1e9 for p in precs},
    }
    if "f16" in res and f32:
        amp = max(abs(v) for v in f32)
        line["f16_minus_f32_over_amplitude"] = [abs(a - b) / amp for a, b in zip(res["f16"], f32)]
    print(json.dumps(line), flush=True)


def run_profile(args, prob):
    """A short pass over the benchmark lattice for ncu: setup, 64 unsampled and
    64 sampled steps (graph-replayed where whole periods allow), the force.
    --profile-nz cuts the lattice along z (same rows, planes and slab plan per
    plane; fewer planes) for captures that must stay within a few GB."""
    import torch

    import paper_2404_02346_gb300 as wlb
    from paper_2404_02346_gb300 import build as B

    B.build()
    if args.profile_nz:
        nx, ny, _ = prob["n"]
        lam = float(args.profile_nz)  # one wavelength along the cut axis
        prob = workloads.problem(3, (nx, ny, args.profile_nz), 2, lam, prob["radius"],
                                 (nx / 2, ny / 2, lam / 8), cp=prob["cp"], n_surface=prob["n_surface"],
                                 n_periods=1, n_avg_periods=1, precision=prob["precision"])
    stream = torch.cuda.Stream()
    with wlb.Solver(prob, stream=stream) as s:
        if args.single_step:
            s.set_two_step(False)
        else:
            if args.tiles:
                s.set_two_step_tiles(args.tiles)
            if args.slab_rows:
                s.set_two_step(True, args.slab_rows)
        info = s.info()
        s.init()
        s.step(args.profile_steps, sample=False)
        s.step(args.profile_steps, sample=True)
        F = s.force()
    print(json.dumps({"profile_run": True, "shape": list(prob["n"]), "force": [float(v) for v in F],
                      "steps_per_launch": info.steps_per_launch, "slab_rows": info.two_step_rows,
                      "segments": info.two_step_segments, "tiles": info.two_step_tiles}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--single-step", action="store_true",
                    help="one step per update launch (default: unsampled steps two per launch)")
    ap.add_argument("--slab-rows", type=int, default=0, help="slab height of the two-step kernel (0: automatic)")
    ap.add_argument("--tiles", type=int, default=0,
                    help="x-tiles per row of the two-step kernel (0: automatic, 1: whole rows)")
    ap.add_argument("--profile", action="store_true", help="short pass for ncu captures")
    ap.add_argument("--profile-steps", type=int, default=64)
    ap.add_argument("--precision", default="f32", choices=["f32", "f16", "f64"],
                    help="population storage (the benchmark workload is FP32)")
    ap.add_argument("--workload", default="sphere512",
                    choices=["sphere512", "sphere256", "ensemble3d", "ensemble2d", "surrogate", "surrogate_infer",
                             "sweep512"],
                    help="sphere512: the benchmark line (512^3, one sweep position per step); sphere256: the "
                         "256^3 sphere; ensembles: batched forces/s; surrogate: learned model (surrogate_infer: "
                         "its inference alone); sweep512: all 16 positions per storage precision in one line")
    ap.add_argument("--epochs", type=int, default=1500, help="surrogate training epochs")
    ap.add_argument("--queries", type=int, default=1 << 20, help="surrogate inference queries")
    ap.add_argument("--positions", type=int, default=16, help="sweep512: the first N of the 16 positions")
    ap.add_argument("--count", type=int, default=0, help="ensembles: lattices (0: 64 in 3D, 512 in 2D)")
    ap.add_argument("--profile-nz", type=int, default=0, help="--profile: planes of a z-cut lattice (0: full)")
    args = ap.parse_args()
    if args.workload == "surrogate":
        run_surrogate(args)
    elif args.workload == "surrogate_infer":
        run_surrogate_infer(args)
    elif args.workload == "sweep512":
        run_sweep(args)
    elif args.workload in ("ensemble3d", "ensemble2d"):
        run_ensemble(args)
    elif args.profile:
        run_profile(args, step_problems(args)[0])
    elif args.impl == "reference":
        run_reference(args, step_problems(args))
    else:
        run_gpu(args, step_problems(args))


if __name__ == "__main__":
    main()
