#!/usr/bin/env python3
"""Benchmark: agent-updates/s of the mechanical-interaction iteration on one
GB300, on the 10M-agent Gaussian-blob workload in the FP32-force form (the
plain FP64 form is timed beside it), with the roofline of the dominant kernel
and the FP64 CPU oracle timed on a bounded same-density sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  Under torchrun every rank advances its own
replica of the workload (weak scaling, no data-path collective); the timed
region is bracketed by a barrier and the slowest rank's time is reported.
"""
import argparse
import ctypes as C
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "agent-updates/s per mechanical step, FP32-force vs plain FP64 form; % HBM peak"
UNIT = "agent-updates/s"
SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0
# algorithmic FP32 work of the force kernel, two models:
#  - the scope table's: 10 flops per candidate pair (the prefilter) and 25 per
#    contact (the force), the model the reported fraction uses;
#  - a tighter count of the kernel's own arithmetic: 8 per candidate (3
#    differences, 3 products, 2 sums for d^2) and 20 per contact (radius sum
#    and square, inverse root and distance, overlap, reduced radius, the two
#    force terms and their difference, the scale and three fused
#    accumulations), reported beside it
FLOP_MODEL = (10, 25)
FLOP_MODEL_KERNEL = (8, 20)
# algorithmic HBM bytes per agent of the force kernel in the FP32 form: own
# record (16) + sorted->storage index (4) + flags and contacts in/out (6) +
# position read (24) and write (24)
FORCE_BYTES_PER_AGENT = 74
# DRAM traffic of the force kernel from an ncu capture, keyed by the hash of
# the kernel's sources (used only while they match the source that runs)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_force_fp32_traffic.json")
HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=10_000_000,
                    help="agents of the blob workload (and of core_shell_leg)")
    ap.add_argument("--sample", type=int, default=0, help="agents of the oracle's CPU sample (0 = auto)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="blobs",
                    choices=["blobs", "ensemble", "core_shell", "core_shell_leg", "lattice", "uniform"],
                    help="blobs is the headline; the others measure the remaining configurations")
    ap.add_argument("--sort-every", type=int, default=10,
                    help="blobs: Morton re-sort cadence (0 = never; the headline workload uses 10)")
    ap.add_argument("--curve", default="morton", choices=["morton", "hilbert"],
                    help="blobs: space-filling curve of the sort (bricks of 4x4x4 boxes along it)")
    ap.add_argument("--lanes", type=int, default=None,
                    help="blobs: FP32 force kernel (bdm_set_force_kernel value; default: the library's)")
    ap.add_argument("--presort", action="store_true",
                    help="blobs: put storage in Morton order (bdm_sort) before the warm-up")
    ap.add_argument("--no-autotune", action="store_true", help="ensemble, core_shell: skip the autotuner")
    ap.add_argument("--no-legs", action="store_true",
                    help="blobs: skip the compact ensemble and core + shell legs of the default line")
    return ap.parse_args()


def workload(n):
    from paper_2301_06984_gb300 import workloads as W
    if n == 10_000_000:
        return W.blobs(n=n, seed=3)
    # same density profile with fewer agents: lengths scale by (n / 1e7)^(1/3)
    sc = (n / 1.0e7) ** (1.0 / 3.0)
    return W.blobs(n=n, seed=3, sigma=150.0 * sc, domain=4000.0 * sc, centre_lo=600.0 * sc, centre_hi=3400.0 * sc)


def config(args):
    return {
        "workload": "blobs-%d: 8 Gaussian blobs (sigma 150 um) in [0,4000]^3 um, diameters U[9,11] um, "
                    "R = L = 11 um, dt 0.01, max displacement 3 um, %s re-sort every %d iterations" % (
                        args.n, args.curve.capitalize(), args.sort_every),
        "n_agents": args.n,
        "precision": "FP32 pair force and accumulation; FP64 cutoff predicate, contact decision and positions",
        "l2_policy": "inputs larger than L2 (about 1 GB touched per iteration vs 129 MB L2); no flush",
        "sort_every": args.sort_every,
        "curve": args.curve,
        "force_kernel": "library default" if args.lanes is None else args.lanes,
        "presort": bool(args.presort),
        "parallelism": "replica per GPU" if args.gpus > 1 else "single GPU",
    }


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        busy = [v for v in sm if mx and v > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def force_source_sha():
    h = hashlib.sha256()
    for f in ("force.cu", "bdm_internal.cuh", "params.cu"):
        with open(os.path.join(ROOT, "paper_2301_06984_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(n_agents):
    """DRAM bytes of one force launch over n_agents, from the machine-readable
    record of an ncu capture (bytes per agent), if that capture was taken on
    the current kernel source; else None."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None, None
    if rec.get("source_sha256") != force_source_sha():
        return None, rec.get("source_sha256")
    return float(rec["dram_bytes_per_agent"]) * n_agents, rec["source_sha256"]


def measured_peaks():
    """Measured peaks (HBM copy GB/s, ...), or the profiling recipe's fallback
    HBM figure when the measured file is absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
            d["_source"] = "of measured"
            return d
    except (OSError, ValueError):
        return {"hbm_gbs": HBM_FALLBACK_GBS, "_source": "of fallback"}


def oracle_timing_lib():
    """The oracle's OpenMP timing build (all host cores) and its thread count,
    or the serial build and 1."""
    from oracle import build_oracle
    from oracle import oracle as O
    path = build_oracle.build_omp()
    if path is None:
        O.lib()
        return None, 1
    return path, None


def cpu_baseline(n_sample, n_steps=2):
    """The FP64 oracle, as it stands (its OpenMP timing build: the per-agent
    force loop over all host cores, same results), over a same-density sample
    of the blob workload.  Returns agent-updates/s, seconds, threads."""
    from oracle import oracle as O
    w = workload(n_sample)
    P = O.make_params(R=11.0, L=11.0, dt=0.01, dmax=3.0, sort_every=10, seed=3)
    path, _ = oracle_timing_lib()
    lib = O.use_library(path) if path else None
    if lib is not None:
        L = lib.__enter__()
        threads = L.orc_threads()
    else:
        threads = 1
    try:
        s = O.State(w.x, w.y, w.z, w.diam)
        t0 = time.perf_counter()
        s.step(P, n_steps)
        dt = time.perf_counter() - t0
    finally:
        if lib is not None:
            lib.__exit__(None, None, None)
    return n_sample * n_steps / dt, dt, threads


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n_s = args.sample or int(min(2_000_000, max(200_000, 6e7 / max(1, args.steps + args.warmup))))
    from oracle import oracle as O
    w = workload(n_s)
    P = O.make_params(R=11.0, L=11.0, dt=0.01, dmax=3.0, sort_every=10, seed=3)
    path, _ = oracle_timing_lib()
    lib = O.use_library(path) if path else None
    threads = lib.__enter__().orc_threads() if lib is not None else 1
    try:
        s = O.State(w.x, w.y, w.z, w.diam)
        s.step(P, args.warmup)
        t0 = time.perf_counter()
        s.step(P, args.steps)
        dt = time.perf_counter() - t0
    finally:
        if lib is not None:
            lib.__exit__(None, None, None)
    v = n_s * args.steps / dt
    cfg = config(args)
    cfg["n_agents"] = n_s
    cfg["workload"] = ("blobs-%d (a same-density sample of the %d-agent workload: lengths scaled by "
                       "(n/1e7)^(1/3)): 8 Gaussian blobs, diameters U[9,11] um, R = L = 11 um, dt 0.01, "
                       "max displacement 3 um, Morton re-sort every 10 iterations" % (n_s, args.n))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d iterations of the FP64 oracle over a %d-agent blob workload of the same "
                                   "density, force loop on %d host threads (OpenMP timing build)"
                                   % (args.steps, n_s, threads)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- other workloads
# algorithmic HBM bytes per agent of the FP32-form iteration, by phase: keys
# 33, scatter 12, brick sort 56, force 74 (32 for a static agent: its index,
# flags, contacts and the position read for the bounding box)
STEP_BYTES_MOVING, STEP_BYTES_STATIC = 33 + 12 + 56 + 74, 33 + 12 + 56 + 32


def reduce_over_ranks(ms, updates, dist, device):
    """Whole-job figures of a timed region: the slowest rank's time and the
    agent-updates of all ranks (identity without a process group)."""
    if dist is None:
        return ms, updates
    import torch
    tm = torch.tensor([ms], dtype=torch.float64, device=device)
    tu = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(tu, op=dist.ReduceOp.SUM)
    return float(tm.item()), float(tu.item())


def timed_steps(sim, k, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_other(args):
    import numpy as np
    import torch

    from paper_2301_06984_gb300 import bdm
    from paper_2301_06984_gb300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "data": "synthetic"}
    if args.workload == "ensemble":
        w = W.ensemble()
        sim = bdm.Simulation.from_workload(w)
        sim.set_workload(w)
        tuning = None
        if not args.no_autotune:
            # box edge, force kernel (threads per box pair) and sort cadence
            tuning = sim.autotune(trial_steps=3)
        sim.step(args.warmup)
        ms = timed_steps(sim, args.steps, stream)
        sim.profile_begin()
        sim.step(1)
        phases = sim.profile_end()
        line["phases_ms_per_step"] = {k: round(v[0], 4) for k, v in phases.items()}
        line.update(value=w.n * args.steps / (ms * 1e-3), ms_per_step=ms / args.steps, dtype="f32",
                    config={"workload": "ensemble-512: 512 independent simulations, 10^U[3,5] agents each, "
                                        "0.25 volume fraction cubes, d = 10 um, dt U[0.005,0.02]; all "
                                        "simulations in one CUDA-graph launch sequence per iteration",
                            "n_agents": w.n, "n_sims": w.n_sims, "autotuned": tuning})
        # baseline: one simulation object (own graph) per member, launched one after another
        sims = []
        for m in range(w.n_sims):
            lo, hi = w.sim_off[m], w.sim_off[m + 1]
            q = bdm.Simulation(R=10.0, capacity=int(hi - lo), dt=float(w.dt_sim[m]), precision="fp32")
            q.set_agents(w.x[lo:hi], w.y[lo:hi], w.z[lo:hi], w.diam[lo:hi])
            q.step(args.warmup)
            sims.append(q)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for q in sims:
            q.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms1 = e0.elapsed_time(e1)
        line["one_launch_per_simulation"] = {"value": w.n * args.steps / (ms1 * 1e-3), "unit": UNIT,
                                             "ms_per_step": ms1 / args.steps}
        line["batched_speedup"] = ms1 / ms
        for q in sims:
            q.close()
    elif args.workload == "core_shell":
        w = W.core_shell()
        sim = bdm.Simulation.from_workload(w)
        sim.set_workload(w)
        tuning = None
        if not args.no_autotune:
            tuning = sim.autotune(trial_steps=3)
        sim.step(args.warmup)
        c0 = sim.counters()
        ms = timed_steps(sim, args.steps, stream)
        c = sim.counters()
        sim.profile_begin()
        sim.step(1)
        phases = sim.profile_end()
        st = c["n_static"]
        bytes_step = STEP_BYTES_MOVING * (w.n - st) + STEP_BYTES_STATIC * st
        peaks = measured_peaks()
        gbs = bytes_step / (ms / args.steps * 1e-3) / 1e9
        line.update(value=w.n * args.steps / (ms * 1e-3), ms_per_step=ms / args.steps, dtype="f32",
                    config={"workload": "core_shell-150M: FCC static core (90%) + random-walk shell (10%), "
                                        "d = 10 um, R = 10 um, static-agent skip on", "n_agents": w.n,
                            "autotuned": tuning},
                    skipped_fraction=st / w.n,
                    roofline={"bound": "hbm", "kernel": "whole iteration", "achieved": gbs,
                              "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                              "frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
                              "traffic": None, "bytes_per_step_algorithmic": bytes_step},
                    phases_ms_per_step={k: round(v[0], 4) for k, v in phases.items()},
                    gpu_launches=c["kernels_launched"] - c0["kernels_launched"])
    else:
        w = W.lattice() if args.workload == "lattice" else W.uniform()
        cap = 4 * w.n + 16 if args.workload == "lattice" else w.n
        vol = (math.pi / 6.0) * w.diam ** 3 if args.workload == "lattice" else None
        sim = bdm.Simulation.from_workload(w, capacity=cap)
        sim.set_agents(w.x, w.y, w.z, w.diam, vol=vol, beh=w.beh)
        total, tms = 0, 0.0
        for t in range(w.steps):
            total += sim.counters()["n_agents"]
            tms += timed_steps(sim, 1, stream)
        line.update(value=total / (tms * 1e-3), ms_per_step=tms / w.steps, steps=w.steps, warmup=0, dtype="f64",
                    config={"workload": w.name + " (FP64 form)", "n_agents_final": sim.counters()["n_agents"]})
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- compact legs of the default line
# Settings measured best for these workloads (box edge; force kernel: -3 = the
# sparse kernel, one thread per agent, for their one to two agents per box;
# sort cadence); the legs use them without re-tuning so that the default run
# stays short.
ENSEMBLE_SETTINGS = dict(box_edge=15.0, lanes=-3, sort_every=10)
CORE_SHELL_SETTINGS = dict(box_edge=15.0, lanes=-3, sort_every=5)


def leg_ensemble(args, steps=10, warmup=3):
    """512 independent simulations: one launch sequence per iteration for all
    members (batched) against one per member, agent-updates/s of each."""
    import torch

    from paper_2301_06984_gb300 import bdm
    from paper_2301_06984_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    w = W.ensemble()
    st = ENSEMBLE_SETTINGS
    sim = bdm.Simulation.from_workload(w, box_edge=st["box_edge"], sort_every=st["sort_every"])
    sim.set_force_kernel(st["lanes"])
    sim.set_workload(w)
    sim.step(warmup)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms = timed_steps(sim, steps, stream)
    sims = []
    for m in range(w.n_sims):
        lo, hi = w.sim_off[m], w.sim_off[m + 1]
        q = bdm.Simulation(R=10.0, capacity=int(hi - lo), dt=float(w.dt_sim[m]), precision="fp32",
                           box_edge=st["box_edge"], sort_every=st["sort_every"])
        q.set_force_kernel(st["lanes"])
        q.set_agents(w.x[lo:hi], w.y[lo:hi], w.z[lo:hi], w.diam[lo:hi])
        q.step(warmup)
        sims.append(q)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k1 = max(1, steps // 2)
    torch.cuda.synchronize()
    e0.record(stream)
    for q in sims:
        q.step(k1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1)
    for q in sims:
        q.close()
    sim.close()
    batched = w.n * steps / (ms * 1e-3)
    per_sim = w.n * k1 / (ms1 * 1e-3)
    return {"workload": "ensemble-512: 512 simulations, 10^U[3,5] agents each (%d in all), d = 10 um, dt "
                        "U[0.005,0.02], FP32 form" % w.n, "settings": st, "steps": steps, "warmup": warmup,
            "batched": {"value": batched, "unit": UNIT, "ms_per_step": ms / steps},
            "one_launch_sequence_per_simulation": {"value": per_sim, "unit": UNIT, "ms_per_step": ms1 / k1,
                                                   "steps": k1},
            "batched_speedup": batched / per_sim, "clocks": clk.summary()}


def leg_core_shell(args, steps=10, warmup=3, n=150_000_000):
    """n agents (150M by default), 90% in a static core: agent-updates/s, the
    skipped fraction, per-phase times and the algorithmic HBM throughput of
    the iteration."""
    import torch

    from paper_2301_06984_gb300 import bdm
    from paper_2301_06984_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    w = W.core_shell(n=n)
    st = CORE_SHELL_SETTINGS
    sim = bdm.Simulation.from_workload(w, box_edge=st["box_edge"], sort_every=st["sort_every"])
    sim.set_force_kernel(st["lanes"])
    sim.set_workload(w)
    sim.step(warmup)
    c0 = sim.counters()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms = timed_steps(sim, steps, stream)
    c = sim.counters()
    sim.profile_begin()
    sim.step(2)
    phases = sim.profile_end()
    sim.close()
    stat = c["n_static"]
    bytes_step = STEP_BYTES_MOVING * (w.n - stat) + STEP_BYTES_STATIC * stat
    peaks = measured_peaks()
    gbs = bytes_step / (ms / steps * 1e-3) / 1e9
    return {"workload": "core_shell-%d: FCC static core (90%%) + random-walk shell (10%%), d = 10 um, R = 10 um, "
                        "static-agent skip on, FP32 form" % w.n, "settings": st, "steps": steps,
            "warmup": warmup, "value": w.n * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "skipped_fraction": stat / w.n,
            "hbm": {"bytes_per_step_algorithmic": bytes_step, "achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"],
                    "frac": gbs / peaks["hbm_gbs"], "peak_source": peaks["_source"]},
            "phases_ms_per_step": {k: round(v[0] / 2, 4) for k, v in phases.items()},
            "counters_last_step": {k: c[k] for k in ("n_agents", "n_static", "n_candidates", "n_neighbors",
                                                     "n_contacts", "n_exact_fallback", "n_fp64_fixup")},
            "gpu_launches": c["kernels_launched"] - c0["kernels_launched"], "clocks": clk.summary()}


# ---------------------------------------------------------------- GPU arm
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "core_shell_leg":
        # the default line's core + shell leg on its own, at --n agents (for
        # profiling a smaller case of the same workload)
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(leg_core_shell(args, steps=args.steps, warmup=max(3, args.warmup), n=args.n)), flush=True)
        return 0
    if args.workload != "blobs":
        return run_other(args)

    import numpy as np
    import torch

    from paper_2301_06984_gb300 import bdm

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    w = workload(args.n)
    stream = torch.cuda.current_stream()
    curve = bdm.CURVE_HILBERT if args.curve == "hilbert" else bdm.CURVE_MORTON
    sim = bdm.Simulation.from_workload(w, precision="fp32", sort_every=args.sort_every, curve=curve)
    if args.lanes is not None:
        sim.set_force_kernel(args.lanes)
    sim.set_workload(w)
    if args.presort:
        sim.sort()
    sim.step(max(3, args.warmup))
    torch.cuda.synchronize()

    # ---- timed region: the production path (one CUDA graph per iteration)
    c0 = sim.counters()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_before = c0["n_agents"]
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1)
    c1 = sim.counters()
    launches = c1["kernels_launched"] - c0["kernels_launched"]
    updates = n_before * args.steps  # no agents are added in this workload
    ms, updates = reduce_over_ranks(ms, updates, dist, "cuda")
    value = updates / (ms * 1e-3)

    # ---- live per-kernel timing over a profiled pass of the same iteration
    kp = max(1, min(args.steps, 10))
    sim.profile_begin()
    cand = cont = agents = 0
    for _ in range(kp):
        sim.step(1)
        c = sim.counters()
        cand += c["n_candidates"]
        cont += c["n_contacts"]
        agents += c["n_agents"]
    phases = sim.profile_end()
    force_ms = phases["force"][0] / kp
    flops = (FLOP_MODEL[0] * cand + FLOP_MODEL[1] * cont) / kp
    flops_k = (FLOP_MODEL_KERNEL[0] * cand + FLOP_MODEL_KERNEL[1] * cont) / kp
    clocks = clk.summary()
    peak_alu = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = flops / (force_ms * 1e-3) / 1e12
    traffic, sha = committed_traffic(agents / kp)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    roofline = {"bound": "alu",
                "kernel": "force phase of the default hybrid launch: k_force<FP32,STEP> (2 to 32 lanes per agent, "
                          "following the agents left in a box) on bricks of 192 agents or more, k_force_sparse on "
                          "the lighter ones",
                "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s", "frac": achieved / peak_alu,
                "traffic": traffic,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (nominal, derived)",
                "flop_model": "%d per candidate pair, %d per contact" % FLOP_MODEL, "flops_per_launch": flops,
                "kernel_flop_model": {"per_candidate": FLOP_MODEL_KERNEL[0], "per_contact": FLOP_MODEL_KERNEL[1],
                                      "achieved": flops_k / (force_ms * 1e-3) / 1e12,
                                      "frac": flops_k / (force_ms * 1e-3) / 1e12 / peak_alu},
                "hbm_view": {"achieved_gbs": FORCE_BYTES_PER_AGENT * agents / kp / (force_ms * 1e-3) / 1e9,
                             "frac": FORCE_BYTES_PER_AGENT * agents / kp / (force_ms * 1e-3) / 1e9 / hbm,
                             "peak_gbs": hbm, "peak_source": peaks["_source"]}}
    phase_ms = {k: round(v[0] / kp, 4) for k, v in phases.items()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config(args),
        "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "phases_ms_per_step": phase_ms,
        "counters_last_step": {k: c1[k] for k in ("n_agents", "n_candidates", "n_neighbors", "n_contacts",
                                                  "n_exact_fallback", "n_fp64_fixup", "n_occupied_bricks",
                                                  "max_brick_agents")},
    }

    # ---- plain FP64 form on the same workload
    if not args.no_fp64:
        s64 = bdm.Simulation.from_workload(w, precision="fp64", sort_every=10)
        s64.set_workload(w)
        s64.step(1)
        k64 = max(1, min(3, args.steps))
        torch.cuda.synchronize()
        e0.record(stream)
        s64.step(k64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        line["fp64_form"] = {"value": args.n * k64 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64 / k64,
                             "steps": k64, "warmup": 1}
        s64.close()

    # ---- end to end through the C ABI with pinned host buffers
    if not args.no_e2e:
        n = args.n
        L = bdm.lib()
        hx = torch.empty(3 * n, dtype=torch.float64, pin_memory=True)
        hd = torch.empty(n, dtype=torch.float64, pin_memory=True)
        hx.numpy()[:] = np.concatenate([w.x, w.y, w.z])
        hd.numpy()[:] = w.diam
        se = bdm.Simulation.from_workload(w, precision="fp32", sort_every=10)
        ke = max(1, min(args.steps, 10))
        nout, st, nu = C.c_int64(), C.c_int64(), C.c_uint64()
        px, pd = C.c_void_p(hx.data_ptr()), C.c_void_p(hd.data_ptr())

        def e2e_step(t):
            se._check(L.bdm_set_agents(se._h, n, px, pd, None, None, None, None, t, n, bdm.BDM_HOST))
            se.step(1)
            se._check(L.bdm_get_agents(se._h, n, px, None, None, None, None, None, C.byref(nout), C.byref(st),
                                       C.byref(nu), bdm.BDM_HOST))

        for t in range(2):
            e2e_step(t)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for t in range(ke):
            e2e_step(2 + t)
        e1.record(stream)
        torch.cuda.synchronize()
        mse = e0.elapsed_time(e1)
        mse, upd = reduce_over_ranks(mse, n * ke, dist, "cuda")
        line["e2e"] = {"value": upd / (mse * 1e-3), "unit": UNIT,
                       "h2d_bytes_per_step": 32 * n, "d2h_bytes_per_step": 24 * n, "steps": ke}
        se.close()

    # ---- the other two throughput configurations, compact (N = 1 only)
    if world == 1 and not args.no_legs:
        line["ensemble_leg"] = leg_ensemble(args)
        line["core_shell_leg"] = leg_core_shell(args)

    # ---- FP64 oracle on the host cores (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_s = args.sample or 2_000_000
        v, dt, threads = cpu_baseline(n_s)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "2 iterations of the FP64 oracle over a %d-agent blob workload of the "
                                          "same density (lengths scaled by (n/1e7)^(1/3)), %.1f s, force loop on "
                                          "%d host threads (OpenMP timing build)" % (n_s, dt, threads)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
