"""Benchmark: particle-steps/s of the collision step at 2^24 particles on GB300.

Workload: the piston-shock tube (box 8 x 1 x 1, periodic in y and z, reflecting wall
at x = 0, piston from x = 8 inward at u_p = 2), N = 2^24, mean free path 0.02
(d0 from lambda = 1/(sqrt(2) n sigma)), dt = 0.1 lambda / sqrt(3), seed 2; synthetic
uniform positions and Maxwellian velocities (kT/m = 1).  The headline value is the
guarded-binary32 path; the binary64 GPU path is timed on the same workload beside it.

One JSON line on rank 0.  Under torchrun each rank runs an independent replica on
its own GPU (the method has no exchange step in this form); value = all ranks'
particle-steps / max over ranks of the timed region.

--impl reference times the CPU oracle (the plain binary64 definition) on a bounded
sample of the same workload: the 8 x 0.25 x 0.25 cross-section of the tube at the
same density (2^20 particles), one oracle step per benchmark step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import kmc_inputs as ki  # noqa: E402

METRIC = "particle-steps/s at 2^24, guarded-FP32 vs FP64 GPU; serve p50/p99 latency"
UNIT = "particle-steps/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# binary32 lanes x 2 flop per FMA x SM count x maximum SM clock (unit counts and
# clocks of the part: 152 SMs, 128 FP32 lanes per SM, 2070 MHz)
ALU_FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# flops of one binary32 pair pre-test: r (3), v (3), |r|^2 (5), |v|^2 (5), bound (2)
FLOPS_PER_PAIR_TEST = 18
# algorithmic bytes of the sort per particle: read the binary64 state and id/last
# (56), write it permuted (56), write the cell-local binary32 mirror (24) and the key (4)
SORT_BYTES_PER_PARTICLE = 140
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal (fractions against it beside the measured peak)


def headline_setup(n: int):
    return ki.piston_setup(n=n, seed=2, profile_bins=256, profile_every=100)


def sample_setup(box_yz: float = 0.25):
    """Cross-section sample of the headline tube: same density, box_yz^2 of the
    particles (1/16 at 0.25)."""
    n_full = 1 << 24
    full = headline_setup(n_full)
    n = int(round(n_full * box_yz * box_yz))
    s = ki.piston_setup(n=n, seed=2, box=(8.0, box_yz, box_yz), profile_bins=0,
                        profile_every=0)
    return s.with_(d0=full.d0, dt=full.dt, name="piston_tube_cross_section")


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def wait_first_sample(self, timeout: float = 3.0):
        t0 = time.time()
        while self.proc and time.time() - t0 < timeout:
            try:
                if os.path.getsize(self.path) > 0:
                    return
            except OSError:
                pass
            time.sleep(0.02)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
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
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x: float, world: int, device=None) -> float:
    """Max over ranks (timing only: no simulation data crosses ranks)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job rate: units all ranks processed / slowest rank's time."""
    return world * units_per_rank / (max_ms / 1e3)


def source_sha(path):
    h = hashlib.sha256()
    with open(path, "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_file: str):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, or None if
    the kernel source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(p)).get(kernel_file)
        src = os.path.join(ROOT, "paper_1310_3437_gb300", "csrc", kernel_file)
        if rec and rec.get("source_sha") == source_sha(src):
            return rec
    except Exception:
        pass
    return None


# --------------------------------------------------------------------------- #
def oracle_sample_rate(max_seconds: float, warmup: int = 0, steps_cap: int = 50,
                       threads: int = 0, box_yz: float = 0.25):
    """Time the oracle on a cross-section sample; returns (rate, steps, seconds,
    threads, setup).  threads = 0: all host threads."""
    import oracle

    s = sample_setup(box_yz)
    st = oracle.State(ki.initial_state(s))
    for k in range(warmup):
        oracle.step(s, st, k, threads=threads)
    t0 = time.perf_counter()
    done = 0
    while done < steps_cap:
        oracle.step(s, st, warmup + done, threads=threads)
        done += 1
        if time.perf_counter() - t0 >= max_seconds:
            break
    dt = time.perf_counter() - t0
    return s.n * done / dt, done, dt, (threads or oracle.max_threads()), s


def run_serving(args, stream, dev):
    """Serving stream at ~70% load: calibrate the aggregate throughput S on a batch of
    requests, then send Poisson arrivals at rate 0.7 S / W (W = mean particle-steps of
    a request) and report latency percentiles and aggregate throughput."""
    import torch

    import paper_1310_3437_gb300 as kmc
    from paper_1310_3437_gb300.serve import Request, Server, summarize

    n_lo, n_hi = 1 << 14, args.serve_n_hi
    st_lo, st_hi = args.serve_steps_lo, args.serve_steps_hi
    setups = ki.serving_requests(args.serve_requests + 16, master_seed=7, n_lo=n_lo, n_hi=n_hi,
                                 steps_lo=st_lo, steps_hi=st_hi)
    cal, rest = setups[:16], setups[16:]
    # calibration: 16 requests admitted at once
    def req(k, q, arrival):
        if args.serve_host_init:
            return Request(rid=k, setup=q, steps=q.steps, arrival=arrival,
                           arrays=(lambda q=q: ki.initial_state(q)))
        return Request(rid=k, setup=q, steps=q.steps, arrival=arrival, init=ki.init_spec(q))

    reqs = [req(k, q, 0.0) for k, q in enumerate(cal)]
    server = Server(budget_bytes=args.serve_budget_gb * 1e9, keep_state=False,
                    stream=stream.cuda_stream)
    done, wall = server.run(reqs)
    S = summarize(done, wall)["particle_steps_per_s"]
    W = ki.mean_loguniform(n_lo, n_hi) * 0.5 * (st_lo + st_hi)
    rate = 0.7 * S / W
    rng = np.random.default_rng(7)
    t = np.cumsum(rng.exponential(1.0 / rate, size=len(rest)))
    reqs = [req(k, q, float(t[k])) for k, q in enumerate(rest)]
    server = Server(budget_bytes=args.serve_budget_gb * 1e9, keep_state=True,
                    stream=stream.cuda_stream)
    done, wall = server.run(reqs)
    sm = summarize(done, wall)
    tests = sum(c["pair_tests"] for r in done for c in r.counts)
    recs = sum(len(r.counts) for r in done)
    if recs != sum(int(r.steps) for r in done):
        raise RuntimeError(f"serving: {recs} step records for {sum(int(r.steps) for r in done)} steps")
    achieved = tests * FLOPS_PER_PAIR_TEST / wall / 1e12
    return {
        "pair_tests_per_s": tests / wall,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / ALU_FP32_PEAK_TFLOPS,
                     "note": "pair tests of all requests over the stream's wall time "
                             "(idle gaps between arrivals included)"},
        "p50_latency_ms": sm["p50_latency_s"] * 1e3, "p99_latency_ms": sm["p99_latency_s"] * 1e3,
        "mean_latency_ms": sm["mean_latency_s"] * 1e3,
        "particle_steps_per_s": sm["particle_steps_per_s"], "requests": sm["requests"],
        "wall_s": sm["wall_s"], "load": 0.7, "arrival_rate_per_s": rate,
        "calibration_particle_steps_per_s": S, "budget_gb": args.serve_budget_gb,
        "mix": f"equilibrium boxes and piston tubes, N log-uniform [{n_lo}, {n_hi}], steps "
               f"U[{st_lo}, {st_hi}], guarded FP32, SplitMix64 seeds from master seed 7",
        "latency": "arrival -> final state and step counts on the host; bursts of at most "
                   "16 group steps end when the live request closest to its end is done",
        "init": ("NumPy arrays generated on the host at admission" if args.serve_host_init
                 else "state drawn on the device at admission (sim_create_init)"),
    }


def run_paper_workloads(args, stream, dev):
    """The paper's own timing workloads at their stated sizes (Fig. 1: 10^8 particles,
    3D; Fig. 3: 4 x 10^7 particles, 2D), equal speeds in random directions, each state
    drawn on the device; guarded FP32, CUDA-event timing of K steps after warm-up."""
    import torch

    import paper_1310_3437_gb300 as kmc

    out = {}
    for fig, name in ((1, "fig1_3d_equal_speed_n1e8"), (3, "fig3_2d_equal_speed_n4e7")):
        setup = ki.paper_timing_setup(fig)
        params = kmc.params_from_setup(setup, precision=kmc.KMC_GUARDED_FP32)
        sim = kmc.Simulation(params, init=ki.init_spec(setup), stream=stream.cuda_stream)
        sim.step(3).sync()
        sim.counts()
        k = args.paper_steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(k)
        e1.record(stream)
        e1.synchronize()
        sim.sync()
        ms = e0.elapsed_time(e1)
        counts = sim.counts()
        cells = counts[-1]["cells"] if counts else 0
        out[name] = {
            "n": setup.n, "steps": k, "ms_per_step": ms / k,
            "particle_steps_per_s": setup.n * k / (ms / 1e3),
            "collisions_per_step": sum(c["collisions"] for c in counts) / max(1, len(counts)),
            "particles_per_cell": setup.n / cells if cells else None,
            "d0": setup.d0, "dt": setup.dt, "planar": setup.planar,
        }
        sim.close()
        torch.cuda.synchronize(dev)
    return out


def run_ensemble(args, stream):
    """Batched ensemble: 256 independent runs of uneven size (N log-uniform in
    [2^12, 2^18], equilibrium boxes and piston tubes) stepped as one group: one launch
    per kernel per step for all runs, the step captured in a CUDA graph.  Reports the
    pair tests beside the particle-steps: the equilibrium boxes keep n sigma of the
    4096-particle box, so their cells hold up to ~360 particles and a particle-step
    costs up to ~10^4 pair tests there, against ~20 in the tube."""
    import torch

    import paper_1310_3437_gb300 as kmc

    setups = ki.ensemble_setups(count=256, steps=args.ensemble_steps)
    sims = [kmc.Simulation(kmc.params_from_setup(q, precision=kmc.KMC_GUARDED_FP32,
                                                 history_cap=args.ensemble_steps + 64),
                           ki.initial_state(q), stream=stream.cuda_stream) for q in setups]
    g = kmc.Group(sims, stream=stream.cuda_stream)
    warm = 3
    for q in sims:
        g.budget(q, warm + args.ensemble_steps)
    g.step(warm)
    g.sync()
    for q in sims:
        q.counts()
    l0 = sims[0].launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(args.ensemble_steps)
    e1.record(stream)
    e1.synchronize()
    g.sync()
    ms = e0.elapsed_time(e1)
    launches = sims[0].launches() - l0
    total_n = sum(q.n for q in setups)
    tests = {"box": 0, "tube": 0}
    psteps = {"box": 0, "tube": 0}
    for q, sim in zip(setups, sims):
        recs = sim.counts()
        if len(recs) != args.ensemble_steps:
            raise RuntimeError(f"ensemble member {q.name}: {len(recs)} step records, "
                               f"expected {args.ensemble_steps}")
        kind = "box" if q.name.startswith("equilibrium") else "tube"
        tests[kind] += sum(c["pair_tests"] for c in recs)
        psteps[kind] += q.n * len(recs)
    secs = ms / 1e3
    all_tests = tests["box"] + tests["tube"]
    achieved = all_tests * FLOPS_PER_PAIR_TEST / secs / 1e12
    out = {"runs": len(setups), "particles": total_n, "steps": args.ensemble_steps,
           "particle_steps_per_s": total_n * args.ensemble_steps / secs,
           "ms_per_group_step": ms / args.ensemble_steps,
           "kernel_launches_per_group_step": launches / args.ensemble_steps,
           "pair_tests_per_s": all_tests / secs,
           "pair_tests_per_particle_step": {k: tests[k] / max(1, psteps[k]) for k in tests},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_FP32_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": achieved / ALU_FP32_PEAK_TFLOPS,
                        "flops_per_pair_test": FLOPS_PER_PAIR_TEST,
                        "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz"},
           "mix": "seeds 1000-1255, N log-uniform [2^12, 2^18], even: equilibrium box, "
                  "odd: piston tube with u_p in [1, 3]; guarded FP32; one CUDA graph per step"}
    g.close()
    for q in sims:
        q.close()
    return out


def run_domains(args, stream):
    """The paper's domain decomposition (Sec. 4) on one GPU: the 2^22-particle piston
    tube (the 2^20 tube's density in an 8 x 2 x 2 box) as 1 and as 4 x slabs, guarded
    binary32, the same steps; the decomposition changes the work, never the result
    (the states are compared)."""
    import torch

    import paper_1310_3437_gb300 as kmc

    n = args.domains_n
    setup = ki.piston_setup(n=n, seed=2, box=(8.0, 2.0, 2.0), profile_bins=0, profile_every=0)
    arrays = ki.initial_state(setup)
    out = {"n": n, "box": list(setup.box), "steps": args.domains_steps}
    states = {}
    for P in (1, 4):
        params = kmc.params_from_setup(setup, precision=kmc.KMC_GUARDED_FP32)
        sim = kmc.Simulation(params, arrays, stream=stream.cuda_stream, domains=P)
        sim.step(2).sync()
        sim.counts()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(args.domains_steps)
        e1.record(stream)
        e1.synchronize()
        sim.sync()
        ms = e0.elapsed_time(e1) / args.domains_steps
        owned, ghosts = sim.domains()
        out[f"p{P}"] = {"ms_per_step": ms, "particle_steps_per_s": n / (ms / 1e3),
                        "owned": owned.tolist(), "ghosts": ghosts.tolist()}
        st, last = sim.state()
        states[P] = [a.copy() for a in st] + [last.copy()]
        sim.close()
    out["identical_states"] = all(np.array_equal(a.view(np.uint8), b.view(np.uint8))
                                  for a, b in zip(states[1], states[4]))
    if not out["identical_states"]:
        raise RuntimeError("domain decomposition: 4 slabs differ from 1")
    return out


def run_launch_overhead(stream):
    """Per-step cost of the launch sequence itself: a 4096-particle box (launch-bound)
    replays its step graph 200 times; us per step and per kernel launch bound what a
    single persistent kernel could save over the graph of per-phase kernels."""
    import torch

    import paper_1310_3437_gb300 as kmc

    setup = ki.equilibrium_setup(n=4096, seed=1)
    sim = kmc.Simulation(kmc.params_from_setup(setup, precision=kmc.KMC_GUARDED_FP32),
                         ki.initial_state(setup), stream=stream.cuda_stream)
    sim.step(5).sync()
    l0 = sim.launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    steps = 200
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    sim.sync()
    per_step = (sim.launches() - l0 - 1) / steps
    us = e0.elapsed_time(e1) * 1e3 / steps
    sim.close()
    return {"n": setup.n, "steps": steps, "us_per_step": us, "launches_per_step": per_step,
            "us_per_launch": us / per_step if per_step else None,
            "note": "graph replay of one step's kernels on a launch-bound 4096-particle box"}


def run_blast(args, stream, dev):
    """The spherical blast at full size (2^27 particles; hot ball of radius 0.1 at 8x
    the background density and 100x its temperature, background lambda 0.005), state
    drawn on the device: guarded binary32 for K steps after one, binary64 for one step
    after one (binary64 runs at about 1/64 of the binary32 rate here), both with pair
    tests, cells and the speed split's fast-particle share."""
    import torch

    import paper_1310_3437_gb300 as kmc

    setup = ki.blast_setup(n=args.blast_n, seed=3)
    out = {"n": setup.n, "d0": setup.d0, "dt": setup.dt, "n_hot": setup.extra["n_hot"]}
    for prec, name, k in ((kmc.KMC_GUARDED_FP32, "fp32", args.blast_steps),
                          (kmc.KMC_FP64, "fp64", args.blast_fp64_steps)):
        if k <= 0:
            continue
        params = kmc.params_from_setup(setup, precision=prec)
        sim = kmc.Simulation(params, init=ki.init_spec(setup), stream=stream.cuda_stream)
        sim.step(1).sync()  # grows the pair buffer if the first step needs more
        sim.counts()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(k)
        e1.record(stream)
        e1.synchronize()
        l1 = sim.launches()
        sim.sync()
        recs = sim.counts()
        if len(recs) != k or sim.launches() != l1:
            raise RuntimeError(f"blast {name}: {len(recs)} step records for {k} steps")
        ms = e0.elapsed_time(e1)
        out[name] = {
            "steps": k, "ms_per_step": ms / k, "particle_steps_per_s": setup.n * k / (ms / 1e3),
            "pair_tests_per_step": float(np.mean([c["pair_tests"] for c in recs])),
            "fast_pair_tests_per_step": float(np.mean([c["fast_tests"] for c in recs])),
            "cells": recs[-1]["cells"],
            "candidate_pairs_per_step": float(np.mean([c["edges"] for c in recs])),
            "collisions_per_step": float(np.mean([c["collisions"] for c in recs]))}
        sim.close()
        torch.cuda.synchronize(dev)
    if "fp32" in out and "fp64" in out:
        out["speedup_fp32_over_fp64"] = out["fp32"]["particle_steps_per_s"] / \
            out["fp64"]["particle_steps_per_s"]
    return out


def run_reference(args):
    world, rank, local = dist_info()
    if rank != 0:
        return
    import oracle

    s = sample_setup()
    st = oracle.State(ki.initial_state(s))
    for k in range(args.warmup):
        oracle.step(s, st, k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.step(s, st, args.warmup + k)
    dt = time.perf_counter() - t0
    rate = s.n * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"piston_tube_n{1 << 24}", "sample": "8x0.25x0.25 cross-section",
                   "n_sample": s.n},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle",
                         "sample": f"{s.n} particles (8x0.25x0.25 cross-section at the same "
                                   f"density), {args.steps} steps after {args.warmup}"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
def run_gpu(args):
    import torch

    import paper_1310_3437_gb300 as kmc

    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    if args.workload == "sample":
        setup = sample_setup()
        n = setup.n
    else:
        n = args.n
        setup = headline_setup(n)
    if world > 1:
        setup = setup.with_(seed=setup.seed + rank)
    t_gen = time.perf_counter()
    arrays = ki.initial_state(setup)
    host_generate_s = time.perf_counter() - t_gen
    dev_arrays = [torch.from_numpy(a).to(dev) for a in arrays]

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return reduce_max(x, world, dev)

    # a dedicated stream: the library launches on it and the events are recorded on it
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    knobs = {"search_kernel": 0, "stencil": 1, "cell_scale": 1.0, "split_min_occ": 0.0}
    tuning = None
    if not args.no_tune:
        from paper_1310_3437_gb300.tune import Autotuner
        tuner = Autotuner(steps=3, warmup=max(2, args.warmup))
        best = tuner.choose(setup, dev_arrays, kmc.KMC_GUARDED_FP32, stream=stream)
        knobs = {k: best[k] for k in knobs}
        tuning = {"chosen": best, "trials": next(iter(tuner.trials.values()))}

    def check_window(sim, first_step, steps, launches_before_sync):
        """The timed steps ran: one step record per step, consecutive from first_step,
        and nothing left for sim_sync to re-run (an overflowing pair buffer skips the
        remaining steps on the device and would move their work out of the window)."""
        recs = sim.counts()
        got = [c["step"] for c in recs]
        if got != list(range(first_step, first_step + steps)):
            raise RuntimeError(f"timed window did not run its {steps} steps: step records "
                               f"{got[:3]}..{got[-3:]} ({len(got)} records)")
        sim.sync()
        if sim.launches() != launches_before_sync:
            raise RuntimeError("sim_sync re-ran steps of the timed window (pair-buffer overflow)")
        return recs

    def timed_run(precision, warm, steps, sample_clocks=False, kn=None, min_ms=0.0,
                  max_windows=1):
        """warm untimed steps, then windows of exactly `steps` steps, each bracketed by
        a barrier and a device synchronisation and timed with CUDA events on the
        simulation's stream.  With more than one window, every window restarts from
        the same state (the one after the warm-up, one more untimed step to capture
        the step's graph), so the windows time the same steps of the same run and the
        median is not shifted by the shock's growth; windows repeat until min_ms of
        timed work (the same number on every rank).  Returns per-window ms (max over
        ranks) and the last window's simulation."""
        kn = knobs if kn is None else kn
        params = kmc.params_from_setup(setup, precision=precision, **kn)
        sim = kmc.Simulation(params, dev_arrays, stream=stream.cuda_stream)
        sim.step(warm).sync()
        sim.counts()
        snap = None
        if max_windows > 1:
            snap = torch.empty(52 * n, dtype=torch.uint8, device=dev)
            sim.state_device(snap)
            torch.cuda.synchronize(dev)
            sim.close()
            f = snap[: 48 * n].view(torch.float64).view(6, n)
            cols = [f[k] for k in range(6)]
            last = snap[48 * n:].view(torch.int32)

        def window_sim():
            if snap is None:
                return sim
            q = kmc.Simulation(kmc.params_from_setup(setup, precision=precision, step0=warm, **kn),
                               cols, last=last, stream=stream.cuda_stream)
            q.step(1).sync()
            q.counts()
            return q

        sampler = ClockSampler(dev.index or 0) if sample_clocks else None
        barrier()
        if sampler:
            sampler.start()
            sampler.wait_first_sample()
        windows, counts, launches = [], [], 0
        nwin = 1
        cur = None
        while len(windows) < nwin:
            if cur is not None and cur is not sim:
                cur.close()
            cur = window_sim()
            step_next = cur.step_index()
            l0 = cur.launches()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cur.step(steps)
            e1.record(stream)
            e1.synchronize()
            barrier()
            windows.append(max_over_ranks(e0.elapsed_time(e1)))
            l1 = cur.launches()
            launches += l1 - l0
            counts += check_window(cur, step_next, steps, l1)
            if len(windows) == 1:
                # the same on every rank: derived from the max-over-ranks time
                nwin = max(1, min(max_windows, math.ceil(min_ms / max(windows[0], 1e-3))))
        clocks = sampler.stop() if sampler else None
        return cur, windows, counts, launches, clocks

    def precision_check(steps):
        """Guarded binary32 (the timed knobs) and binary64 from the same state, one step
        at a time: sorted candidate-pair lists, partners and step counts compared in
        every step, the whole state after the last (Sec. 2: the criteria and the
        closest partner fix the list, so the pre-test precision must not change it)."""
        a = kmc.Simulation(kmc.params_from_setup(setup, precision=kmc.KMC_GUARDED_FP32, **knobs),
                           dev_arrays, stream=stream.cuda_stream)
        b = kmc.Simulation(kmc.params_from_setup(setup, precision=kmc.KMC_FP64), dev_arrays,
                           stream=stream.cuda_stream)
        res = {"steps": steps, "edges_identical": True, "partners_identical": True,
               "counts_identical": True, "edge_sha256_16": []}
        for _ in range(steps):
            a.step(1).sync()
            b.step(1).sync()
            ea, eb = a.edges(), b.edges()
            ha = hashlib.sha256(np.ascontiguousarray(ea).tobytes()).hexdigest()[:16]
            hb = hashlib.sha256(np.ascontiguousarray(eb).tobytes()).hexdigest()[:16]
            res["edge_sha256_16"].append(ha)
            res["edges_identical"] &= ha == hb and ea.shape == eb.shape
            res["partners_identical"] &= bool(np.array_equal(a.partners(), b.partners()))
            ca, cb = a.counts(), b.counts()
            res["counts_identical"] &= [(c["collisions"], c["edges"], c["round_pairs"]) for c in ca] == \
                [(c["collisions"], c["edges"], c["round_pairs"]) for c in cb]
        ba = torch.empty(52 * n, dtype=torch.uint8, device=dev)
        bb = torch.empty_like(ba)
        a.state_device(ba)
        b.state_device(bb)
        torch.cuda.synchronize(dev)
        res["state_identical"] = bool(torch.equal(ba, bb))
        res["candidate_pairs_per_step"] = float(eb.shape[0])
        a.close()
        b.close()
        del ba, bb
        return res

    # ---- guarded binary32 (headline) ----
    sim32, windows32, counts32, launches32, clocks = timed_run(
        kmc.KMC_GUARDED_FP32, args.warmup, args.steps, sample_clocks=True,
        min_ms=args.min_timed_s * 1e3, max_windows=args.max_windows)
    ms32 = float(np.median(windows32))
    value = aggregate_rate(n * args.steps, world, ms32)
    # per-phase times of the next steps, CUDA events on the simulation's stream
    tsteps = max(3, min(args.steps, 10))
    sim32.set_timing(True)
    sim32.step(tsteps).sync()
    ph = sim32.phase_ms()
    tcounts = sim32.counts()
    sim32.set_timing(False)
    tests = np.mean([c["pair_tests"] for c in tcounts]) if tcounts else 0.0
    fast_tests = np.mean([c["fast_tests"] for c in tcounts]) if tcounts else 0.0
    slow_tests = tests - fast_tests
    search_ms = ph["search"] / max(1, ph["steps"])
    slow_ms = ph["search_slow"] / max(1, ph["steps"])
    sort_ms = ph["sort"] / max(1, ph["steps"])
    edges_mean = float(np.mean([c["edges"] for c in counts32])) if counts32 else 0.0
    coll_mean = float(np.mean([c["collisions"] for c in counts32])) if counts32 else 0.0
    sim32.close()

    # ---- binary64 path on the same workload (fewer steps: ~70x slower arithmetic) ----
    fp64 = None
    check = None
    if not args.skip_fp64:
        k64 = max(1, min(args.steps, args.fp64_steps))
        # the binary64 path with its own defaults (the tuner tunes the binary32 path; a
        # binary32-only kernel choice would not carry over)
        kn64 = {"search_kernel": 0, "stencil": 1, "cell_scale": 1.0, "split_min_occ": 0.0}
        sim64, win64, counts64, _, _ = timed_run(kmc.KMC_FP64, args.warmup, k64, kn=kn64)
        v64 = world * n * k64 / (win64[0] / 1e3)
        fp64 = {"value": v64, "unit": UNIT, "steps": k64, "ms_per_step": win64[0] / k64}
        sim64.close()
        check = precision_check(args.check_steps)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.skip_e2e:
        pinned = [torch.from_numpy(a).pin_memory() for a in arrays]
        out = torch.empty(52 * n, dtype=torch.uint8).pin_memory()
        ke = args.steps
        barrier()
        t0 = time.perf_counter()
        params = kmc.params_from_setup(setup, precision=kmc.KMC_GUARDED_FP32, **knobs)
        sim = kmc.Simulation(params, pinned, stream=stream.cuda_stream)
        sim.step(ke)
        kmc.sim_observe(sim.handle, kmc.KMC_OBS_STATE, out.data_ptr(), out.numel())
        torch.cuda.synchronize(dev)
        te = max_over_ranks(time.perf_counter() - t0)
        sim.close()
        e2e = {"value": world * n * ke / te, "unit": UNIT,
               "h2d_bytes_per_step": 48 * n / ke, "d2h_bytes_per_step": 52 * n / ke,
               "job": f"create from pinned host arrays, {ke} steps, state read back"}

    # ---- end to end with the state drawn on the device (no host arrays) ----
    e2e_dinit = None
    if not args.skip_e2e:
        out = torch.empty(52 * n, dtype=torch.uint8).pin_memory()
        ke = args.steps
        spec = ki.init_spec(setup)
        params = kmc.params_from_setup(setup, precision=kmc.KMC_GUARDED_FP32, **knobs)
        barrier()
        t0 = time.perf_counter()
        sim = kmc.Simulation(params, init=spec, stream=stream.cuda_stream)
        torch.cuda.synchronize(dev)
        tc = time.perf_counter() - t0
        sim.step(ke)
        kmc.sim_observe(sim.handle, kmc.KMC_OBS_STATE, out.data_ptr(), out.numel())
        torch.cuda.synchronize(dev)
        te = max_over_ranks(time.perf_counter() - t0)
        sim.close()
        e2e_dinit = {"value": world * n * ke / te, "unit": UNIT, "h2d_bytes_per_step": 0,
                     "d2h_bytes_per_step": 52 * n / ke, "create_ms": tc * 1e3,
                     "host_generate_ms": host_generate_s * 1e3,
                     "job": f"sim_create_init (state drawn on the device), {ke} steps, state "
                            f"read back; host_generate_ms: NumPy generation of the same "
                            f"workload's arrays, which sim_create_init replaces"}

    serve = None
    if not args.skip_serve and rank == 0:
        serve = run_serving(args, stream, dev)
    ensemble = None
    if not args.skip_ensemble and rank == 0:
        ensemble = run_ensemble(args, stream)
    paper = None
    if not args.skip_paper and rank == 0:
        paper = run_paper_workloads(args, stream, dev)
    blast = None
    if not args.skip_blast and rank == 0:
        blast = run_blast(args, stream, dev)
    launch_overhead = run_launch_overhead(stream) if rank == 0 and not args.skip_launch_probe else None
    domains = run_domains(args, stream) if (rank == 0 and not args.skip_domains) else None

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    pk, pk_kind = peaks()
    # dominant kernel: the slow-population search (the row search at this workload),
    # timed alone with CUDA events on the simulation's stream
    achieved_tflops = slow_tests * FLOPS_PER_PAIR_TEST / (slow_ms / 1e3) / 1e12 if slow_ms > 0 else 0.0
    traffic = ncu_traffic("kmc_search.cu")
    roofline = {
        "kernel": "k_search_rows32 (slow-population search, guarded binary32)",
        "bound": "alu",
        "achieved": achieved_tflops,
        "peak": ALU_FP32_PEAK_TFLOPS,
        "unit": "TFLOP/s",
        "frac": achieved_tflops / ALU_FP32_PEAK_TFLOPS,
        "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz",
        "traffic": (traffic["dram_bytes_per_particle"] * n) if traffic else None,
        # the same kernel's HBM fraction beside the ALU one: its measured DRAM bytes per
        # launch over the launch time, against the measured copy bandwidth
        "hbm_frac": (traffic["dram_bytes_per_particle"] * n / (slow_ms / 1e3) / 1e9 / pk["hbm_gbs"])
                    if traffic and slow_ms > 0 else None,
        # what bounds it: the share of issue slots used (ncu, same kernel source)
        "issue_active_pct": traffic.get("issue_active_pct") if traffic else None,
        "flops_per_pair_test": FLOPS_PER_PAIR_TEST,
        "pair_tests_per_launch": float(slow_tests),
        "launch_ms": slow_ms,
    }
    search_phase = {"ms": search_ms, "pair_tests": float(tests), "fast_pair_tests": float(fast_tests),
                    "pair_tests_per_s": tests / (search_ms / 1e3) if search_ms > 0 else None,
                    "kernels": "slow-population search + k_search_fast (fast particles)"}
    sort_gbs = SORT_BYTES_PER_PARTICLE * n / (sort_ms / 1e3) / 1e9 if sort_ms > 0 else 0.0
    roofline_sort = {
        "kernel": "sort phase (k_count, scans, k_scatter, k_gather)",
        "bound": "hbm", "achieved": sort_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
        "frac": sort_gbs / pk["hbm_gbs"], "peak_source": f"{pk_kind} hbm_gbs",
        "frac_of_nominal": sort_gbs / HBM_NOMINAL_GBS,
        "bytes_per_particle": SORT_BYTES_PER_PARTICLE, "launch_ms": sort_ms,
    }
    # the counting sort's key space: every key's count is read, its start written and
    # the count cleared (12 B per key; the fast population, when split, has a second
    # copy of the keys) -- reported beside the per-particle figure, not folded into it
    if counts32 and sort_ms > 0:
        keys = float(np.mean([c["cells"] * (2 if c["fast_tests"] else 1) for c in counts32]))
        kb = SORT_BYTES_PER_PARTICLE * n + 12.0 * keys
        roofline_sort["key_space"] = {
            "keys": keys, "bytes_per_key": 12,
            "achieved_incl_keys": kb / (sort_ms / 1e3) / 1e9,
            "frac_incl_keys": kb / (sort_ms / 1e3) / 1e9 / pk["hbm_gbs"]}

    cpu = None
    cpu1 = None
    if not args.skip_cpu and world >= 1:
        rate, done, secs, threads, s = oracle_sample_rate(args.cpu_seconds, warmup=0)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{s.n} particles (8x0.25x0.25 cross-section of the tube, same "
                         f"density), {done} oracle steps from t=0, {secs:.1f} s"}
        rate1, done1, secs1, _, s1 = oracle_sample_rate(args.cpu_seconds / 2, warmup=0,
                                                        threads=1, box_yz=0.125)
        cpu1 = {"value": rate1, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"{s1.n} particles (8x0.125x0.125 cross-section of the tube, same "
                          f"density), {done1} oracle steps from t=0 on one thread, "
                          f"{secs1:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 pair tests + f64 state",
        "data": "synthetic",
        "config": {"workload": f"piston_tube_n{n}" if args.workload == "tube" else
                   f"piston_tube_cross_section_n{n}", "n": n, "box": list(setup.box),
                   "lambda": 0.02, "d0": setup.d0, "dt": setup.dt, "u_p": setup.piston_u,
                   "precision": "guarded-fp32", "l2": "inputs larger than L2 (state ~1.9 GB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "timed_windows": {"windows": len(windows32), "steps_per_window": args.steps,
                          "first_step": args.warmup + 1 if len(windows32) > 1 else args.warmup,
                          "ms_per_window": windows32, "reported": "median window",
                          "restart": "every window restarts from the state after the warm-up "
                                     "(and one untimed step): the same steps of the same run",
                          "checked": "each window left exactly its steps' records, "
                                     "consecutive, with no re-run at sync"},
        "fp64": fp64,
        "speedup_fp32_over_fp64": (value / fp64["value"]) if fp64 else None,
        "fp32_fp64_edges_identical": (bool(check["edges_identical"] and check["partners_identical"]
                                           and check["counts_identical"] and check["state_identical"])
                                      if check else None),
        "precision_check": check,
        "roofline": roofline,
        "roofline_sort": roofline_sort,
        "phase_ms_per_step": {k: ph[k] / max(1, ph["steps"]) for k in ("sort", "search", "match", "push")},
        "pair_tests_per_s": slow_tests / (slow_ms / 1e3) if slow_ms > 0 else None,
        "search_phase": search_phase,
        "candidate_pairs_per_step": edges_mean, "collisions_per_step": coll_mean,
        "cpu_baseline": cpu,
        "cpu_baseline_1core": cpu1,
        "e2e": e2e,
        "e2e_device_init": e2e_dinit,
        "serve": serve,
        "ensemble": ensemble,
        "paper_workloads": paper,
        "blast": blast,
        "launch_overhead": launch_overhead,
        "domains": domains,
        "tuning": tuning,
        "gpu_launches": int(launches32),
        "gpu_launches_per_window": int(launches32) // max(1, len(windows32)),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if check is not None and not line["fp32_fp64_edges_identical"]:
        raise SystemExit("guarded binary32 and binary64 runs differ (precision_check)")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--workload", default="tube", choices=["tube", "sample"],
                    help="tube: the 2^24 piston tube; sample: its 8x0.25x0.25 cross-section "
                         "(2^20 particles, same density), for profiling")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--check-steps", type=int, default=8,
                    help="steps of the binary32 vs binary64 pair-list comparison")
    ap.add_argument("--min-timed-s", type=float, default=2.0,
                    help="repeat the K-step timed window until this much timed work")
    ap.add_argument("--max-windows", type=int, default=40)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--serve-host-init", action="store_true",
                    help="serving requests carry host arrays instead of a device-init descriptor")
    ap.add_argument("--skip-ensemble", action="store_true")
    ap.add_argument("--skip-launch-probe", action="store_true",
                    help="skip the launch-overhead probe (200 graph replays of a 4096-particle box)")
    ap.add_argument("--skip-paper", action="store_true",
                    help="skip the paper's timing workloads (10^8 3D, 4e7 2D particles)")
    ap.add_argument("--paper-steps", type=int, default=10)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--ensemble-steps", type=int, default=500)
    ap.add_argument("--skip-blast", action="store_true",
                    help="skip the full-size spherical blast (2^27 particles)")
    ap.add_argument("--blast-n", type=int, default=1 << 27)
    ap.add_argument("--skip-domains", action="store_true",
                    help="skip the domain decomposition leg (2^22 tube as 1 and 4 slabs)")
    ap.add_argument("--domains-n", type=int, default=1 << 22)
    ap.add_argument("--domains-steps", type=int, default=10)
    ap.add_argument("--blast-steps", type=int, default=5)
    ap.add_argument("--blast-fp64-steps", type=int, default=1)
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests of the serving stream (the full stream is 10000)")
    ap.add_argument("--serve-n-hi", type=int, default=1 << 22)
    ap.add_argument("--serve-steps-lo", type=int, default=100)
    ap.add_argument("--serve-steps-hi", type=int, default=2000)
    ap.add_argument("--serve-budget-gb", type=float, default=160.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
