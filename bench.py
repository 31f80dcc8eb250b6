#!/usr/bin/env python3
"""Throughput of the sputtered-atom transport hot path on GB300.

A step transports the whole quaternary co-sputter workload (Ni/Pd/Pt/Ru,
4 cathodes tilted 30 deg confocal at 120 mm, 1e7 particles each, Ar 0.5 Pa,
300 K, 100 mm wafer with 200x200 int64 counts + fp64 energy per cathode)
through libsput.so.  The metric is particle-collisions/s (and landed
particles/s), whole job, inputs resident in HBM; ``e2e`` is the same metric
through the host-buffer entry point with the host<->device copies inside.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The JSON line also carries, each measured in this run:
  * ``roofline``: algorithmic lane-ops of the method per launch (a work model
    counted from the run's own flights, partner attempts, collisions, particles
    and the geometry's primitives) over the kernel's CUDA-event time, against
    the FP32 FMA lane-op rate measured by ``sput_microbench``;
  * ``peaks``: the measured FMA, MUFU, Philox and L2-reduction throughputs;
  * ``atomics``: the landing tally's L2 reductions against their measured rate;
  * ``sub``: the other workloads (single Ni 50x50 int32 replayed from a CUDA
    graph, the 512-instance sweep batched vs one launch per instance, the large
    shielded chamber at 3 Pa, and the likelihood-ratio gradient of a 342-point
    composition map against common-random-number finite differences at equal
    standard error).

With N > 1 (torchrun) every rank transports its own replica of the workload
(distinct seeds, no data-path collective: particles are independent) and the
job value is the sum over ranks divided by the slowest rank's time.
``--impl reference`` times the FP64 CPU oracle on bounded samples of the same
workload (rank 0 only).
"""

from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-collisions/sec and landed particles/sec on 1 GB300 vs oracle; roofline fraction"
UNIT = "collisions/s"
WORKLOADS = {
    "quaternary": ("quaternary co-sputter Ni/Pd/Pt/Ru, 4 cathodes tilted 30 deg confocal at 120 mm, "
                   "4 x 1e7 particles, Ar 0.5 Pa 300 K, E_i 400 eV, 100 mm wafer, 200x200 int64 counts + fp64 energy"),
    "sweep": ("batched sweep: 4 cathodes x 16 pressures (0.2-2 Pa log) x 8 tilts (0-40 deg) = 512 instances, "
              "particle counts uniform in [1e5, 1e7] (seed 0), one launch, autotuned launch shape, "
              "100x100 int64 counts per instance"),
    "large": ("large: single Ni cathode, Ar 3 Pa, 64 primitives (57 shields), 512x512 int64 counts + fp64 energy "
              "+ 64-bin energy + 32-bin angle histograms"),
    "single_ni": ("single Ni 2-inch cathode, Ar 0.5 Pa 300 K, E_i 400 eV, 1e5 particles, box chamber, "
                  "100x100 mm substrate at 100 mm, 50x50 int32 counts"),
}
WORKLOAD = WORKLOADS["quaternary"]

# ---------------------------------------------------------------- work model
# Algorithmic lane-operations of the method, per unit (one lane-op = one issue
# slot of one lane: an FP32 or integer operation, a MUFU function, a shared-
# memory load).  The method's own work, independent of how the kernel codes it:
#   Philox4x32-10 block: 10 rounds x (2 mul-hi + 2 mul-lo + 4 xor + 2 key adds)
#   flight (S0 + S4): one Philox block, ln u, the <sigma g>(v) table (ln(1+v/s)
#     + cubic), the inverse mean free path and the position update
#   surface test (S5): 25 FP32 operations per primitive of the geometry
#   partner attempt (S7): one Philox block, Box-Muller (2 ln, 2 sqrt, sin, 2 cos
#     and scaling), relative speed, sigma(g) g from the b_max table, the test
#   collision (S8): the partner envelope lookup, relative velocity and its
#     norm, reduced energy, impact parameter, the deflection from an
#     (ln eps, b) table (1 lg2, 4 loads, bilinear weights), two sincos,
#     the rotation about g and the CM transform
#   particle (S1-S3, S6, S9): two Philox blocks, racetrack / Thompson / cosine
#     inversions and the pose transform, the cell index and tally, the ticket
PHILOX_BLOCK_OPS = 100
OPS_PER_FLIGHT = PHILOX_BLOCK_OPS + 16
OPS_PER_PRIM_TEST = 25
OPS_PER_ATTEMPT = PHILOX_BLOCK_OPS + 35
OPS_PER_COLLISION = 78
OPS_PER_PARTICLE = 2 * PHILOX_BLOCK_OPS + 80
WORK_MODEL = {"philox_block": PHILOX_BLOCK_OPS, "flight": OPS_PER_FLIGHT, "prim_test": OPS_PER_PRIM_TEST,
              "partner_attempt": OPS_PER_ATTEMPT, "collision": OPS_PER_COLLISION, "particle": OPS_PER_PARTICLE}
# Executed active-lane instructions per collision of the current transport
# kernel (ncu smsp__thread_inst_executed.sum / collisions of one launch, small
# case of the workload); the issue share is reported beside the algorithmic
# fraction.  None = no capture of the current build.
EXEC_LANE_INSTR_PER_COLLISION = {"quaternary": 1814.0, "large": 2667.0}
# DRAM bytes (read + write) of one launch of the quaternary workload, from the
# one-pass capture of the current kernel (mean of 5 launches: 4.10 MB read,
# 0.23 MB written); None whenever the kernel changed after the capture.
TRAFFIC_PER_LAUNCH = 4.33e6


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def mean_prims(scene):
    """Primitives tested per flight: the geometry's primitive count, particle-weighted over instances."""
    tot = sum(int(i["n"]) for i in scene.instances)
    return sum(int(i["n"]) * scene.geometries[i["geometry"]]["prim_count"] for i in scene.instances) / max(1, tot)


def algorithmic_lane_ops(st, prims):
    """Lane-ops of the method for one run, from its statistics (a dict of sput_run_stats)."""
    return (st["flights"] * (OPS_PER_FLIGHT + OPS_PER_PRIM_TEST * prims) + st["attempts"] * OPS_PER_ATTEMPT
            + st["collisions"] * OPS_PER_COLLISION + st["particles"] * OPS_PER_PARTICLE)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during a timed region (200 ms period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception as e:  # no nvidia-smi: report nothing rather than guess
            log("clock sampling unavailable:", e)
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        out["samples"] = len(rows)
        out["sm_mhz"] = statistics.median(sm) if sm else None
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        out["sm_max_mhz"] = max(mx) if mx else None
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        out["power_w_max"] = max(pw) if pw else None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower() == "active":
                    reasons.add(nm)
        out["reasons"] = sorted(reasons)
        return out


# ------------------------------------------------------------- reference arm
def sample_scene(workload, n_per_instance):
    """A bounded sample of the workload: every instance with n_per_instance particles."""
    import workloads

    if workload == "quaternary":
        return workloads.scene_quaternary(n_per_cathode=n_per_instance)
    if workload == "sweep":
        return workloads.scene_tilt_pressure_sweep().with_particles(n_per_instance)
    if workload == "single_ni":
        return workloads.scene_single_ni(n=n_per_instance)
    return workloads.scene_large_shielded(n=n_per_instance)


def cpu_oracle_rate(n_per_instance, n_threads=None, workload="quaternary"):
    """Oracle collisions/s and landed/s on a bounded sample of the workload."""
    import numpy as np

    import oracle

    sc = sample_scene(workload, n_per_instance)
    o = oracle.OracleScene(sc)
    n_threads = n_threads or (os.cpu_count() or 1)
    t0 = time.perf_counter()
    out = o.run_all(n_threads=n_threads)
    dt = time.perf_counter() - t0
    coll = int(out["ncoll"].sum())
    landed = int(np.sum(out["prim"] >= 0))
    return {"collisions": coll, "landed": landed, "seconds": dt, "cores": n_threads,
            "particles": sc.total_particles, "instances": len(sc.instances)}


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle

    oracle.build()
    n_per = args.ref_particles
    if args.workload == "sweep":
        n_per = max(1, n_per // 128)
    for _ in range(args.warmup):
        cpu_oracle_rate(max(1, n_per // 8), workload=args.workload)
    tot_c = tot_l = tot_t = 0.0
    cores = 0
    nparts = 0
    for _ in range(args.steps):
        r = cpu_oracle_rate(n_per, workload=args.workload)
        nparts = r["particles"]
        tot_c += r["collisions"]
        tot_l += r["landed"]
        tot_t += r["seconds"]
        cores = r["cores"]
    value = tot_c / tot_t
    sample = f"{nparts} particles ({n_per} per instance) of the workload per step, all host cores"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "landed_per_s": tot_l / tot_t,
        "config": {"workload": WORKLOADS[args.workload], "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ peaks
PEAK_ITERS = {"ffma": 20000, "mufu_lg2": 8000, "mufu_ex2": 8000, "mufu_rsqrt": 8000, "mufu_sin": 8000,
              "philox": 2000, "red_i32": 2000, "red_i64": 2000, "red_f64": 2000}


def measure_peaks(torch, api, dev, n_slots):
    """Measured throughputs (per second) of the units the transport issues to."""
    stream = torch.cuda.current_stream(dev).cuda_stream
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    scratch = torch.zeros(max(8 * n_slots, 4 * 8 * 256 * n_sm), dtype=torch.uint8, device=dev)
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.25)
    out = {}
    for kind, iters in PEAK_ITERS.items():
        r = api.sput_microbench(dev.index, kind, scratch, iters, stream, n_slots=n_slots)
        out[kind] = r.ops_per_s
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    out["unit"] = "lane-ops/s (ffma, mufu_*), Philox4x32-10 blocks/s, L2 reductions/s (red_*)"
    out["red_slots"] = n_slots
    out["clocks"] = {"sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons"), "samples": clk.get("samples")}
    return out


def roofline_entry(stats_list, kernel_ms, prims, peaks, exec_per_coll=None, traffic=None):
    """Algorithmic lane-op roofline of the transport kernel over a list of runs."""
    ops = statistics.mean(algorithmic_lane_ops(s, prims) for s in stats_list)
    coll = statistics.mean(s["collisions"] for s in stats_list)
    t = statistics.mean(kernel_ms) / 1e3
    achieved = ops / t / 1e12
    peak = peaks["ffma"] / 1e12
    e = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tlane-op/s", "frac": achieved / peak,
         "traffic": traffic, "kernel": "transport_kernel", "kernel_ms_mean": statistics.mean(kernel_ms),
         "peak_basis": "measured FP32 FMA lane-op rate of this GPU in this run (sput_microbench ffma)",
         "algorithmic_lane_ops_per_launch": ops, "algorithmic_lane_ops_per_collision": ops / max(1.0, coll),
         "prims_per_flight": prims, "work_model": WORK_MODEL}
    if exec_per_coll is not None:
        e["executed_lane_instr_per_collision"] = exec_per_coll
        e["issue_frac"] = exec_per_coll * coll / t / peaks["ffma"]
    return e


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2411_14413_gb300 as pkg
    import workloads
    from paper_2411_14413_gb300 import _native as N
    from paper_2411_14413_gb300 import api, shard

    dist = None
    if world > 1:
        import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    # CPU baseline first (rank 0, N = 1 only), before the GPU work starts
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_cpu = args.cpu_particles if args.workload != "sweep" else max(1, args.cpu_particles // 128)
        r = cpu_oracle_rate(n_cpu, workload=args.workload)
        cpu = {"value": r["collisions"] / r["seconds"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
               "sample": f"{r['particles']} particles ({n_cpu} per instance) of the workload, "
                         f"{r['seconds']:.1f} s wall on {r['cores']} threads",
               "landed_per_s": r["landed"] / r["seconds"]}
        # the same oracle on one thread, on a quarter of the sample
        r1 = cpu_oracle_rate(max(1, n_cpu // 4), n_threads=1, workload=args.workload)
        cpu["single_thread"] = {"value": r1["collisions"] / r1["seconds"], "unit": UNIT, "cores": 1,
                                "sample": f"{r1['particles']} particles, {r1['seconds']:.1f} s wall on 1 thread"}
        log("cpu baseline:", cpu)

    sc = headline_scene(workloads, args)
    tr = pkg.Transport(sc, device=local_rank, energy=sc.grid["energy"])
    tune = None
    if args.workload == "sweep" or args.autotune:
        tune = tr.autotune(sample_tickets=min(20_000_000, sc.total_particles))
        log("autotune:", {k: getattr(tune, k) for k in ("block_threads", "blocks_per_sm", "ticket_chunk",
                                                          "flags", "best_rate")})
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream(dev)
    seed0 = 1000 * rank

    for w in range(args.warmup):
        st = tr.run(seed=seed0 + 10_000 + w, want_stats=True)
        log(f"warmup {w}: {st.collisions} collisions, kernel {st.kernel_ms:.2f} ms")
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.25)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()                                       # L2 flush, outside the timed events
        ev[k][0].record(stream)
        # asynchronous: the steps are enqueued back to back, so no host wait falls inside the events
        tr.run(seed=seed0 + k, stream=stream.cuda_stream, want_stats=False)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    # each timed step's statistics: the same seeds once more, outside the timed region (a run's
    # counts and tallies depend only on its seed and tickets, so these are the timed steps' own)
    stats = []
    for k in range(args.steps):
        flush.zero_()
        stats.append(tr.run(seed=seed0 + k, stream=stream.cuda_stream, want_stats=True).as_dict())
    coll = sum(s["collisions"] for s in stats)
    landed = sum(s["landed"] for s in stats)
    # the transport kernel's time per launch: the timed events on its stream (they bracket the
    # tally clear, a few microseconds, and the kernel)
    kernel_ms = step_ms
    grid_landings = int(tr.t["counts"].sum())                     # substrate-grid landings of the last step

    # plain form: one launch per instance (identical tallies), timed the same way
    plain = None
    if args.workload == "sweep" and not args.no_plain:
        plain = plain_per_instance(torch, tr, sc, seed0, stream, flush, stats[0]["collisions"])

    # e2e through the host-buffer entry point: instance table H2D + tallies D2H each step
    L = tr.layout
    pin = lambda shape, dt: torch.zeros(shape, dtype=dt, pin_memory=True)
    host = {"counts": pin((L.n_instances, L.ny, L.nx), torch.int64 if L.count_type == 1 else torch.int32),
            "prim_counts": pin((L.n_instances, L.max_prims), torch.int64),
            "timed_out": pin((L.n_instances,), torch.int64)}
    if "energy" in tr.t:
        host["energy"] = pin((L.n_instances, L.ny, L.nx), torch.float64)
    ht = N.sput_tallies()
    for k2, v in host.items():
        setattr(ht, k2, v.data_ptr())
    d2h = sum(v.numel() * v.element_size() for v in host.values())
    h2d = len(sc.instances) * ctypes.sizeof(N.sput_instance)   # the instance table uploaded per step
    e2e_coll = 0
    e2e_t = 0.0
    if not args.no_e2e:
        api.sput_run_host(tr.h, api.run_opts(seed=seed0 + 777), ht)  # warm the staging buffers
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            api.sput_instances_set(tr.h, sc)
            st = api.sput_run_host(tr.h, api.run_opts(seed=seed0 + 500 + k), ht)
            e2e_coll += st.collisions
        e2e_t = time.perf_counter() - t0

    # max over ranks of the time, sum over ranks of the work
    total_ms_all, (coll_all, landed_all) = shard.reduce_job(total_ms, [coll, landed], device=dev)
    e2e_t_all, (e2e_coll_all,) = shard.reduce_job(e2e_t, [e2e_coll], device=dev)
    n_tal = 1 + (1 if "energy" in tr.t else 0)
    tr.close()
    del flush
    if rank != 0:
        return

    # measured peaks of this GPU (after the timed steps, with their own clock record)
    peaks = measure_peaks(torch, api, dev, n_slots=L.n_instances * L.nx * L.ny)
    log("peaks:", {k: v for k, v in peaks.items() if k not in ("unit",)})

    value = coll_all / (total_ms_all / 1e3)
    prims = mean_prims(sc)
    traffic = TRAFFIC_PER_LAUNCH if (args.workload == "quaternary" and args.particles == 10_000_000) else None
    roof = roofline_entry(stats, kernel_ms, prims, peaks, EXEC_LANE_INSTR_PER_COLLISION.get(args.workload), traffic)
    # landing tally: per substrate-grid landing one int64 count and one fp64 energy reduction
    t_kernel = statistics.mean(kernel_ms) / 1e3
    red_i = grid_landings
    red_f = grid_landings * (n_tal - 1)
    atomics = {"achieved": (red_i + red_f) / t_kernel, "unit": "L2 reductions/s",
               "peak_i64": peaks["red_i64"], "peak_f64": peaks["red_f64"],
               "frac": (red_i / peaks["red_i64"] + red_f / peaks["red_f64"]) / t_kernel,
               "per_launch": {"int64": red_i, "fp64": red_f},
               "note": "frac = time the measured L2 reduction rates need for the landing tally's "
                       "reductions / kernel time"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "landed_per_s": landed_all / (total_ms_all / 1e3),
        "config": {"workload": WORKLOADS[args.workload], "particles_per_step_per_gpu": sc.total_particles,
                   "particle_scale": (args.particles / 10_000_000) if args.workload == "sweep" else 1.0,
                   "instances": len(sc.instances), "grid": f"{sc.grid['nx']}x{sc.grid['ny']}",
                   "tallies": "int64 counts + fp64 energy + int64 per-primitive landings",
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "seed": "distinct per step and per rank", "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "atomics": atomics,
        "peaks": peaks,
        "e2e": {"value": (e2e_coll_all / e2e_t_all) if e2e_t_all > 0 else None, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "autotune": None if tune is None else {"block_threads": tune.block_threads, "blocks_per_sm": tune.blocks_per_sm,
                                               "ticket_chunk": tune.ticket_chunk, "flags": tune.flags,
                                               "candidates": tune.n_candidates},
        "plain_per_instance": plain,
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"), "reasons": clk.get("reasons"),
                   "samples": clk.get("samples"), "power_w_max": clk.get("power_w_max")},
        "step_stats": {"collisions_per_step": coll / args.steps, "landed_per_step": landed / args.steps,
                       "flights_per_step": sum(s["flights"] for s in stats) / args.steps,
                       "attempts_per_collision": sum(s["attempts"] for s in stats) / max(1, coll),
                       "step_ms": step_ms},
    }
    if cpu is not None:
        line["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample", "single_thread")}
    if world == 1 and not args.no_extras:
        line["sub"] = run_extras(args, torch, pkg, api, workloads, dev, peaks)
    print(json.dumps(line), flush=True)


def headline_scene(workloads, args):
    if args.workload == "quaternary":
        return workloads.scene_quaternary(n_per_cathode=args.particles)
    if args.workload == "sweep":
        sc = workloads.scene_tilt_pressure_sweep()
        if args.particles != 10_000_000:
            sc = sc.with_particles([max(1, int(i["n"] * args.particles / 10_000_000)) for i in sc.instances])
        return sc
    if args.workload == "single_ni":
        return workloads.scene_single_ni(n=args.particles)
    return workloads.scene_large_shielded(n=args.particles * 100)


def plain_per_instance(torch, tr, sc, seed, stream, flush, collisions, batched=None):
    """The same tickets and seed as one launch per instance, with the tallies compared
    against `batched` (the batched launch's counts for this seed; run again when None)."""
    if batched is None:
        tr.run(seed=seed, stream=stream.cuda_stream, want_stats=False)
        batched = tr.t["counts"].clone()
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    pe0.record(stream)
    off = 0
    for i, inst in enumerate(sc.instances):
        tr.run(seed=seed, stream=stream.cuda_stream, want_stats=False, ticket_begin=off,
               ticket_end=off + inst["n"], accumulate=i > 0)
        off += inst["n"]
    pe1.record(stream)
    torch.cuda.synchronize()
    plain_ms = pe0.elapsed_time(pe1)
    same = bool(torch.equal(batched, tr.t["counts"]))
    return {"launches": len(sc.instances), "ms": plain_ms, "value": collisions / (plain_ms / 1e3), "unit": UNIT,
            "tallies_identical": same,
            "note": "same seed and tickets as the batched launch; integer tallies compared bit for bit"}


# ------------------------------------------------------------- sub-records
def run_extras(args, torch, pkg, api, workloads, dev, peaks):
    out = {}
    for name, fn in (("single_ni", sub_single_ni), ("sweep", sub_sweep), ("large", sub_large),
                     ("adjoint_vs_fd", sub_adjoint_vs_fd), ("inverse_solve", sub_inverse_solve)):
        if args.workload == name:
            continue
        t0 = time.perf_counter()
        try:
            out[name] = fn(args, torch, pkg, api, workloads, dev, peaks)
        except Exception as e:  # a sub-record that fails is reported, the headline stands
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
        log(f"sub {name}:", json.dumps(out[name])[:400])
    return out


def sub_single_ni(args, torch, pkg, api, workloads, dev, peaks):
    """1e5 atoms, 50x50 int32: one launch, then R launches replayed from a CUDA graph."""
    sc = workloads.scene_single_ni(n=100_000)
    tr = pkg.Transport(sc, device=dev.index)
    stream = torch.cuda.current_stream(dev)
    R = 200
    stats = [tr.run(seed=s).as_dict() for s in range(R)]        # per-seed work, untimed
    one_ms = statistics.median(s["kernel_ms"] for s in stats)
    g = tr.graph(stream=stream.cuda_stream)
    for s in range(3):
        api.sput_graph_launch(g, s, stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for s in range(R):
        api.sput_graph_launch(g, s, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    ref = tr.t["counts"].clone()
    tr.run(seed=R - 1, want_stats=False)
    graph_ok = bool(torch.equal(ref, tr.t["counts"]))
    api.sput_graph_destroy(g)
    tr.close()
    coll = sum(s["collisions"] for s in stats)
    # the same workload repeated 100 times inside one launch (1e7 particle ids, one
    # instance): the GPU is filled instead of waiting on the slowest atom of 1e5
    big = workloads.scene_single_ni(n=100 * 100_000)
    trb = pkg.Transport(big, device=dev.index)
    trb.run(seed=98, ticket_end=1_000_000)
    e0.record(stream)
    stb = trb.run(seed=97, stream=stream.cuda_stream).as_dict()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_big = e0.elapsed_time(e1)
    trb.close()
    roof = roofline_entry(stats, [s["kernel_ms"] for s in stats], mean_prims(sc), peaks)
    roof_big = roofline_entry([stb], [stb["kernel_ms"]], mean_prims(big), peaks)
    return {"workload": WORKLOADS["single_ni"], "value": coll / (ms / 1e3), "unit": UNIT,
            "landed_per_s": sum(s["landed"] for s in stats) / (ms / 1e3),
            "launches": R, "ms_per_launch_graph": ms / R, "kernel_ms_single_launch": one_ms,
            "graph_replay_matches_sput_run": graph_ok, "roofline": roof,
            "note": "R seeds of the 1e5-atom workload replayed from one CUDA graph (seed updated per replay), "
                    "inputs resident; kernel_ms_single_launch is one launch's own event time: a launch of 1e5 "
                    "atoms is bound by the latency of its longest trajectories",
            "repeated_in_one_launch": {"particles": big.total_particles, "value": stb["collisions"] / (ms_big / 1e3),
                                       "unit": UNIT, "landed_per_s": stb["landed"] / (ms_big / 1e3), "ms": ms_big,
                                       "roofline": roof_big}}


def sub_sweep(args, torch, pkg, api, workloads, dev, peaks):
    """512 instances in one autotuned launch vs one launch per instance (particle_scale 0.1)."""
    scale = 0.1
    sc = workloads.scene_tilt_pressure_sweep()
    sc = sc.with_particles([max(1, int(i["n"] * scale)) for i in sc.instances])
    tr = pkg.Transport(sc, device=dev.index, energy=False)
    tune = tr.autotune(sample_tickets=min(20_000_000, sc.total_particles))
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    tr.run(seed=99, ticket_end=2_000_000)                       # warm-up
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = tr.run(seed=7, stream=stream.cuda_stream).as_dict()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    plain = plain_per_instance(torch, tr, sc, 7, stream, flush, st["collisions"], batched=tr.t["counts"].clone())
    tr.close()
    roof = roofline_entry([st], [st["kernel_ms"]], mean_prims(sc), peaks)
    return {"workload": WORKLOADS["sweep"], "particle_scale": scale, "particles": sc.total_particles,
            "value": st["collisions"] / (ms / 1e3), "unit": UNIT, "landed_per_s": st["landed"] / (ms / 1e3),
            "ms": ms, "plain_per_instance": plain, "batched_over_plain": plain["ms"] / ms,
            "autotune": {"block_threads": tune.block_threads, "blocks_per_sm": tune.blocks_per_sm,
                         "ticket_chunk": tune.ticket_chunk, "flags": tune.flags},
            "roofline": roof}


def sub_large(args, torch, pkg, api, workloads, dev, peaks):
    """The large shielded chamber at 3 Pa, 1e8 atoms in one launch (the full workload is 1e9)."""
    n = 100_000_000
    sc = workloads.scene_large_shielded(n=n)
    tr = pkg.Transport(sc, device=dev.index, energy=True)
    stream = torch.cuda.current_stream(dev)
    tr.run(seed=99, ticket_end=1_000_000)                      # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = tr.run(seed=3, stream=stream.cuda_stream).as_dict()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    tr.close()
    roof = roofline_entry([st], [st["kernel_ms"]], mean_prims(sc), peaks, EXEC_LANE_INSTR_PER_COLLISION.get("large"))
    return {"workload": WORKLOADS["large"], "particles": n, "particle_scale": n / 1e9,
            "value": st["collisions"] / (ms / 1e3), "unit": UNIT, "landed_per_s": st["landed"] / (ms / 1e3),
            "ms": ms, "collisions_per_particle": st["collisions"] / n,
            "attempts_per_collision": st["attempts"] / max(1, st["collisions"]), "roofline": roof}


def sub_adjoint_vs_fd(args, torch, pkg, api, workloads, dev, peaks):
    """Gradient of a 342-point composition-map loss in (ln p, P_1..P_4): the likelihood-
    ratio adjoint (one run with the score + one boundary run at the cut-off) against
    central finite differences with common random numbers (2 runs per parameter), over
    K seeds.  The cost ratio at equal standard error is (t_fd var_fd) / (t_lr var_lr)."""
    import numpy as np

    from paper_2411_14413_gb300.adjoint import MapSetup
    from workloads import ELEMENTS
    from workloads.measurement import calibration_points, measurement_patches, voltage_points

    quat = ("Ni", "Pd", "Pt", "Ru")
    n_per = 1_000_000
    patch, _pts, ref = measurement_patches()
    cal, volt = [], []
    for s in quat:
        (p1, r1), (p2, r2) = calibration_points(s)
        cal.append([p1, r1, p2, r2, ELEMENTS[s].density, ELEMENTS[s].mass])
        (q1, v1), (q2, v2) = voltage_points(s)
        volt.append([q1, v1, q2, v2])
    sc = workloads.scene_quaternary(n_per_cathode=n_per)
    ms = MapSetup(sc, patch, ref, np.array(cal), device=dev.index, voltage=np.array(volt))
    p0, power = 0.5, np.array([20.0, 30.0, 12.0, 18.0])
    rng = np.random.default_rng(11)
    gcomp = torch.as_tensor(rng.normal(size=(ms.n_points, 4)), device=dev)
    h_lnp, h_pw = 0.05, 2.0
    K = 8
    lr, fd = [], []
    t_lr = t_fd = 0.0
    ms.forward(p0, power, 100)                                  # warm-up
    ms.backward(gcomp, power)
    torch.cuda.synchronize(dev)
    for seed in range(K):
        t0 = time.perf_counter()
        ms.forward(p0, power, seed)
        glogp, gpow = ms.backward(gcomp, power)
        g = np.concatenate([[float(glogp.sum())], gpow.cpu().numpy()])
        t_lr += time.perf_counter() - t0
        lr.append(g)
        t0 = time.perf_counter()
        row = []
        for sgn in (+1, -1):
            row.append(float((gcomp * ms.forward(p0 * math.exp(sgn * h_lnp), power, seed)).sum()))
        d = [(row[0] - row[1]) / (2 * h_lnp)]
        for j in range(4):
            e = np.zeros(4)
            e[j] = h_pw
            lp = float((gcomp * ms.forward(p0, power + e, seed)).sum())
            lm = float((gcomp * ms.forward(p0, power - e, seed)).sum())
            d.append((lp - lm) / (2 * h_pw))
        t_fd += time.perf_counter() - t0
        fd.append(d)
    ms.close()
    lr, fd = np.array(lr), np.array(fd)
    var_lr, var_fd = lr.var(axis=0, ddof=1), fd.var(axis=0, ddof=1)
    names = ["ln_p", "P_Ni", "P_Pd", "P_Pt", "P_Ru"]
    ratio = (t_fd * var_fd) / np.maximum(t_lr * var_lr, 1e-300)
    return {"setup": "quaternary, 1e6 atoms per cathode per run, 342-point map, Table S1 rate and voltage lines, "
                     f"{K} seeds; FD steps ln p +-{h_lnp}, P +-{h_pw} W",
            "runs_per_gradient": {"adjoint": 2, "finite_differences": 10},
            "s_per_gradient": {"adjoint": t_lr / K, "finite_differences": t_fd / K},
            "mean": {"adjoint": dict(zip(names, lr.mean(0).tolist())), "finite_differences": dict(zip(names, fd.mean(0).tolist()))},
            "std": {"adjoint": dict(zip(names, np.sqrt(var_lr).tolist())),
                    "finite_differences": dict(zip(names, np.sqrt(var_fd).tolist()))},
            "cost_ratio_fd_over_adjoint_at_equal_se": dict(zip(names, ratio.tolist()))}


def sub_inverse_solve(args, torch, pkg, api, workloads, dev, peaks):
    """The adjoint workload at its size: 50 Adam steps of the inverse solve for (p, P_1..P_4)
    on the quaternary scene at 1e7 atoms per cathode per step, 342-point map, Table S1 rate
    and voltage lines, to a target transported from random true values (Table 1 ranges)
    with its own seed; each step is a forward run with the score, the composition map, a
    boundary run at the cut-off and the backward kernels."""
    import numpy as np

    from paper_2411_14413_gb300.adjoint import MapSetup, inverse_solve
    from workloads import ELEMENTS
    from workloads.measurement import POWER_RANGE, calibration_points, measurement_patches, voltage_points

    quat = ("Ni", "Pd", "Pt", "Ru")
    rng = np.random.default_rng(20241122)
    true_p = float(math.exp(rng.uniform(math.log(0.3), math.log(1.0))))
    true_pw = np.array([rng.uniform(*POWER_RANGE[s]) for s in quat])
    cal, volt = [], []
    for s in quat:
        (p1, r1), (p2, r2) = calibration_points(s)
        cal.append([p1, r1, p2, r2, ELEMENTS[s].density, ELEMENTS[s].mass])
        (q1, v1), (q2, v2) = voltage_points(s)
        volt.append([q1, v1, q2, v2])
    patch, _pts, ref = measurement_patches()
    sc = workloads.scene_quaternary(n_per_cathode=10_000_000)
    ms = MapSetup(sc, patch, ref, np.array(cal), device=dev.index, voltage=np.array(volt))
    target = ms.forward(true_p, true_pw, seed=987654).clone()
    start = np.array([0.5 * (POWER_RANGE[s][0] + POWER_RANGE[s][1]) for s in quat])
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    hist = inverse_solve(ms, target, math.log(0.5), start, steps=50, lr=0.1, seed=1)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    ms.close()
    frac = lambda x: np.asarray(x) / np.sum(x)
    last = hist[-1]
    return {"setup": "quaternary, 1e7 atoms per cathode per step, 342 points, rate + voltage lines, 50 Adam steps",
            "s_per_step": dt / 50,
            "true": {"p": true_p, "power": true_pw.tolist()}, "fit": {"p": last["p"], "power": last["power"]},
            "p_rel_error": last["p"] / true_p - 1.0,
            "power_fraction_max_error": float(np.abs(frac(last["power"]) - frac(true_pw)).max()),
            "loss": {"first": hist[0]["loss"], "last": last["loss"]}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--particles", type=int, default=None,
                    help="per cathode (quaternary, default 1e7); sweep: counts scaled by particles/1e7 "
                         "(default 1e6, one tenth, so that a run ends in minutes); large: particles x 100 "
                         "(default 1e6 -> 1e8); single_ni: particles (default 1e5)")
    ap.add_argument("--cpu-particles", type=int, default=600, help="oracle sample per cathode")
    ap.add_argument("--ref-particles", type=int, default=400, help="oracle sample per cathode per step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the sub-records of the other workloads")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="quaternary")
    ap.add_argument("--autotune", action="store_true", help="autotune the launch shape before timing")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-launch-per-instance comparison")
    args = ap.parse_args()
    if args.particles is None:
        args.particles = {"quaternary": 10_000_000, "sweep": 1_000_000, "large": 1_000_000,
                          "single_ni": 100_000}[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
