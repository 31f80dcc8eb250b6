#!/usr/bin/env python3
"""Throughput of the sputtered-atom transport hot path on GB300.

A step transports the whole quaternary co-sputter workload (Ni/Pd/Pt/Ru,
4 cathodes tilted 30 deg confocal at 120 mm, 1e7 particles each, Ar 0.5 Pa,
300 K, 100 mm wafer with 200x200 int64 counts + fp64 energy per cathode)
through libsput.so.  The metric is particle-collisions/s (and landed
particles/s), whole job, inputs resident in HBM; ``e2e`` is the same metric
through the host-buffer entry point with the host<->device copies inside.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank transports its own replica of the workload
(distinct seeds, no data-path collective: particles are independent) and the
job value is the sum over ranks divided by the slowest rank's time.
``--impl reference`` times the FP64 CPU oracle on bounded samples of the same
workload (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
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
}
WORKLOAD = WORKLOADS["quaternary"]
# Algorithmic work per collision: active-lane instructions per collision of the
# reference capture of the transport kernel on this workload (ncu
# smsp__thread_inst_executed.sum / collisions of the launch, quaternary scene
# with 2e5 particles per cathode); the figure is kept fixed so that frac
# measures speed against one definition of the work.
LANE_OPS_PER_COLLISION = 4136.0
# DRAM bytes (read + write) of one launch of the quaternary workload, from the
# one-pass capture of the current kernel (mean of 5 launches: 3.11 MB read,
# 0 written; the tallies stay in L2); None whenever the kernel changed after
# the capture.
TRAFFIC_PER_LAUNCH = 3.11e6
LANES_PER_SM_PER_CLK = 128  # 4 SM sub-partitions x 32 lanes issue one instruction per clock each


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (200 ms period)."""

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


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
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
        log("cpu baseline:", cpu)

    if args.workload == "quaternary":
        sc = workloads.scene_quaternary(n_per_cathode=args.particles)
    elif args.workload == "sweep":
        sc = workloads.scene_tilt_pressure_sweep()
        if args.particles != 10_000_000:
            sc = sc.with_particles([max(1, int(i["n"] * args.particles / 10_000_000)) for i in sc.instances])
    else:
        sc = workloads.scene_large_shielded(n=args.particles * 100)
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
    stats = []
    for k in range(args.steps):
        flush.zero_()                                       # L2 flush, outside the timed events
        ev[k][0].record(stream)
        st = tr.run(seed=seed0 + k, stream=stream.cuda_stream, want_stats=True)
        ev[k][1].record(stream)
        stats.append(st.as_dict())
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    coll = sum(s["collisions"] for s in stats)
    landed = sum(s["landed"] for s in stats)
    kernel_ms = [s["kernel_ms"] for s in stats]

    # plain form: one launch per instance (identical tallies), timed the same way
    plain = None
    if args.workload == "sweep" and not args.no_plain:
        torch.cuda.synchronize(dev)
        pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        pe0.record(stream)
        off = 0
        for i, inst in enumerate(sc.instances):
            tr.run(seed=seed0, stream=stream.cuda_stream, want_stats=False, ticket_begin=off,
                   ticket_end=off + inst["n"], accumulate=i > 0)
            off += inst["n"]
        pe1.record(stream)
        torch.cuda.synchronize(dev)
        plain_ms = pe0.elapsed_time(pe1)
        plain = {"launches": len(sc.instances), "ms": plain_ms,
                 "value": stats[0]["collisions"] / (plain_ms / 1e3), "unit": UNIT,
                 "note": "same seed and tickets as step 0; tallies identical to the batched launch"}

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
    h2d = len(sc.instances) * 40
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
    tr.close()
    if rank != 0:
        return

    value = coll_all / (total_ms_all / 1e3)
    props = torch.cuda.get_device_properties(dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * LANES_PER_SM_PER_CLK * sm_max * 1e6 / 1e12   # T lane-ops/s
    mean_kernel_s = statistics.mean(kernel_ms) / 1e3
    coll_per_launch = coll / args.steps
    achieved = LANE_OPS_PER_COLLISION * coll_per_launch / mean_kernel_s / 1e12
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
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tlane-op/s",
                     "frac": achieved / peak,
                     "traffic": TRAFFIC_PER_LAUNCH if (args.workload == "quaternary" and args.particles == 10_000_000) else None,
                     "kernel": "transport_kernel", "kernel_ms_mean": statistics.mean(kernel_ms),
                     "lane_ops_per_collision": LANE_OPS_PER_COLLISION,
                     "peak_basis": f"{props.multi_processor_count} SMs x 128 lanes x {sm_max:.0f} MHz (sm_max_mhz)"},
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
                       "attempts_per_collision": sum(s["attempts"] for s in stats) / max(1, coll),
                       "step_ms": step_ms},
    }
    if cpu is not None:
        line["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--particles", type=int, default=None,
                    help="per cathode (quaternary, default 1e7); sweep: counts scaled by particles/1e7 "
                         "(default 1e6, one tenth, so that a run ends in minutes); large: particles x 100 "
                         "(default 1e6 -> 1e8)")
    ap.add_argument("--cpu-particles", type=int, default=600, help="oracle sample per cathode")
    ap.add_argument("--ref-particles", type=int, default=400, help="oracle sample per cathode per step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="quaternary")
    ap.add_argument("--autotune", action="store_true", help="autotune the launch shape before timing")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-launch-per-instance comparison")
    args = ap.parse_args()
    if args.particles is None:
        args.particles = {"quaternary": 10_000_000, "sweep": 1_000_000, "large": 1_000_000}[args.workload]
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
