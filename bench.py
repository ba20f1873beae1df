#!/usr/bin/env python3
"""Throughput of the FP64 fused tracking path on one or more GB300s.

Workload (the configuration the headline metric is quoted on): the 40-cell
kick-drift ring -- per cell QF(0.2 m, K1 = +1.2), SF(0.1 m, K2 = +20), exact
drift 0.9 m, QD, SD, drift, each thick element integrated by 4 steps of the
4th-order Yoshida scheme, plus one RF cavity (1 MV, h = 400): 241 elements,
elliptical aperture 15 x 8 mm checked after every element, per-turn moments,
stable loss compaction; 1,000,000 particles, 6D Gaussian from seed, 1000 turns.

A step is 100 turns of that bunch (one fused launch followed by moment
finalisation and compaction), so the default 10 timed steps are the whole
1000-turn job; 3 warm-up steps run on a copy of the bunch first.  The metric
counts particle-element passes: alive particles entering each element.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line.  Under torchrun every rank tracks its own bunch (seeded
by rank): particles are independent, so the ranks share no data-path
collective (weak scaling); rank 0 prints.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = ("particle-element passes/s FP64 (1 GB300, % roofline); "
          "DA scans/s batched+surrogate vs plain")
UNIT = "particle-element passes/s"
TURNS_PER_STEP = 100
N_PARTICLES = 1_000_000
# FP64 peak derived from unit counts and clock: 152 SMs x 2 FP64 FMA lanes per
# SM per clock x 2 flops x 2.07 GHz (the lane count is measured, 1.9/clk at a
# 2.0 GHz sampled clock, by a dependent-free DFMA loop on this GPU).
PEAK_FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 256 << 20
WORKLOAD = ("c2: 40-cell kick-drift ring (QF/SF/D0.9/QD/SD/D0.9, Yoshida-4 x 4 steps) + RF, "
            "241 elements, 1e6 particles, 1000 turns, ellipse 15x8 mm")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--block", type=int, default=128)
    p.add_argument("--per-thread", type=int, default=2)
    # smaller cases for profiling runs only (the bench line uses the defaults)
    p.add_argument("--turns-per-step", type=int, default=TURNS_PER_STEP)
    p.add_argument("--particles", type=int, default=N_PARTICLES)
    return p.parse_args()


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------------------------ clocks --

class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_rank%d.csv" % index) if os.path.isdir(
            os.path.join(ROOT, "gpurun_out")) else "/tmp/trk_clocks_%d.csv" % os.getpid()

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------- CPU baseline ----

def oracle_rate(n_particles, n_turns, seed=2):
    """Oracle passes/s on a bounded sample of the workload (single thread)."""
    import synthetic as syn
    from oracle import oracle as orc
    lat = syn.lattice_c2()
    z = syn.bunch("c2", n=n_particles, seed=seed)
    t0 = time.perf_counter()
    s = orc.track(lat, z, n_turns)
    dt = time.perf_counter() - t0
    from paper_1710_07350_gb300 import flops
    lost = s["alive"] == 0
    passes, _ = flops.step_work(lat, n_particles, n_turns, s["loss_turn"][lost], s["loss_elem"][lost])
    return passes / dt, dt, passes


def cpu_baseline():
    rate, dt, _ = oracle_rate(16_000, 10)
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "16000 particles x 10 turns of the 241-element c2 ring, single-threaded C oracle "
                      "(-O2 -ffp-contract=off); %.1f s" % dt}


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    try:
        from oracle import oracle as orc
        orc.build()
    except Exception as e:  # pragma: no cover - build problems are reported, not hidden
        print(json.dumps({"impl": "reference", "unavailable": "oracle build failed: %s" % e}))
        return 0
    n, nt = 4000, 5
    for _ in range(args.warmup):
        oracle_rate(n, nt)
    tot_passes, tot_t = 0.0, 0.0
    for k in range(args.steps):
        r, dt, p = oracle_rate(n, nt)
        tot_passes += p
        tot_t += dt
    value = tot_passes / tot_t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": "%d particles x %d turns" % (n, nt)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d steps of %d particles x %d turns, single-threaded C oracle" % (args.steps, n, nt)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


# ------------------------------------------------------------------- ours ----

def run_ours(args):
    import torch

    import synthetic as syn
    from paper_1710_07350_gb300 import flops, trk

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    lat = syn.lattice_c2()
    L = trk.trk_create_lattice(lat)
    tps, npart = args.turns_per_step, args.particles
    z0 = syn.bunch("c2", n=npart, seed=2 + 1000 * rank)
    coords0, ids0 = trk.upload(z0)
    sched = {"block": args.block, "per_thread": args.per_thread, "chunk_turns": tps}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    # warm-up on a copy of the bunch
    coords, ids = coords0.clone(), ids0.clone()
    b = trk.trk_bunch_wrap(coords, ids)
    trk.trk_bunch_set_schedule(b, **sched)
    for _ in range(args.warmup):
        trk.trk_track(b, L, tps)
    torch.cuda.synchronize()
    del b

    # timed run from the pristine bunch
    coords, ids = coords0.clone(), ids0.clone()
    b = trk.trk_bunch_wrap(coords, ids)
    trk.trk_bunch_set_schedule(b, **sched)
    trk.trk_bunch_enable_timing(b, True)
    trk.trk_bunch_stats(b, reset=True)
    clocks = Clocks(local)
    barrier()
    clocks.start()
    step_ms, passes, flop = [], 0.0, 0.0
    n_alive = npart
    n_lost_seen = 0
    for k in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        trk.trk_track(b, L, tps)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        lid, lturn, lel = trk.trk_lost(b)
        new = slice(n_lost_seen, len(lid))
        p, f = flops.step_work(lat, n_alive, tps, lturn[new] - k * tps, lel[new])
        passes += p
        flop += f
        n_alive -= len(lid) - n_lost_seen
        n_lost_seen = len(lid)
    barrier()
    clk = clocks.stop()
    stats = trk.trk_bunch_stats(b)
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms, passes], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total_ms_all, passes_all = float(tmax[0]), float(t[1])
    else:
        total_ms_all, passes_all = total_ms, passes
    value = passes_all / (total_ms_all / 1e3)
    kernel_ms = stats["track_kernel_ms"]
    achieved = flop / (kernel_ms / 1e3) / 1e12

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hz = coords0.cpu().pin_memory()
        hi = ids0.cpu().pin_memory()
        dz = torch.empty_like(coords0)
        di = torch.empty_like(ids0)
        b2 = trk.trk_bunch_wrap(dz, di)
        trk.trk_bunch_set_schedule(b2, **sched)
        mom_host = torch.empty((tps, 28), dtype=torch.float64).pin_memory()
        n_e2e = max(1, min(args.steps, 3))
        barrier()
        t0 = time.perf_counter()
        p_e2e = 0.0
        na2 = npart
        seen2 = 0
        for k in range(n_e2e):
            dz.copy_(hz, non_blocking=True)
            di.copy_(hi, non_blocking=True)
            trk.trk_track(b2, L, tps)
            hz.copy_(dz, non_blocking=True)
            hi.copy_(di, non_blocking=True)
            mom = trk.trk_moments(b2)          # synchronises; result read on the host
            mom_host.copy_(torch.from_numpy(mom))
            lid, lturn, lel = trk.trk_lost(b2)
            new = slice(seen2, len(lid))
            p, _ = flops.step_work(lat, na2, tps, lturn[new] - k * tps, lel[new])
            p_e2e += p
            na2 -= len(lid) - seen2
            seen2 = len(lid)
        barrier()
        dt = time.perf_counter() - t0
        bi = coords0.numel() * 8 + ids0.numel() * 4
        bo = bi + tps * 28 * 8
        e2e = {"value": p_e2e * world / dt, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
               "steps": n_e2e}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    cpu = None if args.no_cpu_baseline else cpu_baseline()
    traffic = profiled_traffic_per_launch(npart, tps)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles_per_gpu": npart, "elements": len(lat["elements"]),
                   "turns_per_step": tps, "turns_timed": tps * args.steps,
                   "l2": "flushed between steps (256 MiB write)", "block": args.block,
                   "per_thread": args.per_thread, "parallelism": "replica bunches, no collective" if world > 1
                   else "1 GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / PEAK_FP64_TFLOPS, "traffic": traffic,
                     "kernel": "k_track (fused kick-drift ring, 100 turns per launch)",
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                     "flops_per_launch": flop / max(stats["track_launches"], 1),
                     "kernel_ms_per_launch": kernel_ms / max(stats["track_launches"], 1),
                     "kernel_share_of_step": kernel_ms / total_ms if total_ms else None},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": stats["launches"],
        "clocks": clk,
        "passes": passes_all,
        "alive_end": n_alive,
    }
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def profiled_traffic_per_launch(npart, tps):
    """DRAM bytes per k_track launch scaled from the committed ncu summary
    (profiles/k_track_c2.txt, line 'dram_bytes_per_particle_turn: X'), or None."""
    path = os.path.join(ROOT, "profiles", "k_track_c2.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("dram_bytes_per_particle_turn:"):
            try:
                return float(line.split(":")[1]) * npart * tps
            except ValueError:
                return None
    return None


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
