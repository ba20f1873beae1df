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
    p.add_argument("--no-da", action="store_true", help="skip the dynamic-aperture scan measurements")
    p.add_argument("--no-c3", action="store_true", help="skip the wake-linac record of the default line")
    p.add_argument("--no-c4", action="store_true", help="skip the batched-variant record of the default line")
    p.add_argument("--no-sweep", action="store_true", help="skip the particle-count sweeps of the default line")
    p.add_argument("--clocks-dir", default=None, help="where to keep the nvidia-smi samples (default: temp dir)")
    p.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "mlp", "mlp-train", "sweep", "c3sweep", "bend"],
                   help="c2 (default, the headline line); c3 wake linac, c4 batched variants, the "
                        "surrogate's inference (mlp) and training (mlp-train), the particle-count "
                        "sweep of the map ring (sweep) and the sector-bend ring (bend) print their own "
                        "lines")
    p.add_argument("--da-variants", type=int, default=64)
    p.add_argument("--rows", type=int, default=64 * 512 * 512, help="mlp: rows per inference call")
    p.add_argument("--epochs", type=int, default=24, help="mlp-train: epochs")
    p.add_argument("--transverse", action="store_true", help="c3: add the transverse dipole wake")
    p.add_argument("--lsc", action="store_true", help="c3: add impedance space charge after every wake")
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

    def __init__(self, index, directory=None):
        import tempfile
        self.index = index
        self.proc = None
        self.path = os.path.join(directory or tempfile.gettempdir(), "trk_clocks_rank%d.csv" % index)

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

def oracle_rate(n_particles, n_turns, seed=2, threads=1):
    """Oracle passes/s on a bounded sample of the workload: `threads` host
    threads each track an equal slice of one bunch (the C oracle releases the
    interpreter lock while it runs; particles are independent)."""
    import synthetic as syn
    from oracle import oracle as orc
    from paper_1710_07350_gb300 import flops
    lat = syn.lattice_c2()
    z = syn.bunch("c2", n=n_particles * threads, seed=seed)
    parts = np.array_split(z, threads)
    t0 = time.perf_counter()
    if threads == 1:
        outs = [orc.track(lat, parts[0], n_turns)]
    else:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(threads) as ex:
            outs = list(ex.map(lambda zz: orc.track(lat, zz, n_turns), parts))
    dt = time.perf_counter() - t0
    passes = 0.0
    for zz, s in zip(parts, outs):
        lost = s["alive"] == 0
        p, _ = flops.step_work(lat, zz.shape[0], n_turns, s["loss_turn"][lost], s["loss_elem"][lost])
        passes += p
    return passes / dt, dt, passes


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def cpu_baseline():
    """The oracle on all host cores (one slice per core) and on one core."""
    cores = host_cores()
    rate1, dt1, _ = oracle_rate(16_000, 10)
    rate, dt, _ = oracle_rate(4_000, 10, threads=cores)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d threads x 4000 particles x 10 turns of the 241-element c2 ring, C oracle "
                      "(-O2 -ffp-contract=off), %.1f s wall; single thread: 16000 particles x 10 turns, %.1f s"
                      % (cores, dt, dt1),
            "single_thread_value": rate1}


def _threads_map(fn, parts):
    if len(parts) == 1:
        return [fn(parts[0])]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(len(parts)) as ex:
        return list(ex.map(fn, parts))


def da_cpu_baseline():
    """The oracle's dynamic-aperture scan rate on all host cores: one variant's
    512^2 grid sampled every 4th cell in x and y (128^2 cells, 1/16 of a scan),
    1000 turns, split over the cores; scans/s = 1 / (16 x wall time)."""
    import synthetic as syn
    from oracle import oracle as orc
    cores = host_cores()
    n = syn.DA_N
    lat = syn.lattice_c5(0)
    sub = syn.da_particles(n=n).reshape(n, n, 6)[::4, ::4].reshape(-1, 6)
    parts = np.array_split(sub, cores)
    t0 = time.perf_counter()
    _threads_map(lambda zz: orc.track(lat, zz, 1000, moments=False), parts)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / (16.0 * dt), "unit": "DA scans/s", "cores": cores, "kind": "oracle",
            "sample": "variant 0, every 4th cell of the 512^2 grid in x and y (16384 cells = 1/16 of a scan), "
                      "1000 turns, %d threads, %.1f s wall, scaled by 16" % (cores, dt)}


def c3_cpu_baseline(lat):
    """The oracle on the linac: 2e6 particles through 5 of the 200 periods on one
    thread (the wakes need the whole bunch, so the oracle is not split)."""
    import synthetic as syn
    from oracle import oracle as orc
    per = len(lat["elements"]) // syn.C3_PERIODS
    sample = {**lat, "elements": lat["elements"][:5 * per]}
    n = 2_000_000
    z = syn.bunch("c3", n=n)
    t0 = time.perf_counter()
    orc.track(sample, z, 1, moments=False)
    dt = time.perf_counter() - t0
    return {"value": n * len(sample["elements"]) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "2e6 particles through the first 5 of the 200 periods (%d elements), one thread, %.1f s"
                      % (len(sample["elements"]), dt)}


def c4_cpu_baseline():
    """The oracle on the batched-variant ring: the first `cores` variants, 1000
    particles of each through 300 turns, one variant per host thread."""
    import synthetic as syn
    from oracle import oracle as orc
    cores = host_cores()
    vs = syn.c4_variants()[:cores]
    jobs = [(syn.lattice_c4(v), syn.c4_bunch(k, v[2])[:1000]) for k, v in enumerate(vs)]
    t0 = time.perf_counter()
    _threads_map(lambda j: orc.track(j[0], j[1], 300, moments=False), jobs)
    dt = time.perf_counter() - t0
    passes = sum(j[1].shape[0] * len(j[0]["elements"]) * 300 for j in jobs)
    return {"value": passes / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d variants x 1000 particles x 300 turns, one variant per thread, %.1f s wall; passes "
                      "counted as if all survive" % (len(jobs), dt)}


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
    n, nt = 2000, 5
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_rate(n, nt, threads=cores)
    tot_passes, tot_t = 0.0, 0.0
    for k in range(args.steps):
        r, dt, p = oracle_rate(n, nt, threads=cores)
        tot_passes += p
        tot_t += dt
    value = tot_passes / tot_t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": "%d threads x %d particles x %d turns" % (cores, n, nt)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d steps of %d threads x %d particles x %d turns, C oracle"
                                   % (args.steps, cores, n, nt)},
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
    clocks = Clocks(local, args.clocks_dir)
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
    from paper_1710_07350_gb300.dist import combine
    total_ms_all, passes_all = combine(total_ms, passes, device="cuda")
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
    probe = trk.trk_probe_fp64()            # measured FP64 rates, after the timed region
    measured_peak = 2.0 * probe[0] / 1e12
    da = None if args.no_da else run_da(args.da_variants, trk, syn, torch)
    if da is not None and not args.no_cpu_baseline:
        da["cpu_baseline"] = da_cpu_baseline()
    c3 = None if args.no_c3 else c3_record(args, 2, 1, not args.no_cpu_baseline, clocks_index=local)
    c4 = None if args.no_c4 else c4_record(args, 0, not args.no_cpu_baseline, clocks_index=local, plain_stride=8)
    sweep = None if args.no_sweep else {"c3_parts": c3_sweep_record(args), "c1_maps": map_sweep_points()}
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
                     "peak_measured": measured_peak, "frac_of_measured": achieved / measured_peak,
                     "peak_measured_source": "trk_probe_fp64: independent DFMA chains, 4 x 256 threads per SM",
                     "dmul_dadd_rate_vs_dfma": [probe[1] / probe[0], probe[2] / probe[0]],
                     "flops_per_launch": flop / max(stats["track_launches"], 1),
                     "kernel_ms_per_launch": kernel_ms / max(stats["track_launches"], 1),
                     "kernel_share_of_step": kernel_ms / total_ms if total_ms else None},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": stats["launches"],
        "clocks": clk,
        "passes": passes_all,
        "alive_end": n_alive,
        "da": da,
        "c3": c3,
        "c4": c4,
        "sweep": sweep,
    }
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_da(n_var, trk, syn, torch):
    """DA scans/s on the 64-variant, 512^2-cell, 1000-turn workload: plain
    (one lattice per call), batched (all variants in one call) and batched plus
    surrogate triage; the same triage without the network as the ablation.
    One scan = one variant's full grid."""
    import numpy as np
    from paper_1710_07350_gb300 import da_metrics as dm
    n, turns = syn.DA_N, 1000
    L = [trk.trk_create_lattice(syn.lattice_c5(v), moments=False) for v in range(n_var)]
    z = syn.da_particles(n=n)
    x0 = torch.from_numpy(z[:, 0].copy()).cuda()
    y0 = torch.from_numpy(z[:, 2].copy()).cuda()
    trk.trk_da_survival(L[:1], x0[:4096], y0[:4096], [0, 4096], 20)   # warm-up
    torch.cuda.synchronize()
    t = time.perf_counter()
    for v in range(n_var):
        trk.trk_da_survival([L[v]], x0, y0, [0, n * n], turns)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t
    t = time.perf_counter()
    exh = trk.trk_da_survival(L, torch.cat([x0] * n_var), torch.cat([y0] * n_var),
                              [k * n * n for k in range(n_var + 1)], turns)
    torch.cuda.synchronize()
    t_batched = time.perf_counter() - t
    exh = (exh.cpu().numpy().reshape(n_var, n, n) == turns + 1)
    params = torch.from_numpy(syn.c5_params()[:n_var].astype(np.float32)).cuda()
    g = np.random.Generator(np.random.Philox(key=12))
    audit = torch.from_numpy((g.uniform(size=(n_var, n, n)) < 0.005).astype(np.uint8)).cuda()
    # 6 epochs: the fastest surrogate arm at the one-cell boundary (24 / 12 / 8 / 6 / 4 measured)
    stride, epochs, batch = 8, 6, 4096
    ncoarse = n_var * ((n - stride // 2 + stride - 1) // stride) ** 2
    perm = torch.from_numpy(np.stack([g.permutation(ncoarse) for _ in range(epochs)]).astype(np.int32)).cuda()
    out = {"variants": n_var, "grid": [n, n], "turns": turns, "coarse_stride": stride, "band_radius": 2,
           "audit_fraction": 0.005, "sentinel_stride": 5, "expand_radius": 0}
    res = {}
    # the surrogate arm: the network predicts the cells near the nearest-known
    # boundary (use_mlp 2; measured 133 scans/s against 127 with the network on
    # every cell)
    for name, use in (("surrogate", 2), ("nonlearned", 0)):
        net = trk.trk_mlp_create(syn.mlp_init(7)) if use else None
        opts = {"nx": n, "ny": n, "half_width": syn.DA_HALF_WIDTH, "n_turns": turns, "coarse_stride": stride,
                "band_radius": 2, "use_mlp": use, "epochs": epochs, "batch": batch, "lr": 2e-3,
                "sentinel_stride": 5, "expand_radius": 0}
        torch.cuda.synchronize()
        t = time.perf_counter()
        mask, _, st = trk.trk_da_triage(L, params, opts, net=net, audit=audit, perm=perm if use else None)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        mask = mask.cpu().numpy().astype(bool)
        diffs = [dm.boundary_difference(mask[v], exh[v]) for v in range(n_var)]
        res[name] = {"seconds": dt, "scans_per_s": n_var / dt,
                     "boundary_within_1_cell": all(d[0] for d in diffs),
                     "cells_differing": int(sum(d[1] for d in diffs)),
                     "max_cell_distance": int(max(d[2] for d in diffs)),
                     "tracked_fraction": (st["n_tracked"] + st["n_coarse"]) / st["n_cells"],
                     "audit_cells": st["n_audit"], "audit_wrong": st["n_audit_wrong"], "band_passes": st["n_passes"],
                     "network_cells": st["n_region"],
                     "pass_cells": st["pass_cells"], "pass_ms": [round(v, 1) for v in st["pass_ms"]],
                     "ms": {k: st[k] for k in ("ms_coarse", "ms_train", "ms_infer", "ms_band", "ms_retrack")}}
    out["scans_per_s"] = {"plain": n_var / t_plain, "batched": n_var / t_batched,
                          "batched_surrogate": res["surrogate"]["scans_per_s"],
                          "batched_nonlearned_triage": res["nonlearned"]["scans_per_s"]}
    out["surrogate_vs_plain"] = res["surrogate"]["scans_per_s"] / (n_var / t_plain)
    out["triage"] = res
    return out


TRACK_SOURCES = ("paper_1710_07350_gb300/csrc/trk_track.cu", "paper_1710_07350_gb300/csrc/trk_device.cuh",
                 "paper_1710_07350_gb300/csrc/trk_internal.cuh")


def track_source_digest():
    """SHA-256 over the tracking kernel's sources: ties a DRAM capture to the
    kernel build it was taken on."""
    import hashlib
    h = hashlib.sha256()
    for f in TRACK_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic_per_launch(npart, tps):
    """DRAM bytes (read + write) of one k_track launch of this workload from the
    committed ncu summary profiles/k_track_c2.md, whose lines
    'dram_bytes_per_launch: <particles> <turns> <bytes>' and
    'kernel_source_sha256: <digest>' record a capture of exactly this launch
    shape; None when the shape differs or the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "k_track_c2.md")
    if not os.path.exists(path):
        return None
    rec, digest = None, None
    for line in open(path):
        if line.startswith("dram_bytes_per_launch:"):
            try:
                p, t, b = line.split(":")[1].split()
                rec = (int(p), int(t), float(b))
            except ValueError:
                return None
        elif line.startswith("kernel_source_sha256:"):
            digest = line.split(":")[1].strip()
    if rec is None or digest != track_source_digest() or rec[:2] != (npart, tps):
        return None
    return rec[2]


def run_c3(args):
    print(json.dumps(c3_record(args, args.steps, args.warmup, not args.no_cpu_baseline)))
    return 0


def c3_record(args, steps, warmup, with_cpu, clocks_index=None):
    """Wake linac: 10M particles through 200 x [RF, WAKE(4096), drift, quad];
    one step = one pass of the whole linac from the initial bunch."""
    import torch

    import synthetic as syn
    from paper_1710_07350_gb300 import flops, trk
    lat = syn.lattice_c3(transverse=args.transverse, lsc=args.lsc)
    L = trk.trk_create_lattice(lat)
    z0 = syn.bunch("c3")
    if args.transverse:                       # an offset bunch, so that the dipole moments act
        z0[:, 0] += 1.0e-4
        z0[:, 2] -= 5.0e-5
    coords0, ids0 = trk.upload(z0)
    n = z0.shape[0]
    times = []
    clocks = Clocks(clocks_index, args.clocks_dir) if clocks_index is not None else None
    for k in range(warmup + steps):
        if clocks is not None and k == warmup:
            clocks.start()
        coords, ids = coords0.clone(), ids0.clone()
        b = trk.trk_bunch_wrap(coords, ids)
        trk.trk_bunch_set_schedule(b, block=args.block, per_thread=args.per_thread)
        trk.trk_bunch_enable_timing(b, True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        trk.trk_track(b, L, 1)
        e1.record()
        e1.synchronize()
        st = trk.trk_bunch_stats(b)
        if k >= warmup:
            times.append((e0.elapsed_time(e1), st))
        del b
    clk = clocks.stop() if clocks is not None else None
    ms = sum(t for t, _ in times) / len(times)
    kms = sum(st["track_kernel_ms"] for _, st in times) / len(times)
    passes = n * len(lat["elements"])
    _, f = flops.step_work(lat, n, 1)
    f += n * 200 * flops.WAKE_FLOPS_PER_PARTICLE + 200 * flops.wake_conv_flops(syn.C3_NBINS)
    if args.transverse:
        f += n * 200 * flops.TRWAKE_FLOPS_PER_PARTICLE + 200 * 2 * flops.wake_conv_flops(syn.C3_NBINS)
    if args.lsc:
        f += n * 200 * flops.LSC_FLOPS_PER_PARTICLE + 200 * flops.lsc_imp_flops(syn.C3_NBINS)
    extra = (" + transverse dipole wake, offset bunch" if args.transverse else "") + \
            (" + impedance space charge (4096 bins, r_b 1 mm, L 3 m)" if args.lsc else "")
    ach = f / (ms / 1e3) / 1e12
    return {"workload": "c3 wake linac: 200 x [RFCA -10 deg, WAKE 4096 bins%s, drift, quad], 1e7 particles" % extra,
            "metric": UNIT, "value": passes / (ms / 1e3), "ms_per_pass_of_linac": ms,
            "tracking_kernel_share": kms / ms,
            "roofline": {"bound": "alu", "achieved": ach, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / PEAK_FP64_TFLOPS, "flops_per_pass_of_linac": f,
                         "count": "element model (cos, division = 1 flop) + histogram window/bin/kick 14 per "
                                  "particle per wake + nbins (nbins + 1) per convolution"},
            "launches": times[0][1]["launches"], "steps": steps, "warmup": warmup, "clocks": clk,
            "cpu_baseline": c3_cpu_baseline(lat) if with_cpu else None}


def c3_sweep_record(args):
    """Particle-count sweep of the wake linac (20 of its periods: RF cavity,
    4096-bin wake, drift, quadrupole): one pass for 1e6, 1e7 and 1e8 particles
    as one resident bunch, and for 1e8 particles held in 4 parts whose wakes
    are reduced across the parts (trk_track_parts).  Bunches are drawn on the
    device; passes/s counts every particle through every element."""
    import torch

    import synthetic as syn
    from paper_1710_07350_gb300 import trk
    periods = 20
    lat = syn.lattice_c3(periods=periods)
    L = trk.trk_create_lattice(lat)
    ne = len(lat["elements"])
    out = []
    for n, parts in ((1_000_000, 1), (10_000_000, 1), (100_000_000, 1), (100_000_000, 4)):
        z = syn.c3_bunch_device(n)
        sizes = [n // parts] * parts
        sizes[-1] += n - sum(sizes)
        bunches, keep, start = [], [], 0
        for m in sizes:
            coords = z[:, start:start + m].contiguous() if parts > 1 else z
            ids = torch.arange(start, start + m, dtype=torch.int32, device="cuda")
            b = trk.trk_bunch_wrap(coords, ids, n=m)
            trk.trk_bunch_set_schedule(b, block=args.block, per_thread=args.per_thread)
            bunches.append(b)
            keep.append((coords, ids))
            start += m
        if parts > 1:
            del z
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if parts > 1:
            trk.trk_track_parts(bunches, L, 1)
        else:
            trk.trk_track(bunches[0], L, 1)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out.append({"particles": n, "parts": parts, "ms": ms, "passes_per_s": n * ne / (ms / 1e3)})
        del bunches, keep
        if parts == 1:
            del z
        torch.cuda.empty_cache()
    return {"workload": "c3 wake linac, %d periods (%d elements, 4096-bin wakes), one pass" % (periods, ne),
            "metric": UNIT, "points": out,
            "note": "the first point includes the first launches' set-up; bunches drawn on the device"}


def run_bend(args):
    """Sector-bend ring: 1e6 particles, 16 exact sector dipoles between
    kick-drift quadrupoles and drifts per turn, 100 turns per step."""
    import torch

    import synthetic as syn
    from paper_1710_07350_gb300 import flops, trk
    lat = syn.lattice_bend_ring()
    L = trk.trk_create_lattice(lat)
    n, turns = args.particles, args.turns_per_step
    coords0, ids0 = trk.upload(syn.bend_ring_bunch(n))
    times, work = [], []
    for k in range(args.warmup + args.steps):
        b = trk.trk_bunch_wrap(coords0.clone(), ids0.clone())
        trk.trk_bunch_set_schedule(b, block=args.block, per_thread=args.per_thread)
        trk.trk_bunch_enable_timing(b, True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        trk.trk_track(b, L, turns)
        e1.record()
        e1.synchronize()
        st = trk.trk_bunch_stats(b)
        if k >= args.warmup:
            _, lt, le = trk.trk_lost(b)
            times.append((e0.elapsed_time(e1), st))
            work.append(flops.step_work(lat, n, turns, lt, le))
        del b
    ms = sum(t for t, _ in times) / len(times)
    kms = sum(st["track_kernel_ms"] for _, st in times) / len(times)
    passes = sum(p for p, _ in work) / len(work)
    f = sum(w for _, w in work) / len(work)
    print(json.dumps({"workload": "bend ring: 8 x [SBEND 1.5 m pi/8, D0.4, QF, D0.4, SBEND, D0.4, QD, D0.4], "
                                  "%d particles, %d turns per step" % (n, turns),
                      "metric": UNIT, "value": passes / (ms / 1e3), "ms_per_step": ms,
                      "tracking_kernel_share": kms / ms, "achieved_tflops": f / (ms / 1e3) / 1e12,
                      "frac_of_fp64_peak": f / (ms / 1e3) / 1e12 / PEAK_FP64_TFLOPS,
                      "launches": times[0][1]["launches"], "steps": args.steps, "warmup": args.warmup}))
    return 0


def run_c4(args):
    print(json.dumps(c4_record(args, args.warmup, not args.no_cpu_baseline)))
    return 0


def c4_record(args, warmup, with_cpu, clocks_index=None, plain_stride=1):
    """256 lattice variants (log-uniform 1000..65536 particles), 1000 turns:
    batched (autotuned schedule, one CUDA graph per call) against one
    lattice at a time."""
    import torch

    import synthetic as syn
    from paper_1710_07350_gb300 import trk
    vs = syn.c4_variants()
    lats = [syn.lattice_c4(v) for v in vs]
    Ls = [trk.trk_create_lattice(l) for l in lats]
    inputs = [trk.upload(syn.c4_bunch(k, v[2])) for k, v in enumerate(vs)]
    turns = 1000

    def fresh():
        return [trk.trk_bunch_wrap(c.clone(), i.clone()) for c, i in inputs]

    tuned, probe_ms = trk.trk_autotune(fresh(), Ls, 20)
    n_tot = sum(v[2] for v in vs)
    # the plain arm (one lattice per call) on every 8th variant: its rate is
    # per pass, and the whole set would take ~45 s
    plain_idx = list(range(0, len(vs), plain_stride))
    n_plain = sum(vs[k][2] for k in plain_idx)
    res = {}
    clocks = Clocks(clocks_index, args.clocks_dir) if clocks_index is not None else None
    if clocks is not None:
        clocks.start()
    for mode in ("batched", "plain"):
        best = None
        for k in range(warmup + 1):
            bs = fresh()
            torch.cuda.synchronize()
            t = time.perf_counter()
            if mode == "batched":
                B = trk.trk_batch_create(bs, Ls)
                trk.trk_batch_set_schedule(B, **tuned)
                trk.trk_batch_track(B, turns)
            else:
                for j in plain_idx:
                    trk.trk_bunch_set_schedule(bs[j], block=128, per_thread=2, chunk_turns=100)
                    trk.trk_track(bs[j], Ls[j], turns)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            if k >= warmup:
                best = dt
            if mode == "batched":
                alive = sum(trk.trk_n_alive(b) for b in bs)
        res[mode] = best
    clk = clocks.stop() if clocks is not None else None
    passes = n_tot * 60 * turns
    passes_plain = n_plain * 60 * turns
    # the method's count of every variant (the lattices keep their moments); all particles survive
    from paper_1710_07350_gb300 import flops
    f_tot = sum(flops.step_work(l, v[2], turns)[1] for l, v in zip(lats, vs))
    ach = f_tot / res["batched"] / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / PEAK_FP64_TFLOPS, "flops": f_tot,
            "count": "flops.py element model per pass + 54 per particle-turn for the moments; wall time of the "
                     "batched call, host launch included"}
    return {"workload": "c4: 256 variants of the FODO ring + thin sextupoles, %d particles, 1000 turns" % n_tot,
            "metric": UNIT, "value": passes / res["batched"], "batched_value": passes / res["batched"],
            "plain_value": passes_plain / res["plain"], "batched_s": res["batched"], "plain_s": res["plain"],
            "plain_sample": "every %dth variant (%d variants, %d particles), one call each" % (plain_stride, len(plain_idx),
                                                                                             n_plain),
            "speedup": (passes / res["batched"]) / (passes_plain / res["plain"]), "roofline": roof,
            "autotuned_schedule": tuned,
            "alive_end": alive,
            "note": "passes counted as if all survive; wall time of the calls, host launch included", "clocks": clk,
            "cpu_baseline": c4_cpu_baseline() if with_cpu else None}


def run_mlp(args):
    """Surrogate inference: one call over `rows` feature rows (the DA grid's
    16.8 M cells by default), tcgen05 layers; BF16 tensor FLOP/s counted on
    the unpadded network (8 -> 256 -> 256 -> 256 -> 256 -> 1)."""
    import torch

    import synthetic as syn
    from paper_1710_07350_gb300 import trk
    net = trk.trk_mlp_create(syn.mlp_init(7))
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.rand((args.rows, 8), device="cuda", dtype=torch.float32, generator=g) * 2 - 1
    for _ in range(args.warmup):
        trk.trk_mlp_forward(net, X)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        trk.trk_mlp_forward(net, X)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    flops = args.rows * 2.0 * (8 * 256 + 3 * 256 * 256 + 256)
    print(json.dumps({"workload": "surrogate inference, %d rows" % args.rows, "ms_per_call": ms,
                      "rows_per_s": args.rows / (ms / 1e3), "tflops_bf16": flops / (ms / 1e3) / 1e12,
                      "steps": args.steps, "warmup": args.warmup}))
    return 0


def run_mlp_train(args):
    """Surrogate training as the triaged scan runs it: 262 144 samples (64
    variants x 64 x 64 coarse cells), batch 4096, Adam lr 2e-3, `epochs` epochs."""
    import torch

    import synthetic as syn
    from paper_1710_07350_gb300 import trk
    n = 64 * 64 * 64
    g = torch.Generator(device="cuda").manual_seed(6)
    X = torch.rand((n, 8), device="cuda", dtype=torch.float32, generator=g) * 2 - 1
    y = (X[:, 0] ** 2 + X[:, 1] ** 2 < 0.5).float()
    perm = torch.stack([torch.randperm(n, device="cuda", generator=g) for _ in range(args.epochs)]).int()
    times = []
    for k in range(args.warmup + args.steps):
        net = trk.trk_mlp_create(syn.mlp_init(7))
        torch.cuda.synchronize()
        t = time.perf_counter()
        trk.trk_mlp_train(net, X, y, batch=4096, epochs=args.epochs, perm=perm, lr=2e-3)
        torch.cuda.synchronize()
        if k >= args.warmup:
            times.append(time.perf_counter() - t)
    steps = args.epochs * ((n + 4095) // 4096)
    s = sum(times) / len(times)
    print(json.dumps({"workload": "surrogate training, %d samples, batch 4096, %d epochs" % (n, args.epochs),
                      "seconds": s, "adam_steps": steps, "us_per_step": 1e6 * s / steps,
                      "steps": args.steps, "warmup": args.warmup}))
    return 0


def run_sweep(args):
    print(json.dumps({"workload": "c1 map ring particle-count sweep (order 2 and 3 maps)", "metric": UNIT,
                      "points": map_sweep_points()}))
    return 0


def map_sweep_points():
    """Particle-count sweep of the c1 map ring (10 FODO cells, 40 order-2 or
    order-3 maps, rectangle 20 mm): passes/s for N = 1e4 .. 1e8 particles, each
    point about 1e8 particle-turns (turns = 1e8 / N, 1 to 1000) in one launch
    configuration (block 128, 2 particles per thread, 100-turn chunks)."""
    import torch

    import synthetic as syn
    from paper_1710_07350_gb300 import flops, trk
    out = []
    for order in (2, 3):
        lat = syn.lattice_c1(order=order)
        L = trk.trk_create_lattice(lat, moments=False)
        f_pass = float(np.mean(flops.lattice_pass_flops(lat)))
        for n in (10_000, 100_000, 1_000_000, 10_000_000, 100_000_000):
            turns = int(min(1000, max(1, round(1e8 / n))))
            g = torch.Generator(device="cuda").manual_seed(9)
            coords = torch.zeros((6, n), dtype=torch.float64, device="cuda")
            coords[0].normal_(0.0, 2e-4, generator=g)
            coords[2].normal_(0.0, 1e-4, generator=g)
            coords[5].normal_(0.0, 1e-3, generator=g)
            ids = torch.arange(n, dtype=torch.int32, device="cuda")
            b = trk.trk_bunch_wrap(coords, ids)
            trk.trk_bunch_set_schedule(b, block=128, per_thread=2, chunk_turns=100)
            trk.trk_track(b, L, 1)                      # warm-up (first launch, scratch allocation)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            trk.trk_track(b, L, turns)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            alive = trk.trk_n_alive(b)
            passes = float(n) * turns * len(lat["elements"])   # counted as if all survive
            out.append({"order": order, "particles": n, "turns": turns, "ms": ms,
                        "passes_per_s": passes / (ms / 1e3),
                        "tflops": passes * f_pass / (ms / 1e3) / 1e12, "alive_end": alive})
            del b, coords, ids
            torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c3":
        return run_c3(args)
    if args.workload == "c4":
        return run_c4(args)
    if args.workload == "mlp":
        return run_mlp(args)
    if args.workload == "mlp-train":
        return run_mlp_train(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "c3sweep":
        print(json.dumps(c3_sweep_record(args)))
        return 0
    if args.workload == "bend":
        return run_bend(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
