#!/usr/bin/env python
"""Benchmark: photon packets/s and time-to-converged temperature on one GB300.

Workload (one "step"): the flared passive disk on a spherical-polar grid (nr = 200 log-spaced
over 1-1000 AU, ntheta = 128 concentrated at the midplane, nphi = 1, rho ~ r^-1 exp(-z^2/2h^2),
h = 10 AU (r/100 AU)^1.125, radial 550 nm optical depth 100), a 5800 K 1 Lsun star, 1e7 packets
per Lucy iteration, 10 iterations, then one peel-off pass of 1e7 packets into SEDs at 10
inclinations x 250 wavelength bins.  Inputs are synthetic (no dataset).

value     packets propagated per second over the whole step (iterations + peel-off pass), device
          time by CUDA events on the library's stream, inputs resident in HBM; L2 is flushed
          between timed steps (the disk's cell data fit in L2).
e2e       the same step through the C ABI with host buffers: density and starting temperatures
          copied from pinned host memory, temperatures and SEDs copied back, all inside the
          timed region.
roofline  the propagation kernel: algorithmic bytes per launch (20 B per packet cell crossing:
          FP32 density + FP64 accumulator read-modify-write; 4 B per peel-off crossing; 400 B per
          re-emission row) over its measured duration, against the measured HBM copy bandwidth.
time_to_converged_ms      device time of the Lucy iterations until the 99th percentile of the
          iteration change in T is below 2 % (null when the 10 iterations never get there: the
          Monte-Carlo noise of the disk's optically thick midplane is then the floor).
time_to_converged_pda_ms  the same from a separate solve (not in `value`) in which cells entered
          by fewer than --pda-min packets take the partial diffusion approximation (App. A).

``--rows`` instead measures the extensions of the method on their own workloads (one JSON line, not
the headline): the modified random walk against the plain walk on thick grey models and an
embedded envelope, raytracing against peel-off in the disk's imaging pass, Lucy iterations on the
cylindrical disk and the clouds in an external radiation field.

``--impl reference`` times the FP64 CPU oracle (the reference implementation of this build) on
the host cores on a bounded sample of the same workload.  N > 1 GPUs (torchrun) run independent
disk models, one per rank (weak scaling, no collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "photon packets/sec (flared-disk Lucy solve + peel-off SEDs)"
UNIT = "packets/s"
B_CROSS = 20.0
B_PEEL = 4.0
B_REEMIT = 400.0
# DRAM bytes (read + write) per propagation launch, averaged over a step's 12 launches (10 Lucy
# iterations, the imaging pass and its peel pass), from an ncu capture of the current kernels on
# a 2e5-packet case of this workload scaled to 1e7 packets: the Lucy launches touch the resident
# grid and tables once (0.58 MB, independent of the packet count); the peel-event queue (48 B
# per event, 4.74e6 events) and its cell order grow with the packets: 228 MB written by the
# imaging pass, 247 MB read by the peel pass
TRAFFIC_PER_LAUNCH = 40.1e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--kernel", choices=["event", "plain"], default="event")
    ap.add_argument("--packets", type=int, default=10_000_000)
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target length of the CPU oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows", action="store_true",
                    help="measure the extension rows (MRW, raytracing, cylindrical grids, external field) instead")
    ap.add_argument("--pda-min", type=int, default=6000,
                    help="packet entries below which a cell takes the diffusion approximation in the "
                         "time-to-converged solve with PDA (App. A); 0 skips that solve")
    return ap.parse_args()


def workload(n_packets, rank=0):
    from paper_1112_1071_gb300 import workloads as W
    return W.flared_disk(n_packets=n_packets, seed=2 + rank)


def config(args, world):
    return {"workload": "flared_disk spherical 200x128x1, tau_550=100, 1 star; "
                        f"{args.packets:.0e} packets x {args.iters} Lucy iterations + 1 peel-off pass "
                        "(10 inclinations x 250 bins)",
            "grid": "spherical-polar nr=200 ntheta=128 nphi=1", "packets_per_iteration": args.packets,
            "iterations": args.iters, "observers": 10, "sed_bins": 250,
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}",
            "kernel": args.kernel}


def job_throughput(total_ms, e2e_ms, world, packets_step, steps, dist=None, device="cpu"):
    """Whole-job packets/s over `world` ranks that each ran `steps` timed steps of
    `packets_step` packets: the slowest rank's timed total and mean end-to-end step (max over
    ranks) set the time.  Returns (value, e2e value, total_ms, e2e_ms) after the reduction."""
    if dist is not None:
        import torch
        tt = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms, e2e_ms = float(tt[0]), float(tt[1])
    value = world * packets_step * steps / (total_ms * 1e-3)
    return value, world * packets_step / (e2e_ms * 1e-3), total_ms, e2e_ms


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle (CPU) timing
def cpu_oracle_rate(args, seconds):
    """Packets/s of the FP64 oracle on all host cores (threads over packet ranges with private
    accumulators), one Lucy iteration of the disk at its cold-start temperatures, on a packet
    sample sized to take about `seconds`."""
    from oracle.mc import OracleModel
    wl = workload(args.packets)
    om = OracleModel(wl)
    cores = os.cpu_count() or 1
    n = 20_000
    t0 = time.perf_counter()
    om.run_packets(n, 0, nthreads=cores)
    dt = time.perf_counter() - t0
    n2 = int(min(max(n, n * seconds / max(dt, 1e-3)), args.packets))
    t0 = time.perf_counter()
    om.run_packets(n2, 0, nthreads=cores)
    dt2 = time.perf_counter() - t0
    return n2 / dt2, cores, n2, dt2


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    times, rates = [], []
    seconds = max(2.0, min(args.cpu_seconds, 200.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        r, cores, n, dt = cpu_oracle_rate(args, seconds)
        if i >= args.warmup:
            rates.append(r)
            times.append(dt)
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} packets of one Lucy iteration of the disk per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.rows:
        return rows_bench(local)

    import numpy as np
    import torch
    from paper_1112_1071_gb300 import hrt

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    wl = workload(args.packets, rank)
    m = hrt.Model(wl, device=local, stream=stream)
    L = hrt.load()
    kern = hrt.HRT_KERNEL_EVENT if args.kernel == "event" else hrt.HRT_KERNEL_PLAIN
    nc = m.ncells
    T0 = torch.full((nc,), 10.0, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2

    def solve(stats):
        """One step: Lucy iterations from the cold start, then the peel-off pass."""
        hrt.check(m.ctx, L.hrt_set_temperature_device(m.ctx, T0.data_ptr(), nc))
        hrt.check(m.ctx, L.hrt_set_iteration(m.ctx, 0))
        for _ in range(args.iters):
            stats.append(m.run_iteration(n_packets=args.packets, kernel=kern))
        stats.append(m.run_iteration(n_packets=args.packets, kernel=kern, peel=1, update_temperature=0))

    # warm-up
    for _ in range(args.warmup):
        solve([])
    barrier()
    clocks = Clocks(local)
    clocks.start()
    step_ms, all_stats, conv = [], [], []
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        st = []
        ev0.record(stream)
        solve(st)
        ev1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        all_stats.append(st)
        # time to the 2% criterion: iterations until Q_99(delta T) < 1.02
        t, it_conv = 0.0, None
        for i, s in enumerate(st[:-1]):
            t += s["ms_total"]
            if s["converged"] and i > 0:
                it_conv = i + 1
                break
        conv.append((it_conv, t if it_conv else None))
    # time to the 2% criterion with the partial diffusion approximation (App. A) for the cells
    # entered by fewer than --pda-min packets (not part of the timed throughput steps)
    conv_pda, pda_q, pda_cells = [], [], 0
    if args.pda_min > 0:
        for _ in range(args.steps):
            hrt.check(m.ctx, L.hrt_set_temperature_device(m.ctx, T0.data_ptr(), nc))
            hrt.check(m.ctx, L.hrt_set_iteration(m.ctx, 0))
            t, it_conv, qh = 0.0, None, []
            for i in range(args.iters):
                s = m.run_iteration(n_packets=args.packets, kernel=kern, pda_min_visits=args.pda_min)
                t += s["ms_total"]
                qh.append(round(s["Q"], 5))
                pda_cells = s["n_pda"]
                if s["converged"] and i > 0:
                    it_conv = i + 1
                    break
            conv_pda.append((it_conv, t if it_conv else None))
            pda_q = qh
    barrier()
    clk = clocks.stop()

    # ---- end-to-end through the C ABI with host buffers
    rho_h = torch.from_numpy(np.ascontiguousarray(wl.rho.reshape(-1), dtype=np.float32)).pin_memory()
    T0_h = torch.full((nc,), 10.0, dtype=torch.float64).pin_memory()
    T_out = torch.empty(nc, dtype=torch.float64).pin_memory()
    sed_out = torch.empty(m.nobs * wl.nsed, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(max(1, args.steps)):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        hrt.check(m.ctx, L.hrt_set_density(m.ctx, rho_h.data_ptr(), nc))
        hrt.check(m.ctx, L.hrt_set_temperature(m.ctx, T0_h.data_ptr(), nc))
        hrt.check(m.ctx, L.hrt_set_iteration(m.ctx, 0))
        for _ in range(args.iters):
            m.run_iteration(n_packets=args.packets, kernel=kern)
        m.run_iteration(n_packets=args.packets, kernel=kern, peel=1, update_temperature=0)
        hrt.check(m.ctx, L.hrt_get_temperature(m.ctx, T_out.data_ptr(), nc))
        hrt.check(m.ctx, L.hrt_get_sed(m.ctx, sed_out.data_ptr(), sed_out.numel()))
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    barrier()

    packets_step = args.packets * (args.iters + 1)
    ms = statistics.mean(step_ms)
    value, e2e_value, _, _ = job_throughput(sum(step_ms), statistics.mean(e2e_ms), world, packets_step, args.steps,
                                            dist, "cuda")

    # ---- roofline of the propagation kernel (Lucy iterations and the peel-off pass)
    last = all_stats[-1]
    byts = sum(B_CROSS * s["n_crossings"] + B_PEEL * s["n_peel_crossings"] + B_REEMIT * (s["n_absorb"]) for s in last)
    kms = sum(s["ms_propagate"] for s in last)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, src = float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        peak, src = 6800.0, "fallback"
    achieved = byts / (kms * 1e-3) / 1e9
    launches = sum(s["kernel_launches"] for st in all_stats for s in st)
    its, tconv = zip(*conv)
    done = [t for t in tconv if t is not None]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": config(args, world),
            "time_to_converged_ms": statistics.median(done) if done else None,
            "q99_history": [round(s["Q"], 5) for s in last[:-1]],
            "iterations_to_converged": statistics.median([i for i in its if i]) if any(its) else None,
            "time_to_converged_pda_ms": statistics.median([t for _, t in conv_pda if t is not None])
            if any(t is not None for _, t in conv_pda) else None,
            "pda": {"min_visits": args.pda_min, "cells": pda_cells, "q99_history": pda_q,
                    "iterations_to_converged": statistics.median([i for i, _ in conv_pda if i])
                    if any(i for i, _ in conv_pda) else None} if args.pda_min > 0 else None,
            "crossings_per_step": sum(s["n_crossings"] for s in last),
            "peel_crossings_per_step": sum(s["n_peel_crossings"] for s in last),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": TRAFFIC_PER_LAUNCH if kern == hrt.HRT_KERNEL_EVENT else None,
                         "traffic_unit": "bytes per launch (ncu)", "peak_source": src,
                         "kernel": "k_event + k_peel_rays (propagation)" if kern == hrt.HRT_KERNEL_EVENT else "k_plain",
                         "kernel_ms_per_step": kms, "algorithmic_bytes_per_step": byts},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(rho_h.numel() * 4 + T0_h.numel() * 8),
                    "d2h_bytes_per_step": int(T_out.numel() * 8 + sed_out.numel() * 8)},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        if not args.no_cpu_baseline:
            r, cores, n, dt = cpu_oracle_rate(args, args.cpu_seconds)
            line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": f"{n} packets of one Lucy iteration of the disk ({dt:.1f} s)"}
        print(json.dumps(line), flush=True)
    m.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def rows_bench(local):
    """Device times (ms_propagate, CUDA events on the library stream) of the extension rows."""
    import numpy as np
    import torch
    from paper_1112_1071_gb300 import hrt
    from paper_1112_1071_gb300 import workloads as W
    torch.cuda.set_device(local)
    out = {}

    # modified random walk: thick grey models, 1e6 packets, 2nd iteration, gamma 2 / 4 / off
    mrw = {}
    for kind in ("cartesian", "spherical", "cylindrical"):
        wl = W.thick_grey(kind, 1_000_000)
        rows, T = {}, {}
        for gamma in (2.0, 4.0, 0.0):
            m = hrt.Model(wl, device=local)
            for _ in range(2):
                st = m.run_iteration(mrw_gamma=gamma, watchdog_ms=120000)
            rows[f"gamma_{gamma:g}"] = {"ms": st["ms_propagate"], "interactions_per_packet": st["n_interactions"] / 1e6,
                                        "mrw_steps_per_packet": st["n_mrw"] / 1e6, "killed": st["n_killed"]}
            T[gamma] = m.temperature()
        for gamma in (2.0, 4.0):
            d = (T[gamma] - T[0.0]) / T[0.0]
            rows[f"gamma_{gamma:g}"]["dT_vs_plain_mean"] = float(np.abs(d).mean())
        mrw[kind] = rows
    # embedded envelope, tau_550 = 1e5, 1e5 packets, 5 iterations from 10 K
    env = {}
    for gamma in (2.0, 0.0):
        m = hrt.Model(W.embedded_envelope(tau_550=1e5, n_packets=100_000), device=local)
        ms, killed = 0.0, 0
        for _ in range(5):
            st = m.run_iteration(mrw_gamma=gamma, watchdog_ms=120000)
            ms += st["ms_propagate"]
            killed = st["n_killed"]
        env[f"gamma_{gamma:g}"] = {"ms_5_iterations": ms, "killed_last_iteration": killed,
                                   "interactions_per_packet_last": st["n_interactions"] / 1e5}
    mrw["embedded_envelope_tau1e5"] = env
    out["mrw"] = mrw

    # raytracing against peel-off in the disk's imaging pass (1e7 packets, 1e6 dust rays)
    m = hrt.Model(W.flared_disk(n_packets=10_000_000), device=local)
    for _ in range(4):
        m.run_iteration()
    rt = {}
    for rays in (0, 1_000_000):
        st = m.run_iteration(peel=1, update_temperature=0)
        st = m.run_iteration(peel=1, update_temperature=0, raytrace_rays=rays)
        rt[f"rays_{rays}"] = {"ms": st["ms_total"], "peel_crossings": st["n_peel_crossings"]}
    out["raytracing_disk"] = rt

    # Lucy iterations on the cylindrical disk (with external field) and the ISRF clouds
    lucy = {}
    for name, wl in (("cylindrical_disk_isrf", W.cylindrical_disk(n_packets=10_000_000, isrf_dilution=1e-13)),
                     ("isrf_cloud_cartesian", W.isrf_cloud("cartesian", n=64, tau_550=3.0, n_packets=10_000_000)),
                     ("isrf_cloud_spherical", W.isrf_cloud("spherical", n=64, tau_550=3.0, n_packets=10_000_000)),
                     ("isrf_cloud_cylindrical", W.isrf_cloud("cylindrical", n=64, tau_550=3.0, n_packets=10_000_000))):
        m = hrt.Model(wl, device=local)
        for _ in range(3):
            st = m.run_iteration()
        lucy[name] = {"ms": st["ms_propagate"], "packets_per_s": wl.n_packets / (st["ms_propagate"] * 1e-3),
                      "crossings_per_s": st["n_crossings"] / (st["ms_propagate"] * 1e-3)}
    out["lucy_iterations"] = lucy
    print(json.dumps(out))


if __name__ == "__main__":
    sys.exit(main())
