#!/usr/bin/env python
"""Benchmark: photon packets/s and time-to-converged temperature on one GB300.

Workload (one "step", the default ``--workload cloud``): the 3D turbulent cloud, a Cartesian
256^3 grid over a 0.65 pc box with rho = exp(1.5 G), G a k^-11/3 Gaussian random field scaled to
a mean 550 nm optical depth of 10 across the box, 20 stars uniform in the box (T 3000-20000 K,
L 0.1-100 Lsun).  A step is the solve: ``--iters`` (5) Lucy iterations of 1e8 packets from the
10 K cold start, then one imaging pass of 1e8 packets peeled off into 512 x 512 images at 6
wavelengths (1.25, 3.6, 8, 70, 250, 500 um) and the SED at (theta, phi) = (45, 45) degrees.
The cloud's density (64 MiB) and FP64 accumulators (128 MiB) exceed L2.  Inputs are synthetic.

value     packets propagated per second over the whole step (Lucy iterations + imaging pass),
          device time by CUDA events on the library's stream, inputs resident in HBM; L2 is
          flushed (256 MiB write) between timed steps.
e2e       the same step through the C ABI with host buffers: density and starting temperatures
          copied from pinned host memory, temperatures, SED and images copied back, all inside
          the timed region.
roofline  the Lucy propagation kernel (k_event, one launch per iteration): algorithmic bytes per
          launch (20 B per cell crossing: FP32 density + FP64 accumulator read-modify-write;
          400 B per re-emission row) over its CUDA-event duration, against the measured HBM copy
          bandwidth.  `traffic` is the DRAM bytes ncu measured per launch (summary under profiles/).
time_to_converged_ms        device time of the Lucy iterations until the 99th percentile of the
          iteration change of T is below 2 % (Q_99(dT) < 1.02, Eqs. 4-5); null when the Monte-Carlo
          noise floor of Q_99 lies above 1.02 at this packet count (`q99_history` shows the floor).
time_to_converged_delta_ms  the same until the 99th percentile itself changes by less than 2 %
          between iterations (Eq. 6's Delta test, with Q_99 < 2): the iteration has reached its
          noise floor.
plain_gpu  the same step with the one-thread-per-history kernel (k_plain).
cpu_baseline  the FP64 oracle on all host cores on the same mix of passes: a packet sample of a
          cold-start Lucy iteration, of a Lucy iteration at the oracle's own later temperatures and
          of the imaging pass, each rate weighted by the step's packets in that kind of pass.
flared_disk  the L2-resident workload (spherical 200 x 128 x 1 disk, 1e7 packets x 10 iterations
          + a peel-off pass at 10 inclinations x 250 bins), with its kernel's L2 bytes and FP64
          atomics against an L2 copy and an L2 FP64 atomic rate measured in the same process.

``--rows`` instead measures the extensions of the method on their own workloads (one JSON line, not
the headline): the modified random walk against the plain walk on thick grey models and an
embedded envelope, raytracing against peel-off in the disk's imaging pass, Lucy iterations on the
cylindrical disk and the clouds in an external radiation field.

``--impl reference`` times the FP64 CPU oracle (the reference implementation of this build) on
the host cores on a bounded sample of the same workload.  N > 1 GPUs (torchrun) run independent
models, one per rank (weak scaling, no collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "photon packets/sec (Lucy solve + peel-off imaging pass)"
UNIT = "packets/s"
B_CROSS = 20.0
B_PEEL = 4.0
B_REEMIT = 400.0
# DRAM bytes (read + write) per crossing of the Lucy propagation kernel on the 256^3 cloud, from
# an ncu capture of the current k_event (the third Lucy launch of 5e6 packets on the full grid:
# 58.3 GB for 9.55e8 crossings; DRAM traffic there comes from the cache misses of the walk, so it
# grows with the crossings): per launch = this x the launch's crossings
TRAFFIC_PER_CROSSING = 61.1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["cloud", "disk"], default="cloud")
    ap.add_argument("--kernel", choices=["event", "plain"], default="event")
    ap.add_argument("--packets", type=int, default=None, help="packets per pass (cloud 1e8, disk 1e7)")
    ap.add_argument("--iters", type=int, default=None, help="Lucy iterations per step (cloud 5, disk 10)")
    ap.add_argument("--cpu-seconds", type=float, default=18.0, help="target length of the CPU oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the plain-kernel arm and the disk line")
    ap.add_argument("--rows", action="store_true",
                    help="measure the extension rows (MRW, raytracing, cylindrical grids, external field) instead")
    ap.add_argument("--learned", action="store_true",
                    help="time to converged temperatures of held-out 128^3 clouds: the learned warm start plus "
                         "batching against the plain GPU iteration (one JSON line, not the headline)")
    ap.add_argument("--learned-fields", type=int, default=256, help="training fields generated for --learned")
    ap.add_argument("--learned-epochs", type=int, default=10)
    ap.add_argument("--batch", action="store_true",
                    help="the 512 uneven disks of the batched workload at full packet budgets: one persistent "
                         "launch per iteration against the same models one after the other (one JSON line)")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="packet-budget scale for --batch")
    ap.add_argument("--pda-min", type=int, default=6000,
                    help="disk line: packet entries below which a cell takes the diffusion approximation in "
                         "the time-to-converged solve with PDA (App. A); 0 skips that solve")
    a = ap.parse_args()
    if a.packets is None:
        a.packets = 100_000_000 if a.workload == "cloud" else 10_000_000
    if a.iters is None:
        a.iters = 5 if a.workload == "cloud" else 10
    return a


def workload(n_packets, rank=0, name="cloud"):
    """The step's model; rank r of a multi-GPU run gets its own seed (an independent model)."""
    from paper_1112_1071_gb300 import workloads as W
    if name == "cloud":
        return W.turbulent_cloud(n_packets=n_packets, seed=4 + rank)
    return W.flared_disk(n_packets=n_packets, seed=2 + rank)


def describe(name, packets, iters):
    if name == "cloud":
        return (f"turbulent_cloud Cartesian 256^3, 0.65 pc, sigma_lnrho=1.5, mean tau_550=10, 20 stars; "
                f"{packets:.0e} packets x {iters} Lucy iterations from 10 K + 1 imaging pass "
                f"(512x512 images at 6 wavelengths, 1 observer)")
    return (f"flared_disk spherical 200x128x1, tau_550=100, 1 star; {packets:.0e} packets x {iters} Lucy "
            f"iterations from 10 K + 1 peel-off pass (10 inclinations x 250 bins)")


def config(args, world):
    c = {"workload": describe(args.workload, args.packets, args.iters), "packets_per_iteration": args.packets,
         "iterations": args.iters, "l2": "flushed between timed steps (256 MiB write)",
         "parallelism": f"replicas x{world}", "kernel": args.kernel}
    if args.workload == "cloud":
        c.update(grid="cartesian 256x256x256", sources=20, images="6 x 512 x 512", observers=1, sed_bins=250)
    else:
        c.update(grid="spherical-polar nr=200 ntheta=128 nphi=1", observers=10, sed_bins=250)
    return c


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


def converged_at(qs, ms, q_thres=1.02, delta_thres=None):
    """First iteration (1-based, at least the 2nd) that meets the criterion, and the device time
    of the iterations up to it: Q_99 < q_thres, and with delta_thres also Delta = max(Q_prev/Q,
    Q/Q_prev) < delta_thres (Eqs. 5-6).  (None, None) when no iteration meets it."""
    t = 0.0
    for i, (q, m) in enumerate(zip(qs, ms)):
        t += m
        if i == 0:
            continue
        ok = q < q_thres
        if delta_thres is not None:
            ok = ok and max(qs[i - 1] / q, q / qs[i - 1]) < delta_thres
        if ok:
            return i + 1, t
    return None, None


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
_ORACLE_CACHE = {}


def cpu_oracle_rate(wl, iters, seconds, cores=None, refresh=False):
    """Packets/s of the FP64 oracle on all host cores (threads over packet ranges with private
    accumulators) on the step's mix of passes: the cold-start Lucy iteration, a Lucy iteration at
    the oracle's own temperatures after it (the later iterations) and the imaging pass at those
    temperatures.  The first call times each kind of pass at two packet counts, which separates
    its fixed cost (per-thread accumulators over every cell, their sum, the temperature update)
    from its cost per packet; refresh=True re-times one sample of each kind and updates the cost
    per packet (the fixed costs are kept).  The step's CPU time is the sum over its passes of
    (fixed + packets x per packet), for 1, iters - 1 and 1 passes of wl.n_packets; the samples
    take about seconds / 3 each.  Returns (rate, cores, description)."""
    from oracle.mc import OracleModel
    cores = cores or os.cpu_count() or 1
    st = _ORACLE_CACHE.get(id(wl))
    if st is None:
        st = _ORACLE_CACHE[id(wl)] = {"om": OracleModel(wl)}
    om = st["om"]
    part = max(seconds / 3.0, 0.05)

    def cold(n):
        om.T[:] = 10.0
        om.iteration, om.Q_prev = 0, None
        om.run_iteration(n_packets=n, nthreads=cores)

    def lucy(n):
        om.T[:] = st["T1"]
        om.run_packets(n, st["it1"], nthreads=cores)

    def imaging(n):
        om.T[:] = st["T1"]
        om.run_packets(n, 0x80000000 | st["it1"], peel=True, nthreads=cores)

    def timed(fn, n):
        t0 = time.perf_counter()
        fn(n)
        return time.perf_counter() - t0

    def model(fn):
        n0 = max(256, cores * 16)
        t0 = timed(fn, n0)
        n1 = 8 * n0
        per = max((timed(fn, n1) - t0) / (n1 - n0), 1e-9)
        n2 = int(min(max(n1, n0 + part / per), wl.n_packets))
        t2 = timed(fn, n2)
        per = max((t2 - t0) / (n2 - n0), 1e-9)
        return [max(t0 - per * n0, 0.0), per, n2, t2]

    kinds = (("cold", cold), ("lucy", lucy), ("imaging", imaging))
    if "cost" not in st:
        st["cost"] = {}
        st["cost"]["cold"] = model(cold)
        cold(max(256, min(wl.n_packets, int(part / st["cost"]["cold"][1]))))    # the later passes' T
        st["T1"], st["it1"] = om.T.copy(), om.iteration
        st["cost"]["lucy"] = model(lucy)
        st["cost"]["imaging"] = model(imaging)
    elif refresh:
        for name, fn in kinds:
            c = st["cost"][name]
            n = int(min(max(256, part / c[1]), wl.n_packets))
            t = timed(fn, n)
            c[1], c[2], c[3] = max((t - c[0]) / n, 1e-9), n, t
    (f1, c1, n1, t1), (f2, c2, n2, t2), (f3, c3, n3, t3) = (st["cost"][k] for k, _ in kinds)
    N = wl.n_packets
    t_step = (f1 + N * c1) + (iters - 1) * (f2 + N * c2) + (f3 + N * c3)
    rate = N * (iters + 1) / t_step
    desc = (f"fixed cost per pass + packets/s from a small and a large sample of each kind of pass: "
            f"cold-start Lucy iteration {f1:.2f} s + {1 / c1:.3g} packets/s ({n1} packets, {t1:.1f} s), "
            f"Lucy iteration at the oracle's own T after it {f2:.2f} s + {1 / c2:.3g} packets/s ({n2}, {t2:.1f} s), "
            f"imaging pass {f3:.2f} s + {1 / c3:.3g} packets/s ({n3}, {t3:.1f} s); the step is 1 + {iters - 1} + 1 "
            f"passes of {N:.3g} packets")
    return rate, cores, desc


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    wl = workload(args.packets, 0, args.workload)
    times, rates, desc, cores = [], [], "", 1
    seconds = max(0.3, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    cpu_oracle_rate(wl, args.iters, seconds)         # the cost model (fixed costs per kind of pass)
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r, cores, desc = cpu_oracle_rate(wl, args.iters, seconds, refresh=True)
        if i >= args.warmup:
            rates.append(r)
            times.append(time.perf_counter() - t0)
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step: " + desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def l2_peaks(torch):
    """L2-resident peaks measured in this process with CUDA events: the best copy rate over buffer
    pairs of 2-24 MiB (both buffers in L2; read + write bytes) and FP64 atomic adds (index_add_) of
    2^26 values into 25,600 accumulators (the disk's cell count; the index and value streams come
    from HBM)."""
    dev = "cuda"
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l2_gbs, l2_size = 0.0, 0
    for mib in (2, 4, 8, 16, 24):
        a = torch.empty(mib * 1024 * 1024 // 4, dtype=torch.float32, device=dev).uniform_()
        b = torch.empty_like(a)
        for _ in range(5):
            b.copy_(a)
        reps = max(20, 1200 // mib)
        for _ in range(3):
            ev0.record()
            for _ in range(reps):
                b.copy_(a)
            ev1.record()
            torch.cuda.synchronize()
            gbs = 2 * a.numel() * 4 * reps / (ev0.elapsed_time(ev1) * 1e-3) / 1e9
            if gbs > l2_gbs:
                l2_gbs, l2_size = gbs, mib
        del a, b
    n = 1 << 26
    acc = torch.zeros(25600, dtype=torch.float64, device=dev)
    idx = torch.randint(0, 25600, (n,), device=dev)
    val = torch.ones(n, dtype=torch.float64, device=dev)
    acc.index_add_(0, idx, val)
    best = float("inf")
    for _ in range(5):
        ev0.record()
        acc.index_add_(0, idx, val)
        ev1.record()
        torch.cuda.synchronize()
        best = min(best, ev0.elapsed_time(ev1))
    atom = n / (best * 1e-3)
    del acc, idx, val
    return {"l2_copy_gbs": l2_gbs, "l2_fp64_atomics_per_s": atom,
            "how": f"CUDA events: best copy rate over 2-24 MiB buffer pairs (best at {l2_size} MiB); index_add_ of "
                   "2^26 FP64 values into 25,600 accumulators (best of 5)"}


class Runner:
    """One model in one libhrt context and the step that `bench.py` times on it."""

    def __init__(self, hrt, torch, wl, local, stream, kernel, iters):
        self.hrt, self.torch, self.wl, self.iters = hrt, torch, wl, iters
        self.m = hrt.Model(wl, device=local, stream=stream)
        self.L = hrt.load()
        self.kern = hrt.HRT_KERNEL_EVENT if kernel == "event" else hrt.HRT_KERNEL_PLAIN
        self.nc = self.m.ncells
        self.T0 = torch.full((self.nc,), 10.0, dtype=torch.float64, device="cuda")

    def solve(self, stats, pda_min=0, peel=True):
        """One step on device-resident inputs: Lucy iterations from the cold start, then the
        imaging pass."""
        hrt, m = self.hrt, self.m
        hrt.check(m.ctx, self.L.hrt_set_temperature_device(m.ctx, self.T0.data_ptr(), self.nc))
        hrt.check(m.ctx, self.L.hrt_set_iteration(m.ctx, 0))
        for _ in range(self.iters):
            stats.append(m.run_iteration(n_packets=self.wl.n_packets, kernel=self.kern, pda_min_visits=pda_min))
        if peel:
            stats.append(m.run_iteration(n_packets=self.wl.n_packets, kernel=self.kern, peel=1, update_temperature=0))

    def timed_steps(self, steps, warmup, stream, barrier, flush):
        torch = self.torch
        for _ in range(warmup):
            self.solve([])
        barrier()
        ms, stats = [], []
        for _ in range(steps):
            flush.zero_()
            barrier()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            st = []
            ev0.record(stream)
            self.solve(st)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
            stats.append(st)
        return ms, stats

    def e2e_steps(self, steps, barrier, flush):
        """The step through the C ABI with pinned host buffers, copies inside the timed region."""
        import numpy as np
        torch, hrt, m, L, nc = self.torch, self.hrt, self.m, self.L, self.nc
        rho_h = torch.from_numpy(np.ascontiguousarray(self.wl.rho.reshape(-1), dtype=np.float32)).pin_memory()
        T0_h = torch.full((nc,), 10.0, dtype=torch.float64).pin_memory()
        T_out = torch.empty(nc, dtype=torch.float64).pin_memory()
        sed_out = torch.empty(m.nobs * self.wl.nsed, dtype=torch.float64).pin_memory()
        nimg = len(self.wl.img_lam_um) if self.wl.img_nx > 0 else 0
        img_out = torch.empty(max(1, m.nobs * nimg * self.wl.img_nx * self.wl.img_ny), dtype=torch.float64).pin_memory()
        out = []
        for _ in range(max(1, steps)):
            flush.zero_()
            barrier()
            t0 = time.perf_counter()
            hrt.check(m.ctx, L.hrt_set_density(m.ctx, rho_h.data_ptr(), nc))
            hrt.check(m.ctx, L.hrt_set_temperature(m.ctx, T0_h.data_ptr(), nc))
            hrt.check(m.ctx, L.hrt_set_iteration(m.ctx, 0))
            for _ in range(self.iters):
                m.run_iteration(n_packets=self.wl.n_packets, kernel=self.kern)
            m.run_iteration(n_packets=self.wl.n_packets, kernel=self.kern, peel=1, update_temperature=0)
            hrt.check(m.ctx, L.hrt_get_temperature(m.ctx, T_out.data_ptr(), nc))
            hrt.check(m.ctx, L.hrt_get_sed(m.ctx, sed_out.data_ptr(), sed_out.numel()))
            if nimg:
                hrt.check(m.ctx, L.hrt_get_image(m.ctx, img_out.data_ptr(), img_out.numel()))
            torch.cuda.synchronize()
            out.append(1e3 * (time.perf_counter() - t0))
        h2d = int(rho_h.numel() * 4 + T0_h.numel() * 8)
        d2h = int(T_out.numel() * 8 + sed_out.numel() * 8 + (img_out.numel() * 8 if nimg else 0))
        return out, h2d, d2h

    def close(self):
        self.m.close()


def convergence_fields(stats_steps, iters):
    qs = [[s["Q"] for s in st[:iters]] for st in stats_steps]
    ms = [[s["ms_total"] for s in st[:iters]] for st in stats_steps]
    lit = [converged_at(q, m, 1.02) for q, m in zip(qs, ms)]
    dlt = [converged_at(q, m, 2.0, 1.02) for q, m in zip(qs, ms)]

    def med(v):
        v = [x for x in v if x is not None]
        return statistics.median(v) if v else None
    return {"time_to_converged_ms": med([t for _, t in lit]),
            "iterations_to_converged": med([i for i, _ in lit]),
            "time_to_converged_delta_ms": med([t for _, t in dlt]),
            "iterations_to_converged_delta": med([i for i, _ in dlt]),
            "q99_history": [round(q, 5) for q in qs[-1]]}


def lucy_roofline(last, iters, peak, src):
    """Roofline of the Lucy propagation kernel: mean over the step's Lucy launches."""
    lucy = last[:iters]
    byts = statistics.mean(B_CROSS * s["n_crossings"] + B_REEMIT * s["n_absorb"] for s in lucy)
    kms = statistics.mean(s["ms_propagate"] for s in lucy)
    cross = statistics.mean(s["n_crossings"] for s in lucy)
    achieved = byts / (kms * 1e-3) / 1e9
    traffic = TRAFFIC_PER_CROSSING * cross if TRAFFIC_PER_CROSSING else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_unit": "DRAM bytes per launch (ncu)", "peak_source": src,
            "kernel": "k_event (Lucy iteration)", "kernel_ms_per_launch": kms,
            "algorithmic_bytes_per_launch": byts, "crossings_per_launch": cross,
            "crossings_per_s": cross / (kms * 1e-3)}


def disk_line(hrt, torch, local, stream, barrier, flush, steps, warmup, pda_min, l2):
    """The L2-resident flared disk (1e7 packets x 10 iterations + peel-off pass)."""
    wl = workload(10_000_000, 0, "disk")
    r = Runner(hrt, torch, wl, local, stream, "event", 10)
    ms, stats = r.timed_steps(steps, warmup, stream, barrier, flush)
    last = stats[-1]
    packets_step = wl.n_packets * 11
    lucy = last[:10]
    kms = statistics.mean(s["ms_propagate"] for s in lucy)
    byts = statistics.mean(B_CROSS * s["n_crossings"] + B_REEMIT * s["n_absorb"] for s in lucy)
    atoms = statistics.mean(s["n_crossings"] for s in lucy)       # at most one FP64 atomic per crossing
    achieved = byts / (kms * 1e-3) / 1e9
    out = {"workload": describe("disk", wl.n_packets, 10), "packets_per_s": packets_step * steps / (sum(ms) * 1e-3),
           "ms_per_step": statistics.mean(ms), "steps": steps,
           "roofline": {"bound": "l2", "achieved": achieved, "peak": l2["l2_copy_gbs"], "unit": "GB/s",
                        "frac": achieved / l2["l2_copy_gbs"], "peak_source": "measured in this run (L2 copy)",
                        "kernel": "k_event (Lucy iteration)", "kernel_ms_per_launch": kms,
                        "fp64_atomic_bound_per_s": atoms / (kms * 1e-3),
                        "fp64_atomic_frac": atoms / (kms * 1e-3) / l2["l2_fp64_atomics_per_s"]}}
    out.update(convergence_fields(stats, 10))
    if pda_min > 0:
        # time to the criterion with the partial diffusion approximation (App. A) for the cells
        # entered by fewer than pda_min packets (not part of the timed throughput steps)
        st = []
        r.solve(st, pda_min=pda_min, peel=False)
        q = [s["Q"] for s in st]
        it, t = converged_at(q, [s["ms_total"] for s in st], 1.02)
        out["pda"] = {"min_visits": pda_min, "cells": st[-1]["n_pda"], "q99_history": [round(x, 5) for x in q],
                      "iterations_to_converged": it, "time_to_converged_ms": t}
    r.close()
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.rows:
        return rows_bench(local)
    if args.learned:
        return learned_bench(args, local)
    if args.batch:
        return batch_bench(args, local)

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
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2
    wl = workload(args.packets, rank, args.workload)
    run = Runner(hrt, torch, wl, local, stream, args.kernel, args.iters)
    clocks = Clocks(local)
    clocks.start()
    step_ms, all_stats = run.timed_steps(args.steps, args.warmup, stream, barrier, flush)
    barrier()
    clk = clocks.stop()
    e2e_ms, h2d, d2h = run.e2e_steps(min(args.steps, 5), barrier, flush)
    barrier()
    launches = sum(s["kernel_launches"] for st in all_stats for s in st)
    run.close()

    packets_step = args.packets * (args.iters + 1)
    value, e2e_value, _, _ = job_throughput(sum(step_ms), statistics.mean(e2e_ms), world, packets_step, args.steps,
                                            dist, "cuda")
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, src = float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        peak, src = 6800.0, "fallback"
    last = all_stats[-1]
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": config(args, world)}
        line.update(convergence_fields(all_stats, args.iters))
        line.update({
            "lucy_ms_per_iteration": statistics.mean(s["ms_total"] for s in last[:args.iters]),
            "imaging_ms": last[-1]["ms_total"],
            "crossings_per_step": sum(s["n_crossings"] for s in last),
            "peel_crossings_per_step": sum(s["n_peel_crossings"] for s in last),
            "roofline": lucy_roofline(last, args.iters, peak, src),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clk,
        })
    if not args.no_extras and rank == 0:
        # the plain-GPU comparison: the same step with one thread per packet history
        if args.kernel == "event":
            pr = Runner(hrt, torch, wl, local, stream, "plain", args.iters)
            pms, _ = pr.timed_steps(1, 1, stream, barrier, flush)
            pr.close()
            line["plain_gpu"] = {"value": packets_step / (pms[0] * 1e-3), "unit": UNIT, "ms_per_step": pms[0],
                                 "kernel": "k_plain (one thread per history)", "steps": 1, "warmup": 1}
        if args.workload == "cloud":
            l2 = l2_peaks(torch)
            line["l2_peaks"] = l2
            line["flared_disk"] = disk_line(hrt, torch, local, stream, barrier, flush, 3, 2, args.pda_min, l2)
    if line is not None:
        if not args.no_cpu_baseline:
            r, cores, desc = cpu_oracle_rate(wl, args.iters, args.cpu_seconds)
            line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def learned_bench(args, local):
    """Learned warm start (task pattern 4) on the configs of the warm-start workload: 128^3 clouds
    with 1-8 stars (mean tau_550 = 10), a U-Net of widths 32, 64, 192 (2.19M parameters) trained by
    the library's tensor-core kernels on fields that the plain GPU iteration produced, then four
    held-out clouds solved to the Delta test (Q_99 < 2, Delta < 1.02; Eqs. 5-6) three ways with
    1e9 packets per iteration on the same random streams: the plain GPU iteration from 10 K one
    cloud after the other, the cold start batched in one persistent launch per iteration, and the
    warm start batched (inference included)."""
    import ctypes as C
    import torch
    from paper_1112_1071_gb300 import hrt, learned
    torch.cuda.set_device(local)
    L = hrt.load()
    t0 = time.time()
    X, Y, _ = learned.generate(range(1000, 1000 + args.learned_fields), 128, 30_000_000, 4, 10.0, torch)
    gen_s = time.time() - t0
    widths = (C.c_int * 3)(32, 64, 192)
    net = C.c_void_p()
    hrt.check(None, L.hrt_net_create_widths(C.byref(net), local, C.cast(widths, C.c_void_p), 2, 7, None))
    t1 = time.time()
    hist = learned.train(net, X, Y, args.learned_epochs, 1e-3, 4, torch)
    train_s = time.time() - t1
    del X, Y
    row = learned.evaluate_batch(net, range(5000, 5004), 128, 1_000_000_000, 8, 10.0, 2.0, 1.02, torch)
    line = {"metric": "time to converged temperatures, 4 held-out 128^3 clouds (warm start + batching)",
            "value": row["warm_batched_ms"], "unit": "ms", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": row["warm_batched_ms"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (network bf16 x bf16 -> f32)", "data": "synthetic",
            "config": {"workload": "warmstart_cloud 128^3, 1-8 stars, mean tau_550=10; 1e9 packets per iteration; "
                                   "criterion Q_99(dT) < 2 and Delta < 1.02", "training_fields": args.learned_fields,
                       "epochs": args.learned_epochs, "params": int(L.hrt_net_num_params(net))},
            "warm_vs_cold": row, "generation_s": gen_s, "training_s": train_s, "final_loss": hist[-1]}
    print(json.dumps(line), flush=True)
    L.hrt_net_destroy(net)
    return 0


def batch_bench(args, local):
    """Batched models (task pattern 2): the 512 disks of the batched workload (tau_550 1-1e4, uneven
    grids nr 50-400 x ntheta 32-200 x nphi 1-64, packet budgets log-uniform 1e5-1e7 per iteration)
    advance `iters` Lucy iterations in one persistent launch per iteration (captured CUDA graph),
    against the same models run one after the other (each iteration a launch of its own)."""
    import ctypes as C
    import numpy as np
    import torch
    from paper_1112_1071_gb300 import hrt
    from paper_1112_1071_gb300 import workloads as W
    torch.cuda.set_device(local)
    L = hrt.load()
    iters = 2
    wls = W.batched_disks(n_models=512, packet_scale=args.batch_scale)
    npk = np.array([wl.n_packets for wl in wls], np.int64)
    never = hrt.default_params(q_thres=1.0)        # never converged: every model runs every iteration
    # one by one
    ms_one = 0.0
    for wl in wls:
        m = hrt.Model(wl, device=local)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(iters):
            m.run_iteration(params=never)
        torch.cuda.synchronize()
        ms_one += 1e3 * (time.perf_counter() - t0)
        m.close()
    # batched
    models = [hrt.Model(wl, device=local) for wl in wls]
    arr = (C.c_void_p * len(models))(*[m.ctx.value for m in models])
    b = C.c_void_p()
    hrt.check(None, L.hrt_batch_create(C.byref(b), arr, len(models)))
    iters_run = C.c_int()
    hrt.check(None, L.hrt_batch_run(b, npk.ctypes.data, 1, C.byref(never), None, C.byref(iters_run)))   # capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hrt.check(None, L.hrt_batch_run(b, npk.ctypes.data, iters, C.byref(never), None, C.byref(iters_run)))
    torch.cuda.synchronize()
    ms_batch = 1e3 * (time.perf_counter() - t0)
    L.hrt_batch_destroy(b)
    for m in models:
        m.close()
    total = int(npk.sum()) * iters
    cells = int(sum(wl.rho.size for wl in wls))
    line = {"metric": "photon packets/sec, 512 batched disk models (one persistent launch per iteration)",
            "value": total / (ms_batch * 1e-3), "unit": "packets/s", "n_gpus": 1, "steps": iters, "warmup": 1,
            "ms_per_step": ms_batch / iters, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"batched_disks 512 models, {cells} cells, {int(npk.sum())} packets per iteration "
                                   f"(budgets log-uniform 1e5-1e7 x {args.batch_scale:g})", "iterations": iters},
            "one_by_one": {"value": total / (ms_one * 1e-3), "ms_per_step": ms_one / iters},
            "batched_over_one_by_one": ms_one / ms_batch}
    print(json.dumps(line), flush=True)
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
