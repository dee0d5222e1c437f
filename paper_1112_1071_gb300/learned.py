"""Learned warm start for the Lucy iteration: dataset, training and evaluation drivers.

Control flow only: temperature fields come from the library's Monte-Carlo iteration
(hrt_run_iteration), features and targets from hrt_net_features / hrt_net_temperature_target,
training steps from hrt_net_train_step (tensor-core forward and backward kernels, Adam), and
the warm start from hrt_net_warm_start.  torch holds the device tensors.

The experiment: clouds like the turbulent-cloud workload (log-normal density, 1-8 stars) are
solved by the plain iteration from T = 10 K; a network trained on those fields predicts the
temperature of unseen clouds, and the iteration started from that prediction is compared with
the cold start, with the same packets per iteration and the same random streams, on the
method's own convergence test (Sect. 2.4, Eqs. 4-6): iterations and device time (inference
included) until the 99th percentile of the iteration change in T is below 2 %, and until that
percentile stops changing (Delta < 1.02).  The Monte-Carlo iteration decides the result; the two
arms' final temperatures are compared against the Monte-Carlo noise of one iteration.

    python -m paper_1112_1071_gb300.learned --n 128 --train 2000 --test 4 --q-packets 8000000000
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import time

import numpy as np

from . import hrt
from . import workloads as W


def solve(m, packets, max_iter, q_thres=1.02, torch=None):
    """Lucy iterations; returns the per-iteration percentile Q (Eqs. 4-5), device ms and (with
    torch) each iteration's temperatures on the device."""
    L = hrt.load()
    qs, ms, Ts = [], [], []
    for _ in range(max_iter):
        st = m.run_iteration(n_packets=packets, q_thres=q_thres)
        qs.append(st["Q"])
        ms.append(st["ms_total"])
        if torch is not None:
            T = torch.empty(m.ncells, dtype=torch.float64, device="cuda")
            hrt.check(m.ctx, L.hrt_get_temperature_device(m.ctx, T.data_ptr(), T.numel()))
            Ts.append(T)
    return dict(q=qs, ms=ms, T=Ts)


def field(m, torch):
    """(features [n^3 x 2], target [n^3]) of a model as device tensors."""
    L = hrt.load()
    nc = m.ncells
    f = torch.empty(nc * 2, dtype=torch.float32, device="cuda")
    t = torch.empty(nc, dtype=torch.float32, device="cuda")
    hrt.check(m.ctx, L.hrt_net_features(m.ctx, f.data_ptr(), nc * 2))
    hrt.check(m.ctx, L.hrt_net_temperature_target(m.ctx, t.data_ptr(), nc))
    return f, t


def generate(seeds, n, packets, iters, tau, torch, log=None):
    X, Y, info = [], [], []
    for s in seeds:
        wl = W.warmstart_cloud(int(s), n=n, n_packets=packets, n_iter=iters, tau_mean_550=tau)
        m = hrt.Model(wl)
        r = solve(m, packets, iters)
        f, t = field(m, torch)
        X.append(f.view(n, n, n, 2))
        Y.append(t.view(n, n, n))
        info.append(dict(seed=int(s), ms=sum(r["ms"]), q_last=r["q"][-1]))
        m.close()
        if log:
            log(f"field {s}: {sum(r['ms']):.1f} ms, Q {r['q'][-1]:.4f}")
    return torch.stack(X), torch.stack(Y), info


def bench_conv(torch, log, reps=5):
    """Device time per launch of the 'same' 3x3x3 convolution through its three C-ABI hooks
    (tcgen05 fed by TMA, tcgen05 with per-phase cp.async loads, and the mma.sync baseline) on three shapes,
    by CUDA events around reps calls each (the hooks' BF16 conversions included)."""
    L = hrt.load()
    out = []
    for n, d, cin, cout in ((4, 64, 32, 32), (2, 64, 64, 64), (1, 32, 128, 128)):
        x = torch.randn((n, d, d, d, cin), device="cuda")
        w = torch.randn((3, 3, 3, cin, cout), device="cuda") * (27 * cin) ** -0.5
        b = torch.zeros(cout, device="cuda")
        y = torch.empty((n, d, d, d, cout), device="cuda")
        row = dict(shape=f"{n}x{d}^3 {cin}->{cout}", gflop=2 * 27 * cin * cout * n * d ** 3 / 1e9)
        for name, f in (("tcgen05_tma", L.hrt_nn_conv3d), ("tcgen05_phased", L.hrt_nn_conv3d_phased),
                        ("mma_sync", L.hrt_nn_conv3d_mma)):
            for _ in range(2):
                hrt.check(None, f(n, d, d, d, cin, cout, x.data_ptr(), w.data_ptr(), b.data_ptr(), 1, y.data_ptr(), None))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                hrt.check(None, f(n, d, d, d, cin, cout, x.data_ptr(), w.data_ptr(), b.data_ptr(), 1, y.data_ptr(), None))
            e1.record()
            torch.cuda.synchronize()
            row[name + "_ms"] = e0.elapsed_time(e1) / reps
        out.append(row)
        log(json.dumps(row))
    # one U-Net training step (forward, backward, Adam) at batch 2 x 128^3, the warm start's size
    widths = (32, 64, 192)
    wa = (C.c_int * 3)(*widths)
    net = C.c_void_p()
    hrt.check(None, L.hrt_net_create_widths(C.byref(net), 0, C.cast(wa, C.c_void_p), 2, 7, None))
    n, d = 2, 128
    x = torch.randn((n, d, d, d, 2), device="cuda")
    t = torch.randn((n, d, d, d), device="cuda")
    loss = C.c_double()
    for _ in range(2):
        hrt.check(None, L.hrt_net_train_step(net, n, d, d, d, x.data_ptr(), t.data_ptr(), 1e-4, C.byref(loss)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        hrt.check(None, L.hrt_net_train_step(net, n, d, d, d, x.data_ptr(), t.data_ptr(), 1e-4, C.byref(loss)))
    torch.cuda.synchronize()
    row = dict(shape=f"U-Net {widths} training step, batch {n} x {d}^3",
               ms=1e3 * (time.perf_counter() - t0) / reps)
    L.hrt_net_destroy(net)
    out.append(row)
    log(json.dumps(row))
    return out


def train(net, X, Y, epochs, lr, batch, torch, log=None):
    L = hrt.load()
    M, n = X.shape[0], X.shape[1]
    hist = []
    g = torch.Generator(device="cpu").manual_seed(0)
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(M, generator=g)
        tot = 0.0
        lr_ep = lr * (0.5 * (1 + np.cos(np.pi * ep / max(1, epochs))))    # cosine decay
        for b0 in range(0, M - batch + 1, batch):
            idx = perm[b0:b0 + batch].cuda()
            xb = X.index_select(0, idx).contiguous()
            yb = Y.index_select(0, idx).contiguous()
            loss = C.c_double()
            rc = L.hrt_net_train_step(net, batch, n, n, n, xb.data_ptr(), yb.data_ptr(), float(lr_ep), C.byref(loss))
            if rc != 0:
                raise hrt.HrtError(rc, "hrt_net_train_step")
            tot += loss.value
        hist.append(tot / max(1, M // batch))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.5f} ({time.time() - t0:.1f} s)")
    return hist


def converged_at(qs, q_thres=1.02, delta_thres=None):
    """First iteration (1-based) whose percentile meets the criterion: Q_99 < q_thres, and with
    delta_thres also Delta = max(Q_prev/Q, Q/Q_prev) < delta_thres (Eqs. 5-6; from the 2nd
    iteration on); None when no iteration does."""
    for i, q in enumerate(qs):
        if not q < q_thres:
            continue
        if delta_thres is None:
            return i + 1
        if i > 0 and max(qs[i - 1] / q, q / qs[i - 1]) < delta_thres:
            return i + 1
    return None


def evaluate(net, seeds, n, packets, max_iter, tau, torch, log=None):
    """Cold start (10 K) against warm start (the network's prediction, inference time included)
    on held-out clouds, same packets per iteration and same random streams: iterations and device
    time to the criterion Q_99(dT) < 1.02 and to the Delta test (Q_99 < 2, Delta < 1.02), and the
    agreement of the two arms' temperatures at the end against the cold arm's own last change."""
    L = hrt.load()
    rows = []
    for s in seeds:
        wl = W.warmstart_cloud(int(s), n=n, n_packets=packets, n_iter=max_iter, tau_mean_550=tau)
        cold = hrt.Model(wl)
        Tprev = torch.empty(cold.ncells, dtype=torch.float64, device="cuda")
        rc_ = solve(cold, packets, max_iter, torch=torch)
        warm = hrt.Model(wl)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hrt.check(warm.ctx, L.hrt_net_warm_start(net, warm.ctx))
        infer_ms = 1e3 * (time.perf_counter() - t0)
        rw_ = solve(warm, packets, max_iter, torch=torch)
        Tc = torch.empty_like(Tprev)
        Tw = torch.empty_like(Tprev)
        hrt.check(cold.ctx, L.hrt_get_temperature_device(cold.ctx, Tc.data_ptr(), Tc.numel()))
        hrt.check(warm.ctx, L.hrt_get_temperature_device(warm.ctx, Tw.data_ptr(), Tw.numel()))
        dust = torch.as_tensor(wl.rho.reshape(-1) > 0, device="cuda")
        agree = float(((Tw - Tc).abs() / Tc)[dust].mean())
        # the Monte-Carlo noise of one iteration: the cold arm's own change over one more iteration
        Tprev.copy_(Tc)
        cold.run_iteration(n_packets=packets)
        hrt.check(cold.ctx, L.hrt_get_temperature_device(cold.ctx, Tc.data_ptr(), Tc.numel()))
        noise = float(((Tc - Tprev).abs() / Tprev)[dust].mean())
        # distance of every iteration's field to the converged one (the cold arm's last), mean |dT|/T
        dist = {arm: [float(((T - Tprev).abs() / Tprev)[dust].mean()) for T in r["T"]] for arm, r in
                (("cold", rc_), ("warm", rw_))}
        for r in (rc_, rw_):
            r.pop("T")
        row = dict(seed=int(s), sources=len(wl.sources), inference_ms=infer_ms, cold=rc_, warm=rw_,
                   final_mean_dT_warm_vs_cold=agree, mc_noise_mean_dT=noise, dist_to_converged=dist)
        for name, r, extra in (("cold", rc_, 0.0), ("warm", rw_, infer_ms)):
            for crit, it in (("q", converged_at(r["q"], 1.02)), ("delta", converged_at(r["q"], 2.0, 1.02))):
                row[f"{name}_iters_to_{crit}"] = it
                row[f"{name}_ms_to_{crit}"] = (sum(r["ms"][:it]) + extra) if it else None
        rows.append(row)
        if log:
            log(f"cloud {s} ({len(wl.sources)} stars): Q cold {[round(q, 4) for q in rc_['q']]} "
                f"warm {[round(q, 4) for q in rw_['q']]}; to Q99 < 1.02: cold {row['cold_iters_to_q']} it "
                f"{row['cold_ms_to_q']} ms, warm {row['warm_iters_to_q']} it {row['warm_ms_to_q']} ms "
                f"(inference {infer_ms:.1f} ms); final dT warm vs cold {agree:.4f}, MC noise {noise:.4f}")
        cold.close()
        warm.close()
    return rows


def batch_solve(models, packets, max_iter, q_thres, delta_thres):
    """Lucy iterations of several models in one persistent launch per iteration (hrt_batch_run),
    each dropping out once its own convergence test passes; returns (wall ms of the run, per-model
    number of the iteration at which it converged or None)."""
    import torch
    L = hrt.load()
    arr = (C.c_void_p * len(models))(*[m.ctx.value for m in models])
    b = C.c_void_p()
    hrt.check(None, L.hrt_batch_create(C.byref(b), arr, len(models)))
    npk = np.full(len(models), packets, np.int64)
    p = hrt.default_params(q_thres=q_thres, delta_thres=delta_thres)
    stats = (hrt.hrt_iter_stats * len(models))()
    iters = C.c_int()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hrt.check(None, L.hrt_batch_run(b, npk.ctypes.data, max_iter, C.byref(p), stats, C.byref(iters)))
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0)
    L.hrt_batch_destroy(b)
    return ms, [stats[m].iteration + 1 if stats[m].converged else None for m in range(len(models))]


def evaluate_batch(net, seeds, n, packets, max_iter, tau, q_thres, delta_thres, torch, log=None):
    """Time to convergence of several held-out clouds (Sect. 2.4, Eqs. 4-6, with q_thres and
    delta_thres): the plain GPU iteration (cold start from 10 K, one model after the other),
    the cold start batched (one persistent launch per iteration for all clouds, converged clouds
    dropping out), and the warm start batched (the network's prediction for every cloud first,
    its inference time included).  Every arm runs the same packets on the same random streams."""
    L = hrt.load()
    wls = [W.warmstart_cloud(int(s), n=n, n_packets=packets, n_iter=max_iter, tau_mean_550=tau) for s in seeds]
    p = hrt.default_params(q_thres=q_thres, delta_thres=delta_thres)
    # plain: one model at a time, each until its own test passes
    plain_ms, plain_it = 0.0, []
    for wl in wls:
        m = hrt.Model(wl)
        it = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(max_iter):
            st = m.run_iteration(n_packets=packets, params=p)
            if st["converged"]:
                it = i + 1
                break
        torch.cuda.synchronize()
        plain_ms += 1e3 * (time.perf_counter() - t0)
        plain_it.append(it)
        m.close()
    cold = [hrt.Model(wl) for wl in wls]
    cold_ms, cold_it = batch_solve(cold, packets, max_iter, q_thres, delta_thres)
    warm = [hrt.Model(wl) for wl in wls]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m in warm:
        hrt.check(m.ctx, L.hrt_net_warm_start(net, m.ctx))
    torch.cuda.synchronize()
    infer_ms = 1e3 * (time.perf_counter() - t0)
    warm_ms, warm_it = batch_solve(warm, packets, max_iter, q_thres, delta_thres)
    dT = []
    for mc, mw, wl in zip(cold, warm, wls):
        Tc, Tw = mc.temperature(), mw.temperature()
        dust = wl.rho.reshape(-1) > 0
        dT.append(float(np.mean(np.abs(Tw[dust] - Tc[dust]) / Tc[dust])))
        mc.close()
        mw.close()
    row = dict(clouds=len(wls), packets=packets, q_thres=q_thres, delta_thres=delta_thres,
               plain_one_by_one_ms=plain_ms, plain_iterations=plain_it, cold_batched_ms=cold_ms,
               cold_iterations=cold_it, warm_batched_ms=warm_ms + infer_ms, warm_inference_ms=infer_ms,
               warm_iterations=warm_it, final_mean_dT_warm_vs_cold=dT,
               speedup_vs_plain=plain_ms / (warm_ms + infer_ms), speedup_vs_cold_batched=cold_ms / (warm_ms + infer_ms))
    if log:
        log(json.dumps(row))
    return row


def _mean(xs):
    xs = [x for x in xs if x is not None]
    return float(np.mean(xs)) if xs else None


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--tau", type=float, default=10.0, help="mean 550 nm optical depth across the cloud")
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=4)
    ap.add_argument("--q-test", type=int, default=2, help="held-out clouds judged by Q_99(dT) < 1.02")
    ap.add_argument("--packets", type=int, default=30_000_000, help="packets per iteration of a training field")
    ap.add_argument("--iters", type=int, default=4, help="iterations of a training field")
    ap.add_argument("--eval-packets", type=int, default=1_000_000_000,
                    help="packets per iteration of the held-out runs judged by the Delta test")
    ap.add_argument("--q-packets", type=int, default=0,
                    help="packets per iteration of held-out runs judged by Q_99(dT) < 1.02 (0: skip); the "
                         "Monte-Carlo noise floor of Q_99 must lie below 1.02 there")
    ap.add_argument("--eval-iters", type=int, default=6)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--widths", default="32,64,192",
                    help="channels per level, encoder to bottleneck (levels = count - 1); 32,64,192: 2.19M parameters")
    ap.add_argument("--out", default=None)
    ap.add_argument("--bench-conv", action="store_true",
                    help="only time the 3x3x3 convolution (tcgen05 and mma.sync hooks) on three shapes")
    a = ap.parse_args()
    if not 0 <= a.q_packets < 2 ** 32 or not 0 < a.eval_packets < 2 ** 32:
        ap.error("packets per iteration must be below 2^32 (the packet id is one 32-bit word of the Philox counter)")
    log = lambda s: print(s, flush=True)
    L = hrt.load()
    if a.bench_conv:
        bench_conv(torch, log)
        return
    t0 = time.time()
    X, Y, info = generate(range(1000, 1000 + a.train), a.n, a.packets, a.iters, a.tau, torch, log)
    gen_s = time.time() - t0
    widths = [int(w) for w in a.widths.split(",")]
    net = C.c_void_p()
    wa = (C.c_int * len(widths))(*widths)
    hrt.check(None, L.hrt_net_create_widths(C.byref(net), 0, C.cast(wa, C.c_void_p), len(widths) - 1, 7, None))
    t1 = time.time()
    hist = train(net, X, Y, a.epochs, a.lr, a.batch, torch, log)
    train_s = time.time() - t1
    held = range(5000, 5000 + a.test)
    rows = evaluate(net, held, a.n, a.eval_packets, a.eval_iters, a.tau, torch, log)
    batched = [evaluate_batch(net, held, a.n, a.eval_packets, a.eval_iters, a.tau, 2.0, 1.02, torch, log)]
    if a.q_packets > 0:
        batched.append(evaluate_batch(net, held[:a.q_test], a.n, a.q_packets, a.eval_iters, a.tau, 1.02, float("inf"),
                                      torch, log))
    summary = dict(
        grid=a.n, tau_mean_550=a.tau, train_fields=a.train, test_fields=a.test, packets=a.packets,
        iters=a.iters, eval_packets=a.eval_packets, widths=widths, params=int(L.hrt_net_num_params(net)),
        generation_s=gen_s, training_s=train_s, epochs=a.epochs, final_loss=hist[-1],
        inference_ms_mean=_mean([r["inference_ms"] for r in rows]),
        final_mean_dT_warm_vs_cold=_mean([r["final_mean_dT_warm_vs_cold"] for r in rows]),
        mc_noise_mean_dT=_mean([r["mc_noise_mean_dT"] for r in rows]), batched=batched, loss_history=hist, rows=rows,
        fields=info)
    for arm in ("cold", "warm"):
        for crit in ("q", "delta"):
            summary[f"{arm}_iters_to_{crit}_mean"] = _mean([r[f"{arm}_iters_to_{crit}"] for r in rows])
            summary[f"{arm}_ms_to_{crit}_mean"] = _mean([r[f"{arm}_ms_to_{crit}"] for r in rows])
            summary[f"{arm}_reached_{crit}"] = sum(1 for r in rows if r[f"{arm}_iters_to_{crit}"])
    print(json.dumps({k: v for k, v in summary.items() if k not in ("rows", "fields", "loss_history")}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(summary, f, indent=1)
    L.hrt_net_destroy(net)


if __name__ == "__main__":
    main()
