"""Learned warm start for the Lucy iteration: dataset, training and evaluation drivers.

Control flow only: temperature fields come from the library's Monte-Carlo iteration
(hrt_run_iteration), features and targets from hrt_net_features / hrt_net_temperature_target,
training steps from hrt_net_train_step (tensor-core forward and backward kernels, Adam), and
the warm start from hrt_net_warm_start.  torch holds the device tensors.

The experiment: clouds like the turbulent-cloud workload (log-normal density, 1-8 stars) are
solved to convergence by the plain iteration from T = 10 K; a network trained on those fields
predicts the converged temperature of unseen clouds, and the iteration restarted from that
prediction is timed to the same criterion (99th percentile of the iteration change in T below
2 %).  The Monte-Carlo iteration and its convergence test stay the judge.

    python -m paper_1112_1071_gb300.learned --n 64 --train 256 --test 16
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import time

import numpy as np

from . import hrt
from . import workloads as W


def solve(m, packets, max_iter, q_thres=1.02):
    """Lucy iterations until Q_99(delta T) < q_thres; returns (iterations, device ms, Q history)."""
    qs, ms = [], 0.0
    for it in range(max_iter):
        st = m.run_iteration(n_packets=packets, q_thres=q_thres)
        qs.append(st["Q"])
        ms += st["ms_total"]
        if st["converged"]:
            return it + 1, ms, qs
    return None, ms, qs


def field(m, torch):
    """(features [n^3 x 2], target [n^3]) of a model as device tensors."""
    L = hrt.load()
    nc = m.ncells
    f = torch.empty(nc * 2, dtype=torch.float32, device="cuda")
    t = torch.empty(nc, dtype=torch.float32, device="cuda")
    hrt.check(m.ctx, L.hrt_net_features(m.ctx, f.data_ptr(), nc * 2))
    hrt.check(m.ctx, L.hrt_net_temperature_target(m.ctx, t.data_ptr(), nc))
    return f, t


def generate(seeds, n, packets, iters, torch, log=None):
    X, Y, info = [], [], []
    for s in seeds:
        wl = W.warmstart_cloud(int(s), n=n, n_packets=packets, n_iter=iters)
        m = hrt.Model(wl)
        its, ms, qs = solve(m, packets, iters)
        f, t = field(m, torch)
        X.append(f.view(n, n, n, 2))
        Y.append(t.view(n, n, n))
        info.append(dict(seed=int(s), iterations=its, ms=ms, q_last=qs[-1]))
        m.close()
        if log:
            log(f"field {s}: {its} iterations, {ms:.1f} ms, Q {qs[-1]:.4f}")
    return torch.stack(X), torch.stack(Y), info


def train(net, X, Y, epochs, lr, batch, torch, log=None):
    L = hrt.load()
    M, n = X.shape[0], X.shape[1]
    hist = []
    g = torch.Generator(device="cpu").manual_seed(0)
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(M, generator=g)
        tot = 0.0
        for b0 in range(0, M - batch + 1, batch):
            idx = perm[b0:b0 + batch].cuda()
            xb = X.index_select(0, idx).contiguous()
            yb = Y.index_select(0, idx).contiguous()
            loss = C.c_double()
            rc = L.hrt_net_train_step(net, batch, n, n, n, xb.data_ptr(), yb.data_ptr(), lr, C.byref(loss))
            if rc != 0:
                raise hrt.HrtError(rc, "hrt_net_train_step")
            tot += loss.value
        hist.append(tot / max(1, M // batch))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.5f} ({time.time() - t0:.1f} s)")
    return hist


def evaluate(net, seeds, n, packets, max_iter, torch, log=None):
    L = hrt.load()
    rows = []
    for s in seeds:
        wl = W.warmstart_cloud(int(s), n=n, n_packets=packets, n_iter=max_iter)
        cold = hrt.Model(wl)
        ic, mc, qc = solve(cold, packets, max_iter)
        warm = hrt.Model(wl)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hrt.check(warm.ctx, L.hrt_net_warm_start(net, warm.ctx))
        infer_ms = 1e3 * (time.perf_counter() - t0)
        iw, mw, qw = solve(warm, packets, max_iter)
        Tc, Tw = cold.temperature(), warm.temperature()
        rows.append(dict(seed=int(s), cold_iterations=ic, cold_ms=mc, warm_iterations=iw, warm_ms=mw + infer_ms,
                         inference_ms=infer_ms, q_cold=qc, q_warm=qw,
                         mean_abs_dT_over_T=float(np.mean(np.abs(Tw - Tc) / Tc))))
        if log:
            log(f"cloud {s}: cold {ic} it {mc:.1f} ms | warm {iw} it {mw + infer_ms:.1f} ms")
        cold.close()
        warm.close()
    return rows


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--train", type=int, default=256)
    ap.add_argument("--test", type=int, default=16)
    ap.add_argument("--packets", type=int, default=8_000_000, help="packets per iteration of a training field")
    ap.add_argument("--iters", type=int, default=8, help="iterations of a training field")
    ap.add_argument("--eval-packets", type=int, default=300_000_000,
                    help="packets per iteration when timing convergence (noise floor below 2 %%)")
    ap.add_argument("--eval-iters", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--base", type=int, default=32)
    ap.add_argument("--levels", type=int, default=2)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    log = lambda s: print(s, flush=True)
    L = hrt.load()
    t0 = time.time()
    X, Y, info = generate(range(1000, 1000 + a.train), a.n, a.packets, a.iters, torch, log)
    gen_s = time.time() - t0
    net = C.c_void_p()
    hrt.check(None, L.hrt_net_create(C.byref(net), 0, a.base, a.levels, 7, None))
    t1 = time.time()
    hist = train(net, X, Y, a.epochs, a.lr, a.batch, torch, log)
    train_s = time.time() - t1
    rows = evaluate(net, range(5000, 5000 + a.test), a.n, a.eval_packets, a.eval_iters, torch, log)
    ok = [r for r in rows if r["cold_iterations"] and r["warm_iterations"]]
    summary = dict(
        grid=a.n, train_fields=a.train, test_fields=a.test, packets=a.packets, eval_packets=a.eval_packets,
        params=int(L.hrt_net_num_params(net)),
        generation_s=gen_s, training_s=train_s, final_loss=hist[-1], loss_history=hist,
        converged_pairs=len(ok),
        cold_iterations_mean=float(np.mean([r["cold_iterations"] for r in ok])) if ok else None,
        warm_iterations_mean=float(np.mean([r["warm_iterations"] for r in ok])) if ok else None,
        cold_ms_mean=float(np.mean([r["cold_ms"] for r in ok])) if ok else None,
        warm_ms_mean=float(np.mean([r["warm_ms"] for r in ok])) if ok else None,
        mean_abs_dT_over_T=float(np.mean([r["mean_abs_dT_over_T"] for r in rows])),
        rows=rows, fields=info)
    print(json.dumps({k: v for k, v in summary.items() if k not in ("rows", "fields", "loss_history")}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(summary, f, indent=1)
    L.hrt_net_destroy(net)


if __name__ == "__main__":
    main()
