"""Multi-process paths on CPU ranks (gloo, world size 2, 127.0.0.1).

* Packet sharding (Sect. 3): the packets of one iteration are independent, so ranks that run
  disjoint packet-id ranges (each id on its own Philox stream, eps = L / n_total) and add their
  accumulators, SED bins and escape tallies with one all-reduce reproduce the single-process
  iteration.  Checked with the FP64 oracle on two ranks.
* The benchmark's reduction: whole-job throughput from the slowest rank's time, and one
  independent model per rank (weak scaling, no collective on the data path)."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    return dist


def _shard_worker(rank, world, port, n_total, out_dir):
    import torch
    from oracle import mc as M
    from paper_1112_1071_gb300 import workloads as W
    dist = _init(rank, world, port)
    wl = W.tiny_sphere(n_packets=n_total)
    om = M.OracleModel(wl)
    per = n_total // world
    first = rank * per
    n = per if rank < world - 1 else n_total - first
    r = om.run_packets(n, 0, first_packet=first, n_total=n_total, peel=True)
    vec = torch.from_numpy(np.concatenate([r["acc"], r["sed"].ravel(), r["esc"].ravel(),
                                           [r["e_escaped"], r["e_killed"], r["n_crossings"],
                                            r["n_interactions"]]]))
    dist.all_reduce(vec, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(os.path.join(out_dir, "sharded.npy"), vec.numpy())
    dist.destroy_process_group()


def _reduce_worker(rank, world, port, out_dir):
    import bench
    dist = _init(rank, world, port)
    # rank r is slower by (r + 1): the job's time is the slowest rank's
    res = bench.job_throughput(100.0 * (rank + 1), 50.0 * (rank + 1), world, 1000, 2, dist)
    wl = bench.workload(1000, rank)
    np.save(os.path.join(out_dir, f"reduce{rank}.npy"),
            np.array(list(res) + [wl.seed, wl.rho.size, wl.n_packets], dtype=np.float64))
    dist.destroy_process_group()


def _spawn(fn, *args):
    import torch.multiprocessing as mp
    mp.start_processes(fn, args=args, nprocs=2, join=True, start_method="spawn")


def test_packet_shards_reproduce_one_iteration(tmp_path):
    from oracle import mc as M
    from paper_1112_1071_gb300 import workloads as W
    n_total = 6000
    _spawn(_shard_worker, 2, _free_port(), n_total, str(tmp_path))
    vec = np.load(tmp_path / "sharded.npy")
    wl = W.tiny_sphere(n_packets=n_total)
    om = M.OracleModel(wl)
    r = om.run_packets(n_total, 0, peel=True)
    want = np.concatenate([r["acc"], r["sed"].ravel(), r["esc"].ravel(),
                           [r["e_escaped"], r["e_killed"], r["n_crossings"], r["n_interactions"]]])
    # same histories; only the order of the FP64 additions differs
    np.testing.assert_allclose(vec, want, rtol=1e-12, atol=1e-300)
    assert vec[-2:].tolist() == want[-2:].tolist()


def test_benchmark_reduction_over_ranks(tmp_path):
    pytest.importorskip("torch")
    _spawn(_reduce_worker, 2, _free_port(), str(tmp_path))
    r0, r1 = np.load(tmp_path / "reduce0.npy"), np.load(tmp_path / "reduce1.npy")
    # both ranks see the max: 200 ms for 2 ranks x 2 steps x 1000 packets; e2e 100 ms per step
    for r in (r0, r1):
        assert r[0] == pytest.approx(2 * 2 * 1000 / 0.2)
        assert r[1] == pytest.approx(2 * 1000 / 0.1)
        assert r[2] == 200.0 and r[3] == 100.0
    # one independent model per rank: same size, own random streams
    assert r0[4] != r1[4] and r0[5] == r1[5] and r0[6] == r1[6]
