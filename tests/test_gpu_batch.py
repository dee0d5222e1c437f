"""Batched persistent launch (hrt_batch_*): many uneven disk models advance one Lucy iteration
per graph launch.  Every model draws from the same Philox streams as when it runs alone, so
each batched model must reproduce its individually run twin (lockstep level), conserve energy
exactly, and drop out of later launches once its convergence test passes."""
import ctypes as C

import numpy as np
import pytest

from paper_1112_1071_gb300 import hrt
from paper_1112_1071_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(models):
    L = hrt.load()
    arr = (C.c_void_p * len(models))(*[m.ctx.value for m in models])
    b = C.c_void_p()
    assert L.hrt_batch_create(C.byref(b), arr, len(models)) == 0
    return b


def test_batched_models_match_individual_runs():
    L = hrt.load()
    wls = W.batched_disks(n_models=6, size_scale=0.2, packet_scale=0.01, seed=31)
    batched = [hrt.Model(wl) for wl in wls]
    alone = [hrt.Model(wl) for wl in wls]
    npk = np.array([wl.n_packets for wl in wls], np.int64)
    b = _batch(batched)
    p = hrt.default_params(q_thres=1.0)          # never converges: run all iterations
    stats = (hrt.hrt_iter_stats * len(wls))()
    iters = C.c_int()
    assert L.hrt_batch_run(b, npk.ctypes.data, 3, C.byref(p), stats, C.byref(iters)) == 0
    assert iters.value == 3
    for m, (mb, ma) in enumerate(zip(batched, alone)):
        for _ in range(3):
            sa = ma.run_iteration(n_packets=int(npk[m]), q_thres=1.0)
        sb = stats[m]
        assert sb.iteration == 2 and sa["iteration"] == 2
        assert sb.e_escaped + sb.e_killed == pytest.approx(sb.e_emitted, rel=1e-12)
        assert sb.n_crossings == pytest.approx(sa["n_crossings"], rel=2e-3)
        Tb, Ta = mb.temperature(), ma.temperature()
        dust = wls[m].rho.reshape(-1) > 0
        dT = np.abs(Tb[dust] - Ta[dust]) / Ta[dust]
        assert np.median(dT) < 1e-4 and dT.mean() < 0.01, m
        assert sb.Q == pytest.approx(sa["Q"], rel=0.05)
    L.hrt_batch_destroy(b)


def test_batched_models_match_the_oracle_in_lockstep():
    """A mixed batch (two uneven spherical-polar disks and the Cartesian tiny sphere) in one
    persistent launch against the FP64 oracle on each model's own Philox streams: energy
    conservation to FP64 rounding, and per-cell deposits and temperatures in lockstep over two
    Lucy iterations (Sect. 2.3, Eq. 2-3; the second re-emits from the first's temperatures)."""
    from oracle import mc as M
    L = hrt.load()
    wls = W.batched_disks(n_models=2, size_scale=0.15, packet_scale=0.005, seed=34)
    wls.append(W.tiny_sphere(n_packets=20_000))
    models = [hrt.Model(wl) for wl in wls]
    oms = [M.OracleModel(wl) for wl in wls]
    npk = np.array([wl.n_packets for wl in wls], np.int64)
    b = _batch(models)
    p = hrt.default_params(q_thres=1.0)
    stats = (hrt.hrt_iter_stats * len(wls))()
    iters = C.c_int()
    for it in range(2):
        assert L.hrt_batch_run(b, npk.ctypes.data, 1, C.byref(p), stats, C.byref(iters)) == 0
        assert iters.value == 1
        for m, (mb, om) in enumerate(zip(models, oms)):
            ref = om.run_iteration(n_packets=int(npk[m]), nthreads=8)
            sb = stats[m]
            assert sb.iteration == it
            assert sb.e_escaped + sb.e_killed == pytest.approx(om.L_tot, rel=1e-12)
            assert sb.n_crossings == pytest.approx(ref["n_crossings"], rel=2e-3)
            acc, racc = mb.absorbed(), ref["acc"]
            seen = racc > 0
            rel = np.abs(acc[seen] - racc[seen]) / racc[seen]
            assert np.median(rel) < 1e-4, (m, it, np.median(rel))
            assert abs(acc.sum() - racc.sum()) <= 2e-3 * racc.sum(), (m, it)
            T, rT = mb.temperature(), ref["T"]
            dust = om.rho > 0
            dT = np.abs(T[dust] - rT[dust]) / rT[dust]
            assert np.median(dT) < 1e-4 and dT.mean() < 0.01, (m, it, np.median(dT), dT.mean())
    L.hrt_batch_destroy(b)


def test_converged_models_drop_out():
    L = hrt.load()
    wls = W.batched_disks(n_models=5, size_scale=0.2, packet_scale=0.005, seed=32)
    ms = [hrt.Model(wl) for wl in wls]
    npk = np.array([wl.n_packets for wl in wls], np.int64)
    b = _batch(ms)
    p = hrt.default_params(q_thres=1e30)        # passes as soon as Q is finite
    stats = (hrt.hrt_iter_stats * len(wls))()
    iters = C.c_int()
    assert L.hrt_batch_run(b, npk.ctypes.data, 5, C.byref(p), stats, C.byref(iters)) == 0
    assert iters.value == 1
    assert all(stats[m].converged == 1 and stats[m].iteration == 0 for m in range(len(wls)))
    L.hrt_batch_destroy(b)


def test_batch_tune_picks_a_shape_and_caches_it():
    L = hrt.load()
    wls = W.batched_disks(n_models=4, size_scale=0.15, packet_scale=0.005, seed=33)
    ms = [hrt.Model(wl) for wl in wls]
    npk = np.array([wl.n_packets for wl in wls], np.int64)
    b = _batch(ms)
    assert L.hrt_batch_tune(b, npk.ctypes.data) == 0
    assert L.hrt_batch_tune(b, npk.ctypes.data) == 0      # cached
    stats = (hrt.hrt_iter_stats * len(wls))()
    iters = C.c_int()
    assert L.hrt_batch_run(b, npk.ctypes.data, 2, None, stats, C.byref(iters)) == 0
    assert iters.value >= 1
    L.hrt_batch_destroy(b)


@pytest.mark.parametrize("field,value", [("mrw_gamma", 2.0), ("pda_min_visits", 100), ("raytrace_rays", 1000),
                                         ("peel", 1), ("update_temperature", 0)])
def test_batch_rejects_settings_of_single_model_calls(field, value):
    # a batch runs Lucy iterations; the extensions and imaging passes are single-model calls
    L = hrt.load()
    wls = W.batched_disks(n_models=2, size_scale=0.1, packet_scale=0.001, seed=7)
    models = [hrt.Model(wl) for wl in wls]
    b = _batch(models)
    npk = np.array([wl.n_packets for wl in wls], np.int64)
    p = hrt.default_params(**{field: value})
    assert L.hrt_batch_run(b, npk.ctypes.data, 1, C.byref(p), None, None) == hrt.HRT_EINVAL
    assert L.hrt_batch_run(b, npk.ctypes.data, 1, None, None, None) == 0
    L.hrt_batch_destroy(b)
