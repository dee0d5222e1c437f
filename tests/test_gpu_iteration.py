"""Whole-iteration parity of the CUDA path with the FP64 oracle (through the C ABI).

Both implementations draw packet p of iteration i from the same Philox4x32-10 stream, so
their histories agree draw for draw until single-precision geometry moves an interaction
across a wall; per-cell deposits then agree far inside the Monte-Carlo noise.  The tests
hold the GPU to: exact energy conservation; per-cell absorbed energy and temperatures within
1% mean |dT|/T and within 3 sigma of a bootstrap over packet chunks (the aggregate tolerance
of the method); the lockstep agreement itself (most cells within 1e-4); an exact nearest-rank
quantile; peel-off SEDs within 3 sigma; and the closed-form first-flight slab."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import mc as M
from oracle import tables as T
from paper_1112_1071_gb300 import hrt
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import pixel_parity

pytestmark = pytest.mark.gpu

KERNELS = [hrt.HRT_KERNEL_PLAIN, hrt.HRT_KERNEL_EVENT, hrt.HRT_KERNEL_REGROUP]


def _bootstrap_sigma(om, n, nchunk=20, key=0, **kw):
    """Per-cell sigma of the oracle's mean absorbed energy from packet chunks."""
    per = n // nchunk
    parts = np.array([om.run_packets(per, key, first_packet=k * per, n_total=n, **kw)["acc"] for k in range(nchunk)])
    return parts.sum(axis=0), parts.std(axis=0, ddof=1) * math.sqrt(nchunk)


@pytest.mark.parametrize("kernel", KERNELS)
def test_tiny_sphere_iterations_match_oracle(kernel):
    wl = W.tiny_sphere(n_packets=100_000, n_iter=3)
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    for it in range(3):
        st = m.run_iteration(kernel=kernel)
        ref = om.run_iteration(nthreads=8)
        assert st["e_escaped"] + st["e_killed"] + st["e_absorbed"] == pytest.approx(om.L_tot, rel=1e-12)
        assert st["n_packets"] == wl.n_packets
        acc = m.absorbed()
        dust = om.rho > 0
        rel = np.abs(acc - ref["acc"]) / np.maximum(ref["acc"], 1e-300)
        # lockstep: most cells agree far below the Monte-Carlo noise
        assert np.median(rel[dust]) < 1e-4, it
        Tg = m.temperature()
        well = dust & (ref["acc"] > 0)
        dT = np.abs(Tg[well] - ref["T"][well]) / ref["T"][well]
        assert dT.mean() < 0.01 and np.median(dT) < 1e-4, it
        assert st["clamp_low"] == ref["clamp_low"] and st["clamp_high"] == ref["clamp_high"]
        # exact nearest-rank quantile of the GPU's own temperature change
        if it > 0:
            Q = T.percentile_nearest_rank(T.delta(prev_T[dust], Tg[dust]), 0.99)
            assert st["Q"] == Q
            assert st["Q"] == pytest.approx(ref["Q"], rel=0.05)
        prev_T = Tg.copy()


@pytest.mark.parametrize("kernel", KERNELS)
def test_tiny_sphere_within_bootstrap_noise(kernel):
    wl = W.tiny_sphere(n_packets=100_000)
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    m.run_iteration(kernel=kernel)
    acc, sig = _bootstrap_sigma(om, wl.n_packets)
    g = m.absorbed()
    well = (om.rho > 0) & (sig > 0)
    z = np.abs(g[well] - acc[well]) / (math.sqrt(2) * sig[well])
    assert (z > 3).mean() < 0.01
    assert abs(np.mean((g[well] - acc[well]) / acc[well])) < 3 * np.std((g[well] - acc[well]) / acc[well]) / math.sqrt(well.sum()) + 1e-4


@pytest.mark.parametrize("kernel", KERNELS)
def test_flared_disk_iteration_matches_oracle(kernel):
    wl = W.flared_disk(n_packets=200_000, n_r=100, n_theta=64)
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    for it in range(2):
        st = m.run_iteration(kernel=kernel)
        ref = om.run_iteration(nthreads=8)
        assert st["e_escaped"] + st["e_killed"] == pytest.approx(om.L_tot, rel=1e-12)
        acc = m.absorbed()
        seen = ref["acc"] > 0
        rel = np.abs(acc[seen] - ref["acc"][seen]) / ref["acc"][seen]
        assert np.median(rel) < 1e-4
        # crossings agree to the rare histories that diverge
        assert st["n_crossings"] == pytest.approx(ref["n_crossings"], rel=2e-3)
        Tg = m.temperature()
        well = (om.rho > 0) & seen
        dT = np.abs(Tg[well] - ref["T"][well]) / ref["T"][well]
        assert dT.mean() < 0.01


@pytest.mark.parametrize("kernel", KERNELS)
def test_peeloff_sed_and_image_match_oracle(kernel):
    wl = W.tiny_sphere(n_packets=20000)
    wl.img_nx = wl.img_ny = 32
    wl.img_half_extent = 100 * W.AU
    wl.img_lam_um = np.array([1.0, 10.0, 100.0])
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    m.run_iteration(kernel=kernel)
    om.run_iteration(nthreads=8)
    st = m.run_iteration(kernel=kernel, peel=1, update_temperature=0)
    ref = om.run_iteration(peel=True, update=False, nthreads=8)
    sed = m.sed()
    tot_g, tot_o = sed.sum(axis=1), ref["sed"].sum(axis=1)
    np.testing.assert_allclose(tot_g, tot_o, rtol=1e-3)
    big = ref["sed"] > 1e-3 * ref["sed"].max()
    np.testing.assert_allclose(sed[big], ref["sed"][big], rtol=2e-2)
    img = m.image()
    np.testing.assert_allclose(img.sum(axis=(2, 3)), ref["img"].sum(axis=(2, 3)), rtol=2e-2)
    # imaging pass leaves the Lucy state alone
    assert st["Q"] == math.inf


@pytest.mark.parametrize("kernel", KERNELS)
def test_image_pixels_match_oracle_in_lockstep(kernel):
    """Peel-off images with dust (Sect. 2.6.2), pixel by pixel: the same packets on the same
    random streams put their weights into the same pixels at three inclined observers and three
    wavelengths.  Differences come from FP32 against FP64 arithmetic (weights ~1e-7, positions
    at pixel edges) and from the few histories that part over many steps."""
    wl = W.tiny_sphere(n_packets=20000)
    wl.img_nx = wl.img_ny = 32
    wl.img_half_extent = 100 * W.AU
    wl.img_lam_um = np.array([1.0, 10.0, 100.0])
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    m.run_iteration(kernel=kernel)
    om.run_iteration(nthreads=8)
    m.run_iteration(kernel=kernel, peel=1, update_temperature=0)
    ref = om.run_iteration(peel=True, update=False, nthreads=8)
    stats = pixel_parity(m.image(), ref["img"])
    print("image pixels", kernel, stats)
    assert stats["lit"] > 500
    assert stats["median_rel"] < 1e-6
    assert stats["frac_off"] < 0.01
    assert stats["l1_rel"] < 1e-4


@pytest.mark.parametrize("kernel", KERNELS)
def test_peeloff_pass_on_a_fresh_context(kernel):
    # the re-emission rows come from the starting temperatures even before any Lucy iteration
    wl = W.tiny_sphere(n_packets=20000)
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    m.run_iteration(kernel=kernel, peel=1, update_temperature=0)
    ref = om.run_iteration(peel=True, update=False, nthreads=8)
    np.testing.assert_allclose(m.sed().sum(axis=1), ref["sed"].sum(axis=1), rtol=1e-3)


@pytest.mark.parametrize("kernel", KERNELS)
def test_grey_slab_first_flight_closed_form(kernel):
    tau = 1.0
    wl = W.slab(n_layers=8, tau_total=tau, albedo=0.0, n_packets=200_000)
    m = hrt.Model(wl)
    st = m.run_iteration(kernel=kernel, peel=1, terminate_on_absorb=1)
    t = wl.walls[2][-1]
    z0 = wl.sources[0]["pos"][2]
    f_abs = 0.5 * (1 - special.expn(2, tau * (t - z0) / t)) + 0.5 * (1 - special.expn(2, tau * z0 / t))
    sig = math.sqrt(f_abs * (1 - f_abs) / wl.n_packets)
    L = W.LSUN
    assert st["e_absorbed"] / L == pytest.approx(f_abs, abs=4 * sig)
    rho = float(wl.rho.reshape(-1)[0])
    tau_up = rho * 1.0 * (t - z0)
    sed = m.sed()
    for o, inc in enumerate(wl.obs_incl):
        # deterministic: eps/(4 pi) exp(-tau/mu) from every packet (FP32 optical depth)
        assert sed[o].sum() == pytest.approx(L / (4 * math.pi) * math.exp(-tau_up / math.cos(inc)), rel=1e-5)


def test_escape_binning_holds_all_escaping_energy():
    wl = W.tiny_sphere(n_packets=50_000)
    m = hrt.Model(wl)
    st = m.run_iteration()
    esc = m.escape()
    assert esc.sum() == pytest.approx(st["e_escaped"], rel=1e-12)


def test_watchdog_returns_timeout_and_context_survives():
    wl = W.flared_disk(n_packets=2_000_000, n_r=100, n_theta=64)
    m = hrt.Model(wl)
    p = hrt.default_params(watchdog_ms=0.05)
    with pytest.raises(hrt.HrtError) as e:
        m.run_iteration(params=p)
    assert e.value.code == hrt.HRT_ETIMEDOUT
    st = m.run_iteration(n_packets=10_000)
    assert st["e_escaped"] + st["e_killed"] == pytest.approx(st["e_emitted"], rel=1e-12)


def test_input_validation_errors():
    wl = W.tiny_sphere()
    m = hrt.Model(wl)
    L = hrt.load()
    bad = np.full(m.ncells, np.nan, np.float32)
    assert L.hrt_set_density(m.ctx, bad.ctypes.data, bad.size) == hrt.HRT_EINVAL
    short = np.ones(5, np.float32)
    assert L.hrt_set_density(m.ctx, short.ctypes.data, 5) == hrt.HRT_EINVAL
    w = np.array([0.0, 1.0, 0.5])
    assert L.hrt_set_grid_cartesian(m.ctx, 2, 2, 2, w.ctypes.data, w.ctypes.data, w.ctypes.data) == hrt.HRT_EINVAL
    x = np.array([1e20, 0, 0])
    assert L.hrt_add_point_source(m.ctx, x.ctypes.data, 1.0, 5000.0) == hrt.HRT_EINVAL
    assert "outside" in L.hrt_last_error(m.ctx).decode()
    out = np.empty(3)
    assert L.hrt_get_temperature(m.ctx, out.ctypes.data, 3) == hrt.HRT_EINVAL
    # packet shares beyond the iteration's packet range
    for kw in (dict(first_packet=900, n_total=1000), dict(first_packet=-1), dict(n_total=2**32 + 1)):
        with pytest.raises(hrt.HrtError):
            m.run_iteration(n_packets=200, **kw)
    # the context still runs after rejected calls
    st = m.run_iteration(n_packets=1000)
    assert st["n_packets"] == 1000


@pytest.mark.parametrize("name", ["tiny_sphere", "flared_disk"])
def test_event_kernel_reproduces_plain_histories(name):
    # packet p always draws from the same Philox stream, whichever lane runs it, so every
    # launch shape of the event kernel walks the same FP32 histories as the plain kernel;
    # only the order of the FP64 additions differs
    wl = W.WORKLOADS[name](n_packets=60_000)
    if name == "flared_disk":
        wl = W.flared_disk(n_packets=60_000, n_r=80, n_theta=48)
    ref = hrt.Model(wl)
    sp = ref.run_iteration(kernel=hrt.HRT_KERNEL_PLAIN)
    acc0 = ref.absorbed()
    runs = []
    for kern, regroup in [(k, r) for k in (hrt.HRT_KERNEL_EVENT, hrt.HRT_KERNEL_REGROUP) for r in (1, 8, 32)]:
        m = hrt.Model(wl)
        st = m.run_iteration(kernel=kern, regroup_threshold=regroup)
        runs.append(m.absorbed())
        if name == "tiny_sphere":
            # identical FP32 arithmetic in both kernels: same histories; the event kernel merges
            # a lane's FP32 kappa*l products within a cell before its FP64 atomic, the plain
            # kernel adds each product alone, so sums differ at FP32 rounding (< 1e-6)
            np.testing.assert_allclose(runs[-1], acc0, rtol=1e-6, atol=1e-300)
            for k in ("n_crossings", "n_interactions", "n_scatter", "n_absorb", "e_escaped"):
                assert st[k] == sp[k], (regroup, k)
        else:
            # the spherical walk is inlined differently in the two kernels (FMA contraction), so
            # a few histories part at FP32 rounding level, as against the oracle
            seen = acc0 > 0
            rel = np.abs(runs[-1][seen] - acc0[seen]) / acc0[seen]
            assert np.median(rel) < 1e-5
            assert st["n_crossings"] == pytest.approx(sp["n_crossings"], rel=1e-3)
    # the regroup threshold never changes a history (only the merge order of the deposits); nor,
    # on the Cartesian grid, does the form of the event kernel (warp-local or regrouped across
    # warps).  On the spherical grid the two forms are compiled at different register budgets (4
    # and 3 blocks per SM), whose FMA contraction of the walk may differ: there they agree as the
    # event and plain kernels do
    for r in runs[1:3]:
        np.testing.assert_allclose(r, runs[0], rtol=1e-6, atol=1e-300)
    for r in runs[4:6]:
        np.testing.assert_allclose(r, runs[3], rtol=1e-6, atol=1e-300)
    if name == "tiny_sphere":
        np.testing.assert_allclose(runs[3], runs[0], rtol=1e-6, atol=1e-300)
    else:
        seen = runs[0] > 0
        assert np.median(np.abs(runs[3][seen] - runs[0][seen]) / runs[0][seen]) < 1e-5
    # imaging pass: SEDs agree as well
    ref.run_iteration(kernel=hrt.HRT_KERNEL_PLAIN, peel=1, update_temperature=0, n_packets=5000)
    m = hrt.Model(wl)
    m.run_iteration(kernel=hrt.HRT_KERNEL_EVENT)
    m.run_iteration(kernel=hrt.HRT_KERNEL_EVENT, peel=1, update_temperature=0, n_packets=5000)
    sg, sr = m.sed(), ref.sed()
    np.testing.assert_allclose(sg.sum(axis=1), sr.sum(axis=1), rtol=1e-4)
    big = sr > 1e-3 * sr.max()
    np.testing.assert_allclose(sg[big], sr[big], rtol=1e-3)


@pytest.mark.parametrize("name", ["tiny_sphere", "flared_disk"])
def test_peel_queue_overflow_is_peeled_inline_with_the_same_result(name):
    # an imaging pass queues its peel-off events for the peel pass; events past the queue's
    # capacity are walked by the propagation kernel itself: the same rays (equal crossing counts)
    # and the same weights up to the FP32 rounding of each ray's optical depth (the two kernels
    # compile the walk separately, and the compiler may fuse its multiply-adds differently: over
    # n <= a few hundred crossings and tau <= the 40 at which a ray stops, |d tau| stays far
    # below n * 2^-24 * tau < 1e-3)
    wl = W.WORKLOADS[name](n_packets=100_000)
    if name == "flared_disk":
        wl = W.flared_disk(n_packets=100_000, n_r=80, n_theta=48)
        wl.img_nx = wl.img_ny = 32
        wl.img_half_extent = 300 * W.AU
        wl.img_lam_um = np.array([1.0, 100.0])
    runs = []
    for cap in (0, 1000):
        m = hrt.Model(wl)
        m.run_iteration()
        st = m.run_iteration(peel=1, update_temperature=0, peel_queue_events=cap)
        runs.append((st, m.sed(), m.image() if wl.img_nx > 0 else None))
    (s0, sed0, img0), (s1, sed1, img1) = runs
    assert s1["n_peel_crossings"] == s0["n_peel_crossings"] and s1["n_crossings"] == s0["n_crossings"]
    np.testing.assert_allclose(sed1.sum(axis=1), sed0.sum(axis=1), rtol=1e-6)
    np.testing.assert_allclose(sed1, sed0, rtol=1e-3, atol=1e-300)
    if img0 is not None:
        np.testing.assert_allclose(img1, img0, rtol=1e-3, atol=1e-300)
    with pytest.raises(hrt.HrtError):
        hrt.Model(wl).run_iteration(peel=1, update_temperature=0, peel_queue_events=-1)
