"""The remaining setup and read-out calls of the C ABI on the GPU: point sources with a spectrum
of their own (against the oracle's table of it, step by step and over a whole iteration), the
model id that keys the random streams, clearing and re-adding sources, the library stream, the
device read-out of the SEDs and the watchdog report."""
import math

import numpy as np
import pytest

from oracle import mc as M
from paper_1112_1071_gb300 import hrt
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import dev, torch_cuda

pytestmark = pytest.mark.gpu

NU = W.dust_table()[0]


def _own_spectrum_sphere(n_packets=50_000):
    """The tiny sphere with its star given a spectrum of its own: a broken power law that is
    zero over part of the band (exercising the log-log pieces, a zero node and the range ends)."""
    wl = W.tiny_sphere(n_packets=n_packets)
    unu = np.array([NU[10] * 1.01, NU[30], NU[55], NU[70], NU[95] * 0.99])
    f = np.array([1.0, 40.0, 0.0, 5.0, 0.3])
    wl.sources = [dict(pos=s["pos"], L=s["L"], spectrum=(unu, f)) for s in wl.sources]
    return wl


def test_own_spectrum_frequencies_match_oracle():
    torch = torch_cuda()
    wl = _own_spectrum_sphere()
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    rng = np.random.default_rng(9)
    n = 50000
    us = ((rng.integers(0, 2 ** 24, n) + 1) * 2.0 ** -24).astype(np.float32)
    ud, sd = dev(us), dev(np.zeros(n, np.int32))
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    m.step("hrt_step_sample_source", n, sd.data_ptr(), ud.data_ptr(), out.data_ptr())
    got = out.cpu().numpy()
    want = np.array([M.sample_table(om.spec_nu, om.spec_cdf[0], float(us[q])) for q in range(n)])
    rel = np.abs(got - want) / want
    assert (rel > 1e-5).mean() < 1e-3 and np.median(rel) < 1e-6
    # nothing is drawn beyond the source-grid intervals that hold the spectrum's end nodes
    unu = wl.sources[0]["spectrum"][0]
    lo = om.spec_nu[np.searchsorted(om.spec_nu, unu[0]) - 1]
    hi = om.spec_nu[np.searchsorted(om.spec_nu, unu[-1])]
    assert got.min() >= lo * (1 - 1e-6) and got.max() <= hi * (1 + 1e-6)


def _lockstep(st, m, om, ref):
    assert st["e_escaped"] + st["e_killed"] == pytest.approx(om.L_tot, rel=1e-12)
    acc = m.absorbed()
    seen = ref["acc"] > 0
    rel = np.abs(acc[seen] - ref["acc"][seen]) / ref["acc"][seen]
    assert np.median(rel) < 1e-4, np.median(rel)
    assert st["n_crossings"] == pytest.approx(ref["n_crossings"], rel=2e-3)


def test_own_spectrum_iteration_matches_oracle():
    wl = _own_spectrum_sphere()
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    for _ in range(2):
        st = m.run_iteration()
        ref = om.run_iteration(nthreads=16)
        _lockstep(st, m, om, ref)


def test_model_id_keys_the_streams():
    wl = W.tiny_sphere(n_packets=50_000)
    om = M.OracleModel(wl)
    om.model_key = 7
    m = hrt.Model(wl)
    hrt.check(m.ctx, hrt.load().hrt_set_model_id(m.ctx, 7))
    st = m.run_iteration()
    ref = om.run_iteration(nthreads=16)
    _lockstep(st, m, om, ref)
    # other streams: the same model with id 0 deposits differently
    m0 = hrt.Model(wl)
    m0.run_iteration()
    seen = ref["acc"] > 0
    assert np.median(np.abs(m0.absorbed()[seen] / ref["acc"][seen] - 1)) > 1e-3


def test_clearing_and_re_adding_sources_gives_the_same_model():
    wl = W.tiny_sphere(n_packets=50_000)
    fresh = hrt.Model(wl)
    st0 = fresh.run_iteration()
    m = hrt.Model(wl)
    L = hrt.load()
    hrt.check(m.ctx, L.hrt_clear_sources(m.ctx))
    with pytest.raises(hrt.HrtError):
        m.run_iteration()                          # no sources
    for s in wl.sources:
        x = np.asarray(s["pos"], np.float64)
        hrt.check(m.ctx, L.hrt_add_point_source(m.ctx, x.ctypes.data, float(s["L"]), float(s["Teff"])))
    st = m.run_iteration()
    assert st["n_crossings"] == st0["n_crossings"] and st["n_interactions"] == st0["n_interactions"]
    np.testing.assert_allclose(m.absorbed(), fresh.absorbed(), rtol=1e-10)
    np.testing.assert_allclose(m.temperature(), fresh.temperature(), rtol=1e-10)


def test_library_stream_and_device_read_out():
    torch = torch_cuda()
    wl = W.tiny_sphere(n_packets=50_000)
    ref = hrt.Model(wl)
    ref.run_iteration()
    ref.run_iteration(peel=1, update_temperature=0)
    s = torch.cuda.Stream()
    m = hrt.Model(wl)
    hrt.check(m.ctx, hrt.load().hrt_set_stream(m.ctx, s.cuda_stream))
    m.run_iteration()
    st = m.run_iteration(peel=1, update_temperature=0)
    assert st["n_peel_crossings"] > 0
    np.testing.assert_allclose(m.sed(), ref.sed(), rtol=1e-10)
    d = torch.zeros(m.nobs * wl.nsed, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()                        # the fill runs on torch's stream, the read-out on s
    hrt.check(m.ctx, hrt.load().hrt_get_sed_device(m.ctx, d.data_ptr(), d.numel()))
    s.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy().reshape(m.nobs, wl.nsed), m.sed())
    assert hrt.load().hrt_get_sed_device(m.ctx, d.data_ptr(), d.numel() - 1) == hrt.HRT_EINVAL


def test_watchdog_report_after_a_timeout():
    wl = W.flared_disk(n_packets=2_000_000, n_r=100, n_theta=64)
    m = hrt.Model(wl)
    L = hrt.load()
    buf = np.zeros(512, np.float32)
    assert L.hrt_get_watchdog_report(m.ctx, buf.ctypes.data, 511) == hrt.HRT_EINVAL
    with pytest.raises(hrt.HrtError) as e:
        m.run_iteration(params=hrt.default_params(watchdog_ms=0.05))
    assert e.value.code == hrt.HRT_ETIMEDOUT
    r = L.hrt_get_watchdog_report(m.ctx, buf.ctypes.data, 512)
    assert 0 <= r <= 32
    rec = buf.reshape(32, 16)[:r]
    assert np.all(rec[:, 0] == np.rint(rec[:, 0])) and np.all((rec[:, 0] >= 0) & (rec[:, 0] < 16))  # lane modes
    st = m.run_iteration(n_packets=10_000)                      # and the context still works
    assert st["e_escaped"] + st["e_killed"] == pytest.approx(st["e_emitted"], rel=1e-12)


def test_escape_bins_match_oracle():
    """The escape tally by direction cosine and wavelength (Sect. 2.6.1), same packets as the
    oracle's: bin totals within what the few packets that part from lockstep can move."""
    wl = W.tiny_sphere(n_packets=50_000)
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    m.run_iteration()
    ref = om.run_iteration(nthreads=16)
    esc, resc = m.escape(), ref["esc"]
    assert esc.sum() == pytest.approx(resc.sum(), rel=1e-3)
    np.testing.assert_allclose(esc.sum(axis=1), resc.sum(axis=1), rtol=1e-2)
    lam, rlam = esc.sum(axis=0), resc.sum(axis=0)
    big = rlam > 1e-2 * rlam.max()
    np.testing.assert_allclose(lam[big], rlam[big], rtol=2e-2)


def test_spectrum_without_flux_in_the_band_is_rejected():
    wl = W.tiny_sphere(n_packets=1000)
    wl.sources = [dict(pos=(0.0, 0.0, 0.0), L=W.LSUN, spectrum=(np.array([NU[-1] * 2, NU[-1] * 3]), np.ones(2)))]
    m = hrt.Model(wl)
    with pytest.raises(hrt.HrtError) as e:
        m.run_iteration()
    assert e.value.code == hrt.HRT_EINVAL
    assert "no flux" in hrt.load().hrt_last_error(m.ctx).decode()


def test_point_source_checks():
    wl = W.cylindrical_disk(n_R=20, n_z=16, n_packets=1000)
    m = hrt.Model(wl)
    L = hrt.load()
    R_out, z_lo, z_hi = wl.walls[0][-1], wl.walls[1][0], wl.walls[1][-1]
    add = lambda x, Teff=5000.0: L.hrt_add_point_source(m.ctx, np.asarray(x, np.float64).ctypes.data, W.LSUN, Teff)
    # inside the cylinder although farther than R_out from the origin
    assert add([0.97 * R_out, 0.0, 0.9 * z_hi]) == hrt.HRT_OK
    assert add([0.0, 0.0, 1.1 * z_hi]) == hrt.HRT_EINVAL          # beyond an end plane
    assert add([0.0, 0.0, 1.1 * z_lo]) == hrt.HRT_EINVAL
    assert add([0.8 * R_out, 0.8 * R_out, 0.0]) == hrt.HRT_EINVAL  # outside the outer cylinder
    assert add([0.0, 0.0, 0.0], Teff=float("inf")) == hrt.HRT_EINVAL
    x = np.zeros(3)
    for nu in ([0.0, 1e14], [-1e14, 1e14], [1e14, float("nan")], [2e14, 1e14]):
        nu = np.asarray(nu, np.float64)
        f = np.ones(2)
        assert L.hrt_add_point_source_spectrum(m.ctx, x.ctypes.data, W.LSUN, 2, nu.ctypes.data,
                                               f.ctypes.data) == hrt.HRT_EINVAL
    st = m.run_iteration()                                          # the accepted sources run
    assert st["e_escaped"] + st["e_killed"] == pytest.approx(st["e_emitted"], rel=1e-12)


def test_peeloff_checks():
    wl = W.tiny_sphere(n_packets=1000)
    m = hrt.Model(wl)
    L = hrt.load()
    inc, az = np.array([0.3]), np.array([0.0])
    lam = np.array([1.0, -2.0])
    inf = float("inf")

    def peel(nsed=10, lo=0.1, hi=1000.0, nx=0, half=1e15, lam=lam, nimg=1):
        return L.hrt_set_peeloff(m.ctx, 1, inc.ctypes.data, az.ctypes.data, nsed, lo, hi, nx, nx, half, nimg,
                                 lam.ctypes.data)

    assert peel() == hrt.HRT_OK
    assert peel(nx=4) == hrt.HRT_OK
    for bad in (dict(nsed=0), dict(lo=0.0), dict(hi=0.05), dict(hi=inf), dict(nx=4, half=inf), dict(nx=4, half=0.0),
                dict(nx=4, nimg=2), dict(nx=4, nimg=0)):
        assert peel(**bad) == hrt.HRT_EINVAL, bad
    assert peel() == hrt.HRT_OK
    st = m.run_iteration(peel=1, update_temperature=0)
    assert st["n_peel_crossings"] > 0


def test_run_parameter_checks():
    wl = W.tiny_sphere(n_packets=2000)
    m = hrt.Model(wl)
    nan = float("nan")
    for bad in (dict(kernel=5), dict(quantity=2), dict(block_size=128), dict(blocks_per_sm=-1),
                dict(regroup_threshold=33), dict(regroup_threshold=-1), dict(watchdog_ms=-1.0),
                dict(watchdog_ms=nan), dict(q_thres=nan), dict(delta_thres=nan)):
        with pytest.raises(hrt.HrtError) as e:
            m.run_iteration(**bad)
        assert e.value.code == hrt.HRT_EINVAL, bad
    st = m.run_iteration(block_size=256, blocks_per_sm=3, regroup_threshold=32, quantity=1)
    assert st["iteration"] == 0                       # the rejected calls ran nothing
    assert st["e_escaped"] + st["e_killed"] == pytest.approx(st["e_emitted"], rel=1e-12)


@pytest.mark.parametrize("quantity", [0, 1])
def test_resume_from_saved_temperatures_repeats_the_iteration(quantity):
    """Checkpoint/resume: the temperatures and specific energies after iteration i-1, the
    iteration counter (which keys the random streams) and the previous percentile Q^{i-1} (Eqs.
    5-6) are the whole state Lucy iteration i starts from; with them a fresh context repeats the
    iteration, its Q, Delta and converged flag included, for T and for Adot as the quantity."""
    wl = W.tiny_sphere(n_packets=50_000)
    kw = dict(quantity=quantity, q_thres=10.0, delta_thres=10.0)
    a = hrt.Model(wl)
    a.run_iteration(**kw)
    a.run_iteration(**kw)
    T2, A2, conv = a.temperature(), a.specific_energy(), a.convergence_state()
    assert conv[0] == 1 and 1.0 <= conv[1] < math.inf
    st_a = a.run_iteration(**kw)
    b = hrt.Model(wl)
    b.set_temperature(T2)
    b.set_specific_energy(A2)
    b.set_iteration(2)
    b.set_convergence_state(*conv)
    st_b = b.run_iteration(**kw)
    assert st_b["iteration"] == st_a["iteration"] == 2
    for k in ("n_crossings", "n_interactions", "n_scatter", "n_absorb"):
        assert st_b[k] == st_a[k], k
    np.testing.assert_allclose(b.absorbed(), a.absorbed(), rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose(b.temperature(), a.temperature(), rtol=1e-10)
    np.testing.assert_allclose(b.specific_energy(), a.specific_energy(), rtol=1e-10, atol=1e-300)
    assert math.isfinite(st_a["Q"]) and math.isfinite(st_a["Delta"])
    assert st_b["Q"] == pytest.approx(st_a["Q"], rel=1e-9)
    assert st_b["Delta"] == pytest.approx(st_a["Delta"], rel=1e-9)
    assert st_b["converged"] == st_a["converged"] == 1
    # without the saved percentile, Delta is unknown and the run is not converged
    c = hrt.Model(wl)
    c.set_temperature(T2)
    c.set_specific_energy(A2)
    c.set_iteration(2)
    st_c = c.run_iteration(**kw)
    assert st_c["Q"] == pytest.approx(st_a["Q"], rel=1e-9)
    assert math.isinf(st_c["Delta"]) and st_c["converged"] == 0


def test_resume_setters_check_their_arguments():
    wl = W.tiny_sphere(n_packets=1000)
    m = hrt.Model(wl)
    for have, q in ((1, 0.5), (1, float("nan"))):
        with pytest.raises(hrt.HrtError) as e:
            m.set_convergence_state(have, q)
        assert e.value.code == hrt.HRT_EINVAL
    m.set_convergence_state(1, math.inf)
    assert m.convergence_state() == (1, math.inf)
    m.set_convergence_state(0, 0.0)
    assert m.convergence_state() == (0, math.inf)
    bad = np.full(m.ncells, 1.0)
    bad[3] = -1.0
    for arr in (bad, np.full(m.ncells - 1, 1.0)):
        with pytest.raises(hrt.HrtError) as e:
            m.set_specific_energy(arr)
        assert e.value.code == hrt.HRT_EINVAL
