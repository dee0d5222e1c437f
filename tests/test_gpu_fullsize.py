"""Parity at the full sizes of the benchmark workloads, in the launch configuration the
benchmark times (event kernel, tuned launch shape).

A whole iteration at full size is too long for the FP64 oracle, so it is checked by properties
that hold at any size (exact energy conservation, temperatures inside the table, every packet
accounted for); the oracle then checks a sample: a fresh context runs one share of the full
iteration (packet ids first..first+n-1 of n_total, eps = L/n_total) and the oracle runs the same
packet ids on the same Philox streams, so the two agree history by history (lockstep) up to the
rare histories that FP32 geometry moves across a wall."""
import numpy as np
import pytest

from oracle import mc as M
from paper_1112_1071_gb300 import hrt
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import pixel_parity

pytestmark = pytest.mark.gpu


def _share(wl, om, first, n, n_total, nthreads=16, **kw):
    """GPU and oracle results of packet ids first..first+n-1 of the first (n_total-packet)
    iteration, or of the imaging pass, from the starting temperatures."""
    m = hrt.Model(wl)
    st = m.run_iteration(n_packets=n, first_packet=first, n_total=n_total, **kw)
    key = 0 if kw.get("update_temperature", 1) else M.IMAGING_KEY
    ref = om.run_packets(n, key, first_packet=first, n_total=n_total, nthreads=nthreads,
                         peel=bool(kw.get("peel", 0)))
    return m, st, ref


def _lockstep(acc, ref_acc, median_tol, total_tol):
    seen = ref_acc > 0
    rel = np.abs(acc[seen] - ref_acc[seen]) / ref_acc[seen]
    assert np.median(rel) < median_tol, np.median(rel)
    assert abs(acc.sum() - ref_acc.sum()) <= total_tol * ref_acc.sum()
    # no deposits where the oracle has none, beyond the few parted histories
    assert (acc[~seen] > 0).sum() <= 1e-3 * seen.sum() + 5


def test_flared_disk_full_size():
    """200 x 128 disk, 1e7 packets per iteration."""
    wl = W.flared_disk()
    m = hrt.Model(wl)
    # the whole iteration: properties
    st = m.run_iteration()
    assert st["n_packets"] == 10_000_000
    assert st["e_escaped"] + st["e_killed"] == pytest.approx(st["e_emitted"], rel=1e-12)
    assert st["n_killed"] == 0
    T = m.temperature()
    assert np.all(np.isfinite(T)) and T.min() >= 1.0 and T.max() <= 2000.0
    assert (m.absorbed() >= 0).all()
    # a share from the middle of the first iteration's packet range, against the oracle
    om = M.OracleModel(wl)
    n_total, first, n = 10_000_000, 4_321_000, 100_000
    m2, st2, ref = _share(wl, om, first, n, n_total)
    assert st2["e_escaped"] + st2["e_killed"] == pytest.approx(ref["eps"] * n, rel=1e-12)
    assert st2["n_crossings"] == pytest.approx(ref["n_crossings"], rel=2e-3)
    _lockstep(m2.absorbed(), ref["acc"], 1e-4, 2e-3)
    # the peel-off pass at full size on a share: SEDs at 10 inclinations x 250 bins
    m3, st3, ref3 = _share(wl, om, 7_000_000, 20_000, n_total, peel=1, update_temperature=0)
    sed, rs = m3.sed(), ref3["sed"]
    np.testing.assert_allclose(sed.sum(axis=1), rs.sum(axis=1), rtol=1e-3)
    big = rs > 1e-3 * rs.max()
    np.testing.assert_allclose(sed[big], rs[big], rtol=2e-2)


def test_turbulent_cloud_full_size():
    """256^3 log-normal cloud, 20 sources, 1e8 packets per iteration, 512^2 x 6 images."""
    wl = W.turbulent_cloud()
    m = hrt.Model(wl)
    st = m.run_iteration()
    assert st["n_packets"] == 100_000_000
    assert st["e_escaped"] + st["e_killed"] == pytest.approx(st["e_emitted"], rel=1e-12)
    T = m.temperature()
    assert np.all(np.isfinite(T)) and T.min() >= 1.0 and T.max() <= 2000.0
    om = M.OracleModel(wl)
    n_total, first, n = 100_000_000, 61_234_567, 200_000
    m2, st2, ref = _share(wl, om, first, n, n_total)
    assert st2["e_escaped"] + st2["e_killed"] == pytest.approx(ref["eps"] * n, rel=1e-12)
    assert st2["n_crossings"] == pytest.approx(ref["n_crossings"], rel=1e-3)
    _lockstep(m2.absorbed(), ref["acc"], 1e-4, 1e-3)
    # images of an imaging-pass share
    m3, st3, ref3 = _share(wl, om, 33_000_000, 20_000, n_total, peel=1, update_temperature=0)
    img, ri = m3.image(), ref3["img"]
    np.testing.assert_allclose(img.sum(axis=(2, 3)), ri.sum(axis=(2, 3)), rtol=2e-2)
    # pixel by pixel (the share's packets peel into the same 512^2 pixels on both sides)
    stats = pixel_parity(img, ri)
    print("cloud image pixels", stats)
    assert stats["lit"] > 400
    assert stats["median_rel"] < 1e-6 and stats["frac_off"] < 0.01 and stats["l1_rel"] < 1e-4
    np.testing.assert_allclose(m3.sed().sum(axis=1), ref3["sed"].sum(axis=1), rtol=1e-3)
