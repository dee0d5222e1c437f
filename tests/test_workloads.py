"""The seeded synthetic inputs hold the optical depths, shapes and layouts their recipes state
(each checked here from the arrays themselves, not from the builder's own formulas)."""
import math

import numpy as np
import pytest

from paper_1112_1071_gb300 import workloads as W


def _tau_radial(wl, lam_um=0.55):
    """Cell-centre radial optical depth along a ray of the first theta row (spherical grids)."""
    rw = np.asarray(wl.walls[0])
    rho = np.asarray(wl.rho, dtype=np.float64)[0, 0, :]
    return float(np.sum(rho * np.diff(rw)) * W.chi_at_lambda_um(lam_um))


def test_embedded_envelope_has_its_radial_optical_depth_and_power_law():
    wl = W.embedded_envelope(n_r=60, n_theta=8, tau_550=1e5)
    assert np.asarray(wl.rho).shape == (1, 8, 60)
    assert _tau_radial(wl) == pytest.approx(1e5, rel=1e-6)             # FP32 densities
    rw = np.asarray(wl.walls[0])
    rc = 0.5 * (rw[1:] + rw[:-1])
    rho = np.asarray(wl.rho, dtype=np.float64)[0, 3, :]
    slope = np.polyfit(np.log(rc), np.log(rho), 1)[0]
    assert slope == pytest.approx(-1.5, abs=1e-6)
    # every theta row is the same envelope, and the star sits in the empty cavity
    assert np.all(np.asarray(wl.rho)[0] == np.asarray(wl.rho)[0, 0])
    assert rw[0] == pytest.approx(W.AU) and wl.sources[0]["pos"] == (0.0, 0.0, 0.0)


@pytest.mark.parametrize("kind,tau_cell,width_au", [("cartesian", 60.0, 50.0), ("spherical", 50.0, 20.0),
                                                     ("cylindrical", 50.0, 20.0)])
def test_thick_grey_models_have_their_cell_optical_depth(kind, tau_cell, width_au):
    wl = W.thick_grey(kind)
    assert np.all(np.asarray(wl.chi) == 1.0) and np.all(np.asarray(wl.albedo) == 0.5) and wl.g == 0.6
    rho = np.asarray(wl.rho, dtype=np.float64)
    assert np.all(rho == rho.flat[0])
    assert rho.flat[0] * 1.0 * width_au * W.AU == pytest.approx(tau_cell, rel=1e-6)
    assert rho.shape == tuple(len(w) - 1 for w in wl.walls)[::-1]
    moderate = W.thick_grey(kind, tau_cell=3.0)
    assert float(np.asarray(moderate.rho).flat[0]) * width_au * W.AU == pytest.approx(3.0, rel=1e-6)


def test_cylindrical_disk_midplane_column_and_layout():
    wl = W.cylindrical_disk(n_R=120, n_z=96, tau_550=100.0)
    rho = np.asarray(wl.rho, dtype=np.float64)
    assert rho.shape == (1, 96, 120)                                     # [phi][z][R]
    Rw, zw = np.asarray(wl.walls[0]), np.asarray(wl.walls[1])
    # mirror symmetric about the midplane, densest there
    assert np.allclose(rho[0], rho[0, ::-1], rtol=1e-6)
    assert np.all(rho[0, 47] >= rho[0, 0])
    # the model's continuous midplane radial depth is tau_550 with rho ~ 1/R, and it is Gaussian in z
    # with h = 10 AU at 100 AU: the vertical column there is the Gaussian integral sqrt(2 pi) h rho_mid
    # (the z cells resolve h at 100 AU; at 1 AU they do not, so no radial sum of cells is used)
    i = int(np.argmin(np.abs(0.5 * (Rw[1:] + Rw[:-1]) - 100 * W.AU)))
    Rc = 0.5 * (Rw[i] + Rw[i + 1])
    rho_mid = 100.0 / (W.chi_at_lambda_um(0.55) * 100 * W.AU * math.log(300.0)) * (100 * W.AU / Rc)
    h = 10 * W.AU * (Rc / (100 * W.AU)) ** 1.125
    assert float(np.sum(rho[0, :, i] * np.diff(zw))) == pytest.approx(math.sqrt(2 * math.pi) * h * rho_mid, rel=1e-3)
    assert zw[0] == pytest.approx(-zw[-1]) and wl.external_sources == []
    wl2 = W.cylindrical_disk(n_R=20, n_z=16, isrf_dilution=1e-13)
    (e,) = wl2.external_sources
    corner = math.hypot(wl2.walls[0][-1], wl2.walls[1][-1])
    assert e["radius"] > corner                                          # the sphere encloses the grid
    assert e["L"] == pytest.approx(W.isrf_luminosity(e["radius"], 1e-13, 6000.0))


@pytest.mark.parametrize("grid", ["cartesian", "spherical", "cylindrical"])
def test_isrf_cloud_encloses_the_grid_and_has_its_optical_depth(grid):
    wl = W.isrf_cloud(grid, n=8, tau_550=3.0)
    rho = np.asarray(wl.rho, dtype=np.float64)
    assert np.all(rho == rho.flat[0]) and wl.sources == []
    h = 1e4 * W.AU
    size = h if grid == "spherical" else 2 * h
    assert rho.flat[0] * W.chi_at_lambda_um(0.55) * size == pytest.approx(3.0, rel=1e-6)
    (e,) = wl.external_sources
    far = {"cartesian": math.sqrt(3) * h, "spherical": h, "cylindrical": math.sqrt(2) * h}[grid]
    assert e["radius"] > far


def test_tiny_sphere_recipe():
    wl = W.tiny_sphere()
    rho = np.asarray(wl.rho, dtype=np.float64)
    assert rho.shape == (32, 32, 32)
    w = np.asarray(wl.walls[0])
    assert w[0] == pytest.approx(-100 * W.AU) and w[-1] == pytest.approx(100 * W.AU) and w[16] == 0.0
    c = 0.5 * (w[1:] + w[:-1])
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    inside = np.sqrt(xx ** 2 + yy ** 2 + zz ** 2) < 80 * W.AU
    assert np.all(rho[~inside] == 0) and np.all(rho[inside] == rho[inside].flat[0])
    # radial optical depth at 1 micron of the continuous sphere is 1
    assert rho[inside].flat[0] * W.chi_at_lambda_um(1.0) * 80 * W.AU == pytest.approx(1.0, rel=1e-6)
    assert wl.sources == [dict(pos=(0.0, 0.0, 0.0), L=W.LSUN, Teff=5800.0)]
    np.testing.assert_allclose(np.degrees(wl.obs_incl), [12.5, 42.5, 77.5])


def test_flared_disk_recipe():
    wl = W.flared_disk()
    rho = np.asarray(wl.rho, dtype=np.float64)
    assert rho.shape == (1, 128, 200)
    rw, tw = np.asarray(wl.walls[0]), np.asarray(wl.walls[1])
    assert rw[0] == pytest.approx(W.AU) and rw[-1] == pytest.approx(1000 * W.AU)
    q = rw[1:] / rw[:-1]
    np.testing.assert_allclose(q, q[0], rtol=1e-9)                        # log-spaced radii
    dth = np.diff(tw)
    assert tw[0] == 0.0 and tw[-1] == pytest.approx(math.pi) and tw[64] == pytest.approx(math.pi / 2)
    assert dth.argmin() in (63, 64) and dth[0] / dth[63] > 50              # cones crowd the midplane
    np.testing.assert_allclose(dth, dth[::-1], rtol=1e-9)
    np.testing.assert_allclose(rho[0], rho[0, ::-1], rtol=1e-5)            # mirror symmetric
    # midplane radial tau_550 of 100 (the cells next to the midplane are far thinner than h)
    tau = float(np.sum(0.5 * (rho[0, 63] + rho[0, 64]) * np.diff(rw)) * W.chi_at_lambda_um(0.55))
    assert tau == pytest.approx(100.0, rel=2e-3)
    # vertical profile at 100 AU: Gaussian in z with h = 10 AU
    i = int(np.argmin(np.abs(0.5 * (rw[1:] + rw[:-1]) - 100 * W.AU)))
    rc = 0.5 * (rw[i] + rw[i + 1])
    thc = 0.5 * (tw[1:] + tw[:-1])
    z, R = rc * np.cos(thc), rc * np.sin(thc)
    h = 10 * W.AU * (R / (100 * W.AU)) ** 1.125
    col = rho[0, :, i] * (R / (100 * W.AU))                                # remove the 1/R factor
    near = np.abs(z) < 3 * h
    np.testing.assert_allclose(col[near] / np.exp(-0.5 * (z[near] / h[near]) ** 2), col[64] / math.exp(
        -0.5 * (z[64] / h[64]) ** 2), rtol=1e-5)
    assert len(wl.obs_incl) == 10 and wl.nsed == 250
    np.testing.assert_allclose(np.cos(wl.obs_incl), 0.05 + 0.1 * np.arange(10))


def test_batched_disk_parameters_span_their_ranges():
    models = W.batched_disks(size_scale=0.1)
    assert len(models) == 512
    r_in = np.array([m.walls[0][0] for m in models]) / W.AU
    teff = np.array([m.sources[0]["Teff"] for m in models])
    npk = np.array([m.n_packets for m in models])
    assert r_in.min() >= 0.1 and r_in.max() <= 5.0 and teff.min() >= 3000 and teff.max() <= 10000
    assert npk.min() >= 1e5 and npk.max() <= 1e7
    # log-uniform packet budgets and inner radii, uniform temperatures
    from scipy import stats
    assert stats.kstest(np.log10(npk), stats.uniform(5, 2).cdf).pvalue > 1e-3
    assert stats.kstest(np.log10(r_in), stats.uniform(-1, math.log10(50)).cdf).pvalue > 1e-3
    assert stats.kstest(teff, stats.uniform(3000, 7000).cdf).pvalue > 1e-3
    assert len({m.walls[0].size for m in models}) > 5                       # uneven grids


def test_turbulent_cloud_recipe():
    wl = W.turbulent_cloud(n=64, n_packets=1000)
    rho = np.asarray(wl.rho, dtype=np.float64)
    side = 0.65 * W.PC
    assert rho.shape == (64, 64, 64)
    assert rho.mean() * W.chi_at_lambda_um(0.55) * side == pytest.approx(10.0, rel=1e-5)
    lnr = np.log(rho)
    assert lnr.std() == pytest.approx(1.5, rel=1e-4)
    # the log density's power spectrum falls as k^(-11/3)
    P = np.abs(np.fft.rfftn(lnr - lnr.mean())) ** 2
    kx, ky, kz = np.fft.fftfreq(64)[:, None, None], np.fft.fftfreq(64)[None, :, None], np.fft.rfftfreq(64)[None, None, :]
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    kb = np.geomspace(3 / 64, 0.4, 10)
    mids, power = [], []
    for a, b in zip(kb[:-1], kb[1:]):
        sel = (k >= a) & (k < b)
        mids.append(math.sqrt(a * b))
        power.append(P[sel].mean())
    slope = np.polyfit(np.log(mids), np.log(power), 1)[0]
    assert slope == pytest.approx(-11 / 3, abs=0.25)
    assert len(wl.sources) == 20
    pos = np.array([s["pos"] for s in wl.sources])
    assert np.all(np.abs(pos) < side / 2)
    T = np.array([s["Teff"] for s in wl.sources])
    L = np.array([s["L"] for s in wl.sources]) / W.LSUN
    assert T.min() >= 3000 and T.max() <= 20000 and L.min() >= 0.1 and L.max() <= 100
    np.testing.assert_allclose(np.degrees([wl.obs_incl[0], wl.obs_az[0]]), [45.0, 45.0])
    np.testing.assert_allclose(wl.img_lam_um, [1.25, 3.6, 8.0, 70.0, 250.0, 500.0])
