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
