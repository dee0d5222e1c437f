"""Pins of the oracle's external isotropic sources (Sect. 2.1.1) on Cartesian, spherical and
cylindrical grids.

A sphere that emits inwards with the cosine-weighted distribution of an isotropic intensity fills
its interior with a uniform, isotropic field of mean intensity J = L / (4 pi^2 R^2) (times the
spectrum).  Optically thin dust anywhere inside then absorbs Adot = 4 pi int kappa_nu J_nu dnu =
L / (pi R^2) int kappa_nu p(nu) dnu, the same in every cell, with p the packets' spectral pdf.
Every packet escapes in the end (nothing is killed), and a packet that misses the grid carries
no deposit."""
import math

import numpy as np
import pytest

from oracle import mc as M
from oracle import tables as T
from paper_1112_1071_gb300 import workloads as W


def _expected_adot(om, L, R):
    """L / (pi R^2) int kappa(nu) p(nu) dnu with p the piecewise-constant spectrum pdf and kappa
    log-log between the dust nodes (fine midpoint rule inside each spectrum piece)."""
    x = om.spec_nu
    p = np.diff(om.spec_cdf[-1]) / np.diff(x)
    total = 0.0
    for k in range(len(x) - 1):
        nu = np.linspace(x[k], x[k + 1], 33)
        mid = 0.5 * (nu[1:] + nu[:-1])
        chi = np.exp(np.interp(np.log(mid), np.log(om.nu), np.log(om.chi)))
        alb = np.interp(np.log(mid), np.log(om.nu), om.albedo)
        total += p[k] * np.sum((1 - alb) * chi * np.diff(nu))
    return L / (math.pi * R * R) * total


@pytest.mark.parametrize("grid", ["cartesian", "spherical", "cylindrical"])
def test_thin_cloud_in_isotropic_field(grid):
    wl = W.isrf_cloud(grid, n=6, tau_550=1e-4, n_packets=400_000)
    om = M.OracleModel(wl)
    r = om.run_iteration(nthreads=16)
    ext = wl.external_sources[0]
    assert r["e_killed"] == 0
    assert r["e_escaped"] == pytest.approx(om.L_tot, rel=1e-12)
    want = _expected_adot(om, ext["L"], ext["radius"])
    adot = r["adot"]
    # uniform: every cell within its sampling noise, the mean to 1 %
    assert np.mean(adot) == pytest.approx(want, rel=0.01)
    assert np.std(adot) / want < 0.08
    assert np.average(adot, weights=om.vol) == pytest.approx(want, rel=0.01)
    if grid == "cartesian":
        # the central 2^3 cells and the 8 corner cells see the same field
        a = adot.reshape(6, 6, 6)
        centre = a[2:4, 2:4, 2:4].mean()
        corners = a[::5, ::5, ::5].mean()
        assert centre == pytest.approx(corners, rel=0.05)


def test_isrf_luminosity_formula():
    # L = 4 pi R^2 * pi J with J = W sigma T^4 / pi
    L = W.isrf_luminosity(2.0, 1e-3, 100.0)
    assert L == pytest.approx(4 * math.pi * 4.0 * 1e-3 * W.SIGMA_SB * 1e8, rel=1e-14)
