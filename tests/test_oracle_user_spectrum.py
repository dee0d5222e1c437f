"""Pins of the oracle's point sources with a spectrum of their own (Sect. 2.1.1: a source has a
luminosity and a spectrum), read as f_nu interpolated log-log between the given nodes (linearly
where a value is zero), zero outside them, tabulated on the source grid over the dust band and
renormalised so that the in-band part carries all of L:

* a power law given on a few nodes is reproduced exactly (log-log interpolation is exact for it,
  a linear one is not);
* a blackbody given on many nodes gives the blackbody source's table within the interpolation
  error;
* no probability outside the given nodes, and a straight line next to a zero value;
* a whole Lucy iteration with a source whose spectrum is its own blackbody equals, in energy
  and temperatures, the iteration with the built-in blackbody of that temperature.
"""
import math

import numpy as np
import pytest

from oracle import mc as M
from oracle import tables as T
from paper_1112_1071_gb300 import workloads as W

NU = W.dust_table()[0]
NU0, NU1 = float(NU[0]), float(NU[-1])


def _grid(n=1000):
    k = np.arange(n)
    nu = NU0 * (NU1 / NU0) ** (k / (n - 1))
    nu[0], nu[-1] = NU0, NU1
    return nu


def test_power_law_is_reproduced_exactly():
    unu = np.geomspace(NU0 / 3, NU1 * 2, 7)
    f = unu ** -1.3
    nu, cdf = T.user_source_spectrum(NU0, NU1, unu, f)
    np.testing.assert_allclose(nu, _grid(), rtol=0)
    want = np.concatenate([[0.0], np.cumsum(0.5 * (nu[1:] ** -1.3 + nu[:-1] ** -1.3) * np.diff(nu))])
    np.testing.assert_allclose(cdf, want / want[-1], rtol=1e-11, atol=1e-14)
    # a straight-line interpolation of the same nodes is far from it
    lin = np.interp(nu, unu, f)
    clin = np.concatenate([[0.0], np.cumsum(0.5 * (lin[1:] + lin[:-1]) * np.diff(nu))])
    assert np.max(np.abs(clin / clin[-1] - cdf)) > 1e-2


def test_tabulated_blackbody_gives_the_blackbody_table():
    unu = np.geomspace(NU0 / 2, NU1 * 2, 4000)
    _, cdf = T.user_source_spectrum(NU0, NU1, unu, 7.0 * T.planck_bnu(unu, 6000.0))
    _, want = T.source_spectrum(NU0, NU1, 6000.0)
    assert np.max(np.abs(cdf - want)) < 1e-5


def test_nothing_outside_the_nodes_and_a_line_next_to_a_zero():
    nu = _grid()
    a, b = nu[300] * 1.0001, nu[600] * 0.9999
    unu = np.array([a, math.sqrt(a * b), b])
    _, cdf = T.user_source_spectrum(NU0, NU1, unu, np.array([2.0, 1.0, 3.0]))
    below = nu[1:] < a              # pieces whose both ends are below the first node
    assert np.all(cdf[1:][below] == 0.0)
    above = nu[:-1] > b
    assert np.all(cdf[:-1][above] == 1.0)
    # a zero value: linear between the nodes next to it
    unu = np.array([1e13, 2e13, 4e13])
    f = np.array([0.0, 4.0, 8.0])
    assert T.user_spectrum_at(1.5e13, unu, f) == pytest.approx(2.0, rel=1e-15)
    assert T.user_spectrum_at(3e13, unu, f) == pytest.approx(4.0 * 2 ** math.log2(1.5), rel=1e-12)
    assert T.user_spectrum_at(0.9e13, unu, f) == 0.0 and T.user_spectrum_at(4.1e13, unu, f) == 0.0
    assert T.user_spectrum_at(4e13, unu, f) == pytest.approx(8.0, rel=1e-15)


def test_iteration_with_an_own_blackbody_matches_the_built_in_one():
    wl = W.tiny_sphere(n_packets=20_000)
    om_bb = M.OracleModel(wl)
    unu = np.geomspace(NU0 / 2, NU1 * 2, 4000)
    wl2 = W.tiny_sphere(n_packets=20_000)
    wl2.sources = [dict(pos=s["pos"], L=s["L"], spectrum=(unu, T.planck_bnu(unu, s["Teff"]))) for s in wl2.sources]
    om_u = M.OracleModel(wl2)
    a = om_bb.run_iteration(nthreads=8)
    b = om_u.run_iteration(nthreads=8)
    assert b["e_escaped"] + b["e_killed"] == pytest.approx(om_u.L_tot, rel=1e-12)
    assert om_u.L_tot == om_bb.L_tot
    # the same streams draw nearly the same frequencies: temperatures agree to the table error
    dust = om_bb.rho > 0
    dT = np.abs(b["T"][dust] - a["T"][dust]) / a["T"][dust]
    assert dT.mean() < 2e-3
