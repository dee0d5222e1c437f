"""Pins of the oracle's escape tally (Sect. 2.6.1: escaping packets binned by direction and
wavelength; here 10 bins in the direction cosine u_z over [-1, 1] times the SED's wavelength
bins):

* direction: a point source above the midplane of a wide absorbing slab (pure absorber, the
  packets end when absorbed) lets out (L/2) int exp(-tau_face / |mu|) dmu into each bin, with the
  optical depth to the upper face for mu > 0 and to the lower face for mu < 0;
* wavelength: with no dust, a bin holds L times the mass of the source spectrum between its
  edges (the sampled frequency has a piecewise-linear CDF over the spectrum table), and the
  direction bins hold L/10 each.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import mc as M
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import workload_from_walls

AU = W.AU
C_LIGHT = 2.99792458e10


def _slab(rho):
    h = 1.0 * AU
    walls = [np.array([-20 * h, 0.0, 20 * h]), np.array([-20 * h, 0.0, 20 * h]), np.array([-h, 0.0, h])]
    wl = workload_from_walls("cartesian", walls, rho=np.full((2, 2, 2), rho, np.float32))
    wl.sources = [dict(pos=(0.0, 0.0, 0.5 * h), L=W.LSUN, Teff=5800.0)]
    wl.albedo = np.zeros_like(wl.nu)
    return wl, h


def test_direction_bins_of_an_absorbing_slab():
    rho = 1e-18
    wl, h = _slab(rho)
    wl.chi = np.full_like(wl.nu, 1.0 / (float(np.float32(rho)) * h))       # tau = 1 per h
    om = M.OracleModel(wl)
    n = 200_000
    out = om.run_packets(n, 0, terminate_on_absorb=True, nthreads=8)
    esc = out["esc"].sum(axis=1)                                          # over wavelength
    assert esc.sum() == pytest.approx(out["e_escaped"], rel=1e-12)
    eps = om.L_tot / n
    for k in range(10):
        a, b = -1 + 0.2 * k, -1 + 0.2 * (k + 1)
        tau = 0.5 if a >= 0 else 1.5                                      # to the upper / lower face
        p = 0.5 * integrate.quad(lambda mu: math.exp(-tau / abs(mu)), a, b)[0]
        sig = math.sqrt(n * p * (1 - p)) * eps
        assert abs(esc[k] - p * om.L_tot) < 4.5 * sig + 1e-6 * om.L_tot, (k, esc[k] / om.L_tot, p)


def test_wavelength_and_direction_bins_without_dust():
    wl, _ = _slab(0.0)
    om = M.OracleModel(wl)
    n = 200_000
    out = om.run_packets(n, 0, nthreads=8)
    assert out["e_escaped"] == pytest.approx(om.L_tot, rel=1e-12)
    eps = om.L_tot / n
    # direction: isotropic
    esc_mu = out["esc"].sum(axis=1)
    sig = math.sqrt(n * 0.1 * 0.9) * eps
    assert np.all(np.abs(esc_mu - 0.1 * om.L_tot) < 4.5 * sig)
    # wavelength: the spectrum's mass between each bin's edges
    edges_lam = wl.lam_min_um * 1e-4 * (wl.lam_max_um / wl.lam_min_um) ** (np.arange(wl.nsed + 1) / wl.nsed)
    F = lambda nu: np.interp(nu, om.spec_nu, om.spec_cdf[0])
    p = F(C_LIGHT / edges_lam[:-1]) - F(C_LIGHT / edges_lam[1:])
    assert p.sum() == pytest.approx(1.0, abs=1e-12)
    counts = out["esc"].sum(axis=0) / eps                                  # packets per bin
    np.testing.assert_allclose(counts, np.rint(counts), atol=1e-6)
    bound = 5 * np.sqrt(n * p * (1 - p)) + 2                               # (+2: bins of a few packets)
    assert np.all(np.abs(counts - n * p) < bound), np.max(np.abs(counts - n * p) / bound)
    # and the same counts against the masses shifted by one bin, or reversed, are far off
    chi2 = lambda c, q: float(np.sum((c - n * q) ** 2 / (n * q + 1)))
    good = chi2(counts, p)
    assert good < 2 * wl.nsed
    assert chi2(counts[1:], p[:-1]) > 3 * good and chi2(counts[::-1], p) > 100 * good
