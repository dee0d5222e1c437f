"""Pins of the oracle's partial diffusion approximation (App. A), Rosseland mean and packet-entry
counts, against closed forms and special cases that do not go through the oracle's own
discretisation:

* Rosseland mean: grey dust gives chi_R = chi; an adaptive quadrature of the definition with the
  power-law opacity; the infinite-band closed form chi_1 (kT/h nu_1)^beta Gamma(5) zeta(4) /
  (Gamma(5 - beta) zeta(4 - beta)) where the band holds the weight function.
* Diffusion solve: div(D grad x) = 0 with constant D has x = A + B / r between spheres and
  x = A + B ln tan(theta / 2) between cones; the discrete solution converges to them at second
  order.  Equal boundary values give that value exactly; a cell between two azimuthal neighbours
  of equal optical depth takes their mean; a mirror-symmetric problem has a mirror-symmetric
  solution; a region with no well-sampled neighbour keeps its Monte-Carlo temperatures.
* Packet entries: every packet enters the cell it is emitted in; in a grey absorbing slab the
  expected entries of layer l are N E_2(tau_l) / 2 (first flight); thread shards add up exactly.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import mc as M
from oracle import pda
from oracle import tables as T
from paper_1112_1071_gb300 import workloads as W


# ---------------------------------------------------------------- Rosseland mean
def test_rosseland_grey_dust_is_the_opacity():
    nu, _, _, _ = W.dust_table()
    chi = np.full_like(nu, 3.7)
    cr = T.rosseland_mean(nu, chi, W.temperature_nodes()[::50])
    np.testing.assert_allclose(cr, 3.7, rtol=1e-13)


def test_rosseland_against_quadrature_and_closed_form():
    nu, chi, _, _ = W.dust_table()
    beta, chi1, nu1 = W.BETA_DUST, W.CHI_1UM, T.C_LIGHT / 1e-4
    Tn = np.array([30.0, 100.0, 300.0, 1000.0])
    cr = T.rosseland_mean(nu, chi, Tn)
    for t, c in zip(Tn, cr):
        def w(lnv, inv_chi):
            v = math.exp(lnv)
            x = T.H_PLANCK * v / (T.K_BOLTZ * t)
            if x > 700:
                return 0.0
            d = 2 * T.H_PLANCK * v ** 3 / T.C_LIGHT ** 2 * (x / t) * math.exp(-x) / math.expm1(-x) ** 2
            return d * v * (1.0 / (chi1 * (v / nu1) ** beta) if inv_chi else 1.0)
        a, b = math.log(nu[0]), math.log(nu[-1])
        num = integrate.quad(w, a, b, args=(False,), limit=400, epsrel=1e-10)[0]
        den = integrate.quad(w, a, b, args=(True,), limit=400, epsrel=1e-10)[0]
        assert c == pytest.approx(num / den, rel=2e-3), t
    closed = chi1 * (T.K_BOLTZ * Tn / (T.H_PLANCK * nu1)) ** beta * special.gamma(5) * special.zeta(4) / (
        special.gamma(5 - beta) * special.zeta(4 - beta))
    np.testing.assert_allclose(cr[2:], closed[2:], rtol=5e-3)


# ---------------------------------------------------------------- diffusion solve
def _grey_grid(rw, tw, pw):
    """Uniform density and grey dust (chi_R = 1), so D is constant."""
    shape = (len(pw) - 1, len(tw) - 1, len(rw) - 1)
    rho = np.ones(int(np.prod(shape)))
    return [np.asarray(rw, float), np.asarray(tw, float), np.asarray(pw, float)], rho, shape


def _solve(walls, rho, T_mc, visits, n_min=1):
    Tn = np.array([1.0, 1e4])
    return pda.solve(walls, rho, T_mc, np.full_like(T_mc, 100.0), visits, n_min, Tn, np.ones(2))


def _radial_error(n):
    r0, r1 = 1.0, 3.0
    rw = np.linspace(r0, r1, n + 3)            # one boundary cell at each end
    walls, rho, shape = _grey_grid(rw, [0.4, 0.5], [0.0, 2 * math.pi])
    rc = 0.5 * (rw[1:] + rw[:-1])
    xa, xb = 100.0 ** 4, 20.0 ** 4            # T^4 at the boundary cells' centres
    B = (xa - xb) / (1 / rc[0] - 1 / rc[-1])
    A = xa - B / rc[0]
    T_mc = np.full(rc.size, 50.0)
    T_mc[0], T_mc[-1] = 100.0, 20.0
    visits = np.zeros(rc.size, int)
    visits[0] = visits[-1] = 10
    Tg, mask = _solve(walls, rho, T_mc, visits)
    assert mask[1:-1].all() and not mask[0] and not mask[-1]
    x = Tg ** 4
    return np.max(np.abs(x[1:-1] - (A + B / rc[1:-1])) / xa)


def test_radial_solution_converges_to_a_plus_b_over_r():
    e1, e2 = _radial_error(20), _radial_error(40)
    assert e2 < 2e-3 and e2 < 0.35 * e1, (e1, e2)


def _polar_error(n):
    ta, tb = 0.3, 1.3
    tw = np.linspace(ta, tb, n + 3)
    walls, rho, shape = _grey_grid([10.0, 10.5], tw, [0.0, 2 * math.pi])
    tc = 0.5 * (tw[1:] + tw[:-1])
    xa, xb = 80.0 ** 4, 30.0 ** 4
    f = np.log(np.tan(tc / 2))
    B = (xa - xb) / (f[0] - f[-1])
    A = xa - B * f[0]
    T_mc = np.full(tc.size, 50.0)
    T_mc[0], T_mc[-1] = 80.0, 30.0
    visits = np.zeros(tc.size, int)
    visits[0] = visits[-1] = 10
    Tg, mask = _solve(walls, rho, T_mc, visits)
    x = Tg ** 4
    return np.max(np.abs(x[1:-1] - (A + B * f[1:-1])) / xa)


def test_polar_solution_converges_to_log_tan():
    e1, e2 = _polar_error(20), _polar_error(40)
    assert e2 < 2e-3 and e2 < 0.35 * e1, (e1, e2)


def test_azimuthal_cell_takes_the_mean_of_equal_neighbours():
    walls, rho, shape = _grey_grid([1.0, 1.1], [1.0, 1.2], np.linspace(0, 2 * math.pi, 9))
    T_mc = np.full(8, 40.0)
    T_mc[2], T_mc[4] = 30.0, 60.0
    visits = np.full(8, 10)
    visits[3] = 0                                   # one cell between two boundary cells
    Tg, mask = _solve(walls, rho, T_mc, visits)
    assert mask.sum() == 1
    assert Tg[3] ** 4 == pytest.approx(0.5 * (30.0 ** 4 + 60.0 ** 4), rel=1e-12)


def test_equal_boundary_values_are_reproduced():
    rng = np.random.default_rng(3)
    rw = np.geomspace(1.0, 10.0, 9)
    tw = np.linspace(0.2, 2.9, 8)
    pw = np.linspace(0, 2 * math.pi, 5)
    walls = [rw, tw, pw]
    nc = 8 * 7 * 4
    rho = rng.uniform(0.5, 2.0, nc)
    T_mc = np.full(nc, 77.0)
    visits = rng.integers(0, 3, nc)                 # a random diffusion region
    Tg, mask = pda.solve(walls, rho, T_mc, rng.uniform(20, 200, nc), visits, 1,
                         W.temperature_nodes(), np.geomspace(0.1, 10, 1000))
    assert mask.any()
    np.testing.assert_allclose(Tg, 77.0, rtol=1e-10)


def test_mirror_symmetric_problem_has_symmetric_solution():
    rng = np.random.default_rng(4)
    rw = np.geomspace(1.0, 5.0, 7)
    half = np.sort(rng.uniform(0.2, math.pi / 2 - 0.1, 4))
    tw = np.concatenate([[0.0], half, [math.pi / 2], math.pi - half[::-1], [math.pi]])
    n1, n2 = 6, len(tw) - 1
    rho2 = rng.uniform(0.5, 2.0, (n2 // 2, n1))
    rho = np.concatenate([rho2, rho2[::-1]]).reshape(-1)
    T2 = rng.uniform(20, 300, (n2 // 2, n1))
    T_mc = np.concatenate([T2, T2[::-1]]).reshape(-1)
    v2 = rng.integers(0, 3, (n2 // 2, n1))
    visits = np.concatenate([v2, v2[::-1]]).reshape(-1)
    Tg, mask = pda.solve([rw, tw, np.array([0.0, 2 * math.pi])], rho, T_mc, T_mc, visits, 1,
                         W.temperature_nodes(), np.geomspace(0.1, 10, 1000))
    Tg = Tg.reshape(n2, n1)
    assert mask.any()
    np.testing.assert_allclose(Tg, Tg[::-1], rtol=1e-10)


def test_region_without_boundary_keeps_monte_carlo_values():
    walls, rho, shape = _grey_grid(np.linspace(1, 2, 5), [0.5, 0.6], [0.0, 2 * math.pi])
    rho[:] = [1.0, 0.0, 1.0, 1.0]                 # cell 0 isolated by a dust-free cell
    T_mc = np.array([11.0, 10.0, 30.0, 40.0])
    visits = np.array([0, 0, 5, 0])
    Tg, mask = _solve(walls, rho, T_mc, visits)
    assert not mask[0] and mask[3]
    assert Tg[0] == 11.0 and Tg[3] == pytest.approx(30.0, rel=1e-12)


# ---------------------------------------------------------------- packet entries
def test_slab_entries_follow_first_flight():
    n, layers, tau = 40_000, 8, 2.0
    wl = W.slab(n_layers=layers, tau_total=tau, albedo=0.0, n_packets=n)
    om = M.OracleModel(wl)
    r = om.run_packets(n, 0, terminate_on_absorb=True, nthreads=8)
    v = r["visits"].reshape(layers)
    assert v[0] == n                              # every packet starts in the bottom layer
    for l in range(1, layers):
        expect = 0.5 * n * special.expn(2, tau * l / layers)
        assert abs(v[l] - expect) < 5 * math.sqrt(expect) + 5, (l, v[l], expect)
    r1 = om.run_packets(n, 0, terminate_on_absorb=True, nthreads=1)
    np.testing.assert_array_equal(r1["visits"], r["visits"])
