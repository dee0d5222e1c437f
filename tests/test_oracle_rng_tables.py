"""Pins of the FP64 oracle's random numbers and tables against published values and closed
forms (no GPU).  Each test fails for a plausible mistake in the oracle: a wrong Philox
constant or round order, a missing 4 pi or (1 - albedo), a transposed table, a wrong
interpolation base."""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import mc as M
from oracle import tables as T
from paper_1112_1071_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert M.philox4x32_10(ctr, key) == out


def test_uniform_lattice_ends():
    # u = ((x >> 8) + 1) 2^-24 lies in (0, 1]: smallest 2^-24, largest exactly 1.
    assert M.uniform_from_word(0) == 2.0 ** -24
    assert M.uniform_from_word(0xFFFFFFFF) == 1.0
    assert M.uniform_from_word(0x000000FF) == 2.0 ** -24   # low byte discarded
    assert M.uniform_from_word(0x80000000) == (0x800000 + 1) * 2.0 ** -24


def test_planck_integral_closed_form():
    # int B_nu dnu = sigma T^4 / pi (Eq. 3's B(T)).
    for Tk in (30.0, 300.0, 5800.0):
        f = lambda lnnu: float(T.planck_bnu(math.exp(lnnu), Tk)) * math.exp(lnnu)
        val, _ = integrate.quad(f, math.log(1e6), math.log(1e17), limit=400)
        assert val == pytest.approx(T.SIGMA_SB * Tk ** 4 / math.pi, rel=1e-8)


def _power_law_E(Tk, beta=W.BETA_DUST, albedo=W.ALBEDO):
    """E(T) = 4 pi int kappa_nu B_nu dnu for kappa = (1-a) chi1 (nu/nu1)^beta over all nu:
    4 pi (1-a) chi1 nu1^-beta (2h/c^2) (kT/h)^(4+beta) Gamma(4+beta) zeta(4+beta)."""
    nu1 = W.C_LIGHT / W.MICRON
    k = T.K_BOLTZ
    h = T.H_PLANCK
    c = T.C_LIGHT
    return (4 * math.pi * (1 - albedo) * W.CHI_1UM * nu1 ** -beta * 2 * h / c ** 2
            * (k * Tk / h) ** (4 + beta) * special.gamma(4 + beta) * special.zeta(4 + beta))


def test_emission_table_against_power_law_closed_form():
    nu, chi, alb, _ = W.dust_table()
    tab = T.DustTables(nu, chi, alb, W.temperature_nodes())
    # where the band 0.1-1000 um holds the whole emission, the trapezoid table matches the
    # closed form to its quadrature error (~1e-3 with 100 log-spaced nodes)
    for Tk in (20.0, 50.0, 100.0, 300.0, 500.0):
        m = int(np.argmin(np.abs(tab.T - Tk)))
        assert tab.E[m] == pytest.approx(_power_law_E(tab.T[m]), rel=3e-3)
    # kappa_P = E / (4 sigma T^4) then follows the same closed form
    m = int(np.argmin(np.abs(tab.T - 100.0)))
    kp = tab.kappa_planck()[m]
    assert kp == pytest.approx(_power_law_E(tab.T[m]) / (4 * T.SIGMA_SB * tab.T[m] ** 4), rel=3e-3)
    # log-slope 4 + beta
    i1, i2 = (int(np.argmin(np.abs(tab.T - t))) for t in (40.0, 200.0))
    slope = math.log(tab.E[i2] / tab.E[i1]) / math.log(tab.T[i2] / tab.T[i1])
    assert slope == pytest.approx(4 + W.BETA_DUST, abs=5e-3)
    # emissivity rows are normalised cumulative distributions
    assert np.all(np.diff(tab.cdf, axis=1) >= 0)
    assert np.all(tab.cdf[:, 0] == 0) and np.all(tab.cdf[:, -1] == 1)


def test_emission_rows_follow_kappa_B():
    # the pdf of a row on each interval is the trapezoid mean of kappa B_nu; check one
    # interval ratio directly against the integrand.
    nu, chi, alb, _ = W.dust_table()
    tab = T.DustTables(nu, chi, alb, W.temperature_nodes())
    m = 600
    f = (1 - alb) * chi * T.planck_bnu(nu, tab.T[m])
    piece = 0.5 * (f[1:] + f[:-1]) * np.diff(nu)
    p = np.diff(tab.cdf[m])
    np.testing.assert_allclose(p, piece / piece.sum(), rtol=1e-9, atol=1e-15)  # cumsum differencing


def test_temperature_inversion_round_trip_and_clamps():
    nu, chi, alb, _ = W.dust_table()
    tab = T.DustTables(nu, chi, alb, W.temperature_nodes())
    # nodes invert exactly
    Tn, lo, hi = T.temperature_from_adot(tab.E[1:-1], tab.T, tab.E)
    np.testing.assert_allclose(Tn, tab.T[1:-1], rtol=1e-12)
    assert lo == 0 and hi == 0
    # between nodes the answer is inside the bracket and exact for a local power law
    rng = np.random.default_rng(0)
    m = rng.integers(100, 900, 50)
    f = rng.uniform(0, 1, 50)
    Tm = tab.T[m] * (tab.T[m + 1] / tab.T[m]) ** f
    a = tab.E[m] * (tab.E[m + 1] / tab.E[m]) ** f
    Tn, _, _ = T.temperature_from_adot(a, tab.T, tab.E)
    np.testing.assert_allclose(Tn, Tm, rtol=1e-10)
    # clamps
    Tn, lo, hi = T.temperature_from_adot(np.array([0.0, tab.E[0] * 0.5, tab.E[-1] * 2]), tab.T, tab.E)
    assert list(Tn) == [1.0, 1.0, 2000.0] and lo == 2 and hi == 1


def test_emission_row_nearest_in_log_T():
    nodes = W.temperature_nodes()
    lt = np.log(nodes)
    rng = np.random.default_rng(1)
    x = rng.uniform(lt[0] - 0.5, lt[-1] + 0.5, 2000)
    rows = T.emission_row(np.exp(x), nodes)
    brute = np.array([int(np.argmin(np.abs(lt - v))) for v in x])
    np.testing.assert_array_equal(rows, brute)
    # exact midpoint goes to the lower node
    mid = math.exp(0.5 * (lt[10] + lt[11]))
    assert T.emission_row(np.array([mid]), nodes)[0] in (10,)


def test_sample_table_piecewise_constant_pdf():
    x = np.array([1.0, 2.0, 4.0, 5.0])
    cdf = np.array([0.0, 0.25, 0.25, 1.0])   # the middle interval has zero probability
    assert M.sample_table(x, cdf, 0.125) == pytest.approx(1.5)
    assert M.sample_table(x, cdf, 0.25) == pytest.approx(2.0)
    assert M.sample_table(x, cdf, 0.25 + 1e-12) == pytest.approx(4.0, abs=1e-9)
    assert M.sample_table(x, cdf, 1.0) == 5.0
    assert M.sample_table(x, cdf, 0.625) == pytest.approx(4.5)


def test_sampled_spectrum_histogram_matches_row():
    nu, chi, alb, _ = W.dust_table()
    tab = T.DustTables(nu, chi, alb, W.temperature_nodes())
    m = 700
    rng = np.random.default_rng(5)
    us = W.uniforms(20000, rng)
    s = np.array([M.sample_table(nu, tab.cdf[m], u) for u in us])
    counts = np.histogram(s, bins=nu)[0]
    p = np.diff(tab.cdf[m])
    keep = p * len(us) > 20
    chi2 = (((counts - p * len(us)) ** 2 / (p * len(us)))[keep]).sum()
    dof = keep.sum() - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


def test_convergence_nearest_rank_and_paper_parameter_sets():
    assert T.delta(2.0, 1.0) == 2.0 and T.delta(1.0, 2.0) == 2.0 and T.delta(3.0, 3.0) == 1.0
    v = np.arange(1, 101, dtype=float)
    assert T.percentile_nearest_rank(v, 0.99) == 99.0
    assert T.percentile_nearest_rank(v, 0.995) == 100.0
    assert T.percentile_nearest_rank(v, 0.01) == 1.0
    rows = [l.split() for l in open(os.path.join(GOLDEN, "convergence_examples.txt"))
            if l.strip() and not l.startswith("#")]
    for name, p, qt, dt in rows:
        p, qt, dt = float(p), float(qt), float(dt)
        n = 10000
        prev = np.ones(n)
        cur = np.ones(n) * 1.5                     # every cell changed by a factor 1.5 < Q_thres
        k = int(math.floor((1 - p) * n))            # this many cells may change a lot
        cur[:k] = 10.0
        mask = np.ones(n, bool)
        Q, D = T.convergence(prev, cur, mask, p, Q_prev=1.5)
        assert Q == pytest.approx(1.5) and Q < qt and D <= dt, name
        cur[: k + 1] = 10.0                         # one outlier too many
        Q, _ = T.convergence(prev, cur, mask, p, Q_prev=1.5)
        assert Q == 10.0 and Q > qt, name


def test_cell_volumes_sum_to_domain():
    w = W.tiny_sphere(n=4)
    V = T.cell_volumes("cartesian", w.walls)
    assert V.sum() == pytest.approx((200 * W.AU) ** 3, rel=1e-12)
    d = W.flared_disk(n_r=10, n_theta=8, n_phi=3)
    V = T.cell_volumes("spherical", d.walls)
    r0, r1 = d.walls[0][0], d.walls[0][-1]
    assert V.sum() == pytest.approx(4 * math.pi / 3 * (r1 ** 3 - r0 ** 3), rel=1e-12)
