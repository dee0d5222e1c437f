"""Physics pins of the FP64 oracle against closed forms and invariants (no GPU).

* Henyey-Greenstein sampling: analytic CDF, mean cosine = g, normalisation.
* First flight through a grey absorbing slab: absorbed fraction (1 - E2(tau))/2 and the
  Lucy path-length estimator per layer (Eq. 2) against E2 differences.
* Peeling-off (Sect. 2.6.2): the direct stellar term through a slab is deterministic,
  eps/(4 pi) exp(-tau/mu) per packet; an empty grid gives L/(4 pi) to every observer.
* Optically thin limit: Adot(r) = L <kappa>_* / (4 pi r^2) and T ~ r^(-2/(4+beta)).
* Energy conservation: escaped + killed + absorbed = L exactly.
* Sect. 3: packet shards (threads or ranks) add up to one run.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import mc as M
from oracle import tables as T
from paper_1112_1071_gb300 import workloads as W


# ----------------------------------------------------------------- scattering
@pytest.mark.parametrize("g", [0.0, 0.3, 0.6, 0.9, -0.5])
def test_hg_inverse_cdf_against_analytic_cdf(g):
    def cdf(mu):
        if g == 0:
            return 0.5 * (mu + 1)
        return (1 - g * g) / (2 * g) * (1 / math.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))
    for u in np.linspace(1e-6, 1, 57):
        assert cdf(M.hg_mu(g, u)) == pytest.approx(u, abs=1e-12)


def test_hg_phase_normalised_and_mean_cosine():
    g = 0.6
    norm, _ = integrate.quad(lambda mu: 2 * math.pi * M.hg_phase(g, mu), -1, 1)
    mean, _ = integrate.quad(lambda mu: 2 * math.pi * mu * M.hg_phase(g, mu), -1, 1)
    assert norm == pytest.approx(1.0, rel=1e-10)
    assert mean == pytest.approx(g, rel=1e-10)
    rng = np.random.default_rng(2)
    mus = np.array([M.hg_mu(g, u) for u in W.uniforms(40000, rng)])
    assert mus.mean() == pytest.approx(g, abs=4 * mus.std() / math.sqrt(len(mus)))


def test_scatter_direction_frame():
    rng = np.random.default_rng(4)
    for k in range(300):
        u = rng.normal(size=3)
        if k % 10 == 0:
            u = np.array([1e-4, -2e-4, 1.0])           # near the pole: other frame
        u /= np.linalg.norm(u)
        mu, psi = rng.uniform(-1, 1), rng.uniform(0, 2 * math.pi)
        v = M.scatter_dir(u, mu, psi)
        assert np.linalg.norm(v) == pytest.approx(1.0, abs=1e-12)
        assert v @ u == pytest.approx(mu, abs=1e-12)
        if abs(u[2]) < 0.99999:
            e1 = np.cross([0, 0, 1.0], u)
        else:
            e1 = np.cross([0, 1.0, 0], u)
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(u, e1)
        st = math.sqrt(1 - mu * mu)
        assert (v @ e1) == pytest.approx(st * math.cos(psi), abs=1e-12)
        assert (v @ e2) == pytest.approx(st * math.sin(psi), abs=1e-12)


def test_isotropic_directions():
    v = M.isotropic(0.25, 0.125)
    assert v[2] == pytest.approx(-0.5)
    assert math.atan2(v[1], v[0]) == pytest.approx(2 * math.pi * 0.125)
    assert np.linalg.norm(v) == pytest.approx(1.0)


# ----------------------------------------------------------------- first flight
def test_grey_slab_absorption_and_lucy_deposit():
    tau = 1.0
    wl = W.slab(n_layers=8, tau_total=tau, albedo=0.0, n_packets=40000)
    om = M.OracleModel(wl)
    out = om.run_packets(wl.n_packets, 0, peel=True, terminate_on_absorb=True, nthreads=4)
    L = om.L_tot
    t = wl.walls[2][-1]
    z0 = wl.sources[0]["pos"][2]
    tau_up = tau * (t - z0) / t
    tau_dn = tau * z0 / t
    f_abs = 0.5 * (1 - special.expn(2, tau_up)) + 0.5 * (1 - special.expn(2, tau_dn))
    sig = math.sqrt(f_abs * (1 - f_abs) / wl.n_packets)
    assert out["e_absorbed"] / L == pytest.approx(f_abs, abs=4 * sig)
    assert out["e_absorbed"] + out["e_escaped"] + out["e_killed"] == pytest.approx(L, rel=1e-12)
    # Lucy estimator: rho * acc is the absorbed energy rate of the layer in expectation;
    # the spread of 10 disjoint packet chunks gives the Monte-Carlo error
    rho = float(wl.rho.reshape(-1)[0])
    zw = wl.walls[2]
    nchunk = 10
    per = wl.n_packets // nchunk
    chunks = np.array([rho * om.run_packets(per, 0, terminate_on_absorb=True, first_packet=k * per,
                                            n_total=per)["acc"] for k in range(nchunk)])
    mean, se = chunks.mean(axis=0), chunks.std(axis=0, ddof=1) / math.sqrt(nchunk)
    for l in range(len(zw) - 1):
        ta = tau * max(zw[l] - z0, 0.0) / t
        tb = tau * (zw[l + 1] - z0) / t
        expect = 0.5 * L * (special.expn(2, ta) - special.expn(2, tb))
        assert abs(mean[l] - expect) < 4 * se[l] + 2e-3 * expect, l
    # direct stellar term is deterministic: eps/(4 pi) exp(-tau/mu) from every packet
    tau_up_f32 = rho * float(wl.chi[0]) * (t - z0)      # the stored (float32) density
    for o, inc in enumerate(wl.obs_incl):
        want = L / (4 * math.pi) * math.exp(-tau_up_f32 / math.cos(inc))
        assert out["sed"][o].sum() == pytest.approx(want, rel=1e-10)


def test_empty_grid_peel_is_isotropic_and_exact():
    walls = [np.linspace(-1e14, 1e14, 3)] * 3
    nu, chi, alb, g = W.dust_table()
    wl = W.Workload(name="empty", grid_type="cartesian", walls=walls, rho=np.zeros((2, 2, 2), np.float32),
                    nu=nu, chi=chi, albedo=alb, g=g, T_nodes=W.temperature_nodes(),
                    sources=[dict(pos=(1e12, -3e12, 2e12), L=W.LSUN, Teff=5800.0)],
                    obs_incl=np.radians([10.0, 60.0, 120.0]), obs_az=np.radians([0.0, 45.0, 200.0]),
                    n_packets=20000)
    om = M.OracleModel(wl)
    out = om.run_packets(wl.n_packets, 0, peel=True)
    for o in range(3):
        assert out["sed"][o].sum() == pytest.approx(W.LSUN / (4 * math.pi), rel=1e-10)
    # every packet escapes untouched
    assert out["e_escaped"] == pytest.approx(W.LSUN, rel=1e-12) and out["n_interactions"] == 0
    # binned spectrum follows the blackbody (multinomial noise)
    lam_edges = 0.1 * 10 ** (np.arange(251) * 4 / 250) * 1e-4
    frac = out["sed"][0] / out["sed"][0].sum()
    nu_e = T.C_LIGHT / lam_edges
    f = lambda x: float(T.planck_bnu(x, 5800.0))
    tot, _ = integrate.quad(f, nu_e[-1], nu_e[0], limit=500, points=[3e14, 6e14])
    for b in (40, 60, 80, 100):
        pb, _ = integrate.quad(f, nu_e[b + 1], nu_e[b])
        pb /= tot
        sig = math.sqrt(pb / wl.n_packets)
        assert frac[b] == pytest.approx(pb, abs=5 * sig + 2e-3 * pb)


# ----------------------------------------------------------------- optically thin limit
def test_optically_thin_temperature_law():
    wl = W.tiny_sphere(tau_1um=1e-3, n_packets=100000)
    om = M.OracleModel(wl)
    out = om.run_iteration(nthreads=8)
    # source-spectrum-weighted absorption coefficient over the band
    nu = om.nu
    kap = lambda x: (1 - W.ALBEDO) * W.CHI_1UM * (x / (W.C_LIGHT / W.MICRON)) ** W.BETA_DUST
    B = lambda x: float(T.planck_bnu(x, 5800.0))
    num, _ = integrate.quad(lambda ln: kap(math.exp(ln)) * B(math.exp(ln)) * math.exp(ln),
                            math.log(nu[0]), math.log(nu[-1]), limit=400)
    den, _ = integrate.quad(lambda ln: B(math.exp(ln)) * math.exp(ln), math.log(nu[0]), math.log(nu[-1]),
                            limit=400)
    kbar = num / den
    w = wl.walls[0]
    n = len(w) - 1
    xc = 0.5 * (w[1:] + w[:-1])
    # volume average of 1/r^2 over each cell (4^3 midpoint sub-samples)
    sub = (np.arange(4) + 0.5) / 4
    d = w[1] - w[0]
    zz, yy, xx = np.meshgrid(xc, xc, xc, indexing="ij")
    inv_r2 = np.zeros_like(xx)
    for a in sub:
        for b in sub:
            for c in sub:
                inv_r2 += 1.0 / ((xx - d / 2 + a * d) ** 2 + (yy - d / 2 + b * d) ** 2 + (zz - d / 2 + c * d) ** 2)
    inv_r2 /= 64
    expect = om.L_tot * kbar / (4 * math.pi) * inv_r2.reshape(-1)
    r = np.sqrt(xx * xx + yy * yy + zz * zz).reshape(-1) / W.AU
    shell = (r > 25) & (r < 70) & (om.rho > 0)
    ratio = out["adot"][shell].sum() / expect[shell].sum()
    assert ratio == pytest.approx(1.0, abs=0.01)
    # temperature slope -2/(4+beta) where E(T) ~ T^(4+beta)
    slope = np.polyfit(np.log(r[shell]), np.log(out["T"][shell]), 1)[0]
    assert slope == pytest.approx(-2.0 / (4.0 + W.BETA_DUST), abs=0.01)


# ----------------------------------------------------------------- invariants
@pytest.mark.parametrize("name", ["tiny_sphere", "flared_disk"])
def test_energy_conservation_every_iteration(name):
    wl = W.WORKLOADS[name](n_packets=5000)
    om = M.OracleModel(wl)
    for _ in range(2):
        out = om.run_iteration(nthreads=4)
        assert out["e_escaped"] + out["e_killed"] + out["e_absorbed"] == pytest.approx(om.L_tot, rel=1e-12)
        # all-sky photon binning holds every escaping packet whose frequency is in band
        assert out["esc"].sum() == pytest.approx(out["e_escaped"], rel=1e-12)


def test_interaction_cap_kills_and_tallies():
    wl = W.flared_disk(n_packets=2000, tau_550=1e4)
    om = M.OracleModel(wl)
    out = om.run_iteration(max_interactions=3, nthreads=4)
    assert out["n_killed"] > 0
    assert out["e_killed"] == pytest.approx(out["n_killed"] * out["eps"], rel=1e-12)
    assert out["e_escaped"] + out["e_killed"] == pytest.approx(om.L_tot, rel=1e-12)


def test_packet_shards_add_up():
    wl = W.tiny_sphere(n_packets=6000)
    om = M.OracleModel(wl)
    one = om.run_packets(6000, 0, peel=True)
    thr = om.run_packets(6000, 0, peel=True, nthreads=3)
    a = om.run_packets(2500, 0, peel=True, first_packet=0, n_total=6000)
    b = om.run_packets(3500, 0, peel=True, first_packet=2500, n_total=6000)
    for key in ("acc", "sed", "esc"):
        np.testing.assert_allclose(thr[key], one[key], rtol=1e-11, atol=1e-300)
        np.testing.assert_allclose(a[key] + b[key], one[key], rtol=1e-11, atol=1e-300)
    assert one["n_crossings"] == thr["n_crossings"] == a["n_crossings"] + b["n_crossings"]
