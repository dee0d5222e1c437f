"""Pins of the oracle's modified random walk (Sect. 2.2; the published form the paper refers to).

* The sphere of an MRW step lies inside the cell: every point of the sphere at 0.999 times the
  wall distance locates in the cell, and some point of the sphere at 1.02 times it does not
  (the distance is the nearest wall's, on all three grids, with and without holes and phi
  walls).
* The path length solves the diffusion survival probability: P(s) evaluated by the Jacobi
  theta transformation of its series (a different formula, exact for every s) returns the
  uniform deviate, and the mean path is rho chi R0^2 / 2 (the mean first-passage time of
  diffusion from the centre of a sphere).
* A brute-force random walk of isotropic or Henyey-Greenstein scattering in a sphere of large
  optical depth leaves it after the path length the diffusion step predicts, once the transport
  extinction chi (1 - g) and the boundary's extrapolation length (0.7104 mean free paths) are
  counted.
* Whole iterations with the MRW conserve energy exactly and give the temperatures of the plain
  walk on a thick grey cube.
"""
import math

import numpy as np
import pytest

from oracle import mc as M
from oracle import tables as T
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import random_points_in_grid, spherical_test_grid, workload_from_walls


def _fibonacci_sphere(n):
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    phi = math.pi * (1.0 + math.sqrt(5.0)) * k
    s = np.sqrt(1.0 - z * z)
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def _grids():
    cyl_hole = [np.array([0.3, 0.5, 0.9, 1.4, 2.0]) * W.AU, np.array([-1.5, -0.4, 0.0, 0.3, 1.5]) * W.AU,
                np.array([0.0, 1.0, 2.5, 4.0, 2 * math.pi])]
    cyl_axis = [np.array([0.0, 0.5, 0.9, 1.4, 2.0]) * W.AU, cyl_hole[1], np.array([0.0, 2 * math.pi])]
    cart = [np.linspace(-1, 1, 4) * W.AU, np.array([-1.0, -0.2, 0.5, 1.0]) * W.AU, np.linspace(-1, 1, 3) * W.AU]
    return {
        "cartesian": ("cartesian", cart, 0.99 * W.AU),
        "spherical_hole_phi": ("spherical", spherical_test_grid(hole=True, nphi=4), 1.99 * W.AU),
        "spherical_axis": ("spherical", spherical_test_grid(hole=False, nphi=1), 1.99 * W.AU),
        "cylindrical_hole_phi": ("cylindrical", cyl_hole, 1.99 * W.AU),
        "cylindrical_axis": ("cylindrical", cyl_axis, 1.99 * W.AU),
    }


@pytest.mark.parametrize("name", list(_grids()))
def test_wall_distance_is_the_largest_ball_in_the_cell(name):
    gtype, walls, radius = _grids()[name]
    om = M.OracleModel(workload_from_walls(gtype, walls))
    om.struct(np.zeros(om.nc, np.int32))
    rng = np.random.default_rng(7)
    p, _, c = random_points_in_grid(om, 30, rng, radius)
    dirs = _fibonacci_sphere(800)        # 0.13 rad apart; the 1.02 d cap is 0.2 rad wide
    out = np.zeros(3)
    cc = np.zeros(3, np.int32)

    def inside(q, u, cell):
        st = M.lib().or_locate(om._struct, M._ptr(q), M._ptr(u), M._ptr(out), M._ptr(cc, M._ip))
        return st == 0 and np.array_equal(cc, cell) and np.allclose(out, q, rtol=0, atol=0)

    for q in range(len(p)):
        d = M.lib().or_wall_distance(om._struct, M._ptr(p[q]), M._ptr(c[q], M._ip))
        assert d > 0
        assert all(inside(p[q] + 0.999 * d * u, u, c[q]) for u in dirs), (name, q)
        assert not all(inside(p[q] + 1.02 * d * u, u, c[q]) for u in dirs), (name, q)


def _theta_survival(x):
    """P = 1 - 2 sqrt(pi / x) sum_k exp(-pi^2 (2k + 1)^2 / (4 x)) (Jacobi's theta-4 transformation
    of the alternating series)."""
    k = np.arange(8)
    return 1.0 - 2.0 * math.sqrt(math.pi / x) * np.exp(-(math.pi ** 2) * (2 * k + 1) ** 2 / (4.0 * x)).sum()


@pytest.mark.parametrize("tau0", [2.0, 10.0, 300.0])
def test_mrw_path_inverts_the_survival_probability(tau0):
    zetas = np.concatenate([10.0 ** -np.arange(1, 12), np.linspace(0.01, 0.99, 25), 1.0 - 10.0 ** -np.arange(2, 8)])
    for z in zetas:
        s = M.lib().or_mrw_path(tau0, float(z))          # path / R0
        x = math.pi ** 2 * s / (3.0 * tau0)             # pi^2 D s / R0^2 with D = R0 / (3 tau0) per R0
        P = _theta_survival(x)
        assert abs(P - z) <= 1e-12 + 1e-9 * (1.0 - z), (z, P)
    assert M.lib().or_mrw_path(tau0, 1.0) == 0.0


@pytest.mark.parametrize("tau0", [2.0, 50.0])
def test_mrw_mean_path_is_the_mean_first_passage(tau0):
    # E[s] = int_0^1 s(zeta) dzeta = int_0^inf s(e^-t) e^-t dt (Gauss-Laguerre in t)
    t, w = np.polynomial.laguerre.laggauss(120)
    s = np.array([M.lib().or_mrw_path(tau0, math.exp(-ti)) for ti in t])
    assert (w * s).sum() == pytest.approx(tau0 / 2.0, rel=2e-4)


def _hg_mu(g, u):
    if g == 0:
        return 2 * u - 1
    return (1 + g * g - ((1 - g * g) / (1 - g + 2 * g * u)) ** 2) / (2 * g)


def _random_walk_exit_path(tau0, g, n, rng):
    """Pure scattering from the centre of a sphere of radius tau0 (extinction mean free paths):
    total path length to the surface of every walker."""
    pos = np.zeros((n, 3))
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    path = np.zeros(n)
    alive = np.ones(n, bool)
    while alive.any():
        idx = np.flatnonzero(alive)
        step = -np.log(rng.uniform(size=idx.size))
        p, d = pos[idx], u[idx]
        # distance to the sphere along d
        b = (p * d).sum(axis=1)
        c = (p * p).sum(axis=1) - tau0 * tau0
        to_edge = -b + np.sqrt(b * b - c)
        out = step >= to_edge
        path[idx] += np.where(out, to_edge, step)
        pos[idx] = p + d * np.where(out, to_edge, step)[:, None]
        alive[idx[out]] = False
        keep = idx[~out]
        # scatter the walkers still inside
        mu = _hg_mu(g, rng.uniform(size=keep.size))
        psi = 2 * math.pi * rng.uniform(size=keep.size)
        d = u[keep]
        a = np.where(np.abs(d[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
        e1 = np.cross(a, d)
        e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
        e2 = np.cross(d, e1)
        st = np.sqrt(np.maximum(0.0, 1 - mu * mu))[:, None]
        u[keep] = mu[:, None] * d + st * (np.cos(psi)[:, None] * e1 + np.sin(psi)[:, None] * e2)
    return path


@pytest.mark.parametrize("tau0,g", [(20.0, 0.0), (40.0, 0.6)])
def test_mrw_path_matches_a_brute_force_random_walk(tau0, g):
    rng = np.random.default_rng(3)
    walk = _random_walk_exit_path(tau0, g, 3000, rng)
    # the diffusion step for the same sphere: tau0_t = tau0 (1 - g) transport mean free paths
    # (pure scattering: chi_t = chi (1 - g)); path in extinction mean free paths = tau0 * s / R0
    tau_t = tau0 * (1.0 - g)
    zs = (np.arange(20000) + 0.5) / 20000
    s = np.array([max(M.lib().or_mrw_path(tau_t, float(z)), 1.0) for z in zs]) * tau0
    # the random walk leaves a sphere whose radius is effectively larger by the extrapolation
    # length 0.7104 transport mean free paths: mean path (tau_t + 0.71)^2 / 2 / (1 - g)
    ext = ((tau_t + 0.7104) / tau_t) ** 2
    assert walk.mean() / s.mean() == pytest.approx(ext, rel=0.04)
    # the shape of the distribution: quartiles within the same factor
    for q in (0.25, 0.5, 0.75):
        assert np.quantile(walk, q) / np.quantile(s, q) == pytest.approx(ext, rel=0.08)


def _grey_cube(n=10, tau_cell=8.0, g=0.6, n_packets=4000):
    h = 100 * W.AU
    w = np.linspace(-h, h, n + 1)
    nu, chi, alb, _ = W.dust_table()
    chi = np.full_like(nu, 1.0)
    alb = np.full_like(nu, 0.5)
    rho0 = tau_cell / (chi[0] * (2 * h / n))
    wl = W.Workload(name="grey_cube", grid_type="cartesian", walls=[w, w.copy(), w.copy()],
                    rho=np.full((n, n, n), rho0, np.float32), nu=nu, chi=chi, albedo=alb, g=g,
                    T_nodes=W.temperature_nodes(), sources=[dict(pos=(1.0, 2.0, 3.0), L=W.LSUN, Teff=5800.0)],
                    obs_incl=np.radians([30.0]), obs_az=np.zeros(1), n_packets=n_packets, seed=17)
    return wl


def test_mrw_iteration_conserves_energy_and_matches_the_plain_walk():
    # 4^3 cells of 60 extinction mean free paths: the plain walk takes ~7000 interactions per
    # packet; Monte-Carlo noise of the cell temperatures at 8000 packets is 1.5 % (mean) and
    # 4 % (95th percentile) between two seeds
    wl = _grey_cube(n=4, tau_cell=60.0, n_packets=8000)
    plain = M.OracleModel(wl)
    mrw = M.OracleModel(wl)
    rp = plain.run_iteration(nthreads=16)
    rm = mrw.run_iteration(nthreads=16, mrw_gamma=2.0)
    for r, om in ((rp, plain), (rm, mrw)):
        assert r["e_escaped"] + r["e_killed"] == pytest.approx(om.L_tot, rel=1e-12)
        assert r["e_killed"] == 0
    assert rm["n_mrw"] > 0 and rp["n_mrw"] == 0
    assert rm["n_interactions"] < 0.5 * rp["n_interactions"]
    d = (mrw.T - plain.T) / plain.T
    assert np.abs(d).mean() < 0.025, np.abs(d).mean()
    assert np.percentile(np.abs(d), 95) < 0.07
    assert abs(d.mean()) < 0.02
