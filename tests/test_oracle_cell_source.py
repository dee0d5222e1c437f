"""Pins of the oracle's diffuse (cell) sources (Sect. 2.1.1): a cell is picked in proportion to its
luminosity and the packet starts at a point uniform in the cell's volume with an isotropic
direction.

* placement: on all three grids the points of a cell follow, coordinate by coordinate, the exact
  volume CDF of the cell (Kolmogorov-Smirnov), are independent across coordinates (joint
  octant counts against the product of the volume fractions) and lie in the cell;
* whole path: a pure absorber (albedo 0) in a uniform sphere whose cells emit in proportion to
  their volume lets the escape probability of a uniformly emitting sphere out,
  3 / (8 tau^3) (2 tau^2 - 1 + (1 + 2 tau) exp(-2 tau)) (tau the radial optical depth);
* peel-off at emission: an empty Cartesian grid seen face-on images each emitting cell as a
  uniformly filled rectangle carrying its share of L / 4 pi.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import mc as M
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import workload_from_walls

AU = W.AU


def _cells():
    """Grid type, walls and the cell (i, j, k) that the placement tests sample."""
    return {
        "cartesian": ("cartesian", [np.array([-1.0, 0.2, 0.9]) * AU, np.array([-0.5, 0.1, 0.7]) * AU,
                                    np.array([-0.3, 0.4, 1.0]) * AU], (1, 0, 1)),
        "spherical": ("spherical", [np.array([0.0, 0.5, 0.9, 1.4]) * AU, np.array([0.0, 0.4, 1.1, math.pi]),
                                    np.array([0.0, 1.0, 2.5, 2 * math.pi])], (1, 1, 1)),
        "cylindrical": ("cylindrical", [np.array([0.0, 0.5, 0.9, 1.4]) * AU, np.array([-1.0, -0.4, 0.0, 0.6]) * AU,
                                        np.array([0.0, 1.0, 2.5, 2 * math.pi])], (1, 1, 1)),
    }


def _coords(gtype, p):
    """The grid's own coordinates of points p [n][3]."""
    if gtype == "cartesian":
        return p.T
    phi = np.mod(np.arctan2(p[:, 1], p[:, 0]), 2 * math.pi)
    if gtype == "spherical":
        r = np.linalg.norm(p, axis=1)
        return r, np.arccos(np.clip(p[:, 2] / r, -1, 1)), phi
    return np.hypot(p[:, 0], p[:, 1]), p[:, 2], phi


def _volume_cdfs(gtype, lo, hi):
    """Exact CDF of each coordinate of a point uniform in the cell's volume (the volume element
    is dx dy dz, r^2 sin(theta) dr dtheta dphi, or R dR dz dphi)."""
    lin = lambda a: (lambda x: (x - lo[a]) / (hi[a] - lo[a]))
    if gtype == "cartesian":
        return [lin(0), lin(1), lin(2)]
    if gtype == "spherical":
        return [lambda r: (r ** 3 - lo[0] ** 3) / (hi[0] ** 3 - lo[0] ** 3),
                lambda t: (np.cos(lo[1]) - np.cos(t)) / (np.cos(lo[1]) - np.cos(hi[1])), lin(2)]
    return [lambda R: (R ** 2 - lo[0] ** 2) / (hi[0] ** 2 - lo[0] ** 2), lin(1), lin(2)]


@pytest.mark.parametrize("name", list(_cells()))
def test_points_are_uniform_in_the_cell_volume(name):
    gtype, walls, cell = _cells()[name]
    om = M.OracleModel(workload_from_walls(gtype, walls))
    om.struct(np.zeros(om.nc, np.int32))
    rng = np.random.default_rng(3)
    n = 40000
    f = 1.0 - rng.random((n, 3))                             # (0, 1]
    c = np.array(cell, np.int32)
    out = np.zeros(3)
    p = np.empty((n, 3))
    for q in range(n):
        M.lib().or_place_in_cell(om._struct, M._ptr(c, M._ip), M._ptr(np.ascontiguousarray(f[q])), M._ptr(out))
        p[q] = out
    lo = [walls[a][cell[a]] for a in range(3)]
    hi = [walls[a][cell[a] + 1] for a in range(3)]
    x = _coords(gtype, p)
    cdfs = _volume_cdfs(gtype, lo, hi)
    for a in range(3):
        span = hi[a] - lo[a]
        assert np.all(x[a] >= lo[a] - 1e-12 * abs(span) - 1e-9 * AU * (a == 0))
        assert np.all(x[a] <= hi[a] + 1e-12 * abs(span) + 1e-9 * AU * (a == 0))
        assert stats.kstest(x[a], cdfs[a]).pvalue > 1e-4, (name, a)
    # joint: octants split at the coordinates' volume medians hold an eighth each
    med = []
    for a in range(3):
        grid = np.linspace(lo[a], hi[a], 20001)
        med.append(grid[np.searchsorted(cdfs[a](grid), 0.5)])
    octant = sum((x[a] > med[a]).astype(int) << a for a in range(3))
    counts = np.bincount(octant, minlength=8)
    assert stats.chisquare(counts).pvalue > 1e-4, counts
    # every point locates in the cell (direction irrelevant away from the walls)
    ci = np.zeros(3, np.int32)
    po = np.zeros(3)
    u = np.array([0.0, 0.0, 1.0])
    inner = np.all([(x[a] - lo[a] > 1e-6 * (hi[a] - lo[a])) & (hi[a] - x[a] > 1e-6 * (hi[a] - lo[a]))
                    for a in range(3)], axis=0)
    for q in np.flatnonzero(inner)[:2000]:
        assert M.lib().or_locate(om._struct, M._ptr(np.ascontiguousarray(p[q])), M._ptr(u), M._ptr(po),
                                 M._ptr(ci, M._ip)) == 0
        assert tuple(ci) == cell


def _emitting_sphere(tau, n_r=8, n_theta=3, rho=1e-18):
    """Uniform grey pure absorber in a sphere of radius 100 AU (radial optical depth tau) on a
    spherical grid with unequal shells and cones; every cell emits in proportion to its volume."""
    R = 100 * AU
    walls = [R * np.linspace(0, 1, n_r + 1) ** 0.7, np.array([0.0, 0.5, 1.9, math.pi])[: n_theta + 1],
             np.array([0.0, 2 * math.pi])]
    wl = workload_from_walls("spherical", walls, rho=np.full((1, n_theta, n_r), rho, np.float32))
    wl.chi = np.full_like(wl.nu, tau / (float(np.float32(rho)) * R))
    wl.albedo = np.zeros_like(wl.nu)
    wl.sources = []
    om0 = M.OracleModel(W.Workload(**{**wl.__dict__, "sources": [dict(pos=(0.0, 0.0, 0.0), L=1.0, Teff=5800.0)]}))
    wl.cell_source = dict(L=om0.vol * 1e30, Teff=3000.0)
    return wl


@pytest.mark.parametrize("tau", [0.5, 2.0])
def test_uniformly_emitting_sphere_escape_probability(tau):
    wl = _emitting_sphere(tau)
    om = M.OracleModel(wl)
    n = 100_000
    out = om.run_packets(n, 0, terminate_on_absorb=True, nthreads=8)
    assert out["e_escaped"] + out["e_absorbed"] == pytest.approx(om.L_tot, rel=1e-12)
    got = out["e_escaped"] / om.L_tot
    want = 3 / (8 * tau ** 3) * (2 * tau ** 2 - 1 + (1 + 2 * tau) * math.exp(-2 * tau))
    assert abs(got - want) < 4 * math.sqrt(want * (1 - want) / n), (got, want)
    # the same sphere emitting only from its centre lets exp(-tau) out: a different number
    assert abs(math.exp(-tau) - want) > 10 * math.sqrt(want * (1 - want) / n)


def test_face_on_image_of_emitting_cells():
    a = 10 * AU
    walls = [np.array([-a, 0.0, a]), np.array([-a / 2, a / 2]), np.array([-a / 2, a / 2])]
    wl = workload_from_walls("cartesian", walls, rho=np.zeros((1, 1, 2), np.float32))
    wl.sources = []
    wl.cell_source = dict(L=np.array([1.0, 3.0]) * W.LSUN, Teff=5000.0)
    wl.obs_incl, wl.obs_az = np.array([0.0]), np.array([0.0])
    wl.nsed, wl.lam_min_um, wl.lam_max_um = 1, 0.1, 1000.0
    wl.img_nx = wl.img_ny = 8
    wl.img_half_extent = a
    wl.img_lam_um = np.array([1.0])
    om = M.OracleModel(wl)
    n = 80_000
    out = om.run_packets(n, 0, peel=True, nthreads=8)
    L = om.L_tot
    np.testing.assert_allclose(out["sed"].sum(), L / (4 * math.pi), rtol=1e-12)
    img = out["img"][0, 0]
    np.testing.assert_allclose(img.sum(), L / (4 * math.pi), rtol=1e-12)
    # observer on +z, azimuth 0: image x = p . (0, 1, 0) = y, image y = p . ((0,0,1) x (0,1,0)) = -x;
    # pixels of a / 4: the cells span image columns 2-5; cell x < 0 rows 4-7, cell x > 0 rows 0-3
    foot = np.zeros((8, 8), bool)
    foot[:, 2:6] = True
    assert np.all(img[~foot] == 0)
    w = L / (4 * math.pi) / n                                  # one packet's weight
    hits = np.rint(img / w).astype(np.int64)
    np.testing.assert_allclose(hits * w, img, rtol=1e-9)
    upper, lower = hits[4:, 2:6], hits[:4, 2:6]                # cell 0 (L) and cell 1 (3 L)
    share = lower.sum() / n
    assert abs(share - 0.75) < 4 * math.sqrt(0.75 * 0.25 / n)
    for block in (upper, lower):
        assert stats.chisquare(block.reshape(-1)).pvalue > 1e-4
