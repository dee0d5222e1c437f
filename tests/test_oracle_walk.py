"""Pins of the oracle's cell walks (Sect. 2.1.2 grids, Sect. 2.2 propagation) by brute
force: every wall surface is intersected analytically, the crossings are sorted, and each
sub-segment is assigned to a cell by the coordinates of its midpoint.  A wrong wall index,
root choice, cone nappe, half-plane side or hole handling in the oracle fails here."""
import math

import numpy as np
import pytest

from oracle import mc as M
from paper_1112_1071_gb300 import workloads as W


def _model(grid_type, walls, rho=None):
    shape = tuple(len(w) - 1 for w in walls)
    if rho is None:
        rho = np.ones(shape[::-1], np.float32)
    nu, chi, alb, g = W.dust_table(10)
    wl = W.Workload(name="t", grid_type=grid_type, walls=[np.asarray(w, float) for w in walls],
                    rho=rho, nu=nu, chi=chi, albedo=alb, g=g, T_nodes=W.temperature_nodes(20),
                    sources=[dict(pos=(0.0, 0.0, 0.0), L=1.0, Teff=5000.0)])
    om = M.OracleModel(wl)
    om.struct(np.zeros(om.nc, np.int32))
    return om


def _trace(om, p, u):
    segc = np.zeros(4096, np.int64)
    segl = np.zeros(4096)
    p = np.ascontiguousarray(p, float)
    u = np.ascontiguousarray(u, float)
    n = M.lib().or_trace(om._struct, M._ptr(p), M._ptr(u), 4096, M._ptr(segc, M._lp), M._ptr(segl))
    assert 0 <= n < 4096
    return list(zip(segc[:n].tolist(), segl[:n].tolist()))


def _merge(segs, tol):
    out = []
    for c, l in segs:
        if l <= tol:
            continue
        if out and out[-1][0] == c:
            out[-1] = (c, out[-1][1] + l)
        else:
            out.append((c, l))
    return out


def _brute_cart(walls, p, u):
    ts = [0.0]
    t_exit = math.inf
    for a in range(3):
        if u[a] == 0:
            continue
        t = (np.asarray(walls[a]) - p[a]) / u[a]
        ts += [float(v) for v in t if v > 0]
        far = walls[a][-1] if u[a] > 0 else walls[a][0]
        t_exit = min(t_exit, (far - p[a]) / u[a])
    ts = sorted(set(t for t in ts if t <= t_exit) | {t_exit})
    n = [len(w) - 1 for w in walls]
    segs = []
    for t0, t1 in zip(ts[:-1], ts[1:]):
        q = p + 0.5 * (t0 + t1) * u
        idx = [int(np.searchsorted(walls[a], q[a], side="right") - 1) for a in range(3)]
        segs.append(((idx[2] * n[1] + idx[1]) * n[0] + idx[0], t1 - t0))
    return segs


def _brute_sph(walls, p, u):
    rw, tw, pw = (np.asarray(w, float) for w in walls)
    ts = [0.0]
    b = float(p @ u)
    pp = float(p @ p)
    for R in rw:
        disc = b * b - (pp - R * R)
        if disc > 0:
            ts += [t for t in (-b - math.sqrt(disc), -b + math.sqrt(disc)) if t > 0]
    for th in tw[1:-1]:
        c, s = math.cos(th), math.sin(th)
        if abs(c) < 1e-12:
            if u[2] != 0:
                t = -p[2] / u[2]
                if t > 0:
                    ts.append(t)
            continue
        A = u[2] ** 2 * s * s - (u[0] ** 2 + u[1] ** 2) * c * c
        B = p[2] * u[2] * s * s - (p[0] * u[0] + p[1] * u[1]) * c * c
        C = p[2] ** 2 * s * s - (p[0] ** 2 + p[1] ** 2) * c * c
        for t in np.roots([A, 2 * B, C]):
            if abs(t.imag) < 1e-12 and t.real > 0:
                q = p + t.real * u
                if q[2] * c > 0:
                    ts.append(float(t.real))
    if len(pw) > 2:
        for ph in pw[:-1]:
            nx, ny = -math.sin(ph), math.cos(ph)
            den = nx * u[0] + ny * u[1]
            if den != 0:
                t = -(nx * p[0] + ny * p[1]) / den
                q = p + t * u
                if t > 0 and math.cos(ph) * q[0] + math.sin(ph) * q[1] > 0:
                    ts.append(t)
    t_exit = -b + math.sqrt(b * b - (pp - rw[-1] ** 2))
    ts = sorted(set(t for t in ts if t <= t_exit) | {t_exit})
    n = [len(rw) - 1, len(tw) - 1, len(pw) - 1]

    def cell(q):
        r = math.sqrt(float(q @ q))
        if r < rw[0]:
            return None                   # the inner hole holds no cell
        th = math.acos(max(-1.0, min(1.0, q[2] / r)))
        ph = math.atan2(q[1], q[0]) % (2 * math.pi)
        i = int(np.searchsorted(rw, r, side="right") - 1)
        j = int(np.searchsorted(tw, th, side="right") - 1)
        k = int(np.searchsorted(pw, ph, side="right") - 1) if n[2] > 1 else 0
        return (k * n[1] + j) * n[0] + i

    # The crossings above are pinned without their coefficients: every crossing lies on one of
    # the wall surfaces (its polar angle, radius or azimuth equals a wall's), and no wall is
    # crossed inside a sub-segment (points spread along it all fall in its midpoint's cell), so
    # a wrong coefficient or nappe choice, or a missed root, fails here and not only in the oracle.
    for t in ts[1:-1]:
        q = p + t * u
        r = math.sqrt(float(q @ q))
        th = math.acos(max(-1.0, min(1.0, q[2] / r)))
        ph = math.atan2(q[1], q[0]) % (2 * math.pi)
        on = (np.min(np.abs(rw - r)) <= 1e-12 * rw[-1]
              or np.min(np.abs(tw[1:-1] - th)) <= 1e-9
              or (len(pw) > 2 and np.min(np.abs(np.angle(np.exp(1j * (pw - ph))))) <= 1e-9))
        assert on, ("crossing on no wall", p, u, t)
    segs = []
    for t0, t1 in zip(ts[:-1], ts[1:]):
        c = cell(p + 0.5 * (t0 + t1) * u)
        for f in (0.02, 0.1, 0.25, 0.4, 0.6, 0.75, 0.9, 0.98):
            if t1 - t0 > 1e-9 * rw[-1]:
                assert cell(p + (t0 + f * (t1 - t0)) * u) == c, ("wall inside a segment", p, u, t0, t1, f)
        if c is not None:
            segs.append((c, t1 - t0))
    return segs


def _compare(om, brute, walls, scale, n_rays, rng, start_radius):
    for _ in range(n_rays):
        while True:
            p = rng.uniform(-start_radius, start_radius, 3)
            if start_radius is None or np.linalg.norm(p) < start_radius:
                break
        mu = rng.uniform(-1, 1)
        ph = rng.uniform(0, 2 * math.pi)
        u = np.array([math.sqrt(1 - mu * mu) * math.cos(ph), math.sqrt(1 - mu * mu) * math.sin(ph), mu])
        got = _merge(_trace(om, p, u), 1e-9 * scale)
        ref = _merge(brute(walls, p, u), 1e-9 * scale)
        assert [c for c, _ in got] == [c for c, _ in ref], (p, u)
        np.testing.assert_allclose([l for _, l in got], [l for _, l in ref], rtol=1e-8, atol=1e-9 * scale)


def test_cartesian_walk_brute_force():
    rng = np.random.default_rng(7)
    walls = [np.array([-1.0, -0.3, 0.2, 1.0]), np.array([-1.0, 0.5, 1.0]), np.array([-1.0, -0.7, 0.0, 0.1, 1.0])]
    om = _model("cartesian", walls)
    _compare(om, _brute_cart, walls, 1.0, 400, rng, 0.999)


@pytest.mark.parametrize("hole,nphi", [(True, 4), (False, 1), (True, 1)])
def test_spherical_walk_brute_force(hole, nphi):
    rng = np.random.default_rng(8 + nphi)
    rw = np.array([0.3, 0.5, 0.9, 1.4, 2.0]) if hole else np.array([0.0, 0.5, 0.9, 1.4, 2.0])
    tw = np.array([0.0, 0.4, 1.1, math.pi / 2, 2.2, math.pi])
    pw = np.array([0.0, 1.0, 2.5, 4.0, 2 * math.pi]) if nphi == 4 else np.array([0.0, 2 * math.pi])
    walls = [rw, tw, pw]
    om = _model("spherical", walls)
    _compare(om, _brute_sph, walls, 2.0, 400, rng, 1.99)


def test_spherical_disk_grid_near_midplane_and_axis():
    # the production theta spacing: thin midplane cells and wide polar cells
    d = W.flared_disk(n_r=12, n_theta=16, n_phi=1)
    walls = [d.walls[0] / W.AU, d.walls[1], d.walls[2]]
    om = _model("spherical", walls)
    rng = np.random.default_rng(3)
    _compare(om, _brute_sph, walls, 1000.0, 300, rng, 900.0)


def test_tau_through_uniform_sphere_is_density_times_chord():
    rw = np.array([0.0, 0.3, 0.7, 1.0])
    tw = np.array([0.0, 0.5, math.pi / 2, 2.5, math.pi])
    pw = np.array([0.0, 2.0, 4.0, 2 * math.pi])
    om = _model("spherical", [rw, tw, pw], rho=np.full((3, 4, 3), 2.5, np.float32))
    rng = np.random.default_rng(9)
    for _ in range(200):
        p = rng.uniform(-0.55, 0.55, 3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        b = p @ u
        chord = -b + math.sqrt(b * b - (p @ p - 1.0))
        tau = M.lib().or_tau_to_edge(om._struct, M._ptr(p), M._ptr(u), 3.0)
        assert tau == pytest.approx(2.5 * 3.0 * chord, rel=1e-12)


def test_locate_on_walls_follows_direction():
    walls = [np.array([-1.0, 0.0, 1.0])] * 3
    om = _model("cartesian", walls)
    out = np.zeros(3)
    c = np.zeros(3, np.int32)
    for u, want in [((1, 1, 1), (1, 1, 1)), ((-1, -1, -1), (0, 0, 0)), ((1, -1, 0), (1, 0, 0))]:
        u = np.asarray(u, float) / np.linalg.norm(u)
        st = M.lib().or_locate(om._struct, M._ptr(np.zeros(3)), M._ptr(u), M._ptr(out), M._ptr(c, M._ip))
        assert st == 0 and tuple(c) == want


def test_axis_of_a_cylindrical_grid_without_hole_is_inside_the_first_ring():
    # R = 0 bounds no cell when R_0 = 0: a source on the axis starts in ring 0 whatever its
    # direction, and walks out of it as a ray from the axis (the first wall is R_1)
    walls = [np.array([0.0, 1.0, 2.0]) * W.AU, np.array([-1.0, 0.5, 1.0]) * W.AU, np.array([0.0, 2 * math.pi])]
    om = _model("cylindrical", walls)
    out = np.zeros(3)
    c = np.zeros(3, np.int32)
    for u in ((1.0, 0.0, 0.0), (0.0, 0.6, 0.8), (0.0, 0.0, -1.0)):
        u = np.asarray(u)
        st = M.lib().or_locate(om._struct, M._ptr(np.zeros(3)), M._ptr(u), M._ptr(out), M._ptr(c, M._ip))
        assert st == 0 and tuple(c) == (0, 0, 0)
        ax, d = np.zeros(1, np.int32), np.zeros(1, np.int32)
        dist = M.lib().or_cell_exit(om._struct, M._ptr(np.zeros(3)), M._ptr(u), M._ptr(c, M._ip), M._ptr(ax, M._ip),
                                    M._ptr(d, M._ip))
        R_hit = W.AU / math.hypot(u[0], u[1]) if math.hypot(u[0], u[1]) > 0 else math.inf
        z_hit = (0.5 * W.AU / u[2] if u[2] > 0 else -W.AU / u[2]) if u[2] != 0 else math.inf
        assert dist == pytest.approx(min(R_hit, z_hit), rel=1e-12)


def _brute_cyl(walls, p, u):
    Rw, zw, pw = (np.asarray(w, float) for w in walls)
    a = u[0] ** 2 + u[1] ** 2
    b = p[0] * u[0] + p[1] * u[1]
    c0 = p[0] ** 2 + p[1] ** 2
    ts = [0.0]
    t_exit = math.inf
    if a > 0:
        for R in Rw:
            disc = b * b - a * (c0 - R * R)
            if disc > 0:
                ts += [t for t in ((-b - math.sqrt(disc)) / a, (-b + math.sqrt(disc)) / a) if t > 0]
        t_exit = (-b + math.sqrt(b * b - a * (c0 - Rw[-1] ** 2))) / a
    if u[2] != 0:
        ts += [float(t) for t in (zw - p[2]) / u[2] if t > 0]
        t_exit = min(t_exit, ((zw[-1] if u[2] > 0 else zw[0]) - p[2]) / u[2])
    if len(pw) > 2:
        for ph in pw[:-1]:
            nx, ny = -math.sin(ph), math.cos(ph)
            den = nx * u[0] + ny * u[1]
            if den != 0:
                t = -(nx * p[0] + ny * p[1]) / den
                q = p + t * u
                if t > 0 and math.cos(ph) * q[0] + math.sin(ph) * q[1] > 0:
                    ts.append(t)
    ts = sorted(set(t for t in ts if t <= t_exit) | {t_exit})
    n = [len(Rw) - 1, len(zw) - 1, len(pw) - 1]
    segs = []
    for t0, t1 in zip(ts[:-1], ts[1:]):
        q = p + 0.5 * (t0 + t1) * u
        R = math.hypot(q[0], q[1])
        if R < Rw[0]:
            continue                      # the inner vacuum cylinder holds no cell
        ph = math.atan2(q[1], q[0]) % (2 * math.pi)
        i = int(np.searchsorted(Rw, R, side="right") - 1)
        j = int(np.searchsorted(zw, q[2], side="right") - 1)
        k = int(np.searchsorted(pw, ph, side="right") - 1) if n[2] > 1 else 0
        segs.append(((k * n[1] + j) * n[0] + i, t1 - t0))
    return segs


@pytest.mark.parametrize("hole,nphi", [(True, 4), (False, 1), (True, 1)])
def test_cylindrical_walk_brute_force(hole, nphi):
    rng = np.random.default_rng(18 + nphi)
    Rw = np.array([0.3, 0.5, 0.9, 1.4, 2.0]) if hole else np.array([0.0, 0.5, 0.9, 1.4, 2.0])
    zw = np.array([-1.5, -0.4, 0.0, 0.3, 1.5])
    pw = np.array([0.0, 1.0, 2.5, 4.0, 2 * math.pi]) if nphi == 4 else np.array([0.0, 2 * math.pi])
    walls = [Rw, zw, pw]
    om = _model("cylindrical", walls)
    n_done = 0
    for _ in range(400):
        while True:
            p = rng.uniform(-1.99, 1.99, 3)
            p[2] = rng.uniform(-1.49, 1.49)
            if math.hypot(p[0], p[1]) < 1.99:
                break
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        ref = _merge(_brute_cyl(walls, p, u), 1e-9 * 2.0)
        segc, segl = np.zeros(4096, np.int64), np.zeros(4096)
        n = M.lib().or_trace(om._struct, M._ptr(p), M._ptr(u), 4096, M._ptr(segc, M._lp), M._ptr(segl))
        if n < 0:                 # started in the hole and left it through a z plane
            assert ref == [], (p, u)
            n_done += 1
            continue
        got = _merge(list(zip(segc[:n].tolist(), segl[:n].tolist())), 1e-9 * 2.0)
        assert [c for c, _ in got] == [c for c, _ in ref], (p, u)
        np.testing.assert_allclose([l for _, l in got], [l for _, l in ref], rtol=1e-8, atol=1e-9 * 2.0)
        n_done += 1
    assert n_done == 400


def test_cylindrical_volumes_fill_the_annulus():
    from oracle import tables as T
    Rw = np.array([0.3, 0.5, 0.9, 2.0])
    zw = np.array([-1.0, 0.2, 1.5])
    pw = np.array([0.0, 1.0, 2 * math.pi])
    V = T.cell_volumes("cylindrical", [Rw, zw, pw])
    assert V.shape == (2, 2, 3)
    assert V.sum() == pytest.approx(math.pi * (2.0 ** 2 - 0.3 ** 2) * 2.5, rel=1e-14)
