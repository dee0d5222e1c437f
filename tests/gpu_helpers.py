"""Shared helpers of the GPU tests (seeded inputs, oracle models, library models)."""
import math

import numpy as np

from oracle import mc as M
from paper_1112_1071_gb300 import workloads as W


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def dev(a, dtype=None):
    torch = torch_cuda()
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


def spherical_test_grid(hole=True, nphi=4):
    rw = np.array([0.3, 0.5, 0.9, 1.4, 2.0]) * W.AU if hole else np.array([0.0, 0.5, 0.9, 1.4, 2.0]) * W.AU
    tw = np.array([0.0, 0.4, 1.1, math.pi / 2, 2.2, math.pi])
    pw = np.array([0.0, 1.0, 2.5, 4.0, 2 * math.pi]) if nphi == 4 else np.array([0.0, 2 * math.pi])
    return [rw, tw, pw]


def workload_from_walls(grid_type, walls, rho=None, seed=21):
    shape = tuple(len(w) - 1 for w in walls)
    if rho is None:
        rng = np.random.default_rng(seed)
        rho = rng.uniform(0.5, 2.0, shape[::-1]).astype(np.float32) * 1e-18
    nu, chi, alb, g = W.dust_table()
    return W.Workload(name="walls", grid_type=grid_type, walls=[np.asarray(w, float) for w in walls], rho=rho,
                      nu=nu, chi=chi, albedo=alb, g=g, T_nodes=W.temperature_nodes(),
                      sources=[dict(pos=(0.0, 0.0, 0.0), L=W.LSUN, Teff=5800.0)],
                      obs_incl=np.radians([30.0]), obs_az=np.zeros(1), seed=seed)


def random_points_in_grid(om, n, rng, radius):
    """Points strictly inside the grid with their cells located by the oracle."""
    pts, dirs, cells = [], [], []
    out = np.zeros(3)
    c = np.zeros(3, np.int32)
    while len(pts) < n:
        p = rng.uniform(-radius, radius, 3)
        if om.gtype == 1 and np.linalg.norm(p) >= radius:
            continue
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        st = M.lib().or_locate(om._struct, M._ptr(p), M._ptr(u), M._ptr(out), M._ptr(c, M._ip))
        if st != 0 or not np.allclose(out, p):
            continue        # skip points in the hole (the locate moved them)
        pts.append(p.copy())
        dirs.append(u)
        cells.append(c.copy())
    return np.array(pts), np.array(dirs), np.array(cells, np.int32)


def points_in_shell(om, n, rng, r_lo, r_hi, cos_band=None, graze=None):
    """Points with r log-uniform in [r_lo, r_hi] and, with cos_band = c0, |cos theta| >= c0
    (the polar regions); directions isotropic, or with graze = g, inclined to the sphere
    through the point by less than g (|p.u| / |p| < g): rays grazing the spherical walls."""
    pts, dirs, cells = [], [], []
    out = np.zeros(3)
    c = np.zeros(3, np.int32)
    while len(pts) < n:
        r = math.exp(rng.uniform(math.log(r_lo), math.log(r_hi)))
        if cos_band is None:
            mu = rng.uniform(-1.0, 1.0)
        else:
            mu = math.copysign(rng.uniform(cos_band, 1.0), rng.uniform(-1.0, 1.0))
        ph = rng.uniform(0.0, 2.0 * math.pi)
        st = math.sqrt(max(0.0, 1.0 - mu * mu))
        rhat = np.array([st * math.cos(ph), st * math.sin(ph), mu])
        p = r * rhat
        if graze is None:
            u = rng.normal(size=3)
        else:
            t = rng.normal(size=3)
            t -= (t @ rhat) * rhat
            t /= np.linalg.norm(t)
            u = t + rng.uniform(-graze, graze) * rhat
        u /= np.linalg.norm(u)
        s = M.lib().or_locate(om._struct, M._ptr(p), M._ptr(u), M._ptr(out), M._ptr(c, M._ip))
        if s != 0 or not np.allclose(out, p):
            continue
        pts.append(p.copy())
        dirs.append(u)
        cells.append(c.copy())
    return np.array(pts), np.array(dirs), np.array(cells, np.int32)


def grid_scale(wl):
    """L0, the unit the library scales lengths by: the largest |wall| of a Cartesian grid, the
    outer radius of a spherical one, the largest |R| or |z| wall of a cylindrical one."""
    axes = {"cartesian": range(3), "spherical": range(1), "cylindrical": range(2)}[wl.grid_type]
    return max(max(abs(float(wl.walls[a][0])), abs(float(wl.walls[a][-1]))) for a in axes)


def as_device_sees(p, wl):
    """(FP32 positions in cm handed to the step hooks, FP64 positions in cm the oracle gets):
    the hooks scale by an FP32 1/L0, so the oracle is given that rounded position times L0."""
    L0 = grid_scale(wl)
    p32 = np.asarray(p, np.float64).astype(np.float32)
    seen = p32 * np.float32(1.0 / L0)          # FP32 product, rounded like the device's
    return p32, seen.astype(np.float64) * L0


def pixel_parity(img, ref, tol=1e-4):
    """Per-pixel agreement of two images of the same packets (lockstep): over the pixels lit in
    either, the fraction whose values differ by more than tol (relative to the larger), the median
    relative difference, and the summed |difference| relative to the summed reference."""
    import numpy as np
    img = np.asarray(img, np.float64)
    ref = np.asarray(ref, np.float64)
    lit = (img > 0) | (ref > 0)
    big = np.maximum(np.abs(img), np.abs(ref))[lit]
    rel = np.abs(img - ref)[lit] / big
    return {"lit": int(lit.sum()), "frac_off": float((rel > tol).mean()) if lit.any() else 0.0,
            "median_rel": float(np.median(rel)) if lit.any() else 0.0,
            "l1_rel": float(np.abs(img - ref).sum() / max(np.abs(ref).sum(), 1e-300))}
