"""Single-step parity of the CUDA kernels with the FP64 oracle, element by element on the same
inputs and uniform deviates (through the C ABI).  Tolerance: 1e-5 relative with an absolute
floor of 1e-5 x the cell size for distances, as stated for the single steps of the method;
FP64 steps (tables, temperature inversion) to 1e-12; integers (Philox words) bit-exact."""
import math

import numpy as np
import pytest

from oracle import mc as M
from oracle import tables as T
from paper_1112_1071_gb300 import hrt
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import (as_device_sees, dev, points_in_shell, random_points_in_grid, spherical_test_grid,
                               torch_cuda, workload_from_walls)

pytestmark = pytest.mark.gpu


def test_philox_words_bit_exact():
    torch = torch_cuda()
    rng = np.random.default_rng(0)
    n = 100_003
    ctr = rng.integers(0, 2**32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]]
    key[:3] = [[0, 0], [0xFFFFFFFF] * 2, [0xA4093822, 0x299F31D0]]
    c = dev(ctr.view(np.int32))
    k = dev(key.view(np.int32))
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    lib = hrt.load()
    assert lib.hrt_step_philox(n, c.data_ptr(), k.data_ptr(), out.data_ptr(), None) == 0
    got = out.cpu().numpy().view(np.uint32)
    for i in list(range(3)) + list(rng.integers(3, n, 300)):
        assert list(got[i]) == M.philox4x32_10(ctr[i], key[i])


@pytest.mark.parametrize("kind", ["cartesian", "spherical_hole_phi", "spherical_disk", "disk_inner_rim",
                                  "disk_polar", "disk_grazing"])
def test_cell_exit_matches_oracle(kind):
    """Random rays; the disk cases also sample the regions where the FP32 solves are most
    exposed: the first shells outside the inner hole, the polar cones, and rays inclined by
    less than 2 % to the spheres (grazing the inner sphere and the cones)."""
    torch = torch_cuda()
    rng = np.random.default_rng(1)
    if kind == "cartesian":
        wl = W.tiny_sphere()
        radius = 99.0 * W.AU
    elif kind == "spherical_hole_phi":
        wl = workload_from_walls("spherical", spherical_test_grid())
        radius = 1.99 * W.AU
    else:
        wl = W.flared_disk(n_r=50, n_theta=64)
        radius = 990 * W.AU
    om = M.OracleModel(wl)
    om.struct(np.zeros(om.nc, np.int32))
    r_in = wl.walls[0][0]
    if kind == "disk_inner_rim":
        p, u, c = points_in_shell(om, 4000, rng, r_in, 1.5 * r_in)
    elif kind == "disk_polar":
        p, u, c = points_in_shell(om, 4000, rng, r_in, 0.99 * wl.walls[0][-1], cos_band=math.cos(0.15))
    elif kind == "disk_grazing":
        p, u, c = points_in_shell(om, 4000, rng, r_in, 0.99 * wl.walls[0][-1], graze=0.02)
    else:
        p, u, c = random_points_in_grid(om, 4000, rng, radius)
    # both sides see the same inputs: FP32 directions, and the scaled FP32 position the device
    # computes from the FP32 cm position it is given
    p32, p = as_device_sees(p, wl)
    u = u.astype(np.float32).astype(np.float64)
    want = np.empty(len(p))
    want_ax = np.empty(len(p), np.int32)
    a = np.zeros(1, np.int32)
    d = np.zeros(1, np.int32)
    for q in range(len(p)):
        want[q] = M.lib().or_cell_exit(om._struct, M._ptr(p[q]), M._ptr(u[q]), M._ptr(c[q], M._ip),
                                       M._ptr(a, M._ip), M._ptr(d, M._ip))
        want_ax[q] = a[0] * 2 + (1 if d[0] > 0 else 0)
    m = hrt.Model(wl)
    dist = torch.empty(len(p), dtype=torch.float32, device="cuda")
    ex = torch.empty(len(p), dtype=torch.int32, device="cuda")
    pd, ud, cd = dev(p32), dev(u.astype(np.float32)), dev(c)
    m.step("hrt_step_cell_exit", len(p), pd.data_ptr(), ud.data_ptr(), cd.data_ptr(), dist.data_ptr(), ex.data_ptr())
    got = dist.cpu().numpy().astype(np.float64)
    gax = ex.cpu().numpy()
    # cell size scale for the absolute floor
    if wl.grid_type == "cartesian":
        size = np.diff(wl.walls[0]).min()
    else:
        r = np.linalg.norm(p, axis=1)
        size = np.maximum(r * 1e-3, np.diff(wl.walls[0]).min())
    # 1e-5 relative, plus 1e-5 of the cell size and four FP32 ulps of the position for exits
    # that approach zero length; rays grazing a cone at a small angle amplify the FP32
    # rounding of the quadratic, so up to 0.4% of random rays may exceed it
    tol = 1e-5 * np.abs(want) + 1e-5 * size + 2.4e-7 * np.linalg.norm(p, axis=1)
    bad = np.abs(got - want) > tol
    assert bad.mean() < 4e-3, (kind, np.flatnonzero(bad)[:5], got[bad][:5], want[bad][:5])
    assert (np.abs(got - want) > 20 * tol).mean() < 5e-4
    agree = gax == want_ax
    assert agree.mean() > 0.998


@pytest.mark.parametrize("kind", ["cartesian", "spherical_disk"])
def test_tau_to_edge_matches_oracle(kind):
    torch = torch_cuda()
    rng = np.random.default_rng(2)
    wl = W.tiny_sphere() if kind == "cartesian" else W.flared_disk(n_r=60, n_theta=64)
    radius = 99 * W.AU if kind == "cartesian" else 990 * W.AU
    om = M.OracleModel(wl)
    om.struct(np.zeros(om.nc, np.int32))
    p, u, _ = random_points_in_grid(om, 3000, rng, radius)
    p32, p = as_device_sees(p, wl)
    u = u.astype(np.float32).astype(np.float64)
    nus = np.exp(rng.uniform(np.log(wl.nu[0]), np.log(wl.nu[-1]), len(p))).astype(np.float32).astype(np.float64)
    want = np.empty(len(p))
    for q in range(len(p)):
        chi, _ = _oracle_dust(om, nus[q])
        want[q] = M.lib().or_tau_to_edge(om._struct, M._ptr(p[q]), M._ptr(u[q]), chi)
    m = hrt.Model(wl)
    tau = torch.empty(len(p), dtype=torch.float32, device="cuda")
    pd, ud, nd = dev(p32), dev(u.astype(np.float32)), dev(nus.astype(np.float32))
    m.step("hrt_step_tau_to_edge", len(p), pd.data_ptr(), ud.data_ptr(), nd.data_ptr(), tau.data_ptr())
    got = tau.cpu().numpy().astype(np.float64)
    tol = 2e-5 * np.abs(want) + 1e-6
    bad = np.abs(got - want) > tol
    assert bad.mean() < 2e-3, (np.flatnonzero(bad)[:5], got[bad][:5], want[bad][:5])


def _oracle_dust(om, nu):
    lnu = np.log(om.nu)
    j = int(np.clip(np.searchsorted(om.nu, nu, side="right") - 1, 0, len(om.nu) - 2))
    t = (math.log(nu) - lnu[j]) / (lnu[j + 1] - lnu[j])
    chi = math.exp((1 - t) * math.log(om.chi[j]) + t * math.log(om.chi[j + 1]))
    alb = (1 - t) * om.albedo[j] + t * om.albedo[j + 1]
    return chi, alb


def test_hg_scatter_matches_oracle():
    torch = torch_cuda()
    rng = np.random.default_rng(3)
    n = 20000
    u = rng.normal(size=(n, 3))
    u[::97] = [1e-4, 2e-4, 1.0]
    u /= np.linalg.norm(u, axis=1)[:, None]
    u = u.astype(np.float32).astype(np.float64)
    u1 = W.uniforms(n, rng)
    u2 = W.uniforms(n, rng)
    m = hrt.Model(W.tiny_sphere())
    out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    ud, a, b = dev(u.astype(np.float32)), dev(u1.astype(np.float32)), dev(u2.astype(np.float32))
    m.step("hrt_step_hg_scatter", n, ud.data_ptr(), a.data_ptr(), b.data_ptr(), out.data_ptr())
    got = out.cpu().numpy()
    for q in range(n):
        want = M.scatter_dir(u[q], M.hg_mu(0.6, u1[q]), 2 * math.pi * u2[q])
        assert np.abs(got[q] - want).max() < 2e-5, (q, got[q], want)


def test_frequency_sampling_matches_oracle():
    torch = torch_cuda()
    rng = np.random.default_rng(4)
    wl = W.tiny_sphere()
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    n = 20000
    rows = rng.integers(0, len(wl.T_nodes), n).astype(np.int32)
    us = W.uniforms(n, rng)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    rd, ud = dev(rows), dev(us.astype(np.float32))
    m.step("hrt_step_sample_emission", n, rd.data_ptr(), ud.data_ptr(), out.data_ptr())
    got = out.cpu().numpy()
    want = np.array([M.sample_table(om.nu, om.cdf_emit[rows[q]], us[q]) for q in range(n)])
    rel = np.abs(got - want) / want
    # the device row is FP32: a draw landing within one FP32 ulp of a node may pick the
    # neighbouring interval, which moves nu by far less than an interval but more than 1e-5
    assert (rel > 1e-5).mean() < 1e-3 and np.median(rel) < 1e-6
    # source spectrum
    srcs = np.zeros(n, np.int32)
    out2 = torch.empty(n, dtype=torch.float32, device="cuda")
    sd = dev(srcs)
    m.step("hrt_step_sample_source", n, sd.data_ptr(), ud.data_ptr(), out2.data_ptr())
    got = out2.cpu().numpy()
    want = np.array([M.sample_table(om.spec_nu, om.spec_cdf[0], us[q]) for q in range(n)])
    rel = np.abs(got - want) / want
    assert (rel > 1e-5).mean() < 1e-3 and np.median(rel) < 1e-6


def test_tables_and_temperature_inversion_fp64():
    torch = torch_cuda()
    wl = W.tiny_sphere()
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    E, cdf = m.tables()
    np.testing.assert_allclose(E, om.dust.E, rtol=1e-12)
    np.testing.assert_allclose(cdf, om.dust.cdf, atol=2e-7)
    rng = np.random.default_rng(5)
    A = np.exp(rng.uniform(np.log(E[0]) - 1, np.log(E[-1]) + 1, 50000))
    A[:3] = [E[0], E[10], E[-1]]
    out = torch.empty(len(A), dtype=torch.float64, device="cuda")
    Ad = dev(A)
    m.step("hrt_step_temperature", len(A), Ad.data_ptr(), out.data_ptr())
    want, _, _ = T.temperature_from_adot(A, om.T_nodes, om.dust.E)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-12)


def test_ray_tangent_to_a_sphere_wall_terminates():
    # a peel ray from a point on the sphere r_15 of the disk grid, exactly perpendicular to the
    # radius there: in FP32 it must not cross the wall back and forth
    torch = torch_cuda()
    wl = W.flared_disk()
    L0 = wl.walls[0][-1]
    r15 = wl.walls[0][15] / L0
    u = np.array([0.526783, 0.0, 0.85])
    u /= np.linalg.norm(u)
    v = np.array([-u[2], 0.0, u[0]])                   # perpendicular to u in the x-z plane
    q = np.array([0.0, 1.0, 0.0])
    rng = np.random.default_rng(6)
    pts, dirs = [], []
    for k in range(256):
        a = rng.uniform(0, 2 * np.pi)
        rad = np.cos(a) * v + np.sin(a) * q                # radius direction perpendicular to u
        pts.append(rad * r15 * L0)
        dirs.append(u)
    p = np.array(pts).astype(np.float32)
    d = np.array(dirs).astype(np.float32)
    om = M.OracleModel(wl)
    om.struct(np.zeros(om.nc, np.int32))
    m = hrt.Model(wl)
    nus = np.full(len(p), 3e14, np.float32)
    tau = torch.empty(len(p), dtype=torch.float32, device="cuda")
    pd, ud, nd = dev(p), dev(d), dev(nus)
    m.step("hrt_step_tau_to_edge", len(p), pd.data_ptr(), ud.data_ptr(), nd.data_ptr(), tau.data_ptr())
    got = tau.cpu().numpy()
    chi, _ = _oracle_dust(om, 3e14)
    want = np.array([M.lib().or_tau_to_edge(om._struct, M._ptr(p[k].astype(np.float64)),
                                            M._ptr(d[k].astype(np.float64)), chi) for k in range(len(p))])
    assert np.all(np.isfinite(got))
    # rays that start on a wall and graze it are ill-conditioned in FP32: 1e-3 here
    np.testing.assert_allclose(got, want, rtol=1e-3, atol=1e-6)
