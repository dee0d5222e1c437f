"""Raytracing of point-source and dust emission (Sect. 2.6.3) on the GPU against the FP64 oracle.

Both sides hold the same temperatures; the dust rays draw from the same Philox streams (cell from
the emission CDF, point in the cell), so the rays coincide, and the columns to the grid edge
agree to FP32 walk rounding; the bin integrals differ only by quadrature order (3- against
8-point Gauss-Legendre per piece).  The packets of the same imaging pass are peeled off only at
scatterings on both sides."""
import math

import numpy as np
import pytest

from oracle import mc as M
from oracle import raytrace as RT
from paper_1112_1071_gb300 import hrt
from paper_1112_1071_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _compare(wl, T_field, n_packets, n_rays, kernel):
    m = hrt.Model(wl)
    m.set_temperature(T_field)
    st = m.run_iteration(n_packets=n_packets, kernel=kernel, peel=1, update_temperature=0, raytrace_rays=n_rays)
    om = M.OracleModel(wl)
    om.T = T_field.copy()
    ref = om.run_packets(n_packets, M.IMAGING_KEY, peel=True, raytrace=True, nthreads=16)
    sed_rt, img_rt, _ = RT.raytrace(om, n_rays, RT.RAYTRACE_KEY)
    want = ref["sed"] + sed_rt
    got = m.sed()
    np.testing.assert_allclose(got.sum(axis=1), want.sum(axis=1), rtol=2e-4)
    big = want > 1e-3 * want.max()
    np.testing.assert_allclose(got[big], want[big], rtol=2e-3)
    if om.nimg:
        wimg = ref["img"] + img_rt
        np.testing.assert_allclose(m.image().sum(axis=(2, 3)), wimg.sum(axis=(2, 3)), rtol=2e-3)
    return st, got


@pytest.mark.parametrize("kernel", [hrt.HRT_KERNEL_PLAIN, hrt.HRT_KERNEL_EVENT])
def test_raytraced_sphere_matches_oracle(kernel):
    wl = W.tiny_sphere(n_packets=2000)
    wl.img_nx = wl.img_ny = 32
    wl.img_half_extent = 100 * W.AU
    wl.img_lam_um = np.array([1.0, 24.0, 100.0])
    n = 32 ** 3
    rng = np.random.default_rng(5)
    T_field = rng.uniform(15.0, 80.0, n)
    _compare(wl, T_field, 2000, 20_000, kernel)


def test_raytraced_disk_matches_oracle():
    wl = W.flared_disk(n_packets=2000, n_r=80, n_theta=48)
    rw = wl.walls[0]
    rc = 0.5 * (rw[1:] + rw[:-1]) / rw[0]
    T_field = np.broadcast_to(np.clip(400.0 * rc ** -0.45, 8.0, 1500.0), (48, 80)).reshape(-1).copy()
    st, got = _compare(wl, T_field, 2000, 20_000, hrt.HRT_KERNEL_EVENT)
    assert st["n_peel_crossings"] > 0


def test_raytracing_needs_an_imaging_pass_and_valid_count():
    wl = W.tiny_sphere(n_packets=1000)
    m = hrt.Model(wl)
    with pytest.raises(hrt.HrtError):
        m.run_iteration(n_packets=1000, peel=1, update_temperature=0, raytrace_rays=-1)
    # in a Lucy iteration the setting is ignored (no SEDs are made)
    st = m.run_iteration(n_packets=1000, raytrace_rays=1000)
    assert st["e_escaped"] + st["e_killed"] == pytest.approx(st["e_emitted"], rel=1e-12)
