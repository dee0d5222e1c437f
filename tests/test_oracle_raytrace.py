"""Pins of the oracle's raytracing of source and dust emission (Sect. 2.6.3):

* an empty grid passes a point source's whole luminosity: sum over bins = L / 4 pi exactly (the
  quadrature is exact on the piecewise-constant spectrum);
* grey dust: a source at the centre of a uniform sphere of radial optical depth tau arrives
  attenuated by exactly exp(-tau) in every bin;
* grey dust in a uniform sphere of uniform temperature: the mean transmission of the emission
  is the escape probability of a uniform sphere, 3 / (8 tau^3) (2 tau^2 - 1 + (1 + 2 tau)
  exp(-2 tau)) (within the sampling error of the rays);
* rays pick cells in proportion to their emitted luminosity m E(T);
* an image that holds the whole object collects the SED bin of its wavelength.
"""
import math

import numpy as np
import pytest

from oracle import mc as M
from oracle import raytrace as RT
from oracle import tables as T
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import workload_from_walls


def _grey(wl, chi=1.0):
    wl.chi = np.full_like(wl.nu, chi)
    wl.albedo = np.zeros_like(wl.nu)
    return wl


def _sphere(tau, n_r=1, rho=1e-18):
    """Spherical grid without a hole, uniform density, grey dust with chi set for tau."""
    R = 100 * W.AU
    walls = [np.linspace(0, R, n_r + 1), np.array([0.0, math.pi]), np.array([0.0, 2 * math.pi])]
    wl = workload_from_walls("spherical", walls, rho=np.full((1, 1, n_r), rho, np.float32))
    return _grey(wl, chi=tau / (rho * R)), R


def test_empty_grid_passes_the_source_luminosity():
    wl = W.tiny_sphere(n_packets=10)
    wl.rho[:] = 0
    om = M.OracleModel(wl)
    om.struct(np.zeros(om.nc, np.int32))
    sed = np.zeros((om.nobs, wl.nsed))
    img = np.zeros((om.nobs, om.nimg, wl.img_ny, wl.img_nx))
    RT.sources(om, sed, img)
    np.testing.assert_allclose(sed.sum(axis=1) * 4 * math.pi, om.L_tot, rtol=1e-12)


def test_grey_sphere_source_attenuation():
    tau = 1.7
    wl, R = _sphere(tau)
    om = M.OracleModel(wl)
    om.struct(np.zeros(om.nc, np.int32))
    sed = np.zeros((om.nobs, wl.nsed))
    img = np.zeros((om.nobs, om.nimg, wl.img_ny, wl.img_nx))
    RT.sources(om, sed, img)
    # the unattenuated spectrum from an empty copy of the grid
    wl0, _ = _sphere(tau)
    wl0.rho[:] = 0
    om0 = M.OracleModel(wl0)
    om0.struct(np.zeros(om0.nc, np.int32))
    sed0 = np.zeros_like(sed)
    RT.sources(om0, sed0, np.zeros_like(img))
    big = sed0 > 1e-6 * sed0.max()
    tau_f32 = wl.chi[0] * float(om.rho[0]) * R       # the density is held in FP32
    np.testing.assert_allclose(sed[big] / sed0[big], math.exp(-tau_f32), rtol=1e-12)


@pytest.mark.parametrize("tau", [0.3, 2.0])
def test_uniform_sphere_escape_probability(tau):
    wl, R = _sphere(tau)
    om = M.OracleModel(wl)
    om.T = np.full(om.nc, 50.0)
    n = 20000
    sed, img, cells = RT.raytrace(om, n, RT.RAYTRACE_KEY)
    # remove the point source's share (its own exp(-tau) term) to keep the dust emission
    src = np.zeros_like(sed)
    om.struct(np.zeros(om.nc, np.int32))
    RT.sources(om, src, np.zeros_like(img))
    L_dust = float((om.rho * om.vol).sum() * T.interp_loglog(50.0, om.T_nodes, om.dust.E))
    got = (sed - src).sum(axis=1) * 4 * math.pi / L_dust
    want = 3 / (8 * tau ** 3) * (2 * tau ** 2 - 1 + (1 + 2 * tau) * math.exp(-2 * tau))
    # sampling error of the mean of exp(-tau_ray): below 0.5/sqrt(n)
    np.testing.assert_allclose(got, want, atol=4 * 0.5 / math.sqrt(n))


def test_rays_pick_cells_by_luminosity():
    walls = [np.linspace(0, 4 * W.AU, 3), np.linspace(0, 1 * W.AU, 2), np.linspace(0, 1 * W.AU, 2)]
    wl = _grey(workload_from_walls("cartesian", walls, rho=np.full((1, 1, 2), 1e-20, np.float32)))
    om = M.OracleModel(wl)
    om.T = np.array([30.0, 45.0])
    E = T.interp_loglog(om.T, om.T_nodes, om.dust.E)      # emission per gram at each T (Eq. 3)
    share = E[1] / E.sum()
    n = 8000
    _, _, cells = RT.raytrace(om, n, RT.RAYTRACE_KEY)
    frac = (cells == 1).mean()
    assert abs(frac - share) < 4 * math.sqrt(share * (1 - share) / n)


def test_image_holds_the_sed_bin():
    wl = W.tiny_sphere(n_packets=10)
    wl.img_nx = wl.img_ny = 16
    wl.img_half_extent = 101 * W.AU
    wl.img_lam_um = np.array([2.0, 100.0])
    om = M.OracleModel(wl)
    om.T = np.full(om.nc, 40.0)
    sed, img, _ = RT.raytrace(om, 3000, RT.RAYTRACE_KEY)
    for l, b in enumerate(om.img_bin):
        np.testing.assert_allclose(img[:, l].sum(axis=(1, 2)), sed[:, b], rtol=1e-12)
