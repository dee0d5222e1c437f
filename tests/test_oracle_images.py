"""Pins of the oracle's peel-off images (Sect. 2.6.2): a point source in an empty grid is imaged,
by every packet's peel-off at emission, into one pixel that holds L / 4 pi, at the projection of
the source onto the sky plane: its distance from the image centre is the source's distance from
the line of sight through the origin, |p - (p.n) n|, for any observer direction n; and for the
observer on +z at azimuth 0 the sky axes are e_x = +y, e_y = -x.  For inclined observers the lit
pixel holds the source's coordinates along e_x (horizontal, at azimuth + 90 degrees) and
e_y = n x e_x, written out here from that convention."""
import math

import numpy as np
import pytest

from oracle import mc as M
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import workload_from_walls

AU = W.AU


def _image_of_point(p_au, incl, az, half_au=10.0, npix=200, n=2000):
    walls = [np.array([-half_au, half_au]) * AU] * 3
    wl = workload_from_walls("cartesian", [w.copy() for w in walls], rho=np.zeros((1, 1, 1), np.float32))
    wl.sources = [dict(pos=tuple(float(v) * AU for v in p_au), L=W.LSUN, Teff=5000.0)]
    wl.obs_incl, wl.obs_az = np.array([incl]), np.array([az])
    wl.nsed, wl.lam_min_um, wl.lam_max_um = 1, 0.05, 2000.0
    wl.img_nx = wl.img_ny = npix
    wl.img_half_extent = half_au * AU
    wl.img_lam_um = np.array([1.0])
    om = M.OracleModel(wl)
    out = om.run_packets(n, 0, peel=True, nthreads=4)
    return om, out["img"][0, 0], out["sed"][0]


@pytest.mark.parametrize("incl,az", [(0.0, 0.0), (0.4, 1.1), (1.2, -2.0), (math.pi / 2, 0.3), (2.5, 4.0)])
def test_point_source_images_at_its_sky_projection(incl, az):
    p = np.array([3.13, -2.37, 4.21])                 # off the pixel edges
    om, img, sed = _image_of_point(p, incl, az)
    L4 = om.L_tot / (4 * math.pi)
    assert sed.sum() == pytest.approx(L4, rel=1e-12)
    nz = np.argwhere(img > 0)
    assert len(nz) == 1
    iy, ix = nz[0]
    assert img[iy, ix] == pytest.approx(L4, rel=1e-12)
    pix = 20.0 / 200                                              # AU per pixel
    cx, cy = -10.0 + (ix + 0.5) * pix, -10.0 + (iy + 0.5) * pix  # pixel centre on the sky (AU)
    n = np.array([math.sin(incl) * math.cos(az), math.sin(incl) * math.sin(az), math.cos(incl)])
    d = np.linalg.norm(p - p.dot(n) * n)
    assert abs(math.hypot(cx, cy) - d) <= pix * math.sqrt(0.5) + 1e-9
    # the lit pixel holds the source's sky coordinates in the stated basis: e_x horizontal,
    # perpendicular to n (azimuth + 90 degrees), e_y = n x e_x; (e_x, e_y, n) is right-handed, so
    # a rotated or mirrored sky basis puts the source in another pixel
    ex = np.array([math.cos(az + math.pi / 2), math.sin(az + math.pi / 2), 0.0])
    ey = np.cross(n, ex)
    assert np.allclose(np.cross(ex, ey), n, atol=1e-12) and abs(ex @ n) < 1e-12
    sx, sy = float(p @ ex), float(p @ ey)
    assert -10.0 + ix * pix <= sx < -10.0 + (ix + 1) * pix, (sx, ix)
    assert -10.0 + iy * pix <= sy < -10.0 + (iy + 1) * pix, (sy, iy)


@pytest.mark.parametrize("incl,az", [(0.7, 0.9), (2.2, -1.3)])
def test_image_orientation_follows_the_source(incl, az):
    """Moving the source along the sky axis e_x moves its pixel along +x only; along e_y, +y only."""
    n = np.array([math.sin(incl) * math.cos(az), math.sin(incl) * math.sin(az), math.cos(incl)])
    ex = np.array([-math.sin(az), math.cos(az), 0.0])
    ey = np.cross(n, ex)
    p0 = np.array([0.93, -1.37, 1.21])
    pix0 = np.argwhere(_image_of_point(p0, incl, az, n=200)[1] > 0)[0]
    pxs = np.argwhere(_image_of_point(p0 + 2.0 * ex, incl, az, n=200)[1] > 0)[0]
    pys = np.argwhere(_image_of_point(p0 + 2.0 * ey, incl, az, n=200)[1] > 0)[0]
    assert pxs[0] == pix0[0] and pxs[1] == pix0[1] + 20            # 2 AU = 20 pixels along +x
    assert pys[1] == pix0[1] and pys[0] == pix0[0] + 20            # and along +y


def test_sky_axes_of_the_face_on_observer():
    p = np.array([3.13, -2.37, 4.21])                 # off the pixel edges
    _, img, _ = _image_of_point(p, 0.0, 0.0)
    iy, ix = np.argwhere(img > 0)[0]
    pix = 0.1
    assert -10.0 + ix * pix <= p[1] < -10.0 + (ix + 1) * pix      # e_x = +y
    assert -10.0 + iy * pix <= -p[0] < -10.0 + (iy + 1) * pix     # e_y = n x e_x = -x
