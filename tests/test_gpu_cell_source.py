"""Diffuse (cell) sources (Sect. 2.1.1) on the GPU against the FP64 oracle (through the C ABI):
a cell picked in proportion to its luminosity, a point uniform in its volume, an isotropic
direction and the source's spectrum, drawn in the same order from the same Philox streams on
both sides, so whole iterations stay in lockstep; an imaging pass peels the emission off; an
empty grid seen face-on images each emitting cell as a filled rectangle."""
import math

import numpy as np
import pytest

from oracle import mc as M
from paper_1112_1071_gb300 import hrt
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import spherical_test_grid, workload_from_walls

pytestmark = pytest.mark.gpu

KERNELS = [hrt.HRT_KERNEL_PLAIN, hrt.HRT_KERNEL_EVENT, hrt.HRT_KERNEL_REGROUP]


def _walls(grid):
    if grid == "cartesian":
        return [np.linspace(-2, 2, 7) * W.AU, np.linspace(-1.5, 2, 6) * W.AU, np.linspace(-2, 1.5, 5) * W.AU]
    if grid == "spherical":
        return spherical_test_grid(hole=True, nphi=4)
    return [np.array([0.3, 0.5, 0.9, 1.4, 2.0]) * W.AU, np.array([-1.5, -0.4, 0.0, 0.3, 1.5]) * W.AU,
            np.array([0.0, 1.0, 2.5, 4.0, 2 * math.pi])]


def _model(grid, n_packets=100_000):
    """A star at the origin plus half a solar luminosity emitted by the cells in proportion to
    their dust mass (a 4000 K population embedded in the dust), tau_550 of 1-3 across the grid."""
    wl = workload_from_walls(grid, _walls(grid))
    om = M.OracleModel(wl)
    mass = om.rho * om.vol
    wl.cell_source = dict(L=0.5 * W.LSUN * mass / mass.sum(), Teff=4000.0)
    wl.n_packets = n_packets
    return wl


def _lockstep(m, st, om, ref):
    assert st["e_escaped"] + st["e_killed"] == pytest.approx(om.L_tot, rel=1e-12)
    acc = m.absorbed()
    seen = ref["acc"] > 0
    rel = np.abs(acc[seen] - ref["acc"][seen]) / ref["acc"][seen]
    assert np.median(rel) < 1e-4, np.median(rel)
    assert st["n_crossings"] == pytest.approx(ref["n_crossings"], rel=2e-3)
    assert st["n_interactions"] == pytest.approx(ref["n_interactions"], rel=2e-3)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("grid", ["cartesian", "spherical", "cylindrical"])
def test_cell_source_iterations_match_oracle(grid, kernel):
    wl = _model(grid)
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    for _ in range(2):
        st = m.run_iteration(kernel=kernel)
        ref = om.run_iteration(nthreads=16)
        _lockstep(m, st, om, ref)
        dT = np.abs(m.temperature() - ref["T"]) / ref["T"]
        assert dT.mean() < 3e-3


@pytest.mark.parametrize("kernel", KERNELS)
def test_cell_source_imaging_pass_matches_oracle(kernel):
    wl = _model("spherical", n_packets=50_000)
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    m.run_iteration(kernel=kernel)
    om.run_iteration(nthreads=16)
    m.run_iteration(kernel=kernel, peel=1, update_temperature=0)
    ref = om.run_iteration(peel=True, update=False, nthreads=16)
    sed, rs = m.sed(), ref["sed"]
    np.testing.assert_allclose(sed.sum(axis=1), rs.sum(axis=1), rtol=2e-3)
    big = rs > 1e-3 * rs.max()
    np.testing.assert_allclose(sed[big], rs[big], rtol=2e-2)


@pytest.mark.parametrize("kernel", KERNELS)
def test_face_on_image_of_emitting_cells_matches_oracle(kernel):
    a = 10 * W.AU
    walls = [np.array([-a, 0.0, a]), np.array([-a / 2, a / 2]), np.array([-a / 2, a / 2])]
    wl = workload_from_walls("cartesian", walls, rho=np.zeros((1, 1, 2), np.float32))
    wl.sources = []
    wl.cell_source = dict(L=np.array([1.0, 3.0]) * W.LSUN, Teff=5000.0)
    wl.obs_incl, wl.obs_az = np.array([0.0]), np.array([0.0])
    wl.nsed, wl.lam_min_um, wl.lam_max_um = 1, 0.05, 2000.0         # one bin holding the whole band
    wl.img_nx = wl.img_ny = 8
    wl.img_half_extent = a
    wl.img_lam_um = np.array([1.0])
    n = 80_000
    om = M.OracleModel(wl)
    ref = om.run_iteration(n_packets=n, peel=True, update=False, nthreads=16)
    m = hrt.Model(wl)
    st = m.run_iteration(n_packets=n, kernel=kernel, peel=1, update_temperature=0)
    assert st["e_escaped"] == pytest.approx(om.L_tot, rel=1e-12)
    w = om.L_tot / (4 * math.pi) / n                           # one packet's weight
    img, rimg = m.image()[0, 0], ref["img"][0, 0]
    # every packet lands in the image; the peel pass forms each weight in FP32 (bins are FP64)
    assert img.sum() == pytest.approx(om.L_tot / (4 * math.pi), rel=1e-6)
    hits, rhits = np.rint(img / w).astype(np.int64), np.rint(rimg / w).astype(np.int64)
    # the same packets on both sides: pixels differ only where an FP32 position sits on a pixel edge
    assert np.abs(hits - rhits).max() <= 3
    assert abs(hits[:4].sum() - rhits[:4].sum()) <= 3
