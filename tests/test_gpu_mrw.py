"""The modified random walk (Sect. 2.2) on the GPU against the FP64 oracle (through the C ABI):
the nearest-wall distance and the path-length solve step by step, then whole iterations on all
three grid types.

A step's sphere radius is the distance to the nearest wall, which depends on the position, so a
chain of steps amplifies rounding of the position (by about 1.2x per step on the cubes here):
FP32 and FP64 histories stay in lockstep through chains of a few steps and part after many
tens.  Models whose packets take ~5 steps each are therefore compared packet for packet (same
Philox streams: counts and per-cell deposits at the lockstep level), and models whose packets
take ~100 steps each are compared statistically (temperatures within the Monte-Carlo noise of
8000 packets, which is 1-2 % per cell)."""
import math

import numpy as np
import pytest

from oracle import mc as M
from paper_1112_1071_gb300 import hrt
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import as_device_sees, dev, random_points_in_grid, spherical_test_grid, torch_cuda
from tests.gpu_helpers import workload_from_walls
from tests.test_oracle_mrw import _grids

pytestmark = pytest.mark.gpu

KERNELS = [hrt.HRT_KERNEL_PLAIN, hrt.HRT_KERNEL_EVENT]


@pytest.mark.parametrize("name", list(_grids()))
def test_wall_distance_matches_oracle(name):
    torch = torch_cuda()
    gtype, walls, radius = _grids()[name]
    wl = workload_from_walls(gtype, walls)
    om = M.OracleModel(wl)
    om.struct(np.zeros(om.nc, np.int32))
    p, _, c = random_points_in_grid(om, 3000, np.random.default_rng(11), radius)
    p32, p = as_device_sees(p, wl)
    want = np.array([M.lib().or_wall_distance(om._struct, M._ptr(p[q]), M._ptr(c[q], M._ip)) for q in range(len(p))])
    m = hrt.Model(wl)
    out = torch.empty(len(p), dtype=torch.float32, device="cuda")
    pd, cd = dev(p32), dev(c)
    m.step("hrt_step_wall_distance", len(p), pd.data_ptr(), cd.data_ptr(), out.data_ptr())
    got = out.cpu().numpy().astype(np.float64)
    # FP32 positions: the distance is good to a few ulps of |p|
    tol = 1e-5 * want + 8 * 2.0 ** -24 * np.linalg.norm(p, axis=1)
    assert (np.abs(got - want) <= tol).all(), np.max(np.abs(got - want) / tol)


def test_mrw_path_matches_oracle():
    torch = torch_cuda()
    rng = np.random.default_rng(5)
    n = 20000
    tau0 = np.exp(rng.uniform(math.log(1.0), math.log(1e4), n)).astype(np.float32)
    # the library's uniforms ((x >> 8) + 1) 2^-24, including both ends of (0, 1]
    zeta = ((rng.integers(0, 2 ** 24, n) + 1) * 2.0 ** -24).astype(np.float32)
    zeta[:3] = [2.0 ** -24, 1.0 - 2.0 ** -24, 1.0]
    want = np.array([M.lib().or_mrw_path(float(t), float(z)) for t, z in zip(tau0, zeta)])
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    t_d, z_d = dev(tau0), dev(zeta)
    hrt.check(None, hrt.load().hrt_step_mrw_path(n, t_d.data_ptr(), z_d.data_ptr(), out.data_ptr(), None))
    got = out.cpu().numpy().astype(np.float64)
    assert got[2] == 0.0 and want[2] == 0.0
    np.testing.assert_allclose(got, want, rtol=2e-6)


def _thick(kind, n_packets=3000):
    """Optically thick models whose cells are many transport mean free paths across: the grey
    models of the workloads module, and a non-grey cube (the synthetic dust, thick at the
    temperatures reached: chi_t and kappa_P vary with T)."""
    if kind != "nongrey":
        return W.thick_grey(kind, n_packets)
    w = np.linspace(-100 * W.AU, 100 * W.AU, 5)
    wl = workload_from_walls("cartesian", [w, w.copy(), w.copy()], rho=np.ones((4, 4, 4), np.float32))
    wl.sources = [dict(pos=(W.AU, 2 * W.AU, 3 * W.AU), L=W.LSUN, Teff=5800.0)]
    wl.rho[:] = np.float32(1e5 / (W.chi_at_lambda_um(0.55) * 50 * W.AU))
    wl.n_packets = n_packets
    return wl


def _moderate(kind, n_packets=3000):
    """Cells of 3-6 extinction mean free paths: with gamma = 1 (2 for the non-grey model) the
    packets take ~5 MRW steps each, short chains that stay in lockstep."""
    if kind == "nongrey":
        return _thick(kind, n_packets), 2.0
    return W.thick_grey(kind, n_packets, tau_cell=6.0 if kind == "cartesian" else 3.0), 1.0


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("kind", ["cartesian", "spherical", "cylindrical", "nongrey"])
def test_mrw_iterations_match_oracle_in_lockstep(kind, kernel):
    wl, gamma = _moderate(kind)
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    for it in range(2):
        st = m.run_iteration(kernel=kernel, mrw_gamma=gamma)
        ref = om.run_iteration(nthreads=16, mrw_gamma=gamma)
        if it == 1 or kind != "nongrey":        # the non-grey dust is thick only once warm
            assert ref["n_mrw"] > 1000
        assert st["e_escaped"] + st["e_killed"] == pytest.approx(om.L_tot, rel=1e-12)
        assert st["n_mrw"] == pytest.approx(ref["n_mrw"], rel=1e-3)
        assert st["n_interactions"] == pytest.approx(ref["n_interactions"], rel=1e-3)
        acc = m.absorbed()
        seen = ref["acc"] > 0
        rel = np.abs(acc[seen] - ref["acc"][seen]) / ref["acc"][seen]
        assert np.median(rel) < 1e-4, np.median(rel)
        dT = np.abs(m.temperature() - ref["T"]) / ref["T"]
        assert dT.mean() < 1e-3


_THICK_REF = {}


def _thick_reference(kind):
    if kind not in _THICK_REF:
        wl = _thick(kind, n_packets=8000)
        om = M.OracleModel(wl)
        _THICK_REF[kind] = (wl, om, om.run_iteration(nthreads=16, mrw_gamma=2.0))
    return _THICK_REF[kind]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("kind", ["cartesian", "spherical", "cylindrical"])
def test_mrw_thick_models_match_oracle_statistically(kind, kernel):
    wl, om, ref = _thick_reference(kind)
    m = hrt.Model(wl)
    st = m.run_iteration(kernel=kernel, mrw_gamma=2.0)
    assert ref["n_mrw"] > 50 * wl.n_packets                   # long chains: ~100 steps per packet
    assert st["e_escaped"] + st["e_killed"] == pytest.approx(om.L_tot, rel=1e-12)
    assert st["e_killed"] == 0
    # totals of heavy-tailed per-packet counts: within 3 %
    assert st["n_mrw"] == pytest.approx(ref["n_mrw"], rel=0.03)
    assert st["n_interactions"] == pytest.approx(ref["n_interactions"], rel=0.03)
    d = (m.temperature() - ref["T"]) / ref["T"]
    assert np.abs(d).mean() < 0.02 and np.percentile(np.abs(d), 95) < 0.05 and abs(d.mean()) < 0.01


@pytest.mark.parametrize("kernel", KERNELS)
def test_mrw_imaging_pass_matches_oracle(kernel):
    wl, gamma = _moderate("spherical", n_packets=3000)
    om = M.OracleModel(wl)
    m = hrt.Model(wl)
    m.run_iteration(kernel=kernel, mrw_gamma=gamma)
    om.run_iteration(nthreads=16, mrw_gamma=gamma)
    st = m.run_iteration(kernel=kernel, peel=1, update_temperature=0, mrw_gamma=gamma)
    ref = om.run_iteration(peel=True, update=False, nthreads=16, mrw_gamma=gamma)
    assert ref["n_mrw"] > 1000
    assert st["n_mrw"] == pytest.approx(ref["n_mrw"], rel=1e-3)
    sed, rs = m.sed(), ref["sed"]
    np.testing.assert_allclose(sed.sum(axis=1), rs.sum(axis=1), rtol=2e-3)
    big = rs > 1e-3 * rs.max()
    np.testing.assert_allclose(sed[big], rs[big], rtol=2e-2)


def test_mrw_argument_checks():
    wl = _thick("cartesian", n_packets=1000)
    m = hrt.Model(wl)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(hrt.HrtError):
            m.run_iteration(mrw_gamma=bad)
    st = m.run_iteration(mrw_gamma=0.0)
    assert st["n_mrw"] == 0
