"""The library's host copy of a source's own spectrum (the header the device table builder and the
run's input check share) against the oracle's statement of it, and the check that rejects a
spectrum without flux in the dust band (CPU: the header is plain C++ outside nvcc)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import tables as T
from paper_1112_1071_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1112_1071_gb300", "csrc")

_SRC = r"""
#include "user_spectrum.h"
extern "C" double us_eval(double v, const double* x, const double* f, int n) { return hrt::user_spectrum(v, x, f, n); }
extern "C" int us_has_flux(const double* g, int ng, const double* x, const double* f, int n) {
    return hrt::user_spectrum_has_flux(g, ng, x, f, n) ? 1 : 0;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("us")
    src, so = d / "us.cpp", d / "libus.so"
    src.write_text(_SRC)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    L.us_eval.argtypes = [ctypes.c_double, dp, dp, ctypes.c_int]
    L.us_eval.restype = ctypes.c_double
    L.us_has_flux.argtypes = [dp, ctypes.c_int, dp, dp, ctypes.c_int]
    L.us_has_flux.restype = ctypes.c_int
    return L


def _p(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _grid():
    nu = W.dust_table()[0]
    k = np.arange(1000)
    g = nu[0] * (nu[-1] / nu[0]) ** (k / 999)
    g[0], g[-1] = nu[0], nu[-1]
    return g


def test_host_spectrum_matches_the_oracle(lib):
    rng = np.random.default_rng(2)
    x = np.sort(rng.uniform(1e12, 1e15, 9))
    f = rng.uniform(0.1, 5.0, 9)
    f[[2, 6]] = 0.0                                           # pieces next to zeros are straight lines
    xs, fs = np.ascontiguousarray(x), np.ascontiguousarray(f)
    vs = np.concatenate([rng.uniform(0.5e12, 1.2e15, 4000), x])
    for v in vs:
        got = lib.us_eval(float(v), _p(xs), _p(fs), len(x))
        want = T.user_spectrum_at(float(v), x, f)
        assert got == pytest.approx(want, rel=1e-13, abs=1e-300), v


def test_spectra_without_flux_in_the_band_are_caught(lib):
    g = np.ascontiguousarray(_grid())
    has = lambda x, f: lib.us_has_flux(_p(g), len(g), _p(np.asarray(x, float)), _p(np.asarray(f, float)), len(x))
    assert has([g[0] * 0.5, g[-1] * 2], [1.0, 1.0]) == 1                 # covers the band
    assert has([g[100] * 1.001, g[101] * 0.999], [1.0, 1.0]) == 0        # between two grid nodes
    assert has([g[-1] * 2, g[-1] * 3], [1.0, 1.0]) == 0                   # above the band
    assert has([g[10], g[20], g[30]], [0.0, 0.0, 0.0]) == 0               # no flux anywhere
    assert has([g[10], g[20], g[30]], [0.0, 1.0, 0.0]) == 1
    # the check is the oracle's CDF being defined
    for x, f in ([[g[100] * 1.001, g[101] * 0.999], [1.0, 1.0]], [[g[10], g[20], g[30]], [0.0, 1.0, 0.0]]):
        vals = np.array([T.user_spectrum_at(v, np.asarray(x), np.asarray(f)) for v in g])
        assert (vals.max() > 0) == bool(has(x, f))
