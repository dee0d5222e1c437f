"""The learned warm start (task pattern 4) against the cold start, judged by the method itself.

A small network is trained here, by the library's own tensor-core kernels, on temperature
fields that the plain GPU iteration produced for seeded 32^3 clouds (log-normal density, 1-8
stars, mean 550 nm optical depth 100).  On held-out clouds, the iteration started from the
network's prediction is compared with the cold start from 10 K, with the same packets on the
same random streams; the Monte-Carlo iteration and its convergence test (Sect. 2.4, Eqs. 4-6)
decide.  What the warm start gains on such clouds is a better start: its first iteration changes
the field less (Q_99 of the iteration change) and ends closer to the converged temperatures than
the cold start's first iteration.  It never converges later, and both arms end on the same
temperatures (the warm start does not change the answer).  On these clouds the plain iteration
itself reaches its Monte-Carlo floor within three iterations, so both arms meet the Delta test
in about the same number of iterations."""
import ctypes as C

import pytest

from paper_1112_1071_gb300 import hrt, learned
from tests.gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

N, TAU = 32, 100.0


def test_warm_start_starts_closer_and_converges_to_the_same_temperatures():
    torch = torch_cuda()
    L = hrt.load()
    X, Y, _ = learned.generate(range(1000, 1064), N, 10_000_000, 5, TAU, torch)
    widths = (C.c_int * 3)(32, 64, 64)
    net = C.c_void_p()
    assert L.hrt_net_create_widths(C.byref(net), 0, C.cast(widths, C.c_void_p), 2, 7, None) == 0
    hist = learned.train(net, X, Y, 20, 2e-3, 8, torch)
    assert hist[-1] < 0.2 * hist[0]
    rows = learned.evaluate(net, [5000, 5001, 5002], N, 30_000_000, 6, TAU, torch, print)
    for r in rows:
        qc, qw = r["cold"]["q"], r["warm"]["q"]
        dc, dw = r["dist_to_converged"]["cold"], r["dist_to_converged"]["warm"]
        # the first iteration from the prediction changes the field less than from 10 K, and ends
        # closer to the converged temperatures
        assert qw[0] < qc[0], (qc, qw)
        assert dw[0] < dc[0], (dc, dw)
        ic = learned.converged_at(qc, 2.0, 1.02)
        iw = learned.converged_at(qw, 2.0, 1.02)
        assert ic is not None and iw is not None and iw <= ic, (qc, qw)
        # equal accuracy: the same packets on the same streams end on the same temperatures
        assert r["final_mean_dT_warm_vs_cold"] <= r["mc_noise_mean_dT"], r
    L.hrt_net_destroy(net)
