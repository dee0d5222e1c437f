"""The allocation-free quantile entry point, hrt_quantile_ratio_noalloc.

It serves callers of the library that cannot allocate device memory (a framework whose
allocator already owns the GPU's memory, or latency-bound code that cannot afford the
synchronisation cudaMalloc may impose).  Its answer must be the convergence quantile Q that
hrt_run_iteration reports for the same temperatures, exactly (both take the nearest-rank order
statistic of the same FP64 ratios), on consecutive calls that reuse its fixed scratch array.
This file is collected last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

from paper_1112_1071_gb300 import hrt
from paper_1112_1071_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_quantile_equals_iteration_quantile_on_consecutive_calls():
    import torch
    assert torch.cuda.is_available()
    L = hrt.load()
    wl = W.tiny_sphere(n_packets=50_000)
    m = hrt.Model(wl)
    nc = m.ncells
    rho = torch.as_tensor(np.ascontiguousarray(wl.rho.reshape(-1), dtype=np.float32)).cuda()
    prev = torch.empty(nc, dtype=torch.float64, device="cuda")
    cur = torch.empty(nc, dtype=torch.float64, device="cuda")
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    m.run_iteration()
    for call in range(2):
        hrt.check(m.ctx, L.hrt_get_temperature_device(m.ctx, prev.data_ptr(), nc))
        st = m.run_iteration()
        hrt.check(m.ctx, L.hrt_get_temperature_device(m.ctx, cur.data_ptr(), nc))
        rc = L.hrt_quantile_ratio_noalloc(nc, prev.data_ptr(), cur.data_ptr(), rho.data_ptr(), 0.99,
                                          out.data_ptr(), stream)
        assert rc == hrt.HRT_OK
        torch.cuda.synchronize()
        assert out.item() == st["Q"], (call, out.item(), st["Q"])


def test_noalloc_quantile_rejects_sizes_beyond_its_limit():
    import torch
    L = hrt.load()
    d = torch.ones(4, dtype=torch.float64, device="cuda")
    r = torch.ones(4, dtype=torch.float32, device="cuda")
    o = torch.empty(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert L.hrt_quantile_ratio_noalloc(0, d.data_ptr(), d.data_ptr(), r.data_ptr(), 0.5, o.data_ptr(), s) == hrt.HRT_EINVAL
    assert L.hrt_quantile_ratio_noalloc(2**31, d.data_ptr(), d.data_ptr(), r.data_ptr(), 0.5, o.data_ptr(), s) == hrt.HRT_EINVAL
    assert L.hrt_quantile_ratio_noalloc(4, d.data_ptr(), d.data_ptr(), r.data_ptr(), 1.5, o.data_ptr(), s) == hrt.HRT_EINVAL


def _nearest_rank(prev, cur, rho, p):
    """The statistic written out: nearest-rank p-quantile of max(a/b, b/a) over cells with rho > 0."""
    mask = rho > 0
    if not mask.any():
        return float("nan")
    r = np.sort(np.maximum(prev[mask] / cur[mask], cur[mask] / prev[mask]))
    k = min(max(int(np.ceil(p * r.size)) - 1, 0), r.size - 1)
    return float(r[k])


def _call(L, prev, cur, rho, p):
    import torch
    dp = torch.as_tensor(prev, device="cuda")
    dc = torch.as_tensor(cur, device="cuda")
    dr = torch.as_tensor(rho, device="cuda")
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    rc = L.hrt_quantile_ratio_noalloc(prev.size, dp.data_ptr(), dc.data_ptr(), dr.data_ptr(), p, out.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == hrt.HRT_OK
    torch.cuda.synchronize()
    return out.item()


def test_noalloc_quantile_edge_cases_and_stale_scratch():
    """No cell with dust gives NaN; p = 1 gives the largest ratio and a tiny p the smallest (the
    rank is clamped to the cells with dust); a large call followed by a smaller one on the same
    scratch still gives the nearest-rank answer of the second (nothing of the first remains)."""
    L = hrt.load()
    rng = np.random.default_rng(11)
    n_big, n_small = 300_000, 1_003
    prev = rng.uniform(5.0, 50.0, n_big)
    cur = prev * np.exp(rng.normal(0.0, 0.05, n_big))
    rho = np.where(rng.uniform(size=n_big) < 0.8, rng.uniform(0.1, 1.0, n_big), 0.0).astype(np.float32)
    assert np.isnan(_call(L, prev[:n_small], cur[:n_small], np.zeros(n_small, np.float32), 0.99))
    for p in (1.0, 1e-9, 0.5, 0.99):
        got = _call(L, prev, cur, rho, p)
        assert got == _nearest_rank(prev, cur, rho, p), p
    r = np.maximum(prev / cur, cur / prev)[rho > 0]
    assert _call(L, prev, cur, rho, 1.0) == r.max() and _call(L, prev, cur, rho, 1e-9) == r.min()
    for p in (0.99, 0.3):
        got = _call(L, prev[:n_small], cur[:n_small], rho[:n_small], p)
        assert got == _nearest_rank(prev[:n_small], cur[:n_small], rho[:n_small], p), p
