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
