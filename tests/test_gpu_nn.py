"""Learned warm start on the GPU (through the C ABI) against the FP64 network oracle.

The kernels take BF16 inputs and weights and accumulate in FP32, so the oracle is evaluated
on the same BF16-rounded numbers; outputs stored in BF16 are compared to a few BF16 ulps, FP32
reductions (weight and bias gradients) to 1e-3."""
import ctypes as C

import numpy as np
import pytest

from oracle import nn as N
from paper_1112_1071_gb300 import hrt
from paper_1112_1071_gb300 import workloads as W
from tests.gpu_helpers import dev, torch_cuda

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round float32 values to BF16 (nearest even) and back."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def close(got, want, rel):
    scale = np.sqrt(np.mean(want ** 2)) + 1e-30
    err = np.abs(got - want)
    assert np.all(err <= rel * np.abs(want) + rel * scale), (err.max(), scale)


@pytest.mark.parametrize("cin,cout,relu", [(32, 64, 1), (16, 32, 0), (64, 32, 1), (64, 128, 1), (48, 96, 0)])
def test_conv3d_forward_matches_oracle(cin, cout, relu):
    torch = torch_cuda()
    rng = np.random.default_rng(cin + cout)
    n, d, h, w = 2, 6, 8, 10
    x = bf16(rng.normal(size=(n, d, h, w, cin)))
    wt = bf16(rng.normal(size=(3, 3, 3, cin, cout)) / np.sqrt(27 * cin))
    b = rng.normal(size=cout).astype(np.float32).astype(np.float64)
    y = torch.empty((n, d, h, w, cout), dtype=torch.float32, device="cuda")
    L = hrt.load()
    xd, wd, bd = dev(x.astype(np.float32)), dev(wt.astype(np.float32)), dev(b.astype(np.float32))
    assert L.hrt_nn_conv3d(n, d, h, w, cin, cout, xd.data_ptr(), wd.data_ptr(), bd.data_ptr(), relu, y.data_ptr(),
                           None) == 0
    got = y.cpu().numpy().astype(np.float64)
    for s in range(n):
        ref = N.conv3d(x[s], wt, b)
        if relu:
            ref = np.maximum(ref, 0)
        close(got[s], ref, 8e-3)      # one BF16 rounding of the output


@pytest.mark.parametrize("cin,cout", [(32, 64), (64, 128), (96, 32), (192, 64), (32, 192)])
def test_conv3d_backward_matches_oracle(cin, cout):
    # weight gradients on tcgen05 in brick form: output channels in the MMA's rows (32 -> 64,
    # 64 -> 128; 32 -> 192 in two blocks, the second with 64 real rows) or input channels (96 -> 32,
    # 192 -> 64 in two blocks); the network's first layer (16 input channels) runs the stacked-tap
    # kernel and is checked in the network gradient test
    torch = torch_cuda()
    rng = np.random.default_rng(7)
    n, d, h, w = 2, 4, 6, 8
    x = bf16(rng.normal(size=(n, d, h, w, cin)))
    wt = bf16(rng.normal(size=(3, 3, 3, cin, cout)) / np.sqrt(27 * cin))
    g = bf16(rng.normal(size=(n, d, h, w, cout)))
    L = hrt.load()
    dx = torch.empty((n, d, h, w, cin), dtype=torch.float32, device="cuda")
    dw = torch.empty((27, cin, cout), dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    xd, wd, gd = dev(x.astype(np.float32)), dev(wt.astype(np.float32)), dev(g.astype(np.float32))
    assert L.hrt_nn_conv3d_backward(n, d, h, w, cin, cout, xd.data_ptr(), wd.data_ptr(), gd.data_ptr(), dx.data_ptr(),
                                    dw.data_ptr(), db.data_ptr(), None) == 0
    rdx, rdw, rdb = np.zeros(x.shape), np.zeros(wt.shape), np.zeros(cout)
    for s in range(n):
        a, bw, c = N.conv3d_backward(x[s], wt, g[s])
        rdx[s] = a
        rdw += bw
        rdb += c
    close(dx.cpu().numpy().astype(np.float64), rdx, 8e-3)
    close(dw.cpu().numpy().reshape(wt.shape).astype(np.float64), rdw, 1e-3)
    close(db.cpu().numpy().astype(np.float64), rdb, 1e-3)


# Sizes that span several 16 x 8-voxel bricks per plane and a ragged tail in x and y, so that
# interior halos between bricks, many blocks per plane and (weight gradient) the split of the
# voxels over many blocks with FP32 atomics are all exercised; the last three have more output
# tiles than the GPU has SMs, so persistent blocks run several tiles each.  The first two: a grid
# one tile wide (W <= 8: one tile per work item) and W = 17 (the last pair of tiles holds one
# column).
MULTI_BRICK = [((2, 5, 7, 6), 32, 64), ((1, 4, 16, 17), 32, 32),
               ((1, 4, 18, 34), 32, 32), ((2, 8, 32, 32), 64, 32), ((2, 8, 32, 32), 16, 32),
               ((1, 6, 20, 36), 32, 128), ((2, 8, 32, 64), 32, 64), ((1, 6, 20, 36), 64, 192),
               ((3, 9, 33, 41), 16, 32)]


@pytest.mark.parametrize("shape,cin,cout", MULTI_BRICK)
def test_conv3d_forward_multi_brick_matches_oracle(shape, cin, cout):
    torch = torch_cuda()
    n, d, h, w = shape
    rng = np.random.default_rng(d * h + cin)
    x = bf16(rng.normal(size=(n, d, h, w, cin)))
    wt = bf16(rng.normal(size=(3, 3, 3, cin, cout)) / np.sqrt(27 * cin))
    b = rng.normal(size=cout).astype(np.float32).astype(np.float64)
    y = torch.empty((n, d, h, w, cout), dtype=torch.float32, device="cuda")
    L = hrt.load()
    xd, wd, bd = dev(x.astype(np.float32)), dev(wt.astype(np.float32)), dev(b.astype(np.float32))
    assert L.hrt_nn_conv3d(n, d, h, w, cin, cout, xd.data_ptr(), wd.data_ptr(), bd.data_ptr(), 1, y.data_ptr(),
                           None) == 0
    got = y.cpu().numpy().astype(np.float64)
    for s in range(n):
        close(got[s], np.maximum(N.conv3d(x[s], wt, b), 0), 8e-3)


@pytest.mark.parametrize("shape,cin,cout", [((1, 4, 18, 34), 32, 32), ((2, 8, 32, 32), 64, 32),
                                            ((2, 8, 32, 32), 32, 64)])
def test_conv3d_backward_multi_brick_matches_oracle(shape, cin, cout):
    torch = torch_cuda()
    n, d, h, w = shape
    rng = np.random.default_rng(d * w + cout)
    x = bf16(rng.normal(size=(n, d, h, w, cin)))
    wt = bf16(rng.normal(size=(3, 3, 3, cin, cout)) / np.sqrt(27 * cin))
    g = bf16(rng.normal(size=(n, d, h, w, cout)))
    L = hrt.load()
    dx = torch.empty((n, d, h, w, cin), dtype=torch.float32, device="cuda")
    dw = torch.empty((27, cin, cout), dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    xd, wd, gd = dev(x.astype(np.float32)), dev(wt.astype(np.float32)), dev(g.astype(np.float32))
    assert L.hrt_nn_conv3d_backward(n, d, h, w, cin, cout, xd.data_ptr(), wd.data_ptr(), gd.data_ptr(), dx.data_ptr(),
                                    dw.data_ptr(), db.data_ptr(), None) == 0
    rdx, rdw, rdb = np.zeros(x.shape), np.zeros(wt.shape), np.zeros(cout)
    for s in range(n):
        a, bw, c = N.conv3d_backward(x[s], wt, g[s])
        rdx[s] = a
        rdw += bw
        rdb += c
    close(dx.cpu().numpy().astype(np.float64), rdx, 8e-3)
    close(dw.cpu().numpy().reshape(wt.shape).astype(np.float64), rdw, 1e-3)
    close(db.cpu().numpy().astype(np.float64), rdb, 1e-3)


def _net(base=32, levels=1, seed=5):
    L = hrt.load()
    net = C.c_void_p()
    assert L.hrt_net_create(C.byref(net), 0, base, levels, seed, None) == 0
    return net


def _unpack(flat, base, levels):
    """Packed parameter vector -> oracle parameter list."""
    P = N.init_unet(base, levels, cin=2, seed=0)
    q = 0
    for k, (w, b) in enumerate(P):
        if w.ndim == 5:
            P[k][0] = flat[q:q + w.size].reshape(w.shape).astype(np.float64); q += w.size
            P[k][1] = flat[q:q + b.size].astype(np.float64); q += b.size
        else:
            P[k][0] = flat[q:q + w.size].reshape(w.shape).astype(np.float64); q += w.size
            P[k][1] = flat[q:q + 1].astype(np.float64); q += 1
    assert q == flat.size
    return P


def test_network_forward_and_gradient_match_oracle():
    torch = torch_cuda()
    L = hrt.load()
    base, levels = 32, 1
    net = _net(base, levels)
    npar = L.hrt_net_num_params(net)
    flat = np.empty(npar, np.float32)
    assert L.hrt_net_get_params(net, flat.ctypes.data, npar) == 0
    # BF16-representable parameters so that both sides use the same numbers
    flat = bf16(flat).astype(np.float32)
    assert L.hrt_net_set_params(net, flat.ctypes.data, npar) == 0
    P = _unpack(flat, base, levels)
    rng = np.random.default_rng(9)
    x = bf16(rng.normal(size=(1, 8, 8, 8, 2)))
    t = rng.normal(size=(1, 8, 8, 8)).astype(np.float32).astype(np.float64)
    xd, td = dev(x.astype(np.float32)), dev(t.astype(np.float32))
    y = torch.empty((1, 8, 8, 8), dtype=torch.float32, device="cuda")
    assert L.hrt_net_forward(net, 1, 8, 8, 8, xd.data_ptr(), y.data_ptr()) == 0
    ref = N.unet_forward(P, x[0], levels)
    got = y.cpu().numpy()[0].astype(np.float64)
    # BF16 activations through five layers: a few percent of the output scale
    assert np.sqrt(np.mean((got - ref) ** 2)) < 0.03 * np.sqrt(np.mean(ref ** 2)) + 1e-3
    grad = np.empty(npar, np.float32)
    loss = C.c_double()
    assert L.hrt_net_gradients(net, 1, 8, 8, 8, xd.data_ptr(), td.data_ptr(), grad.ctypes.data, npar, C.byref(loss)) == 0
    rloss, G = N.unet_grad(P, x[0], t[0], levels)
    assert loss.value == pytest.approx(rloss, rel=0.02)
    # every parameter tensor's gradient element by element against the oracle, relative to
    # |r| + rms of that tensor's r; BF16 activations and output gradients stored between layers
    # set the tolerance
    q = 0
    worst = []
    for k, (gw, gb) in enumerate(G):
        for r in (gw.reshape(-1), gb.reshape(-1)):
            gg = grad[q:q + r.size].astype(np.float64)
            q += r.size
            rms = np.sqrt(np.mean(r ** 2)) + 1e-30
            err = np.abs(gg - r) / (np.abs(r) + rms)
            worst.append((k, r.size, float(np.percentile(err, 99)), float(np.median(err)), float(err.max())))
    assert q == npar
    print("per-layer gradient error (layer, size, p99, median, max)", worst)
    # the median and 99 % of every tensor's elements; the rest are elements whose sum nearly
    # cancels or that a ReLU decided differently (BF16 against FP64 pre-activations)
    for k, size, p99, med, _ in worst:
        assert med < 0.03 and p99 < 0.3, (k, size, p99, med)
    L.hrt_net_destroy(net)


def test_training_step_reduces_the_loss():
    torch = torch_cuda()
    L = hrt.load()
    net = _net(32, 2, seed=11)
    rng = np.random.default_rng(12)
    x = dev(rng.normal(size=(2, 16, 16, 16, 2)).astype(np.float32))
    xs = x.cpu().numpy()
    t = dev((0.5 * xs[..., 0] + 0.25 * xs[..., 1] + 0.1).astype(np.float32))
    losses = []
    for _ in range(120):
        loss = C.c_double()
        assert L.hrt_net_train_step(net, 2, 16, 16, 16, x.data_ptr(), t.data_ptr(), 2e-3, C.byref(loss)) == 0
        losses.append(loss.value)
    assert losses[-1] < 0.25 * losses[0], losses[::20]
    L.hrt_net_destroy(net)


def test_warm_start_writes_the_network_prediction():
    torch = torch_cuda()
    L = hrt.load()
    wl = W.turbulent_cloud(n=32, n_sources=3, n_packets=10000, img_n=0, img_lam_um=(), seed=21)
    m = hrt.Model(wl)
    net = _net(32, 2, seed=13)
    nc = m.ncells
    feats = torch.empty(nc * 2, dtype=torch.float32, device="cuda")
    assert L.hrt_net_features(m.ctx, feats.data_ptr(), nc * 2) == 0
    f = feats.cpu().numpy().reshape(32, 32, 32, 2)
    rho = wl.rho.astype(np.float64)
    np.testing.assert_allclose(f[..., 0], (np.log10(rho) + 21.5), rtol=1e-5, atol=1e-5)
    y = torch.empty(nc, dtype=torch.float32, device="cuda")
    assert L.hrt_net_forward(net, 1, 32, 32, 32, feats.data_ptr(), y.data_ptr()) == 0
    assert L.hrt_net_warm_start(net, m.ctx) == 0
    T = m.temperature()
    want = np.clip(10 ** (1.5 + 0.5 * y.cpu().numpy().astype(np.float64)), 1.0, 2000.0)
    np.testing.assert_allclose(T, want, rtol=1e-5)
    # the Lucy iteration runs from it
    st = m.run_iteration()
    assert st["e_escaped"] + st["e_killed"] == pytest.approx(st["e_emitted"], rel=1e-12)
    L.hrt_net_destroy(net)


def test_tcgen05_conv_equals_the_mma_sync_baseline():
    """The TMA-fed tcgen05 kernel, the per-phase tcgen05 kernel and the warp-level mma.sync kernel
    accumulate the same BF16 products in FP32; after the BF16 store they agree to one BF16 ulp
    (summation order)."""
    torch = torch_cuda()
    rng = np.random.default_rng(3)
    L = hrt.load()
    for n, d, h, w, cin, cout in [(1, 9, 10, 11, 32, 32), (2, 5, 6, 7, 64, 64), (1, 6, 20, 36, 64, 192),
                                  (2, 4, 17, 9, 16, 128)]:
        x = dev(rng.normal(size=(n, d, h, w, cin)).astype(np.float32))
        wt = dev((rng.normal(size=(3, 3, 3, cin, cout)) / np.sqrt(27 * cin)).astype(np.float32))
        b = dev(rng.normal(size=cout).astype(np.float32))
        y1 = torch.empty((n, d, h, w, cout), dtype=torch.float32, device="cuda")
        y2 = torch.empty_like(y1)
        assert L.hrt_nn_conv3d(n, d, h, w, cin, cout, x.data_ptr(), wt.data_ptr(), b.data_ptr(), 1, y1.data_ptr(), None) == 0
        assert L.hrt_nn_conv3d_mma(n, d, h, w, cin, cout, x.data_ptr(), wt.data_ptr(), b.data_ptr(), 1, y2.data_ptr(),
                                   None) == 0
        y3 = torch.empty_like(y1)
        assert L.hrt_nn_conv3d_phased(n, d, h, w, cin, cout, x.data_ptr(), wt.data_ptr(), b.data_ptr(), 1,
                                      y3.data_ptr(), None) == 0
        a, c, p = y1.cpu().numpy(), y2.cpu().numpy(), y3.cpu().numpy()
        # one BF16 ulp of the value, or of a small fraction of the output scale where the sum of
        # 27 Cin products nearly cancels (the FP32 summation orders then differ by more)
        floor = 2.0 ** -7 * 0.01 * np.sqrt(np.mean(c.astype(np.float64) ** 2))
        assert np.all(np.abs(a - c) <= 2.0 ** -7 * np.abs(c) + floor)
        assert np.all(np.abs(a - p) <= 2.0 ** -7 * np.abs(p) + floor)

