"""Pins of the FP64 network oracle (no GPU): the convolution against scipy's n-d correlation,
every gradient against central finite differences, pooling/upsampling adjointness."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import nn as N


def test_conv3d_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(5, 6, 7, 3))
    w = rng.normal(size=(3, 3, 3, 3, 4))
    b = rng.normal(size=4)
    y = N.conv3d(x, w, b)
    for o in range(4):
        ref = np.full(x.shape[:3], b[o])
        for i in range(3):
            ref += ndimage.correlate(x[..., i], w[..., i, o], mode="constant", cval=0.0)
        np.testing.assert_allclose(y[..., o], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_gradients_by_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 4, 3, 2))
    w = rng.normal(size=(3, 3, 3, 2, 3))
    b = rng.normal(size=3)
    r = rng.normal(size=(3, 4, 3, 3))
    loss = lambda x_, w_, b_: float((N.conv3d(x_, w_, b_) * r).sum())
    dx, dw, db = N.conv3d_backward(x, w, r)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 1, 1), (2, 3, 2, 0)]:
        e = np.zeros_like(x); e[idx] = h
        assert dx[idx] == pytest.approx((loss(x + e, w, b) - loss(x - e, w, b)) / (2 * h), rel=1e-6, abs=1e-8)
    for idx in [(0, 0, 0, 0, 0), (1, 1, 1, 1, 2), (2, 0, 1, 0, 1)]:
        e = np.zeros_like(w); e[idx] = h
        assert dw[idx] == pytest.approx((loss(x, w + e, b) - loss(x, w - e, b)) / (2 * h), rel=1e-6, abs=1e-8)
    e = np.zeros_like(b); e[1] = h
    assert db[1] == pytest.approx((loss(x, w, b + e) - loss(x, w, b - e)) / (2 * h), rel=1e-6)


def test_pool_and_upsample_are_adjoint_to_their_gradients():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(4, 4, 6, 3))
    y = rng.normal(size=(2, 2, 3, 3))
    assert float((N.avgpool2(x) * y).sum()) == pytest.approx(float((x * N.avgpool2_backward(y)).sum()), rel=1e-12)
    assert float((N.upsample2(y) * x).sum()) == pytest.approx(float((y * N.upsample2_backward(x)).sum()), rel=1e-12)
    assert N.avgpool2(np.ones((2, 2, 2, 1)))[0, 0, 0, 0] == 1.0


def test_unet_gradient_by_finite_differences():
    rng = np.random.default_rng(3)
    levels = 1
    P = N.init_unet(base=3, levels=levels, cin=2, seed=4)
    x = rng.normal(size=(4, 4, 4, 2))
    t = rng.normal(size=(4, 4, 4))
    loss, G = N.unet_grad(P, x, t, levels)
    assert loss == pytest.approx(N.unet_loss(P, x, t, levels), rel=1e-12)
    h = 1e-6
    for k in range(len(P)):
        for part in (0, 1):
            a = P[k][part]
            idx = tuple(rng.integers(0, s) for s in a.shape)
            old = a[idx]
            a[idx] = old + h; lp = N.unet_loss(P, x, t, levels)
            a[idx] = old - h; lm = N.unet_loss(P, x, t, levels)
            a[idx] = old
            assert G[k][part][idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9), (k, part, idx)
