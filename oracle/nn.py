"""FP64 ORACLE of the learned warm start's layers (numpy, direct loops over the 27 taps).

Test infrastructure only (tests and the smoke check): the CUDA network kernels are checked
against these definitions on small tensors.  Layout: channels last, x[z, y, x, c]; 3x3x3
weights w[dz, dy, dx, c_in, c_out]; zero padding of one voxel ("same" convolution).

* conv3d:     y[v, o] = b[o] + sum_{d, i} x[v + d - 1, i] w[d, i, o]
* its gradients by the chain rule: dx[v, i] = sum_{d, o} dy[v - d + 1, o] w[d, i, o],
  dw[d, i, o] = sum_v x[v + d - 1, i] dy[v, o], db[o] = sum_v dy[v, o]
* 2x average pooling, 2x nearest upsampling, channel concatenation, ReLU and their gradients
* the encoder-decoder (U-Net) the library trains, for finite-difference pins
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in range(3) for dy in range(3) for dx in range(3)]


def pad1(x):
    return np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))


def conv3d(x, w, b):
    """'Same' 3x3x3 convolution (cross-correlation) with bias."""
    D, H, W, _ = x.shape
    xp = pad1(np.asarray(x, np.float64))
    y = np.zeros((D, H, W, w.shape[-1])) + np.asarray(b, np.float64)
    for dz, dy, dx in TAPS:
        y += xp[dz:dz + D, dy:dy + H, dx:dx + W, :] @ np.asarray(w[dz, dy, dx], np.float64)
    return y


def conv3d_backward(x, w, dy):
    D, H, W, _ = x.shape
    xp = pad1(np.asarray(x, np.float64))
    dyp = pad1(np.asarray(dy, np.float64))
    dw = np.zeros(w.shape)
    dx = np.zeros(x.shape)
    for dz, dyy, dxx in TAPS:
        dw[dz, dyy, dxx] = np.einsum("zyxi,zyxo->io", xp[dz:dz + D, dyy:dyy + H, dxx:dxx + W, :], dy)
        # dx[v] += dy[v - d + 1] w[d]^T ; dyp index v - d + 1 + 1 = v + 2 - d
        dx += dyp[2 - dz:2 - dz + D, 2 - dyy:2 - dyy + H, 2 - dxx:2 - dxx + W, :] @ np.asarray(w[dz, dyy, dxx], np.float64).T
    db = dy.sum(axis=(0, 1, 2))
    return dx, dw, db


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def avgpool2_backward(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, 0), 2, 1), 2, 2) / 8.0


def upsample2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def upsample2_backward(dy):
    D, H, W, C = dy.shape
    return dy.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def init_unet(base, levels, cin=2, seed=0):
    """Parameters of the encoder-decoder: per level two 3x3x3 convs (encoder), the bottleneck,
    then per level an upsampled concat and two convs (decoder), and a 1x1x1 head."""
    rng = np.random.default_rng(seed)
    P = []

    def conv(ci, co):
        bound = np.sqrt(6.0 / (27 * ci))
        P.append([rng.uniform(-bound, bound, (3, 3, 3, ci, co)), np.zeros(co)])

    ch = [base * 2 ** l for l in range(levels + 1)]
    c = cin
    for l in range(levels):
        conv(c, ch[l]); conv(ch[l], ch[l]); c = ch[l]
    conv(c, ch[levels]); conv(ch[levels], ch[levels]); c = ch[levels]
    for l in reversed(range(levels)):
        conv(c + ch[l], ch[l]); conv(ch[l], ch[l]); c = ch[l]
    P.append([rng.uniform(-1, 1, (c, 1)) / np.sqrt(c), np.zeros(1)])
    return P


def unet_forward(P, x, levels):
    """Returns the output [D,H,W] and the saved activations."""
    acts = {}
    h = x
    k = 0
    skips = []
    for l in range(levels):
        for _ in range(2):
            h = relu(conv3d(h, *P[k])); k += 1
        skips.append(h)
        h = avgpool2(h)
    for _ in range(2):
        h = relu(conv3d(h, *P[k])); k += 1
    for l in reversed(range(levels)):
        h = np.concatenate([upsample2(h), skips[l]], axis=-1)
        for _ in range(2):
            h = relu(conv3d(h, *P[k])); k += 1
    w, b = P[k]
    return (h @ w)[..., 0] + b[0]


def unet_loss(P, x, target, levels):
    y = unet_forward(P, x, levels)
    return 0.5 * np.mean((y - target) ** 2)


def unet_grad(P, x, target, levels):
    """Loss 0.5 mean((y - t)^2) and its gradient for every parameter (chain rule, layer by layer)."""
    # forward, keeping every conv input and output
    rec = []
    h = x
    k = 0
    skips = []
    for l in range(levels):
        for _ in range(2):
            z = conv3d(h, *P[k]); rec.append((h, z)); h = relu(z); k += 1
        skips.append(h)
        h = avgpool2(h)
    for _ in range(2):
        z = conv3d(h, *P[k]); rec.append((h, z)); h = relu(z); k += 1
    ups = []
    for l in reversed(range(levels)):
        ups.append(h.shape[-1])
        h = np.concatenate([upsample2(h), skips[l]], axis=-1)
        for _ in range(2):
            z = conv3d(h, *P[k]); rec.append((h, z)); h = relu(z); k += 1
    w, b = P[k]
    y = (h @ w)[..., 0] + b[0]
    n = y.size
    loss = 0.5 * np.mean((y - target) ** 2)
    G = [None] * len(P)
    dy = (y - target) / n
    G[k] = [h.reshape(-1, h.shape[-1]).T @ dy.reshape(-1, 1), np.array([dy.sum()])]
    dh = dy[..., None] * w[:, 0]
    # decoder (reverse)
    ci = len(rec) - 1
    dskips = [None] * levels
    for l in range(levels):                    # walk the decoder back: level 0 ran last
        for _ in range(2):
            hin, z = rec[ci]
            dz = dh * (z > 0)
            dh, dw_, db_ = conv3d_backward(hin, P[ci][0], dz)
            G[ci] = [dw_, db_]
            ci -= 1
        cu = ups[levels - 1 - l]
        dskips[l] = dh[..., cu:]
        dh = upsample2_backward(dh[..., :cu])
    for _ in range(2):
        hin, z = rec[ci]
        dz = dh * (z > 0)
        dh, dw_, db_ = conv3d_backward(hin, P[ci][0], dz)
        G[ci] = [dw_, db_]
        ci -= 1
    for l in reversed(range(levels)):
        dh = avgpool2_backward(dh) + dskips[l]
        for _ in range(2):
            hin, z = rec[ci]
            dz = dh * (z > 0)
            dh, dw_, db_ = conv3d_backward(hin, P[ci][0], dz)
            G[ci] = [dw_, db_]
            ci -= 1
    return loss, G
