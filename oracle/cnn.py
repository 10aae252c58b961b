"""CPU oracle of the learned scatter estimator.  TEST INFRASTRUCTURE ONLY.

numpy FP64 forward and backward of the 4-level convolutional
encoder-decoder (conv3x3 + ReLU per level, 2x2 average pooling, nearest 2x
upsampling with skip concatenation, 1x1 output added to input channel 0,
mean-squared-error loss).
With emulate=True the values the GPU stores in BF16 are rounded to BF16 at
the same points: the network input, the weights, every stored activation,
and the activation gradients that enter the two products of a convolution's
backward pass.  Shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def specs(c):
    """(ci, co, ks, relu) of the eight convolutions, in parameter order."""
    return [(2, c, 3, 1), (c, 2 * c, 3, 1), (2 * c, 4 * c, 3, 1), (4 * c, 8 * c, 3, 1),
            (12 * c, 4 * c, 3, 1), (6 * c, 2 * c, 3, 1), (3 * c, c, 3, 1), (c, 1, 1, 0)]


def n_params(c):
    return sum(co * ci * k * k + co for ci, co, k, _ in specs(c))


def unflatten(flat, c):
    out, off = [], 0
    for ci, co, k, _ in specs(c):
        w = np.asarray(flat[off:off + co * ci * k * k], np.float64).reshape(co, ci, k, k)
        off += w.size
        b = np.asarray(flat[off:off + co], np.float64)
        off += co
        out.append((w, b))
    return out


def flatten(grads):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in grads])


def im2col(x, k):
    """[B, C, H, W] -> [B*H*W, C*k*k] with zero padding k // 2."""
    B, C, H, W = x.shape
    h = k // 2
    xp = np.pad(x, ((0, 0), (0, 0), (h, h), (h, h)))
    cols = np.empty((B, H, W, C, k, k))
    for ky in range(k):
        for kx in range(k):
            cols[:, :, :, :, ky, kx] = xp[:, :, ky:ky + H, kx:kx + W].transpose(0, 2, 3, 1)
    return cols.reshape(B * H * W, C * k * k)


def col2im(dcols, shape, k):
    B, C, H, W = shape
    h = k // 2
    d = dcols.reshape(B, H, W, C, k, k)
    dxp = np.zeros((B, C, H + 2 * h, W + 2 * h))
    for ky in range(k):
        for kx in range(k):
            dxp[:, :, ky:ky + H, kx:kx + W] += d[:, :, :, :, ky, kx].transpose(0, 3, 1, 2)
    return dxp[:, :, h:h + H, h:h + W]


def conv(x, w, b):
    """Cross-correlation with zero padding (the convolution of CNNs)."""
    B, C, H, W = x.shape
    co, _, k, _ = w.shape
    y = im2col(x, k) @ w.reshape(co, -1).T + b
    return y.reshape(B, H, W, co).transpose(0, 3, 1, 2)


def pool(x):
    return 0.25 * ((x[:, :, 0::2, 0::2] + x[:, :, 0::2, 1::2]) + (x[:, :, 1::2, 0::2] + x[:, :, 1::2, 1::2]))


def pool_back(d):
    return 0.25 * np.repeat(np.repeat(d, 2, axis=2), 2, axis=3)


def up(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up_back(d):
    return (d[:, :, 0::2, 0::2] + d[:, :, 0::2, 1::2]) + (d[:, :, 1::2, 0::2] + d[:, :, 1::2, 1::2])


def forward(x, flat, c, emulate=True):
    r = bf16 if emulate else (lambda v: np.asarray(v, np.float64))
    P = unflatten(flat, c)
    W = [(r(w), b) for w, b in P]
    cache = {"W": W, "c": c, "emulate": emulate}

    def layer(i, inp):
        w, b = W[i]
        z = conv(inp, w, b)
        y = np.maximum(z, 0.0) if specs(c)[i][3] else z
        return y

    x_in = np.asarray(x, np.float64)
    x = r(x)
    e1 = r(layer(0, x)); p1 = r(pool(e1))
    e2 = r(layer(1, p1)); p2 = r(pool(e2))
    e3 = r(layer(2, p2)); p3 = r(pool(e3))
    e4 = r(layer(3, p3))
    c3 = np.concatenate([up(e4), e3], axis=1); d3 = r(layer(4, c3))
    c2 = np.concatenate([up(d3), e2], axis=1); d2 = r(layer(5, c2))
    c1 = np.concatenate([up(d2), e1], axis=1); d1 = r(layer(6, c1))
    out = layer(7, d1) + x_in[:, 0:1]      # residual: a correction to input channel 0
    cache.update(x=x, e1=e1, p1=p1, e2=e2, p2=p2, e3=e3, p3=p3, e4=e4, c3=c3, d3=d3, c2=c2, d2=d2, c1=c1, d1=d1,
                 out=out)
    return out, cache


def backward(cache, target):
    """Loss = mean (out - target)^2 and the flat gradient of every parameter."""
    c, W = cache["c"], cache["W"]
    r = bf16 if cache["emulate"] else (lambda v: v)
    out = cache["out"]
    n = out.size
    loss = float(np.mean((out - target) ** 2))
    grads = [None] * 8

    def layer_back(i, dy, y, x):
        w, _ = W[i]
        k = w.shape[2]
        dz = dy * (y > 0) if specs(c)[i][3] else dy
        db = dz.sum(axis=(0, 2, 3))
        dzr = r(dz)
        co = w.shape[0]
        dz2 = dzr.transpose(0, 2, 3, 1).reshape(-1, co)
        dw = (dz2.T @ im2col(x, k)).reshape(w.shape)
        grads[i] = (dw, db)
        return col2im(dz2 @ w.reshape(co, -1), x.shape, k)

    g = 2.0 * (out - target) / n
    gd1 = layer_back(7, g, out, cache["d1"])
    gc1 = layer_back(6, gd1, cache["d1"], cache["c1"])
    gd2 = up_back(gc1[:, :2 * c]); ge1 = gc1[:, 2 * c:]
    gc2 = layer_back(5, gd2, cache["d2"], cache["c2"])
    gd3 = up_back(gc2[:, :4 * c]); ge2 = gc2[:, 4 * c:]
    gc3 = layer_back(4, gd3, cache["d3"], cache["c3"])
    ge4 = up_back(gc3[:, :8 * c]); ge3 = gc3[:, 8 * c:]
    gp3 = layer_back(3, ge4, cache["e4"], cache["p3"])
    ge3 = ge3 + pool_back(gp3)
    gp2 = layer_back(2, ge3, cache["e3"], cache["p2"])
    ge2 = ge2 + pool_back(gp2)
    gp1 = layer_back(1, ge2, cache["e2"], cache["p1"])
    ge1 = ge1 + pool_back(gp1)
    layer_back(0, ge1, cache["e1"], cache["x"])
    return loss, flatten(grads)


def init_params(c, seed):
    """He-normal weights, zero biases (independent of the GPU's initialiser)."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co, k, _ in specs(c):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (ci * k * k)), co * ci * k * k))
        parts.append(np.zeros(co))
    return np.concatenate(parts)
