"""Pins of the CNN oracle: the convolution against scipy's correlate, BF16
rounding against torch's cast, pooling / upsampling adjointness, and the
backward pass against central finite differences in FP64."""
import numpy as np
import pytest
from scipy import signal

import oracle.cnn as cnn


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).normal(0, 10, 100000).astype(np.float32)
    x[:4] = [1.0, 1.00390625, 1.01171875, -3.0e-39]
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cnn.bf16(x), ref)


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 9, 11))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = cnn.conv(x, w, b)
    for bi in range(2):
        for co in range(4):
            ref = sum(signal.correlate2d(x[bi, ci], w[co, ci], mode="same") for ci in range(3)) + b[co]
            np.testing.assert_allclose(y[bi, co], ref, rtol=1e-12, atol=1e-12)


def test_pool_and_up_adjoints():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 3, 8, 12))
    d = rng.normal(size=(2, 3, 4, 6))
    assert np.isclose(np.sum(cnn.pool(x) * d), np.sum(x * cnn.pool_back(d)))
    y = rng.normal(size=(2, 3, 4, 6))
    e = rng.normal(size=(2, 3, 8, 12))
    assert np.isclose(np.sum(cnn.up(y) * e), np.sum(y * cnn.up_back(e)))


def test_backward_matches_finite_differences():
    c, H, W = 2, 8, 16
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 2, H, W))
    t = rng.normal(size=(2, 1, H, W))
    p = cnn.init_params(c, 4) + 0.05 * rng.normal(size=cnn.n_params(c))
    _, cache = cnn.forward(x, p, c, emulate=False)
    loss, g = cnn.backward(cache, t)
    idx = rng.choice(p.size, 40, replace=False)
    eps = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        lp = cnn.backward(cnn.forward(x, pp, c, emulate=False)[1], t)[0]
        lm = cnn.backward(cnn.forward(x, pm, c, emulate=False)[1], t)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (i, fd, g[i])
