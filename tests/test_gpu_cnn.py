"""GPU parity of the learned scatter estimator's kernels against the CPU
oracle: the tcgen05 BF16 GEMM against a library matrix product of the same
BF16 inputs, and the network's forward pass and parameter gradients against
the FP64 oracle that rounds to BF16 at the same points.

Tolerances: the GEMM accumulates in FP32, so each element is within
2^-20 (16 FP32 ulps) of the sum of the absolute values of its products.  The network
differs from the emulating oracle only by FP32 accumulation order and the
rare BF16 rounding that this flips: 2e-3 relative (norm) on the output,
2e-2 on each layer's gradients.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle.cnn as cnn  # noqa: E402


@pytest.fixture(scope="module")
def gd():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_6367_gb300 import build, gdrr
    build.build()
    gdrr.lib()
    return gdrr


@pytest.mark.parametrize("M,N,K,splits", [(128, 32, 64, 1), (200, 37, 192, 1), (1000, 130, 640, 1),
                                          (77, 300, 3456, 4), (4096, 64, 576, 1), (64, 896, 2048, 8)])
def test_gemm_bf16(gd, M, N, K, splits):
    rng = np.random.default_rng(M * 7 + N)
    a = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    b = torch.from_numpy(rng.normal(size=(N, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    c = gd.gdrr_gemm_bf16(a, b, splits)
    torch.cuda.synchronize()
    ad, bd = a.double().cpu().numpy(), b.double().cpu().numpy()
    ref = ad @ bd.T
    # FP32 accumulation: error within a few ulps of the sum of |products|
    bound = 2.0**-20 * (np.abs(ad) @ np.abs(bd).T)
    err = np.abs(c.cpu().numpy() - ref)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("M, N, K, splits", [(1000, 256, 320, 1),    # TMA path, 256-wide tiles, ragged M
                                             (130, 200, 128, 1),     # TMA path, 128-wide tiles, ragged M and N
                                             (4096, 512, 1024, 3),   # TMA path, K split across CTAs
                                             (300, 128, 64, 1),      # one K slice
                                             (512, 384, 2048, 1),    # ring wraps many times
                                             (8192, 2048, 64, 1),    # persistent: 3-4 tiles per CTA
                                             (4000, 1024, 384, 3),   # persistent with K splits (atomics)
                                             (3000, 768, 128, 1),    # persistent, fewer tiles than SMs
                                             (5000, 32, 896, 1),     # persistent 32-wide, deep ring wraps
                                             (3000, 64, 1728, 1),    # persistent 64-wide
                                             (1000, 48, 512, 3)])    # persistent 64-wide, ragged N, K splits
def test_gemm_bf16_tma_path(gd, M, N, K, splits):
    rng = np.random.default_rng(M + 3 * N + K)
    a = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    b = torch.from_numpy(rng.normal(size=(N, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    c = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    gd.gdrr_gemm_bf16(a, b, splits, out=c)
    torch.cuda.synchronize()
    ad, bd = a.double().cpu().numpy(), b.double().cpu().numpy()
    ref = ad @ bd.T
    bound = 2.0**-20 * (np.abs(ad) @ np.abs(bd).T) * max(1, splits)
    err = np.abs(c.cpu().numpy() - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_gemm_bf16_strided_and_unaligned_operands(gd):
    # row strides above K give the same products; a base off a 16-byte
    # boundary is refused before any launch (operand rows are read in 16-byte
    # pieces)
    rng = np.random.default_rng(77)
    M, N, K = 257, 192, 192
    big_a = torch.from_numpy(rng.normal(size=(M, K + 64)).astype(np.float32)).to(torch.bfloat16).cuda()
    big_b = torch.from_numpy(rng.normal(size=(N + 1, K + 8)).astype(np.float32)).to(torch.bfloat16).cuda()
    a = big_a[:, :K]                      # lda = K + 64
    b = big_b[:N, :K]                     # ldb = K + 8
    ad, bd = a.double().cpu().numpy(), b.double().cpu().numpy()
    c = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    gd.gdrr_gemm_bf16(a, b, 1, out=c)
    torch.cuda.synchronize()
    bound = 2.0**-20 * (np.abs(ad) @ np.abs(bd).T)
    assert np.all(np.abs(c.cpu().numpy() - ad @ bd.T) <= bound)
    b_off = big_b.reshape(-1)[4:4 + N * (K + 8)].view(N, K + 8)[:, :K]    # base 8 bytes off
    with pytest.raises(gd.GdrrError) as ei:
        gd.gdrr_gemm_bf16(a, b_off, 1, out=c)
    assert ei.value.code == -1


# Grids that take each product form: at 32 x 32 the 16 x 16 and 32 x 32
# levels tile into 128-pixel row groups (implicit GEMM) and the 8 x 8 and
# 4 x 4 levels take the column matrix; at the estimator's 96 x 128 every
# level but 12 x 16 tiles (one, two and four rows per tile); at 16 x 256 a
# tile is half an image row.
@pytest.mark.parametrize("H,W,B", [(32, 32, 2), (96, 128, 2), (16, 256, 1)])
def test_cnn_forward_backward_against_oracle(gd, H, W, B):
    c = 32
    rng = np.random.default_rng(9)
    x = rng.normal(size=(B, 2, H, W)).astype(np.float32)
    t = rng.normal(size=(B, 1, H, W)).astype(np.float32)
    p = cnn.init_params(c, 5).astype(np.float32)
    p += (0.01 * rng.normal(size=p.size)).astype(np.float32)      # non-zero biases
    net = gd.Cnn(B, H, W, c)
    assert net.n_params == cnn.n_params(c)
    net.set_params(p)
    out = net.forward(torch.from_numpy(x).cuda())
    loss = net.backward(torch.from_numpy(t).cuda())
    g = net.get_grads()
    o_out, cache = cnn.forward(x.astype(np.float64), p.astype(np.float64), c, emulate=True)
    o_loss, o_g = cnn.backward(cache, t.astype(np.float64))
    out = out.cpu().numpy()
    assert np.linalg.norm(out - o_out) / np.linalg.norm(o_out) < 2e-3
    assert loss == pytest.approx(o_loss, rel=5e-3)
    off = 0
    for i, (ci, co, k, _) in enumerate(cnn.specs(c)):
        for name, size in (("w", co * ci * k * k), ("b", co)):
            gg, og = g[off:off + size], o_g[off:off + size]
            off += size
            rel = np.linalg.norm(gg - og) / max(np.linalg.norm(og), 1e-30)
            assert rel < 2e-2, (i, name, rel)
    net.close()


def test_cnn_training_reduces_loss(gd):
    c, H, W, B = 32, 32, 48, 4
    rng = np.random.default_rng(2)
    yy, xx = np.mgrid[0:H, 0:W]
    base = np.exp(-((xx - W / 2) ** 2 + (yy - H / 2) ** 2) / 200.0)
    t = np.stack([base * (1 + 0.2 * i) for i in range(B)])[:, None].astype(np.float32)
    x = np.concatenate([t + 0.3 * rng.normal(size=t.shape), 0.5 * t], axis=1).astype(np.float32)
    net = gd.Cnn(B, H, W, c, seed=3)
    xt, tt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    losses = []
    for _ in range(60):
        net.forward(xt)
        losses.append(net.backward(tt))
        net.adam_step(1e-3)
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])
    net.close()


def test_training_is_bit_reproducible(gd):
    # at the estimator's size the first layers split their weight-gradient pixel
    # sums across CTAs; the partial products are added in a fixed order, so
    # two trainings from the same start end bit-identical
    rng = np.random.default_rng(3)
    H, W, B, c = 96, 128, 16, 32
    x = torch.from_numpy(rng.normal(size=(B, 2, H, W)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(size=(B, 1, H, W)).astype(np.float32)).cuda()
    params = []
    for _ in range(2):
        net = gd.Cnn(B, H, W, c, seed=4)
        for _ in range(5):
            net.forward(x)
            net.backward(t)
            net.adam_step(1e-3)
        params.append(net.get_params())
        net.close()
    np.testing.assert_array_equal(params[0], params[1])
