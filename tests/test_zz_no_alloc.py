"""The allocation-free denoiser against the context-based one.

gdrr_denoise_scatter_static exists for callers that cannot allocate device
memory: a plug-in whose host application fixes its device-memory budget and
owns the allocator, or code that must not call cudaMalloc / cudaFree because
those calls can synchronise the device.  It keeps its scratch in a static
device array shared by every call.  Two calls in a row, of different sizes
and data, must each match gdrr_denoise_scatter on the same input within the
image-step tolerance of the parity tests; sizes beyond the array's maximum
are rejected.  This file is collected last so that a failure here leaves
every other test already run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-11          # the FP64 image-step tolerance of tests/test_gpu_parity.py


@pytest.fixture(scope="module")
def gd():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_6367_gb300 import build, gdrr
    build.build()
    gdrr.lib()
    return gdrr


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_denoiser_matches_context_denoiser(gd):
    from paper_1204_6367_gb300 import inputs
    lib = gd.lib()
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream()
    with gd.Context(inputs.small_problem()) as ctx:
        for nv, nu, scale, beta, iters in ((96, 128, 0.37, 0.02, 300), (40, 56, 2.5, 0.05, 120)):
            counts = rng.poisson(800.0 * (1.0 + 0.3 * np.sin(np.arange(nu) / 9.0))[None, :], (nv, nu))
            s_hat = torch.from_numpy(counts.astype(np.float64) * scale).cuda()
            ref = gd.gdrr_denoise_scatter(ctx, s_hat, scale, beta, 0.8, iters)
            got = torch.full_like(s_hat, float("nan"))
            rc = lib.gdrr_denoise_scatter_static(_ptr(s_hat), _ptr(got), nu, nv, scale, beta, 0.8, iters,
                                                 ctypes.c_void_p(stream.cuda_stream))
            assert rc == 0, lib.gdrr_error_string(rc)
            torch.cuda.synchronize()
            np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=RTOL)


def test_static_denoiser_rejects_oversize(gd):
    lib = gd.lib()
    nv, nu = 257, 256                       # 65792 pixels > the 65536-pixel maximum
    assert nv * nu > gd.STATIC_DENOISE_MAX_PIXELS
    a = torch.ones((nv, nu), dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    rc = lib.gdrr_denoise_scatter_static(_ptr(a), _ptr(b), nu, nv, 1.0, 0.05, 0.8, 3, None)
    assert rc == -1 and lib.gdrr_error_string(rc) == b"invalid argument"
