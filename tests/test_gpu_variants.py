"""GPU parity of the method's variants against the oracle:

* Monte Carlo without density interpolation (the paper's speed variant) and
  with scatter filters (first-order Compton, first-order Rayleigh, multiple):
  bit-exact int64 tallies, counters and event records;
* Siddon ray tracing: FP32/FP64 GPU against the FP64 oracle, rtol 2e-4 (the
  ray-tracing tolerance of tests/test_gpu_parity.py).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1204_6367_gb300 import inputs  # noqa: E402

NTH = os.cpu_count() or 1


@pytest.fixture(scope="module")
def gd():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_6367_gb300 import build, gdrr
    build.build()
    gdrr.lib()
    return gdrr


def _gpu(gd, prob, n, seed, phi=0.0, records=False, **opts):
    with gd.Context(prob) as ctx:
        gd.gdrr_set_options(ctx, **opts)
        stats = torch.zeros(gd.GDRR_NSTATS, dtype=torch.int64, device="cuda")
        rec = torch.zeros(n * gd.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda") if records else None
        p, s = gd.gdrr_mc_project(ctx, n, seed, phi, stats=stats, records=rec)
        gd.gdrr_sync(ctx)
        return p.cpu().numpy(), s.cpu().numpy(), gd.stats_dict(stats), (gd.records_array(rec) if records else None)


@pytest.mark.parametrize("nearest,filt", [(1, 0), (0, 1), (0, 2), (0, 3), (1, 3)])
def test_variants_bit_exact_small(gd, small, nearest, filt):
    n = 500_000
    tp, ts, st, _ = _gpu(gd, small, n, 12, 0.6, nearest_voxel=nearest, scatter_filter=filt)
    otp, ots, ost, _ = oracle.mc_run(small, n, seed=12, phi=0.6, threads=NTH, nearest_voxel=bool(nearest),
                                     scatter_filter=filt)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)


def test_nearest_voxel_records_and_torso(gd):
    prob = inputs.torso_problem(vox=4.0, nu=128, nv=96, det_px=0.776 * 4)
    tp, ts, st, rec = _gpu(gd, prob, 3000, 2, 1.0, records=True, nearest_voxel=1)
    otp, ots, ost, orec = oracle.mc_run(prob, 3000, seed=2, phi=1.0, records=True, nearest_voxel=True)
    for f in oracle.RECORD_DTYPE.names:
        np.testing.assert_array_equal(rec[f], orec[f], err_msg=f)
    n = 300_000
    tp, ts, st, _ = _gpu(gd, prob, n, 5, 2.0, nearest_voxel=1, scatter_filter=1)
    otp, ots, ost, _ = oracle.mc_run(prob, n, seed=5, phi=2.0, threads=NTH, nearest_voxel=True, scatter_filter=1)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)


def test_siddon_small_and_torso(gd, small):
    with gd.Context(small) as ctx:
        for phi in (0.0, 0.9):
            P = gd.gdrr_raytrace_primary_siddon(ctx, phi).cpu().numpy()
            ref = oracle.rt_primary_siddon(small, phi=phi)
            np.testing.assert_allclose(P, ref, rtol=2e-4, atol=1e-12 * ref.max())
    prob = inputs.torso_problem()
    pix = np.random.default_rng(3).integers(0, prob.nu * prob.nv, 150)
    with gd.Context(prob) as ctx:
        for phi in (0.0, 2.2):
            P = gd.gdrr_raytrace_primary_siddon(ctx, phi).cpu().numpy().ravel()[pix]
            ref = oracle.rt_primary_siddon(prob, phi=phi, pixels=pix)
            np.testing.assert_allclose(P, ref, rtol=2e-4, atol=1e-12 * ref.max())
