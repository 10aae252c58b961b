"""FP32 transport against the FP64 oracle on the same random streams, at
1, 2 and 4 mm voxels of the same torso.

Both sides draw identical Philox words per history, so every difference
between them is the FP32 rounding of the GPU transport: a history whose
decisions all agree ends in the same pixel with (nearly) the same deposit.
The test bounds the fraction of histories whose outcome or pixel differ and
the relative difference of the 4x4-binned primary and scatter images, and
prints the per-pixel error report.
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


@pytest.mark.parametrize("vox,n", [(4.0, 2_000_000), (2.0, 2_000_000), (1.0, 1_000_000)])
def test_fp32_transport_against_fp64(gd, vox, n):
    prob = inputs.torso_problem(vox=vox)
    with gd.Context(prob) as ctx:
        rec = torch.zeros(n * gd.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        p, s = gd.gdrr_mc_project(ctx, n, 5, records=rec)
        gd.gdrr_sync(ctx)
        gp, gs, grec = p.cpu().numpy(), s.cpu().numpy(), gd.records_array(rec)
    op, os_, _, orec = oracle.mc_run(prob, n, seed=5, precision=64, threads=NTH, records=True)
    same = (grec["outcome"] == orec["outcome"]) & (grec["pixel"] == orec["pixel"])
    frac_same = float(same.mean())
    report = {"vox_mm": vox, "histories": n, "same_outcome_and_pixel": frac_same}
    for name, g, o in (("primary", gp, op), ("scatter", gs, os_)):
        gb = oracle.bin_tally(g, 4).astype(np.float64)
        ob = oracle.bin_tally(o, 4).astype(np.float64)
        m = ob > np.percentile(ob, 50)
        rel = np.abs(gb - ob)[m] / ob[m]
        report[name] = {"total_rel_diff": float(abs(gb.sum() - ob.sum()) / ob.sum()),
                        "pixel_rel_diff_mean": float(rel.mean()), "pixel_rel_diff_max": float(rel.max())}
        assert report[name]["total_rel_diff"] < 2e-3, report
    print("precision report:", report)
    assert frac_same > 0.995, report
