"""GPU parity of the local-majorant tracking option against the CPU oracle.

With local majorants the transport draws differently from the global
majorant's Woodcock tracking, so it is compared with the oracle's own
local-majorant tracking: per-history event records, counters (the cell
crossings included) and int64 tallies bit for bit, in both start paths (the
source pass without records, inline starts with them), every launch
configuration, 2, 4 and 8 material slots, and the general kernel's options.
At scale, against the global majorant: the same images within the statistics.
"""
import math
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


def _run(gd, prob, n, seed, phi=0.0, angle_index=0, offset=0, records=False, shift=0, **opts):
    with gd.Context(prob) as ctx:
        gd.gdrr_set_options(ctx, local_majorant=1, cell_shift=shift, **opts)
        o = gd.gdrr_get_options(ctx)
        assert o["local_majorant"] == 1
        stats = torch.zeros(gd.GDRR_NSTATS, dtype=torch.int64, device="cuda")
        rec = torch.zeros(n * gd.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda") if records else None
        prim, scat = gd.gdrr_mc_project(ctx, n, seed, phi, angle_index, offset, stats=stats, records=rec)
        gd.gdrr_sync(ctx)
        return (prim.cpu().numpy(), scat.cpu().numpy(), gd.stats_dict(stats),
                gd.records_array(rec) if records else None, o["cell_shift"])


def _same(got, prob, n, seed, phi=0.0, angle_index=0, records=False, **oopts):
    tp, ts, st, rec, shift = got
    otp, ots, ost, orec = oracle.mc_run(prob, n, seed=seed, phi=phi, angle_index=angle_index, records=records,
                                        threads=1 if records else NTH, local_majorant=True, cell_shift=shift,
                                        **oopts)
    if records:
        for f in oracle.RECORD_DTYPE.names:
            np.testing.assert_array_equal(rec[f], orec[f], err_msg=f)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)
    return ost


@pytest.mark.parametrize("shift", [1, 3])
def test_tiny_run_event_by_event(gd, small, shift):
    n = 1000
    st = _same(_run(gd, small, n, 1, records=True, shift=shift), small, n, 1, records=True)
    assert st["crossings"] > 0


@pytest.mark.parametrize("phi", [0.0, 1.1])
def test_small_problem_1e6_bit_exact(gd, small, phi):
    # no records: the source pass starts the histories
    n = 1_000_000
    _same(_run(gd, small, n, 3, phi=phi, angle_index=5, shift=2), small, n, 3, phi=phi, angle_index=5)


def test_torso_4mm_default_cells_bit_exact(gd):
    # the default cells of the option are about 32 mm: 8 voxels of 4 mm
    prob = inputs.torso_problem(vox=4.0, nu=128, nv=96, det_px=0.776 * 4)
    n = 300_000
    got = _run(gd, prob, n, 11, phi=0.4, angle_index=2)
    assert got[4] == 3
    st = _same(got, prob, n, 11, phi=0.4, angle_index=2)
    assert st["steps"] < 0.25 * 46 * n


def _slot_problem(which):
    rng = np.random.default_rng(17)
    if which == "two":                                     # 2 slots: a bone block in air
        prob = inputs.uniform_slab_problem(nx=20, ny=18, nz=17, nu=16, nv=16, det_px=3.0, pencil=False, mat_id=0,
                                           density=0.0012, materials=[inputs.AIR, inputs.BONE])
        prob.material[4:12, 3:15, 9:19] = 1
        prob.density[4:12, 3:15, 9:19] = rng.uniform(1.2, 1.9, (8, 12, 10)).astype(np.float32)
    else:                                                  # 8 slots: slabs of eight materials
        mats = [inputs.AIR, inputs.WATER, inputs.BONE, inputs.LUNG, inputs.ALUMINIUM,
                inputs.WATER, inputs.BONE, inputs.LUNG]
        prob = inputs.uniform_slab_problem(nx=16, ny=15, nz=19, nu=16, nv=16, det_px=3.0, pencil=False,
                                           materials=mats)
        prob.material[:] = ((np.arange(19) // 3) % 8).astype(np.uint8)[:, None, None]
        prob.density[:] = rng.uniform(0.0, 2.6, prob.density.shape).astype(np.float32)
    prob.form_factor = None
    return prob


@pytest.mark.parametrize("which", ["two", "eight"])
@pytest.mark.parametrize("shift", [1, 2, 6])
def test_material_slots_and_cell_sizes(gd, which, shift):
    # ragged grids (no cell size divides 20 x 18 x 17 or 16 x 15 x 19), one
    # cell for the whole box at shift 6
    prob = _slot_problem(which)
    _same(_run(gd, prob, 1500, 21, phi=0.7, records=True, shift=shift), prob, 1500, 21, phi=0.7, records=True)
    _same(_run(gd, prob, 200_000, 5, phi=2.1, shift=shift), prob, 200_000, 5, phi=2.1)


@pytest.mark.parametrize("opts", [dict(nearest_voxel=1), dict(scatter_filter=1), dict(scatter_filter=3),
                                  dict(rayleigh_form_factor=1)])
def test_general_kernel_options(gd, small, opts):
    oopts = {"nearest_voxel": bool(opts.get("nearest_voxel", 0)), "scatter_filter": opts.get("scatter_filter", 0),
             "rayleigh_ff": bool(opts.get("rayleigh_form_factor", 0))}
    n = 1500
    _same(_run(gd, small, n, 23, phi=0.5, records=True, shift=2, **opts), small, n, 23, phi=0.5, records=True,
          **oopts)
    n = 200_000
    _same(_run(gd, small, n, 29, phi=1.5, shift=1, **opts), small, n, 29, phi=1.5, **oopts)


@pytest.mark.parametrize("opts", [dict(block_size=64, hist_per_thread=1, batch_min=1),
                                  dict(block_size=128, hist_per_thread=64, batch_min=32),
                                  dict(block_size=256, hist_per_thread=3, batch_min=3, blocks_per_sm=1),
                                  dict(block_size=512, hist_per_thread=8, batch_min=20),
                                  dict(photon_pool=2, hist_per_thread=5)])
def test_launch_configuration_invariance(gd, small, opts):
    # the pool form does not carry the option: photon_pool runs the lane form
    n = 200_003
    _same(_run(gd, small, n, 7, phi=0.3, shift=2, **opts), small, n, 7, phi=0.3)


def test_option_checks(gd, small):
    # the option's default cells are about 32 mm: 8 voxels of 4 mm, 16 of
    # 2 mm, 32 of 1 mm, 64 of 0.5 mm
    for vox, shift in ((4.0, 3), (2.0, 4), (1.0, 5), (0.5, 6)):
        prob = inputs.uniform_slab_problem(nx=8, ny=8, nz=8, vox=vox)
        with gd.Context(prob) as ctx:
            gd.gdrr_set_options(ctx, local_majorant=1)
            assert gd.gdrr_get_options(ctx)["cell_shift"] == shift
            gd.gdrr_set_options(ctx, local_majorant=0)
            assert gd.gdrr_get_options(ctx)["cell_shift"] == max(1, round(math.log2(4.0 / vox)))
    with gd.Context(small) as ctx:
        gd.gdrr_set_options(ctx, local_majorant=1)
        assert gd.gdrr_get_options(ctx)["batch_min"] == 24          # the option's default
        gd.gdrr_set_options(ctx, local_majorant=0)
        assert gd.gdrr_get_options(ctx)["batch_min"] == 16
        for bad in (dict(local_majorant=2), dict(local_majorant=-1), dict(local_majorant=1, cell_shift=-1)):
            with pytest.raises(gd.GdrrError):
                gd.gdrr_set_options(ctx, **bad)
        assert gd.gdrr_get_options(ctx)["local_majorant"] == 0


def test_full_size_2mm_torso_windows_and_global_majorant(gd):
    # The 2 mm torso at 2e7 histories with the option's defaults: history
    # windows equal the oracle bit for bit, the run equals its split parts,
    # and it agrees with the global majorant's run within the statistics
    # (total primary and scatter, 16 x 16-pixel blocks) with a quarter of
    # its flights or fewer.
    prob = inputs.torso_problem(vox=2.0)
    n = 20_000_000
    with gd.Context(prob) as ctx:
        sg = torch.zeros(gd.GDRR_NSTATS, dtype=torch.int64, device="cuda")
        gp, gs = gd.gdrr_mc_project(ctx, n, 5, stats=sg)
        gd.gdrr_set_options(ctx, local_majorant=1, batch_min=24)
        assert gd.gdrr_get_options(ctx)["cell_shift"] == 4
        sl = torch.zeros(gd.GDRR_NSTATS, dtype=torch.int64, device="cuda")
        lp, ls = gd.gdrr_mc_project(ctx, n, 3, stats=sl)
        parts_p, parts_s = gd.new_tallies(ctx)
        for lo, hi in ((0, 7_000_000), (7_000_000, n)):
            gd.gdrr_mc_project(ctx, hi - lo, 3, history_offset=lo, prim=parts_p, scat=parts_s)
        gd.gdrr_sync(ctx)
        assert torch.equal(lp, parts_p) and torch.equal(ls, parts_s)
        for off in (0, 12_345_678, n - 20_000):
            wp, ws = gd.gdrr_mc_project(ctx, 20_000, 3, history_offset=off)
            otp, ots, _, _ = oracle.mc_run(prob, 20_000, seed=3, history_offset=off, threads=NTH,
                                           local_majorant=True, cell_shift=4)
            np.testing.assert_array_equal(wp.cpu().numpy(), otp)
            np.testing.assert_array_equal(ws.cpu().numpy(), ots)
        g, l = gd.stats_dict(sg), gd.stats_dict(sl)
    assert l["steps"] < 0.25 * g["steps"] and l["crossings"] > 0 and g["crossings"] == 0
    for k in ("tally_primary", "tally_scatter", "rayleigh", "compton", "photo", "miss"):
        assert abs(g[k] - l[k]) < 4.0 * math.sqrt(2.0 * max(g[k], l[k])) + 2, (k, g[k], l[k])
    for a, b, key in ((gp, lp, "tally_primary"), (gs, ls, "tally_scatter")):
        A = a.cpu().numpy().reshape(24, 16, 32, 16).sum(axis=(1, 3)).astype(np.float64)
        B = b.cpu().numpy().reshape(24, 16, 32, 16).sum(axis=(1, 3)).astype(np.float64)
        unit = (A.sum() + B.sum()) / (g[key] + l[key])
        sig = 1.5 * np.sqrt((A + B) / unit) * unit
        assert np.all(np.abs(A - B) <= 5.0 * sig + 3.0 * unit), np.abs(A - B).max() / unit


def test_batched_scan_and_graph_carry_the_option(gd, small):
    # one persistent launch over all angles, and its CUDA-graph replay, give
    # each angle's per-angle local-majorant tallies; one angle against the oracle
    angles = np.linspace(0, 2 * math.pi, 5, endpoint=False)
    budgets = np.array([20_000, 7, 0, 55_555, 31_000], np.uint64)
    with gd.Context(small) as ctx:
        gd.gdrr_set_options(ctx, local_majorant=1, cell_shift=2)
        bp, bs = gd.gdrr_mc_project_batched(ctx, angles, budgets, 23)
        for a in range(angles.size):
            p, s = gd.gdrr_mc_project(ctx, int(budgets[a]), 23, float(angles[a]), a)
            assert torch.equal(bp[a], p) and torch.equal(bs[a], s), a
        scan = gd.gdrr_scan_create(ctx, angles, budgets, 23, zero_tallies=True)
        scan.launch()
        scan.launch()
        gd.gdrr_sync(ctx)
        assert torch.equal(scan.prim, bp) and torch.equal(scan.scat, bs)
        scan.close()
    otp, ots, _, _ = oracle.mc_run(small, 55_555, seed=23, phi=float(angles[3]), angle_index=3, threads=NTH,
                                   local_majorant=True, cell_shift=2)
    np.testing.assert_array_equal(bp[3].cpu().numpy(), otp)
    np.testing.assert_array_equal(bs[3].cpu().numpy(), ots)


def test_autotune_keeps_the_option(gd, small):
    # the autotuner times lane-form configurations only and keeps the option
    with gd.Context(small) as ctx:
        gd.gdrr_set_options(ctx, local_majorant=1, cell_shift=2)
        ref = gd.gdrr_mc_project(ctx, 150_000, 8)
        best = gd.gdrr_autotune(ctx, 0.0, 200_000, 3)
        assert best["local_majorant"] == 1 and best["cell_shift"] == 2 and best["photon_pool"] == -1
        got = gd.gdrr_mc_project(ctx, 150_000, 8)
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])


def test_vacuum_cells_anisotropic_voxels_and_step_limit(gd, small):
    # cells of bound zero (vacuum) are crossed without spending depth; the
    # cell planes follow each axis's own voxel edge; a history that reaches
    # max_steps at a flight draw ends as the oracle's does
    import copy
    prob = copy.deepcopy(small)
    prob.density[prob.material == 0] = 0.0                  # air becomes vacuum
    prob.voxel = (4.0, 3.0, 5.0)
    n = 1500
    for shift in (1, 2):
        _same(_run(gd, prob, n, 41, phi=0.9, records=True, shift=shift), prob, n, 41, phi=0.9, records=True)
    _same(_run(gd, prob, 200_000, 43, phi=2.3, shift=2), prob, 200_000, 43, phi=2.3)
    st = _same(_run(gd, prob, 3000, 47, phi=0.2, records=True, shift=1, max_steps=2), prob, 3000, 47, phi=0.2,
               records=True, max_steps=2)
    assert st["step_limit"] > 0
