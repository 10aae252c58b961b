"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer outputs (random words, int64 tallies, transport counters, per-history
event records) must match the oracle's FP32 transport bit for bit: both sides
perform the same IEEE operations in the same order.  The ray-traced primary
is FP32 on the GPU against an FP64 oracle: tolerance 2e-4 relative.  The
path integrals (up to ~1000 midpoints) are summed in FP32, about 1e-5
relative; the midpoints carry ~1e-4 mm of FP32 position error 1.5 m from the
source; a radiological length of at most ~10 turns both into at most 1e-4
relative through exp(-x).  Image-domain steps are FP64 on both sides: 1e-15
to 1e-13 for single operations, 1e-11 for the Eq. 5 iteration (hundreds of
contracting sweeps, each adding a rounding).
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
RT_RTOL = 2e-4


@pytest.fixture(scope="module")
def gd():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_6367_gb300 import build, gdrr
    build.build()
    gdrr.lib()
    return gdrr


def _run_gpu(gd, prob, n, seed, phi=0.0, angle_index=0, offset=0, records=False, **opts):
    with gd.Context(prob) as ctx:
        if opts:
            gd.gdrr_set_options(ctx, **opts)
        stats = torch.zeros(gd.GDRR_NSTATS, dtype=torch.int64, device="cuda")
        rec = torch.zeros(n * gd.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda") if records else None
        prim, scat = gd.gdrr_mc_project(ctx, n, seed, phi, angle_index, offset, stats=stats, records=rec)
        gd.gdrr_sync(ctx)
        return (prim.cpu().numpy(), scat.cpu().numpy(), gd.stats_dict(stats),
                gd.records_array(rec) if records else None)


def test_stream_words_bit_exact(gd):
    for seed, a, h0 in [(1, 0, 0), (0xFEDCBA9876543210, 63, (1 << 32) - 3), (12345, 7, 10**12)]:
        w = gd.gdrr_stream_words(seed, a, h0, 64, 3).cpu().numpy().view(np.uint32)
        torch.cuda.synchronize()
        ref = np.stack([oracle.stream_words(seed, a, h0 + i, 3) for i in range(64)])
        np.testing.assert_array_equal(w, ref)


def test_tiny_run_event_by_event(gd, small):
    n = 1000
    tp, ts, st, rec = _run_gpu(gd, small, n, seed=1, records=True)
    otp, ots, ost, orec = oracle.mc_run(small, n, seed=1, records=True)
    for f in oracle.RECORD_DTYPE.names:
        np.testing.assert_array_equal(rec[f], orec[f], err_msg=f)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)


@pytest.mark.parametrize("phi", [0.0, 1.1])
def test_small_problem_1e6_bit_exact(gd, small, phi):
    n = 1_000_000
    tp, ts, st, _ = _run_gpu(gd, small, n, seed=3, phi=phi, angle_index=5)
    otp, ots, ost, _ = oracle.mc_run(small, n, seed=3, phi=phi, angle_index=5, threads=NTH)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)


def test_torso_4mm_polyenergetic_bit_exact(gd):
    prob = inputs.torso_problem(vox=4.0, nu=128, nv=96, det_px=0.776 * 4)
    n = 300_000
    tp, ts, st, _ = _run_gpu(gd, prob, n, seed=11, phi=0.4, angle_index=2)
    otp, ots, ost, _ = oracle.mc_run(prob, n, seed=11, phi=0.4, angle_index=2, threads=NTH)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)


@pytest.mark.parametrize("opts", [dict(photon_pool=-1, block_size=64, hist_per_thread=1, batch_min=1),
                                  dict(photon_pool=-1, block_size=128, hist_per_thread=64, batch_min=32),
                                  dict(photon_pool=-1, block_size=256, hist_per_thread=3, batch_min=3,
                                       blocks_per_sm=1),
                                  dict(photon_pool=-1, block_size=512, hist_per_thread=8, batch_min=20),
                                  dict(photon_pool=1, hist_per_thread=1),
                                  dict(photon_pool=3, hist_per_thread=64),
                                  dict(photon_pool=2, hist_per_thread=5, blocks_per_sm=1)])
def test_launch_configuration_invariance(gd, small, opts):
    n = 200_003
    ref = _run_gpu(gd, small, n, seed=5)
    got = _run_gpu(gd, small, n, seed=5, **opts)
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[1])
    assert got[2] == ref[2]


def test_split_and_accumulate(gd, small):
    n, k = 300_000, 123_457
    with gd.Context(small) as ctx:
        full = gd.gdrr_mc_project(ctx, n, 9)
        a_p, a_s = gd.gdrr_mc_project(ctx, k, 9)
        gd.gdrr_mc_project(ctx, n - k, 9, history_offset=k, prim=a_p, scat=a_s)
        gd.gdrr_sync(ctx)
        assert torch.equal(full[0], a_p) and torch.equal(full[1], a_s)


def test_source_pass_segments_and_inline_start_agree(gd, small):
    """With default options the transport starts histories from the source
    pass's records, in passes of at most 2^27 histories.  A call of 1.5e8
    histories takes two passes; the same histories split at another point
    (two calls) and a call whose histories start inline (records requested)
    give the same tallies and counters."""
    n, k = 150_000_000, 90_000_000
    with gd.Context(small) as ctx:
        s_full = torch.zeros(gd.GDRR_NSTATS, dtype=torch.int64, device="cuda")
        full = gd.gdrr_mc_project(ctx, n, 5, stats=s_full)
        s_split = torch.zeros(gd.GDRR_NSTATS, dtype=torch.int64, device="cuda")
        a_p, a_s = gd.gdrr_mc_project(ctx, k, 5, stats=s_split)
        gd.gdrr_mc_project(ctx, n - k, 5, history_offset=k, prim=a_p, scat=a_s, stats=s_split)
        gd.gdrr_sync(ctx)
        assert torch.equal(full[0], a_p) and torch.equal(full[1], a_s)
        assert torch.equal(s_full, s_split)
        # inline starts (the records path) on a window of the same histories
        m = 200_000
        s_w = torch.zeros(gd.GDRR_NSTATS, dtype=torch.int64, device="cuda")
        w_p, w_s = gd.gdrr_mc_project(ctx, m, 5, history_offset=k - m // 2, stats=s_w)
        s_r = torch.zeros(gd.GDRR_NSTATS, dtype=torch.int64, device="cuda")
        rec = torch.zeros(m * gd.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        r_p, r_s = gd.gdrr_mc_project(ctx, m, 5, history_offset=k - m // 2, stats=s_r, records=rec)
        gd.gdrr_sync(ctx)
        assert torch.equal(w_p, r_p) and torch.equal(w_s, r_s) and torch.equal(s_w, s_r)


def test_zero_photons_is_a_noop(gd, small):
    with gd.Context(small) as ctx:
        p, s = gd.new_tallies(ctx)
        p += 5
        gd.gdrr_mc_project(ctx, 0, 1, prim=p, scat=s)
        gd.gdrr_sync(ctx)
        assert int(p.sum()) == 5 * p.numel() and int(s.abs().sum()) == 0


def test_edge_phantoms(gd):
    # one voxel; vacuum; eight materials; a single-pixel detector
    one = inputs.uniform_slab_problem(nx=1, ny=1, nz=1, vox=30.0, nu=5, nv=3, det_px=4.0, pencil=False)
    vac = inputs.uniform_slab_problem(mat_id=0, density=0.0, nu=7, nv=5, pencil=False)
    mats = [inputs.AIR, inputs.WATER, inputs.BONE, inputs.LUNG, inputs.ALUMINIUM,
            inputs.WATER, inputs.BONE, inputs.AIR]
    eight = inputs.uniform_slab_problem(nx=9, ny=8, nz=7, nu=6, nv=6, det_px=3.0, materials=mats, pencil=False)
    eight.material[:] = (np.arange(eight.material.size) % 8).reshape(eight.material.shape)
    eight.density[:] = np.linspace(0.1, 2.5, eight.density.size).reshape(eight.density.shape)
    single = inputs.uniform_slab_problem(nu=1, nv=1, det_px=2.0)
    for prob in (one, vac, eight, single):
        tp, ts, st, _ = _run_gpu(gd, prob, 20_000, seed=4, phi=0.3)
        otp, ots, ost, _ = oracle.mc_run(prob, 20_000, seed=4, phi=0.3, threads=NTH)
        assert st == ost
        np.testing.assert_array_equal(tp, otp)
        np.testing.assert_array_equal(ts, ots)


def test_step_limit_counted(gd, small):
    tp, ts, st, _ = _run_gpu(gd, small, 5000, seed=1, max_steps=2)
    otp, ots, ost, _ = oracle.mc_run(small, 5000, seed=1, max_steps=2)
    assert st == ost and st["step_limit"] > 0
    np.testing.assert_array_equal(tp, otp)


def test_batched_equals_per_angle(gd, small):
    angles = np.linspace(0, 2 * math.pi, 6, endpoint=False)
    budgets = np.array([3000, 0, 25_000, 1, 9_999, 40_000], np.uint64)
    with gd.Context(small) as ctx:
        bp, bs = gd.gdrr_mc_project_batched(ctx, angles, budgets, 17)
        for a in range(angles.size):
            p, s = gd.gdrr_mc_project(ctx, int(budgets[a]), 17, float(angles[a]), a)
            assert torch.equal(bp[a], p) and torch.equal(bs[a], s), a
    otp, ots, _, _ = oracle.mc_run(small, 9_999, seed=17, phi=float(angles[4]), angle_index=4, threads=NTH)
    np.testing.assert_array_equal(bp[4].cpu().numpy(), otp)
    np.testing.assert_array_equal(bs[4].cpu().numpy(), ots)


def test_raytrace_small(gd, small):
    with gd.Context(small) as ctx:
        for phi in (0.0, 0.9):
            P = gd.gdrr_raytrace_primary(ctx, phi).cpu().numpy()
            ref = oracle.rt_primary(small, phi=phi)
            np.testing.assert_allclose(P, ref, rtol=RT_RTOL, atol=1e-12 * ref.max())


def test_raytrace_torso_sampled(gd):
    # full-size 2 mm torso (512 x 384 detector): sampled pixels, the oracle's
    # per-channel FP64 trace against the GPU's per-material FP32 trace
    prob = inputs.torso_problem()
    rng = np.random.default_rng(0)
    pix = np.concatenate([rng.integers(0, prob.nu * prob.nv, 120), [0, prob.nu - 1, prob.nu * prob.nv - 1]])
    with gd.Context(prob) as ctx:
        for phi in (0.0, 1.3):
            P = gd.gdrr_raytrace_primary(ctx, phi).cpu().numpy().ravel()[pix]
            ref = oracle.rt_primary(prob, phi=phi, pixels=pix)
            np.testing.assert_allclose(P, ref, rtol=RT_RTOL, atol=1e-12 * ref.max())


def test_image_steps_match_oracle(gd, small):
    rng = np.random.default_rng(3)
    t = torch.from_numpy(rng.integers(0, 2**45, (64, 64), dtype=np.int64)).cuda()
    with gd.Context(small) as ctx:
        fin = gd.gdrr_finalize(ctx, t, 123456).cpu().numpy()
        np.testing.assert_allclose(fin, oracle.finalize(t.cpu().numpy(), 123456), rtol=1e-15)
        b = gd.gdrr_bin_tally(ctx, t, 4).cpu().numpy()
        np.testing.assert_array_equal(b, oracle.bin_tally(t.cpu().numpy(), 4))
        coarse = torch.from_numpy(rng.uniform(1, 100, (16, 16))).cuda()
        up = gd.gdrr_upsample(ctx, coarse, 4).cpu().numpy()
        np.testing.assert_allclose(up, oracle.upsample(coarse.cpu().numpy(), 4), rtol=1e-13)
        s_hat = torch.from_numpy(rng.poisson(500.0, (24, 32)).astype(np.float64) * 0.37).cuda()
        den = gd.gdrr_denoise_scatter(ctx, s_hat, 0.37, 0.02, 0.8, 400).cpu().numpy()
        ref = oracle.denoise(s_hat.cpu().numpy() / 0.37, 0.02, 0.8, 400) * 0.37
        np.testing.assert_allclose(den, ref, rtol=1e-11)
        a, p, c, d = (torch.from_numpy(rng.normal(size=(8, 8))).cuda() for _ in range(4))
        n = gd.gdrr_noise_calibrate(ctx, a, p, c, d, 10**8, 0.4, 5.2913e9).cpu().numpy()
        np.testing.assert_allclose(n, oracle.noise_scale(*(x.cpu().numpy() for x in (a, p, c, d)), 10**8, 0.4, 5.2913e9),
                                   rtol=1e-14)


def test_finalize_flags_overflow(gd, small):
    t = torch.tensor([1, -5, 3], dtype=torch.int64, device="cuda")
    with gd.Context(small) as ctx:
        with pytest.raises(gd.GdrrError) as e:
            gd.gdrr_finalize(ctx, t, 10)
        assert e.value.code == -4


def test_full_size_torso_sampled_windows(gd):
    # The 2 mm torso at 1e8 histories in the default launch configuration:
    # the full run equals the sum of its split parts, and history windows of
    # the same streams (start, middle, end) equal the oracle bit for bit.
    prob = inputs.torso_problem()
    n = 100_000_000
    with gd.Context(prob) as ctx:
        full_p, full_s = gd.gdrr_mc_project(ctx, n, 1)
        parts_p, parts_s = gd.new_tallies(ctx)
        for lo, hi in ((0, 37_000_000), (37_000_000, 81_234_567), (81_234_567, n)):
            gd.gdrr_mc_project(ctx, hi - lo, 1, history_offset=lo, prim=parts_p, scat=parts_s)
        gd.gdrr_sync(ctx)
        assert torch.equal(full_p, parts_p) and torch.equal(full_s, parts_s)
        for off in (0, 55_555_555, n - 40_000):
            wp, ws = gd.gdrr_mc_project(ctx, 40_000, 1, history_offset=off)
            otp, ots, _, _ = oracle.mc_run(prob, 40_000, seed=1, history_offset=off, threads=NTH)
            np.testing.assert_array_equal(wp.cpu().numpy(), otp)
            np.testing.assert_array_equal(ws.cpu().numpy(), ots)


def test_full_size_1mm_torso_sampled_windows(gd):
    # The 1 mm torso (512 x 512 x 256 voxels: 537 MB of records, beyond L2)
    # at 1e8 histories in the default launch configuration and macro cells:
    # history windows of the full run's streams (start, middle, end) equal
    # the oracle bit for bit, and the full run equals its split parts.
    prob = inputs.torso_problem(vox=1.0)
    n = 100_000_000
    with gd.Context(prob) as ctx:
        assert gd.gdrr_get_options(ctx)["cell_shift"] == 2          # 4 mm cells of 1 mm voxels
        full_p, full_s = gd.gdrr_mc_project(ctx, n, 3)
        parts_p, parts_s = gd.new_tallies(ctx)
        for lo, hi in ((0, 61_000_000), (61_000_000, n)):
            gd.gdrr_mc_project(ctx, hi - lo, 3, history_offset=lo, prim=parts_p, scat=parts_s)
        gd.gdrr_sync(ctx)
        assert torch.equal(full_p, parts_p) and torch.equal(full_s, parts_s)
        for off in (0, 42_424_242, n - 30_000):
            wp, ws = gd.gdrr_mc_project(ctx, 30_000, 3, history_offset=off)
            otp, ots, _, _ = oracle.mc_run(prob, 30_000, seed=3, history_offset=off, threads=NTH)
            np.testing.assert_array_equal(wp.cpu().numpy(), otp)
            np.testing.assert_array_equal(ws.cpu().numpy(), ots)


def _pooled(chunks):
    """Per-pixel estimate and variance of a tally summed over k independent
    chunks.  A tally is a compound-Poisson sum of deposits, Var = R * mean,
    with one dispersion ratio R per image pooled over well-filled pixels."""
    c = np.asarray(chunks, np.float64)
    m, v = c.mean(0), c.var(0, ddof=1)
    keep = m > np.percentile(m, 50)
    R = v[keep].sum() / m[keep].sum()
    tot = c.sum(0)
    return tot, tot * R


def test_statistical_agreement_with_fp64_oracle(gd, small):
    # Large-run statistics against the independent FP64 transport: >= 99.7 %
    # of pixels within 3 combined sigma, total scatter within 0.5 % (+3 sigma).
    n_g, k_g = 100_000_000, 20
    n_o, k_o = 40_000_000, 20
    with gd.Context(small) as ctx:
        cg_p, cg_s = [], []
        for i in range(k_g):
            p, s = gd.gdrr_mc_project(ctx, n_g // k_g, 1, history_offset=i * (n_g // k_g))
            cg_p.append(p.cpu().numpy()); cg_s.append(s.cpu().numpy())
    co_p, co_s = [], []
    for i in range(k_o):
        p, s, _, _ = oracle.mc_run(small, n_o // k_o, seed=77, history_offset=i * (n_o // k_o), precision=64,
                                   threads=NTH)
        co_p.append(p); co_s.append(s)
    for cg, co in ((cg_p, co_p), (cg_s, co_s)):
        tg, vg = _pooled(cg)
        to, vo = _pooled(co)
        g, o = tg / n_g, to / n_o
        var = vg / n_g**2 + vo / n_o**2
        keep = (tg > 0) | (to > 0)
        z = (g - o)[keep] / np.sqrt(var[keep])
        n_pix = z.size
        # 99.7 % within 3 sigma is the Gaussian expectation itself (99.73 %);
        # over n_pix pixels the observed fraction scatters binomially around
        # it, so allow its own 3-sigma band, and check the z distribution.
        frac = float(np.mean(np.abs(z) < 3.0))
        band = 3.0 * math.sqrt(0.0027 * 0.9973 / n_pix)
        assert frac >= 0.997 - band, (frac, band)
        assert abs(float(z.mean())) < 4.0 / math.sqrt(n_pix), float(z.mean())
        assert abs(float(z.std()) - 1.0) < 0.05, float(z.std())
    sg, so = np.sum(cg_s) / n_g, np.sum(co_s) / n_o
    sig = math.sqrt(_pooled(cg_s)[1].sum() / n_g**2 + _pooled(co_s)[1].sum() / n_o**2)
    assert abs(sg - so) <= 0.005 * so + 3 * sig, (sg, so, sig)


def _bin(t, f):
    nv, nu = t.shape
    return t.reshape(nv // f, f, nu // f, f).sum(axis=(1, 3))


def test_full_size_torso_statistical_agreement(gd, torso):
    # The headline workload (2 mm poly-energetic torso, 120 kVp, bowtie,
    # 512 x 384 detector): the FP32 GPU transport at 1e8 histories against the
    # independent FP64 oracle at 4e7 on the host cores, on other random
    # streams.  Per pixel: >= 99.7 % within 3 combined sigma (the binomial
    # band of reading 16) with mean z ~ 0 and sd(z) ~ 1; total scatter within
    # 0.5 % + 3 sigma.  The pixels are 8 x 8 bins of the detector (64 x 48):
    # at 4e7 histories the oracle leaves ~0.5 scattered photons per full-
    # resolution pixel, where a 3-sigma Gaussian band means nothing, and ~30
    # per bin.
    n_g, k_g = 100_000_000, 20
    n_o, k_o = 40_000_000, 20
    f = 8
    with gd.Context(torso) as ctx:
        gd.gdrr_autotune(ctx, 0.0, 10_000_000, 1)
        cg_p, cg_s = [], []
        for i in range(k_g):
            p, s = gd.gdrr_mc_project(ctx, n_g // k_g, 1, history_offset=i * (n_g // k_g))
            cg_p.append(_bin(p.cpu().numpy(), f)); cg_s.append(_bin(s.cpu().numpy(), f))
    co_p, co_s = [], []
    for i in range(k_o):
        p, s, _, _ = oracle.mc_run(torso, n_o // k_o, seed=77, history_offset=i * (n_o // k_o), precision=64,
                                   threads=NTH)
        co_p.append(_bin(p, f)); co_s.append(_bin(s, f))
    for cg, co in ((cg_p, co_p), (cg_s, co_s)):
        tg, vg = _pooled(cg)
        to, vo = _pooled(co)
        g, o = tg / n_g, to / n_o
        var = vg / n_g**2 + vo / n_o**2
        keep = (tg > 0) | (to > 0)
        z = (g - o)[keep] / np.sqrt(var[keep])
        n_pix = z.size
        assert n_pix > 2500
        frac = float(np.mean(np.abs(z) < 3.0))
        band = 3.0 * math.sqrt(0.0027 * 0.9973 / n_pix)
        assert frac >= 0.997 - band, (frac, band)
        assert abs(float(z.mean())) < 4.0 / math.sqrt(n_pix), float(z.mean())
        assert abs(float(z.std()) - 1.0) < 0.05, float(z.std())
    sg, so = np.sum(cg_s) / n_g, np.sum(co_s) / n_o
    sig = math.sqrt(_pooled(cg_s)[1].sum() / n_g**2 + _pooled(co_s)[1].sum() / n_o**2)
    assert abs(sg - so) <= 0.005 * so + 3 * sig, (sg, so, sig)


def test_scan_graph_replays_equal_batched(gd, small):
    angles = np.linspace(0, 2 * math.pi, 5, endpoint=False)
    budgets = np.array([20_000, 7, 0, 55_555, 31_000], np.uint64)
    with gd.Context(small) as ctx:
        bp, bs = gd.gdrr_mc_project_batched(ctx, angles, budgets, 23)
        scan = gd.gdrr_scan_create(ctx, angles, budgets, 23, zero_tallies=True)
        scan.launch()
        scan.launch()
        gd.gdrr_sync(ctx)
        assert torch.equal(scan.prim, bp) and torch.equal(scan.scat, bs)
        acc = gd.gdrr_scan_create(ctx, angles, budgets, 23, zero_tallies=False)
        acc.launch()
        acc.launch()
        gd.gdrr_sync(ctx)
        assert torch.equal(acc.prim, 2 * bp) and torch.equal(acc.scat, 2 * bs)
        scan.close()
        acc.close()


def test_autotune_keeps_results(gd, small):
    with gd.Context(small) as ctx:
        ref = gd.gdrr_mc_project(ctx, 150_000, 8)
        best = gd.gdrr_autotune(ctx, 0.0, 200_000, 3)
        assert best["block_size"] in (64, 128, 256, 512) and 8 <= best["batch_min"] <= 32
        assert best["photon_pool"] in (-1, 1, 2, 3)
        assert best["hist_per_thread"] in (1, 8, 64)
        assert gd.gdrr_get_options(ctx)["batch_min"] == best["batch_min"]
        got = gd.gdrr_mc_project(ctx, 150_000, 8)
        gd.gdrr_sync(ctx)
        assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])


def test_anisotropic_voxels_and_rotated_imager(gd):
    # voxels of 2 x 3 x 2.5 mm, imager turned by theta = 0.2 rad off the
    # source-opposite position, gantry at 0.8 rad
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0, nx=20, ny=14, nz=12, nu=40, nv=30, det_px=2.0,
                                       pencil=False)
    prob.voxel = (2.0, 3.0, 2.5)
    prob.theta = 0.2
    rng = np.random.default_rng(8)
    prob.material[:] = rng.integers(0, 3, prob.material.shape).astype(np.uint8)
    prob.density[:] = rng.uniform(0.05, 2.0, prob.density.shape).astype(np.float32)
    tp, ts, st, _ = _run_gpu(gd, prob, 300_000, seed=19, phi=0.8, angle_index=3)
    otp, ots, ost, _ = oracle.mc_run(prob, 300_000, seed=19, phi=0.8, angle_index=3, threads=NTH)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)
    with gd.Context(prob) as ctx:
        P = gd.gdrr_raytrace_primary(ctx, 0.8).cpu().numpy()
        Ps = gd.gdrr_raytrace_primary_siddon(ctx, 0.8).cpu().numpy()
    ref = oracle.rt_primary(prob, phi=0.8)
    refs = oracle.rt_primary_siddon(prob, phi=0.8)
    np.testing.assert_allclose(P, ref, rtol=RT_RTOL, atol=1e-12 * ref.max())
    np.testing.assert_allclose(Ps, refs, rtol=RT_RTOL, atol=1e-12 * refs.max())


def test_hardened_bowtie_columns(gd):
    # per-column spectra behind an aluminium bowtie: the source energy depends
    # on the detector column the photon heads for
    prob = inputs.torso_problem(vox=8.0, seed=3, kvp=120.0, nu=64, nv=48, det_px=6.208, hardened_bowtie=True)
    assert prob.spec_cols is not None
    tp, ts, st, _ = _run_gpu(gd, prob, 400_000, seed=31, phi=1.1, angle_index=2)
    otp, ots, ost, _ = oracle.mc_run(prob, 400_000, seed=31, phi=1.1, angle_index=2, threads=NTH)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)
    with gd.Context(prob) as ctx:
        P = gd.gdrr_raytrace_primary(ctx, 1.1).cpu().numpy()
        Ps = gd.gdrr_raytrace_primary_siddon(ctx, 1.1).cpu().numpy()
    ref = oracle.rt_primary(prob, phi=1.1)
    refs = oracle.rt_primary_siddon(prob, phi=1.1)
    np.testing.assert_allclose(P, ref, rtol=RT_RTOL, atol=1e-12 * ref.max())
    np.testing.assert_allclose(Ps, refs, rtol=RT_RTOL, atol=1e-12 * refs.max())


def test_single_bin_columns_event_by_event(gd):
    # one energy per column: every record's source energy is fixed by its column
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0, nx=16, ny=16, nz=8, nu=24, nv=6, det_px=1.2,
                                       pencil=False)
    e, _ = inputs.kramers_spectrum(kvp=100.0, bin_kev=5.0)
    prob.spec_e, prob.spec_w = e, np.ones(e.size) / e.size
    cols = np.zeros((prob.nu, e.size))
    cols[np.arange(prob.nu), (np.arange(prob.nu) * 5) % e.size] = 1.0
    prob.spec_cols = cols
    n = 5000
    tp, ts, st, rec = _run_gpu(gd, prob, n, seed=4, records=True)
    otp, ots, ost, orec = oracle.mc_run(prob, n, seed=4, records=True)
    for f in oracle.RECORD_DTYPE.names:
        np.testing.assert_array_equal(rec[f], orec[f], err_msg=f)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)


@pytest.mark.parametrize("nearest", [False, True])
def test_rayleigh_form_factor_event_by_event(gd, small, nearest):
    # form-factor Rayleigh angles and the per-corner material pick, history by history
    n = 3000
    tp, ts, st, rec = _run_gpu(gd, small, n, seed=23, phi=0.5, records=True, rayleigh_form_factor=1,
                               nearest_voxel=int(nearest))
    otp, ots, ost, orec = oracle.mc_run(small, n, seed=23, phi=0.5, records=True, rayleigh_ff=True,
                                        nearest_voxel=nearest)
    for f in oracle.RECORD_DTYPE.names:
        np.testing.assert_array_equal(rec[f], orec[f], err_msg=f)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)
    assert np.any(rec["ray_material"] > 0)


def test_rayleigh_form_factor_mixture_bit_exact(gd):
    # water / bone checkerboard: every Rayleigh event meets a mixture of materials
    prob = inputs.uniform_slab_problem(mat_id=1, nx=16, ny=16, nz=16, nu=32, nv=32, det_px=1.0, pencil=False)
    z, y, x = np.indices(prob.material.shape)
    prob.material[:] = (1 + (x + y + z) % 2).astype(np.uint8)
    tp, ts, st, _ = _run_gpu(gd, prob, 1_000_000, seed=29, rayleigh_form_factor=1)
    otp, ots, ost, _ = oracle.mc_run(prob, 1_000_000, seed=29, threads=NTH, rayleigh_ff=True)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)


def test_rayleigh_form_factor_narrows_single_rayleigh_scatter(gd):
    # pencil beam through water, single-Rayleigh scatter only: the detector
    # (128 mm at 500 mm behind the slab) sees scattering angles below ~7 deg;
    # the form factor puts most Rayleigh events there, Thomson spreads them
    # over the sphere
    prob = inputs.uniform_slab_problem(mat_id=1, nx=16, ny=16, nz=16, nu=64, nv=64, det_px=2.0)
    n = 4_000_000
    _, _, st_ff, _ = _run_gpu(gd, prob, n, seed=37, rayleigh_form_factor=1, scatter_filter=2)
    _, _, st_th, _ = _run_gpu(gd, prob, n, seed=37, scatter_filter=2)
    assert st_th["tally_scatter"] > 100
    assert st_ff["tally_scatter"] > 20 * st_th["tally_scatter"], (st_ff, st_th)


def test_rayleigh_form_factor_option_checks(gd, small):
    prob = inputs.small_problem()
    prob.form_factor = None
    with gd.Context(prob) as ctx:
        with pytest.raises(gd.GdrrError):
            gd.gdrr_set_options(ctx, rayleigh_form_factor=1)
        x = 0.01 * np.arange(500)       # reaches 4.99 1/Angstrom; 150 keV backscatter needs 12.1
        with pytest.raises(gd.GdrrError):
            gd.gdrr_set_form_factor(ctx, np.stack([inputs.form_factor(m, x) for m in
                                                   (inputs.AIR, inputs.WATER, inputs.BONE)]), 0.01)
        gd.gdrr_set_form_factor(ctx, small.form_factor, small.ff_dx)
        gd.gdrr_set_options(ctx, rayleigh_form_factor=1)
        with pytest.raises(gd.GdrrError):
            gd.gdrr_set_form_factor(ctx, None, 0.0)      # refused while the option is on


def test_create_rejects_bad_voxels(gd, small):
    # voxel validation runs in the device staging kernel
    bad_mat = small.material.copy()
    bad_mat[0, 0, 0] = 7
    neg = small.density.copy()
    neg[1, 2, 3] = -1.0
    nan = small.density.copy()
    nan[0, 0, 1] = np.nan
    inf = small.density.copy()
    inf[5, 5, 5] = np.inf
    for field, arr in (("material", bad_mat), ("density", neg), ("density", nan), ("density", inf)):
        prob = inputs.small_problem()
        setattr(prob, field, arr)
        with pytest.raises(gd.GdrrError) as ei:
            gd.Context(prob)
        assert ei.value.code == -1
    with gd.Context(inputs.small_problem()) as ctx:       # the device is still usable
        assert gd.gdrr_raytrace_primary(ctx, 0.0).sum().item() > 0


def test_eight_materials_at_512_threads(gd):
    # 8 materials x 512 threads need 48 KB of per-thread coefficients: above the
    # default dynamic shared-memory cap, which the launch raises
    prob = inputs.uniform_slab_problem(mat_id=1, nx=12, ny=12, nz=12, nu=24, nv=24, det_px=3.0, pencil=False,
                                       materials=[inputs.AIR, inputs.WATER, inputs.BONE, inputs.LUNG,
                                                  inputs.ALUMINIUM, inputs.WATER, inputs.BONE, inputs.LUNG])
    rng = np.random.default_rng(21)
    prob.material[:] = rng.integers(0, 8, prob.material.shape).astype(np.uint8)
    prob.density[:] = rng.uniform(0.1, 2.0, prob.density.shape).astype(np.float32)
    prob.form_factor = None
    n = 100_000
    ref = oracle.mc_run(prob, n, seed=3, threads=NTH)
    # the lane form at 512 threads, and the pool form (8 materials: its largest pool)
    for opts in (dict(block_size=512, photon_pool=-1), dict(photon_pool=3), dict(photon_pool=1)):
        got = _run_gpu(gd, prob, n, seed=3, **opts)
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_array_equal(got[1], ref[1])
        assert got[2] == ref[2]


def test_roofline_probes(gd):
    # the machine ceilings the bench reports the transport against
    l2 = gd.gdrr_probe_l2_gather(32 << 20)
    fp32 = gd.gdrr_probe_fp32()
    assert 100.0 < l2 < 50_000.0          # GB/s of 8-byte words
    assert 5.0 < fp32 < 500.0             # TFLOP/s
    with pytest.raises(gd.GdrrError):
        gd.gdrr_probe_l2_gather(1 << 10)  # below the 1 MiB minimum


def test_maximum_bins_and_materials(gd):
    # 512 spectrum channels (the library's limit) with 8 materials: transport
    # bit-exact, both ray tracers within tolerance
    mats = [inputs.AIR, inputs.WATER, inputs.BONE, inputs.LUNG, inputs.ALUMINIUM,
            inputs.WATER, inputs.BONE, inputs.LUNG]
    prob = inputs.uniform_slab_problem(nx=10, ny=9, nz=8, nu=12, nv=10, det_px=3.0, materials=mats, pencil=False)
    rng = np.random.default_rng(5)
    prob.material[:] = rng.integers(0, 8, prob.material.shape).astype(np.uint8)
    prob.density[:] = rng.uniform(0.05, 2.5, prob.density.shape).astype(np.float32)
    prob.spec_e = np.linspace(10.25, 139.75, 512)
    prob.spec_w = rng.uniform(0.1, 1.0, 512)
    prob.form_factor = None
    tp, ts, st, _ = _run_gpu(gd, prob, 100_000, seed=8, phi=2.0)
    otp, ots, ost, _ = oracle.mc_run(prob, 100_000, seed=8, phi=2.0, threads=NTH)
    assert st == ost
    np.testing.assert_array_equal(tp, otp)
    np.testing.assert_array_equal(ts, ots)
    with gd.Context(prob) as ctx:
        P = gd.gdrr_raytrace_primary(ctx, 2.0).cpu().numpy()
        Ps = gd.gdrr_raytrace_primary_siddon(ctx, 2.0).cpu().numpy()
    np.testing.assert_allclose(P, oracle.rt_primary(prob, phi=2.0), rtol=RT_RTOL)
    np.testing.assert_allclose(Ps, oracle.rt_primary_siddon(prob, phi=2.0), rtol=RT_RTOL)
    prob.spec_e = np.linspace(10.25, 139.75, 513)
    prob.spec_w = np.ones(513)
    with pytest.raises(gd.GdrrError) as ei:
        gd.Context(prob)
    assert ei.value.code == -6


def _run_cells(gd, prob, n, seed, phi, shift, records=False):
    with gd.Context(prob) as ctx:
        gd.gdrr_set_options(ctx, cell_shift=shift)
        assert gd.gdrr_get_options(ctx)["cell_shift"] == shift
        stats = torch.zeros(gd.GDRR_NSTATS, dtype=torch.int64, device="cuda")
        rec = torch.zeros(n * gd.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda") if records else None
        prim, scat = gd.gdrr_mc_project(ctx, n, seed, phi, 0, 0, stats=stats, records=rec)
        gd.gdrr_sync(ctx)
        return (prim.cpu().numpy(), scat.cpu().numpy(), gd.stats_dict(stats), gd.cell_skips(stats),
                gd.records_array(rec) if records else None)


def _cell_problem(which):
    if which == "torso":                                   # 4 material slots
        return inputs.torso_problem(vox=4.0, nu=128, nv=96, det_px=0.776 * 4)
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


@pytest.mark.parametrize("which", ["two", "torso", "eight"])
def test_cell_bound_changes_no_decision(gd, which):
    # the macro-cell test skips the corner gathers only of collisions that
    # are virtual anyway: every event record, counter and tally is the same
    # with cells of 2, 8 or 64 voxels and without the test, and the oracle's
    prob = _cell_problem(which)
    n, seed, phi = 1500, 21, 0.7
    base = _run_cells(gd, prob, n, seed, phi, -1, records=True)
    assert base[3] == 0
    otp, ots, ost, orec = oracle.mc_run(prob, n, seed=seed, phi=phi, records=True)
    for f in oracle.RECORD_DTYPE.names:
        np.testing.assert_array_equal(base[4][f], orec[f], err_msg=f)
    assert base[2] == ost
    np.testing.assert_array_equal(base[0], otp)
    np.testing.assert_array_equal(base[1], ots)
    for shift in (1, 3, 6):
        got = _run_cells(gd, prob, n, seed, phi, shift, records=True)
        for f in gd.RECORD_DTYPE.names:
            np.testing.assert_array_equal(got[4][f], base[4][f], err_msg=f"{f} at cell_shift {shift}")
        assert got[2] == base[2]
        np.testing.assert_array_equal(got[0], base[0])
        np.testing.assert_array_equal(got[1], base[1])
    off = _run_cells(gd, prob, 200_000, 5, 2.1, -1)
    on = _run_cells(gd, prob, 200_000, 5, 2.1, 3)
    np.testing.assert_array_equal(on[0], off[0])
    np.testing.assert_array_equal(on[1], off[1])
    assert on[2] == off[2] and off[3] == 0
    assert 0 < on[3] <= on[2]["virtual"]


def test_cell_bound_skips_most_virtual_collisions_in_the_torso(gd):
    # the torso's majorant is set by dense bone; in air, lung and soft-tissue
    # cells most tentative collisions lie above the cell's bound
    prob = inputs.torso_problem(vox=4.0, nu=128, nv=96, det_px=0.776 * 4)
    _, _, st, skips, _ = _run_cells(gd, prob, 300_000, 9, 0.2, 3)
    assert skips > 0.6 * st["virtual"]


def test_cell_shift_option_checks(gd, small):
    # the default cells are about 4 mm: 2 voxels of 2 mm, 4 of 1 mm, 8 of 0.5 mm
    # (at least 2 voxels: 8 mm at 4 mm voxels)
    for vox, shift in ((4.0, 1), (2.0, 1), (1.0, 2), (0.5, 3)):
        prob = inputs.uniform_slab_problem(nx=8, ny=8, nz=8, vox=vox)
        with gd.Context(prob) as ctx:
            assert gd.gdrr_get_options(ctx)["cell_shift"] == shift
    with gd.Context(small) as ctx:
        for bad in (-2, 7):
            with pytest.raises(gd.GdrrError):
                gd.gdrr_set_options(ctx, cell_shift=bad)
        gd.gdrr_set_options(ctx, cell_shift=5)
        gd.gdrr_set_options(ctx, cell_shift=0)                     # zero: the default
        assert gd.gdrr_get_options(ctx)["cell_shift"] == 1


def test_negative_zero_density_is_zero(gd):
    # a density of -0 is a density of zero: staged as +0, it neither lowers a
    # material's largest density (the majorant) nor the cell table
    prob = _cell_problem("two")
    prob.density[5, 5, 10] = 0.0                                   # a bone voxel
    neg = _cell_problem("two")
    neg.density[5, 5, 10] = -0.0
    assert np.signbit(neg.density[5, 5, 10])
    n = 100_000
    a = _run_cells(gd, prob, n, 3, 0.4, 3)
    b = _run_cells(gd, neg, n, 3, 0.4, 3)
    otp, ots, ost, _ = oracle.mc_run(neg, n, seed=3, phi=0.4, threads=NTH)
    for got in (a, b):
        assert got[2] == ost
        np.testing.assert_array_equal(got[0], otp)
        np.testing.assert_array_equal(got[1], ots)
