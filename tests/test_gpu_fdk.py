"""GPU FDK reconstruction and synthetic scans (Section 3.5) against the oracle.

The filter and backprojection run in FP32 on the GPU against the oracle's
FP64.  Tolerances: the filter sums at most nu/2 products of magnitude up to
max|q| / (2 tau) with FP32 rounding 6e-8 each, so 1e-5 max|q| / tau bounds
it; the backprojection sums n_views bilinear samples (FP32, positions good
to ~1e-5 pixel), so 1e-4 of the volume's largest magnitude bounds it.

The scan tests reproduce the paper's demonstrations on a synthetic water
cylinder with a bone rod: no cupping with a mono-energetic source, a cupping
artifact with a poly-energetic one (beam hardening, Fig. 9(a)-(b)), a lower
reconstruction when scatter enters (Fig. 9(c)), the ring shadow of scatter
behind a bowtie (Fig. 9(d)), and noise that scales as 1/sqrt(mAs) (Fig. 10).
Every view's scatter denoiser runs with a 4-pixel smoothing length (beta
from the view's mean count), inside the range where Eq. 5 converges.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import fdk as ofdk  # noqa: E402
from paper_1204_6367_gb300 import inputs  # noqa: E402
from test_oracle_fdk import SHADOW_EDGES, _ball_projections, radial_means, water_cylinder  # noqa: E402


@pytest.fixture(scope="module")
def gd():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_6367_gb300 import build, gdrr
    build.build()
    gdrr.lib()
    return gdrr


def _geo(gd, sad, sdd, nu, nv, du, dv, shape, vox):
    return gd.fdk_geometry(sad, sdd, nu, nv, du, dv, shape, vox)


@pytest.mark.parametrize("nu, nv", [(200, 12), (701, 5)])
def test_filter_matches_oracle(gd, nu, nv):
    rng = np.random.default_rng(nu)
    sad, sdd, du, dv = 1000.0, 1500.0, 0.9, 1.1
    g = rng.uniform(0.0, 3.0, (4, nv, nu)).astype(np.float32)
    geo = _geo(gd, sad, sdd, nu, nv, du, dv, (4, 4, 4), (1.0, 1.0, 1.0))
    got = gd.gdrr_fdk_filter(geo, torch.from_numpy(g).cuda()).cpu().numpy().astype(np.float64)
    ref = ofdk.fdk_filter(g.astype(np.float64), sad, sdd, du, dv)
    tau = du * sad / sdd
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5 * float(np.abs(g).max()) / tau)


def test_backprojection_matches_oracle(gd):
    # ragged grid against the 32 x 8 x 8 tiles, 150 views (two launches),
    # unequally spaced angles, an arbitrary view weight
    rng = np.random.default_rng(3)
    sad, sdd, nu, nv, du, dv = 800.0, 1300.0, 96, 40, 1.3, 1.7
    shape, vox = (13, 20, 37), (1.7, 2.1, 2.3)
    n = 150
    angles = np.sort(rng.uniform(0.0, 2.0 * math.pi, n))
    q = rng.normal(0.0, 1.0, (n, nv, nu)).astype(np.float32)
    geo = _geo(gd, sad, sdd, nu, nv, du, dv, shape, vox)
    got = gd.gdrr_fdk_backproject(geo, torch.from_numpy(q).cuda(), angles, d_beta=0.037).cpu().numpy()
    ref = ofdk.fdk_backproject(q.astype(np.float64), angles, 0.037, sad, sdd, du, dv, shape, vox)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-4 * float(np.abs(ref).max()))


def test_backprojection_in_batches_equals_one_call(gd):
    rng = np.random.default_rng(4)
    sad, sdd, nu, nv, du, dv = 1000.0, 1500.0, 64, 24, 2.0, 2.0
    shape, vox = (10, 30, 30), (2.0, 2.0, 2.0)
    n = 200
    angles = np.arange(n) * (2.0 * math.pi / n)
    q = torch.from_numpy(rng.normal(0.0, 1.0, (n, nv, nu)).astype(np.float32)).cuda()
    geo = _geo(gd, sad, sdd, nu, nv, du, dv, shape, vox)
    one = gd.gdrr_fdk_backproject(geo, q, angles, d_beta=0.01)
    vol = gd.gdrr_fdk_backproject(geo, q[:128].contiguous(), angles[:128], d_beta=0.01)
    gd.gdrr_fdk_backproject(geo, q[128:].contiguous(), angles[128:], d_beta=0.01, volume=vol, accumulate=True)
    assert torch.equal(one, vol)


def test_ball_reconstruction_matches_oracle(gd):
    sad, sdd = 1000.0, 1500.0
    nu, nv, du, dv = 128, 64, 1.6, 1.6
    n_proj = 180
    angles = np.arange(n_proj) * (2.0 * math.pi / n_proj)
    centre, radius, mu = (12.0, -6.0, 8.0), 25.0, 0.02
    g = _ball_projections(angles, sad, sdd, nu, nv, du, dv, centre, radius, mu)
    shape, vox = (32, 48, 48), (2.0, 2.0, 2.0)
    geo = _geo(gd, sad, sdd, nu, nv, du, dv, shape, vox)
    got = gd.fdk(geo, torch.from_numpy(g.astype(np.float32)).cuda(), angles).cpu().numpy()
    ref = ofdk.fdk(g.astype(np.float32).astype(np.float64), angles, sad, sdd, du, dv, shape, vox)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-4 * float(np.abs(ref).max()))


def test_air_scan_and_line_integrals(gd):
    for hardened in (False, True):
        prob = inputs.torso_problem(vox=8.0, seed=3, nu=64, nv=48, det_px=6.208, hardened_bowtie=hardened)
        empty = inputs.torso_problem(vox=8.0, seed=3, nu=64, nv=48, det_px=6.208, hardened_bowtie=hardened)
        empty.density[:] = 0.0
        with gd.Context(prob) as ctx:
            I0 = gd.gdrr_air_scan(ctx)
            P = gd.gdrr_raytrace_primary(ctx, 0.4)
            g = gd.gdrr_line_integrals(P, I0, 1e-6).cpu().numpy()
            I0 = I0.cpu().numpy()
        np.testing.assert_allclose(I0, oracle.rt_primary(empty, phi=0.0), rtol=1e-6)
        ref = ofdk.line_integrals(P.cpu().numpy(), I0, 1e-6)
        np.testing.assert_allclose(g, ref, rtol=1e-6, atol=1e-6)


def _cylinder(poly):
    p = inputs.small_problem(n_vox=64, vox=2.0, n_det=128, det_px=2.0)
    if poly:
        p.spec_e, p.spec_w = inputs.kramers_spectrum(kvp=100.0, bin_kev=2.0)
    return p


def _regions():
    c = (np.arange(64) + 0.5 - 32) * 2.0
    Y, X = np.meshgrid(c, c, indexing="ij")
    r = np.hypot(X, Y)
    centre = r < 10.0
    periphery = (r > 35.0) & (r < 45.0) & ~((X > 5.0) & (np.abs(Y) < 20.0))    # away from the bone rod
    return centre, periphery


def test_scan_beam_hardening_and_scatter(gd):
    from paper_1204_6367_gb300 import scan
    centre, periphery = _regions()
    out = {}
    for name, poly, comp in (("mono", False, "P"), ("poly", True, "P"), ("poly_ps", True, "PS")):
        prob = _cylinder(poly)
        with gd.Context(prob) as ctx:
            angles, sig = scan.scan(ctx, 90, comp, n_photons=2_000_000, seed=5, bin_factor=4, iters=1000,
                                    smoothing_px=4.0)
            vol = scan.reconstruct(ctx, angles, sig, prob.material.shape, prob.voxel).cpu().numpy()
        mid = vol[vol.shape[0] // 2]
        out[name] = (mid[centre].mean(), mid[periphery].mean())
    cup = {k: (v[1] - v[0]) / v[1] for k, v in out.items()}
    mu_w = float(_cylinder(False).mu_hat[1, :, 59].astype(np.float64).sum() * 0.1)
    assert out["mono"][0] == pytest.approx(mu_w, rel=0.01)
    assert abs(cup["mono"]) < 0.005                 # no cupping without beam hardening
    assert cup["poly"] > 0.015                      # beam hardening cups the water (Fig. 9(b))
    assert out["poly_ps"][0] < 0.99 * out["poly"][0]   # scatter lowers the reconstruction (Fig. 9(c))


def test_scan_noise_scales_with_mas(gd):
    from paper_1204_6367_gb300 import scan
    centre, _ = _regions()
    prob = _cylinder(False)
    sig = {}
    with gd.Context(prob) as ctx:
        # the paper's zeta (Section 3.3) gives alpha = sqrt(n_sim / (zeta mAs)) =
        # 0.019 at 0.1 mAs: noise of about 2 % of the signal, where -ln is close
        # to linear
        for mas in (0.1, 1.0):
            angles, s = scan.scan(ctx, 60, "PSN", n_photons=200_000, seed=9, mas=mas, zeta=5.2913e9, iters=1000,
                                  smoothing_px=4.0)
            sig[mas] = s
        _, s_ps = scan.scan(ctx, 60, "PS", n_photons=200_000, seed=9, iters=1000, smoothing_px=4.0)
        vols = {k: scan.reconstruct(ctx, angles, v, prob.material.shape, prob.voxel).cpu().numpy() for k, v in
                sig.items()}
        v_ps = scan.reconstruct(ctx, angles, s_ps, prob.material.shape, prob.voxel).cpu().numpy()
    z = vols[1.0].shape[0] // 2
    sd = {k: float((v[z] - v_ps[z])[centre].std()) for k, v in vols.items()}
    # the noise image scales as 1 / sqrt(mAs) (Section 2.6, Fig. 10)
    assert sd[0.1] / sd[1.0] == pytest.approx(math.sqrt(10.0), rel=0.05)


def test_denoised_view_converges_and_low_counts_warn(gd):
    prob = _cylinder(True)
    with gd.Context(prob) as ctx:
        r = gd.project(ctx, 2_000_000, 5, 0.3, iters=2000, smoothing_px=4.0)
        cs, beta = r["count_scale"], r["beta"]
        res = oracle.optimality_residual(r["S_coarse"].cpu().numpy() / cs, r["S_hat_coarse"].cpu().numpy() / cs, beta)
        assert np.abs(res).max() < 1e-6                     # Eq. 4 holds: the iteration converged
        # a fixed beta at a low count: beta * mean count far below the
        # stability floor omega / (8 (1 - omega)) = 0.5
        assert gd.denoise_stability_floor(0.8) == pytest.approx(0.5)
        with pytest.warns(RuntimeWarning, match="diverges"):
            gd.project(ctx, 200_000, 5, 0.3, beta=0.02, iters=50)


def test_scan_scatter_shadow_follows_the_bowtie(gd):
    # the full orbit through the library (independent streams per view)
    from paper_1204_6367_gb300 import scan
    deficit = {}
    for bowtie in (0.0, 30.0):
        prob = water_cylinder(bowtie)
        with gd.Context(prob) as ctx:
            vol = {}
            for comp in ("P", "PS"):
                angles, sig = scan.scan(ctx, 90, comp, n_photons=2_000_000, seed=3, iters=1500, smoothing_px=4.0)
                v = scan.reconstruct(ctx, angles, sig, prob.material.shape, prob.voxel).cpu().numpy()
                vol[comp] = radial_means(v[v.shape[0] // 2], 2.0, 64, SHADOW_EDGES)
        deficit[bowtie] = vol["P"] - vol["PS"]
    centre, middle, ring = deficit[0.0]
    assert centre > 1.1 * middle > 1.2 * ring > 0                 # no bowtie: cupping, deepest at the centre
    centre, middle, ring = deficit[30.0]
    assert ring > 1.3 * middle and ring > 2.5 * abs(centre)       # bowtie: the shadow is a ring (Fig. 9(d))
