"""Pins of the oracle's FDK reconstruction (the cone-beam reconstruction that
Section 3.5 applies to simulated scans).

* The Ram-Lak kernel's discrete-time Fourier transform is |f| inside the
  Nyquist band (Kak & Slaney): the filter's shape and scale.
* A uniform ball, projected analytically (exact chords), reconstructs to its
  attenuation coefficient inside, to zero outside, at its own position (an
  off-centre ball catches mirrored axes and wrong rotation senses) and with
  its own radius.
* Scans the oracle's ray tracer computes (Section 2.3) of the water cylinder
  with an off-axis bone rod, mono-energetic, reconstruct to mu(60 keV) of
  water and of bone at the places the phantom puts them: the projection
  geometry and the reconstruction geometry agree.
* Scatter artifacts (Section 3.5, Fig. 9(c)-(d)): on a centred water
  cylinder, 100 kVp, the denoised Monte Carlo scatter lowers the
  reconstruction most at the centre without a bowtie (cupping), while behind
  a bowtie the centre is spared and the deficit moves out to a ring near the
  periphery: the ring shadow the paper traces to the interplay of scatter and
  bowtie.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import fdk
from paper_1204_6367_gb300 import inputs


def _ball_projections(angles, sad, sdd, nu, nv, du, dv, centre, radius, mu):
    """Exact line integrals mu * chord through a ball, at pixel centres."""
    c = np.asarray(centre, np.float64)
    out = np.zeros((len(angles), nv, nu))
    u = (np.arange(nu) + 0.5 - 0.5 * nu) * du
    v = (np.arange(nv) + 0.5 - 0.5 * nv) * dv
    V, U = np.meshgrid(v, u, indexing="ij")
    for i, phi in enumerate(angles):
        n = np.array([math.cos(phi), math.sin(phi), 0.0])
        eu = np.array([math.sin(phi), -math.cos(phi), 0.0])
        S = -sad * n
        C = (sdd - sad) * n[None, None, :] + U[..., None] * eu + V[..., None] * np.array([0.0, 0.0, 1.0])
        d = C - S
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        w = c - S
        t0 = d @ w
        dist2 = w @ w - t0 * t0
        out[i] = mu * 2.0 * np.sqrt(np.maximum(radius * radius - dist2, 0.0))
    return out


def test_ramp_kernel_is_the_band_limited_ramp():
    tau = 0.7
    n = 20001
    h = fdk.ramp_kernel(n, tau)
    k = np.arange(-(n - 1), n)
    for f in (0.02 / tau, 0.1 / tau, 0.3 / tau, 0.49 / tau):
        H = tau * np.sum(h * np.cos(2.0 * math.pi * f * k * tau))
        assert H == pytest.approx(f, rel=1e-6)
    assert abs(tau * h.sum()) < 1e-4 / tau          # no DC response
    assert np.all(h[k % 2 == 0][k[k % 2 == 0] != 0] == 0.0)


def test_uniform_ball_reconstructs_in_place():
    sad, sdd = 1000.0, 1500.0
    nu, nv, du, dv = 128, 64, 1.6, 1.6
    n_proj = 180
    angles = np.arange(n_proj) * (2.0 * math.pi / n_proj)
    centre, radius, mu = (12.0, -6.0, 8.0), 25.0, 0.02
    g = _ball_projections(angles, sad, sdd, nu, nv, du, dv, centre, radius, mu)
    shape, vox = (32, 48, 48), (2.0, 2.0, 2.0)
    f = fdk.fdk(g, angles, sad, sdd, du, dv, shape, vox)
    nz, ny, nx = shape
    x = (np.arange(nx) + 0.5 - 0.5 * nx) * vox[0]
    y = (np.arange(ny) + 0.5 - 0.5 * ny) * vox[1]
    z = (np.arange(nz) + 0.5 - 0.5 * nz) * vox[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    inside = r < 0.6 * radius
    outside = (r > 1.3 * radius) & (np.abs(Z) < 20.0)
    assert f[inside].mean() == pytest.approx(mu, rel=0.01)
    assert f[inside].std() < 0.03 * mu
    assert abs(f[outside].mean()) < 0.02 * mu
    # position: centroid of the thresholded ball; size: the volume above mu/2
    m = f > 0.5 * mu
    cen = [float((X * m).sum() / m.sum()), float((Y * m).sum() / m.sum()), float((Z * m).sum() / m.sum())]
    np.testing.assert_allclose(cen, centre, atol=0.5)
    r_eq = (m.sum() * np.prod(vox) * 3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
    assert r_eq == pytest.approx(radius, abs=1.0)


def test_ray_traced_scan_reconstructs_the_phantom():
    prob = inputs.small_problem()
    air = inputs.small_problem()
    air.density[:] = 0.0
    n_proj = 90
    angles = np.arange(n_proj) * (2.0 * math.pi / n_proj)
    I0 = oracle.rt_primary(air, phi=0.0)
    g = np.stack([fdk.line_integrals(oracle.rt_primary(prob, phi=float(a)), I0) for a in angles])
    nz, ny, nx = prob.material.shape
    f = fdk.fdk(g, angles, prob.sad, prob.sdd, prob.du, prob.dv, (nz, ny, nx), prob.voxel)
    mu60 = prob.mu_hat[:, :, 59].astype(np.float64).sum(axis=1) * 0.1      # 1/mm per g/cm^3
    mid = f[nz // 2]
    mat = prob.material[nz // 2]
    rho = prob.density[nz // 2].astype(np.float64)

    def interior(mask):
        # voxels whose 8 in-plane neighbours share the material (away from edges)
        m = mask.copy()
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                m &= np.roll(np.roll(mask, dy, 0), dx, 1)
        return m

    water, bone = interior(mat == 1), interior(mat == 2)
    assert water.sum() > 50 and bone.sum() >= 4
    assert mid[water].mean() == pytest.approx(float((mu60[1] * rho[water]).mean()), rel=0.03)
    assert mid[bone].mean() == pytest.approx(float((mu60[2] * rho[bone]).mean()), rel=0.05)
    # the rod sits at +x: its mirror image across x = 0 holds water, not bone
    assert mid[:, ::-1][bone].mean() == pytest.approx(float(mu60[1]), rel=0.05)


def test_wide_fan_mid_plane_is_exact():
    # the fan-beam formula is exact in the orbit plane: with a short source
    # distance the cosine and 1/U^2 weights change each view by tens of per
    # cent, and the reconstruction still returns mu to 1e-3
    sad, sdd = 150.0, 300.0
    nu, nv, du, dv = 256, 16, 1.2, 1.2
    n_proj = 360
    angles = np.arange(n_proj) * (2.0 * math.pi / n_proj)
    centre, radius, mu = (20.0, -10.0, 0.0), 25.0, 0.02
    g = _ball_projections(angles, sad, sdd, nu, nv, du, dv, centre, radius, mu)
    shape, vox = (3, 64, 64), (1.5, 1.5, 1.0)
    f = fdk.fdk(g, angles, sad, sdd, du, dv, shape, vox)[1]
    c = (np.arange(64) + 0.5 - 32) * 1.5
    Y, X = np.meshgrid(c, c, indexing="ij")
    r = np.hypot(X - centre[0], Y - centre[1])
    inside = r < 0.7 * radius
    assert np.abs(f[inside] / mu - 1.0).max() < 1e-3
    # outside the ball, within the circle every view covers (the fan's
    # half-width at the nearest source distance): view-sampling streaks of
    # about 1 % of mu on average
    fov = np.hypot(X, Y) < 40.0
    out = (r > 1.2 * radius) & fov
    assert np.abs(f[out]).mean() < 0.02 * mu and np.abs(f[out]).max() < 0.06 * mu


def water_cylinder(bowtie_mm):
    """Centred water cylinder (r = 50 mm, 64^3 voxels of 2 mm) in air, 100 kVp
    Kramers spectrum in 2 keV bins, 128 x 128 detector of 2 mm, and an
    aluminium bowtie of 0 .. bowtie_mm (0: none)."""
    p = inputs.small_problem(n_vox=64, vox=2.0, n_det=128, det_px=2.0)
    p.material, p.density = inputs.cylinder_phantom(64, 2.0, r_bone=10.0, bone_x=500.0)   # rod outside the box
    p.spec_e, p.spec_w = inputs.kramers_spectrum(kvp=100.0, bin_kev=2.0)
    p.fluence = inputs.fluence_map(p.nu, p.nv, p.du, p.dv, p.sdd, p.spec_e, p.spec_w, bowtie_mm)
    return p


def radial_means(slice_, vox, n, edges):
    """Mean of a [n, n] transverse slice over the annuli [edges[i], edges[i+1]) (mm)."""
    c = (np.arange(n) + 0.5 - 0.5 * n) * vox
    Y, X = np.meshgrid(c, c, indexing="ij")
    r = np.hypot(X, Y)
    return np.array([slice_[(r >= a) & (r < b)].mean() for a, b in zip(edges[:-1], edges[1:])])


SHADOW_EDGES = (0.0, 12.0, 36.0, 48.0)     # centre disc, middle annulus, ring near the 50 mm surface


def test_scatter_shadow_follows_the_bowtie():
    # the cylinder is rotationally symmetric, so one view, replicated over
    # the orbit, stands for the scan (the ray-traced P is the same at every
    # angle; the scatter is the same in distribution)
    n_views, n = 90, 2_000_000
    angles = np.arange(n_views) * (2.0 * math.pi / n_views)
    deficit = {}
    for bowtie in (0.0, 30.0):
        p = water_cylinder(bowtie)
        P = oracle.rt_primary(p, 0.0)
        _, ts, st, _ = oracle.mc_run(p, n, seed=3, threads=8)
        s_hat = oracle.finalize(ts, n)
        scale = s_hat.sum() / st["tally_scatter"]              # count scale: mean deposit per scattered photon
        counts = oracle.finalize(oracle.bin_tally(ts, 4), n) / scale
        beta = 16.0 / counts.mean()                            # a 4-pixel smoothing length
        s_c = oracle.denoise(counts, beta, iters=1500)
        assert np.abs(oracle.optimality_residual(s_c, counts, beta)).max() < 1e-6
        S = oracle.upsample(s_c * scale, 4)
        empty = water_cylinder(bowtie)
        empty.density[:] = 0.0
        I0 = oracle.rt_primary(empty, 0.0)
        vol = {}
        for name, sig in (("P", P), ("PS", P + S)):
            g = fdk.line_integrals(np.broadcast_to(sig, (n_views,) + sig.shape),
                                   np.broadcast_to(I0, (n_views,) + sig.shape))
            v = fdk.fdk(g, angles, p.sad, p.sdd, p.du, p.dv, p.material.shape, p.voxel)
            vol[name] = radial_means(v[v.shape[0] // 2], 2.0, 64, SHADOW_EDGES)
        deficit[bowtie] = vol["P"] - vol["PS"]
    centre, middle, ring = deficit[0.0]
    assert centre > 1.1 * middle > 1.2 * ring > 0                 # no bowtie: cupping, deepest at the centre
    centre, middle, ring = deficit[30.0]
    assert ring > 1.3 * middle and ring > 2.5 * abs(centre)       # bowtie: the shadow is a ring (Fig. 9(d))
