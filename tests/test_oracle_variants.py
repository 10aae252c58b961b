"""Pins of the oracle's variants of the method:

* Monte Carlo without density interpolation (the voxel's own value; the
  speed variant of the paper's appendix, Fig. 11): Beer-Lambert through a
  transverse density step, where only the voxel containing the beam counts;
* Siddon ray tracing (Section 2.3's alternative): closed-form chords, and
  brute-force sampling of the piecewise-constant field along the ray;
* the paper's pairing of the two (Fig. 11): MC primary without density
  interpolation matches the Siddon primary;
* scatter filters (Section 2.4: tally a specific type of scatter): single
  Compton, single Rayleigh and multiple scatter partition the scatter tally.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1204_6367_gb300 import inputs


def _mu_mm(prob, mat_id, e):
    tab = prob.mu_hat[mat_id].astype(np.float64).sum(axis=0)
    eg = prob.e0 + prob.de * np.arange(tab.size)
    return 0.1 * float(np.interp(e, eg, tab))


def test_nearest_voxel_transverse_step():
    # density steps in y; the pencil beam runs along x inside voxel row j:
    # only that row's density matters without interpolation
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0, nx=16, ny=16, nz=16, nu=32, nv=32, det_px=0.5)
    dens = np.linspace(0.4, 2.0, 16).astype(np.float32)
    prob.density[:] = dens[None, :, None]
    iu, iv = 26, 16                     # u = +5.25 mm -> y = -3.5 mm at the isocentre: row 6 of 16 (2 mm voxels)
    prob.fluence[:] = 0.0
    prob.fluence[iv, iu] = 1.0
    n = 300000
    _, _, st, _ = oracle.mc_run(prob, n, seed=3, threads=8, nearest_voxel=True)
    frac = st["tally_primary"] / n
    row = int(math.floor((-3.5 + 16.0) / 2.0))
    expect = math.exp(-float(dens[row]) * _mu_mm(prob, 1, 60.0) * 32.0)
    sigma = math.sqrt(expect * (1 - expect) / n)
    assert abs(frac - expect) < 3 * sigma, (frac, expect)
    # with interpolation the same beam sees a different density
    _, _, st2, _ = oracle.mc_run(prob, n, seed=3, threads=8)
    assert abs(st2["tally_primary"] / n - expect) > 5 * sigma


@pytest.mark.parametrize("phi", [0.0, 0.7, 2.5])
def test_siddon_homogeneous_chords(phi):
    prob = inputs.uniform_slab_problem(mat_id=2, density=1.3, nx=12, ny=10, nz=9, nu=10, nv=8, det_px=4.0,
                                       pencil=False)
    got = oracle.rt_primary_siddon(prob, phi=phi)
    ref = oracle.rt_primary(prob, phi=phi)          # both exact for a homogeneous box
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_siddon_matches_dense_sampling():
    rng = np.random.default_rng(4)
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0, nx=7, ny=6, nz=5, nu=6, nv=5, det_px=3.0,
                                       pencil=False)
    prob.material[:] = rng.integers(0, 3, prob.material.shape).astype(np.uint8)
    prob.density[:] = rng.uniform(0.1, 2.0, prob.density.shape).astype(np.float32)
    phi = 0.4
    got = oracle.rt_primary_siddon(prob, phi=phi).ravel()
    # brute force: midpoint rule with 200000 samples of the piecewise-constant field
    ang = phi
    S = np.array([-prob.sad * math.cos(phi), -prob.sad * math.sin(phi), 0.0])
    P = (prob.sdd - prob.sad) * np.array([math.cos(ang), math.sin(ang), 0.0])
    eu = np.array([math.sin(ang), -math.cos(ang), 0.0])
    nz, ny, nx = prob.material.shape
    half = 0.5 * np.array([nx, ny, nz]) * np.array(prob.voxel)
    mu_m = np.array([_mu_mm(prob, m, 60.0) for m in range(3)])
    w = prob.fluence.ravel() / prob.fluence.sum()
    for j in range(prob.nu * prob.nv):
        iu, iv = j % prob.nu, j // prob.nu
        C = P + (iu + 0.5 - 0.5 * prob.nu) * prob.du * eu + np.array([0, 0, (iv + 0.5 - 0.5 * prob.nv) * prob.dv])
        d = (C - S) / np.linalg.norm(C - S)
        with np.errstate(divide="ignore"):
            t1, t2 = (-half - S) / d, (half - S) / d
        t0, t3 = np.max(np.minimum(t1, t2)), np.min(np.maximum(t1, t2))
        if t3 <= t0:
            assert got[j] == pytest.approx(w[j] * 60.0, rel=1e-12)
            continue
        m = 200000
        ts = t0 + (np.arange(m) + 0.5) * (t3 - t0) / m
        x = S[None] + ts[:, None] * d[None]
        idx = np.clip(np.floor((x + half) / np.array(prob.voxel)).astype(int), 0, np.array([nx, ny, nz]) - 1)
        rho = prob.density[idx[:, 2], idx[:, 1], idx[:, 0]].astype(np.float64)
        mat = prob.material[idx[:, 2], idx[:, 1], idx[:, 0]]
        rad = np.sum(rho * mu_m[mat]) * (t3 - t0) / m
        assert got[j] == pytest.approx(w[j] * 60.0 * math.exp(-rad), rel=2e-3)


def test_nearest_voxel_mc_matches_siddon(small):
    n = 2_000_000
    tp, _, _, _ = oracle.mc_run(small, n, seed=8, threads=8, nearest_voxel=True)
    p_mc = oracle.finalize(tp, n)
    p_rt = oracle.rt_primary_siddon(small)
    m = p_rt > 0.05 * p_rt.max()
    assert abs(p_mc[m].sum() / p_rt[m].sum() - 1.0) < 0.01
    assert abs(np.mean((p_mc[m] - p_rt[m]) / p_rt[m])) < 0.01


def test_scatter_filters_partition_the_scatter(small):
    n = 200000
    _, s_all, _, rec_all = oracle.mc_run(small, n, seed=6, threads=4, records=True)
    parts = []
    for f in (1, 2, 3):
        tp, s_f, _, rec = oracle.mc_run(small, n, seed=6, threads=4, scatter_filter=f, records=True)
        parts.append(s_f)
        sel = rec["outcome"] == 1
        if f == 1:
            assert np.all((rec["n_compton"][sel] == 1) & (rec["n_rayleigh"][sel] == 0))
        if f == 2:
            assert np.all((rec["n_rayleigh"][sel] == 1) & (rec["n_compton"][sel] == 0))
        if f == 3:
            assert np.all(rec["n_rayleigh"][sel] + rec["n_compton"][sel] >= 2)
    np.testing.assert_array_equal(parts[0] + parts[1] + parts[2], s_all)
    assert parts[0].sum() > parts[2].sum() > parts[1].sum() > 0
