"""Pins of the oracle's ray-traced primary (Section 2.3, Eq. 1).

Closed forms: for a field that trilinear interpolation reproduces exactly
along the ray (constant, or any profile along a voxel-centre line), the
midpoint sum of Eq. 1's discretisation equals the exact line integral, so
P = w * sum_E phi r exp(-mu(E) * chord).  And the paper's own consistency
check (Section 3.1, Fig. 5): the MC primary agrees with the ray-traced one.
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


def _ray(prob, iu, iv, phi=0.0):
    ang = phi + prob.theta
    aid = prob.sdd - prob.sad
    S = np.array([-prob.sad * math.cos(phi), -prob.sad * math.sin(phi), 0.0])
    P = aid * np.array([math.cos(ang), math.sin(ang), 0.0])
    eu = np.array([math.sin(ang), -math.cos(ang), 0.0])
    ev = np.array([0.0, 0.0, 1.0])
    C = P + (iu + 0.5 - 0.5 * prob.nu) * prob.du * eu + (iv + 0.5 - 0.5 * prob.nv) * prob.dv * ev
    d = C - S
    return S, d / np.linalg.norm(d)


def _box_chord(prob, S, d):
    nz, ny, nx = prob.material.shape
    half = 0.5 * np.array([nx * prob.voxel[0], ny * prob.voxel[1], nz * prob.voxel[2]])
    with np.errstate(divide="ignore"):
        t1 = (-half - S) / d
        t2 = (half - S) / d
    tmin = np.max(np.minimum(t1, t2))
    tmax = np.min(np.maximum(t1, t2))
    return max(0.0, tmax - tmin)


@pytest.mark.parametrize("phi", [0.0, 0.3, 1.2, 2.9])
def test_homogeneous_box_chords(phi):
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.3, nx=20, ny=14, nz=10, nu=16, nv=12,
                                       det_px=3.0, pencil=False)
    pix = np.arange(prob.nu * prob.nv)
    got = oracle.rt_primary(prob, phi=phi, pixels=pix)
    mu = float(np.float32(1.3)) * _mu_mm(prob, 1, 60.0)   # density is stored as float32
    w = prob.fluence.ravel() / prob.fluence.sum()
    for j in pix:
        S, d = _ray(prob, j % prob.nu, j // prob.nu, phi)
        expect = w[j] * 60.0 * math.exp(-mu * _box_chord(prob, S, d))
        assert got[j] == pytest.approx(expect, rel=1e-12, abs=1e-300)


def test_polyenergetic_slab():
    prob = inputs.uniform_slab_problem(mat_id=2, density=1.6, nx=12)
    e, wts = inputs.kramers_spectrum()
    prob.spec_e, prob.spec_w = e, wts
    j = (prob.nv // 2) * prob.nu + prob.nu // 2
    got = oracle.rt_primary(prob, pixels=[j])[0]
    S, d = _ray(prob, prob.nu // 2, prob.nv // 2)
    L = _box_chord(prob, S, d)
    r = lambda x: float(np.interp(x, prob.r0 + prob.dr * np.arange(prob.response.size), prob.response.astype(np.float64)))
    expect = sum(wi * r(ei) * math.exp(-float(np.float32(1.6)) * _mu_mm(prob, 2, ei) * L) for ei, wi in zip(e, wts))
    assert got == pytest.approx(expect, rel=1e-12)


def test_density_profile_along_beam():
    # Along a voxel-centre line the trilinear integral is dx * sum(rho): the
    # midpoint rule of Eq. 1's discretisation reproduces it for the
    # piecewise-linear field when intervals nest in the voxel half-grid.
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0, nx=24, ny=15, nz=15, nu=1, nv=1,
                                       det_px=0.001, sad=1000.0, sdd=1500.0)
    prof = np.random.default_rng(0).uniform(0.1, 2.0, 24).astype(np.float32)
    prob.density[:] = prof[None, None, :]
    got = oracle.rt_primary(prob, pixels=[0])[0]
    expect = 60.0 * math.exp(-prob.voxel[0] * float(prof.astype(np.float64).sum()) * _mu_mm(prob, 1, 60.0))
    assert got == pytest.approx(expect, rel=1e-9)


def test_mc_primary_matches_rt(small):
    # Section 3.1 / Fig. 5: MC primary with density interpolation agrees with
    # the tri-linear ray-traced primary.  Mean relative difference <= 1 % over
    # pixels carrying > 5 % of the peak, and per-pixel z-scores look normal.
    n = 2_000_000
    tp, _, _, _ = oracle.mc_run(small, n, seed=21, threads=8)
    p_mc = oracle.finalize(tp, n)
    p_rt = oracle.rt_primary(small)
    m = p_rt > 0.05 * p_rt.max()
    assert abs(p_mc[m].sum() / p_rt[m].sum() - 1.0) < 0.01
    assert abs(np.mean((p_mc[m] - p_rt[m]) / p_rt[m])) < 0.01
    # per-pixel: counts are ~binomial; in-pixel variation of the path length
    # gives the MC pixel a slightly different mean than the centre ray, so
    # assess the bulk, not the tail.
    counts = tp[m] / (60.0 * 2**24)
    mean = p_rt[m] / 60.0 * n
    z = (counts - mean) / np.sqrt(mean)
    assert np.mean(np.abs(z) < 3) > 0.97
