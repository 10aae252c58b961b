"""Pins of the oracle's Monte Carlo transport (Section 2.4) against closed
forms and invariants.

Beer-Lambert narrow-beam transmission: the fraction of source photons that
reach the aimed pixel unscattered is exp(-integral of mu along the ray).  With
the trilinear field and clamp-to-edge faces, the integral of mu along a
voxel-centre line equals the voxel size times the sum of the voxel mu values,
whatever the profile, so a slab of any density / material profile along the
beam has a closed-form transmission.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1204_6367_gb300 import inputs


def _mu_mm(prob, mat_id, e):
    """total mass attenuation of material mat_id at energy e, mm^-1 per g/cm^3,
    by linear interpolation of the float table (the model's own definition)."""
    tab = prob.mu_hat[mat_id].astype(np.float64).sum(axis=0)
    eg = prob.e0 + prob.de * np.arange(tab.size)
    return 0.1 * float(np.interp(e, eg, tab))


def _transmission(prob, n, seed=1):
    _, _, st, _ = oracle.mc_run(prob, n, seed=seed, threads=8)
    return st["tally_primary"] / n, st


def _check_binomial(frac, expect, n, nsig=3.0):
    sigma = math.sqrt(expect * (1 - expect) / n)
    assert abs(frac - expect) < nsig * sigma, (frac, expect, sigma)


@pytest.mark.parametrize("mat_id,density,energy", [(1, 1.0, 60.0), (2, 1.85, 60.0), (1, 1.0, 25.0), (2, 1.4, 110.0)])
def test_narrow_beam_homogeneous(mat_id, density, energy):
    prob = inputs.uniform_slab_problem(mat_id=mat_id, density=density, energy=energy)
    n = 400000
    frac, _ = _transmission(prob, n)
    thickness = prob.material.shape[2] * prob.voxel[0]     # beam runs along +x at phi = 0
    expect = math.exp(-density * _mu_mm(prob, mat_id, energy) * thickness)
    _check_binomial(frac, expect, n)


def test_narrow_beam_two_materials():
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0)
    prob.material[:, :, 8:] = 2
    prob.density[:, :, 8:] = 1.85
    n = 400000
    frac, _ = _transmission(prob, n)
    dx = prob.voxel[0]
    expect = math.exp(-(8 * dx * 1.0 * _mu_mm(prob, 1, 60.0) + 8 * dx * 1.85 * _mu_mm(prob, 2, 60.0)))
    _check_binomial(frac, expect, n)


def test_narrow_beam_density_ramp():
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0, nx=24)
    ramp = np.linspace(0.2, 2.4, 24).astype(np.float32)
    prob.density[:] = ramp[None, None, :]
    n = 400000
    frac, _ = _transmission(prob, n)
    expect = math.exp(-prob.voxel[0] * float(ramp.astype(np.float64).sum()) * _mu_mm(prob, 1, 60.0))
    _check_binomial(frac, expect, n)


def test_loose_majorant_does_not_bias():
    # A dense bone voxel far from the beam raises the majorant (more virtual
    # collisions) but must not change the transmission.
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0)
    n = 400000
    frac0, st0 = _transmission(prob, n)
    prob.material[0, 0, 0] = 2
    prob.density[0, 0, 0] = 8.0
    frac1, st1 = _transmission(prob, n)
    assert st1["virtual"] > 5 * st0["virtual"] + 1000
    thickness = prob.material.shape[2] * prob.voxel[0]
    expect = math.exp(-_mu_mm(prob, 1, 60.0) * thickness)
    _check_binomial(frac0, expect, n)
    _check_binomial(frac1, expect, n)


def test_first_interaction_fractions():
    # In a homogeneous medium the first real collision is Rayleigh, Compton or
    # photoelectric with probabilities mu_R : mu_C : mu_P at the source energy.
    prob = inputs.uniform_slab_problem(mat_id=2, density=1.85, energy=40.0, nx=32, ny=32, nz=32)
    n = 300000
    _, _, _, rec = oracle.mc_run(prob, n, seed=2, threads=8, records=True)
    first = rec["first_interaction"]
    counts = np.array([(first == k).sum() for k in (1, 2, 3)], np.float64)
    tab = prob.mu_hat[2].astype(np.float64)
    eg = prob.e0 + prob.de * np.arange(tab.shape[1])
    mu = np.array([np.interp(40.0, eg, tab[k]) for k in range(3)])
    expected = mu / mu.sum() * counts.sum()
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(chi2, 2) > 0.01, (counts, expected)


def test_energy_conservation(small):
    _, _, _, rec = oracle.mc_run(small, 50000, seed=4, records=True)
    out = rec["outcome"]
    esrc = rec["e_source"].astype(np.float64)
    escaped = (out == 0) | (out == 1) | (out == 4)
    absorbed = (out == 2) | (out == 3)
    assert escaped.any() and absorbed.any()
    lhs = rec["e_final"].astype(np.float64) + rec["e_deposited"]
    np.testing.assert_allclose(lhs[escaped], esrc[escaped], rtol=1e-6)
    np.testing.assert_allclose(rec["e_deposited"][absorbed], esrc[absorbed], rtol=1e-6)
    # unscattered photons keep their energy
    prim = out == 0
    np.testing.assert_array_equal(rec["e_final"][prim], rec["e_source"][prim])
    assert np.all(rec["n_rayleigh"][prim] + rec["n_compton"][prim] == 0)


def test_split_and_thread_invariance(small):
    n = 40000
    tp, ts, st, _ = oracle.mc_run(small, n, seed=9)
    tp1, ts1, st1, _ = oracle.mc_run(small, 17000, seed=9)
    tp2, ts2, st2, _ = oracle.mc_run(small, n - 17000, seed=9, history_offset=17000)
    np.testing.assert_array_equal(tp, tp1 + tp2)
    np.testing.assert_array_equal(ts, ts1 + ts2)
    tp8, ts8, st8, _ = oracle.mc_run(small, n, seed=9, threads=7)
    np.testing.assert_array_equal(tp, tp8)
    np.testing.assert_array_equal(ts, ts8)
    assert st == st8
    assert {k: st1[k] + st2[k] for k in st} == st


def test_vacuum_reproduces_source(small):
    # Zero density everywhere: every photon flies straight to the pixel it was
    # aimed at; pixel counts follow w(u), energies follow phi(E).
    prob = inputs.torso_problem(vox=16.0, nu=32, nv=24, det_px=0.776 * 16)
    prob.density[:] = 0.0
    n = 300000
    tp, ts, st, rec = oracle.mc_run(prob, n, seed=12, threads=8, records=True)
    assert st["tally_primary"] == n and ts.sum() == 0 and st["steps"] <= n
    counts = np.bincount(rec["pixel"], minlength=prob.nu * prob.nv).astype(np.float64)
    expected = prob.fluence.ravel() / prob.fluence.sum() * n
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(chi2, counts.size - 1) > 0.01
    e_idx = np.searchsorted(prob.spec_e.astype(np.float32), rec["e_source"])
    ecounts = np.bincount(e_idx, minlength=prob.spec_e.size).astype(np.float64)
    eexp = prob.spec_w / prob.spec_w.sum() * n
    keep = eexp > 5
    chi2 = ((ecounts[keep] - eexp[keep]) ** 2 / eexp[keep]).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 0.01
    # primary tally is exactly r(E) * 2^24 per photon
    q = np.rint(np.interp(rec["e_source"].astype(np.float32), prob.r0 + prob.dr * np.arange(prob.response.size),
                          prob.response) * 2.0**24)
    assert abs(tp.sum() - q.sum()) <= n * 2


def test_step_limit_is_reported(small):
    _, _, st, rec = oracle.mc_run(small, 2000, seed=1, max_steps=2, records=True)
    assert st["step_limit"] > 0
    assert np.all(rec["n_steps"] <= 2)


def test_rejects_bad_geometry(small):
    import copy
    bad = copy.copy(small)
    bad.sdd = 1030.0          # imager plane cuts the phantom box
    with pytest.raises(ValueError):
        oracle.mc_run(bad, 10)


def _pixel_average(fn, u_c, v_c, du, dv, n=24):
    g = (np.arange(n) + 0.5) / n - 0.5
    return float(np.mean([[fn(u_c + a * du, v_c + b * dv) for a in g] for b in g]))


@pytest.mark.parametrize("axis", ["y", "z"])
def test_narrow_beam_transverse_linear_field(axis):
    # Density linear across the beam (in y or z), beam off a voxel-centre line:
    # the trilinear field is exactly linear there, so the line integral is the
    # chord length times the density at the chord's midpoint.  Catches wrong
    # interpolation weights or corner indices in the transverse directions.
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0, nx=16, ny=16, nz=16, nu=32, nv=32, det_px=0.5)
    vox = prob.voxel[0]
    centres = (np.arange(16) + 0.5) * vox - 8 * vox
    a, b = 1.0, 0.04
    ramp = (a + b * centres).astype(np.float32)
    if axis == "y":
        prob.density[:] = ramp[None, :, None]
    else:
        prob.density[:] = ramp[:, None, None]
    iu, iv = 26, 4          # beam well off the centre lines in both y and z
    prob.fluence[:] = 0.0
    prob.fluence[iv, iu] = 1.0
    n = 400000
    frac, _ = _transmission(prob, n)
    mu = _mu_mm(prob, 1, 60.0)
    S = np.array([-prob.sad, 0.0, 0.0])
    half = 8 * vox

    def trans(u, v):
        D = np.array([prob.sdd - prob.sad, -u, v])      # phi = 0: e_u = (0,-1,0), e_v = z
        d = (D - S) / np.linalg.norm(D - S)
        t0, t1 = (-half - S[0]) / d[0], (half - S[0]) / d[0]
        mid = S + 0.5 * (t0 + t1) * d
        coord = mid[1] if axis == "y" else mid[2]
        rho = a + b * coord
        return math.exp(-mu * rho * (t1 - t0))

    u_c = (iu + 0.5 - 0.5 * prob.nu) * prob.du
    v_c = (iv + 0.5 - 0.5 * prob.nv) * prob.dv
    expect = _pixel_average(trans, u_c, v_c, prob.du, prob.dv)
    _check_binomial(frac, expect, n)


@pytest.mark.parametrize("phi,theta", [(0.0, 0.0), (0.7, 0.0), (2.2, 0.15)])
def test_vacuum_photon_lands_in_aimed_pixel(phi, theta):
    # Asymmetric source: only one off-centre pixel is lit; in vacuum every
    # photon must be tallied there, for any gantry angle and imager angle.
    prob = inputs.uniform_slab_problem(mat_id=0, density=0.0, nu=12, nv=10, det_px=2.0)
    prob.theta = theta
    prob.fluence[:] = 0.0
    prob.fluence[7, 2] = 1.0
    _, _, st, rec = oracle.mc_run(prob, 5000, seed=3, phi=phi, records=True)
    assert st["tally_primary"] == 5000
    # FP32 positions carry ~1e-4 mm of rounding at these distances, so a point
    # drawn within that of a pixel edge may cross into the neighbour.
    pix = rec["pixel"]
    assert np.mean(pix == 7 * prob.nu + 2) > 0.998
    iu, iv = pix % prob.nu, pix // prob.nu
    assert np.all((np.abs(iu - 2) <= 1) & (np.abs(iv - 7) <= 1))
