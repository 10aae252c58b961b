"""Pins of the oracle's Rayleigh form-factor option.

Rayleigh scattering has the differential cross section (r_e^2 / 2)(1 + cos^2)
F^2(x) with x = sin(theta/2) E / (hc); the paper samples the angle with the
techniques of its dose engine (Section 2.4) without stating them.  The
library's default stays Thomson (F = const).  Pins:

* with the synthetic form factor on a fine table, the sampled angles follow
  the analytic law (1 + cos^2) F^2(x), integrated by quadrature;
* on a coarse table, they follow the law the method defines exactly (F^2
  linear in x^2 between nodes), which checks the in-interval inversion;
* a constant form factor reduces to the Thomson law;
* the distribution narrows as the energy rises;
* at a trilinear mixture point the form factor's material is picked in
  proportion to its share of the Rayleigh coefficient: on a water/bone
  checkerboard the bone share is mu_R(bone) / (mu_R(bone) + mu_R(water)).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1204_6367_gb300 import inputs

HC = 12.398419843320026          # keV Angstrom
MATS = [inputs.AIR, inputs.WATER, inputs.BONE]


def _prob(dx=None, n=None, table=None):
    prob = inputs.uniform_slab_problem(mat_id=1, nx=8, ny=8, nz=8)
    if dx is not None:
        x = dx * np.arange(n)
        prob.form_factor = np.stack([inputs.form_factor(m, x) for m in MATS]).astype(np.float32)
        prob.ff_dx = dx
    if table is not None:
        prob.form_factor = table
    return prob


def _chi2(samples, pdf, edges, breakpoints=None):
    """Chi-square of a histogram of samples against a density given up to its norm."""
    lo, hi = edges[0], edges[-1]
    tot = integrate.quad(pdf, lo, hi, limit=2000, points=breakpoints)[0]
    exp = []
    for a, b in zip(edges[:-1], edges[1:]):
        pts = None if breakpoints is None else [p for p in breakpoints if a < p < b]
        exp.append(integrate.quad(pdf, a, b, limit=2000, points=pts or None)[0])
    exp = np.array(exp) / tot * samples.size
    obs = np.histogram(samples, edges)[0]
    return float(((obs - exp) ** 2 / exp).sum())


# 20 bins: chi-square with 19 dof has mean 19 and sd 6.2; 55 is p ~ 1e-5
CHI2_MAX = 55.0


@pytest.mark.parametrize("e, m", [(5.0, 1), (60.0, 1), (20.0, 2), (140.0, 2), (90.0, 0)])
def test_sampler_follows_the_analytic_law(e, m):
    prob = _prob(dx=0.005, n=2560)
    c = oracle.sample_rayleigh_ff(prob, e, m, 300000, seed=11).astype(np.float64)
    xm = e / HC
    s = xm * xm * (1.0 - c) / 2.0
    z = MATS[m].z_eff
    b = (0.45 * (z / inputs.WATER.z_eff) ** (1.0 / 3.0)) ** 2
    pdf = lambda t: (1.0 + (1.0 - 2.0 * t / (xm * xm)) ** 2) / (1.0 + t / b) ** 4
    edges = np.quantile(s, np.linspace(0, 1, 21))
    edges[0], edges[-1] = 0.0, xm * xm
    assert _chi2(s, pdf, edges) < CHI2_MAX


def test_coarse_table_follows_the_piecewise_linear_law():
    dx, n = 0.1, 130
    prob = _prob(dx=dx, n=n)
    e, m = 12.0, 1                      # x_max ~ 0.97: ten intervals, strongly curved F^2
    c = oracle.sample_rayleigh_ff(prob, e, m, 300000, seed=5).astype(np.float64)
    xm = e / HC
    smax = xm * xm
    s = smax * (1.0 - c) / 2.0
    F = prob.form_factor[m].astype(np.float64)
    nodes = (dx * np.arange(n)) ** 2
    g = F * F
    pdf = lambda t: (1.0 + (1.0 - 2.0 * t / smax) ** 2) * np.interp(t, nodes, g)
    edges = np.quantile(s, np.linspace(0, 1, 21))
    edges[0], edges[-1] = 0.0, smax
    bp = [p for p in nodes if 0 < p < smax]
    assert _chi2(s, pdf, edges, bp) < CHI2_MAX


def test_constant_form_factor_is_thomson():
    table = np.ones((3, 640), np.float32) * np.array([[7.0], [8.0], [9.0]], np.float32)
    prob = _prob(table=table)
    c = oracle.sample_rayleigh_ff(prob, 60.0, 1, 300000, seed=9).astype(np.float64)
    edges = np.linspace(-1, 1, 21)
    assert _chi2(c, lambda t: 1.0 + t * t, edges) < CHI2_MAX
    assert np.mean(c * c) == pytest.approx(0.4, abs=0.004)


def test_forward_peaking_grows_with_energy():
    prob = _prob()
    means = [oracle.sample_rayleigh_ff(prob, e, 1, 50000, seed=2).astype(np.float64).mean()
             for e in (10.0, 20.0, 40.0, 80.0, 150.0)]
    assert np.all(np.diff(means) > 0) and means[-1] > 0.99 and means[0] < 0.95


@pytest.mark.parametrize("nearest", [False, True])
def test_material_pick_in_a_mixture(nearest):
    prob = inputs.uniform_slab_problem(mat_id=1, nx=16, ny=16, nz=16, nu=32, nv=32, det_px=1.0, pencil=False)
    z, y, x = np.indices(prob.material.shape)
    prob.material[:] = (1 + (x + y + z) % 2).astype(np.uint8)       # water / bone checkerboard
    n = 300000
    _, _, st, rec = oracle.mc_run(prob, n, seed=17, threads=8, records=True, rayleigh_ff=True,
                                  nearest_voxel=nearest)
    one = rec["n_rayleigh"] == 1
    k = int(one.sum())
    assert k > 3000
    assert set(np.unique(rec["ray_material"][one])) <= {1, 2}
    frac_bone = float(np.mean(rec["ray_material"][one] == 2))
    r = float(prob.mu_hat[2, inputs.RAYLEIGH, 59] / prob.mu_hat[1, inputs.RAYLEIGH, 59])
    expect = r / (1.0 + r)
    assert abs(frac_bone - expect) < 4 * math.sqrt(expect * (1 - expect) / k) + 0.01, (frac_bone, expect)
    # histories without a Rayleigh event keep the field at zero
    assert np.all(rec["ray_material"][rec["n_rayleigh"] == 0] == 0)


def test_form_factor_table_must_reach_the_backscatter_momentum():
    prob = _prob(dx=0.01, n=500)        # reaches 4.99 1/Angstrom, 150 keV needs 12.1
    with pytest.raises(ValueError):
        oracle.mc_run(prob, 10, rayleigh_ff=True)
