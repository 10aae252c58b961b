"""Pins of the oracle's interaction samplers against closed forms.

Compton: the sampled polar cosine follows the Klein-Nishina law
  dsigma/dOmega ~ P^2 (P + 1/P - sin^2 theta),  P = E'/E = 1 / (1 + a (1 - cos theta)),
and E' = E P (Compton formula).  Rayleigh (no form factor): Thomson's
(1 + cos^2 theta).  Azimuth: uniform.  Rotation: the new direction makes the
sampled angle with the old one and stays a unit vector.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle

ME = 510.99895


def kn_pdf(mu, e):
    a = e / ME
    p = 1.0 / (1.0 + a * (1.0 - mu))
    return p * p * (p + 1.0 / p - (1.0 - mu * mu))


def _chi2_pvalue(samples, edges, cdf_bins):
    counts, _ = np.histogram(samples, edges)
    expected = cdf_bins / cdf_bins.sum() * counts.sum()
    chi2 = ((counts - expected) ** 2 / expected).sum()
    return stats.chi2.sf(chi2, len(counts) - 1)


@pytest.mark.parametrize("e", [20.0, 60.0, 120.0])
def test_klein_nishina_angle(e):
    n = 400000
    mu, e_out = oracle.sample_compton(e, n, seed=3)
    mu = mu.astype(np.float64)
    assert np.all(mu >= -1.0 - 1e-6) and np.all(mu <= 1.0 + 1e-6)
    edges = np.linspace(-1.0, 1.0, 41)
    probs = np.array([integrate.quad(kn_pdf, lo, hi, args=(e,))[0] for lo, hi in zip(edges[:-1], edges[1:])])
    assert _chi2_pvalue(mu, edges, probs) > 0.01


@pytest.mark.parametrize("e", [20.0, 60.0, 120.0])
def test_compton_energy(e):
    n = 200000
    mu, e_out = oracle.sample_compton(e, n, seed=5)
    mu = mu.astype(np.float64)
    e_out = e_out.astype(np.float64)
    # Compton formula per sample
    np.testing.assert_allclose(e_out, e / (1.0 + (e / ME) * (1.0 - mu)), rtol=2e-6)
    # mean scattered energy against the closed-form KN average
    norm = integrate.quad(kn_pdf, -1, 1, args=(e,))[0]
    mean = integrate.quad(lambda m: kn_pdf(m, e) * e / (1 + (e / ME) * (1 - m)), -1, 1)[0] / norm
    assert abs(e_out.mean() - mean) < 4.0 * e_out.std() / math.sqrt(n)


def test_thomson_angle():
    mu = oracle.sample_rayleigh(400000, seed=7).astype(np.float64)
    edges = np.linspace(-1.0, 1.0, 41)
    prim = lambda m: m + m**3 / 3.0
    probs = prim(edges[1:]) - prim(edges[:-1])
    assert _chi2_pvalue(mu, edges, probs) > 0.01


def test_azimuth_uniform():
    c, s = oracle.sample_azimuth(400000, seed=11)
    c = c.astype(np.float64)
    s = s.astype(np.float64)
    np.testing.assert_allclose(c * c + s * s, 1.0, atol=1e-6)
    phi = np.arctan2(s, c)
    edges = np.linspace(-math.pi, math.pi, 37)
    assert _chi2_pvalue(phi, edges, np.diff(edges)) > 0.01


def test_rotate_keeps_angle_and_norm():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if rng.random() < 0.05:
            d = np.array([0.0, 0.0, rng.choice([-1.0, 1.0])])
        ct = rng.uniform(-1, 1)
        ph = rng.uniform(-math.pi, math.pi)
        out = oracle.rotate(d.astype(np.float32), ct, math.cos(ph), math.sin(ph)).astype(np.float64)
        d32 = d.astype(np.float32).astype(np.float64)
        assert abs(np.linalg.norm(out) - 1.0) < 1e-6
        assert abs(np.dot(out, d32) - ct) < 5e-6


def test_rotate_azimuth_is_uniform_about_the_axis():
    # For a fixed old direction and polar angle, sweeping the azimuth must
    # sweep the new direction uniformly around the old one: the component
    # along a fixed perpendicular axis is then cos(phi + const).
    d = np.array([0.3, -0.5, 0.8124]); d /= np.linalg.norm(d)
    ct = 0.25
    phis = np.linspace(-math.pi, math.pi, 721)[:-1]
    outs = np.array([oracle.rotate(d.astype(np.float32), ct, math.cos(p), math.sin(p)) for p in phis], np.float64)
    e1 = np.cross(d, [0.0, 0.0, 1.0]); e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    proj = outs - np.outer(outs @ d, d)
    ang = np.unwrap(np.arctan2(proj @ e2, proj @ e1))
    steps = np.diff(ang)
    np.testing.assert_allclose(np.abs(steps), 2 * math.pi / 720, rtol=1e-3)
    np.testing.assert_allclose(np.linalg.norm(proj, axis=1), math.sqrt(1 - ct * ct), atol=1e-5)
