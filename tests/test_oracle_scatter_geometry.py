"""First-order Compton and Rayleigh scatter on the detector, against a
deterministic integral of their physics.

A pencil beam of 60 keV photons crosses a thin water cube; the oracle's
transport tallies the photons that scattered exactly once, by Compton, and
then reached the imager without a further interaction (the single-Compton
filter of Section 2.4).  The same signal follows from the physics alone:

    T_k = < integral over the beam chord of  mu_C e^{-mu s}
            x integral over pixel k of  (1/sigma) dsigma_KN/dOmega(theta) dOmega
            x E'(theta) e^{-mu(E') d_out} >_beam,

with mu from the same material table, Klein-Nishina's angular law
normalised by its numerically integrated total, dOmega = cos(psi) dA / r^2,
E' = E / (1 + (E / m_e c^2)(1 - cos theta)) and d_out the path from the
scatter point to the cube's surface.  Here it is evaluated by midpoint
quadrature over the beam's cross-section, its depth and each pixel's area:
no sampling, none of the oracle's code.  A wrong scattering frame, azimuth,
exit geometry, imager coordinate, scattered energy or response would move
the rings of the scatter image away from it.  The single-Rayleigh filter
gives the same check with the Thomson law, and with Thomson times the form
factor (Rayleigh with form factors), in place of Klein-Nishina.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1204_6367_gb300 import inputs

MEC2 = 510.99895


def _kn(mu, e):
    """Klein-Nishina dsigma/dOmega / r_e^2 at cos theta = mu, and E'."""
    e2 = e / (1.0 + (e / MEC2) * (1.0 - mu))
    r = e2 / e
    return 0.5 * r * r * (r + 1.0 / r - (1.0 - mu * mu)), e2


HC = 12.398419843320026          # keV Angstrom


def _angular_law(prob, law, e):
    """(1/sigma) dsigma/dOmega as a function of cos theta, and the scattered
    energy, for the three first-order laws: Klein-Nishina (Compton), Thomson
    (Rayleigh) and Thomson times the form factor F^2 of water (Rayleigh with
    form factors; F^2 linear in s = x^2 between the table's nodes, x =
    sin(theta / 2) E / hc, as the method defines it)."""
    if law == "compton":
        sigma = 2.0 * math.pi * integrate.quad(lambda m: _kn(m, e)[0], -1.0, 1.0, epsabs=0, epsrel=1e-12)[0]
        return lambda mu: (_kn(mu, e)[0] / sigma, _kn(mu, e)[1])
    if law == "rayleigh":
        return lambda mu: (3.0 / (16.0 * math.pi) * (1.0 + mu * mu), np.full_like(mu, e))
    f = prob.form_factor[1].astype(np.float64)
    s_nodes = (np.arange(f.size) * prob.ff_dx) ** 2
    smax = (e / HC) ** 2

    def f2(mu):
        return np.interp(smax * (1.0 - mu) / 2.0, s_nodes, f * f)
    grid = np.linspace(-1.0, 1.0, 400001)
    sigma = 2.0 * math.pi * np.trapezoid((1.0 + grid * grid) * f2(grid), grid)
    return lambda mu: ((1.0 + mu * mu) * f2(mu) / sigma, np.full_like(mu, e))


def _mu(prob, k, e):
    """mu in 1/mm of water at density rho for interaction k (0 R, 1 C, 2 P; None: total),
    linear in E between the table's nodes (the method's mu(E))."""
    tab = prob.mu_hat[1].astype(np.float64)             # material 1: water, cm^2/g
    e0, de = prob.e0, prob.de
    x = (np.asarray(e, np.float64) - e0) / de
    i = np.clip(np.floor(x).astype(int), 0, tab.shape[1] - 2)
    f = x - i
    t = tab.sum(axis=0) if k is None else tab[k]
    return (t[i] + f * (t[i + 1] - t[i])) * 0.1 * float(prob.density.flat[0])


def _exit_distance(X, d, half):
    """Distance from points X inside the cube [-half, half]^3 along unit d to its surface."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(d > 0, (half - X) / d, np.where(d < 0, (-half - X) / d, np.inf))
    return t.min(axis=-1)


def _expected(prob, half, law="compton", n_depth=64, n_beam=4, n_sub=3):
    E = float(prob.spec_e[0])
    sad, sdd, nu, nv, du, dv = prob.sad, prob.sdd, prob.nu, prob.nv, prob.du, prob.dv
    S = np.array([-sad, 0.0, 0.0])                      # angle 0: source on -x, imager at x = sdd - sad
    eu, ev = np.array([0.0, -1.0, 0.0]), np.array([0.0, 0.0, 1.0])
    pdf = _angular_law(prob, law, E)
    muC, muT = _mu(prob, 1 if law == "compton" else 0, E), _mu(prob, None, E)
    # detector sub-points: pixel centres and area elements
    iu, iv = np.meshgrid(np.arange(nu), np.arange(nv))
    off = (np.arange(n_sub) + 0.5) / n_sub
    ou, ov = np.meshgrid(off, off)
    au = ((iu[..., None, None] + ou) - 0.5 * nu) * du                 # [nv, nu, sub, sub]
    av = ((iv[..., None, None] + ov) - 0.5 * nv) * dv
    D = (sdd - sad) * np.array([1.0, 0.0, 0.0]) + au[..., None] * eu + av[..., None] * ev
    dA = du * dv / (n_sub * n_sub)
    # the pencil: uniform over the fluence map's one lit pixel
    ju, jv = nu // 2, nv // 2
    bo = (np.arange(n_beam) + 0.5) / n_beam
    T = np.zeros((nv, nu))
    for bu in bo:
        for bv in bo:
            C = (sdd - sad) * np.array([1.0, 0.0, 0.0]) + ((ju + bu) - 0.5 * nu) * du * eu \
                + ((jv + bv) - 0.5 * nv) * dv * ev
            d0 = (C - S) / np.linalg.norm(C - S)
            ts = [((-half - S[a]) / d0[a], (half - S[a]) / d0[a]) for a in range(3) if d0[a] != 0.0]
            t_in = max(min(p) for p in ts)
            t_out = min(max(p) for p in ts)
            dt = (t_out - t_in) / n_depth
            for j in range(n_depth):
                t = t_in + (j + 0.5) * dt
                X = S + t * d0
                R = D - X
                r = np.linalg.norm(R, axis=-1)
                d1 = R / r[..., None]
                cos_psi = d1[..., 0]
                w, e2 = pdf(d1 @ d0)
                d_out = _exit_distance(X, d1, half)
                f = w * cos_psi / (r * r) * dA * e2 * np.exp(-_mu(prob, None, e2) * d_out)
                T += dt * muC * math.exp(-muT * (t - t_in)) * f.sum(axis=(2, 3))
    return T / (n_beam * n_beam)


@pytest.mark.parametrize("energy, sdd, n_det, det_px", [
    (60.0, 1500.0, 32, 8.0),       # the CT geometry: small angles, little energy loss
    (120.0, 1060.0, 64, 4.0),      # imager 44 mm behind the cube: angles to 70 degrees, E' down 13 %
])
def test_single_compton_image_matches_its_integral(energy, sdd, n_det, det_px):
    prob = inputs.uniform_slab_problem(nx=16, ny=16, nz=16, vox=2.0, mat_id=1, density=0.2, energy=energy,
                                       nu=n_det, nv=n_det, det_px=det_px, pencil=True, sdd=sdd)
    n = 4_000_000
    _, ts, st, _ = oracle.mc_run(prob, n, seed=7, threads=8, scatter_filter=1)
    got = oracle.finalize(ts, n)                          # keV per source photon
    want = _expected(prob, half=16.0)
    # rings around the beam's spot on the imager, and the whole image
    iu, iv = np.meshgrid(np.arange(prob.nu), np.arange(prob.nv))
    rho = np.hypot(iu + 0.5 - (prob.nu // 2 + 0.5), iv + 0.5 - (prob.nv // 2 + 0.5))
    q = n_det // 8
    for lo, hi in ((0, q), (q, 2 * q), (2 * q, 3 * q), (3 * q, 4 * q), (4 * q, 6 * q), (0, 6 * q)):
        m = (rho >= lo) & (rho < hi)
        g, w = got[m].sum(), want[m].sum()
        counts = w * n / (0.92 * energy)                  # photons, at a little under E each
        tol = 4.0 / math.sqrt(counts) + 0.002      # statistics, and the quadrature (< 2e-4)
        assert g == pytest.approx(w, rel=tol), (lo, hi, g, w, counts)


@pytest.mark.parametrize("law", ["rayleigh", "rayleigh_ff"])
def test_single_rayleigh_image_matches_its_integral(law):
    # Thomson, and Thomson times the form factor (forward-peaked: half of F at
    # about 11 degrees for water at 60 keV), on the close imager; full-density
    # water for enough Rayleigh events (the attenuation is in the integral)
    prob = inputs.uniform_slab_problem(nx=16, ny=16, nz=16, vox=2.0, mat_id=1, density=1.0, energy=60.0,
                                       nu=64, nv=64, det_px=4.0, pencil=True, sdd=1060.0)
    n = 4_000_000
    _, ts, st, _ = oracle.mc_run(prob, n, seed=9, threads=8, scatter_filter=2, rayleigh_ff=(law == "rayleigh_ff"))
    got = oracle.finalize(ts, n)
    want = _expected(prob, half=16.0, law=law)
    iu, iv = np.meshgrid(np.arange(prob.nu), np.arange(prob.nv))
    rho = np.hypot(iu + 0.5 - (prob.nu // 2 + 0.5), iv + 0.5 - (prob.nv // 2 + 0.5))
    for lo, hi in ((0, 4), (4, 8), (8, 16), (16, 24), (24, 48), (0, 48)):
        m = (rho >= lo) & (rho < hi)
        g, w = got[m].sum(), want[m].sum()
        counts = w * n / 60.0
        tol = 4.0 / math.sqrt(counts) + 0.002
        assert g == pytest.approx(w, rel=tol), (law, lo, hi, g, w, counts)
