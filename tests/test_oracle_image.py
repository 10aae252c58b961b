"""Pins of the oracle's image-domain steps.

Step 3 (Section 2.5): the Eq. 5 iteration must converge to the minimiser of
the convex energy of Eq. 2, i.e. to a zero of the discrete optimality
condition Eq. 4, independently of the start (convexity), leave a constant
image unchanged, and reduce to the data as beta -> 0.  Linearised, it must
multiply each cosine mode of a flat image by the closed-form growth factor,
which puts its convergence floor at beta S = omega / (8 (1 - omega)).
Step 4 (Section 2.6): the printed calibration example, the 1/sqrt(n) noise
law, and recovery of a known zeta.
"""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle
from tests.golden.load import load


def _smooth_poisson(shape=(24, 32), scale=400.0, seed=0, length=6.0):
    rng = np.random.default_rng(seed)
    v, u = np.mgrid[0:shape[0], 0:shape[1]]
    truth = scale * (1.0 + 0.5 * np.sin(u / length) * np.cos(v / (length * 0.8)))
    return truth, rng.poisson(truth).astype(np.float64)


def test_paper_omega_constant():
    assert load("paper_constants.txt")["omega"] == 0.8


def test_denoise_reaches_eq4_fixed_point():
    _, s_hat = _smooth_poisson()
    beta = 0.05
    s = oracle.denoise(s_hat, beta, omega=0.8, iters=6000)
    res = oracle.optimality_residual(s, s_hat, beta)
    assert np.abs(res).max() < 1e-9


def test_denoise_minimises_eq2_energy():
    # Independent check: minimise the discrete Eq. 2 energy with a library
    # optimiser (L-BFGS-B) and compare with the relaxation iteration.
    truth, s_hat = _smooth_poisson(shape=(10, 12), scale=50.0, seed=3)
    beta = 0.08
    def f(x):
        s = x.reshape(s_hat.shape)
        gx = np.diff(s, axis=1)
        gy = np.diff(s, axis=0)
        e = np.sum(s - s_hat * np.log(s)) + 0.5 * beta * (np.sum(gx**2) + np.sum(gy**2))
        g = 1.0 - s_hat / s
        lap = np.zeros_like(s)
        lap[:, :-1] += gx; lap[:, 1:] -= gx
        lap[:-1, :] += gy; lap[1:, :] -= gy
        return e, (g - beta * lap).ravel()
    res = optimize.minimize(f, np.maximum(s_hat, 1.0).ravel(), jac=True, method="L-BFGS-B",
                            bounds=[(1e-6, None)] * s_hat.size, options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 20000})
    s_ref = res.x.reshape(s_hat.shape)
    s = oracle.denoise(s_hat, beta, omega=0.8, iters=20000)
    np.testing.assert_allclose(s, s_ref, rtol=2e-5)


def test_denoise_independent_of_start():
    _, s_hat = _smooth_poisson(seed=1)
    beta = 0.05
    a = oracle.denoise(s_hat, beta, iters=8000)
    b = oracle.denoise(s_hat, beta, iters=8000, s0=np.full_like(s_hat, s_hat.mean()))
    np.testing.assert_allclose(a, b, rtol=1e-8)


def _cosine_mode(nv, nu, kv, ku):
    # eigenvectors of the neighbour sum with replicate edges: along an axis of
    # n pixels cos(pi k (i + 1/2) / n) has eigenvalue 2 cos(pi k / n)
    j, i = np.indices((nv, nu))
    v = np.cos(math.pi * ku * (i + 0.5) / nu) * np.cos(math.pi * kv * (j + 0.5) / nv)
    return v, 2.0 * math.cos(math.pi * ku / nu) + 2.0 * math.cos(math.pi * kv / nv)


@pytest.mark.parametrize("omega", [0.8, 0.5])
@pytest.mark.parametrize("mode", ["checkerboard", "smooth"])
@pytest.mark.parametrize("beta_c", [0.45, 0.55, 1.0, 3.0])
def test_denoise_linear_growth_factor(omega, mode, beta_c):
    # Linearising Eq. 5 at the fixed point S = S^ = c of a flat image: a
    # perturbation along an eigenvector of the neighbour sum (eigenvalue lam)
    # is multiplied every iteration by
    #     g = 1 - omega + (omega / 4) (lam - 1 / (beta c)),
    # since d/dS (S^ / S) = -S^ / S^2 = -1 / c there.  A wrong relaxation
    # weight, neighbour sum or sign of the data term changes g.
    nv, nu, c = 24, 30, 50.0
    v, lam = _cosine_mode(nv, nu, *((nv - 1, nu - 1) if mode == "checkerboard" else (1, 2)))
    g = 1.0 - omega + omega / 4.0 * (lam - 1.0 / beta_c)
    # as many iterations (2 .. 12) as keep the perturbation above 1e-3 of its start
    k = 12 if abs(g) ** 12 >= 1e-3 else max(2, int(math.log(1e-3) / math.log(abs(g))))
    eps = 1e-6
    beta = beta_c / c
    s = oracle.denoise(np.full((nv, nu), c), beta, omega=omega, iters=k, s0=c + eps * v)
    amp = float(((s - c) * v).sum() / (v * v).sum()) / eps
    assert amp == pytest.approx(g**k, rel=1e-5)


def test_denoise_stability_bound():
    # The checkerboard (lam -> -4) limits the iteration: |g| < 1 needs
    # beta S > omega / (8 (1 - omega)) counts (0.5 at the paper's omega = 0.8),
    # and no beta makes it stable for omega >= 1.  On a flat image at
    # beta S = 0.45 a tiny checkerboard grows; at 0.55 it dies out.
    c, shape = 40.0, (32, 40)
    v, _ = _cosine_mode(*shape, shape[0] - 1, shape[1] - 1)
    amp = {}
    for beta_c in (0.45, 0.55):
        s = oracle.denoise(np.full(shape, c), beta_c / c, omega=0.8, iters=400, s0=c + 1e-6 * v)
        amp[beta_c] = np.abs(s - c).max()
    assert amp[0.45] > 1e-3 and amp[0.55] < 1e-9


def test_denoise_constant_and_small_beta():
    c = np.full((16, 20), 123.0)
    np.testing.assert_allclose(oracle.denoise(c, 0.3, iters=50), c, rtol=1e-14)
    # beta -> 0 leaves the data term alone: S -> S^.  The Eq. 5 iteration is
    # stable only while beta * S > omega / (8 (1 - omega)) counts (the
    # checkerboard bound above), so shrink beta within that range.
    _, s_hat = _smooth_poisson(seed=2)
    dist = [np.linalg.norm(oracle.denoise(s_hat, b, iters=4000) - s_hat) / np.linalg.norm(s_hat)
            for b in (0.05, 0.02, 0.008)]
    assert dist[0] > dist[1] > dist[2] and dist[2] < 0.07


def test_denoise_reduces_noise():
    truth, s_hat = _smooth_poisson(shape=(48, 64), scale=400.0, seed=4, length=20.0)
    s = oracle.denoise(s_hat, 0.01, iters=3000)
    err_raw = np.linalg.norm(s_hat - truth) / np.linalg.norm(truth)
    err_den = np.linalg.norm(s - truth) / np.linalg.norm(truth)
    assert err_den < 0.4 * err_raw


def test_zeta_printed_example():
    g = load("paper_noise_calibration.txt")
    zeta = g["n_sim"] / g["k"] ** 2
    assert zeta == pytest.approx(g["zeta"], rel=g["rel_tol"])
    # the fit reproduces it from exact data on the line ratio = k / sqrt(I)
    inv_sqrt = 1.0 / np.sqrt(np.array([0.1, 0.2, 0.4, 0.8, 1.6]))
    z, k = oracle.fit_zeta(inv_sqrt, g["k"] * inv_sqrt, g["n_sim"])
    assert k == pytest.approx(g["k"], rel=1e-12)
    assert z == pytest.approx(g["zeta"], rel=g["rel_tol"])


def test_fit_recovers_known_zeta():
    rng = np.random.default_rng(7)
    n_sim, zeta = 1e8, 3.3e9
    mas = np.array([0.2, 0.4, 0.63, 1.0, 1.6, 2.5])
    k = math.sqrt(n_sim / zeta)
    ratio = k / np.sqrt(mas) * (1 + 0.002 * rng.standard_normal(mas.size))
    z, _ = oracle.fit_zeta(1 / np.sqrt(mas), ratio, n_sim)
    assert z == pytest.approx(zeta, rel=0.01)


def test_noise_scale_law():
    # N = N^ sqrt(n_sim / (zeta I)): a noise image drawn at n_sim photons,
    # scaled to zeta*I photons, has the standard deviation of one drawn there.
    rng = np.random.default_rng(5)
    p = np.full((64, 64), 0.3)
    n_sim, zeta, mas = 1e6, 5.2913e9, 0.4
    p_hat = rng.binomial(int(n_sim), p) / n_sim
    n = oracle.noise_scale(p_hat, p, np.zeros_like(p), np.zeros_like(p), n_sim, mas, zeta)
    expect_sd = math.sqrt(p[0, 0] * (1 - p[0, 0]) / (zeta * mas))
    assert n.std() == pytest.approx(expect_sd, rel=0.03)
    np.testing.assert_allclose(n, (p_hat - p) * math.sqrt(n_sim / (zeta * mas)), rtol=1e-15)


def test_mc_noise_variance_scales_with_photons(small):
    # Section 2.6: the MC noise amplitude goes as 1/sqrt(n_sim).
    p_rt = oracle.rt_primary(small)
    sds = []
    for n in (50000, 800000):
        tp, _, _, _ = oracle.mc_run(small, n, seed=31, threads=8)
        m = p_rt > 0.2 * p_rt.max()
        sds.append(np.std((oracle.finalize(tp, n) - p_rt)[m]))
    assert sds[0] / sds[1] == pytest.approx(4.0, rel=0.08)


def test_bin_and_upsample():
    rng = np.random.default_rng(0)
    t = rng.integers(0, 2**40, size=(16, 24), dtype=np.int64)
    b = oracle.bin_tally(t, 4)
    assert b.shape == (4, 6) and b.sum() == t.sum() and b[1, 2] == t[4:8, 8:12].sum()
    # a linear coarse image is reproduced exactly by bilinear interpolation
    # away from the clamped border, and the per-pixel values sum back
    jj, ii = np.mgrid[0:6, 0:8]
    coarse = 3.0 + 2.0 * ii + 0.5 * jj
    fine = oracle.upsample(coarse, 4)
    v, u = np.mgrid[0:24, 0:32]
    lin = (3.0 + 2.0 * ((u + 0.5) / 4 - 0.5) + 0.5 * ((v + 0.5) / 4 - 0.5)) / 16.0
    inner = (slice(2, -2), slice(2, -2))
    np.testing.assert_allclose(fine[inner], lin[inner], rtol=1e-13)
