"""Pins of the oracle's Step 3 scalars and of its Steps 2-4 chain.

The count scale (the mean signal one detected scattered photon leaves,
Section 2.5's Poisson fidelity read on the count scale) is pinned by physics
the transport fixes exactly: with Rayleigh scattering alone and an ideal
energy-integrating response r(E) = E, a scattered photon keeps its source
energy, so every detected scattered photon of a 60 keV beam leaves exactly
60 keV, and the count scale is 60 keV per source photon divided by n.  With
Compton scattering the scattered photons lose energy, so the scale must fall
below that and above the smallest scattered energy.  The smoothing rule for
beta is pinned by the Eq. 5 convergence floor of the denoiser: a smoothing
length of one coarse pixel keeps beta S at 1 on a flat image and converges,
while the same rule at 0.6 px (beta S = 0.36, below the 0.5 floor at omega =
0.8) grows a checkerboard.
"""
import copy

import numpy as np
import pytest

import oracle
from paper_1204_6367_gb300 import inputs


def _rayleigh_only(prob):
    p = copy.copy(prob)
    mu = np.array(prob.mu_hat, np.float32, copy=True)
    mu[:, 0, :] *= 20.0                      # enough Rayleigh events to count
    mu[:, 1:, :] = 0.0                       # no Compton, no photoelectric absorption
    p.mu_hat = mu
    return p


def test_count_scale_is_the_source_energy_without_energy_loss():
    prob = _rayleigh_only(inputs.small_problem())
    n = 200_000
    tp, ts, st, _ = oracle.mc_run(prob, n, seed=3)
    assert st["tally_scatter"] > 1000 and st["compton"] == 0 and st["photo"] == 0
    cs = oracle.count_scale(ts, n, st["tally_scatter"])
    assert cs == pytest.approx(60.0 / n, rel=1e-12)
    # the primary tally gives the same per-photon value, but divided by the
    # scattered count it does not
    assert float(np.sum(oracle.finalize(tp, n))) / st["tally_scatter"] != pytest.approx(60.0 / n, rel=1e-3)


def test_count_scale_with_compton_lies_below_the_source_energy():
    prob = inputs.small_problem()
    n = 200_000
    _, ts, st, _ = oracle.mc_run(prob, n, seed=4)
    cs = oracle.count_scale(ts, n, st["tally_scatter"])
    # 60 keV Compton: E' >= E / (1 + 2 E / 511) = 48.8 keV after one scattering
    assert 30.0 / n < cs < 60.0 / n
    assert cs * n > 0.9 * 55.0          # most detected scatter is single and forward


def test_count_scale_without_scatter_is_one_photon_share():
    assert oracle.count_scale(np.zeros((4, 4), np.int64), 1000, 0) == 1.0 / 1000


@pytest.mark.parametrize("length,grows", [(1.0, False), (0.6, True)])
def test_smoothing_beta_and_the_convergence_floor(length, grows):
    rng = np.random.default_rng(2)
    n_scat, shape = 96 * 128 * 40, (96, 128)
    mean = oracle.mean_coarse_count(n_scat, shape[0] * shape[1])
    assert mean == 40.0
    beta = oracle.smoothing_beta(length, n_scat, shape[0] * shape[1])
    flat = np.full(shape, mean)
    kick = 1e-3 * mean * (-1.0) ** np.add.outer(np.arange(shape[0]), np.arange(shape[1]))
    s = oracle.denoise(flat, beta, 0.8, 200, s0=flat + kick)
    amp = np.abs(s - flat).max()
    assert (amp > 1e-3 * mean) == grows, amp


def test_project_chain_composes_the_steps():
    prob = inputs.small_problem()
    n = 100_000
    tp, ts, st, _ = oracle.mc_run(prob, n, seed=5)
    P = oracle.rt_primary(prob)
    r = oracle.project_chain(P, tp, ts, n, st["tally_scatter"], bin_factor=4, smoothing_px=2.0, iters=50)
    assert r["S_hat_coarse"].shape == (16, 16) and r["S"].shape == (64, 64)
    # the coarse grid holds the same signal; the upsampled S conserves the
    # coarse total (bilinear interpolation of a block sum over factor^2)
    assert r["S_hat_coarse"].sum() == pytest.approx(r["S_hat"].sum(), rel=1e-12)
    assert r["beta"] == pytest.approx(4.0 / (st["tally_scatter"] / 256.0))
    np.testing.assert_allclose(r["N"], oracle.noise_scale(r["P_hat"], P, r["S_hat"], r["S"], n, 0.4, 5.2913e9))
