"""Pins of the oracle's energy-dependent bowtie (per-column source spectra).

Section 2.1 defines the source as a spectrum phi(E) times a fluence map w(u)
after the bowtie.  An aluminium bowtie also hardens the spectrum off axis, so
the oracle optionally takes one spectrum per detector column.  Pins:

* identical column spectra reduce exactly to the separable source;
* a column whose spectrum has a single bin emits only that energy (catches a
  row/column mix-up and a wrong CDF row);
* narrow-beam transmission through a water slab follows Beer-Lambert with the
  column's own spectrum, for both the Monte Carlo and the ray tracer, and
  differs measurably from the separable spectrum's.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1204_6367_gb300 import inputs


def _spectral_slab(nu=32, nv=8, det_px=1.5, pencil_col=None):
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0, nx=16, ny=16, nz=8, nu=nu, nv=nv,
                                       det_px=det_px, pencil=False)
    e, w = inputs.kramers_spectrum(kvp=100.0, al_mm=2.5, bin_kev=5.0)
    prob.spec_e, prob.spec_w = e, w
    prob.spec_cols = inputs.bowtie_column_spectra(nu, det_px, prob.sdd, e, w, bowtie_mm=30.0)
    if pencil_col is not None:
        prob.fluence[:] = 0.0
        prob.fluence[nv // 2, pencil_col] = 1.0
    return prob


def _mu_mm(prob, mat_id, e):
    tab = prob.mu_hat[mat_id].astype(np.float64).sum(axis=0)
    eg = prob.e0 + prob.de * np.arange(tab.size)
    return 0.1 * np.interp(e, eg, tab)


def test_bowtie_columns_harden_off_axis():
    e, w = inputs.kramers_spectrum(kvp=120.0, bin_kev=1.0)
    cols = inputs.bowtie_column_spectra(65, 4.0, 1500.0, e, w, bowtie_mm=30.0)
    mean_e = (cols * e).sum(1) / cols.sum(1)
    # the centre column sees no aluminium; the mean energy rises towards the edges
    np.testing.assert_array_equal(cols[32], w)
    assert np.all(np.diff(mean_e[32:]) > 0) and np.all(np.diff(mean_e[:33]) < 0)
    np.testing.assert_allclose(mean_e, mean_e[::-1], rtol=1e-12)


def test_identical_columns_reduce_to_separable(small):
    prob = small
    ref = oracle.mc_run(prob, 20000, seed=5, phi=0.3, threads=4, records=True)
    ref_rt = oracle.rt_primary(prob, phi=0.3)
    ref_sd = oracle.rt_primary_siddon(prob, phi=0.3)
    prob.spec_cols = np.tile(np.asarray(prob.spec_w, np.float64), (prob.nu, 1))
    try:
        got = oracle.mc_run(prob, 20000, seed=5, phi=0.3, threads=4, records=True)
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_array_equal(got[1], ref[1])
        assert got[2] == ref[2]
        np.testing.assert_array_equal(got[3], ref[3])
        np.testing.assert_array_equal(oracle.rt_primary(prob, phi=0.3), ref_rt)
        np.testing.assert_array_equal(oracle.rt_primary_siddon(prob, phi=0.3), ref_sd)
    finally:
        prob.spec_cols = None


def test_single_bin_columns_fix_the_source_energy():
    # vacuum: every history is a primary that lands in (or, at a pixel edge
    # in FP32, next to) the column it was aimed at
    prob = _spectral_slab(nu=24, nv=6, det_px=1.2)
    prob.density[:] = 0.0
    nb = prob.spec_e.size
    cols = np.zeros((prob.nu, nb))
    pick = (np.arange(prob.nu) * 5) % nb
    cols[np.arange(prob.nu), pick] = 1.0
    prob.spec_cols = cols
    _, _, _, rec = oracle.mc_run(prob, 20000, seed=12, threads=4, records=True)
    assert np.all(rec["outcome"] == 0)
    iu = rec["pixel"] % prob.nu
    e32 = prob.spec_e.astype(np.float32)
    hit = rec["e_source"] == e32[pick[iu]]
    assert hit.mean() > 0.995
    near = (rec["e_source"] == e32[pick[np.maximum(iu - 1, 0)]]) | \
           (rec["e_source"] == e32[pick[np.minimum(iu + 1, prob.nu - 1)]])
    assert np.all(hit | near)
    assert np.unique(iu).size == prob.nu


@pytest.mark.parametrize("col", [16, 30])
def test_pencil_transmission_follows_the_column_spectrum(col):
    prob = _spectral_slab(pencil_col=col)
    n = 400000
    _, _, st, _ = oracle.mc_run(prob, n, seed=21, threads=8)
    wc = prob.spec_cols[col] / prob.spec_cols[col].sum()
    u = (col + 0.5 - 0.5 * prob.nu) * prob.du
    L = 32.0 * math.hypot(prob.sad, u * prob.sad / prob.sdd) / prob.sad   # chord of the slab along x
    T = np.exp(-_mu_mm(prob, 1, prob.spec_e) * L)
    expect = float((wc * T).sum())
    sigma = math.sqrt(expect * (1 - expect) / n)
    frac = st["tally_primary"] / n
    assert abs(frac - expect) < 3.5 * sigma, (frac, expect)
    # the separable spectrum predicts a different transmission off axis
    sep = float((prob.spec_w / prob.spec_w.sum() * T).sum())
    if col == 30:
        assert abs(frac - sep) > 8 * sigma
    # the ray tracer: ideal response -> signal = w_j sum_b phi_u(b) E_b T_b
    for rt in (oracle.rt_primary, oracle.rt_primary_siddon):
        img = rt(prob)
        j = prob.nv // 2
        # a pixel spans a small range of chords; the centre ray sets the value
        assert img[j, col] == pytest.approx(float((wc * prob.spec_e * T).sum()), rel=2e-3)
