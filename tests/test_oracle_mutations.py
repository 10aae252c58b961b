"""The oracle's pins must catch plausible mistakes.

Each case below plants one mistake (a dropped term, a wrong sign or index, a
swapped operand) in a temporary copy of the oracle, rebuilds it, and runs
the oracle pin tests against that copy.  The test passes when the pins fail.
Mistakes are planted only in the CPU oracle, never in GPU code.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (file, original text, planted text, what it breaks, pin files expected to catch it)
MUTATIONS = [
    ("mc_history.inc", "if (r1 <= (RC(1) + ta) / (RC(9) + ta)) {", "if (r1 <= (RC(1) + ta) / (RC(8) + ta)) {",
     "Kahn branch probability", "test_oracle_sampling.py"),
    ("mc_history.inc", "if (r3 <= RC(0.5) * (ct * ct + RC(1) / x)) break;", "if (r3 <= RC(0.5) * (ct * ct + x)) break;",
     "Kahn second-branch acceptance", "test_oracle_sampling.py"),
    ("mc_history.inc", "nw_ = w * ct - st * t * cp;", "nw_ = w * ct + st * t * cp;",
     "rotation sign", "test_oracle_sampling.py"),
    ("mc_history.inc", "*sp = RC(2) * a * b * inv;", "*sp = RC(2) * a * a * inv;",
     "azimuth sine", "test_oracle_sampling.py"),
    ("mc_history.inc", "if (RC(2) * b <= RC(1) + mu * mu || rs->ctr[0] >= ORC_MAX_BLOCKS) return mu;",
     "if (b <= RC(1) + mu * mu || rs->ctr[0] >= ORC_MAX_BLOCKS) return mu;",
     "Thomson acceptance", "test_oracle_sampling.py"),
    ("mc_history.inc", "w0[a] = RC(1) - t; w1[a] = t;", "w0[a] = t; w1[a] = RC(1) - t;",
     "trilinear weights swapped", "test_oracle_transport.py"),
    ("mc_history.inc", "channel = t <= muR ? 1 : (t <= muR + muC ? 2 : 3);", "channel = t <= muR ? 1 : (t <= muR + muR ? 2 : 3);",
     "interaction channels mixed up", "test_oracle_transport.py"),
    ("mc_history.inc", "REAL s = -LOGR(xi_s) * inv_mumax;", "REAL s = -LOGR(xi_s) * (RC(1.1) * inv_mumax);",
     "free path scale", "test_oracle_transport.py"),
    ("mc_history.inc", "for (int corner = 0; corner < n_corner; ++corner) muT = muT + a[corner] * cT[mc[corner]];",
     "for (int corner = 0; corner < n_corner; ++corner) muT = a[corner] * cT[mc[corner]];",
     "dropped corner terms", "test_oracle_transport.py"),
    ("mc_history.inc", "cT[m] = (cR[m] + cC[m]) + cP[m];", "cT[m] = cR[m] + cC[m];",
     "photoelectric missing from the total", "test_oracle_transport.py"),
    ("mc_history.inc", "int64_t iy = cy ? i1[1] : i0[1];", "int64_t iy = cy ? i1[0] : i0[0];",
     "wrong corner index", "test_oracle_transport.py"),
    ("mc_history.inc", "REAL fu = au * GEO(idu) + GEO(hu);", "REAL fu = -au * GEO(idu) + GEO(hu);",
     "detector u axis flipped", "test_oracle_transport.py"),
    ("mc_history.inc", "scattered = 1;\n                r.n_rayleigh++;", "r.n_rayleigh++;",
     "Rayleigh not marked as scatter", "test_oracle_transport.py"),
    ("mc_history.inc", "r.e_deposited += (double)e - (double)e2;", "r.e_deposited += (double)e;",
     "energy ledger", "test_oracle_transport.py"),
    ("gdrr_oracle.c", "if (xi <= cdf[mid]) hi = mid; else lo = mid + 1;", "if (xi < cdf[mid]) hi = mid; else lo = mid + 1;",
     "inverse-CDF boundary (harmless for continuous xi, must NOT be required)", None),
    ("gdrr_oracle.c", "uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;", "uint32_t n2 = (uint32_t)(p0 >> 32) ^ c1 ^ k1;",
     "Philox round word", "test_oracle_rng.py"),
    ("gdrr_oracle.c", "k1 += 0xBB67AE85u;", "k1 += 0x9E3779B9u;",
     "Philox key schedule", "test_oracle_rng.py"),
    ("gdrr_oracle.c", "float poly = (float)(1.0 / 3.0) + s2 * ((float)(1.0 / 5.0)", "float poly = (float)(1.0 / 3.0) + s2 * ((float)(1.0 / 6.0)",
     "log series term", "test_oracle_rng.py"),
    ("gdrr_oracle.c", "major[e] = (float)(mx * (1.0 + 1e-5));", "major[e] = (float)(mx * 0.8);",
     "majorant below mu", "test_oracle_transport.py"),
    ("gdrr_oracle.c", "rad += dl * orc_mu_at(&c, x, &mu_e[(size_t)b * p->n_mat]);", "rad += 0.5 * orc_mu_at(&c, x, &mu_e[(size_t)b * p->n_mat]);",
     "ray-tracing interval length", "test_oracle_rt.py"),
    ("gdrr_oracle.c", "double tt = tmin + (s + 0.5) * dl, x[3];", "double tt = tmin + s * dl, x[3];",
     "interval end point instead of midpoint", "test_oracle_rt.py"),
    ("mc_history.inc", "c->cdf_e_cols + (size_t)iu * p->n_bins", "c->cdf_e_cols + (size_t)iv * p->n_bins",
     "column spectrum indexed by the detector row", "test_oracle_bowtie.py"),
    ("gdrr_oracle.c", "double* col = orc_build_cdf(p->bin_w_cols + (size_t)u * p->n_bins, p->n_bins);",
     "double* col = orc_build_cdf(p->bin_w, p->n_bins);",
     "column spectra ignored by the energy sampler", "test_oracle_bowtie.py"),
    ("mc_history.inc", "acc = acc + a[corner] * cR[mc[corner]];", "acc = acc + a[corner];",
     "form-factor material picked by corner weight alone", "test_oracle_rayleigh_ff.py"),
    ("mc_history.inc", "REAL s = S[lo - 1] + RC(2) * D / (g0 + SQRTR(q));", "REAL s = S[lo - 1] + D / g0;",
     "form-factor interval inverted as if F^2 were constant", "test_oracle_rayleigh_ff.py"),
    ("mc_history.inc", "REAL xmax = e * GEO(inv_hc);", "REAL xmax = RC(0.5) * e * GEO(inv_hc);",
     "momentum transfer of a wavelength off by two", "test_oracle_rayleigh_ff.py"),
    ("gdrr_oracle.c", "acc += 0.5 * (f0 * f0 + f1 * f1) * (c->gd.ff_s[j] - c->gd.ff_s[j - 1]);",
     "acc += 0.5 * (f0 + f1) * (c->gd.ff_s[j] - c->gd.ff_s[j - 1]);",
     "form factor not squared in the cumulative", "test_oracle_rayleigh_ff.py"),
    ("fdk.py", "e0, e1 = math.sin(phi), -math.cos(phi)", "e0, e1 = -math.sin(phi), math.cos(phi)",
     "reconstruction u axis mirrored", "test_oracle_fdk.py"),
    ("fdk.py", "out[i, r] = 0.5 * tau * full[nu - 1:2 * nu - 1]", "out[i, r] = tau * full[nu - 1:2 * nu - 1]",
     "full-scan factor 1/2 of the filter dropped", "test_oracle_fdk.py"),
    ("fdk.py", "f += d_beta * val / (U * U)", "f += d_beta * val",
     "FDK distance weight dropped", "test_oracle_fdk.py"),
    ("fdk.py", "w = sad / np.sqrt(sad * sad + a[None, :] ** 2 + b[:, None] ** 2)", "w = 1.0",
     "FDK cosine weight dropped", "test_oracle_fdk.py"),
    ("fdk.py", "h[odd] = -1.0 / (np.pi * k[odd] * tau) ** 2", "h[odd] = -1.0 / (np.pi * k[odd] * tau ** 2)",
     "Ram-Lak odd taps", "test_oracle_fdk.py"),
    ("oracle.py", "sigma - (1.0 / beta) * (1.0 - s_hat / s)", "sigma - (1.0 / beta) * (1.0 - s / s_hat)",
     "denoiser fidelity term", "test_oracle_image.py"),
    ("oracle.py", "sigma = ((p[1:-1, 2:] + p[2:, 1:-1]) + p[1:-1, :-2]) + p[:-2, 1:-1]\n        s = ",
     "sigma = ((p[1:-1, 2:] + p[2:, 1:-1]) + p[1:-1, :-2]) + p[1:-1, 1:-1]\n        s = ",
     "denoiser stencil", "test_oracle_image.py"),
    ("mc_history.inc", "*e_out = e / x;", "*e_out = e;",
     "Compton-scattered photon keeps its energy", "test_oracle_scatter_geometry.py"),
    ("mc_history.inc", "nw_ = w * ct - st * t * cp;", "nw_ = w * ct + st * t * cp;",
     "rotation sign, seen through multiple scattering", "test_oracle_analog.py"),
    ("mc_history.inc", "channel = t <= muR ? 1 : (t <= muR + muC ? 2 : 3);",
     "channel = t <= muR ? 1 : (t <= muR + muR ? 2 : 3);",
     "interaction channels, seen in the scatter image", "test_oracle_analog.py"),
    ("mc_history.inc", "int64_t q = (int64_t)LLRINTR(FN(response)(c, e) * RC(16777216.0));",
     "int64_t q = (int64_t)LLRINTR(FN(response)(c, (REAL)r.e_source) * RC(16777216.0));",
     "detector response at the source energy", "test_oracle_scatter_geometry.py"),
    ("oracle.py", "s = (1.0 - omega) * s + (omega / 4.0) * (sigma", "s = (1.0 - omega) * s + (omega / 2.0) * (sigma",
     "denoiser relaxation weight", "test_oracle_image.py"),
    ("oracle.py", "        p = np.pad(s, 1, mode=\"edge\")\n        sigma", "        p = np.pad(s, 1, mode=\"wrap\")\n        sigma",
     "denoiser edges wrap around instead of replicating", "test_oracle_image.py"),
    ("oracle.py", "return n_hat * np.sqrt(float(n_sim) / (zeta * mas))", "return n_hat * np.sqrt(float(n_sim) * (zeta * mas))",
     "noise scaling", "test_oracle_image.py"),
    ("oracle.py", "scale = total / max(1, int(n_scat))", "scale = total / max(1, int(n_photons))",
     "count scale divided by the source photons", "test_oracle_project.py"),
    ("oracle.py", "total = float(np.sum(finalize(scat_tally, n_photons)))", "total = float(np.sum(scat_tally))",
     "count scale from the raw fixed-point tally", "test_oracle_project.py"),
    ("oracle.py", "return smoothing_px * smoothing_px / max(", "return smoothing_px / max(",
     "smoothing length not squared", "test_oracle_project.py"),
    ("mc_history.inc", "return GEO(lo)[a] + ((REAL)(j << c->p->cell_shift) + RC(0.5)) * GEO(vox)[a];",
     "return GEO(lo)[a] + ((REAL)(j << c->p->cell_shift) + RC(0)) * GEO(vox)[a];",
     "local-majorant cell planes half a voxel off", "test_oracle_local_majorant.py"),
    ("mc_history.inc", "tau = tau - bt;", "tau = tau - RC(0.5) * bt;",
     "optical depth of a crossed cell half spent", "test_oracle_local_majorant.py"),
    ("mc_history.inc", "REAL sc = tau / b;", "REAL sc = tau * b;",
     "tentative collision distance inverted", "test_oracle_local_majorant.py"),
    ("mc_history.inc", "nk[a] += d[a] > RC(0) ? 1 : -1;", "nk[a] += 1;",
     "cells stepped forward along negative directions", "test_oracle_local_majorant.py"),
    ("mc_history.inc", "REAL f = (x[a] - GEO(lo)[a]) * GEO(ivox)[a] - RC(0.5);",
     "REAL f = (x[a] - GEO(lo)[a]) * GEO(ivox)[a];",
     "entry cell by the containing voxel instead of the lower corner", "test_oracle_local_majorant.py"),
    ("mc_history.inc", "REAL t = (REAL)uf[1] * maj;", "REAL t = (REAL)uf[1] * mumax;",
     "local tentative collisions tested against the global majorant", "test_oracle_local_majorant.py"),
    ("gdrr_oracle.c", "v1[a] = (k[a] + 1) << s;", "v1[a] = ((k[a] + 1) << s) - 1;",
     "cell cover without the next voxel layer", "test_oracle_local_majorant.py"),
]


def _run_pins(tmp, pin_file):
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", os.path.join("tests", pin_file)]
    return subprocess.run(cmd, cwd=tmp, env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("case", [m for m in MUTATIONS if m[4]], ids=lambda m: m[3])
def test_pins_catch_planted_mistake(case, tmp_path):
    fname, old, new, _, pin_file = case
    tmp = str(tmp_path)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(tmp, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(tmp, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutations.py"))
    path = os.path.join(tmp, "oracle", fname)
    src = open(path).read()
    assert src.count(old) == 1, f"mutation anchor not unique in {fname}: {old!r}"
    open(path, "w").write(src.replace(old, new))
    res = _run_pins(tmp, pin_file)
    assert res.returncode != 0, f"pins in {pin_file} did not catch: {case[3]}\n{res.stdout[-2000:]}"
