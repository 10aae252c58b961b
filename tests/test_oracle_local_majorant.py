"""Pins of the oracle's local-majorant tracking, the option beside the paper's
global Woodcock majorant (Section 2.4).

Delta tracking stays exact for any majorant that bounds mu along the flight.
The option takes one per macro cell: per material the largest density over the
cell's voxels and the next layer, times the material's coefficient, raised by
2^-10.  What fixes it, independently of the oracle's code:
  * the cell table is a maximum over a set of voxels: brute force;
  * the bound is never below the trilinear mixture anywhere in the cell (the
    reason for the extra voxel layer): random points in fp64;
  * a flight of optical depth tau ends where the integral of the
    piecewise-constant majorant along the ray reaches tau, or leaves the box
    when the integral to the box face is smaller: a fine numerical integral;
  * the images are those of the global majorant: Beer-Lambert narrow-beam
    transmission and the analog transport of `analog_transport.py`;
  * it takes fewer flights than the global majorant where densities differ.
"""
import math

import numpy as np
import pytest

import oracle
from analog_transport import transport
from paper_1204_6367_gb300 import inputs

MARGIN = 1.0 + 2.0**-10


def _blocky_problem(seed=3, shape=(9, 13, 20), voxel=(2.0, 1.5, 3.0)):
    """A phantom of random 3-voxel blocks of three materials and a vacuum
    corner, anisotropic voxels, sizes that no cell size divides."""
    rng = np.random.default_rng(seed)
    prob = inputs.uniform_slab_problem(nx=shape[2], ny=shape[1], nz=shape[0])
    nz, ny, nx = shape
    blocks = rng.integers(0, 3, size=(nz // 3 + 1, ny // 3 + 1, nx // 3 + 1))
    mat = np.kron(blocks, np.ones((3, 3, 3), np.int64))[:nz, :ny, :nx].astype(np.uint8)
    den = rng.uniform(0.2, 2.0, size=(nz, ny, nx)).astype(np.float32)
    den[mat == 0] = 0.0012
    den[:3, :4, :5] = 0.0                     # vacuum: cells of bound zero
    prob.material, prob.density, prob.voxel = mat, den, voxel
    return prob


def _table(prob, s):
    """Per cell and material the largest density over the voxels
    [k 2^s, (k + 1) 2^s] of each axis (clamped to the phantom)."""
    nz, ny, nx = prob.material.shape
    nm = prob.mu_hat.shape[0]
    nc = [((n - 1) >> s) + 1 for n in (nz, ny, nx)]
    out = np.zeros(nc + [nm], np.float32)
    for kz in range(nc[0]):
        for ky in range(nc[1]):
            for kx in range(nc[2]):
                sl = tuple(slice(k << s, min((k + 1) << s, n - 1) + 1) for k, n in zip((kz, ky, kx), (nz, ny, nx)))
                m, d = prob.material[sl].ravel(), prob.density[sl].ravel()
                for i in range(nm):
                    if (m == i).any():
                        out[kz, ky, kx, i] = d[m == i].max()
    return out


def _mu_tot(prob, e):
    """Total coefficient per material at e (mm^-1 per g/cm^3), the float table
    interpolated linearly."""
    tab = (prob.mu_hat.astype(np.float64) * 0.1).astype(np.float32).astype(np.float64)
    eg = prob.e0 + prob.de * np.arange(tab.shape[2])
    return np.array([np.interp(e, eg, tab[m].sum(axis=0)) for m in range(tab.shape[0])])


def _box(prob):
    nz, ny, nx = prob.material.shape
    vox = np.array(prob.voxel, np.float64)
    n = np.array([nx, ny, nz], np.float64)
    return -0.5 * n * vox, 0.5 * n * vox, vox, np.array([nx, ny, nz])


def _cells_of(prob, s, x):
    """Cells (x, y, z order) of points x [..., 3]: the lower trilinear corner
    max(floor((x - lo) / vox - 1/2), 0), shifted down by s."""
    lo, _, vox, n = _box(prob)
    g = np.maximum(np.floor((x - lo) / vox - 0.5), 0).astype(np.int64) >> s
    return np.minimum(g, ((n - 1) >> s))


def _mixture(prob, x, mu_m):
    """mu at points x [..., 3]: the trilinear mixture of the eight corner
    voxels (clamp to edge), fp64."""
    lo, _, vox, n = _box(prob)
    f = (x - lo) / vox - 0.5
    g = np.floor(f).astype(np.int64)
    t = f - g
    out = np.zeros(x.shape[:-1])
    for c in range(8):
        bits = [(c >> a) & 1 for a in range(3)]
        idx = [np.clip(g[..., a] + bits[a], 0, n[a] - 1) for a in range(3)]
        w = np.ones(x.shape[:-1])
        for a in range(3):
            w = w * (t[..., a] if bits[a] else 1.0 - t[..., a])
        rho = prob.density[idx[2], idx[1], idx[0]].astype(np.float64)
        m = prob.material[idx[2], idx[1], idx[0]]
        out += w * rho * mu_m[m]
    return out


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_cell_table_is_the_cover_maximum(s):
    prob = _blocky_problem()
    np.testing.assert_array_equal(oracle.lm_cells(prob, s), _table(prob, s))


@pytest.mark.parametrize("s", [1, 2])
def test_bound_covers_the_mixture(s):
    # Random points, many near cell planes: mu there never exceeds the bound
    # of the point's cell.  A cover without the next voxel layer fails this.
    prob = _blocky_problem()
    rng = np.random.default_rng(5)
    lo, hi, vox, _ = _box(prob)
    x = lo + (hi - lo) * rng.random((200000, 3))
    near = rng.random(200000) < 0.5            # snap half of them next to a plane
    k = np.round((x - lo) / vox - 0.5) // (1 << s) * (1 << s)
    x[near] = (lo + (k + 0.5) * vox + rng.uniform(-1e-3, 1e-3, (200000, 3)))[near]
    x = np.clip(x, lo, hi)
    tab = _table(prob, s).astype(np.float64)
    for e in (30.0, 60.0, 110.0):
        mu_m = _mu_tot(prob, e)
        cz, cy, cx = [_cells_of(prob, s, x)[:, a] for a in (2, 1, 0)]
        b = (tab[cz, cy, cx] * mu_m).max(axis=1) * MARGIN
        mu = _mixture(prob, x, mu_m)
        assert np.all(mu <= b * (1 + 1e-9)), (mu - b).max()
        assert (mu > 0.9 * b).mean() > 0.002     # and it is tight in places


def _depth_along(prob, s, e, pos, d, t_end, dt):
    """Midpoint samples of the majorant along the ray up to t_end: sample
    times, the majorant there, the cells."""
    t = (np.arange(int(math.ceil(t_end / dt))) + 0.5) * dt
    t = t[t < t_end]
    x = pos[None, :] + t[:, None] * d[None, :]
    cells = _cells_of(prob, s, x)
    tab = _table(prob, s).astype(np.float64)
    b = (tab[cells[:, 2], cells[:, 1], cells[:, 0]] * _mu_tot(prob, e)).max(axis=1) * MARGIN
    return t, b, cells


def _box_exit(prob, pos, d):
    lo, hi, _, _ = _box(prob)
    te = np.inf
    for a in range(3):
        if d[a] > 0:
            te = min(te, (hi[a] - pos[a]) / d[a])
        elif d[a] < 0:
            te = min(te, (lo[a] - pos[a]) / d[a])
    return te


@pytest.mark.parametrize("s", [1, 2])
def test_flight_spends_the_optical_depth_of_the_majorant(s):
    # One flight from random points along random (and axis-parallel, and
    # diagonal) directions: where it stops, the integral of the majorant along
    # the ray equals tau; when it leaves the box, the integral to the face is
    # below tau.  The cells it crossed are the ones the ray passes.
    prob = _blocky_problem()
    rng = np.random.default_rng(11)
    lo, hi, vox, _ = _box(prob)
    e = 60.0
    dirs = [np.array(v, np.float64) for v in ((1, 0, 0), (0, -1, 0), (0, 0, 1), (1, 1, 0), (-1, 1, 1))]
    n_ok = n_cross_ok = n_hits = n_esc = n_b_ok = 0
    cases = 150
    for i in range(cases):
        pos = lo + (hi - lo) * rng.uniform(0.02, 0.98, 3)
        d = dirs[i % len(dirs)] if i < 20 else rng.normal(size=3)
        d = d / np.linalg.norm(d)
        tau = rng.exponential(1.0) * (0.3 if i % 2 else 3.0)
        hit, x, b, n = oracle.lm_walk(prob, s, pos, d, e, tau, precision=64)
        t_exit = _box_exit(prob, pos, d)
        dt = 2e-3 * vox.min()
        t, bs, cells = _depth_along(prob, s, e, pos, d, t_exit, dt)
        depth = np.concatenate([[0.0], np.cumsum(bs * dt)])
        tol = 3 * bs.max() * dt * (1 + np.count_nonzero(np.any(np.diff(cells, axis=0) != 0, axis=1)))
        if hit:
            n_hits += 1
            t_or = float(np.dot(x - pos, d))
            assert np.allclose(x, pos + t_or * d, atol=1e-9)
            assert 0 <= t_or <= t_exit + 1e-9
            j = min(int(t_or / dt), len(t) - 1)
            d_at = depth[j] + bs[j] * (t_or - j * dt)
            assert abs(d_at - tau) <= tol, (i, d_at, tau, tol)
            # the bound returned is the one of the cell the flight ended in
            xb = pos + max(t_or - 1e-7, 0.0) * d
            cb = _cells_of(prob, s, xb[None, :])[0]
            bb = (_table(prob, s).astype(np.float64)[cb[2], cb[1], cb[0]] * _mu_tot(prob, e)).max() * MARGIN
            n_b_ok += b == pytest.approx(bb, rel=1e-12)
            k = max(int(t_or / dt - 0.5), 0)
            brute = int(np.count_nonzero(np.any(np.diff(cells[:k + 1], axis=0) != 0, axis=1)))
        else:
            n_esc += 1
            assert depth[-1] <= tau + tol, (i, depth[-1], tau)
            brute = int(np.count_nonzero(np.any(np.diff(cells, axis=0) != 0, axis=1)))
        n_ok += 1
        n_cross_ok += n == brute
    assert n_ok == cases and n_hits > 30 and n_esc > 30
    assert n_cross_ok >= 0.95 * cases, n_cross_ok
    assert n_b_ok >= n_hits - 2, (n_b_ok, n_hits)


def test_fp32_flight_follows_the_fp64_flight():
    prob = _blocky_problem()
    rng = np.random.default_rng(12)
    lo, hi, _, _ = _box(prob)
    agree = 0
    for i in range(200):
        pos = lo + (hi - lo) * rng.uniform(0.02, 0.98, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        tau = rng.exponential(1.0)
        h64, x64, b64, n64 = oracle.lm_walk(prob, 1, pos, d, 60.0, tau, precision=64)
        h32, x32, b32, n32 = oracle.lm_walk(prob, 1, pos, d, 60.0, tau, precision=32)
        if h64 == h32 and n64 == n32 and np.allclose(x32, x64, atol=1e-3) and (not h64 or b32 == pytest.approx(b64, rel=1e-5)):
            agree += 1
    assert agree >= 196


def _mu_mm(prob, mat_id, e):
    tab = prob.mu_hat[mat_id].astype(np.float64).sum(axis=0)
    eg = prob.e0 + prob.de * np.arange(tab.size)
    return 0.1 * float(np.interp(e, eg, tab))


def _check_binomial(frac, expect, n, nsig=3.0):
    sigma = math.sqrt(expect * (1 - expect) / n)
    assert abs(frac - expect) < nsig * sigma, (frac, expect, sigma)


@pytest.mark.parametrize("s", [1, 2])
def test_narrow_beam_two_materials_and_ramp(s):
    # Water then bone along the beam, and a density ramp: the cells along the
    # beam have different bounds, so the flights cross cells of unequal depth.
    n = 400000
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0)
    prob.material[:, :, 8:] = 2
    prob.density[:, :, 8:] = 1.85
    _, _, st, _ = oracle.mc_run(prob, n, seed=1, threads=8, local_majorant=True, cell_shift=s)
    dx = prob.voxel[0]
    expect = math.exp(-(8 * dx * 1.0 * _mu_mm(prob, 1, 60.0) + 8 * dx * 1.85 * _mu_mm(prob, 2, 60.0)))
    _check_binomial(st["tally_primary"] / n, expect, n)
    assert st["crossings"] > n

    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0, nx=24)
    ramp = np.linspace(0.2, 2.4, 24).astype(np.float32)
    prob.density[:] = ramp[None, None, :]
    _, _, st, _ = oracle.mc_run(prob, n, seed=2, threads=8, local_majorant=True, cell_shift=s)
    expect = math.exp(-prob.voxel[0] * float(ramp.astype(np.float64).sum()) * _mu_mm(prob, 1, 60.0))
    _check_binomial(st["tally_primary"] / n, expect, n)


def test_loose_cell_far_from_the_beam_changes_nothing():
    # Dense bone far from the beam raises the global majorant but not the
    # bounds of the cells the beam crosses: local majorants keep the flights
    # of the water-only phantom, and the transmission.
    prob = inputs.uniform_slab_problem(mat_id=1, density=1.0)
    n = 200000
    _, _, st0, _ = oracle.mc_run(prob, n, seed=1, threads=8, local_majorant=True, cell_shift=1)
    prob.material[0, 0, 0] = 2
    prob.density[0, 0, 0] = 8.0
    _, _, st1, _ = oracle.mc_run(prob, n, seed=1, threads=8, local_majorant=True, cell_shift=1)
    _, _, stw, _ = oracle.mc_run(prob, n, seed=1, threads=8)
    # unscattered photons never enter the bone's cell: their histories are the
    # same draw for draw; scattered ones rarely do
    assert st1["tally_primary"] == st0["tally_primary"]
    assert abs(st1["steps"] - st0["steps"]) < 0.01 * st0["steps"]
    assert stw["virtual"] > 5 * st1["virtual"] + 1000
    expect = math.exp(-_mu_mm(prob, 1, 60.0) * prob.material.shape[2] * prob.voxel[0])
    _check_binomial(st1["tally_primary"] / n, expect, n)


def test_local_majorant_matches_analog_transport():
    # The layered phantom of the global-majorant pin (water, a lung-density
    # slice, bone): primary and the scatter image of all orders, ring by ring.
    prob = inputs.uniform_slab_problem(nx=16, ny=16, nz=16, vox=2.0, mat_id=1, density=1.0, energy=60.0,
                                       nu=64, nv=64, det_px=4.0, pencil=True, sdd=1060.0)
    prob.density[:, :, 3] = 0.3
    prob.material[:, :, 8:] = 2
    prob.density[:, :, 8:] = 1.85
    n = 2_000_000
    a_prim, a_scat = transport(prob, n, seed=1, half=16.0)
    tp, ts, st, _ = oracle.mc_run(prob, n, seed=5, threads=8, local_majorant=True, cell_shift=1)
    o_prim, o_scat = oracle.finalize(tp, n), oracle.finalize(ts, n)
    c = a_prim.sum() * n / 60.0
    assert o_prim.sum() == pytest.approx(a_prim.sum(), rel=4.0 * math.sqrt(2.0 / c) + 0.002)
    iu, iv = np.meshgrid(np.arange(prob.nu), np.arange(prob.nv))
    rho = np.hypot(iu + 0.5 - (prob.nu // 2 + 0.5), iv + 0.5 - (prob.nv // 2 + 0.5))
    for lo, hi in ((0, 4), (4, 8), (8, 16), (16, 24), (24, 48), (0, 48)):
        m = (rho >= lo) & (rho < hi)
        a, o = a_scat[m].sum(), o_scat[m].sum()
        c = a * n / 57.0
        assert o == pytest.approx(a, rel=4.0 * math.sqrt(2.0 / c) + 0.002), (lo, hi, o, a, c)


def test_torso_fewer_flights_same_images():
    # The torso at 8 mm with its bowtie and 120 kVp spectrum: the local
    # majorants cut the flights and agree with the global majorant's images
    # and event counts within the statistics of the two runs.
    prob = inputs.torso_problem(vox=8.0, nu=64, nv=48, det_px=0.776 * 8)
    n = 300000
    tw, sw, stw, _ = oracle.mc_run(prob, n, seed=7, threads=8)
    tl, sl, stl, _ = oracle.mc_run(prob, n, seed=8, threads=8, local_majorant=True, cell_shift=1)
    assert stl["steps"] < 0.5 * stw["steps"] and stl["crossings"] > 0 and stw["crossings"] == 0
    for k in ("tally_primary", "tally_scatter", "miss", "rayleigh", "compton", "photo"):
        a, b = stw[k], stl[k]
        assert abs(a - b) < 4.0 * math.sqrt(2.0 * max(a, b)) + 2, (k, a, b)
    for a, b, key in ((tw, tl, "tally_primary"), (sw, sl, "tally_scatter")):
        # 4 x 4 pixel blocks; photon counts in a block are about its tally over
        # the mean tally per photon, and their spread sets the tolerance
        A = a.reshape(12, 4, 16, 4).sum(axis=(1, 3)).astype(np.float64)
        B = b.reshape(12, 4, 16, 4).sum(axis=(1, 3)).astype(np.float64)
        unit = (A.sum() + B.sum()) / (stw[key] + stl[key])
        sig = 1.5 * np.sqrt((A + B) / unit) * unit
        assert np.all(np.abs(A - B) <= 5.0 * sig + 3.0 * unit), np.abs(A - B).max() / unit


def test_fp64_histories_follow_the_fp32_histories(small):
    # The same streams in FP32 (the parity reference) and FP64 (the accuracy
    # reference): rounding can flip a decision only where it sits within
    # ~1e-7 of a threshold, so nearly every history ends the same way, and
    # the per-history counts agree.
    n = 20000
    _, _, s32, r32 = oracle.mc_run(small, n, seed=13, records=True, local_majorant=True, cell_shift=2)
    _, _, s64, r64 = oracle.mc_run(small, n, seed=13, records=True, local_majorant=True, cell_shift=2,
                                   precision=64)
    same = (r32["outcome"] == r64["outcome"]) & (r32["pixel"] == r64["pixel"]) & \
           (r32["n_steps"] == r64["n_steps"]) & (r32["rng_blocks"] == r64["rng_blocks"])
    assert same.mean() > 0.995, same.mean()
    for k in ("steps", "virtual", "rayleigh", "compton", "photo", "crossings"):
        assert abs(s32[k] - s64[k]) <= 0.005 * s32[k] + 5, (k, s32[k], s64[k])
