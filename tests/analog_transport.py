"""An independent analog photon transport for a homogeneous cube, for
testing the oracle by brute force.

It shares nothing with the oracle's transport but the problem's tables: free
paths are drawn from the exponential law of the local total coefficient (no
Woodcock tracking), Klein-Nishina angles by rejection from the uniform law of
cos theta, Thomson angles by inverting their cumulative (Cardano's formula),
azimuths as uniform angles, and new directions from an explicit orthonormal
frame.  Random numbers come from numpy's generator.  Photons are transported
in vectorised rounds: each round moves every live photon to its next
interaction or out of the cube.
"""
import math

import numpy as np

MEC2 = 510.99895


def _coeffs(prob, e):
    """mu_R, mu_C, mu_P in 1/mm of the cube's material at energies e (linear
    between the table's 1 keV nodes)."""
    m = int(prob.material.flat[0])
    rho = float(prob.density.flat[0])
    tab = prob.mu_hat[m].astype(np.float64)
    x = (e - prob.e0) / prob.de
    i = np.clip(np.floor(x).astype(int), 0, tab.shape[1] - 2)
    f = x - i
    return [(tab[k, i] + f * (tab[k, i + 1] - tab[k, i])) * 0.1 * rho for k in range(3)]


def _frame_rotate(d, ct, phi):
    """Directions at polar angle acos(ct) and azimuth phi about unit vectors d."""
    k = np.zeros_like(d)
    k[np.arange(len(d)), np.argmin(np.abs(d), axis=1)] = 1.0      # the axis least aligned with d
    a = np.cross(d, k)
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = np.cross(d, a)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    out = ct[:, None] * d + (st * np.cos(phi))[:, None] * a + (st * np.sin(phi))[:, None] * b
    return out / np.linalg.norm(out, axis=1, keepdims=True)


def _thomson(rng, n):
    """cos theta with density (3/8)(1 + mu^2) on [-1, 1]: the real root of
    mu^3 + 3 mu + 4 - 8 u = 0."""
    q = 4.0 - 8.0 * rng.random(n)
    disc = np.sqrt(q * q / 4.0 + 1.0)
    return np.cbrt(-q / 2.0 + disc) + np.cbrt(-q / 2.0 - disc)


def _klein_nishina(rng, e):
    """cos theta from Klein-Nishina at energies e, by rejection from the
    uniform law (the law's maximum, at cos theta = 1, is 1 in these units)."""
    mu = np.empty_like(e)
    todo = np.arange(len(e))
    while todo.size:
        m = 2.0 * rng.random(todo.size) - 1.0
        r = 1.0 / (1.0 + (e[todo] / MEC2) * (1.0 - m))
        w = 0.5 * r * r * (r + 1.0 / r - (1.0 - m * m))
        ok = rng.random(todo.size) < w
        mu[todo[ok]] = m[ok]
        todo = todo[~ok]
    return mu


def transport(prob, n, seed, half):
    """Primary and scatter images (keV per source photon) of a pencil beam
    (the fluence map's one lit pixel) through a homogeneous cube
    [-half, half]^3, imager at angle 0 (source on -x, imager plane x = sdd -
    sad, u along -y, v along z), ideal response r(E) = E."""
    rng = np.random.default_rng(seed)
    sad, sdd, nu, nv, du, dv = prob.sad, prob.sdd, prob.nu, prob.nv, prob.du, prob.dv
    jv, ju = np.unravel_index(int(np.argmax(prob.fluence)), prob.fluence.shape)
    E0 = float(prob.spec_e[0])
    xd = sdd - sad
    # source rays to uniform points in the lit pixel
    au = ((ju + rng.random(n)) - 0.5 * nu) * du
    av = ((jv + rng.random(n)) - 0.5 * nv) * dv
    S = np.array([-sad, 0.0, 0.0])
    tgt = np.stack([np.full(n, xd), -au, av], axis=1)
    d = tgt - S
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    # entry into the cube (the pencil always hits it)
    with np.errstate(divide="ignore"):
        t1 = (-half - S) / d
        t2 = (half - S) / d
    t_in = np.max(np.minimum(t1, t2), axis=1)
    x = S + t_in[:, None] * d
    e = np.full(n, E0)
    scattered = np.zeros(n, bool)
    prim = np.zeros((nv, nu))
    scat = np.zeros((nv, nu))
    live = np.arange(n)
    while live.size:
        xl, dl, el = x[live], d[live], e[live]
        muR, muC, muP = _coeffs(prob, el)
        muT = muR + muC + muP
        s = -np.log(1.0 - rng.random(live.size)) / muT
        with np.errstate(divide="ignore", invalid="ignore"):
            te = np.where(dl > 0, (half - xl) / dl, np.where(dl < 0, (-half - xl) / dl, np.inf))
        d_exit = np.maximum(te.min(axis=1), 0.0)
        out = s >= d_exit
        # leaving photons: straight to the imager plane
        if out.any():
            idx = live[out]
            xo = xl[out] + d_exit[out, None] * dl[out]
            do = dl[out]
            ok = do[:, 0] > 0
            t = np.where(ok, (xd - xo[:, 0]) / np.where(ok, do[:, 0], 1.0), -1.0)
            ok &= t >= 0
            pu = -(xo[:, 1] + t * do[:, 1])
            pv = xo[:, 2] + t * do[:, 2]
            iu = np.floor(pu / du + 0.5 * nu).astype(np.int64)
            iv = np.floor(pv / dv + 0.5 * nv).astype(np.int64)
            ok &= (iu >= 0) & (iu < nu) & (iv >= 0) & (iv < nv)
            for img, sel in ((prim, ok & ~scattered[idx]), (scat, ok & scattered[idx])):
                np.add.at(img, (iv[sel], iu[sel]), e[idx[sel]])
        # interacting photons
        stay = ~out
        idx = live[stay]
        x[idx] = xl[stay] + s[stay, None] * dl[stay]
        u = rng.random(idx.size) * muT[stay]
        ray = u < muR[stay]
        comp = ~ray & (u < muR[stay] + muC[stay])
        # photoelectric: absorbed
        r_idx = idx[ray]
        if r_idx.size:
            d[r_idx] = _frame_rotate(d[r_idx], _thomson(rng, r_idx.size), 2.0 * math.pi * rng.random(r_idx.size))
            scattered[r_idx] = True
        c_idx = idx[comp]
        if c_idx.size:
            ct = _klein_nishina(rng, e[c_idx])
            e[c_idx] = e[c_idx] / (1.0 + (e[c_idx] / MEC2) * (1.0 - ct))
            d[c_idx] = _frame_rotate(d[c_idx], ct, 2.0 * math.pi * rng.random(c_idx.size))
            scattered[c_idx] = True
        live = np.concatenate([r_idx, c_idx])
        live = live[e[live] >= 1.0]
    return prim / n, scat / n
