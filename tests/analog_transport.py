"""An independent analog photon transport for a phantom that varies along x
only (layers of voxels), for testing the oracle by brute force.

It shares nothing with the oracle's transport but the problem's tables.  The
method's trilinear field of such a phantom is linear in x between voxel
centres and constant beyond the outer centres (clamp to edge), so the
optical depth along a ray is a piecewise-quadratic function of x: free paths
are drawn by inverting it exactly for an exponential optical depth (no
Woodcock tracking).  Klein-Nishina angles come by rejection from the uniform
law of cos theta, Thomson angles by inverting their cumulative (Cardano's
formula), azimuths as uniform angles, new directions from an explicit
orthonormal frame, random numbers from numpy's generator.  Photons are
transported in vectorised rounds: each round moves every live photon to its
next interaction or out of the box.
"""
import math

import numpy as np

MEC2 = 510.99895


class _Layers:
    """Coefficients of a phantom whose voxels vary along x only."""

    def __init__(self, prob):
        mat, den = prob.material, prob.density
        if not ((mat == mat[:1, :1, :]).all() and (den == den[:1, :1, :]).all()):
            raise ValueError("the analog transport needs a phantom that varies along x only")
        nx = mat.shape[2]
        vox = float(prob.voxel[0])
        self.half = 0.5 * nx * vox
        self.m = mat[0, 0, :].astype(np.int64)
        self.rho = den[0, 0, :].astype(np.float64)
        centres = (np.arange(nx) + 0.5) * vox - self.half
        self.knots = np.concatenate([[-self.half], centres, [self.half]])
        self.tab = prob.mu_hat.astype(np.float64) * 0.1           # 1/mm per g/cm^3, [m, k, e]
        self.e0, self.de = prob.e0, prob.de

    def knot_mu(self, e):
        """mu_k at the knots for energies e: [N, knots, 3] (linear in E between
        the table's nodes; the end knots repeat the outer centres)."""
        x = (e - self.e0) / self.de
        i = np.clip(np.floor(x).astype(np.int64), 0, self.tab.shape[2] - 2)
        f = (x - i)[:, None, None]
        t = self.tab[:, :, i] + f.transpose(1, 2, 0) * (self.tab[:, :, i + 1] - self.tab[:, :, i])   # [M, 3, N]
        cen = self.rho[None, :, None] * t[self.m].transpose(2, 0, 1)                           # [N, nx, 3]
        return np.concatenate([cen[:, :1], cen, cen[:, -1:]], axis=1)

    def coeffs(self, x, e):
        """mu_R, mu_C, mu_P at positions x (the x coordinate) for energies e."""
        mu = self.knot_mu(e)
        j = np.clip(np.searchsorted(self.knots, x, side="right") - 1, 0, len(self.knots) - 2)
        f = np.clip((x - self.knots[j]) / (self.knots[j + 1] - self.knots[j]), 0.0, 1.0)
        r = np.arange(len(x))
        v = mu[r, j] + f[:, None] * (mu[r, j + 1] - mu[r, j])
        return v[:, 0], v[:, 1], v[:, 2]

    def free_path(self, x0, dx, e, tau):
        """Distance along rays (x coordinate x0, direction cosine dx) at which
        the optical depth of mu_T reaches tau; inf when it is not reached
        before the last knot."""
        mu = self.knot_mu(e).sum(axis=2)                                        # [N, K]
        K = self.knots
        h = np.diff(K)
        seg = 0.5 * (mu[:, 1:] + mu[:, :-1]) * h[None, :]
        C = np.concatenate([np.zeros((len(x0), 1)), np.cumsum(seg, axis=1)], axis=1)

        def F(x):                                                               # integral of mu_T from -half
            j = np.clip(np.searchsorted(K, x, side="right") - 1, 0, len(K) - 2)
            r = np.arange(len(x))
            slope = (mu[r, j + 1] - mu[r, j]) / h[j]
            dxk = x - K[j]
            return C[r, j] + dxk * mu[r, j] + 0.5 * slope * dxk * dxk

        s = np.full(len(x0), np.inf)
        flat = np.abs(dx) < 1e-12
        if flat.any():                                                          # parallel to the layers
            mT = sum(self.coeffs(x0[flat], e[flat]))
            s[flat] = tau[flat] / mT
        ok = ~flat
        if ok.any():
            r = np.nonzero(ok)[0]
            T = F(x0[r]) + np.sign(dx[r]) * tau[r] * np.abs(dx[r])
            inside = (T >= 0.0) & (T <= C[r, -1])
            r, T = r[inside], T[inside]
            j = np.clip((C[r] <= T[:, None]).sum(axis=1) - 1, 0, len(K) - 2)
            m0 = mu[r, j]
            slope = (mu[r, j + 1] - m0) / h[j]
            q = T - C[r, j]
            delta = 2.0 * q / (m0 + np.sqrt(np.maximum(m0 * m0 + 2.0 * slope * q, 0.0)))
            s[r] = (K[j] + delta - x0[r]) / dx[r]
        return s


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
    med = _Layers(prob)
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
        s = med.free_path(xl[:, 0], dl[:, 0], el, -np.log(1.0 - rng.random(live.size)))
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
        muR, muC, muP = med.coeffs(x[idx, 0], e[idx])
        u = rng.random(idx.size) * (muR + muC + muP)
        ray = u < muR
        comp = ~ray & (u < muR + muC)
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
