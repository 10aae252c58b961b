"""CPU oracle of the cone-beam reconstruction used to view simulated scans.
TEST INFRASTRUCTURE ONLY.

Section 3.5 reconstructs CBCT images from simulated projections with "an FDK
algorithm" (Feldkamp, Davis and Kress, JOSA A 1984) and no further detail.
This module writes out the textbook form (Kak and Slaney, Principles of
Computerized Tomographic Imaging, Ch. 3, equally spaced fan beam, extended
to the cone by Feldkamp's weighting) in numpy FP64, for the circular orbit of
Section 2.1 with the imager opposite the source:

  1. line integrals g = -ln(I / I0), I0 the air scan (no object);
  2. virtual detector at the isocentre: a = u SAD / SDD, b = v SAD / SDD,
     sample spacing tau = du SAD / SDD;
  3. cosine weighting Q = g SAD / sqrt(SAD^2 + a^2 + b^2);
  4. ramp filtering of each detector row with the Ram-Lak kernel
     h(0) = 1 / (4 tau^2), h(n even) = 0, h(n odd) = -1 / (n pi tau)^2,
     as the linear convolution Qf(n) = tau sum_k h(n - k) Q(k) / 2 (the 1/2
     of the full-scan fan-beam formula), zero outside the row;
  5. voxel-driven backprojection f(x) = sum_beta dbeta Qf(a(x), b(x)) / U^2,
     U = (SAD + x.n) / SAD, a(x) = SAD (x.e_u) / (SAD + x.n),
     b(x) = SAD z / (SAD + x.n), n the unit vector from the source through
     the isocentre, e_u the detector's u axis, bilinear interpolation of Qf
     on the pixel-centre grid, zero outside the detector.

Nothing here imports the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np


def line_integrals(signal, air, floor=1e-6):
    """g = -ln(I / I0), with I clamped below at floor * I0."""
    s = np.asarray(signal, np.float64)
    a = np.asarray(air, np.float64)
    return -np.log(np.maximum(s, floor * a) / a)


def ramp_kernel(n_taps, tau):
    """Ram-Lak kernel h(k tau) for k = -(n_taps-1) .. n_taps-1 (Kak & Slaney)."""
    k = np.arange(-(n_taps - 1), n_taps)
    h = np.zeros(k.size)
    h[k == 0] = 1.0 / (4.0 * tau * tau)
    odd = (k % 2) != 0
    h[odd] = -1.0 / (np.pi * k[odd] * tau) ** 2
    return h


def fdk_filter(proj, sad, sdd, du, dv):
    """Cosine-weighted, ramp-filtered projections [n_proj, nv, nu] (FP64)."""
    p = np.asarray(proj, np.float64)
    n_proj, nv, nu = p.shape
    mag = sad / sdd
    a = (np.arange(nu) + 0.5 - 0.5 * nu) * du * mag
    b = (np.arange(nv) + 0.5 - 0.5 * nv) * dv * mag
    w = sad / np.sqrt(sad * sad + a[None, :] ** 2 + b[:, None] ** 2)
    tau = du * mag
    h = ramp_kernel(nu, tau)
    out = np.empty_like(p)
    for i in range(n_proj):
        q = p[i] * w
        for r in range(nv):
            full = np.convolve(q[r], h)             # length 3 nu - 2, index k + (nu - 1) is output k
            out[i, r] = 0.5 * tau * full[nu - 1:2 * nu - 1]
    return out


def fdk_backproject(filtered, angles, d_beta, sad, sdd, du, dv, shape, voxel):
    """Voxel-driven FDK backprojection onto a grid [nz, ny, nx] of voxel size
    (dx, dy, dz) mm centred on the isocentre.  Returns mu in 1/mm (FP64)."""
    q = np.asarray(filtered, np.float64)
    n_proj, nv, nu = q.shape
    nz, ny, nx = shape
    dx, dy, dz = voxel
    mag = sad / sdd
    tau_u, tau_v = du * mag, dv * mag
    x = (np.arange(nx) + 0.5 - 0.5 * nx) * dx
    y = (np.arange(ny) + 0.5 - 0.5 * ny) * dy
    z = (np.arange(nz) + 0.5 - 0.5 * nz) * dz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = np.zeros(shape)
    for i in range(n_proj):
        phi = float(angles[i])
        n0, n1 = math.cos(phi), math.sin(phi)          # source -> isocentre
        e0, e1 = math.sin(phi), -math.cos(phi)         # detector u axis
        depth = sad + X * n0 + Y * n1
        a = sad * (X * e0 + Y * e1) / depth
        b = sad * Z / depth
        fu = a / tau_u + 0.5 * nu - 0.5
        fv = b / tau_v + 0.5 * nv - 0.5
        iu = np.floor(fu).astype(np.int64)
        iv = np.floor(fv).astype(np.int64)
        wu = fu - iu
        wv = fv - iv
        val = np.zeros(shape)
        for cu, cv, w in ((0, 0, (1 - wu) * (1 - wv)), (1, 0, wu * (1 - wv)),
                          (0, 1, (1 - wu) * wv), (1, 1, wu * wv)):
            ju, jv = iu + cu, iv + cv
            ok = (ju >= 0) & (ju < nu) & (jv >= 0) & (jv < nv)
            samp = np.zeros(shape)
            samp[ok] = q[i, jv[ok], ju[ok]]
            val += w * samp
        U = depth / sad
        f += d_beta * val / (U * U)
    return f


def fdk(proj, angles, sad, sdd, du, dv, shape, voxel, d_beta=None):
    """Full FDK of line-integral projections [n_proj, nv, nu] over a full scan."""
    n_proj = len(angles)
    if d_beta is None:
        d_beta = 2.0 * math.pi / n_proj
    return fdk_backproject(fdk_filter(proj, sad, sdd, du, dv), angles, d_beta, sad, sdd, du, dv, shape, voxel)
