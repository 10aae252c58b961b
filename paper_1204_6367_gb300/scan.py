"""Synthetic CBCT scans and their reconstruction (Section 3.5).

Section 3.5 simulates a full orbit of projections and reconstructs them with
FDK to show what realistic projections carry into the image: beam hardening
from a poly-energetic source, scatter artifacts, and noise whose amplitude
follows the mAs level (Fig. 9, Fig. 10).  A scan here is the gDRR pipeline
(Steps 1-4 of Section 2.2) at equally spaced gantry angles over 2 pi, with a
choice of components:

  "P"    the ray-traced primary (Step 1);
  "PS"   primary plus the denoised Monte Carlo scatter (Steps 1-3);
  "PSN"  primary, scatter and the noise scaled to the mAs level (Steps 1-4).

Each view draws its own random streams (angle index = view index).  The
reconstruction takes line integrals against the air scan and runs the FDK
filter and backprojection kernels.  Every step runs in libgdrr kernels; this
module only sequences the calls.
"""
from __future__ import annotations

import math

from . import gdrr


def full_orbit(n_views: int):
    import numpy as np
    return np.arange(n_views) * (2.0 * math.pi / n_views)


def scan(ctx, n_views: int, components: str = "P", n_photons: int = 1_000_000, seed: int = 1,
         mas: float = 0.4, zeta: float = 5.2913e9, bin_factor: int = 4, beta: float = 0.02, iters: int = 300,
         smoothing_px: float | None = None):
    """Signals [n_views, nv, nu] FP64 (per source photon) of a full orbit.

    beta / smoothing_px set the scatter denoiser of each view as in
    gdrr.project (smoothing_px: beta from the view's mean scatter count)."""
    import torch
    if components not in ("P", "PS", "PSN"):
        raise ValueError("components must be 'P', 'PS' or 'PSN'")
    if ctx.prob.theta != 0.0:
        raise ValueError("the reconstruction geometry needs the imager opposite the source (theta = 0)")
    angles = full_orbit(n_views)
    sig = torch.empty((n_views, ctx.nv, ctx.nu), dtype=torch.float64, device="cuda")
    for i, a in enumerate(angles):
        if components == "P":
            gdrr.gdrr_raytrace_primary(ctx, float(a), out=sig[i])
            continue
        r = gdrr.project(ctx, n_photons, seed, float(a), bin_factor=bin_factor, beta=beta, iters=iters, mas=mas,
                         zeta=zeta, angle_index=i, smoothing_px=smoothing_px)
        s = r["P"] + r["S"]
        if components == "PSN":
            s = s + r["N"]
        sig[i].copy_(s)
    return angles, sig


def reconstruct(ctx, angles, signal, shape, voxel, floor_rel: float = 1e-6):
    """FDK volume [nz, ny, nx] FP32 (attenuation, 1/mm) of a scan's signals."""
    I0 = gdrr.gdrr_air_scan(ctx)
    g = gdrr.gdrr_line_integrals(signal, I0.expand_as(signal).contiguous(), floor_rel)
    p = ctx.prob
    geo = gdrr.fdk_geometry(p.sad, p.sdd, ctx.nu, ctx.nv, p.du, p.dv, shape, voxel)
    return gdrr.fdk(geo, g, angles)
