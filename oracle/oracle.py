"""Python side of the CPU oracle.  TEST INFRASTRUCTURE ONLY.

The Monte Carlo and ray-tracing steps live in plain C (gdrr_oracle.c) because
a Python loop over 1e6 photon histories would take hours; this module loads
that library with ctypes and adds the image-domain steps of the paper, written
directly in numpy FP64:

  * Step 3, Section 2.5: Poisson denoising of the scatter signal by the
    relaxation iteration of Eq. 5 (the optimality condition of Eq. 2-4);
  * Step 4, Section 2.6: the noise N = (P^ - P) + (S^ - S) scaled by
    sqrt(n_sim / (zeta I)), and the zeta fit zeta = n_sim / k^2 from the slope
    k of sigma_X / sigma_N^ against 1 / sqrt(I).

Nothing here imports the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, f) for f in ("gdrr_oracle.c", "mc_history.inc", "oracle.h")]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

FIXED_POINT_BITS = 24           # tally unit: 2^-24 keV
N_STATS = 12
STAT_NAMES = ("histories", "steps", "virtual", "rayleigh", "compton", "photo",
              "tally_primary", "tally_scatter", "miss", "cutoff", "step_limit", "crossings")
OUTCOMES = ("primary", "scatter", "photo", "cutoff", "miss", "step_limit")

RECORD_DTYPE = np.dtype([
    ("n_steps", "<u4"), ("n_virtual", "<u4"), ("n_rayleigh", "<u4"), ("n_compton", "<u4"),
    ("n_photo", "<u4"), ("outcome", "<u4"), ("rng_blocks", "<u4"), ("first_interaction", "<u4"),
    ("pixel", "<i4"), ("e_source", "<f4"), ("e_final", "<f4"), ("ray_material", "<u4"),
    ("e_deposited", "<f8")])


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, no FMA contraction, no fast-math)."""
    with _lock:
        newest = max(os.path.getmtime(s) for s in _SRC)
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
        os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-pthread", _SRC[0], "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("sad", ctypes.c_double), ("sdd", ctypes.c_double), ("theta", ctypes.c_double),
        ("nu", ctypes.c_int), ("nv", ctypes.c_int), ("du", ctypes.c_double), ("dv", ctypes.c_double),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("vx", ctypes.c_double), ("vy", ctypes.c_double), ("vz", ctypes.c_double),
        ("material", ctypes.c_void_p), ("density", ctypes.c_void_p),
        ("n_mat", ctypes.c_int), ("n_e", ctypes.c_int), ("e0", ctypes.c_double), ("de", ctypes.c_double),
        ("mu_hat", ctypes.c_void_p),
        ("n_bins", ctypes.c_int), ("bin_e", ctypes.c_void_p), ("bin_w", ctypes.c_void_p),
        ("bin_w_cols", ctypes.c_void_p),
        ("fluence", ctypes.c_void_p),
        ("n_r", ctypes.c_int), ("r0", ctypes.c_double), ("dr", ctypes.c_double),
        ("response", ctypes.c_void_p),
        ("e_cut", ctypes.c_double), ("max_steps", ctypes.c_int),
        ("nearest_voxel", ctypes.c_int), ("scatter_filter", ctypes.c_int),
        ("rayleigh_ff", ctypes.c_int), ("n_ff", ctypes.c_int), ("ff_dx", ctypes.c_double),
        ("ff", ctypes.c_void_p),
        ("local_majorant", ctypes.c_int), ("cell_shift", ctypes.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        L.orc_mc_run.argtypes = [vp, ctypes.c_double, ctypes.c_uint32, u64, u64, u64, i32, i32, vp, vp, vp, vp]
        L.orc_mc_run.restype = i32
        L.orc_rt_primary.argtypes = [vp, ctypes.c_double, vp, i32, vp]
        L.orc_rt_primary.restype = i32
        L.orc_rt_primary_siddon.argtypes = [vp, ctypes.c_double, vp, i32, vp]
        L.orc_rt_primary_siddon.restype = i32
        L.orc_majorant.argtypes = [vp, vp]
        L.orc_majorant.restype = i32
        L.orc_lm_cells.argtypes = [vp, vp]
        L.orc_lm_cells.restype = i32
        L.orc_lm_walk.argtypes = [vp, i32, vp, vp, ctypes.c_double, ctypes.c_double, vp]
        L.orc_lm_walk.restype = i32
        L.orc_logf.argtypes = [ctypes.c_float]
        L.orc_logf.restype = ctypes.c_float
        L.orc_logf_many.argtypes = [vp, vp, i32]
        L.orc_philox_many.argtypes = [vp, vp, vp, i32]
        L.orc_stream_words.argtypes = [u64, ctypes.c_uint32, u64, i32, vp]
        L.orc_sample_compton.argtypes = [ctypes.c_float, u64, i32, vp, vp]
        L.orc_sample_rayleigh.argtypes = [u64, i32, vp]
        L.orc_sample_rayleigh_ff.argtypes = [vp, ctypes.c_float, i32, u64, i32, vp]
        L.orc_sample_rayleigh_ff.restype = i32
        L.orc_sample_azimuth.argtypes = [u64, i32, vp, vp]
        L.orc_rotate.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, vp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class _Marshalled:
    """Keeps the contiguous arrays alive while C reads them."""

    def __init__(self, prob, e_cut=1.0, max_steps=100000, nearest_voxel=0, scatter_filter=0, rayleigh_ff=0,
                 local_majorant=0, cell_shift=0):
        self.material = np.ascontiguousarray(prob.material, np.uint8)
        self.density = np.ascontiguousarray(prob.density, np.float32)
        self.mu_hat = np.ascontiguousarray(prob.mu_hat, np.float32)
        self.spec_e = np.ascontiguousarray(prob.spec_e, np.float64)
        self.spec_w = np.ascontiguousarray(prob.spec_w, np.float64)
        self.fluence = np.ascontiguousarray(prob.fluence, np.float64)
        self.response = np.ascontiguousarray(prob.response, np.float32)
        cols = getattr(prob, "spec_cols", None)
        self.spec_cols = None if cols is None else np.ascontiguousarray(cols, np.float64)
        nz, ny, nx = self.material.shape
        s = _Problem()
        s.sad, s.sdd, s.theta = prob.sad, prob.sdd, prob.theta
        s.nu, s.nv, s.du, s.dv = prob.nu, prob.nv, prob.du, prob.dv
        s.nx, s.ny, s.nz = nx, ny, nz
        s.vx, s.vy, s.vz = prob.voxel
        s.material, s.density = _ptr(self.material).value, _ptr(self.density).value
        s.n_mat, s.n_e = self.mu_hat.shape[0], self.mu_hat.shape[2]
        s.e0, s.de = prob.e0, prob.de
        s.mu_hat = _ptr(self.mu_hat).value
        s.n_bins = self.spec_e.size
        s.bin_e, s.bin_w = _ptr(self.spec_e).value, _ptr(self.spec_w).value
        s.bin_w_cols = None if self.spec_cols is None else _ptr(self.spec_cols).value
        s.fluence = _ptr(self.fluence).value
        s.n_r, s.r0, s.dr = self.response.size, prob.r0, prob.dr
        s.response = _ptr(self.response).value
        s.e_cut, s.max_steps = e_cut, max_steps
        s.nearest_voxel, s.scatter_filter = int(nearest_voxel), int(scatter_filter)
        s.rayleigh_ff = int(rayleigh_ff)
        s.local_majorant, s.cell_shift = int(local_majorant), int(cell_shift)
        ff = getattr(prob, "form_factor", None)
        if rayleigh_ff and ff is None:
            raise ValueError("rayleigh_ff needs the problem's form_factor table")
        if ff is not None:
            self.ff = np.ascontiguousarray(ff, np.float32)
            s.n_ff, s.ff_dx, s.ff = self.ff.shape[1], float(prob.ff_dx), _ptr(self.ff).value
        self.struct = s


def mc_run(prob, n_histories, seed=1, phi=0.0, angle_index=0, history_offset=0, precision=32,
           threads=1, records=False, e_cut=1.0, max_steps=100000, nearest_voxel=False, scatter_filter=0,
           rayleigh_ff=False, local_majorant=False, cell_shift=1):
    """Monte Carlo projection (Section 2.4).  Returns (tally_p, tally_s, stats, records)
    with int64 fixed-point tallies shaped [nv, nu].  nearest_voxel: no density
    interpolation (the paper's speed variant); scatter_filter: 0 all scatter,
    1 single Compton, 2 single Rayleigh, 3 multiple scatter; rayleigh_ff: the
    Rayleigh angle takes the problem's form factors (else Thomson);
    local_majorant: delta tracking with one majorant per macro cell of
    2^cell_shift voxels per edge instead of the global one."""
    m = _Marshalled(prob, e_cut, max_steps, nearest_voxel, scatter_filter, rayleigh_ff, local_majorant,
                    cell_shift)
    tp = np.zeros((prob.nv, prob.nu), np.int64)
    ts = np.zeros((prob.nv, prob.nu), np.int64)
    st = np.zeros(N_STATS, np.uint64)
    rec = np.zeros(n_histories, RECORD_DTYPE) if records else None
    rc = lib().orc_mc_run(ctypes.byref(m.struct), phi, angle_index, n_histories, seed, history_offset,
                          precision, threads, _ptr(tp), _ptr(ts), _ptr(st),
                          _ptr(rec) if records else None)
    if rc:
        raise ValueError(f"oracle mc_run rejected the problem (rc={rc})")
    return tp, ts, dict(zip(STAT_NAMES, (int(x) for x in st))), rec


def lm_cells(prob, cell_shift):
    """The local-majorant cell table: [ncz, ncy, ncx, n_mat] largest densities."""
    m = _Marshalled(prob, cell_shift=cell_shift)
    nz, ny, nx = m.material.shape
    nc = [((n - 1) >> cell_shift) + 1 for n in (nz, ny, nx)]
    out = np.zeros(nc + [m.mu_hat.shape[0]], np.float32)
    if lib().orc_lm_cells(ctypes.byref(m.struct), _ptr(out)):
        raise ValueError("oracle lm_cells rejected the problem")
    return out


def lm_walk(prob, cell_shift, pos, direction, e, tau, precision=64):
    """One local-majorant free flight: (hit, position, bound, crossings)."""
    m = _Marshalled(prob, cell_shift=cell_shift)
    p = np.ascontiguousarray(pos, np.float64)
    d = np.ascontiguousarray(direction, np.float64)
    out = np.zeros(5)
    rc = lib().orc_lm_walk(ctypes.byref(m.struct), precision, _ptr(p), _ptr(d), float(e), float(tau), _ptr(out))
    if rc < 0:
        raise ValueError("oracle lm_walk rejected the problem")
    return bool(rc), out[:3].copy(), float(out[3]), int(out[4])


def rt_primary(prob, phi=0.0, pixels=None):
    """Ray-traced primary (Section 2.3, Eq. 1) in FP64; per source photon."""
    m = _Marshalled(prob)
    if pixels is None:
        out = np.zeros(prob.nv * prob.nu)
        rc = lib().orc_rt_primary(ctypes.byref(m.struct), phi, None, 0, _ptr(out))
        out = out.reshape(prob.nv, prob.nu)
    else:
        px = np.ascontiguousarray(pixels, np.int32)
        out = np.zeros(px.size)
        rc = lib().orc_rt_primary(ctypes.byref(m.struct), phi, _ptr(px), px.size, _ptr(out))
    if rc:
        raise ValueError(f"oracle rt_primary rejected the problem (rc={rc})")
    return out


def rt_primary_siddon(prob, phi=0.0, pixels=None):
    """Siddon ray-traced primary (exact voxel path lengths), FP64; per source photon."""
    m = _Marshalled(prob)
    if pixels is None:
        out = np.zeros(prob.nv * prob.nu)
        rc = lib().orc_rt_primary_siddon(ctypes.byref(m.struct), phi, None, 0, _ptr(out))
        out = out.reshape(prob.nv, prob.nu)
    else:
        px = np.ascontiguousarray(pixels, np.int32)
        out = np.zeros(px.size)
        rc = lib().orc_rt_primary_siddon(ctypes.byref(m.struct), phi, _ptr(px), px.size, _ptr(out))
    if rc:
        raise ValueError(f"oracle rt_primary_siddon rejected the problem (rc={rc})")
    return out


def majorant(prob):
    m = _Marshalled(prob)
    out = np.zeros(m.mu_hat.shape[2], np.float32)
    if lib().orc_majorant(ctypes.byref(m.struct), _ptr(out)):
        raise ValueError("bad problem")
    return out


def logf(x):
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty_like(x)
    lib().orc_logf_many(_ptr(x), _ptr(out), x.size)
    return out


def philox(ctr, key):
    """Philox4x32-10 of counters [n,4] under keys [n,2] -> [n,4] uint32."""
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, np.uint32).reshape(-1, 2), (ctr.shape[0], 2)))
    out = np.empty_like(ctr)
    lib().orc_philox_many(_ptr(ctr), _ptr(key), _ptr(out), ctr.shape[0])
    return out


def stream_words(seed, angle_index, hid, n_blocks):
    out = np.empty(4 * n_blocks, np.uint32)
    lib().orc_stream_words(seed, angle_index, hid, n_blocks, _ptr(out))
    return out


def sample_compton(e_kev, n, seed=1):
    c = np.empty(n, np.float32)
    e = np.empty(n, np.float32)
    lib().orc_sample_compton(e_kev, seed, n, _ptr(c), _ptr(e))
    return c, e


def sample_rayleigh(n, seed=1):
    c = np.empty(n, np.float32)
    lib().orc_sample_rayleigh(seed, n, _ptr(c))
    return c


def sample_rayleigh_ff(prob, e_kev, material, n, seed=1):
    """Rayleigh cos(theta) with the form factor of `material` at e_kev (FP32 path)."""
    m = _Marshalled(prob, rayleigh_ff=1)
    c = np.empty(n, np.float32)
    rc = lib().orc_sample_rayleigh_ff(ctypes.byref(m.struct), e_kev, material, seed, n, _ptr(c))
    if rc:
        raise ValueError("oracle rejected the form-factor problem")
    return c


def sample_azimuth(n, seed=1):
    c = np.empty(n, np.float32)
    s = np.empty(n, np.float32)
    lib().orc_sample_azimuth(seed, n, _ptr(c), _ptr(s))
    return c, s


def rotate(d, ct, cp, sp):
    d = np.ascontiguousarray(d, np.float32)
    out = np.empty(3, np.float32)
    lib().orc_rotate(_ptr(d), ct, cp, sp, _ptr(out))
    return out


# --------------------------------------------------------------------------
# Image-domain steps, FP64 numpy.

def finalize(tally, n_photons):
    """Fixed-point tally -> signal per source photon (Section 2.6: MC results
    are normalised by the number of source photons)."""
    return np.asarray(tally, np.float64) * 2.0**-FIXED_POINT_BITS / float(n_photons)


def bin_tally(tally, f):
    """Exact integer f x f binning of a [nv, nu] tally (coarse scatter grid)."""
    nv, nu = tally.shape
    return tally.reshape(nv // f, f, nu // f, f).sum(axis=(1, 3))


def upsample(coarse, f):
    """Bilinear interpolation of a coarse f x f-binned image back to the fine
    grid, divided by f^2 (a binned sum -> a per-fine-pixel value); coarse
    pixel centres sit at fine coordinate (I + 1/2) f - 1/2, edges clamp."""
    cv, cu = coarse.shape
    def axis(n_fine, n_coarse):
        x = (np.arange(n_fine) + 0.5) / f - 0.5
        i0 = np.floor(x).astype(np.int64)
        t = x - i0
        return np.clip(i0, 0, n_coarse - 1), np.clip(i0 + 1, 0, n_coarse - 1), t
    v0, v1, tv = axis(cv * f, cv)
    u0, u1, tu = axis(cu * f, cu)
    c = np.asarray(coarse, np.float64)
    top = c[v0][:, u0] * (1 - tu) + c[v0][:, u1] * tu
    bot = c[v1][:, u0] * (1 - tu) + c[v1][:, u1] * tu
    return (top * (1 - tv)[:, None] + bot * tv[:, None]) / (f * f)


def denoise(s_hat, beta, omega=0.8, iters=500, eps=1e-3, s0=None):
    """Step 3, Section 2.5: minimise  sum (S - S^ log S) + beta/2 |grad S|^2
    (Eq. 2) by iterating Eq. 5,

        S <- (1 - omega) S + omega/4 [ Sigma S - (1/beta)(1 - S^/S) ],

    with Sigma S = S(i+1,j) + S(i,j+1) + S(i-1,j) + S(i,j-1), starting from
    S^(0) = S^ (Section 2.5).  Every right-hand side uses the previous iterate
    (the paper's superscript k throughout).  Readings where the paper is
    silent: replicate (zero-flux) edges, S kept >= eps so that S^/S and log S
    stay defined.  Input is on the count scale (Poisson fidelity).  Array
    index [j, i]: i runs along u (fast axis), j along v."""
    s_hat = np.asarray(s_hat, np.float64)
    s = np.maximum(s_hat if s0 is None else np.asarray(s0, np.float64), eps)
    for _ in range(iters):
        p = np.pad(s, 1, mode="edge")
        sigma = ((p[1:-1, 2:] + p[2:, 1:-1]) + p[1:-1, :-2]) + p[:-2, 1:-1]
        s = (1.0 - omega) * s + (omega / 4.0) * (sigma - (1.0 / beta) * (1.0 - s_hat / s))
        s = np.maximum(s, eps)
    return s


def count_scale(scat_tally, n_photons, n_scat):
    """The count scale of Step 3 (Section 2.5 needs counts for the Poisson
    fidelity of Eq. 2; reading: the mean signal one detected scattered
    photon leaves): the scatter image per source photon, summed, over the
    number of scattered photons tallied.  With none tallied the scale is one
    photon's share, 1 / n_photons."""
    total = float(np.sum(finalize(scat_tally, n_photons)))
    scale = total / max(1, int(n_scat))
    return scale if scale > 0 else 1.0 / n_photons


def mean_coarse_count(n_scat, n_coarse):
    """Scattered photons tallied per coarse pixel (at least one photon in all)."""
    return max(1, int(n_scat)) / n_coarse


def smoothing_beta(smoothing_px, n_scat, n_coarse):
    """beta of Eq. 2 for a smoothing length in coarse pixels: the Laplacian term
    of Eq. 4 balances the fidelity term over a length L where beta S ~ L^2,
    so beta = L^2 / (mean count per coarse pixel)."""
    return smoothing_px * smoothing_px / max(mean_coarse_count(n_scat, n_coarse), 1e-6)


def project_chain(P, prim_tally, scat_tally, n_photons, n_scat, bin_factor=4, beta=0.02, smoothing_px=None,
                  omega=0.8, iters=300, mas=0.4, zeta=5.2913e9):
    """Steps 2-4 of Section 2.2 after the transport, in the paper's order, from
    the int64 tallies and the ray-traced primary P: signals per source photon
    (Section 2.6), the coarse scatter grid, Eq. 5 on the count scale, bilinear
    upsampling, and the scaled noise N."""
    P_hat = finalize(prim_tally, n_photons)
    S_hat = finalize(scat_tally, n_photons)
    S_hat_c = finalize(bin_tally(scat_tally, bin_factor), n_photons)
    cs = count_scale(scat_tally, n_photons, n_scat)
    if smoothing_px is not None and smoothing_px > 0:
        beta = smoothing_beta(smoothing_px, n_scat, S_hat_c.size)
    S_c = denoise(S_hat_c / cs, beta, omega, iters) * cs
    S = upsample(S_c, bin_factor)
    N = noise_scale(P_hat, P, S_hat, S, n_photons, mas, zeta)
    return dict(P_hat=P_hat, S_hat=S_hat, S_hat_coarse=S_hat_c, S_coarse=S_c, S=S, N=N, count_scale=cs, beta=beta)


def optimality_residual(s, s_hat, beta):
    """Eq. 4: (1 - S^/S) - beta (Sigma S - 4 S), per pixel, replicate edges."""
    p = np.pad(s, 1, mode="edge")
    sigma = ((p[1:-1, 2:] + p[2:, 1:-1]) + p[1:-1, :-2]) + p[:-2, 1:-1]
    return (1.0 - s_hat / s) - beta * (sigma - 4.0 * s)


def energy(s, s_hat, beta):
    """Discrete Eq. 2: sum (S - S^ log S) + beta/2 sum |grad S|^2 (forward differences)."""
    gx = np.diff(s, axis=1)
    gy = np.diff(s, axis=0)
    return float(np.sum(s - s_hat * np.log(s)) + 0.5 * beta * (np.sum(gx**2) + np.sum(gy**2)))


def noise_scale(p_hat, p, s_hat, s, n_sim, mas, zeta):
    """Step 4, Section 2.6: N = alpha ((P^ - P) + (S^ - S)), alpha = sqrt(n_sim / (zeta I))."""
    n_hat = (np.asarray(p_hat, np.float64) - p) + (np.asarray(s_hat, np.float64) - s)
    return n_hat * np.sqrt(float(n_sim) / (zeta * mas))


def fit_zeta(inv_sqrt_mas, ratio, n_sim):
    """Section 2.6: sigma_X/sigma_N^ = k / sqrt(I) (a line through the origin,
    Eq. 6), least-squares slope k, zeta = n_sim / k^2.  Returns (zeta, k)."""
    x = np.asarray(inv_sqrt_mas, np.float64)
    y = np.asarray(ratio, np.float64)
    k = float(np.dot(x, y) / np.dot(x, x))
    return float(n_sim) / (k * k), k
