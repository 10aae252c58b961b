"""Python binding of libgdrr (include/gdrr.h): argument marshalling only.

Every step of the projection runs in the library's CUDA kernels; this module
turns torch tensors into device pointers and CUDA streams into handles, and
raises GdrrError on a non-zero return code.  It never falls back to another
implementation: if libgdrr.so is missing or cannot load, the first call
raises.  Function names are those of the C ABI.
"""
from __future__ import annotations

import ctypes
import math
import os
import warnings

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgdrr.so")

GDRR_NSTATS = 13
# the method's event counters; slot 11 (cell_skips) is the kernel's own count
# of virtual collisions the macro-cell bound decided without corner gathers,
# slot 12 the cell crossings of flights with local majorants
STAT_NAMES = ("histories", "steps", "virtual", "rayleigh", "compton", "photo",
              "tally_primary", "tally_scatter", "miss", "cutoff", "step_limit")
ST_CELL_SKIPS = 11
ST_CELL_CROSSINGS = 12
TALLY_BITS = 24
RECORD_DTYPE = np.dtype([
    ("n_steps", "<u4"), ("n_virtual", "<u4"), ("n_rayleigh", "<u4"), ("n_compton", "<u4"),
    ("n_photo", "<u4"), ("outcome", "<u4"), ("rng_blocks", "<u4"), ("first_interaction", "<u4"),
    ("pixel", "<i4"), ("e_source", "<f4"), ("e_final", "<f4"), ("ray_material", "<u4"),
    ("e_deposited", "<f8")])


class GdrrError(RuntimeError):
    def __init__(self, call, code):
        msg = _lib_or_none().gdrr_error_string(code).decode() if _lib_or_none() else str(code)
        super().__init__(f"{call} failed: {msg} ({code})")
        self.code = code


class Geometry(ctypes.Structure):
    _fields_ = [("sad_mm", ctypes.c_double), ("sdd_mm", ctypes.c_double), ("theta_rad", ctypes.c_double),
                ("nu", ctypes.c_int32), ("nv", ctypes.c_int32), ("du_mm", ctypes.c_double), ("dv_mm", ctypes.c_double)]


class Phantom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx_mm", ctypes.c_double), ("dy_mm", ctypes.c_double), ("dz_mm", ctypes.c_double),
                ("material", ctypes.c_void_p), ("density", ctypes.c_void_p)]


class Materials(ctypes.Structure):
    _fields_ = [("n_materials", ctypes.c_int32), ("n_energies", ctypes.c_int32),
                ("e0_kev", ctypes.c_double), ("de_kev", ctypes.c_double), ("mu_hat", ctypes.c_void_p)]


class Spectrum(ctypes.Structure):
    _fields_ = [("n_bins", ctypes.c_int32), ("energy_kev", ctypes.c_void_p), ("weight", ctypes.c_void_p),
                ("column_weight", ctypes.c_void_p)]


class Bowtie(ctypes.Structure):
    _fields_ = [("fluence", ctypes.c_void_p)]


class Detector(ctypes.Structure):
    _fields_ = [("n_energies", ctypes.c_int32), ("e0_kev", ctypes.c_double), ("de_kev", ctypes.c_double),
                ("response", ctypes.c_void_p)]


class McOptions(ctypes.Structure):
    _fields_ = [("e_cut_kev", ctypes.c_double), ("max_steps", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("hist_per_thread", ctypes.c_int32),
                ("batch_min", ctypes.c_int32), ("nearest_voxel", ctypes.c_int32),
                ("scatter_filter", ctypes.c_int32), ("rayleigh_form_factor", ctypes.c_int32),
                ("cell_shift", ctypes.c_int32), ("photon_pool", ctypes.c_int32),
                ("local_majorant", ctypes.c_int32)]


class Projection(ctypes.Structure):
    _fields_ = [("angle_rad", ctypes.c_double), ("angle_index", ctypes.c_uint32), ("n_photons", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("bin_factor", ctypes.c_int32), ("beta", ctypes.c_double),
                ("smoothing_px", ctypes.c_double), ("omega", ctypes.c_double), ("iters", ctypes.c_int32),
                ("mAs", ctypes.c_double), ("zeta", ctypes.c_double)]


class ProjectionOut(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("P", "P_hat", "S_hat", "S", "N", "S_hat_coarse", "S_coarse",
                                               "prim_tally", "scat_tally", "stats")]


class ProjectionInfo(ctypes.Structure):
    _fields_ = [("count_scale", ctypes.c_double), ("beta", ctypes.c_double), ("mean_count", ctypes.c_double),
                ("tally_scatter", ctypes.c_uint64), ("step_limit", ctypes.c_uint64), ("below_floor", ctypes.c_int32),
                ("denoise_fused", ctypes.c_int32), ("transport_ms", ctypes.c_float), ("denoise_ms", ctypes.c_float),
                ("total_ms", ctypes.c_float)]


class FdkGeometry(ctypes.Structure):
    _fields_ = [("sad_mm", ctypes.c_double), ("sdd_mm", ctypes.c_double), ("nu", ctypes.c_int32),
                ("nv", ctypes.c_int32), ("du_mm", ctypes.c_double), ("dv_mm", ctypes.c_double),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx_mm", ctypes.c_double), ("dy_mm", ctypes.c_double), ("dz_mm", ctypes.c_double)]


class FormFactor(ctypes.Structure):
    _fields_ = [("n_x", ctypes.c_int32), ("dx_inv_angstrom", ctypes.c_double), ("form_factor", ctypes.c_void_p)]


_lib = None


def _lib_or_none():
    return _lib


def lib():
    """Load libgdrr.so (built by __graft_entry__.build() or build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgdrr.so not found at {LIB_PATH}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, u32, u64, i64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_int64, ctypes.c_double)
        sig = {
            "gdrr_create": [vp, vp, vp, vp, vp, vp, vp, vp],
            "gdrr_destroy": [vp],
            "gdrr_set_options": [vp, vp],
            "gdrr_set_form_factor": [vp, vp],
            "gdrr_get_options": [vp, vp],
            "gdrr_sync": [vp],
            "gdrr_raytrace_primary": [vp, dbl, vp],
            "gdrr_raytrace_primary_siddon": [vp, dbl, vp],
            "gdrr_mc_project": [vp, dbl, u32, u64, u64, u64, vp, vp, vp, vp],
            "gdrr_mc_project_batched": [vp, i32, vp, vp, u64, vp, vp, vp],
            "gdrr_finalize": [vp, vp, i64, u64, vp],
            "gdrr_bin_tally": [vp, vp, i32, i32, i32, vp],
            "gdrr_upsample": [vp, vp, i32, i32, i32, vp],
            "gdrr_denoise_scatter": [vp, vp, vp, i32, i32, dbl, dbl, dbl, i32],
            "gdrr_denoise_scatter_static": [vp, vp, i32, i32, dbl, dbl, dbl, i32, vp],
            "gdrr_noise_calibrate": [vp, vp, vp, vp, vp, i64, u64, dbl, dbl, vp],
            "gdrr_fit_zeta": [vp, vp, i32, u64, vp, vp],
            "gdrr_stream_words": [u64, u32, u64, i32, i32, vp, vp],
            "gdrr_gather_roofline": [vp, u64, vp],
            "gdrr_scan_create": [vp, i32, vp, vp, u64, vp, vp, vp, i32, vp],
            "gdrr_scan_launch": [vp],
            "gdrr_scan_destroy": [vp],
            "gdrr_autotune": [vp, dbl, u64, u64, vp],
            "gdrr_gemm_bf16": [vp, i32, vp, i32, vp, i32, i32, i32, i32, i32, vp],
            "gdrr_scale_to_f32": [vp, i64, dbl, vp, vp],
            "gdrr_scale_to_f64": [vp, i64, dbl, vp, vp],
            "gdrr_cnn_create": [i32, i32, i32, i32, u64, vp, vp],
            "gdrr_cnn_destroy": [vp],
            "gdrr_cnn_num_params": [vp, vp],
            "gdrr_cnn_get_params": [vp, vp],
            "gdrr_cnn_set_params": [vp, vp],
            "gdrr_cnn_get_grads": [vp, vp],
            "gdrr_cnn_forward": [vp, i32, vp, vp],
            "gdrr_cnn_backward": [vp, vp, vp],
            "gdrr_cnn_adam_step": [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float],
            "gdrr_air_scan": [vp, vp],
            "gdrr_probe_l2_gather": [i64, vp, vp],
            "gdrr_probe_fp32": [vp, vp],
            "gdrr_line_integrals": [vp, vp, i64, dbl, vp, vp],
            "gdrr_fdk_filter": [vp, i32, vp, vp, vp],
            "gdrr_fdk_backproject": [vp, i32, vp, dbl, vp, vp, i32, vp],
            "gdrr_project": [vp, vp, vp, vp],
            "gdrr_probe_bounded_wait": [u64, vp],
            "gdrr_release_memory": [],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None if name in ("gdrr_destroy", "gdrr_scan_destroy", "gdrr_cnn_destroy") else ctypes.c_int
        L.gdrr_error_string.argtypes = [ctypes.c_int]
        L.gdrr_error_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(call, rc):
    if rc != 0:
        raise GdrrError(call, rc)


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t, dtype, numel=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream), stream


class Context:
    """Owns a gdrr_ctx: the staged phantom, tables and scratch of one problem."""

    def __init__(self, prob, stream=None):
        import torch
        self._handle = None
        self.prob = prob
        self.nu, self.nv = int(prob.nu), int(prob.nv)
        h, self.stream = _stream_handle(stream)
        keep = dict(
            material=np.ascontiguousarray(prob.material, np.uint8),
            density=np.ascontiguousarray(prob.density, np.float32),
            mu_hat=np.ascontiguousarray(prob.mu_hat, np.float32),
            spec_e=np.ascontiguousarray(prob.spec_e, np.float64),
            spec_w=np.ascontiguousarray(prob.spec_w, np.float64),
            fluence=np.ascontiguousarray(prob.fluence, np.float64),
            response=np.ascontiguousarray(prob.response, np.float32))
        nz, ny, nx = keep["material"].shape
        geo = Geometry(prob.sad, prob.sdd, prob.theta, self.nu, self.nv, prob.du, prob.dv)
        ph = Phantom(nx, ny, nz, prob.voxel[0], prob.voxel[1], prob.voxel[2],
                     _np_ptr(keep["material"]), _np_ptr(keep["density"]))
        mt = Materials(keep["mu_hat"].shape[0], keep["mu_hat"].shape[2], prob.e0, prob.de, _np_ptr(keep["mu_hat"]))
        cols = getattr(prob, "spec_cols", None)
        if cols is not None:
            keep["spec_cols"] = np.ascontiguousarray(cols, np.float64)
            if keep["spec_cols"].shape != (self.nu, keep["spec_e"].size):
                raise ValueError("spec_cols must be [nu, n_bins]")
        sp = Spectrum(keep["spec_e"].size, _np_ptr(keep["spec_e"]), _np_ptr(keep["spec_w"]),
                      _np_ptr(keep["spec_cols"]) if cols is not None else None)
        bt = Bowtie(_np_ptr(keep["fluence"]))
        dt = Detector(keep["response"].size, prob.r0, prob.dr, _np_ptr(keep["response"]))
        handle = ctypes.c_void_p()
        torch.cuda.current_device()   # make sure torch has set up the primary context
        _check("gdrr_create", lib().gdrr_create(ctypes.byref(geo), ctypes.byref(ph), ctypes.byref(mt),
                                                ctypes.byref(sp), ctypes.byref(bt), ctypes.byref(dt), h,
                                                ctypes.byref(handle)))
        self._handle = handle
        ff = getattr(prob, "form_factor", None)
        if ff is not None:
            gdrr_set_form_factor(self, ff, prob.ff_dx)

    @property
    def handle(self):
        if self._handle is None:
            raise RuntimeError("context is closed")
        return self._handle

    def close(self):
        if self._handle is not None:
            lib().gdrr_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- the C ABI, one wrapper per call -------------------------------------

def gdrr_create(prob, stream=None) -> Context:
    return Context(prob, stream)


def gdrr_destroy(ctx: Context):
    ctx.close()


def gdrr_release_memory():
    """Return the unused blocks of the contexts' device memory pools."""
    _check("gdrr_release_memory", lib().gdrr_release_memory())


def gdrr_set_options(ctx: Context, **kw):
    o = McOptions()
    _check("gdrr_get_options", lib().gdrr_get_options(ctx.handle, ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    if "local_majorant" in kw:           # the defaults of the chosen tracking
        if "cell_shift" not in kw:
            o.cell_shift = 0
        if "batch_min" not in kw:
            o.batch_min = 0
    _check("gdrr_set_options", lib().gdrr_set_options(ctx.handle, ctypes.byref(o)))


def gdrr_set_form_factor(ctx: Context, form_factor, dx_inv_angstrom: float):
    """Rayleigh form factors F(x) [n_materials, n_x] on x_j = j * dx (1/Angstrom),
    or None to remove them."""
    if form_factor is None:
        f = FormFactor(0, 0.0, None)
        _check("gdrr_set_form_factor", lib().gdrr_set_form_factor(ctx.handle, ctypes.byref(f)))
        return
    t = np.ascontiguousarray(form_factor, np.float32)
    f = FormFactor(t.shape[1], float(dx_inv_angstrom), _np_ptr(t))
    _check("gdrr_set_form_factor", lib().gdrr_set_form_factor(ctx.handle, ctypes.byref(f)))


def gdrr_get_options(ctx: Context) -> dict:
    o = McOptions()
    _check("gdrr_get_options", lib().gdrr_get_options(ctx.handle, ctypes.byref(o)))
    return {k: getattr(o, k) for k, _ in McOptions._fields_}


def gdrr_sync(ctx: Context):
    _check("gdrr_sync", lib().gdrr_sync(ctx.handle))


def gdrr_raytrace_primary(ctx: Context, angle_rad: float, out=None):
    import torch
    if out is None:
        out = torch.empty((ctx.nv, ctx.nu), dtype=torch.float64, device="cuda")
    _check("gdrr_raytrace_primary",
           lib().gdrr_raytrace_primary(ctx.handle, float(angle_rad), _dev_ptr(out, torch.float64, ctx.nu * ctx.nv, "P")))
    return out


def gdrr_raytrace_primary_siddon(ctx: Context, angle_rad: float, out=None):
    import torch
    if out is None:
        out = torch.empty((ctx.nv, ctx.nu), dtype=torch.float64, device="cuda")
    _check("gdrr_raytrace_primary_siddon",
           lib().gdrr_raytrace_primary_siddon(ctx.handle, float(angle_rad),
                                              _dev_ptr(out, torch.float64, ctx.nu * ctx.nv, "P")))
    return out


def new_tallies(ctx: Context, n_angles: int | None = None):
    import torch
    shape = (ctx.nv, ctx.nu) if n_angles is None else (n_angles, ctx.nv, ctx.nu)
    return (torch.zeros(shape, dtype=torch.int64, device="cuda"),
            torch.zeros(shape, dtype=torch.int64, device="cuda"))


def gdrr_mc_project(ctx: Context, n_photons: int, seed: int, angle_rad: float = 0.0, angle_index: int = 0,
                    history_offset: int = 0, prim=None, scat=None, stats=None, records=None):
    """Accumulates into prim / scat (int64 [nv, nu], created zeroed if None)."""
    import torch
    if prim is None or scat is None:
        prim, scat = new_tallies(ctx)
    npix = ctx.nu * ctx.nv
    sp = _dev_ptr(stats, torch.int64, GDRR_NSTATS, "stats") if stats is not None else None
    rp = None
    if records is not None:
        if records.dtype != torch.uint8 or records.numel() != n_photons * RECORD_DTYPE.itemsize:
            raise ValueError("records must be a uint8 CUDA tensor of n_photons * record size bytes")
        rp = _dev_ptr(records, torch.uint8, None, "records")
    _check("gdrr_mc_project",
           lib().gdrr_mc_project(ctx.handle, float(angle_rad), int(angle_index), int(n_photons), int(seed),
                                 int(history_offset), _dev_ptr(prim, torch.int64, npix, "prim"),
                                 _dev_ptr(scat, torch.int64, npix, "scat"), sp, rp))
    return prim, scat


def gdrr_mc_project_batched(ctx: Context, angles_rad, budgets, seed: int, prim=None, scat=None, stats=None):
    import torch
    angles = np.ascontiguousarray(angles_rad, np.float64)
    bud = np.ascontiguousarray(budgets, np.uint64)
    if angles.size != bud.size:
        raise ValueError("angles and budgets differ in length")
    if prim is None or scat is None:
        prim, scat = new_tallies(ctx, angles.size)
    n = angles.size * ctx.nu * ctx.nv
    sp = _dev_ptr(stats, torch.int64, GDRR_NSTATS, "stats") if stats is not None else None
    _check("gdrr_mc_project_batched",
           lib().gdrr_mc_project_batched(ctx.handle, angles.size, _np_ptr(angles), _np_ptr(bud), int(seed),
                                         _dev_ptr(prim, torch.int64, n, "prim"), _dev_ptr(scat, torch.int64, n, "scat"),
                                         sp))
    return prim, scat


class Scan:
    """A multi-angle scan captured as a CUDA graph (gdrr_scan_create)."""

    def __init__(self, ctx: Context, angles_rad, budgets, seed: int, prim=None, scat=None, stats=None,
                 zero_tallies: bool = True):
        import torch
        self.ctx = ctx
        self.angles = np.ascontiguousarray(angles_rad, np.float64)
        self.budgets = np.ascontiguousarray(budgets, np.uint64)
        if prim is None or scat is None:
            prim, scat = new_tallies(ctx, self.angles.size)
        self.prim, self.scat, self.stats = prim, scat, stats
        n = self.angles.size * ctx.nu * ctx.nv
        h = ctypes.c_void_p()
        sp = _dev_ptr(stats, torch.int64, GDRR_NSTATS, "stats") if stats is not None else None
        _check("gdrr_scan_create",
               lib().gdrr_scan_create(ctx.handle, self.angles.size, _np_ptr(self.angles), _np_ptr(self.budgets),
                                      int(seed), _dev_ptr(prim, torch.int64, n, "prim"),
                                      _dev_ptr(scat, torch.int64, n, "scat"), sp, int(bool(zero_tallies)),
                                      ctypes.byref(h)))
        self._h = h

    def launch(self):
        _check("gdrr_scan_launch", lib().gdrr_scan_launch(self._h))
        return self.prim, self.scat

    def close(self):
        if self._h is not None:
            lib().gdrr_scan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gdrr_scan_create(ctx: Context, angles_rad, budgets, seed: int, prim=None, scat=None, stats=None,
                     zero_tallies: bool = True) -> Scan:
    return Scan(ctx, angles_rad, budgets, seed, prim, scat, stats, zero_tallies)


def gdrr_scan_launch(scan: Scan):
    return scan.launch()


def gdrr_scan_destroy(scan: Scan):
    scan.close()


def gdrr_autotune(ctx: Context, angle_rad: float = 0.0, n_probe: int = 10_000_000, seed: int = 1) -> dict:
    o = McOptions()
    _check("gdrr_autotune", lib().gdrr_autotune(ctx.handle, float(angle_rad), int(n_probe), int(seed),
                                                ctypes.byref(o)))
    return {k: getattr(o, k) for k, _ in McOptions._fields_}


def gdrr_finalize(ctx: Context, tally, n_photons: int, out=None):
    import torch
    if out is None:
        out = torch.empty(tally.shape, dtype=torch.float64, device="cuda")
    _check("gdrr_finalize", lib().gdrr_finalize(ctx.handle, _dev_ptr(tally, torch.int64, None, "tally"), tally.numel(),
                                                int(n_photons), _dev_ptr(out, torch.float64, tally.numel(), "out")))
    return out


def gdrr_bin_tally(ctx: Context, tally, factor: int, out=None):
    import torch
    nv, nu = tally.shape[-2:]
    if out is None:
        out = torch.empty((nv // factor, nu // factor), dtype=torch.int64, device="cuda")
    _check("gdrr_bin_tally", lib().gdrr_bin_tally(ctx.handle, _dev_ptr(tally, torch.int64, nu * nv, "tally"), nu, nv,
                                                  int(factor), _dev_ptr(out, torch.int64, (nu // factor) * (nv // factor), "out")))
    return out


def gdrr_upsample(ctx: Context, coarse, factor: int, out=None):
    import torch
    cv, cu = coarse.shape
    if out is None:
        out = torch.empty((cv * factor, cu * factor), dtype=torch.float64, device="cuda")
    _check("gdrr_upsample", lib().gdrr_upsample(ctx.handle, _dev_ptr(coarse, torch.float64, cu * cv, "coarse"), cu, cv,
                                                int(factor), _dev_ptr(out, torch.float64, cu * cv * factor * factor, "out")))
    return out


def gdrr_denoise_scatter(ctx: Context, s_hat, count_scale: float, beta: float, omega: float = 0.8,
                         iters: int = 500, out=None):
    import torch
    nv, nu = s_hat.shape
    if out is None:
        out = torch.empty_like(s_hat)
    _check("gdrr_denoise_scatter",
           lib().gdrr_denoise_scatter(ctx.handle, _dev_ptr(s_hat, torch.float64, nu * nv, "s_hat"),
                                      _dev_ptr(out, torch.float64, nu * nv, "out"), nu, nv, float(count_scale),
                                      float(beta), float(omega), int(iters)))
    return out


STATIC_DENOISE_MAX_PIXELS = 65536


def gdrr_denoise_scatter_static(s_hat, count_scale: float, beta: float, omega: float = 0.8, iters: int = 500,
                                out=None, stream=None):
    """The denoiser without a context and without device allocation inside the
    library (its scratch is a static device array shared by all calls)."""
    import torch
    nv, nu = s_hat.shape
    if out is None:
        out = torch.empty_like(s_hat)
    dev = torch.cuda.current_device()
    if s_hat.device.index != dev or out.device.index != dev:
        raise ValueError("gdrr_denoise_scatter_static runs on the current device: s_hat and out must live there")
    h, _ = _stream_handle(stream)
    _check("gdrr_denoise_scatter_static",
           lib().gdrr_denoise_scatter_static(_dev_ptr(s_hat, torch.float64, nu * nv, "s_hat"),
                                             _dev_ptr(out, torch.float64, nu * nv, "out"), nu, nv,
                                             float(count_scale), float(beta), float(omega), int(iters), h))
    return out


def gdrr_noise_calibrate(ctx: Context, p_hat, p, s_hat, s, n_sim: int, mas: float, zeta: float, out=None):
    import torch
    n = p_hat.numel()
    if out is None:
        out = torch.empty_like(p_hat)
    ptrs = [_dev_ptr(t, torch.float64, n, nm) for t, nm in ((p_hat, "p_hat"), (p, "p"), (s_hat, "s_hat"), (s, "s"))]
    _check("gdrr_noise_calibrate", lib().gdrr_noise_calibrate(ctx.handle, *ptrs, n, int(n_sim), float(mas), float(zeta),
                                                              _dev_ptr(out, torch.float64, n, "out")))
    return out


def gdrr_fit_zeta(inv_sqrt_mas, ratio, n_sim: int):
    x = np.ascontiguousarray(inv_sqrt_mas, np.float64)
    y = np.ascontiguousarray(ratio, np.float64)
    z, k = ctypes.c_double(), ctypes.c_double()
    _check("gdrr_fit_zeta", lib().gdrr_fit_zeta(_np_ptr(x), _np_ptr(y), x.size, int(n_sim), ctypes.byref(z),
                                                ctypes.byref(k)))
    return z.value, k.value


def gdrr_stream_words(seed: int, angle_index: int, hid0: int, n_hist: int, n_blocks: int, stream=None):
    import torch
    out = torch.empty((n_hist, 4 * n_blocks), dtype=torch.int32, device="cuda")
    h, _ = _stream_handle(stream)
    _check("gdrr_stream_words", lib().gdrr_stream_words(int(seed), int(angle_index), int(hid0), int(n_hist),
                                                        int(n_blocks), _dev_ptr(out, torch.int32, None, "out"), h))
    return out


def gdrr_gather_roofline(ctx: Context, n_cells: int) -> float:
    """Seconds the transport's corner gathers alone take for n_cells cells."""
    sec = ctypes.c_double()
    _check("gdrr_gather_roofline", lib().gdrr_gather_roofline(ctx.handle, int(n_cells), ctypes.byref(sec)))
    return sec.value


def gdrr_probe_l2_gather(working_set_bytes: int = 32 << 20, stream=None) -> float:
    """GB/s of random 8-byte loads over an L2-resident working set."""
    h, _ = _stream_handle(stream)
    out = ctypes.c_double()
    _check("gdrr_probe_l2_gather", lib().gdrr_probe_l2_gather(int(working_set_bytes), ctypes.byref(out), h))
    return out.value


def gdrr_probe_bounded_wait(limit_ns: int, stream=None) -> int:
    """Return code of a bounded device wait on a flag nothing sets (-7: timed out)."""
    h, _ = _stream_handle(stream)
    return lib().gdrr_probe_bounded_wait(int(limit_ns), h)


def gdrr_probe_fp32(stream=None) -> float:
    """FP32 FMA throughput in TFLOP/s."""
    h, _ = _stream_handle(stream)
    out = ctypes.c_double()
    _check("gdrr_probe_fp32", lib().gdrr_probe_fp32(ctypes.byref(out), h))
    return out.value


def stats_dict(stats) -> dict:
    """The method's event counters and the cell crossings (the oracle counts
    the same ones); stats a device tensor or a host array."""
    v = (stats.cpu().numpy() if hasattr(stats, "cpu") else np.asarray(stats)).view(np.uint64)
    d = dict(zip(STAT_NAMES, (int(x) for x in v)))
    d["crossings"] = int(v[ST_CELL_CROSSINGS])
    return d


def cell_skips(stats) -> int:
    """Virtual collisions the macro-cell bound decided without corner gathers."""
    return int(stats.cpu().numpy().view(np.uint64)[ST_CELL_SKIPS])


def records_array(records) -> np.ndarray:
    return records.cpu().numpy().view(RECORD_DTYPE)


# ---- one full projection: Steps 1-4 of Section 2.2 ------------------------

def denoise_stability_floor(omega: float = 0.8) -> float:
    """Smallest beta * S (S in counts) at which the Eq. 5 iteration converges.

    Linearised at its fixed point, Eq. 5 multiplies a perturbation along an
    eigenvector of the neighbour sum (eigenvalue lam in (-4, 4]) by
    1 - omega + (omega / 4) (lam - 1 / (beta S)) per iteration.  The
    checkerboard (lam -> -4) bounds it: |.| < 1 needs beta S > omega / (8 (1 - omega)),
    0.5 at omega = 0.8; for omega >= 1 no beta converges."""
    if not 0.0 < omega < 1.0:
        return math.inf
    return omega / (8.0 * (1.0 - omega))


def project(ctx: Context, n_photons: int, seed: int, angle_rad: float = 0.0, bin_factor: int = 4,
            beta: float = 0.02, omega: float = 0.8, iters: int = 300, mas: float = 0.4,
            zeta: float = 5.2913e9, stats=None, angle_index: int = 0, smoothing_px: float | None = None,
            out: dict | None = None, allow_step_limit: bool = False):
    """One projection through gdrr_project: P (ray traced), P^ and S^ (MC), S
    (denoised, coarse and full), N (scaled noise), and the int64 tallies.

    Every step and every scalar is computed by the library on the device;
    this wrapper only allocates the outputs (or takes them from ``out``, a
    dict of preallocated CUDA tensors with the keys of the result) and reads
    the scalars the call returns.  The denoiser runs on the bin_factor x
    bin_factor coarse scatter grid on the count scale (the mean signal of one
    detected scattered photon).  beta is in counts^-1; smoothing_px, when
    given, replaces it by smoothing_px^2 / (mean coarse count).  A warning
    says when beta times the mean count is below the Eq. 5 convergence floor.
    stats, when given, receives this projection's counters (overwritten).
    GDRR_ERR_STEP_LIMIT raises unless allow_step_limit is true.
    """
    import torch
    nv, nu = ctx.nv, ctx.nu
    if nu % bin_factor or nv % bin_factor:
        raise ValueError("detector size must be a multiple of bin_factor")
    cu, cv = nu // bin_factor, nv // bin_factor
    o = dict(out or {})

    def buf(key, shape, dtype):
        if key not in o or o[key] is None:
            o[key] = torch.empty(shape, dtype=dtype, device="cuda")
        return o[key]

    if stats is not None:
        o["stats"] = stats
    f64 = torch.float64
    specs = (("P", (nv, nu), f64), ("P_hat", (nv, nu), f64), ("S_hat", (nv, nu), f64), ("S", (nv, nu), f64),
             ("N", (nv, nu), f64), ("S_hat_coarse", (cv, cu), f64), ("S_coarse", (cv, cu), f64),
             ("prim", (nv, nu), torch.int64), ("scat", (nv, nu), torch.int64), ("stats", (GDRR_NSTATS,), torch.int64))
    ptr = {k: _dev_ptr(buf(k, shp, dt), dt, math.prod(shp), k) for k, shp, dt in specs}
    po = ProjectionOut(ptr["P"], ptr["P_hat"], ptr["S_hat"], ptr["S"], ptr["N"], ptr["S_hat_coarse"],
                       ptr["S_coarse"], ptr["prim"], ptr["scat"], ptr["stats"])
    pr = Projection(float(angle_rad), int(angle_index), int(n_photons), int(seed), int(bin_factor), float(beta),
                    float(smoothing_px) if smoothing_px is not None else 0.0, float(omega), int(iters), float(mas),
                    float(zeta))
    info = ProjectionInfo()
    rc = lib().gdrr_project(ctx.handle, ctypes.byref(pr), ctypes.byref(po), ctypes.byref(info))
    if rc != 0 and not (allow_step_limit and rc == -5):
        raise GdrrError("gdrr_project", rc)
    if info.below_floor:
        warnings.warn(f"beta * mean scatter count = {info.beta * info.mean_count:.3g} is below "
                      f"{denoise_stability_floor(omega):.3g}: the Eq. 5 iteration diverges on most of the image "
                      "(raise beta, n_photons or bin_factor, or pass smoothing_px)", RuntimeWarning, stacklevel=2)
    res = {k: o[k] for k, _, _ in specs}
    res.update(count_scale=info.count_scale, beta=info.beta, mean_count=info.mean_count,
               step_limit=info.step_limit, denoise_fused=bool(info.denoise_fused),
               transport_ms=info.transport_ms, denoise_ms=info.denoise_ms, total_ms=info.total_ms)
    return res


# ---- reconstruction of simulated scans (Section 3.5) ----------------------

def gdrr_air_scan(ctx: Context, out=None):
    """Unattenuated signal I0 [nv, nu] FP64 of the context's source and detector."""
    import torch
    if out is None:
        out = torch.empty((ctx.nv, ctx.nu), dtype=torch.float64, device="cuda")
    _check("gdrr_air_scan", lib().gdrr_air_scan(ctx.handle, _dev_ptr(out, torch.float64, ctx.nu * ctx.nv, "I0")))
    return out


def gdrr_line_integrals(signal, air, floor_rel: float = 1e-6, out=None, stream=None):
    """g = -ln(max(I, floor I0) / I0), FP32, same shape as signal."""
    import torch
    if out is None:
        out = torch.empty(signal.shape, dtype=torch.float32, device="cuda")
    h, _ = _stream_handle(stream)
    n = signal.numel()
    _check("gdrr_line_integrals", lib().gdrr_line_integrals(_dev_ptr(signal, torch.float64, None, "signal"),
                                                            _dev_ptr(air, torch.float64, n, "air"), n,
                                                            float(floor_rel), _dev_ptr(out, torch.float32, n, "out"),
                                                            h))
    return out


def fdk_geometry(sad, sdd, nu, nv, du, dv, shape, voxel) -> FdkGeometry:
    nz, ny, nx = shape
    return FdkGeometry(float(sad), float(sdd), int(nu), int(nv), float(du), float(dv), int(nx), int(ny), int(nz),
                       float(voxel[0]), float(voxel[1]), float(voxel[2]))


def gdrr_fdk_filter(geo: FdkGeometry, proj, out=None, stream=None):
    """Cosine-weighted Ram-Lak filtering of line integrals [n_proj, nv, nu] FP32."""
    import torch
    if out is None:
        out = torch.empty_like(proj)
    h, _ = _stream_handle(stream)
    n_proj = proj.shape[0]
    _check("gdrr_fdk_filter", lib().gdrr_fdk_filter(ctypes.byref(geo), n_proj,
                                                    _dev_ptr(proj, torch.float32, n_proj * geo.nu * geo.nv, "proj"),
                                                    _dev_ptr(out, torch.float32, n_proj * geo.nu * geo.nv, "out"), h))
    return out


def gdrr_fdk_backproject(geo: FdkGeometry, filtered, angles, d_beta=None, volume=None, accumulate=False,
                         stream=None):
    """Voxel-driven FDK backprojection into [nz, ny, nx] FP32 (1/mm)."""
    import torch
    ang = np.ascontiguousarray(angles, np.float64)
    n_proj = ang.size
    if d_beta is None:
        d_beta = 2.0 * math.pi / n_proj
    if volume is None:
        volume = torch.empty((geo.nz, geo.ny, geo.nx), dtype=torch.float32, device="cuda")
        accumulate = False
    h, _ = _stream_handle(stream)
    _check("gdrr_fdk_backproject",
           lib().gdrr_fdk_backproject(ctypes.byref(geo), n_proj, _np_ptr(ang), float(d_beta),
                                      _dev_ptr(filtered, torch.float32, n_proj * geo.nu * geo.nv, "filtered"),
                                      _dev_ptr(volume, torch.float32, geo.nx * geo.ny * geo.nz, "volume"),
                                      1 if accumulate else 0, h))
    return volume


def fdk(geo: FdkGeometry, proj, angles, d_beta=None, stream=None):
    """Full FDK reconstruction of line integrals [n_proj, nv, nu] FP32."""
    return gdrr_fdk_backproject(geo, gdrr_fdk_filter(geo, proj, stream=stream), angles, d_beta, stream=stream)


# ---- tensor-core GEMM and the learned scatter estimator ------------------

def gdrr_scale_to_f32(src, scale: float, out, stream=None):
    import torch
    h, _ = _stream_handle(stream)
    _check("gdrr_scale_to_f32", lib().gdrr_scale_to_f32(_dev_ptr(src, torch.float64, None, "src"), src.numel(),
                                                        float(scale), _dev_ptr(out, torch.float32, src.numel(), "out"),
                                                        h))
    return out


def gdrr_scale_to_f64(src, scale: float, out, stream=None):
    import torch
    h, _ = _stream_handle(stream)
    _check("gdrr_scale_to_f64", lib().gdrr_scale_to_f64(_dev_ptr(src, torch.float32, None, "src"), src.numel(),
                                                        float(scale), _dev_ptr(out, torch.float64, src.numel(), "out"),
                                                        h))
    return out


def _row_major_ptr(t, dtype, name):
    """Device pointer of a 2-D CUDA tensor whose rows are contiguous (any row stride)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dim() != 2:
        raise TypeError(f"{name} must be a 2-D CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.stride(1) != 1:
        raise ValueError(f"{name} rows must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def gdrr_gemm_bf16(a, b, splits: int = 1, out=None, stream=None):
    """C = A . B^T for BF16 CUDA tensors A [M, K], B [N, K] (K a multiple of 64;
    rows contiguous, row strides multiples of 8 elements)."""
    import torch
    M, K = a.shape
    N = b.shape[0]
    if out is None:
        out = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    h, _ = _stream_handle(stream)
    _check("gdrr_gemm_bf16", lib().gdrr_gemm_bf16(_row_major_ptr(a, torch.bfloat16, "A"), a.stride(0),
                                                  _row_major_ptr(b, torch.bfloat16, "B"), b.stride(0),
                                                  _row_major_ptr(out, torch.float32, "C"), out.stride(0),
                                                  M, N, K, int(splits), h))
    return out


class Cnn:
    """gdrr_cnn: the learned scatter estimator (forward, backward, Adam)."""

    def __init__(self, max_batch: int, height: int, width: int, base_channels: int = 32, seed: int = 1,
                 stream=None):
        h, self.stream = _stream_handle(stream)
        self.max_batch, self.height, self.width, self.c = max_batch, height, width, base_channels
        self._h = ctypes.c_void_p()
        _check("gdrr_cnn_create", lib().gdrr_cnn_create(max_batch, height, width, base_channels, int(seed), h,
                                                        ctypes.byref(self._h)))
        n = ctypes.c_int64()
        _check("gdrr_cnn_num_params", lib().gdrr_cnn_num_params(self._h, ctypes.byref(n)))
        self.n_params = n.value

    def get_params(self):
        out = np.empty(self.n_params, np.float32)
        _check("gdrr_cnn_get_params", lib().gdrr_cnn_get_params(self._h, _np_ptr(out)))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        if p.size != self.n_params:
            raise ValueError("wrong parameter count")
        _check("gdrr_cnn_set_params", lib().gdrr_cnn_set_params(self._h, _np_ptr(p)))

    def get_grads(self):
        out = np.empty(self.n_params, np.float32)
        _check("gdrr_cnn_get_grads", lib().gdrr_cnn_get_grads(self._h, _np_ptr(out)))
        return out

    def forward(self, x, out=None):
        import torch
        B = x.shape[0]
        if out is None:
            out = torch.empty((B, 1, self.height, self.width), dtype=torch.float32, device="cuda")
        _check("gdrr_cnn_forward", lib().gdrr_cnn_forward(self._h, B, _dev_ptr(x, torch.float32,
                                                                                B * 2 * self.height * self.width, "x"),
                                                          _dev_ptr(out, torch.float32, None, "out")))
        return out

    def backward(self, target) -> float:
        import torch
        loss = ctypes.c_double()
        _check("gdrr_cnn_backward", lib().gdrr_cnn_backward(self._h, _dev_ptr(target, torch.float32, None, "target"),
                                                            ctypes.byref(loss)))
        return loss.value

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check("gdrr_cnn_adam_step", lib().gdrr_cnn_adam_step(self._h, lr, beta1, beta2, eps))

    def close(self):
        if self._h is not None and self._h.value:
            lib().gdrr_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
