"""The C ABI library loads without a GPU and exports every symbol declared in
include/gdrr.h; host-side argument validation rejects bad inputs before any
CUDA call (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "gdrr.h")).read()
    return sorted(set(re.findall(r"GDRR_API\s+[^;(]*?\b(gdrr_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1204_6367_gb300 import build, gdrr
    build.build()
    return gdrr.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gdrr_create", "gdrr_raytrace_primary", "gdrr_mc_project", "gdrr_denoise_scatter",
                     "gdrr_noise_calibrate", "gdrr_finalize", "gdrr_destroy", "gdrr_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_library_exports_nothing_else(lib):
    import subprocess
    from paper_1204_6367_gb300 import gdrr
    out = subprocess.run(["nm", "-D", "--defined-only", gdrr.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("gdrr_")}
    assert exported == set(_declared())


def test_error_strings(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.gdrr_error_string(code)
    assert lib.gdrr_error_string(-99) == b"unknown error"


def test_fit_zeta_host_only(lib):
    from paper_1204_6367_gb300 import gdrr
    from tests.golden.load import load
    g = load("paper_noise_calibration.txt")
    x = 1 / np.sqrt(np.array([0.1, 0.4, 1.6]))
    z, k = gdrr.gdrr_fit_zeta(x, g["k"] * x, int(g["n_sim"]))
    assert z == pytest.approx(g["zeta"], rel=g["rel_tol"]) and k == pytest.approx(g["k"])
    with pytest.raises(gdrr.GdrrError):
        gdrr.gdrr_fit_zeta(np.zeros(3), np.ones(3), 10)


def _create_rc(prob, **override):
    """gdrr_create on a problem with fields overridden; validation runs before
    any CUDA call, so rejected inputs return without touching a device."""
    from paper_1204_6367_gb300 import gdrr
    L = gdrr.lib()
    mat = np.ascontiguousarray(override.pop("material", prob.material), np.uint8)
    den = np.ascontiguousarray(override.pop("density", prob.density), np.float32)
    mu = np.ascontiguousarray(override.pop("mu_hat", prob.mu_hat), np.float32)
    se = np.ascontiguousarray(prob.spec_e, np.float64)
    sw = np.ascontiguousarray(override.pop("spec_w", prob.spec_w), np.float64)
    fl = np.ascontiguousarray(override.pop("fluence", prob.fluence), np.float64)
    rs = np.ascontiguousarray(prob.response, np.float32)
    nz, ny, nx = mat.shape
    geo = gdrr.Geometry(prob.sad, override.pop("sdd", prob.sdd), prob.theta, prob.nu, prob.nv, prob.du, prob.dv)
    ph = gdrr.Phantom(nx, ny, nz, *prob.voxel, mat.ctypes.data, den.ctypes.data)
    mt = gdrr.Materials(override.pop("n_materials", mu.shape[0]), mu.shape[2], prob.e0, prob.de, mu.ctypes.data)
    sp = gdrr.Spectrum(se.size, se.ctypes.data, sw.ctypes.data)
    bt = gdrr.Bowtie(fl.ctypes.data)
    dt = gdrr.Detector(rs.size, prob.r0, prob.dr, rs.ctypes.data)
    h = ctypes.c_void_p()
    return L.gdrr_create(ctypes.byref(geo), ctypes.byref(ph), ctypes.byref(mt), ctypes.byref(sp), ctypes.byref(bt),
                         ctypes.byref(dt), None, ctypes.byref(h))


def test_create_rejects_bad_inputs(lib, small):
    # the host checks these before any CUDA call (invalid voxels are found
    # by the device staging kernel: tests/test_gpu_parity.py)
    assert _create_rc(small, spec_w=-small.spec_w) == -1
    assert _create_rc(small, fluence=np.zeros_like(small.fluence)) == -1
    assert _create_rc(small, sdd=1030.0) == -1          # imager plane cuts the box
    assert _create_rc(small, n_materials=9) in (-1, -6)


def test_null_arguments(lib):
    assert lib.gdrr_create(None, None, None, None, None, None, None, None) == -1
    assert lib.gdrr_mc_project(None, 0.0, 0, 10, 1, 0, None, None, None, None) == -1
    assert lib.gdrr_raytrace_primary(None, 0.0, None) == -1
    assert lib.gdrr_denoise_scatter(None, None, None, 4, 4, 1.0, 1.0, 0.8, 1) == -1
    assert lib.gdrr_stream_words(1, 0, 0, -1, 1, None, None) == -1
    assert lib.gdrr_project(None, None, None, None) == -1
    assert lib.gdrr_probe_bounded_wait(0, None) == -1


def test_projection_structs_match_the_header():
    # the binding's ctypes layouts against the C declarations, field by field
    import re
    from paper_1204_6367_gb300 import gdrr
    text = open(os.path.join(ROOT, "include", "gdrr.h")).read()
    for cname, cls in (("gdrr_projection", gdrr.Projection), ("gdrr_projection_out", gdrr.ProjectionOut),
                       ("gdrr_projection_info", gdrr.ProjectionInfo), ("gdrr_mc_options", gdrr.McOptions)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + r";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"\b(\w+)\s*;", body)
        assert fields == [f for f, _ in cls._fields_], cname


def test_stats_layout_matches_the_header():
    # the counters' enum of the header and the binding's slots: the method's
    # eleven counters, then the cell-test skips and the cell crossings
    import re
    from paper_1204_6367_gb300 import gdrr
    text = open(os.path.join(ROOT, "include", "gdrr.h")).read()
    body = re.search(r"enum \{\s*(GDRR_ST_HISTORIES[^}]*)\}", text).group(1)
    names = [n.split("=")[0].strip() for n in body.replace("\n", " ").split(",") if n.strip()]
    assert names[-1] == "GDRR_NSTATS" and len(names) - 1 == gdrr.GDRR_NSTATS
    assert names.index("GDRR_ST_CELL_SKIPS") == gdrr.ST_CELL_SKIPS
    assert names.index("GDRR_ST_CELL_CROSSINGS") == gdrr.ST_CELL_CROSSINGS
    v = np.arange(gdrr.GDRR_NSTATS, dtype=np.uint64) * 3 + 1
    d = gdrr.stats_dict(v.view(np.int64))
    assert [d[k] for k in gdrr.STAT_NAMES] == [int(x) for x in v[:len(gdrr.STAT_NAMES)]]
    assert d["crossings"] == int(v[gdrr.ST_CELL_CROSSINGS]) and "cell_skips" not in d


def test_option_helper_takes_the_tracking_defaults(monkeypatch):
    # gdrr_set_options reads the context's options, applies the keywords and
    # writes them back; switching the tracking resets cell_shift and batch_min
    # to 0 (the library's defaults for that tracking) unless they are given
    import ctypes as ct
    from paper_1204_6367_gb300 import gdrr
    written = []

    class FakeLib:
        def gdrr_get_options(self, handle, ref):
            o = ct.cast(ref, ct.POINTER(gdrr.McOptions)).contents
            o.cell_shift, o.batch_min, o.block_size, o.local_majorant = 1, 16, 512, 0
            return 0

        def gdrr_set_options(self, handle, ref):
            o = ct.cast(ref, ct.POINTER(gdrr.McOptions)).contents
            written.append({k: getattr(o, k) for k, _ in gdrr.McOptions._fields_})
            return 0

    monkeypatch.setattr(gdrr, "lib", lambda: FakeLib())

    class Ctx:
        handle = None

    gdrr.gdrr_set_options(Ctx(), local_majorant=1)
    gdrr.gdrr_set_options(Ctx(), local_majorant=1, cell_shift=3, batch_min=20)
    gdrr.gdrr_set_options(Ctx(), block_size=256)
    assert (written[0]["local_majorant"], written[0]["cell_shift"], written[0]["batch_min"]) == (1, 0, 0)
    assert (written[1]["cell_shift"], written[1]["batch_min"]) == (3, 20)
    assert (written[2]["cell_shift"], written[2]["batch_min"], written[2]["block_size"]) == (1, 16, 256)
    with pytest.raises(KeyError):
        gdrr.gdrr_set_options(Ctx(), no_such_option=1)
