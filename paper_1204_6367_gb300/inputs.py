"""Seeded synthetic inputs for the gDRR projection problem.

This module only *builds inputs*: voxel phantoms, material attenuation tables,
source spectra, bowtie fluence maps and detector response curves.  It holds none
of the method's arithmetic (no transport, ray tracing, denoising or noise
scaling) and imports nothing else from this package, so both the CUDA path and
the CPU oracle may consume what it returns.

The paper (Section 2.1) defines the inputs of a projection: a voxel phantom with
a material index i(x) and a density rho(x) per voxel, mass attenuation
coefficients mu_hat_k(i, E) for k = Rayleigh, Compton, photoelectric, a detector
response r(E), a source spectrum phi(E) and a fluence map w(u) defined after the
bowtie filter.  The paper's own phantoms, Boone spectra and NIST tables are not
available, so the values here are synthetic stand-ins with the shapes of the
paper's workloads (Section 2.7: SAD 1000 mm, SDD 1500 mm, 512x384 detector at
0.776 mm).

Units: mm, keV, g/cm^3 for density, cm^2/g for mass attenuation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Physical constants (CODATA 2018).
ELECTRON_RADIUS_CM = 2.8179403262e-13
AVOGADRO = 6.02214076e23
ELECTRON_REST_KEV = 510.99895

# Interaction order of the tables, as in the paper's labelling k = 1, 2, 3.
RAYLEIGH, COMPTON, PHOTO = 0, 1, 2


@dataclass(frozen=True)
class Material:
    name: str
    z_eff: float          # effective atomic number for the power laws
    z_over_a: float       # electrons per nucleon (mol e- / g)
    nominal_density: float


AIR = Material("air", 7.64, 0.499, 0.0012)
WATER = Material("water", 7.42, 0.555, 1.0)
BONE = Material("bone", 13.8, 0.530, 1.85)
LUNG = Material("lung", 7.42, 0.555, 0.3)     # water composition, low density
ALUMINIUM = Material("aluminium", 13.0, 0.482, 2.699)


def klein_nishina_sigma_cm2(e_kev: np.ndarray) -> np.ndarray:
    """Total Klein-Nishina cross section per free electron (cm^2)."""
    a = np.asarray(e_kev, dtype=np.float64) / ELECTRON_REST_KEV
    l = np.log1p(2.0 * a)
    term = ((1.0 + a) / a**2) * (2.0 * (1.0 + a) / (1.0 + 2.0 * a) - l / a) \
        + l / (2.0 * a) - (1.0 + 3.0 * a) / (1.0 + 2.0 * a) ** 2
    return 2.0 * math.pi * ELECTRON_RADIUS_CM**2 * term


# Power-law constants chosen so that water at 60 keV has photoelectric 0.01 and
# Rayleigh 0.007 cm^2/g (photo ~ Z^4/E^3, Rayleigh ~ Z^2/E^2 per gram).
_C_PHOTO = 0.01 * 60.0**3 / WATER.z_eff**4
_C_RAYL = 0.007 * 60.0**2 / WATER.z_eff**2


def mass_attenuation(mat: Material, e_kev: np.ndarray) -> np.ndarray:
    """[3, len(e)] table of mu_hat_k(E) in cm^2/g, k = Rayleigh, Compton, photo."""
    e = np.asarray(e_kev, dtype=np.float64)
    out = np.empty((3, e.size))
    out[RAYLEIGH] = _C_RAYL * mat.z_eff**2 / e**2
    out[COMPTON] = klein_nishina_sigma_cm2(e) * AVOGADRO * mat.z_over_a
    out[PHOTO] = _C_PHOTO * mat.z_eff**4 / e**3
    return out


@dataclass
class Problem:
    """One projection problem: everything the paper lists as gDRR input."""
    # geometry (Section 2.1, Fig. 1)
    sad: float
    sdd: float
    theta: float
    nu: int
    nv: int
    du: float
    dv: float
    # voxel phantom: uint8 material [nz, ny, nx] and float32 density
    material: np.ndarray
    density: np.ndarray
    voxel: tuple  # (dx, dy, dz) mm
    # material tables: float32 [n_mat, 3, n_e] cm^2/g on e0 + i*de
    mu_hat: np.ndarray
    e0: float
    de: float
    # spectrum: bin energies (keV) and weights phi (sum 1)
    spec_e: np.ndarray
    spec_w: np.ndarray
    # fluence map after the bowtie, float64 [nv, nu], sum 1
    fluence: np.ndarray
    # detector response: float32 table of deposited keV on r0 + i*dr
    response: np.ndarray
    r0: float
    dr: float
    name: str = ""
    meta: dict = field(default_factory=dict)
    # optional per-detector-column spectra [nu, n_bins] (energy-dependent bowtie
    # hardening); None keeps the separable phi(E) w(u) source of Section 2.1
    spec_cols: np.ndarray | None = None
    # optional Rayleigh form factors F(x) per material [n_mat, n_x] float32 on
    # x_j = j * ff_dx (1/Angstrom, x = sin(theta/2) / lambda)
    form_factor: np.ndarray | None = None
    ff_dx: float = 0.02

    @property
    def shape(self):
        return self.material.shape


ENERGY_GRID = (1.0, 1.0, 150)   # e0 = 1 keV, step 1 keV, 150 nodes up to 150 keV


def material_table(materials) -> np.ndarray:
    e0, de, n = ENERGY_GRID
    e = e0 + de * np.arange(n)
    return np.stack([mass_attenuation(m, e) for m in materials]).astype(np.float32)


FF_GRID = (0.02, 640)   # x_j = j * 0.02 1/Angstrom, j < 640 (to 12.78; 150 keV backscatter is 12.1)


def form_factor(mat: Material, x: np.ndarray) -> np.ndarray:
    """Synthetic coherent form factor F(x): Z_eff (1 + (x/x0)^2)^-2 with
    x0 = 0.45 (Z_eff / 7.42)^(1/3) 1/Angstrom, a hydrogen-like fall-off that
    halves F near x = 0.29 1/Angstrom for water.  Stands in for tabulated
    (Hubbell) form factors, which are not available here."""
    x0 = 0.45 * (mat.z_eff / WATER.z_eff) ** (1.0 / 3.0)
    return mat.z_eff / (1.0 + (np.asarray(x, np.float64) / x0) ** 2) ** 2


def form_factor_table(materials) -> np.ndarray:
    dx, n = FF_GRID
    x = dx * np.arange(n)
    return np.stack([form_factor(m, x) for m in materials]).astype(np.float32)


def response_table(kind: str) -> np.ndarray:
    """Detector response r(E) in keV deposited per incident photon of energy E."""
    e0, de, n = ENERGY_GRID
    e = e0 + de * np.arange(n)
    if kind == "ideal":
        r = e.copy()
    elif kind == "csi":
        k = 100.0**3 * math.log(2.0)          # 50 % absorption at 100 keV
        r = e * (1.0 - np.exp(-k / e**3))
    else:
        raise ValueError(kind)
    return r.astype(np.float32)


def kramers_spectrum(kvp: float = 120.0, al_mm: float = 2.5, e_lo: float = 10.0,
                     bin_kev: float = 1.0):
    """Kramers photon-number spectrum (E_max - E)/E filtered by aluminium.

    Returns bin-centre energies and normalised weights.  Stands in for Boone's
    spectrum model, whose data tables are not available here.
    """
    edges = np.arange(e_lo, kvp + 0.5 * bin_kev, bin_kev)
    e = 0.5 * (edges[:-1] + edges[1:])
    mu_al = mass_attenuation(ALUMINIUM, e).sum(axis=0) * ALUMINIUM.nominal_density
    w = (kvp - e) / e * np.exp(-mu_al * al_mm * 0.1)
    return e, w / w.sum()


def _pixel_offsets(nu, nv, du, dv):
    u = (np.arange(nu) + 0.5 - 0.5 * nu) * du
    v = (np.arange(nv) + 0.5 - 0.5 * nv) * dv
    return np.meshgrid(u, v)   # [nv, nu]


def fluence_map(nu, nv, du, dv, sdd, spec_e=None, spec_w=None, bowtie_mm=0.0):
    """w(u): point-source solid angle per pixel (cos^3) times bowtie transmission.

    The bowtie is aluminium whose thickness grows quadratically with the fan
    angle from 0 at the centre to ``bowtie_mm`` at the detector edge.
    """
    uu, vv = _pixel_offsets(nu, nv, du, dv)
    cos_g = sdd / np.sqrt(sdd**2 + uu**2 + vv**2)
    w = cos_g**3
    if bowtie_mm > 0.0:
        gamma = np.arctan(np.abs(uu) / sdd)
        gmax = math.atan(0.5 * nu * du / sdd)
        t_cm = 0.1 * bowtie_mm * (gamma / gmax) ** 2
        mu_al = mass_attenuation(ALUMINIUM, spec_e).sum(axis=0) * ALUMINIUM.nominal_density
        trans = (spec_w[None, None, :] * np.exp(-mu_al[None, None, :] * t_cm[..., None])).sum(-1)
        w = w * trans
    return w / w.sum()


def bowtie_column_spectra(nu, du, sdd, spec_e, spec_w, bowtie_mm=30.0):
    """Spectrum of each detector column behind the aluminium bowtie: the
    primary spectrum times the transmission of that column's thickness
    (0 at the centre, bowtie_mm at the edge, quadratic in fan angle).
    Rows are the column spectra [nu, n_bins], not normalised."""
    u = (np.arange(nu) + 0.5 - 0.5 * nu) * du
    gamma = np.arctan(np.abs(u) / sdd)
    gmax = math.atan(0.5 * nu * du / sdd)
    t_cm = 0.1 * bowtie_mm * (gamma / gmax) ** 2
    mu_al = mass_attenuation(ALUMINIUM, spec_e).sum(axis=0) * ALUMINIUM.nominal_density
    return spec_w[None, :] * np.exp(-mu_al[None, :] * t_cm[:, None])


def _voxel_centres(n, d):
    return (np.arange(n) + 0.5) * d - 0.5 * n * d


def cylinder_phantom(n=32, vox=4.0, r_water=50.0, r_bone=10.0, bone_x=25.0):
    """Water cylinder (axis z) in air with an off-axis bone rod."""
    c = _voxel_centres(n, vox)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    mat = np.zeros((n, n, n), np.uint8)
    den = np.full((n, n, n), AIR.nominal_density, np.float32)
    water = x**2 + y**2 <= r_water**2
    mat[water] = 1
    den[water] = WATER.nominal_density
    bone = (x - bone_x) ** 2 + y**2 <= r_bone**2
    mat[bone] = 2
    den[bone] = BONE.nominal_density
    return mat, den


def torso_phantom(shape=(128, 256, 256), vox=2.0, seed=1):
    """Seeded ellipsoid torso: water body, bone inclusions, two lungs, in air.

    ``shape`` is (nz, ny, nx).  The same seed gives the same anatomy at any
    voxel size, so the torso can be voxelised at 1, 2 and 4 mm.
    """
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    cz, cy, cx = (_voxel_centres(nz, vox), _voxel_centres(ny, vox), _voxel_centres(nx, vox))
    mat = np.zeros(shape, np.uint8)
    den = np.full(shape, AIR.nominal_density, np.float32)
    zz, yy, xx = np.meshgrid(cz, cy, cx, indexing="ij", sparse=True)

    def ellipsoid(c, r):
        return ((xx - c[0]) / r[0]) ** 2 + ((yy - c[1]) / r[1]) ** 2 + ((zz - c[2]) / r[2]) ** 2 <= 1.0

    body = ellipsoid((0.0, 0.0, 0.0), (170.0, 110.0, 1e9))
    mat[body] = 1
    den[body] = WATER.nominal_density
    for side in (-1.0, 1.0):
        c = (side * rng.uniform(60, 80), rng.uniform(-5, 15), rng.uniform(-20, 20))
        r = (rng.uniform(45, 60), rng.uniform(50, 65), rng.uniform(90, 120))
        lung = ellipsoid(c, r) & body
        mat[lung] = 3
        den[lung] = rng.uniform(0.2, 0.4)
    # spine, sternum and four rib-like arcs
    bones = [((0.0, -80.0 + rng.uniform(-5, 5), 0.0), (16.0, 14.0, 1e9)),
             ((0.0, 95.0, rng.uniform(-30, 30)), (18.0, 6.0, 70.0))]
    for _ in range(4):
        ang = rng.uniform(0.15, 0.45) * math.pi * (1 if rng.random() < 0.5 else -1)
        px, py = 150.0 * math.sin(ang) * 0.93, -100.0 * math.cos(ang) * 0.85
        bones.append(((px, py, rng.uniform(-80, 80)), (rng.uniform(8, 14), rng.uniform(5, 8), rng.uniform(40, 90))))
    for c, r in bones:
        b = ellipsoid(c, r) & body
        mat[b] = 2
        den[b] = rng.uniform(1.4, 1.9)
    return mat, den


def small_problem(n_vox=32, vox=4.0, n_det=64, det_px=4.0, energy=60.0, name="cylinder-32"):
    """32^3 water cylinder with bone rod, mono-energetic 60 keV point source,
    64x64 detector of 4 mm pixels, ideal energy-integrating response."""
    mat, den = cylinder_phantom(n_vox, vox)
    sdd = 1500.0
    return Problem(
        sad=1000.0, sdd=sdd, theta=0.0, nu=n_det, nv=n_det, du=det_px, dv=det_px,
        material=mat, density=den, voxel=(vox, vox, vox),
        mu_hat=material_table([AIR, WATER, BONE]), e0=ENERGY_GRID[0], de=ENERGY_GRID[1],
        form_factor=form_factor_table([AIR, WATER, BONE]), ff_dx=FF_GRID[0],
        spec_e=np.array([energy]), spec_w=np.array([1.0]),
        fluence=fluence_map(n_det, n_det, det_px, det_px, sdd),
        response=response_table("ideal"), r0=ENERGY_GRID[0], dr=ENERGY_GRID[1],
        name=name)


def torso_problem(vox=2.0, seed=1, kvp=120.0, nu=512, nv=384, det_px=0.776, bowtie_mm=30.0,
                  name=None, hardened_bowtie=False):
    """Ellipsoid torso at ``vox`` mm (256x256x128 at 2 mm), 120 kVp Kramers
    spectrum with 2.5 mm Al, aluminium bowtie 0-30 mm, 512x384 detector of
    0.776 mm pixels, CsI-like response."""
    extent = (256.0, 512.0, 512.0)
    shape = tuple(int(round(e / vox)) for e in extent)
    mat, den = torso_phantom(shape, vox, seed)
    spec_e, spec_w = kramers_spectrum(kvp)
    sdd = 1500.0
    return Problem(
        sad=1000.0, sdd=sdd, theta=0.0, nu=nu, nv=nv, du=det_px, dv=det_px,
        material=mat, density=den, voxel=(vox, vox, vox),
        mu_hat=material_table([AIR, WATER, BONE, LUNG]), e0=ENERGY_GRID[0], de=ENERGY_GRID[1],
        form_factor=form_factor_table([AIR, WATER, BONE, LUNG]), ff_dx=FF_GRID[0],
        spec_e=spec_e, spec_w=spec_w,
        fluence=fluence_map(nu, nv, det_px, det_px, sdd, spec_e, spec_w, bowtie_mm),
        response=response_table("csi"), r0=ENERGY_GRID[0], dr=ENERGY_GRID[1],
        name=name or f"torso-{shape[2]}x{shape[1]}x{shape[0]}-{vox:g}mm",
        spec_cols=bowtie_column_spectra(nu, det_px, sdd, spec_e, spec_w, bowtie_mm) if hardened_bowtie else None)


def uniform_slab_problem(nx=16, ny=16, nz=16, vox=2.0, mat_id=1, density=1.0, energy=60.0,
                         nu=8, nv=8, det_px=1.0, materials=None, pencil=True, sad=1000.0, sdd=1500.0):
    """A homogeneous box phantom with a narrow (single-pixel) beam: the
    textbook narrow-beam transmission geometry."""
    mats = materials if materials is not None else [AIR, WATER, BONE]
    mat = np.full((nz, ny, nx), mat_id, np.uint8)
    den = np.full((nz, ny, nx), density, np.float32)
    flu = np.zeros((nv, nu))
    if pencil:
        flu[nv // 2, nu // 2] = 1.0
    else:
        flu[:] = 1.0 / flu.size
    return Problem(
        sad=sad, sdd=sdd, theta=0.0, nu=nu, nv=nv, du=det_px, dv=det_px,
        material=mat, density=den, voxel=(vox, vox, vox),
        mu_hat=material_table(mats), e0=ENERGY_GRID[0], de=ENERGY_GRID[1],
        form_factor=form_factor_table(mats), ff_dx=FF_GRID[0],
        spec_e=np.array([energy]), spec_w=np.array([1.0]), fluence=flu,
        response=response_table("ideal"), r0=ENERGY_GRID[0], dr=ENERGY_GRID[1],
        name="slab")


def batched_budgets(n_angles=64, lo=1e7, hi=5e7, seed=1):
    """Per-angle history budgets drawn uniformly from [lo, hi] and angles
    spread uniformly over 360 degrees (the multi-angle scan workload)."""
    rng = np.random.default_rng(seed)
    budgets = rng.uniform(lo, hi, n_angles).astype(np.uint64)
    angles = np.arange(n_angles) * (2.0 * math.pi / n_angles)
    return angles, budgets
