/*
 * gdrr.h -- C ABI of the GB300 gDRR projection library (libgdrr.so).
 *
 * gDRR (Jia et al., arXiv:1204.6367) computes a cone-beam CT projection as
 * primary P(u), scatter S(u) and noise N(u) (Section 2.2, Fig. 3):
 *   Step 1  ray-traced primary                      gdrr_raytrace_primary
 *   Step 2  Monte Carlo primary and scatter tallies  gdrr_mc_project[_batched]
 *           and their conversion to signal           gdrr_finalize
 *   Step 3  Poisson denoising of the scatter         gdrr_denoise_scatter
 *   Step 4  noise N = alpha (N_P + N_S), zeta fit    gdrr_noise_calibrate, gdrr_fit_zeta
 *
 * Conventions for every call:
 *  - Units: lengths mm, energies keV, density g/cm^3, mass attenuation cm^2/g.
 *  - Host input structs and arrays are borrowed for the duration of the call
 *    and deep-copied by gdrr_create; the caller may free them afterwards.
 *  - Pointers named *_dev are device pointers owned by the caller (for example
 *    torch tensors); every kernel runs on the context's stream and the call
 *    returns without synchronising unless stated.  Results are valid after the
 *    stream is synchronised (gdrr_sync does that and reports kernel errors).
 *  - Images are row-major [nv][nu] (u fastest).  The phantom is x-fastest:
 *    index = x + nx * (y + ny * z), box centred on the isocentre.
 *  - Return value: GDRR_OK (0) or a negative GDRR_ERR_* code; no call throws.
 *    A context is not thread-safe; use one context per host thread.
 */
#ifndef GDRR_H
#define GDRR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GDRR_API __attribute__((visibility("default")))
#else
#define GDRR_API
#endif

enum {
    GDRR_OK = 0,
    GDRR_ERR_INVALID_ARG = -1,   /* a size, pointer or value is out of range      */
    GDRR_ERR_CUDA = -2,          /* a CUDA runtime call failed                     */
    GDRR_ERR_OOM = -3,           /* device allocation failed                       */
    GDRR_ERR_TALLY_OVERFLOW = -4,/* an int64 tally would exceed its headroom       */
    GDRR_ERR_STEP_LIMIT = -5,    /* histories hit the free-flight limit            */
    GDRR_ERR_UNSUPPORTED = -6,   /* valid input this build does not handle         */
    GDRR_ERR_TIMEOUT = -7        /* a bounded device-side wait gave up             */
};

/* How the two run-time conditions reach the caller.
 *  - GDRR_ERR_STEP_LIMIT: a history that reaches gdrr_mc_options.max_steps
 *    free flights is dropped and counted in stats[GDRR_ST_STEP_LIMIT].  The
 *    asynchronous transport calls (gdrr_mc_project, _batched, scans) return
 *    before the kernel runs, so they report it only through that counter;
 *    gdrr_project, which synchronises, returns GDRR_ERR_STEP_LIMIT when the
 *    counter of its projection is non-zero (its outputs are still written).
 *  - GDRR_ERR_TIMEOUT: kernels that wait on other CTAs or on the tensor-core
 *    pipeline bound every wait (about a second) and then record a timeout
 *    instead of spinning on.  Synchronising calls (gdrr_project,
 *    gdrr_gemm_bf16, the learned estimator's backward) return it directly;
 *    for asynchronous calls on a context the next gdrr_sync returns it (and
 *    clears the record).  The context stays usable; the outputs of the call
 *    that timed out are not defined. */

/* Maximum number of materials the transport kernels handle. */
#define GDRR_MAX_MATERIALS 8
/* Fixed-point tally unit: 2^-GDRR_TALLY_BITS keV per count. */
#define GDRR_TALLY_BITS 24

typedef struct gdrr_ctx gdrr_ctx;

/* Scanner geometry, Section 2.1 / Fig. 1: the source rotates in the xOy plane
 * at distance sad_mm from the isocentre O, at angle phi between SO and +x; the
 * imager is perpendicular to xOy and to OP, at AID = sdd_mm - sad_mm from O,
 * with theta_rad the angle between SO and OP (0: opposite the source).  The
 * detector frame (u, v) has its origin at P, v parallel to z, u = OP x z
 * normalised; nu x nv pixels of du_mm x dv_mm centred on P. */
typedef struct {
    double sad_mm, sdd_mm, theta_rad;
    int32_t nu, nv;
    double du_mm, dv_mm;
} gdrr_geometry;

/* Voxel phantom, Section 2.1: a material index i(x) and a density rho(x) per
 * voxel.  Densities must be finite and >= 0; indices < n_materials. */
typedef struct {
    int32_t nx, ny, nz;
    double dx_mm, dy_mm, dz_mm;
    const uint8_t* material;   /* host, nx*ny*nz */
    const float* density;      /* host, nx*ny*nz, g/cm^3 */
} gdrr_phantom;

/* Mass attenuation mu_hat_k(i, E) of each material, Section 2.1, for
 * k = 0 Rayleigh, 1 Compton, 2 photoelectric, tabulated on the energy grid
 * e0_kev + j * de_kev, j < n_energies (linear interpolation between nodes).
 * Layout [n_materials][3][n_energies], cm^2/g, host. */
typedef struct {
    int32_t n_materials, n_energies;
    double e0_kev, de_kev;
    const float* mu_hat;
} gdrr_materials;

/* Source spectrum phi(E) after the bowtie, Section 2.1: n_bins energy
 * channels (keV) and non-negative weights (normalised by the library).
 * column_weight (host, may be NULL) makes the spectrum depend on the detector
 * column, as behind a bowtie that hardens the beam off axis: [nu][n_bins]
 * non-negative weights, each column normalised by the library and each with a
 * positive sum; the photon heading for pixel (iu, iv) then draws its energy
 * from column iu, and the ray tracer weights pixel (iu, iv) by that column's
 * spectrum.  With NULL, weight serves every column (the separable source). */
typedef struct {
    int32_t n_bins;
    const double* energy_kev;
    const double* weight;
    const double* column_weight;
} gdrr_spectrum;

/* Photon fluence map w(u) after the bowtie, Section 2.1: the probability of
 * a source photon heading for each detector pixel, [nv][nu], non-negative,
 * normalised by the library. */
typedef struct {
    const double* fluence;
} gdrr_bowtie;

/* Detector response r(E), Section 2.1: energy (keV) recorded for an incoming
 * photon of energy E, tabulated on r0_kev + j * dr_kev (linear interpolation). */
typedef struct {
    int32_t n_energies;
    double e0_kev, de_kev;
    const float* response;
} gdrr_detector;

/* Transport options (defaults in brackets).  Zero means "default". */
typedef struct {
    double e_cut_kev;          /* absorb photons below this energy [1.0]           */
    int32_t max_steps;         /* free flights per history before giving up [1e5]  */
    int32_t block_size;        /* threads per block, multiple of 32, <= 512 [256]   */
    int32_t blocks_per_sm;     /* resident blocks per SM for the persistent grid [by occupancy] */
    int32_t hist_per_thread;   /* histories a warp claims per lane at a time [8]    */
    int32_t batch_min;         /* lanes of a warp that must be waiting for an
                                  interaction, a tally or a new history before the
                                  warp serves them together, 1..32 [16; 24 with
                                  local_majorant, whose short flights bring the
                                  services more often]                              */
    int32_t nearest_voxel;     /* 1: no density interpolation, each point takes its
                                  voxel's density and material (the speed variant of
                                  the paper's appendix); 0: trilinear [0]           */
    int32_t scatter_filter;    /* scattered photons the scatter counter takes
                                  (Section 2.4): 0 all, 1 exactly one Compton and no
                                  Rayleigh, 2 exactly one Rayleigh and no Compton,
                                  3 two or more interactions; the others count as
                                  missing the detector [0]                           */
    int32_t rayleigh_form_factor; /* 1: Rayleigh polar angle from (1 + cos^2) F^2(x)
                                  with the form factors set by gdrr_set_form_factor
                                  (the material picked among the interaction point's
                                  corner voxels in proportion to their Rayleigh
                                  coefficient); 0: Thomson (1 + cos^2), the paper's
                                  default reading [0]                                 */
    int32_t cell_shift;        /* macro cells of 2^cell_shift voxels per edge, 1..6;
                                  -1: none; [0: cells of about 4 mm, cell_shift =
                                  round(log2(4 mm / smallest voxel edge)) in 1..6].
                                  Before gathering the eight corner voxels of
                                  a tentative collision, the transport compares it with
                                  a bound on mu over the macro cell that holds the
                                  corners (the largest density of each material there
                                  times the material's coefficient, raised by 2^-10
                                  against rounding); a tentative collision above it is
                                  virtual without the gathers.  The bound is never below
                                  the mu the gathers would give, so with the global
                                  majorant tallies, counters and records are the same
                                  for every cell_shift; only GDRR_ST_CELL_SKIPS and the
                                  time change.  With local_majorant the cells are the
                                  majorant itself, and the draws depend on their size.
                                  Changing it rebuilds the cell table (not while a scan
                                  exists).                                              */
    int32_t photon_pool;       /* photons per thread, 1..3, in the shared-memory pool
                                  of the pool form of the transport: blocks of 256
                                  threads move photons between warps so that free
                                  flights, corner gathers, interactions, tallies and
                                  new histories each run on full warps (block_size and
                                  batch_min do not apply to it); -1: the lane form, one
                                  photon per lane with warp-batched services.  Runs
                                  with records, nearest_voxel, scatter_filter,
                                  rayleigh_form_factor or local_majorant always take
                                  the lane form.  Tallies, counters and records are
                                  the same for every choice.  On the 2 mm torso the
                                  pool form ran at 125-158 ms per 1e8 histories
                                  against 75 ms for the lane form, so the lane form is
                                  the default and the autotuner times both [-1]       */
    int32_t local_majorant;    /* 1: delta tracking with local majorants, an option
                                  beside the paper's global Woodcock majorant: the
                                  macro-cell bounds (cell_shift, which must not be -1)
                                  serve as a piecewise-constant majorant, and each free
                                  flight spends its optical depth -ln xi cell by cell
                                  along the ray; a tentative collision is real with
                                  probability mu / (its cell's bound).  The expected
                                  images are those of the global majorant; the draws,
                                  and so the per-history results, differ.  With
                                  cell_shift 0 the cells are then about 32 mm
                                  (round(log2(32 mm / smallest voxel edge)) in 1..6).
                                  On the 2 mm torso it ran at 64 ms per 1e8 histories
                                  (batch_min 24) against 75 ms for the global
                                  majorant: 6.5 flights and 11.5 cell crossings per
                                  history instead of 46 flights.
                                  Runs the lane form; GDRR_ST_CELL_CROSSINGS counts the
                                  cell crossings; 0: the global majorant [0]           */
} gdrr_mc_options;

/* Transport counters, accumulated by every gdrr_mc_project* call (device
 * array of GDRR_NSTATS uint64 in this order).  The first eleven count events
 * of the method (GDRR_ST_STEPS: free flights); GDRR_ST_CELL_SKIPS counts the
 * virtual collisions (included in GDRR_ST_VIRTUAL) that the macro-cell bound
 * decided without gathering corner voxels (see gdrr_mc_options.cell_shift;
 * global majorant only); GDRR_ST_CELL_CROSSINGS the macro-cell crossings of
 * the free flights with local majorants (gdrr_mc_options.local_majorant). */
enum {
    GDRR_ST_HISTORIES = 0, GDRR_ST_STEPS, GDRR_ST_VIRTUAL, GDRR_ST_RAYLEIGH, GDRR_ST_COMPTON,
    GDRR_ST_PHOTO, GDRR_ST_TALLY_PRIMARY, GDRR_ST_TALLY_SCATTER, GDRR_ST_MISS, GDRR_ST_CUTOFF,
    GDRR_ST_STEP_LIMIT, GDRR_ST_CELL_SKIPS, GDRR_ST_CELL_CROSSINGS, GDRR_NSTATS
};

/* Per-history event record (tiny parity runs only). outcome: 0 primary tally,
 * 1 scatter tally, 2 photoelectric absorption, 3 energy cut-off, 4 missed the
 * detector, 5 step limit.  first_interaction: 0 none, 1 Rayleigh, 2 Compton,
 * 3 photoelectric.  rng_blocks: Philox blocks the history consumed. */
typedef struct {
    uint32_t n_steps, n_virtual, n_rayleigh, n_compton;
    uint32_t n_photo, outcome, rng_blocks, first_interaction;
    int32_t pixel;
    float e_source, e_final;
    uint32_t ray_material;   /* material of the last form-factor Rayleigh event, else 0 */
    double e_deposited;
} gdrr_history_record;

/* Create a context: validates and deep-copies the inputs, stages the phantom
 * and tables on the current CUDA device, and binds cuda_stream (a
 * cudaStream_t; NULL = the legacy default stream) to every later call.
 * Fails with GDRR_ERR_INVALID_ARG when an input is inconsistent (sizes,
 * negative weights, material index out of range, imager plane cutting the
 * phantom box), GDRR_ERR_UNSUPPORTED for more than GDRR_MAX_MATERIALS
 * materials.  *out is set only on success.  Follows Section 2.1 (inputs) and
 * Section 4 (the package takes phantom, geometry, source and detector). */
GDRR_API int gdrr_create(const gdrr_geometry* geometry, const gdrr_phantom* phantom,
                         const gdrr_materials* materials, const gdrr_spectrum* spectrum,
                         const gdrr_bowtie* bowtie, const gdrr_detector* detector,
                         void* cuda_stream, gdrr_ctx** out);

/* Release every device buffer of the context (synchronises its stream).
 * A context's device buffers come from one stream-ordered memory pool per
 * device that keeps the blocks of destroyed contexts for the next ones (a
 * context of the 2 mm torso holds about 3.4 GB after a 1e8-history
 * projection, 3.2 GB of it source records); gdrr_release_memory hands them
 * back. */
GDRR_API void gdrr_destroy(gdrr_ctx* ctx);

/* Return the unused blocks of the contexts' device memory pools (on every
 * device), and the page-locked host staging blocks kept for reuse, to the
 * driver; memory of live contexts stays.  GDRR_ERR_CUDA if a pool cannot be
 * trimmed or a host block freed. */
GDRR_API int gdrr_release_memory(void);

/* Static description of an error code. */
GDRR_API const char* gdrr_error_string(int code);

/* Set / read transport options; invalid values give GDRR_ERR_INVALID_ARG. */
GDRR_API int gdrr_set_options(gdrr_ctx* ctx, const gdrr_mc_options* options);
GDRR_API int gdrr_get_options(const gdrr_ctx* ctx, gdrr_mc_options* options);

/* Synchronise the context stream; returns GDRR_ERR_CUDA on a kernel fault
 * or a failed self-check of the transport's photon bookkeeping,
 * GDRR_ERR_TIMEOUT when a bounded device-side wait of an earlier call on the
 * context gave up since the last gdrr_sync. */
GDRR_API int gdrr_sync(gdrr_ctx* ctx);

/* Step 1, Section 2.3, Eq. 1: P(u) = w(u) sum_E phi(E) r(E) exp(-int mu dl)
 * for the ray from the source to each pixel centre at gantry angle
 * angle_rad.  The ray inside the phantom box is cut into equal intervals no
 * longer than half the smallest voxel size, mu taken at interval midpoints
 * with the trilinear field.  P_dev: caller-owned device double[nv*nu],
 * overwritten, per source photon (keV). */
GDRR_API int gdrr_raytrace_primary(gdrr_ctx* ctx, double angle_rad, double* P_dev);

/* Step 1 with Siddon's algorithm (the paper's faster alternative, Section
 * 2.3 and appendix): exact path lengths through the piecewise-constant voxel
 * field (each voxel's own density and material) along the ray to each pixel
 * centre.  P_dev as for gdrr_raytrace_primary. */
GDRR_API int gdrr_raytrace_primary_siddon(gdrr_ctx* ctx, double angle_rad, double* P_dev);

/* Step 2, Section 2.4: transport n_photons source photons with Woodcock
 * tracking, photoelectric / Compton (Klein-Nishina) / Rayleigh (Thomson)
 * interactions, and tally r(E) at the detector pixel each escaping photon
 * hits, into the primary counter when it never scattered, else the scatter
 * counter.  History h (h = history_offset .. history_offset + n_photons - 1)
 * draws from Philox4x32-10 with key = seed, counter = (block, angle_index,
 * h lo, h hi), so any split of the history range sums to the same tallies.
 * prim_dev / scat_dev: caller-owned device int64[nv*nu], ACCUMULATED (not
 * cleared) in units of 2^-24 keV.  stats_dev: NULL or device
 * uint64[GDRR_NSTATS], accumulated.  records_dev: NULL or device
 * gdrr_history_record[n_photons], written (debug / parity use; slower).
 * With default options and no records, the source points, directions and
 * energies are first sampled by a separate full-warp pass into a workspace
 * the context owns (32 bytes per history, at most 2^27 histories per pass,
 * allocated on first use; a scan keeps its own); the arithmetic is the same,
 * and when the workspace cannot be allocated the transport samples them
 * itself, with the same results. */
GDRR_API int gdrr_mc_project(gdrr_ctx* ctx, double angle_rad, uint32_t angle_index,
                             uint64_t n_photons, uint64_t seed, uint64_t history_offset,
                             int64_t* prim_dev, int64_t* scat_dev, uint64_t* stats_dev,
                             gdrr_history_record* records_dev);

/* Step 2 for a multi-angle scan in one persistent launch: angle a
 * (a < n_angles) at angles_rad[a] (host) transports budgets[a] (host)
 * histories with angle_index = a and history ids 0 .. budgets[a]-1, so each
 * angle's tallies equal gdrr_mc_project(angle_index = a, history_offset = 0).
 * prim_dev / scat_dev: device int64[n_angles][nv*nu], accumulated.
 * stats_dev: NULL or device uint64[GDRR_NSTATS], accumulated over angles. */
GDRR_API int gdrr_mc_project_batched(gdrr_ctx* ctx, int32_t n_angles, const double* angles_rad,
                                     const uint64_t* budgets, uint64_t seed, int64_t* prim_dev,
                                     int64_t* scat_dev, uint64_t* stats_dev);

/* A multi-angle scan captured once as a CUDA graph and replayed by
 * gdrr_scan_launch: each replay runs the same work as
 * gdrr_mc_project_batched(angles_rad, budgets, seed) in one persistent launch
 * (work counter reset + transport kernel), preceded by zeroing prim_dev /
 * scat_dev when zero_tallies != 0 (else replays accumulate).  The job table,
 * launch configuration (the context's options at creation) and buffers are
 * fixed at creation; prim_dev / scat_dev / stats_dev (device, caller-owned,
 * as for the batched call; stats_dev may be NULL) must outlive the scan.
 * Creation allocates the job table and counters and synchronises. */
typedef struct gdrr_scan gdrr_scan;
GDRR_API int gdrr_scan_create(gdrr_ctx* ctx, int32_t n_angles, const double* angles_rad, const uint64_t* budgets,
                              uint64_t seed, int64_t* prim_dev, int64_t* scat_dev, uint64_t* stats_dev,
                              int32_t zero_tallies, gdrr_scan** out);
/* Enqueue one replay of the scan on its context's stream. */
GDRR_API int gdrr_scan_launch(gdrr_scan* scan);
/* Release the scan (synchronises its context's stream). */
GDRR_API void gdrr_scan_destroy(gdrr_scan* scan);

/* Coherent (Rayleigh) form factors F(x, i) of each material, for the
 * rayleigh_form_factor option: tabulated on x_j = j * dx_inv_angstrom,
 * j < n_x, with x = sin(theta/2) / lambda in 1/Angstrom; layout
 * [n_materials][n_x], host, finite, >= 0, F(0) > 0.  The grid must reach the
 * backscatter momentum transfer E_max / hc of the largest energy of the
 * material tables (hc = 12.398419843320026 keV Angstrom).  The library builds
 * the cumulative of F^2 over x^2 (trapezoid sums, F^2 linear in x^2 between
 * nodes) per material; the draw of x^2 inverts it exactly.  A second call
 * replaces the tables; form_factor == NULL removes them (and is refused while
 * the option is on).  Synchronises the context's stream. */
typedef struct {
    int32_t n_x;
    double dx_inv_angstrom;
    const float* form_factor;
} gdrr_form_factor;
GDRR_API int gdrr_set_form_factor(gdrr_ctx* ctx, const gdrr_form_factor* ff);

/* ---- Reconstruction of simulated scans (Section 3.5) ---------------------- */

/* The unattenuated signal I0 of every pixel (an air scan): w(u) times the
 * response-weighted spectrum sum_b phi_u(b) r(E_b), per source photon, the
 * signal gdrr_raytrace_primary gives for an empty phantom.  FP64 device
 * [nv][nu], caller-owned.  Asynchronous on the context stream. */
GDRR_API int gdrr_air_scan(gdrr_ctx* ctx, double* I0_dev);

/* Line integrals g = -ln(max(I, floor_rel I0) / I0) of n pixels: signal and
 * air scan FP64 device arrays, out FP32 device; 0 < floor_rel < 1 keeps the
 * logarithm finite where the signal is zero or negative (noise).  No
 * context; asynchronous on cuda_stream (a cudaStream_t, NULL = legacy). */
GDRR_API int gdrr_line_integrals(const double* signal_dev, const double* air_dev, int64_t n, double floor_rel,
                                 float* out_dev, void* cuda_stream);

/* Geometry of an FDK reconstruction: the circular orbit of Section 2.1
 * (source at sad_mm from the isocentre, imager at sdd_mm from the source,
 * opposite it: theta = 0), the detector grid, and the output voxel grid of
 * nx x ny x nz voxels of dx x dy x dz mm centred on the isocentre. */
typedef struct {
    double sad_mm, sdd_mm;
    int32_t nu, nv;
    double du_mm, dv_mm;
    int32_t nx, ny, nz;
    double dx_mm, dy_mm, dz_mm;
} gdrr_fdk_geometry;

/* FDK step 1 (Feldkamp, Davis & Kress 1984; Kak & Slaney's equally spaced
 * fan-beam form): on the virtual detector at the isocentre (spacing
 * tau = du SAD / SDD), weight each line integral by SAD / sqrt(SAD^2 + a^2 +
 * b^2) and convolve each row with the Ram-Lak kernel (h(0) = 1 / (4 tau^2),
 * h(odd n) = -1 / (n pi tau)^2, 0 otherwise) times tau / 2, zeros outside
 * the row.  proj_dev and filtered_dev: FP32 device [n_proj][nv][nu] (may not
 * alias).  nu <= 4096 (GDRR_ERR_UNSUPPORTED beyond).  No context;
 * asynchronous on cuda_stream. */
GDRR_API int gdrr_fdk_filter(const gdrr_fdk_geometry* geometry, int32_t n_proj, const float* proj_dev,
                             float* filtered_dev, void* cuda_stream);

/* FDK step 2: voxel-driven backprojection f(x) = sum_views d_beta
 * (SAD / (SAD + x.n))^2 Qf(a(x), b(x)) of the filtered views taken at the
 * gantry angles angles_rad (host, n_proj values; n = (cos phi, sin phi, 0)
 * points from the source through the isocentre), bilinear on the pixel-centre
 * grid with zeros outside the detector.  d_beta is the angular weight of one
 * view (2 pi / n_proj for a full scan of equally spaced views).  volume_dev:
 * FP32 device [nz][ny][nx], attenuation in 1/mm; accumulate = 1 adds to it
 * (so views may come in batches), 0 overwrites it.  The grid must keep every
 * voxel between the source and the isocentre plane's far side at every angle
 * (half-diagonal of the x-y extent < sad_mm), else GDRR_ERR_INVALID_ARG.  No
 * context; asynchronous on cuda_stream. */
GDRR_API int gdrr_fdk_backproject(const gdrr_fdk_geometry* geometry, int32_t n_proj, const double* angles_rad,
                                  double d_beta, const float* filtered_dev, float* volume_dev, int32_t accumulate,
                                  void* cuda_stream);

/* Roofline probes (machine ceilings, not part of the method).
 * gdrr_probe_l2_gather: 8-byte loads at pseudo-random indices over a
 * working set of the largest power of two <= working_set_bytes (1 MiB ...
 * 4 GiB; 32 MiB fits in L2), *gbs_out = GB/s of 8-byte words.
 * gdrr_probe_fp32: independent FMA chains, *tflops_out = FP32 TFLOP/s (two
 * flops per FMA).  Both allocate their buffers, run one warm-up and one timed
 * launch on cuda_stream, and synchronise. */
GDRR_API int gdrr_probe_l2_gather(int64_t working_set_bytes, double* gbs_out, void* cuda_stream);
GDRR_API int gdrr_probe_fp32(double* tflops_out, void* cuda_stream);

/* Check of the bounded device-side wait (not part of the method): one CTA
 * waits, with the same bounded wait the denoiser's row bands use, for a flag
 * that nothing sets.  The wait gives up after limit_ns nanoseconds (1 ..
 * 2e9) and the call returns GDRR_ERR_TIMEOUT; GDRR_OK would mean the flag was
 * seen.  Allocates 16 bytes, runs on cuda_stream, synchronises. */
GDRR_API int gdrr_probe_bounded_wait(uint64_t limit_ns, void* cuda_stream);

/* Autotuner: time gdrr_mc_project of n_probe histories at angle_rad for each
 * launch configuration of a fixed grid (the lane form: block size 64 / 128 /
 * 256 / 512, batch_min 8 .. 32, hist_per_thread 1 / 8 / 64; the pool form:
 * photon_pool 1 / 2 / 3, hist_per_thread 1 / 8 / 64), into scratch tallies, and
 * keep the fastest as the context's options (also copied to *best_out when
 * not NULL).  Tallies do not depend on these options, only the speed does.
 * Synchronises. */
GDRR_API int gdrr_autotune(gdrr_ctx* ctx, double angle_rad, uint64_t n_probe, uint64_t seed,
                           gdrr_mc_options* best_out);

/* Tally -> signal per source photon in FP64 (Section 2.6: MC results are
 * normalised by the number of source photons): out = tally * 2^-24 / n_photons.
 * n elements; tally_dev int64, signal_dev double, both caller-owned device.
 * Fails with GDRR_ERR_TALLY_OVERFLOW (after a stream sync) if any tally is
 * negative, which only an int64 wrap-around can produce. */
GDRR_API int gdrr_finalize(gdrr_ctx* ctx, const int64_t* tally_dev, int64_t n,
                           uint64_t n_photons, double* signal_dev);

/* Exact integer factor x factor binning of a [nv][nu] int64 tally to
 * [nv/factor][nu/factor] (the coarse scatter grid); nu, nv multiples of factor. */
GDRR_API int gdrr_bin_tally(gdrr_ctx* ctx, const int64_t* tally_dev, int32_t nu, int32_t nv,
                            int32_t factor, int64_t* out_dev);

/* Bilinear interpolation of a coarse [cv][cu] image (a factor x factor binned
 * sum) to the fine [cv*factor][cu*factor] grid, divided by factor^2.  Coarse
 * pixel centres sit at fine coordinate (I + 1/2) factor - 1/2; edges clamp. */
GDRR_API int gdrr_upsample(gdrr_ctx* ctx, const double* coarse_dev, int32_t cu, int32_t cv,
                           int32_t factor, double* fine_dev);

/* Step 3, Section 2.5, Eq. 2-5: denoise a Poisson-noisy scatter image by
 *   S <- (1 - omega) S + omega/4 [Sigma S - (1/beta)(1 - S^/S)]
 * for iters iterations from S = max(S^, eps), every term using the previous
 * iterate, replicate edges, S kept >= eps = 1e-3 counts.  The iteration runs
 * on the count scale: S^ / count_scale (count_scale > 0 is the signal of one
 * detected photon); the result is returned on the input scale.  The paper uses
 * omega = 0.8.  Linearised at its fixed point the iteration converges while
 * beta * S > omega / (8 (1 - omega)) in counts (0.5 at omega = 0.8; a
 * checkerboard is the first pattern to grow below it), and for no beta when
 * omega >= 1.  Below that floor the result oscillates and is not the Eq. 4
 * solution; no error is returned.  S_hat_dev, S_dev: caller-owned device
 * double[nv*nu]. */
GDRR_API int gdrr_denoise_scatter(gdrr_ctx* ctx, const double* S_hat_dev, double* S_dev,
                                  int32_t nu, int32_t nv, double count_scale, double beta,
                                  double omega, int32_t iters);

/* Largest image, in pixels, that gdrr_denoise_scatter_static accepts. */
#define GDRR_STATIC_DENOISE_MAX_PIXELS 65536

/* The scatter denoiser of gdrr_denoise_scatter without a context and without
 * allocating device memory, for callers that cannot allocate: a plug-in
 * given a fixed device-memory budget by its host application, or code that
 * must not call cudaMalloc / cudaFree because they can synchronise the
 * device.  The paper has no counterpart; it computes exactly what
 * gdrr_denoise_scatter computes, with the same arguments.
 *  - Scratch: a file-scope device array of 2 * GDRR_STATIC_DENOISE_MAX_PIXELS
 *    doubles (1 MiB) that every GPU loading the library holds until exit.
 *    Images with nu * nv > GDRR_STATIC_DENOISE_MAX_PIXELS are rejected with
 *    GDRR_ERR_INVALID_ARG.
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any
 *    stream capture.  The address is kept for the life of the process: after
 *    cudaDeviceReset on a device (or a release and re-creation of its primary
 *    context) the array may move, so do not call this entry point on that
 *    device again in the same process.
 *  - Every call on a device shares the one array, and the array keeps the
 *    last call's contents (each call writes every element it reads before
 *    reading it, so nothing needs clearing).  Calls that overlap on the GPU
 *    (on different streams, or from different host threads) race on it and
 *    must be ordered by the caller.
 *  - Runs on cuda_stream (a cudaStream_t, NULL = legacy default stream) on the
 *    current device; returns without synchronising.  S_hat_dev, S_dev:
 *    caller-owned device double[nv * nu]. */
GDRR_API int gdrr_denoise_scatter_static(const double* S_hat_dev, double* S_dev, int32_t nu, int32_t nv,
                                         double count_scale, double beta, double omega, int32_t iters,
                                         void* cuda_stream);

/* ---- One whole projection: Steps 1-4 of Section 2.2 / Fig. 3 -------------- */

/* What gdrr_project simulates.  beta and smoothing_px choose the Eq. 2
 * regularisation weight: with smoothing_px > 0, beta = smoothing_px^2 /
 * (mean scatter count per coarse pixel), a smoothing length in coarse pixels
 * that keeps the Eq. 5 iteration convergent at any photon count (see
 * gdrr_denoise_scatter); otherwise beta (counts^-1) is used as given. */
typedef struct {
    double angle_rad;        /* gantry angle phi                                   */
    uint32_t angle_index;    /* Philox counter word of this projection's streams   */
    uint64_t n_photons;      /* source photons n_sim, > 0                          */
    uint64_t seed;           /* Philox key                                         */
    int32_t bin_factor;      /* coarse scatter grid of bin_factor^2 pixels; nu and
                                nv multiples of it                                  */
    double beta;             /* Eq. 2 weight in counts^-1 when smoothing_px <= 0   */
    double smoothing_px;     /* > 0: beta from the mean coarse count (see above)   */
    double omega;            /* Eq. 5 relaxation, 0 < omega < 2 (paper: 0.8)       */
    int32_t iters;           /* Eq. 5 iterations, >= 0                             */
    double mAs;              /* exposure I of the noise scaling, > 0               */
    double zeta;             /* photons per mAs of the noise scaling, > 0          */
} gdrr_projection;

/* Caller-owned device outputs of gdrr_project, all overwritten.  Required:
 * P, P_hat, S_hat, S, N (FP64 [nv][nu]).  Optional (NULL: not returned; the
 * context keeps its own scratch instead): S_hat_coarse and S_coarse (FP64
 * [nv/f][nu/f], f = bin_factor), prim_tally and scat_tally (int64 [nv][nu],
 * the projection's fixed-point tallies), stats (uint64[GDRR_NSTATS], this
 * projection's counters; zeroed by the call, not accumulated). */
typedef struct {
    double* P;
    double* P_hat;
    double* S_hat;
    double* S;
    double* N;
    double* S_hat_coarse;
    double* S_coarse;
    int64_t* prim_tally;
    int64_t* scat_tally;
    uint64_t* stats;
} gdrr_projection_out;

/* Scalars gdrr_project derived on the device, copied to the host at its end. */
typedef struct {
    double count_scale;      /* signal of one detected scattered photon: scatter
                                tally sum / scattered photons tallied (1/n_photons
                                when none was tallied)                              */
    double beta;             /* the Eq. 2 weight the denoiser used                 */
    double mean_count;       /* scattered photons tallied per coarse pixel (>= 1
                                photon in total)                                    */
    uint64_t tally_scatter;  /* scattered photons tallied                          */
    uint64_t step_limit;     /* histories dropped at max_steps                     */
    int32_t below_floor;     /* 1: beta * mean_count < omega / (8 (1 - omega)), the
                                Eq. 5 iteration diverges on most of the image      */
    int32_t denoise_fused;   /* 1: the denoiser ran as one launch (else one launch
                                per iteration)                                     */
    float transport_ms;      /* CUDA-event time of the transport launch (Step 2)   */
    float denoise_ms;        /* CUDA-event time of the Eq. 5 iteration             */
    float total_ms;          /* CUDA-event time of the whole call's device work    */
} gdrr_projection_info;

/* Steps 1-4 of Section 2.2 in one call, every step a kernel on the context
 * stream (Step 1 on a side stream of the context, forked from and joined
 * back to it, so that the ray trace fills the SMs the transport leaves at
 * its end) and every scalar computed on the device:
 *   1  P = ray-traced primary (gdrr_raytrace_primary);
 *   2  fixed-point tallies of n_photons histories (gdrr_mc_project with
 *      history_offset 0, into zeroed tallies), P^ and S^ per source photon
 *      (gdrr_finalize);
 *   3  S^ binned to the coarse grid (gdrr_bin_tally + gdrr_finalize), the count
 *      scale and beta (gdrr_projection_info), the Eq. 5 denoiser on the count
 *      scale (gdrr_denoise_scatter), S = its bilinear upsampling
 *      (gdrr_upsample);
 *   4  N = ((P^ - P) + (S^ - S)) sqrt(n_photons / (zeta mAs))
 *      (gdrr_noise_calibrate).
 * Each output equals what that sequence of calls gives.  The call
 * synchronises the stream once, at its end, to read the scalars back:
 * GDRR_ERR_STEP_LIMIT when histories hit max_steps, GDRR_ERR_TALLY_OVERFLOW
 * when a tally wrapped, GDRR_ERR_TIMEOUT when the denoiser's bounded wait gave
 * up; info (host, may be NULL) is filled in every one of these cases.  The
 * first call on a context allocates its scratch (tallies, coarse images,
 * scalars): about 2 nu nv (8 + 0.3) bytes. */
GDRR_API int gdrr_project(gdrr_ctx* ctx, const gdrr_projection* proj, const gdrr_projection_out* out,
                          gdrr_projection_info* info);

/* Step 4, Section 2.6, Eq. 4 and the scaling equation that follows it:
 * N = ((P^ - P) + (S^ - S)) sqrt(n_sim / (zeta * mAs)), element-wise over n
 * pixels; all arrays caller-owned device double. */
GDRR_API int gdrr_noise_calibrate(gdrr_ctx* ctx, const double* P_hat_dev, const double* P_dev,
                                  const double* S_hat_dev, const double* S_dev, int64_t n,
                                  uint64_t n_sim, double mAs, double zeta, double* N_dev);

/* Step 4 calibration, Section 2.6: fit sigma_X / sigma_N^ = k / sqrt(I)
 * (least squares through the origin) over n host points, zeta = n_sim / k^2.
 * Host-only; zeta_out and k_out are host pointers (k_out may be NULL). */
GDRR_API int gdrr_fit_zeta(const double* inv_sqrt_mAs, const double* ratio, int32_t n,
                           uint64_t n_sim, double* zeta_out, double* k_out);

/* Memory-roofline probe of the transport: n_cells trilinear cells at
 * pseudo-random positions, each gathering the same eight voxel records with
 * the same layout and index arithmetic as a Woodcock free flight, and nothing
 * else.  *seconds_out (host) receives the device time of those gathers; the
 * call synchronises the context stream.  Not part of the paper's method: it
 * measures the ceiling the transport's gather rate is compared with. */
GDRR_API int gdrr_gather_roofline(gdrr_ctx* ctx, uint64_t n_cells, double* seconds_out);

/* dst = (float)(src * scale) and dst = (double)src * scale over n device
 * elements (packing images into the learned estimator's FP32 input and
 * back); run on cuda_stream. */
GDRR_API int gdrr_scale_to_f32(const double* src_dev, int64_t n, double scale, float* dst_dev, void* cuda_stream);
GDRR_API int gdrr_scale_to_f64(const float* src_dev, int64_t n, double scale, double* dst_dev, void* cuda_stream);

/* BF16 tensor-core GEMM (tcgen05): C[M x N] (FP32, row length ldc) = A[M x K]
 * . B[N x K]^T with A and B BF16 device matrices whose rows are K-contiguous
 * (row lengths lda, ldb, multiples of 8 elements; A_dev and B_dev 16-byte
 * aligned, C_dev 4-byte aligned, else GDRR_ERR_INVALID_ARG before any launch);
 * K a multiple of 64.  Outputs wider than 64 columns take the TMA-fed
 * pipelined kernel.  With
 * splits > 1 the K range is split across CTAs that add into C, which the
 * caller zeroes first.  Synchronises; GDRR_ERR_TIMEOUT reports a tensor-core
 * pipeline wait that gave up.  Not in the paper: the building block of the learned
 * scatter estimator's convolutions. */
GDRR_API int gdrr_gemm_bf16(const void* A_dev, int32_t lda, const void* B_dev, int32_t ldb, float* C_dev, int32_t ldc,
                            int32_t M, int32_t N, int32_t K, int32_t splits, void* cuda_stream);

/* ---- Learned scatter estimator ----------------------------------------------
 * Not in the paper.  A 4-level convolutional encoder-decoder (base_channels
 * channels at full resolution, doubling per level; 2 x 2 average pooling,
 * nearest 2x upsampling with skip concatenation, ReLU, a 1x1 output layer
 * whose result is added to input channel 0, so the network learns a
 * correction to that channel) that maps (low-photon scatter estimate,
 * ray-traced primary) to scatter, trained
 * on pairs the method itself generates.  BF16 weights and activations, FP32
 * accumulation on the tensor cores; FP32 master weights, gradients and Adam
 * state.  Inputs are device FP32 [batch][2][height][width], outputs and
 * targets [batch][1][height][width]; height and width multiples of 8;
 * base_channels a multiple of 8, at most 64 (else GDRR_ERR_INVALID_ARG).
 * Parameters flatten layer by layer as (weights [co][ci][ky][kx], biases
 * [co]), encoder first, then decoder, then the 1x1 layer.  Convolutions whose
 * grid tiles into 128-pixel groups of whole rows (or of part of one row) run
 * as implicit GEMMs on the tensor cores; the others, and the weight
 * gradients, through column matrices. */
typedef struct gdrr_cnn gdrr_cnn;
GDRR_API int gdrr_cnn_create(int32_t max_batch, int32_t height, int32_t width, int32_t base_channels, uint64_t seed,
                             void* cuda_stream, gdrr_cnn** out);
GDRR_API void gdrr_cnn_destroy(gdrr_cnn* net);
GDRR_API int gdrr_cnn_num_params(const gdrr_cnn* net, int64_t* count);
/* Host FP32 copies of the parameters / of the last backward's gradients. */
GDRR_API int gdrr_cnn_get_params(gdrr_cnn* net, float* host);
GDRR_API int gdrr_cnn_set_params(gdrr_cnn* net, const float* host);   /* also resets the Adam state */
GDRR_API int gdrr_cnn_get_grads(gdrr_cnn* net, float* host);
/* Forward pass of batch inputs; out_dev may be NULL (activations are kept for backward). */
GDRR_API int gdrr_cnn_forward(gdrr_cnn* net, int32_t batch, const float* in_dev, float* out_dev);
/* Mean-squared-error loss against target_dev and the gradients of every
 * parameter for the last forward pass (overwritten, not accumulated);
 * *loss_out (host) receives the loss.  Synchronises; GDRR_ERR_TIMEOUT
 * reports a tensor-core pipeline wait that gave up. */
GDRR_API int gdrr_cnn_backward(gdrr_cnn* net, const float* target_dev, double* loss_out);
/* One Adam update of every parameter from the last gradients. */
GDRR_API int gdrr_cnn_adam_step(gdrr_cnn* net, float lr, float beta1, float beta2, float eps);

/* Parity hook: the Philox words of n_hist history streams (ids hid0 ..),
 * n_blocks blocks each, exactly as the transport draws them.  out_dev:
 * device uint32[n_hist][4 * n_blocks].  Runs on cuda_stream. */
GDRR_API int gdrr_stream_words(uint64_t seed, uint32_t angle_index, uint64_t hid0, int32_t n_hist,
                               int32_t n_blocks, uint32_t* out_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GDRR_H */
