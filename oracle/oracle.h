/*
 * CPU oracle for the gDRR projection path (arXiv:1204.6367).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-purpose CPU
 * restatement of what the paper computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Units: lengths mm, energies keV, density g/cm^3, mass attenuation cm^2/g.
 * Phantom index order: x fastest, idx = x + nx*(y + ny*z), box centred on the
 * isocentre.
 *
 * Parity status of each function is stated beside it; all are pinned by the
 * CPU tests (closed forms, library routines, invariants).
 */
#ifndef GDRR_ORACLE_H
#define GDRR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    /* geometry, Section 2.1 / Fig. 1 */
    double sad, sdd, theta;
    int nu, nv;
    double du, dv;
    /* voxel phantom, Section 2.1: material index i(x) and density rho(x) */
    int nx, ny, nz;
    double vx, vy, vz;
    const uint8_t* material;
    const float* density;
    /* mass attenuation mu_hat_k(i, E), k = Rayleigh, Compton, photo; [m][k][e] */
    int n_mat, n_e;
    double e0, de;
    const float* mu_hat;
    /* source spectrum phi(E): bin energies and weights; optionally one spectrum
     * per detector column [nu][n_bins] (bowtie hardening), else NULL */
    int n_bins;
    const double* bin_e;
    const double* bin_w;
    const double* bin_w_cols;
    /* fluence map w(u) after the bowtie, [nv][nu] */
    const double* fluence;
    /* detector response r(E) on r0 + i*dr */
    int n_r;
    double r0, dr;
    const float* response;
    /* transport options */
    double e_cut;      /* photons below this energy are absorbed (keV) */
    int max_steps;     /* per-history free-flight limit */
    int nearest_voxel; /* 0: trilinear density interpolation (Section 2.4); 1: the voxel's own value */
    int scatter_filter;/* which scattered photons the scatter counter takes (Section 2.4 option):
                          0 all, 1 exactly one Compton and no Rayleigh, 2 exactly one Rayleigh and no
                          Compton, 3 two or more interactions; others count as missing the detector */
    /* Rayleigh angular law: 0 Thomson (1 + cos^2); 1 (1 + cos^2) F^2(x) with the
     * form factor F(x, i) of each material on x_j = j * ff_dx (1/Angstrom,
     * x = sin(theta/2) / lambda), [n_mat][n_ff] */
    int rayleigh_ff;
    int n_ff;
    double ff_dx;
    const float* ff;
    /* Free-flight majorant: 0 the global one of Woodcock tracking (Section 2.4);
     * 1 local majorants, one per macro cell of 2^cell_shift voxels per edge
     * (cell_shift 0..10): delta tracking with a piecewise-constant majorant,
     * the optical depth of each flight spent cell by cell along the ray.  An
     * option beside the paper's method; the expected images are the same. */
    int local_majorant;
    int cell_shift;
} orc_problem;

/* One record per history, for tiny-run event-by-event parity. */
typedef struct {
    uint32_t n_steps, n_virtual, n_rayleigh, n_compton;
    uint32_t n_photo, outcome, rng_blocks, first_interaction;
    int32_t pixel;
    float e_source, e_final;
    uint32_t ray_material;   /* material of the last form-factor Rayleigh event, else 0 */
    double e_deposited;
} orc_record;

enum { ORC_OUT_PRIMARY = 0, ORC_OUT_SCATTER = 1, ORC_OUT_PHOTO = 2, ORC_OUT_CUTOFF = 3,
       ORC_OUT_MISS = 4, ORC_OUT_STEP_LIMIT = 5 };
enum { ORC_INT_NONE = 0, ORC_INT_RAYLEIGH = 1, ORC_INT_COMPTON = 2, ORC_INT_PHOTO = 3 };

/* stats[] order */
enum { ORC_ST_HISTORIES = 0, ORC_ST_STEPS, ORC_ST_VIRTUAL, ORC_ST_RAYLEIGH, ORC_ST_COMPTON,
       ORC_ST_PHOTO, ORC_ST_TALLY_P, ORC_ST_TALLY_S, ORC_ST_MISS, ORC_ST_CUTOFF,
       ORC_ST_STEP_LIMIT, ORC_ST_CROSSINGS, ORC_NSTATS };

/* Philox4x32-10 (Salmon et al., SC'11).  Pinned against cuRAND's host generator. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Natural log of a positive normal float by the atanh series (textbook). */
float orc_logf(float x);
void orc_logf_many(const float* x, float* out, int n);
void orc_philox_many(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n);
/* Stream words for history hid: n_blocks Philox blocks, counter (k, angle, hid lo, hid hi). */
void orc_stream_words(uint64_t seed, uint32_t angle_index, uint64_t hid, int n_blocks, uint32_t* out);

/* Angular samplers on their own, for the closed-form pins.  Sample i uses the
 * stream of history id i; the sampler starts at the first word of the stream. */
void orc_sample_compton(float e_kev, uint64_t seed, int n, float* cos_out, float* e_out);
void orc_sample_rayleigh(uint64_t seed, int n, float* cos_out);
void orc_sample_azimuth(uint64_t seed, int n, float* cos_out, float* sin_out);
void orc_rotate(const float d[3], float ct, float cp, float sp, float out[3]);

/* Monte Carlo projection (Section 2.4).  Tallies ACCUMULATE into tally_p /
 * tally_s (int64 fixed point, 2^-24 keV units, [nv][nu]).  precision is 32
 * (FP32 transport: the parity reference) or 64 (FP64 transport: the accuracy
 * reference).  stats has ORC_NSTATS entries (accumulated).  records, if not
 * NULL, receives one record per history.  Returns 0 or a negative error. */
int orc_mc_run(const orc_problem* p, double phi, uint32_t angle_index, uint64_t n_histories,
               uint64_t seed, uint64_t history_offset, int precision, int n_threads,
               int64_t* tally_p, int64_t* tally_s, uint64_t* stats, orc_record* records);

/* Ray-traced primary, Eq. 1, FP64, for the listed flat pixel indices (all
 * pixels when pixels == NULL).  out[i] is P at pixels[i] per source photon. */
int orc_rt_primary(const orc_problem* p, double phi, const int32_t* pixels, int n_pixels,
                   double* out);

/* Siddon ray-traced primary (Section 2.3's alternative; Siddon 1985), FP64:
 * exact path lengths through the piecewise-constant voxel field, one trace
 * per energy channel. */
int orc_rt_primary_siddon(const orc_problem* p, double phi, const int32_t* pixels, int n_pixels, double* out);

/* Derived tables, exposed for the pins. */
int orc_majorant(const orc_problem* p, float* node_out /* n_e */);

/* Local majorants: the macro-cell table, per cell (x fastest) and material,
 * the largest density over the voxels [c 2^s, (c + 1) 2^s] of each axis
 * (clamped to the phantom), [ncz][ncy][ncx][n_mat]; and one free flight of
 * the tracking with that table (precision 32 or 64) from pos along unit dir
 * at energy e with optical depth tau: returns 1 at a tentative collision
 * (out = position, bound there, cell crossings), 0 when the ray leaves the
 * box first (out = last position inside, 0, crossings), negative on error. */
int orc_lm_cells(const orc_problem* p, float* out);
int orc_lm_walk(const orc_problem* p, int precision, const double pos[3], const double dir[3], double e,
                double tau, double out[5]);

#ifdef __cplusplus
}
#endif
#endif
