/*
 * CPU oracle for the gDRR projection path (arXiv:1204.6367).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library.  It is a plain, slow
 * restatement of the paper's method that shares no code with the CUDA path.
 *
 *   - Philox4x32-10 random streams (Salmon et al., SC'11), one per history;
 *   - the Monte Carlo step of Section 2.4 (mc_history.inc), FP32 and FP64;
 *   - the tri-linear ray-traced primary of Section 2.3, Eq. 1, in FP64.
 *
 * Build flags keep every floating-point operation an IEEE-rounded single
 * operation (-ffp-contract=off, no fast-math), so that the FP32 transport is
 * a bit-level reference for any implementation that performs the same
 * operations in the same order.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_MAT 16

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: ten rounds of the Philox S-box over a 128-bit counter with a
 * 64-bit key bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
} orc_stream;

/* The stream of a history: Philox blocks with counter (k, angle index, hid lo,
 * hid hi), k = 0, 1, 2, ..., key = (seed lo, seed hi).  Every draw site takes
 * the next whole block: the source (block 0, four uniforms), each free flight
 * (two uniforms), each rejection attempt of an angular sampler (two or three
 * uniforms); words a site does not use are dropped. */
static void orc_stream_init(orc_stream* s, uint64_t seed, uint32_t angle_index, uint64_t hid) {
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
    s->ctr[0] = 0;
    s->ctr[1] = angle_index;
    s->ctr[2] = (uint32_t)hid;
    s->ctr[3] = (uint32_t)(hid >> 32);
}

/* Uniform on (0, 1]: the top 24 bits plus one, times 2^-24 (exact in FP32). */
static float orc_uniform(uint32_t w) {
    return (float)((w >> 8) + 1u) * (float)(1.0 / 16777216.0);
}

/* The next block of the stream as four uniforms. */
static void orc_next_block(orc_stream* s, float u[4]) {
    uint32_t w[4];
    orc_philox4x32_10(s->ctr, s->key, w);
    s->ctr[0] += 1;
    for (int i = 0; i < 4; ++i) u[i] = orc_uniform(w[i]);
}

void orc_stream_words(uint64_t seed, uint32_t angle_index, uint64_t hid, int n_blocks, uint32_t* out) {
    orc_stream s;
    orc_stream_init(&s, seed, angle_index, hid);
    for (int b = 0; b < n_blocks; ++b) {
        orc_philox4x32_10(s.ctr, s.key, out + 4 * b);
        s.ctr[0] += 1;
    }
}

/* ------------------------------------------------------------------------ */
/* ln(x) for a positive normal float: x = m * 2^e with m in [sqrt(1/2), sqrt(2)),
 * ln m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ... + s^11/11), s = (m-1)/(m+1),
 * ln x = e ln2 + ln m, with ln 2 split into a 12-bit head and a tail so that
 * e * head is exact.  The series is the textbook Taylor series of atanh;
 * |s| <= 0.1716 so the first omitted term is below 2^-30 relative. */
float orc_logf(float x) {
    union { float f; uint32_t u; } v;
    v.f = x;
    int e = (int)((v.u >> 23) & 0xffu) - 127;
    v.u = (v.u & 0x007fffffu) | 0x3f800000u;          /* m in [1, 2) */
    if (v.u > 0x3fb504f3u) {                           /* m > sqrt(2): halve */
        v.u -= 0x00800000u;
        e += 1;
    }
    float m = v.f;
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float poly = (float)(1.0 / 3.0) + s2 * ((float)(1.0 / 5.0) + s2 * ((float)(1.0 / 7.0)
               + s2 * ((float)(1.0 / 9.0) + s2 * (float)(1.0 / 11.0))));
    float lm = 2.0f * s + (2.0f * s) * (s2 * poly);
    float ln2_hi = (float)(2839.0 / 4096.0);
    float ln2_lo = (float)(0.69314718055994530942 - 2839.0 / 4096.0);
    float fe = (float)e;
    return fe * ln2_hi + (fe * ln2_lo + lm);
}

void orc_logf_many(const float* x, float* out, int n) {
    for (int i = 0; i < n; ++i) out[i] = orc_logf(x[i]);
}

void orc_philox_many(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n) {
    for (int i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* Smallest j with xi <= cdf[j] (inverse-CDF sampling; cdf[n-1] == 1). */
static int orc_cdf_search(const double* cdf, int n, double xi) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (xi <= cdf[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* Derived per-projection quantities in both precisions. */
#define GEO_FIELDS(T)                                                         \
    T S[3], n[3], P[3], eu[3], ev[3], lo[3], hi[3], ivox[3], vox[3];          \
    T hu, hv, du, dv, idu, idv, e0, inv_de, r0, inv_dr, e_cut;                \
    T* tab;   /* [m][k][e] mm^-1 per g/cm^3 */                                \
    T* major; /* [e] majorant node values, mm^-1 */                           \
    T* resp;  /* [n_r] keV */                                                 \
    T* bin_e; /* [n_bins] keV */                                              \
    T* ff_s;  /* [n_ff] squared momentum transfer x_j^2, 1/Angstrom^2 */       \
    T* ff_a;  /* [m][n_ff] cumulative of F^2 over x^2 (trapezoid) */           \
    T* ff_g;  /* [m][n_ff] F^2 on the nodes */                                 \
    T inv_hc, ff_idx;  /* 1/(hc) in 1/(keV Angstrom); 1/ff_dx */

typedef struct { GEO_FIELDS(float) } orc_geo_f;
typedef struct { GEO_FIELDS(double) } orc_geo_d;

typedef struct {
    const orc_problem* p;
    int dims[3];
    double* cdf_pix;
    double* cdf_e;
    double* cdf_e_cols;   /* [nu][n_bins] when the spectrum depends on the column */
    orc_geo_f gf;
    orc_geo_d gd;
    /* local majorants: cells per axis and the per-cell, per-material largest
     * density (orc_lm_build), NULL without the option */
    int nc[3];
    float* lm_rho;
} orc_ctx;

static double* orc_build_cdf(const double* w, int n) {
    double* c = (double*)malloc(sizeof(double) * (size_t)n);
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(w[i] >= 0.0)) { free(c); return NULL; }
        s += w[i];
        c[i] = s;
    }
    if (!(s > 0.0)) { free(c); return NULL; }
    for (int i = 0; i < n; ++i) c[i] = c[i] / s;
    return c;
}

/* Woodcock majorant on the energy nodes: the largest total mu over materials,
 * each at the largest density present for that material, with a 1e-5 relative
 * margin for rounding.  Between nodes the larger bracketing node is used, which
 * bounds the linear interpolant and the convex trilinear mixture. */
static void orc_build_major(const orc_problem* p, const float* tab, float* major) {
    double rho_max[ORC_MAX_MAT];
    for (int m = 0; m < p->n_mat; ++m) rho_max[m] = 0.0;
    size_t nv = (size_t)p->nx * p->ny * p->nz;
    for (size_t v = 0; v < nv; ++v) {
        double r = (double)p->density[v];
        if (r > rho_max[p->material[v]]) rho_max[p->material[v]] = r;
    }
    for (int e = 0; e < p->n_e; ++e) {
        double mx = 0.0;
        for (int m = 0; m < p->n_mat; ++m) {
            const float* t = tab + (size_t)m * 3 * p->n_e;
            double tot = ((double)t[e] + (double)t[p->n_e + e]) + (double)t[2 * p->n_e + e];
            double v = rho_max[m] * tot;
            if (v > mx) mx = v;
        }
        major[e] = (float)(mx * (1.0 + 1e-5));
    }
}

/* The macro cells of the local-majorant option.  Cell k of an axis (2^s
 * voxels per edge, s = cell_shift) holds the points whose lower trilinear
 * corner, max(floor((x - lo) / vox - 1/2), 0), has index k 2^s ... (k + 1) 2^s
 * - 1; the eight corners of such a point lie among the voxels k 2^s ...
 * (k + 1) 2^s, which is the cover whose largest density per material the
 * table keeps.  Every corner term rho_c mu(m_c, E) of the mixture is then at
 * most max_m rho_max(cell, m) mu(m, E), and so is the mixture (its weights sum
 * to one).  Written as that definition: for each cell, a scan of its cover. */
static int orc_lm_build(orc_ctx* c) {
    const orc_problem* p = c->p;
    const int s = p->cell_shift;
    if (s < 0 || s > 10) return -1;
    for (int a = 0; a < 3; ++a) c->nc[a] = ((c->dims[a] - 1) >> s) + 1;
    size_t ncell = (size_t)c->nc[0] * c->nc[1] * c->nc[2];
    c->lm_rho = (float*)calloc(ncell * (size_t)p->n_mat, sizeof(float));
    if (!c->lm_rho) return -1;
    for (int kz = 0; kz < c->nc[2]; ++kz)
        for (int ky = 0; ky < c->nc[1]; ++ky)
            for (int kx = 0; kx < c->nc[0]; ++kx) {
                float* r = c->lm_rho + (((size_t)kz * c->nc[1] + ky) * c->nc[0] + kx) * p->n_mat;
                int k[3] = {kx, ky, kz}, v0[3], v1[3];
                for (int a = 0; a < 3; ++a) {
                    v0[a] = k[a] << s;
                    v1[a] = (k[a] + 1) << s;
                    if (v1[a] > c->dims[a] - 1) v1[a] = c->dims[a] - 1;
                }
                for (int z = v0[2]; z <= v1[2]; ++z)
                    for (int y = v0[1]; y <= v1[1]; ++y)
                        for (int x = v0[0]; x <= v1[0]; ++x) {
                            size_t v = (size_t)x + (size_t)p->nx * ((size_t)y + (size_t)p->ny * z);
                            float rho = p->density[v];
                            if (rho > r[p->material[v]]) r[p->material[v]] = rho;
                        }
            }
    return 0;
}

static int orc_ctx_init(orc_ctx* c, const orc_problem* p, double phi) {
    memset(c, 0, sizeof *c);
    c->p = p;
    if (p->n_mat < 1 || p->n_mat > ORC_MAX_MAT || p->n_e < 2 || p->n_r < 2 || p->n_bins < 1
        || p->nu < 1 || p->nv < 1 || p->nx < 1 || p->ny < 1 || p->nz < 1)
        return -1;
    size_t nvox = (size_t)p->nx * p->ny * p->nz;
    for (size_t v = 0; v < nvox; ++v)
        if (p->material[v] >= p->n_mat || !(p->density[v] >= 0.0f)) return -1;
    c->dims[0] = p->nx; c->dims[1] = p->ny; c->dims[2] = p->nz;
    c->cdf_pix = orc_build_cdf(p->fluence, p->nu * p->nv);
    c->cdf_e = orc_build_cdf(p->bin_w, p->n_bins);
    if (!c->cdf_pix || !c->cdf_e) return -1;
    if (p->bin_w_cols) {
        c->cdf_e_cols = (double*)malloc(sizeof(double) * (size_t)p->nu * p->n_bins);
        for (int u = 0; u < p->nu; ++u) {
            double* col = orc_build_cdf(p->bin_w_cols + (size_t)u * p->n_bins, p->n_bins);
            if (!col) return -1;
            memcpy(c->cdf_e_cols + (size_t)u * p->n_bins, col, sizeof(double) * (size_t)p->n_bins);
            free(col);
        }
    }

    /* geometry (Fig. 1): source at SAD on the -SO side, imager at AID = SDD - SAD
     * along OP, which makes angle theta with SO; v axis parallel to z. */
    double ang = phi + p->theta, aid = p->sdd - p->sad;
    double S[3] = {-p->sad * cos(phi), -p->sad * sin(phi), 0.0};
    double n[3] = {cos(ang), sin(ang), 0.0};
    double P[3] = {aid * cos(ang), aid * sin(ang), 0.0};
    double eu[3] = {sin(ang), -cos(ang), 0.0};
    double ev[3] = {0.0, 0.0, 1.0};
    double vox[3] = {p->vx, p->vy, p->vz};
    for (int k = 0; k < 3; ++k) {
        double half = 0.5 * c->dims[k] * vox[k];
        c->gd.S[k] = S[k]; c->gd.n[k] = n[k]; c->gd.P[k] = P[k];
        c->gd.eu[k] = eu[k]; c->gd.ev[k] = ev[k];
        c->gd.lo[k] = -half; c->gd.hi[k] = half; c->gd.ivox[k] = 1.0 / vox[k];
        c->gf.S[k] = (float)S[k]; c->gf.n[k] = (float)n[k]; c->gf.P[k] = (float)P[k];
        c->gf.eu[k] = (float)eu[k]; c->gf.ev[k] = (float)ev[k];
        c->gf.lo[k] = (float)(-half); c->gf.hi[k] = (float)half;
        c->gf.ivox[k] = (float)(1.0 / vox[k]);
        c->gd.vox[k] = vox[k];
        c->gf.vox[k] = (float)vox[k];
    }
    /* The source must lie outside the box and the whole box on the source
     * side of the imager plane, so that a photon leaving the box towards the
     * plane always meets it ahead of the box. */
    {
        int src_in = 1;
        for (int k = 0; k < 3; ++k)
            if (!(S[k] > c->gd.lo[k] && S[k] < c->gd.hi[k])) src_in = 0;
        if (src_in) return -1;
        for (int corner = 0; corner < 8; ++corner) {
            double q[3];
            for (int k = 0; k < 3; ++k) q[k] = ((corner >> k) & 1) ? c->gd.hi[k] : c->gd.lo[k];
            double side = (q[0] - P[0]) * n[0] + (q[1] - P[1]) * n[1] + (q[2] - P[2]) * n[2];
            if (!(side < 0.0)) return -1;
        }
        double s_side = (S[0] - P[0]) * n[0] + (S[1] - P[1]) * n[1] + (S[2] - P[2]) * n[2];
        if (!(s_side < 0.0)) return -1;
    }
    c->gd.hu = 0.5 * p->nu; c->gd.hv = 0.5 * p->nv; c->gd.du = p->du; c->gd.dv = p->dv;
    c->gd.idu = 1.0 / p->du; c->gd.idv = 1.0 / p->dv;
    c->gd.e0 = p->e0; c->gd.inv_de = 1.0 / p->de; c->gd.r0 = p->r0; c->gd.inv_dr = 1.0 / p->dr;
    c->gd.e_cut = p->e_cut;
    c->gf.hu = (float)(0.5 * p->nu); c->gf.hv = (float)(0.5 * p->nv);
    c->gf.du = (float)p->du; c->gf.dv = (float)p->dv;
    c->gf.idu = (float)(1.0 / p->du); c->gf.idv = (float)(1.0 / p->dv);
    c->gf.e0 = (float)p->e0; c->gf.inv_de = (float)(1.0 / p->de);
    c->gf.r0 = (float)p->r0; c->gf.inv_dr = (float)(1.0 / p->dr);
    c->gf.e_cut = (float)p->e_cut;

    /* tables: mu_hat in cm^2/g times 0.1 -> mm^-1 per g/cm^3 */
    size_t nt = (size_t)p->n_mat * 3 * p->n_e;
    c->gf.tab = (float*)malloc(sizeof(float) * nt);
    c->gd.tab = (double*)malloc(sizeof(double) * nt);
    for (size_t i = 0; i < nt; ++i) {
        c->gf.tab[i] = (float)((double)p->mu_hat[i] * 0.1);
        c->gd.tab[i] = (double)c->gf.tab[i];
    }
    c->gf.major = (float*)malloc(sizeof(float) * (size_t)p->n_e);
    c->gd.major = (double*)malloc(sizeof(double) * (size_t)p->n_e);
    orc_build_major(p, c->gf.tab, c->gf.major);
    for (int e = 0; e < p->n_e; ++e) c->gd.major[e] = (double)c->gf.major[e];
    c->gf.resp = (float*)malloc(sizeof(float) * (size_t)p->n_r);
    c->gd.resp = (double*)malloc(sizeof(double) * (size_t)p->n_r);
    for (int i = 0; i < p->n_r; ++i) { c->gf.resp[i] = p->response[i]; c->gd.resp[i] = p->response[i]; }
    c->gf.bin_e = (float*)malloc(sizeof(float) * (size_t)p->n_bins);
    c->gd.bin_e = (double*)malloc(sizeof(double) * (size_t)p->n_bins);
    for (int i = 0; i < p->n_bins; ++i) { c->gf.bin_e[i] = (float)p->bin_e[i]; c->gd.bin_e[i] = p->bin_e[i]; }

    /* Rayleigh form factors: the polar angle follows (1 + cos^2) F^2(x) with
     * x = sin(theta/2) E / (hc), i.e. x^2 = x_max^2 (1 - cos) / 2; x^2 is drawn
     * from F^2 taken linear in x^2 between the table's nodes (its cumulative
     * A(x^2) is the trapezoid sum, quadratic within an interval) and accepted
     * with (1 + cos^2) / 2.  The grid must reach x_max of the table's largest
     * energy; F(0) > 0. */
    if (p->rayleigh_ff) {
        const double hc = 12.398419843320026;   /* keV Angstrom (CODATA 2018) */
        if (!p->ff || p->n_ff < 2 || !(p->ff_dx > 0.0)) return -1;
        double e_max = p->e0 + (double)(p->n_e - 1) * p->de;
        if ((double)(p->n_ff - 1) * p->ff_dx < e_max / hc) return -1;
        size_t nf = (size_t)p->n_ff;
        c->gf.ff_s = (float*)malloc(sizeof(float) * nf);
        c->gd.ff_s = (double*)malloc(sizeof(double) * nf);
        c->gf.ff_a = (float*)malloc(sizeof(float) * nf * (size_t)p->n_mat);
        c->gd.ff_a = (double*)malloc(sizeof(double) * nf * (size_t)p->n_mat);
        c->gf.ff_g = (float*)malloc(sizeof(float) * nf * (size_t)p->n_mat);
        c->gd.ff_g = (double*)malloc(sizeof(double) * nf * (size_t)p->n_mat);
        for (int j = 0; j < p->n_ff; ++j) {
            double x = (double)j * p->ff_dx;
            c->gd.ff_s[j] = x * x;
            c->gf.ff_s[j] = (float)(x * x);
        }
        for (int m = 0; m < p->n_mat; ++m) {
            const float* F = p->ff + (size_t)m * nf;
            if (!(F[0] > 0.0f)) return -1;
            double acc = 0.0;
            for (int j = 0; j < p->n_ff; ++j) {
                if (!(F[j] >= 0.0f) || !isfinite(F[j])) return -1;
                if (j > 0) {
                    double f0 = (double)F[j - 1], f1 = (double)F[j];
                    acc += 0.5 * (f0 * f0 + f1 * f1) * (c->gd.ff_s[j] - c->gd.ff_s[j - 1]);
                }
                c->gd.ff_a[(size_t)m * nf + j] = acc;
                c->gf.ff_a[(size_t)m * nf + j] = (float)acc;
                double g = (double)F[j] * (double)F[j];
                c->gd.ff_g[(size_t)m * nf + j] = g;
                c->gf.ff_g[(size_t)m * nf + j] = (float)g;
            }
        }
        c->gd.inv_hc = 1.0 / hc;
        c->gf.inv_hc = (float)(1.0 / hc);
        c->gd.ff_idx = 1.0 / p->ff_dx;
        c->gf.ff_idx = (float)(1.0 / p->ff_dx);
    }
    if (p->local_majorant && orc_lm_build(c)) return -1;
    return 0;
}

static void orc_ctx_free(orc_ctx* c) {
    free(c->cdf_pix); free(c->cdf_e); free(c->cdf_e_cols);
    free(c->gf.tab); free(c->gd.tab); free(c->gf.major); free(c->gd.major);
    free(c->gf.resp); free(c->gd.resp); free(c->gf.bin_e); free(c->gd.bin_e);
    free(c->gf.ff_s); free(c->gd.ff_s); free(c->gf.ff_a); free(c->gd.ff_a);
    free(c->gf.ff_g); free(c->gd.ff_g);
    free(c->lm_rho);
}

int orc_majorant(const orc_problem* p, float* node_out) {
    orc_ctx c;
    if (orc_ctx_init(&c, p, 0.0)) { orc_ctx_free(&c); return -1; }
    memcpy(node_out, c.gf.major, sizeof(float) * (size_t)p->n_e);
    orc_ctx_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The history, once per precision. */
#define REAL float
#define ORC_MAX_BLOCKS (1u << 24)   /* Philox blocks per history after which samplers stop rejecting */
#define ORC_LM_MARGIN 1.0009765625  /* local-majorant bounds are raised by 2^-10 */

#define FN(name) name##_f32
#define GEO(x) (c->gf.x)
#define LOGR(x) orc_logf(x)
#define SQRTR(x) sqrtf(x)
#define FLOORR(x) floorf(x)
#define LLRINTR(x) llrintf(x)
#include "mc_history.inc"
#undef REAL
#undef FN
#undef GEO
#undef LOGR
#undef SQRTR
#undef FLOORR
#undef LLRINTR

#define REAL double
#define FN(name) name##_f64
#define GEO(x) (c->gd.x)
#define LOGR(x) log(x)
#define SQRTR(x) sqrt(x)
#define FLOORR(x) floor(x)
#define LLRINTR(x) llrint(x)
#include "mc_history.inc"
#undef REAL
#undef FN
#undef GEO
#undef LOGR
#undef SQRTR
#undef FLOORR
#undef LLRINTR

int orc_lm_cells(const orc_problem* p, float* out) {
    orc_problem q = *p;
    q.local_majorant = 1;
    orc_ctx c;
    if (orc_ctx_init(&c, &q, 0.0)) { orc_ctx_free(&c); return -1; }
    memcpy(out, c.lm_rho, sizeof(float) * (size_t)c.nc[0] * c.nc[1] * c.nc[2] * (size_t)p->n_mat);
    orc_ctx_free(&c);
    return 0;
}

int orc_lm_walk(const orc_problem* p, int precision, const double pos[3], const double dir[3], double e,
                double tau, double out[5]) {
    if (precision != 32 && precision != 64) return -1;
    orc_problem q = *p;
    q.local_majorant = 1;
    orc_ctx c;
    if (orc_ctx_init(&c, &q, 0.0)) { orc_ctx_free(&c); return -1; }
    int hit = precision == 64 ? lm_walk_once_f64(&c, pos, dir, e, tau, out) : lm_walk_once_f32(&c, pos, dir, e, tau, out);
    orc_ctx_free(&c);
    return hit;
}

/* ------------------------------------------------------------------------ */
/* Samplers on their own (for the angular-distribution pins). */
void orc_sample_compton(float e_kev, uint64_t seed, int n, float* cos_out, float* e_out) {
    for (int i = 0; i < n; ++i) {
        orc_stream s;
        orc_stream_init(&s, seed, 0, (uint64_t)i);
        compton_f32(&s, e_kev, &cos_out[i], &e_out[i]);
    }
}

void orc_sample_rayleigh(uint64_t seed, int n, float* cos_out) {
    for (int i = 0; i < n; ++i) {
        orc_stream s;
        orc_stream_init(&s, seed, 0, (uint64_t)i);
        cos_out[i] = rayleigh_f32(&s);
    }
}

int orc_sample_rayleigh_ff(const orc_problem* p, float e_kev, int material, uint64_t seed, int n,
                           float* cos_out) {
    orc_ctx c;
    if (!p->rayleigh_ff || material < 0 || material >= p->n_mat || orc_ctx_init(&c, p, 0.0)) return -1;
    for (int i = 0; i < n; ++i) {
        orc_stream s;
        orc_stream_init(&s, seed, 0, (uint64_t)i);
        cos_out[i] = rayleigh_ff_f32(&c, &s, e_kev, material);
    }
    orc_ctx_free(&c);
    return 0;
}

void orc_sample_azimuth(uint64_t seed, int n, float* cos_out, float* sin_out) {
    for (int i = 0; i < n; ++i) {
        orc_stream s;
        orc_stream_init(&s, seed, 0, (uint64_t)i);
        azimuth_f32(&s, &cos_out[i], &sin_out[i]);
    }
}

void orc_rotate(const float d[3], float ct, float cp, float sp, float out[3]) {
    float t[3] = {d[0], d[1], d[2]};
    rotate_f32(t, ct, cp, sp);
    out[0] = t[0]; out[1] = t[1]; out[2] = t[2];
}

/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_ctx* c;
    uint64_t begin, end, seed, offset;
    uint32_t angle_index;
    int precision;
    int64_t* tp;
    int64_t* ts;
    uint64_t st[ORC_NSTATS];
    orc_record* records;
} orc_job;

static void* orc_worker(void* arg) {
    orc_job* j = (orc_job*)arg;
    for (uint64_t i = j->begin; i < j->end; ++i) {
        orc_record* rec = j->records ? &j->records[i] : NULL;
        if (j->precision == 64)
            run_history_f64(j->c, j->offset + i, j->angle_index, j->seed, j->tp, j->ts, j->st, rec);
        else
            run_history_f32(j->c, j->offset + i, j->angle_index, j->seed, j->tp, j->ts, j->st, rec);
    }
    return NULL;
}

int orc_mc_run(const orc_problem* p, double phi, uint32_t angle_index, uint64_t n_histories,
               uint64_t seed, uint64_t history_offset, int precision, int n_threads,
               int64_t* tally_p, int64_t* tally_s, uint64_t* stats, orc_record* records) {
    if (precision != 32 && precision != 64) return -1;
    orc_ctx c;
    if (orc_ctx_init(&c, p, phi)) { orc_ctx_free(&c); return -1; }
    if (n_threads < 1) n_threads = 1;
    if ((uint64_t)n_threads > n_histories) n_threads = n_histories > 0 ? (int)n_histories : 1;
    size_t npix = (size_t)p->nu * p->nv;
    orc_job* jobs = (orc_job*)calloc((size_t)n_threads, sizeof(orc_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int t = 0; t < n_threads; ++t) {
        orc_job* j = &jobs[t];
        j->c = &c;
        j->begin = n_histories * (uint64_t)t / (uint64_t)n_threads;
        j->end = n_histories * (uint64_t)(t + 1) / (uint64_t)n_threads;
        j->seed = seed; j->offset = history_offset; j->angle_index = angle_index;
        j->precision = precision;
        j->tp = (int64_t*)calloc(npix, sizeof(int64_t));
        j->ts = (int64_t*)calloc(npix, sizeof(int64_t));
        j->records = records;
        if (n_threads == 1) orc_worker(j);
        else pthread_create(&th[t], NULL, orc_worker, j);
    }
    for (int t = 0; t < n_threads; ++t) {
        if (n_threads > 1) pthread_join(th[t], NULL);
        orc_job* j = &jobs[t];
        for (size_t i = 0; i < npix; ++i) { tally_p[i] += j->tp[i]; tally_s[i] += j->ts[i]; }
        for (int k = 0; k < ORC_NSTATS; ++k) stats[k] += j->st[k];
        free(j->tp); free(j->ts);
    }
    free(jobs); free(th);
    orc_ctx_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Ray-traced primary (Section 2.3, Eq. 1) in FP64, literally: for every energy
 * channel of the spectrum, the ray from the source to the pixel centre is cut
 * inside the phantom box into equal intervals no longer than half the smallest
 * voxel size, mu(x, E) is taken at each interval midpoint with the trilinear
 * field, and P = w(u) * sum_E phi(E) r(E) exp(-sum_j dl mu(x_j, E)). */
static double orc_mu_at(const orc_ctx* c, const double x[3], const double* mu_e) {
    const orc_problem* p = c->p;
    int i0[3], i1[3];
    double w0[3], w1[3];
    for (int a = 0; a < 3; ++a) {
        double fa = (x[a] - c->gd.lo[a]) * c->gd.ivox[a] - 0.5;
        int f0 = (int)floor(fa);
        double t = fa - f0;
        int f1 = f0 + 1;
        int n_a = c->dims[a];
        f0 = f0 < 0 ? 0 : (f0 > n_a - 1 ? n_a - 1 : f0);
        f1 = f1 < 0 ? 0 : (f1 > n_a - 1 ? n_a - 1 : f1);
        i0[a] = f0; i1[a] = f1; w0[a] = 1.0 - t; w1[a] = t;
    }
    double mu = 0.0;
    for (int corner = 0; corner < 8; ++corner) {
        int cx = corner & 1, cy = (corner >> 1) & 1, cz = corner >> 2;
        int64_t v = (int64_t)(cx ? i1[0] : i0[0])
                  + (int64_t)p->nx * ((cy ? i1[1] : i0[1]) + (int64_t)p->ny * (cz ? i1[2] : i0[2]));
        double w = (cx ? w1[0] : w0[0]) * (cy ? w1[1] : w0[1]) * (cz ? w1[2] : w0[2]);
        mu += w * (double)p->density[v] * mu_e[p->material[v]];
    }
    return mu;
}

static double orc_interp_d(const double* t, double e0, double de, int n, double e) {
    double fi = (e - e0) / de;
    if (fi < 0.0) fi = 0.0;
    if (fi > n - 1) fi = n - 1;
    int i = (int)fi;
    if (i > n - 2) i = n - 2;
    double f = fi - i;
    return t[i] + f * (t[i + 1] - t[i]);
}

/* Siddon's algorithm (Siddon, Med. Phys. 12, 1985): the parametric values
 * where the ray crosses the voxel planes x = lo + i dx (and y, z) inside the
 * box, merged in increasing order; each consecutive pair bounds a segment
 * inside one voxel, found from the segment midpoint; the radiological length
 * is the sum of segment length times that voxel's mu. */
static int orc_cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int orc_rt_primary_siddon(const orc_problem* p, double phi, const int32_t* pixels, int n_pixels, double* out) {
    orc_ctx c;
    if (orc_ctx_init(&c, p, phi)) { orc_ctx_free(&c); return -1; }
    int npix_all = p->nu * p->nv;
    if (!pixels) n_pixels = npix_all;
    double* mu_e = (double*)malloc(sizeof(double) * (size_t)p->n_bins * p->n_mat);
    double* wr = (double*)malloc(sizeof(double) * (size_t)p->n_bins);
    double* tot = (double*)malloc(sizeof(double) * (size_t)p->n_e);
    double* rsp = (double*)malloc(sizeof(double) * (size_t)p->n_r);
    double wsum = 0.0, fsum = 0.0;
    for (int b = 0; b < p->n_bins; ++b) wsum += p->bin_w[b];
    for (int i = 0; i < p->n_r; ++i) rsp[i] = p->response[i];
    for (int m = 0; m < p->n_mat; ++m) {
        for (int e = 0; e < p->n_e; ++e) {
            const float* t = p->mu_hat + (size_t)m * 3 * p->n_e;
            tot[e] = 0.1 * ((double)t[e] + (double)t[p->n_e + e] + (double)t[2 * p->n_e + e]);
        }
        for (int b = 0; b < p->n_bins; ++b)
            mu_e[(size_t)b * p->n_mat + m] = orc_interp_d(tot, p->e0, p->de, p->n_e, p->bin_e[b]);
    }
    for (int b = 0; b < p->n_bins; ++b)
        wr[b] = (p->bin_w[b] / wsum) * orc_interp_d(rsp, p->r0, p->dr, p->n_r, p->bin_e[b]);
    /* per-column spectra: channel weights phi_u(E) r(E) of each column */
    double* wr_cols = NULL;
    if (p->bin_w_cols) {
        wr_cols = (double*)malloc(sizeof(double) * (size_t)p->nu * p->n_bins);
        for (int u = 0; u < p->nu; ++u) {
            const double* wc = p->bin_w_cols + (size_t)u * p->n_bins;
            double cs = 0.0;
            for (int b = 0; b < p->n_bins; ++b) cs += wc[b];
            for (int b = 0; b < p->n_bins; ++b)
                wr_cols[(size_t)u * p->n_bins + b] = (wc[b] / cs) * orc_interp_d(rsp, p->r0, p->dr, p->n_r, p->bin_e[b]);
        }
    }
    for (int i = 0; i < npix_all; ++i) fsum += p->fluence[i];
    const int dims[3] = {p->nx, p->ny, p->nz};
    const double vox[3] = {p->vx, p->vy, p->vz};
    double* alpha = (double*)malloc(sizeof(double) * (size_t)(p->nx + p->ny + p->nz + 8));
    double* seg_len = (double*)malloc(sizeof(double) * (size_t)(p->nx + p->ny + p->nz + 8));
    int64_t* seg_vox = (int64_t*)malloc(sizeof(int64_t) * (size_t)(p->nx + p->ny + p->nz + 8));
    for (int k = 0; k < n_pixels; ++k) {
        int j = pixels ? pixels[k] : k;
        int iu = j % p->nu, iv = j / p->nu;
        double au = (iu + 0.5 - 0.5 * p->nu) * p->du, av = (iv + 0.5 - 0.5 * p->nv) * p->dv;
        double S[3], d[3], L = 0.0;
        for (int a = 0; a < 3; ++a) {
            S[a] = c.gd.S[a];
            d[a] = c.gd.P[a] + au * c.gd.eu[a] + av * c.gd.ev[a] - S[a];
            L += d[a] * d[a];
        }
        L = sqrt(L);
        for (int a = 0; a < 3; ++a) d[a] /= L;
        double tmin = 0.0, tmax = L;
        int hit = 1;
        for (int a = 0; a < 3; ++a) {
            if (d[a] != 0.0) {
                double t1 = (c.gd.lo[a] - S[a]) / d[a], t2 = (c.gd.hi[a] - S[a]) / d[a];
                if (t1 > t2) { double t = t1; t1 = t2; t2 = t; }
                if (t1 > tmin) tmin = t1;
                if (t2 < tmax) tmax = t2;
            } else if (S[a] < c.gd.lo[a] || S[a] > c.gd.hi[a]) {
                hit = 0;
            }
        }
        int na = 0, nseg = 0;
        if (hit && tmax > tmin) {
            alpha[na++] = tmin;
            alpha[na++] = tmax;
            for (int a = 0; a < 3; ++a) {
                if (d[a] == 0.0) continue;
                for (int i = 0; i <= dims[a]; ++i) {
                    double t = (c.gd.lo[a] + i * vox[a] - S[a]) / d[a];
                    if (t > tmin && t < tmax) alpha[na++] = t;
                }
            }
            qsort(alpha, (size_t)na, sizeof(double), orc_cmp_double);
            for (int i = 0; i + 1 < na; ++i) {
                double len = alpha[i + 1] - alpha[i];
                if (len <= 0.0) continue;
                double tm = 0.5 * (alpha[i] + alpha[i + 1]);
                int64_t vi[3];
                for (int a = 0; a < 3; ++a) {
                    int g = (int)floor((S[a] + tm * d[a] - c.gd.lo[a]) / vox[a]);
                    vi[a] = g < 0 ? 0 : (g > dims[a] - 1 ? dims[a] - 1 : g);
                }
                seg_len[nseg] = len;
                seg_vox[nseg++] = vi[0] + (int64_t)p->nx * (vi[1] + (int64_t)p->ny * vi[2]);
            }
        }
        double sig = 0.0;
        for (int b = 0; b < p->n_bins; ++b) {
            double rad = 0.0;
            for (int s = 0; s < nseg; ++s)
                rad += seg_len[s] * (double)p->density[seg_vox[s]] * mu_e[(size_t)b * p->n_mat + p->material[seg_vox[s]]];
            sig += (wr_cols ? wr_cols[(size_t)iu * p->n_bins + b] : wr[b]) * exp(-rad);
        }
        out[k] = (p->fluence[j] / fsum) * sig;
    }
    free(alpha); free(seg_len); free(seg_vox);
    free(mu_e); free(wr); free(wr_cols); free(tot); free(rsp);
    orc_ctx_free(&c);
    return 0;
}

int orc_rt_primary(const orc_problem* p, double phi, const int32_t* pixels, int n_pixels, double* out) {
    orc_ctx c;
    if (orc_ctx_init(&c, p, phi)) { orc_ctx_free(&c); return -1; }
    int npix_all = p->nu * p->nv;
    if (!pixels) n_pixels = npix_all;
    /* per-channel total mass attenuation per material (mm^-1 per g/cm^3),
     * spectrum weight phi and response r at the channel energy */
    double* mu_e = (double*)malloc(sizeof(double) * (size_t)p->n_bins * p->n_mat);
    double* wr = (double*)malloc(sizeof(double) * (size_t)p->n_bins);
    double wsum = 0.0;
    for (int b = 0; b < p->n_bins; ++b) wsum += p->bin_w[b];
    double* tot = (double*)malloc(sizeof(double) * (size_t)p->n_e);
    double* rsp = (double*)malloc(sizeof(double) * (size_t)p->n_r);
    for (int i = 0; i < p->n_r; ++i) rsp[i] = p->response[i];
    for (int m = 0; m < p->n_mat; ++m) {
        for (int e = 0; e < p->n_e; ++e) {
            const float* t = p->mu_hat + (size_t)m * 3 * p->n_e;
            tot[e] = 0.1 * ((double)t[e] + (double)t[p->n_e + e] + (double)t[2 * p->n_e + e]);
        }
        for (int b = 0; b < p->n_bins; ++b)
            mu_e[(size_t)b * p->n_mat + m] = orc_interp_d(tot, p->e0, p->de, p->n_e, p->bin_e[b]);
    }
    for (int b = 0; b < p->n_bins; ++b)
        wr[b] = (p->bin_w[b] / wsum) * orc_interp_d(rsp, p->r0, p->dr, p->n_r, p->bin_e[b]);
    /* per-column spectra: channel weights phi_u(E) r(E) of each column */
    double* wr_cols = NULL;
    if (p->bin_w_cols) {
        wr_cols = (double*)malloc(sizeof(double) * (size_t)p->nu * p->n_bins);
        for (int u = 0; u < p->nu; ++u) {
            const double* wc = p->bin_w_cols + (size_t)u * p->n_bins;
            double cs = 0.0;
            for (int b = 0; b < p->n_bins; ++b) cs += wc[b];
            for (int b = 0; b < p->n_bins; ++b)
                wr_cols[(size_t)u * p->n_bins + b] = (wc[b] / cs) * orc_interp_d(rsp, p->r0, p->dr, p->n_r, p->bin_e[b]);
        }
    }
    double fsum = 0.0;
    for (int i = 0; i < npix_all; ++i) fsum += p->fluence[i];
    double vmin = p->vx < p->vy ? p->vx : p->vy;
    if (p->vz < vmin) vmin = p->vz;

    for (int k = 0; k < n_pixels; ++k) {
        int j = pixels ? pixels[k] : k;
        int iu = j % p->nu, iv = j / p->nu;
        double au = (iu + 0.5 - 0.5 * p->nu) * p->du;
        double av = (iv + 0.5 - 0.5 * p->nv) * p->dv;
        double d[3], S[3];
        double L = 0.0;
        for (int a = 0; a < 3; ++a) {
            S[a] = c.gd.S[a];
            d[a] = c.gd.P[a] + au * c.gd.eu[a] + av * c.gd.ev[a] - S[a];
            L += d[a] * d[a];
        }
        L = sqrt(L);
        for (int a = 0; a < 3; ++a) d[a] /= L;
        double tmin = 0.0, tmax = L;
        int hit = 1;
        for (int a = 0; a < 3; ++a) {
            if (d[a] != 0.0) {
                double t1 = (c.gd.lo[a] - S[a]) / d[a], t2 = (c.gd.hi[a] - S[a]) / d[a];
                if (t1 > t2) { double t = t1; t1 = t2; t2 = t; }
                if (t1 > tmin) tmin = t1;
                if (t2 < tmax) tmax = t2;
            } else if (S[a] < c.gd.lo[a] || S[a] > c.gd.hi[a]) {
                hit = 0;
            }
        }
        double chord = (hit && tmax > tmin) ? tmax - tmin : 0.0;
        int nint = chord > 0.0 ? (int)ceil(chord / (0.5 * vmin)) : 0;
        double dl = nint > 0 ? chord / nint : 0.0;
        double sig = 0.0;
        for (int b = 0; b < p->n_bins; ++b) {
            double rad = 0.0;
            for (int s = 0; s < nint; ++s) {
                double tt = tmin + (s + 0.5) * dl, x[3];
                for (int a = 0; a < 3; ++a) x[a] = S[a] + tt * d[a];
                rad += dl * orc_mu_at(&c, x, &mu_e[(size_t)b * p->n_mat]);
            }
            sig += (wr_cols ? wr_cols[(size_t)iu * p->n_bins + b] : wr[b]) * exp(-rad);
        }
        out[k] = (p->fluence[j] / fsum) * sig;
    }
    free(mu_e); free(wr); free(wr_cols); free(tot); free(rsp);
    orc_ctx_free(&c);
    return 0;
}
