// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gdrr.h"

namespace gdrr {

// Voxel records are stored in bricks of 4 x 2 x 2 voxels (16 records of 8
// bytes = one 128-byte line), bricks x fastest.  The record of voxel (x, y, z)
// sits at brick_x(x) + brick_y(y, bsy) + brick_z(z, bsz) with bsy = 16 * nbx,
// bsz = 16 * nbx * nby (nbx, nby: bricks per row and per column).
__host__ __device__ __forceinline__ int brick_x(int x) { return ((x >> 2) << 4) + (x & 3); }
__host__ __device__ __forceinline__ int brick_y(int y, int bsy) { return (y >> 1) * bsy + ((y & 1) << 2); }
__host__ __device__ __forceinline__ int brick_z(int z, int bsz) { return (z >> 1) * bsz + ((z & 1) << 3); }

// Philox4x32-10 round keys of a seed: k_r = (lo + r * 0x9E3779B9, hi + r * 0xBB67AE85).
struct RoundKeys {
    uint32_t k0[10], k1[10];
};

inline RoundKeys round_keys(uint64_t seed) {
    RoundKeys rk;
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = (uint32_t)seed + (uint32_t)r * 0x9E3779B9u;
        rk.k1[r] = (uint32_t)(seed >> 32) + (uint32_t)r * 0xBB67AE85u;
    }
    return rk;
}

// Per-angle imager frame in FP32 (Section 2.1, Fig. 1).
struct Frame {
    float S[3];    // source position
    float n[3];    // imager normal, direction OP
    float P[3];    // imager centre
    float eu[3];   // detector u axis
    float ev[3];   // detector v axis (z)
};

// One angle of a (possibly batched) transport launch.
struct Job {
    Frame f;
    uint32_t angle_index;
    uint32_t pad;
    uint64_t first;        // first flattened history of this job
    uint64_t count;        // histories of this job
    uint64_t hid_offset;   // history id of the job's first history
    int64_t* tally_p;      // [nv*nu]
    int64_t* tally_s;      // [nv*nu]
};

// Everything the transport kernel reads, by value.
struct McParams {
    // phantom box and bricked voxel records {density bits, material}
    int nx, ny, nz;
    int bsy, bsz;
    float lo[3], hi[3], ivox[3];
    const uint2* vox;
    // material tables, mm^-1 per g/cm^3, [m][k][e]; majorant nodes [e]
    int n_mat, n_e;
    float e0, inv_de;
    const float* tab;
    const float* major;
    // detector response
    int n_r;
    float r0, inv_dr;
    const float* resp;
    // source: pixel and energy inverse CDFs with guide tables
    int npix, n_guide_pix;
    const uint32_t* kcdf_pix;      // floor(cdf * 2^24): integer thresholds of the inverse CDF
    const int* guide_pix;
    int n_bins, n_guide_e;
    const uint32_t* kcdf_e;        // [n_bins], or [nu][n_bins] with per-column spectra
    const int* guide_e;            // [n_guide_e], or [nu][n_guide_e]
    int e_col;                     // 1: the energy tables hold one row per detector column
    const float* bin_e;
    // detector grid
    int nu, nv;
    float hu, hv, du, dv, idu, idv;
    // options
    float e_cut;
    int max_steps;
    RoundKeys rk;                  // Philox round keys of the seed
    // jobs
    const Job* jobs;
    int n_jobs;
    uint64_t total;                // sum of job counts
    unsigned long long* counter;   // work counter (flattened histories claimed)
    unsigned long long* stats;     // GDRR_NSTATS
    gdrr_history_record* records;  // NULL or [total]
    int chunk;                     // histories a warp claims at a time
    int batch_min;                 // waiting lanes that trigger a warp's service batch
    int nearest_voxel;             // 1: each point takes its voxel's value (no interpolation)
    int scatter_filter;            // 0 all scatter, 1 single Compton, 2 single Rayleigh, 3 multiple
    // Rayleigh form factors (ray_ff = 1): nodes s_j = x_j^2, cumulative A and
    // F^2 per material [m][n_ff], 1/(hc) and 1/dx
    int ray_ff, n_ff;
    const float* ff_s;
    const float* ff_a;
    const float* ff_g;
    float inv_hc, ff_idx;
    // macro cells of 2^cshift voxels per edge: per cell and material the
    // largest density over the voxels [c 2^s, (c + 1) 2^s] of each axis (the
    // cell and the next voxel), [cell][NM] with NM the kernel's material
    // slots; NULL disables the early virtual-collision test
    const float* cells;
    int cshift, ncx, ncy, ncz;
    // local majorants (lm = 1): the cell bounds serve as the free flights'
    // majorant; the cells' planes need the voxel edges
    int lm;
    float vox_mm[3];
    int* status;                   // NULL, or where a bounded loop that gave up records it
    int pool_tail, pool_park_min;  // pool form: tail width and parking minimum (0: defaults)
    // the launch covers flattened histories seg0 .. seg0 + total - 1; with src
    // != NULL their source points were sampled by the source pass: src[2 i],
    // src[2 i + 1] = {px, py, pz, dx}, {dy, dz, E, job + 1 as bits, or 0 when
    // the history ended there} for history seg0 + i
    uint64_t seg0;
    const float4* src;
};

// Bounded waits on flags that another CTA publishes (release store, acquire
// load, both at GPU scope).  Every spin ends after limit_ns nanoseconds of
// %globaltimer, so a flag that is never set costs a bounded delay and a
// recorded timeout, not a hung GPU.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until flags[j] >= want for the neighbour bands j = b - 1 and b + 1
// that exist (0 <= j < G); false once limit_ns has passed.
__device__ __forceinline__ bool wait_band_neighbours(const unsigned* flags, int b, int G, unsigned want,
                                                     unsigned long long limit_ns) {
    const unsigned long long t0 = globaltimer_ns();
    for (int j = b - 1; j <= b + 1; j += 2) {
        if (j < 0 || j >= G) continue;
        while (ld_acquire_u32(flags + j) < want) {
            if (globaltimer_ns() - t0 > limit_ns) return false;
        }
    }
    return true;
}

// Material slots of the transport kernel (and of a macro-cell record) for
// n_mat materials: 2, 4 or 8.
__host__ __device__ __forceinline__ int material_slots(int n_mat) { return n_mat <= 2 ? 2 : (n_mat <= 4 ? 4 : 8); }

// Ray-tracing parameters.
struct RtParams {
    int nx, ny, nz;
    int bsy, bsz;
    float lo[3], hi[3], ivox[3];
    const uint2* vox;
    int n_mat, n_bins;
    const float* mu_rt;     // [n_bins][n_mat] total mu_hat at the channel energy, mm^-1 per g/cm^3
    const float* wr;        // [n_bins] phi_b r(E_b), phi normalised
    const float* wr_cols;   // NULL, or [nu][n_bins] per-column phi_b r(E_b)
    const double* wnorm;    // [npix] normalised fluence
    int nu, nv;
    float hu, hv, du, dv;
    float half_step;        // half the smallest voxel size
    Frame f;
};

cudaError_t launch_mc(const McParams& p, int block, int grid, bool records, cudaStream_t s);
// The source pass of the lane form (default options, no records): samples
// the source point, direction and energy of histories p.seg0 .. p.seg0 +
// p.total - 1 into p.src, and tallies and counts those that miss the box.
cudaError_t launch_mc_source(const McParams& p, cudaStream_t s);
constexpr size_t MC_SRC_BYTES = 32;    // bytes of one history's source record
int mc_occupancy_blocks(int n_mat, int block, bool records, bool lm);
// The photon-pool form of the transport (default options, no records):
// blocks of pool_threads() threads, per_thread photons per thread in the
// shared-memory pool; 0 blocks per SM when the pool does not fit.
cudaError_t launch_mc_pool(const McParams& p, int per_thread, int grid, cudaStream_t s);
int mc_pool_occupancy_blocks(int n_mat, int per_thread);
int pool_threads();
cudaError_t launch_rt(const RtParams& p, double* out, cudaStream_t s);
cudaError_t launch_rt_siddon(const RtParams& p, double* out, cudaStream_t s);
cudaError_t launch_air(const RtParams& p, double* out, cudaStream_t s);
cudaError_t launch_gather_probe(const McParams& p, uint64_t n_cells, int grid, unsigned int* sink, cudaStream_t s);
cudaError_t launch_stream_words(uint64_t seed, uint32_t angle_index, uint64_t hid0, int n_hist,
                                int n_blocks, uint32_t* out, cudaStream_t s);

cudaError_t launch_finalize(const int64_t* t, int64_t n, double scale, double* out, int* bad, cudaStream_t s);
cudaError_t launch_bin(const int64_t* t, int nu, int nv, int f, int64_t* out, cudaStream_t s);
cudaError_t launch_upsample(const double* c, int cu, int cv, int f, double* out, cudaStream_t s);
cudaError_t launch_noise(const double* ph, const double* p, const double* sh, const double* sc, int64_t n,
                         double alpha, double* out, cudaStream_t s);
// Eq. 5 denoiser, one launch per iteration: scratch of denoise_scratch_doubles
// doubles; count scale and beta from scal_dev[0], [1] when scal_dev is not
// NULL, else the host values.
cudaError_t launch_denoise(const double* s_hat, double* s, int nu, int nv, double count_scale, double beta,
                           const double* scal_dev, double omega, int iters, double* scratch, cudaStream_t stream);
size_t denoise_scratch_doubles(int nu, int nv);
// Eq. 5 denoiser in one cooperative launch (images that fit its row bands):
// scratch of denoise_fused_scratch_bytes; a wait that gives up sets *status.
bool denoise_fused_fits(int nu, int nv);
size_t denoise_fused_scratch_bytes(int nu, int nv);
cudaError_t launch_denoise_fused(const double* s_hat, double* s_out, int nu, int nv, double count_scale,
                                 double beta, const double* scal_dev, double omega, int iters, void* scratch,
                                 int* status, cudaStream_t stream);
// gdrr_project's Step 3 scalars from the coarse scatter tally and the counters.
cudaError_t launch_project_scalars(const int64_t* coarse, int n, const unsigned long long* stats,
                                   double tally_to_signal, double inv_n_photons, double beta, double smoothing_px,
                                   double floor_, double* scal, cudaStream_t s);
cudaError_t launch_scale_to_f32(const double* a, int64_t n, double scale, float* out, cudaStream_t s);
cudaError_t launch_scale_to_f64(const float* a, int64_t n, double scale, double* out, cudaStream_t s);

}  // namespace gdrr
