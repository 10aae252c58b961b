// Host side of libgdrr: the C ABI declared in include/gdrr.h.
//
// gdrr_create validates and deep-copies the inputs of Section 2.1.  The voxel
// phantom is copied as is and staged by one device kernel (validation, the
// per-material maximum density, the bricked records); the derived tables are
// built on the host in FP64 (material coefficients in mm^-1, the Woodcock
// majorant, inverse-CDF tables of the fluence map and of the spectrum or the
// per-column spectra, the ray-tracing channel tables).  Every other call only
// enqueues kernels on the context stream, apart from the documented
// synchronising ones.
#include <math.h>
#include <cmath>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <mutex>
#include <new>
#include <vector>

#include "gdrr_internal.cuh"

using namespace gdrr;

// What gdrr_project reads back at its end (pinned host memory).
struct ProjHost {
    double scal[8];                         // count scale, beta, mean count, below floor, scattered photons
    unsigned long long stats[GDRR_NSTATS];
    int overflow;
    int status;
};

struct gdrr_ctx {
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;    // the device's pool for the context's device memory
    int device = 0;
    int n_sm = 0;
    // inputs (host copies of the scalars)
    gdrr_geometry geo{};
    int nx = 0, ny = 0, nz = 0;
    int bsy = 0, bsz = 0;          // brick strides of the staged voxel records
    double vox[3] = {0, 0, 0};
    int n_mat = 0, n_e = 0, n_r = 0, n_bins = 0;
    double e0 = 0, de = 0, r0 = 0, dr = 0;
    // staged device data: one 8-byte record {density bits, material} per voxel
    uint2* d_vox = nullptr;
    float* d_tab = nullptr;
    float* d_major = nullptr;
    float* d_resp = nullptr;
    float* d_bin_e = nullptr;
    uint32_t* d_kcdf_pix = nullptr;
    int* d_guide_pix = nullptr;
    uint32_t* d_kcdf_e = nullptr;
    int* d_guide_e = nullptr;
    double* d_wnorm = nullptr;
    float* d_mu_rt = nullptr;
    float* d_wr = nullptr;
    float* d_wr_cols = nullptr;   // [nu][n_bins] with per-column spectra, else NULL
    // Rayleigh form factors: nodes s_j = x_j^2 [n_ff], cumulative and F^2 [m][n_ff]
    float* d_ff_s = nullptr;
    float* d_ff_a = nullptr;
    float* d_ff_g = nullptr;
    int n_ff = 0;
    float ff_idx = 0.0f;
    // macro-cell table of the early virtual-collision test (NULL: none)
    float* d_cells = nullptr;
    int cell_shift = -1, ncx = 0, ncy = 0, ncz = 0;
    int n_scans = 0;              // live scans, which captured the table pointers
    int e_col = 0;                // 1: energy CDFs hold one row per detector column
    int n_guide_pix = 0, n_guide_e = 0;
    // scratch owned by the context
    unsigned long long* d_counter = nullptr;
    unsigned long long* d_stats = nullptr;   // used when the caller passes none
    int* d_flag = nullptr;
    Job* d_jobs = nullptr;
    int jobs_cap = 0;
    double* d_denoise = nullptr;
    size_t denoise_cap = 0;          // bytes
    int64_t* d_tune = nullptr;       // autotuner scratch tallies, 2 * nu * nv
    int* d_status = nullptr;         // timeouts of bounded device waits since the last gdrr_sync
    void* d_arena = nullptr;         // one allocation holding the tables and counters above
    float4* d_src = nullptr;         // source records of the lane form's source pass
    uint64_t src_cap = 0;            // ... in histories
    // gdrr_project scratch: tallies, coarse tally and images, device scalars,
    // and the pinned host block the scalars come back through
    void* d_proj = nullptr;
    ProjHost* h_proj = nullptr;      // page-locked, from the reuse list
    size_t h_proj_cap = 0;
    cudaEvent_t ev_proj[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};   // step / transport / denoise
    // gdrr_project's side stream (the ray trace, beside the transport) and
    // its fork and join events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    gdrr_mc_options opt{};
};

// A multi-angle scan captured once as a CUDA graph: (optionally) zero the
// tallies, reset the work counter, run the persistent transport kernel over
// all angles.  Replays reuse the captured launch configuration and buffers.
struct gdrr_scan {
    gdrr_ctx* ctx = nullptr;
    gdrr::Job* d_jobs = nullptr;
    unsigned long long* d_counter = nullptr;
    unsigned long long* d_stats = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t total = 0;
    float4* d_src = nullptr;  // the scan's own source records (the graph captured the pointer)
    uint64_t src_cap = 0;
    bool counted = false;     // included in ctx->n_scans
};

namespace {

// The device status record: bits 1 and 2, a bounded wait or loop that gave
// up (GDRR_ERR_TIMEOUT); bit 4, a failed self-check of the transport's
// photon bookkeeping (GDRR_ERR_CUDA).
int status_code(int status) { return (status & 4) ? GDRR_ERR_CUDA : GDRR_ERR_TIMEOUT; }

int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return GDRR_OK;
    return e == cudaErrorMemoryAllocation ? GDRR_ERR_OOM : GDRR_ERR_CUDA;
}

// Device memory of contexts.  Each device gets one stream-ordered pool, made
// on first use, that keeps the blocks its contexts free (its release
// threshold is the largest value): a context made after another one reuses
// those blocks instead of mapping new memory (the transport's source records
// alone take 3.2 GB at 1e8 histories), and destroying a context frees on its
// stream instead of waiting for the device at every buffer.
// gdrr_release_memory hands the unused blocks back.
constexpr int MAX_POOL_DEVICES = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pool[MAX_POOL_DEVICES] = {};

cudaError_t device_pool(int dev, cudaMemPool_t* out) {
    if (dev < 0 || dev >= MAX_POOL_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pool[dev] = p;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

// A context buffer of the given size from its device's pool, ordered on the
// context's stream; and its release, ordered after the work queued there.
cudaError_t dalloc(const gdrr_ctx* c, void** p, size_t bytes) {
    return cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 1), c->pool, c->stream);
}
template <typename T>
cudaError_t dalloc(const gdrr_ctx* c, T** p, size_t bytes) {
    return dalloc(c, reinterpret_cast<void**>(p), bytes);
}
void dfree(const gdrr_ctx* c, void* p) {
    if (p) cudaFreeAsync(p, c->stream);
}

// Page-locked host blocks (staging of the context's tables, the staging
// kernel's counters, gdrr_project's scalars), kept for reuse: a page-locked
// allocation costs far more than the copies it serves, and contexts come and
// go.  take_pinned hands out the smallest free block that is large enough.
struct Pinned {
    void* p = nullptr;
    size_t cap = 0;
};
std::mutex g_host_mutex;
std::vector<Pinned> g_host_free;

Pinned take_pinned(size_t bytes) {
    {
        std::lock_guard<std::mutex> lock(g_host_mutex);
        size_t best = g_host_free.size();
        for (size_t i = 0; i < g_host_free.size(); ++i)
            if (g_host_free[i].cap >= bytes && (best == g_host_free.size() || g_host_free[i].cap < g_host_free[best].cap))
                best = i;
        if (best < g_host_free.size()) {
            const Pinned b = g_host_free[best];
            g_host_free.erase(g_host_free.begin() + (std::ptrdiff_t)best);
            return b;
        }
    }
    Pinned b;
    b.cap = std::max<size_t>(bytes, 4096);
    if (cudaMallocHost(&b.p, b.cap) != cudaSuccess) {
        cudaGetLastError();
        return Pinned();
    }
    return b;
}

void give_pinned(Pinned b) {
    if (!b.p) return;
    std::lock_guard<std::mutex> lock(g_host_mutex);
    g_host_free.push_back(b);
}

#define TRY_CUDA(x)                               \
    do {                                          \
        cudaError_t _e = (x);                     \
        if (_e != cudaSuccess) return cuda_err(_e); \
    } while (0)

template <typename T>
int upload(const gdrr_ctx* c, T** dst, const T* src, size_t n) {
    TRY_CUDA(dalloc(c, dst, std::max<size_t>(n, 1) * sizeof(T)));
    if (n) TRY_CUDA(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return GDRR_OK;
}

// The context's small tables and counters in one device allocation, staged
// in one page-locked host block and copied once: each piece starts on a
// 256-byte boundary; pieces without source data are zero.  The sources must
// stay alive until commit, which waits for the copy.
struct Arena {
    struct Piece {
        const void* src;
        size_t off, bytes;
    };
    std::vector<Piece> pieces;
    std::vector<std::function<void(char*)>> bind;
    size_t size = 0;
    template <typename T>
    void add(T** dst, const T* src, size_t n) {
        const size_t off = (size + 255) / 256 * 256;
        const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
        pieces.push_back({n ? src : nullptr, off, bytes});
        size = off + bytes;
        bind.push_back([dst, off](char* base) { *dst = reinterpret_cast<T*>(base + off); });
    }
    int commit(const gdrr_ctx* c, void** base) {
        Pinned st = take_pinned(size);
        std::vector<char> pageable;                   // only when page-locked memory is short
        char* h = static_cast<char*>(st.p);
        if (!h) {
            pageable.resize(size);
            h = pageable.data();
        }
        memset(h, 0, size);
        for (const Piece& q : pieces)
            if (q.src) memcpy(h + q.off, q.src, q.bytes);
        cudaError_t e = dalloc(c, base, size);
        if (e == cudaSuccess) e = cudaMemcpyAsync(*base, h, size, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        give_pinned(st);
        TRY_CUDA(e);
        for (auto& b : bind) b(static_cast<char*>(*base));
        return GDRR_OK;
    }
};

// Device staging of the voxel phantom: one thread per voxel (x fastest)
// checks its material index and density, raises its block's maximum density
// for the material (float bits of non-negative values order like the
// values, so an unsigned atomicMax is exact), and writes its 8-byte record to
// the bricked layout; each block then raises the global maxima once per
// material.  aux[0] counts invalid voxels; aux[1 + m] holds material m's
// maximum density bits.
__global__ void stage_voxels_kernel(const uint8_t* __restrict__ mat, const float* __restrict__ den, int nx, int ny,
                                    int nz, int n_mat, int bsy, int bsz, uint2* __restrict__ vox,
                                    unsigned int* __restrict__ aux) {
    __shared__ unsigned int s_max[GDRR_MAX_MATERIALS];
    __shared__ unsigned int s_bad;
    if (threadIdx.x < GDRR_MAX_MATERIALS) s_max[threadIdx.x] = 0u;
    if (threadIdx.x == 0) s_bad = 0u;
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)nx * ny * nz;
    if (v < n) {
        const int x = (int)(v % nx);
        const int y = (int)((v / nx) % ny);
        const int z = (int)(v / ((int64_t)nx * ny));
        const uint32_t m = mat[v];
        const float d = den[v];
        // -0 is stored as +0 so that the float bits order like the values
        const uint32_t bits = d == 0.0f ? 0u : __float_as_uint(d);
        if (m >= (uint32_t)n_mat || !(d >= 0.0f) || !isfinite(d)) {
            atomicAdd(&s_bad, 1u);
        } else {
            atomicMax(&s_max[m], bits);
            vox[(size_t)brick_x(x) + brick_y(y, bsy) + brick_z(z, bsz)] = make_uint2(bits, m);
        }
    }
    __syncthreads();
    if (threadIdx.x < n_mat && s_max[threadIdx.x]) atomicMax(aux + 1 + threadIdx.x, s_max[threadIdx.x]);
    if (threadIdx.x == 0 && s_bad) atomicAdd(aux, s_bad);
}

// Macro-cell table of the early virtual-collision test.  Cell c of an axis
// covers voxels [c 2^shift, (c + 1) 2^shift] (its own and the next one): the
// corners a point can touch whose lower corner lies in the cell.  Each voxel
// raises its material's entry in every cell that covers it (at most two per
// axis); float bits of non-negative densities order like the values, so an
// unsigned atomicMax is exact.  cells: zeroed [cell][slots] words.
__global__ void build_cells_kernel(const uint2* __restrict__ vox, int nx, int ny, int nz, int bsy, int bsz, int shift,
                                   int ncx, int ncy, int slots, unsigned int* __restrict__ cells) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (int64_t)nx * ny * nz) return;
    const int x = (int)(v % nx);
    const int y = (int)((v / nx) % ny);
    const int z = (int)(v / ((int64_t)nx * ny));
    const uint2 r = vox[(size_t)brick_x(x) + brick_y(y, bsy) + brick_z(z, bsz)];
    if (r.x == 0u) return;                       // zero density raises nothing
    const int mask = (1 << shift) - 1;
    const int cx1 = x >> shift, cy1 = y >> shift, cz1 = z >> shift;
    const int cx0 = (x > 0 && (x & mask) == 0) ? cx1 - 1 : cx1;
    const int cy0 = (y > 0 && (y & mask) == 0) ? cy1 - 1 : cy1;
    const int cz0 = (z > 0 && (z & mask) == 0) ? cz1 - 1 : cz1;
    for (int cz = cz0; cz <= cz1; ++cz)
        for (int cy = cy0; cy <= cy1; ++cy)
            for (int cx = cx0; cx <= cx1; ++cx)
                atomicMax(cells + ((size_t)(cz * ncy + cy) * ncx + cx) * slots + r.y, r.x);
}

// (Re)build the macro-cell table for cells of 2^shift voxels per edge, or
// drop it (shift < 0).  Synchronises the context stream.
int build_cells(gdrr_ctx* c, int shift, bool sync) {
    cudaStream_t s = c->stream;
    if (sync && cudaStreamSynchronize(s) != cudaSuccess) return GDRR_ERR_CUDA;
    dfree(c, c->d_cells);
    c->d_cells = nullptr;
    c->cell_shift = -1;
    if (shift < 0) return GDRR_OK;
    const int ncx = ((c->nx - 1) >> shift) + 1, ncy = ((c->ny - 1) >> shift) + 1, ncz = ((c->nz - 1) >> shift) + 1;
    const int slots = material_slots(c->n_mat);
    const size_t bytes = (size_t)ncx * ncy * ncz * slots * sizeof(float);
    if (dalloc(c, &c->d_cells, bytes) != cudaSuccess) {
        c->d_cells = nullptr;
        return GDRR_ERR_OOM;
    }
    int rc = cuda_err(cudaMemsetAsync(c->d_cells, 0, bytes, s));
    if (!rc) {
        const int64_t nvox = (int64_t)c->nx * c->ny * c->nz;
        const int block = 256;
        build_cells_kernel<<<(unsigned)((nvox + block - 1) / block), block, 0, s>>>(
            c->d_vox, c->nx, c->ny, c->nz, c->bsy, c->bsz, shift, ncx, ncy, slots,
            reinterpret_cast<unsigned int*>(c->d_cells));
        rc = cuda_err(cudaGetLastError());
    }
    if (!rc && sync) rc = cuda_err(cudaStreamSynchronize(s));
    if (rc) {
        dfree(c, c->d_cells);
        c->d_cells = nullptr;
        return rc;
    }
    c->cell_shift = shift;
    c->ncx = ncx; c->ncy = ncy; c->ncz = ncz;
    return GDRR_OK;
}

// Copy the host phantom to the device and stage it into ctx->d_vox (n_rec
// bricked records, padding zero).  Returns the per-material maximum density
// in rho_max, or GDRR_ERR_INVALID_ARG when a voxel is invalid.  Synchronises.
// Queues the phantom's staging on the context stream: the copies, the staging
// kernel and the read-back of its counters into aux (page-locked, 1 + n_mat
// words), which are valid once the stream has been synchronised; then
// stage_phantom_finish checks them.
int stage_phantom(gdrr_ctx* c, const gdrr_phantom& ph, size_t n_rec, unsigned int* aux) {
    const int64_t nvox = (int64_t)ph.nx * ph.ny * ph.nz;
    cudaStream_t s = c->stream;
    // the inputs staged in one temporary allocation: densities, counters,
    // material indices (each on a 256-byte boundary)
    const size_t den_bytes = (size_t)nvox * sizeof(float);
    const size_t aux_off = (den_bytes + 255) / 256 * 256;
    const size_t mat_off = aux_off + 256 * (size_t)((sizeof(unsigned int) * (1 + c->n_mat) + 255) / 256);
    char* d_tmp = nullptr;
    float* d_den = nullptr;
    unsigned int* d_aux = nullptr;
    uint8_t* d_mat = nullptr;
    int rc = GDRR_OK;
    const size_t aux_bytes = sizeof(unsigned int) * (1 + (size_t)c->n_mat);
    do {
        if ((rc = cuda_err(dalloc(c, &c->d_vox, n_rec * sizeof(uint2))))) break;
        if ((rc = cuda_err(cudaMemsetAsync(c->d_vox, 0, n_rec * sizeof(uint2), s)))) break;
        if ((rc = cuda_err(dalloc(c, &d_tmp, mat_off + (size_t)nvox)))) break;
        d_den = reinterpret_cast<float*>(d_tmp);
        d_aux = reinterpret_cast<unsigned int*>(d_tmp + aux_off);
        d_mat = reinterpret_cast<uint8_t*>(d_tmp + mat_off);
        if ((rc = cuda_err(cudaMemcpyAsync(d_den, ph.density, den_bytes, cudaMemcpyHostToDevice, s)))) break;
        if ((rc = cuda_err(cudaMemcpyAsync(d_mat, ph.material, (size_t)nvox, cudaMemcpyHostToDevice, s)))) break;
        if ((rc = cuda_err(cudaMemsetAsync(d_aux, 0, aux_bytes, s)))) break;
        const int block = 256;
        stage_voxels_kernel<<<(unsigned)((nvox + block - 1) / block), block, 0, s>>>(
            d_mat, d_den, ph.nx, ph.ny, ph.nz, c->n_mat, c->bsy, c->bsz, c->d_vox, d_aux);
        if ((rc = cuda_err(cudaGetLastError()))) break;
        if ((rc = cuda_err(cudaMemcpyAsync(aux, d_aux, aux_bytes, cudaMemcpyDeviceToHost, s)))) break;
    } while (0);
    dfree(c, d_tmp);                                  // after the read-back, in stream order
    return rc;
}

// The staging's counters, read back by stage_phantom: any invalid voxel
// rejects the phantom; else each material's largest density.
int stage_phantom_finish(const gdrr_ctx* c, const unsigned int* aux, std::vector<double>& rho_max) {
    if (aux[0]) return GDRR_ERR_INVALID_ARG;
    rho_max.assign(c->n_mat, 0.0);
    for (int m = 0; m < c->n_mat; ++m) {
        float r;
        memcpy(&r, &aux[1 + m], sizeof r);
        rho_max[m] = (double)r;
    }
    return GDRR_OK;
}

// Inverse-CDF table of non-negative weights: running FP64 sum, divided by the
// total (last entry exactly 1).  Empty vector on invalid weights.
std::vector<double> build_cdf(const double* w, int n) {
    std::vector<double> c(n);
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(w[i] >= 0.0) || !std::isfinite(w[i])) return {};
        s += w[i];
        c[i] = s;
    }
    if (!(s > 0.0)) return {};
    for (int i = 0; i < n; ++i) c[i] = c[i] / s;
    return c;
}

// Integer thresholds of an inverse CDF: a uniform xi = k 2^-24 (k integer,
// 1 <= k <= 2^24) satisfies xi <= cdf[j] exactly when k <= floor(cdf[j] 2^24),
// since cdf[j] 2^24 is exact in FP64.
std::vector<uint32_t> kcdf_of(const std::vector<double>& cdf) {
    std::vector<uint32_t> k(cdf.size());
    for (size_t i = 0; i < cdf.size(); ++i) {
        const double v = floor(ldexp(cdf[i], 24));
        k[i] = (uint32_t)std::min(v, 16777216.0);
    }
    return k;
}

// Guide table: g[i] = first j with cdf[j] >= i / G (a starting point only;
// the device search corrects it in both directions).
std::vector<int> build_guide(const std::vector<double>& cdf, int G) {
    std::vector<int> g(G);
    int j = 0;
    const int n = (int)cdf.size();
    for (int i = 0; i < G; ++i) {
        const double t = (double)i / (double)G;
        while (j < n - 1 && cdf[j] < t) ++j;
        g[i] = j;
    }
    return g;
}

// The imager frame at gantry angle phi (Fig. 1), computed in FP64, stored FP32.
Frame make_frame(const gdrr_geometry& g, double phi) {
    const double ang = phi + g.theta_rad, aid = g.sdd_mm - g.sad_mm;
    const double S[3] = {-g.sad_mm * cos(phi), -g.sad_mm * sin(phi), 0.0};
    const double n[3] = {cos(ang), sin(ang), 0.0};
    const double P[3] = {aid * cos(ang), aid * sin(ang), 0.0};
    const double eu[3] = {sin(ang), -cos(ang), 0.0};
    const double ev[3] = {0.0, 0.0, 1.0};
    Frame f;
    for (int k = 0; k < 3; ++k) {
        f.S[k] = (float)S[k]; f.n[k] = (float)n[k]; f.P[k] = (float)P[k];
        f.eu[k] = (float)eu[k]; f.ev[k] = (float)ev[k];
    }
    return f;
}

// The source must be outside the voxel box and the whole box (and source)
// strictly on the source side of the imager plane.
bool geometry_ok(const gdrr_ctx* c, double phi) {
    const double ang = phi + c->geo.theta_rad, aid = c->geo.sdd_mm - c->geo.sad_mm;
    const double S[3] = {-c->geo.sad_mm * cos(phi), -c->geo.sad_mm * sin(phi), 0.0};
    const double n[3] = {cos(ang), sin(ang), 0.0};
    const double P[3] = {aid * cos(ang), aid * sin(ang), 0.0};
    const int dims[3] = {c->nx, c->ny, c->nz};
    double lo[3], hi[3];
    bool src_in = true;
    for (int k = 0; k < 3; ++k) {
        hi[k] = 0.5 * dims[k] * c->vox[k];
        lo[k] = -hi[k];
        if (!(S[k] > lo[k] && S[k] < hi[k])) src_in = false;
    }
    if (src_in) return false;
    for (int corner = 0; corner < 8; ++corner) {
        double side = 0.0;
        for (int k = 0; k < 3; ++k) side += (((corner >> k) & 1 ? hi[k] : lo[k]) - P[k]) * n[k];
        if (!(side < 0.0)) return false;
    }
    double s_side = 0.0;
    for (int k = 0; k < 3; ++k) s_side += (S[k] - P[k]) * n[k];
    return s_side < 0.0;
}

void fill_box(const gdrr_ctx* c, float lo[3], float hi[3], float ivox[3]) {
    const int dims[3] = {c->nx, c->ny, c->nz};
    for (int k = 0; k < 3; ++k) {
        const double half = 0.5 * dims[k] * c->vox[k];
        lo[k] = (float)(-half);
        hi[k] = (float)half;
        ivox[k] = (float)(1.0 / c->vox[k]);
    }
}

double interp_d(const std::vector<double>& t, double e0, double de, double e) {
    const int n = (int)t.size();
    double fi = (e - e0) / de;
    fi = std::min(std::max(fi, 0.0), (double)(n - 1));
    int i = std::min((int)fi, n - 2);
    const double f = fi - i;
    return t[i] + f * (t[i + 1] - t[i]);
}

void set_defaults(gdrr_mc_options* o) {
    if (o->e_cut_kev <= 0.0) o->e_cut_kev = 1.0;
    if (o->max_steps <= 0) o->max_steps = 100000;
    if (o->block_size <= 0) o->block_size = 256;
    if (o->hist_per_thread <= 0) o->hist_per_thread = 8;
    if (o->batch_min <= 0) o->batch_min = o->local_majorant ? 24 : 16;
    if (o->photon_pool == 0) o->photon_pool = -1;
}

// Default macro cells: about 4 mm on a side, 2^s voxels of the smallest voxel
// edge with s = round(log2(4 mm / edge)) in 1..6.  On the torso, cells of 4 mm
// ran faster than 2, 8 or 16 mm at 1 mm voxels and faster than 8 or 16 mm at
// 2 mm (tighter bounds, fewer gathers, against a larger table that stays in
// L2); the results do not depend on the choice.  With local majorants the
// cells are the flights' majorant and every cell a flight passes costs a
// crossing: about 32 mm by default (on the 2 mm torso, 8, 16, 32 and 64 mm
// cells gave 92.2, 71.8, 70.3 and 87.5 ms per 1e8 histories).
int default_cell_shift(const gdrr_ctx* c, bool local_majorant) {
    const double v = std::min(c->vox[0], std::min(c->vox[1], c->vox[2]));
    const int s = (int)std::lround(std::log2((local_majorant ? 32.0 : 4.0) / v));
    return std::min(6, std::max(1, s));
}

int free_ctx(gdrr_ctx* c) {
    if (!c) return GDRR_OK;
    if (c->side) cudaStreamSynchronize(c->side);   // a projection's ray trace reads the tables
    cudaStreamSynchronize(c->stream);
    void* bufs[] = {c->d_vox, c->d_arena, c->d_jobs, c->d_denoise, c->d_tune,
                    c->d_ff_s, c->d_ff_a, c->d_ff_g, c->d_cells, c->d_proj, c->d_src};
    if (c->pool)
        for (void* b : bufs) dfree(c, b);
    Pinned hp;
    hp.p = c->h_proj;
    hp.cap = c->h_proj_cap;
    give_pinned(hp);
    for (cudaEvent_t e : c->ev_proj)
        if (e) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    delete c;
    return GDRR_OK;
}

}  // namespace

extern "C" {

GDRR_API const char* gdrr_error_string(int code) {
    switch (code) {
        case GDRR_OK: return "ok";
        case GDRR_ERR_INVALID_ARG: return "invalid argument";
        case GDRR_ERR_CUDA: return "CUDA runtime error";
        case GDRR_ERR_OOM: return "device out of memory";
        case GDRR_ERR_TALLY_OVERFLOW: return "int64 tally overflow";
        case GDRR_ERR_STEP_LIMIT: return "histories hit the free-flight limit";
        case GDRR_ERR_UNSUPPORTED: return "unsupported input";
        case GDRR_ERR_TIMEOUT: return "a bounded device-side wait gave up";
        default: return "unknown error";
    }
}

GDRR_API int gdrr_create(const gdrr_geometry* geometry, const gdrr_phantom* phantom,
                         const gdrr_materials* materials, const gdrr_spectrum* spectrum,
                         const gdrr_bowtie* bowtie, const gdrr_detector* detector, void* cuda_stream,
                         gdrr_ctx** out) {
    if (!geometry || !phantom || !materials || !spectrum || !bowtie || !detector || !out)
        return GDRR_ERR_INVALID_ARG;
    const gdrr_geometry& g = *geometry;
    if (!(g.sad_mm > 0 && g.sdd_mm > g.sad_mm && g.nu > 0 && g.nv > 0 && g.du_mm > 0 && g.dv_mm > 0)
        || !std::isfinite(g.theta_rad))
        return GDRR_ERR_INVALID_ARG;
    if ((int64_t)g.nu * g.nv > (1 << 28)) return GDRR_ERR_INVALID_ARG;
    const gdrr_phantom& ph = *phantom;
    if (ph.nx <= 0 || ph.ny <= 0 || ph.nz <= 0 || !(ph.dx_mm > 0 && ph.dy_mm > 0 && ph.dz_mm > 0)
        || !ph.material || !ph.density)
        return GDRR_ERR_INVALID_ARG;
    const int64_t nbrick_rec = (int64_t)16 * ((ph.nx + 3) / 4) * ((ph.ny + 1) / 2) * ((ph.nz + 1) / 2);
    if (nbrick_rec >= ((int64_t)1 << 31)) return GDRR_ERR_UNSUPPORTED;
    const gdrr_materials& mt = *materials;
    if (mt.n_materials <= 0 || mt.n_energies < 2 || !(mt.de_kev > 0) || !mt.mu_hat) return GDRR_ERR_INVALID_ARG;
    if (mt.n_materials > GDRR_MAX_MATERIALS) return GDRR_ERR_UNSUPPORTED;
    const gdrr_spectrum& sp = *spectrum;
    if (sp.n_bins <= 0 || !sp.energy_kev || !sp.weight) return GDRR_ERR_INVALID_ARG;
    if (sp.n_bins > 512) return GDRR_ERR_UNSUPPORTED;
    const gdrr_detector& dt = *detector;
    if (dt.n_energies < 2 || !(dt.de_kev > 0) || !dt.response || !bowtie->fluence) return GDRR_ERR_INVALID_ARG;

    const int64_t nt = (int64_t)mt.n_materials * 3 * mt.n_energies;
    for (int64_t i = 0; i < nt; ++i)
        if (!(mt.mu_hat[i] >= 0.0f) || !std::isfinite(mt.mu_hat[i])) return GDRR_ERR_INVALID_ARG;
    for (int i = 0; i < dt.n_energies; ++i)
        if (!std::isfinite(dt.response[i])) return GDRR_ERR_INVALID_ARG;
    for (int i = 0; i < sp.n_bins; ++i)
        if (!(sp.energy_kev[i] > 0.0) || !std::isfinite(sp.energy_kev[i])) return GDRR_ERR_INVALID_ARG;

    const int npix = g.nu * g.nv;
    std::vector<double> cdf_pix = build_cdf(bowtie->fluence, npix);
    std::vector<double> cdf_e = build_cdf(sp.weight, sp.n_bins);
    if (cdf_pix.empty() || cdf_e.empty()) return GDRR_ERR_INVALID_ARG;
    // per-column spectra (energy-dependent bowtie): one CDF row per column
    const bool e_col = sp.column_weight != nullptr;
    std::vector<std::vector<double>> cdf_cols;
    if (e_col) {
        cdf_cols.resize(g.nu);
        for (int u = 0; u < g.nu; ++u) {
            cdf_cols[u] = build_cdf(sp.column_weight + (size_t)u * sp.n_bins, sp.n_bins);
            if (cdf_cols[u].empty()) return GDRR_ERR_INVALID_ARG;
        }
    }

    gdrr_ctx* c = new (std::nothrow) gdrr_ctx();
    if (!c) return GDRR_ERR_OOM;
    c->stream = (cudaStream_t)cuda_stream;
    c->geo = g;
    c->nx = ph.nx; c->ny = ph.ny; c->nz = ph.nz;
    c->vox[0] = ph.dx_mm; c->vox[1] = ph.dy_mm; c->vox[2] = ph.dz_mm;
    c->n_mat = mt.n_materials; c->n_e = mt.n_energies; c->e0 = mt.e0_kev; c->de = mt.de_kev;
    c->n_r = dt.n_energies; c->r0 = dt.e0_kev; c->dr = dt.de_kev;
    c->n_bins = sp.n_bins;
    set_defaults(&c->opt);
    if (!geometry_ok(c, 0.0)) { delete c; return GDRR_ERR_INVALID_ARG; }

    int rc = GDRR_OK;
    Pinned aux_blk;                   // the staging kernel's counters, read back
    do {
        if (cudaGetDevice(&c->device) != cudaSuccess) { rc = GDRR_ERR_CUDA; break; }
        if ((rc = cuda_err(device_pool(c->device, &c->pool)))) break;
        if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
            rc = GDRR_ERR_CUDA;
            break;
        }
        // material coefficients in mm^-1 per g/cm^3 (mu_hat cm^2/g * 0.1)
        std::vector<float> tab(nt);
        for (int64_t i = 0; i < nt; ++i) tab[i] = (float)((double)mt.mu_hat[i] * 0.1);
        // the phantom is validated, reduced and bricked on the device, and the
        // macro-cell table built from it, while the host builds the tables below
        cudaStream_t s = c->stream;
        const int nbx = (ph.nx + 3) / 4, nby = (ph.ny + 1) / 2, nbz = (ph.nz + 1) / 2;
        c->bsy = 16 * nbx;
        c->bsz = 16 * nbx * nby;
        aux_blk = take_pinned(sizeof(unsigned int) * (1 + (size_t)mt.n_materials));
        if (!aux_blk.p) { rc = GDRR_ERR_OOM; break; }
        unsigned int* aux = static_cast<unsigned int*>(aux_blk.p);
        if ((rc = stage_phantom(c, ph, (size_t)16 * nbx * nby * nbz, aux))) break;
        if (c->opt.cell_shift == 0) c->opt.cell_shift = default_cell_shift(c, false);
        if ((rc = build_cells(c, c->opt.cell_shift, false))) break;
        std::vector<float> bin_e(sp.n_bins);
        for (int b = 0; b < sp.n_bins; ++b) bin_e[b] = (float)sp.energy_kev[b];
        c->n_guide_pix = npix;
        c->n_guide_e = std::max(sp.n_bins, 16);
        std::vector<int> guide_pix = build_guide(cdf_pix, c->n_guide_pix);
        std::vector<int> guide_e;
        std::vector<uint32_t> kcdf_e;
        if (e_col) {
            for (int u = 0; u < g.nu; ++u) {
                const std::vector<int> gu = build_guide(cdf_cols[u], c->n_guide_e);
                const std::vector<uint32_t> ku = kcdf_of(cdf_cols[u]);
                guide_e.insert(guide_e.end(), gu.begin(), gu.end());
                kcdf_e.insert(kcdf_e.end(), ku.begin(), ku.end());
            }
        } else {
            guide_e = build_guide(cdf_e, c->n_guide_e);
            kcdf_e = kcdf_of(cdf_e);
        }
        c->e_col = e_col ? 1 : 0;
        // ray-tracing channel tables: total mu_hat per material at each
        // channel energy (FP64 interpolation), and phi_b r(E_b)
        std::vector<float> mu_rt((size_t)sp.n_bins * mt.n_materials);
        std::vector<float> wr(sp.n_bins);
        double wsum = 0.0;
        for (int b = 0; b < sp.n_bins; ++b) wsum += sp.weight[b];
        std::vector<double> tot(mt.n_energies), rsp(dt.n_energies);
        for (int i = 0; i < dt.n_energies; ++i) rsp[i] = dt.response[i];
        for (int m = 0; m < mt.n_materials; ++m) {
            const float* t = mt.mu_hat + (size_t)m * 3 * mt.n_energies;
            for (int e = 0; e < mt.n_energies; ++e)
                tot[e] = 0.1 * ((double)t[e] + (double)t[mt.n_energies + e] + (double)t[2 * mt.n_energies + e]);
            for (int b = 0; b < sp.n_bins; ++b)
                mu_rt[(size_t)b * mt.n_materials + m] = (float)interp_d(tot, mt.e0_kev, mt.de_kev, sp.energy_kev[b]);
        }
        for (int b = 0; b < sp.n_bins; ++b)
            wr[b] = (float)((sp.weight[b] / wsum) * interp_d(rsp, dt.e0_kev, dt.de_kev, sp.energy_kev[b]));
        std::vector<float> wr_cols;
        if (e_col) {
            wr_cols.resize((size_t)g.nu * sp.n_bins);
            for (int u = 0; u < g.nu; ++u) {
                const double* wc = sp.column_weight + (size_t)u * sp.n_bins;
                double cs = 0.0;
                for (int b = 0; b < sp.n_bins; ++b) cs += wc[b];
                for (int b = 0; b < sp.n_bins; ++b)
                    wr_cols[(size_t)u * sp.n_bins + b] =
                        (float)((wc[b] / cs) * interp_d(rsp, dt.e0_kev, dt.de_kev, sp.energy_kev[b]));
            }
        }
        double fsum = 0.0;
        for (int i = 0; i < npix; ++i) fsum += bowtie->fluence[i];
        std::vector<double> wnorm(npix);
        for (int i = 0; i < npix; ++i) wnorm[i] = bowtie->fluence[i] / fsum;
        const std::vector<uint32_t> kcdf_pix = kcdf_of(cdf_pix);

        // the staging's counters: valid phantom, each material's largest density
        if ((rc = cuda_err(cudaStreamSynchronize(s)))) break;
        std::vector<double> rho_max;
        if ((rc = stage_phantom_finish(c, aux, rho_max))) break;
        // Woodcock majorant nodes: max over materials of the largest density of
        // that material times its total coefficient, with a 1e-5 margin.
        std::vector<float> major(mt.n_energies);
        for (int e = 0; e < mt.n_energies; ++e) {
            double mx = 0.0;
            for (int m = 0; m < mt.n_materials; ++m) {
                const float* t = tab.data() + (size_t)m * 3 * mt.n_energies;
                const double tot = ((double)t[e] + (double)t[mt.n_energies + e]) + (double)t[2 * mt.n_energies + e];
                mx = std::max(mx, rho_max[m] * tot);
            }
            major[e] = (float)(mx * (1.0 + 1e-5));
        }

        Arena ar;
        ar.add(&c->d_tab, tab.data(), tab.size());
        ar.add(&c->d_major, major.data(), major.size());
        ar.add(&c->d_resp, dt.response, (size_t)dt.n_energies);
        ar.add(&c->d_bin_e, bin_e.data(), bin_e.size());
        ar.add(&c->d_kcdf_pix, kcdf_pix.data(), kcdf_pix.size());
        ar.add(&c->d_guide_pix, guide_pix.data(), guide_pix.size());
        ar.add(&c->d_kcdf_e, kcdf_e.data(), kcdf_e.size());
        ar.add(&c->d_guide_e, guide_e.data(), guide_e.size());
        ar.add(&c->d_wnorm, wnorm.data(), wnorm.size());
        ar.add(&c->d_mu_rt, mu_rt.data(), mu_rt.size());
        ar.add(&c->d_wr, wr.data(), wr.size());
        if (e_col) ar.add(&c->d_wr_cols, wr_cols.data(), wr_cols.size());
        ar.add(&c->d_counter, (const unsigned long long*)nullptr, 1);
        ar.add(&c->d_stats, (const unsigned long long*)nullptr, GDRR_NSTATS);
        ar.add(&c->d_flag, (const int*)nullptr, 1);
        ar.add(&c->d_status, (const int*)nullptr, 1);
        if ((rc = ar.commit(c, &c->d_arena))) break;       // waits for its copy
    } while (0);
    // no copy may still target the counters' block when it goes back
    if (cudaStreamSynchronize(c->stream) != cudaSuccess && !rc) rc = GDRR_ERR_CUDA;
    give_pinned(aux_blk);
    if (rc) { free_ctx(c); return rc; }
    *out = c;
    return GDRR_OK;
}

GDRR_API void gdrr_destroy(gdrr_ctx* ctx) { free_ctx(ctx); }

GDRR_API int gdrr_release_memory(void) {
    {
        std::lock_guard<std::mutex> lock(g_pool_mutex);
        for (cudaMemPool_t p : g_pool)
            if (p && cudaMemPoolTrimTo(p, 0) != cudaSuccess) return GDRR_ERR_CUDA;
    }
    // the page-locked host blocks on the reuse list (none of them in use)
    std::lock_guard<std::mutex> lock(g_host_mutex);
    int rc = GDRR_OK;
    for (const Pinned& b : g_host_free)
        if (cudaFreeHost(b.p) != cudaSuccess) rc = GDRR_ERR_CUDA;
    g_host_free.clear();
    return rc;
}

GDRR_API int gdrr_set_options(gdrr_ctx* ctx, const gdrr_mc_options* o) {
    if (!ctx || !o) return GDRR_ERR_INVALID_ARG;
    gdrr_mc_options n = *o;
    set_defaults(&n);
    if (n.block_size % 32 || n.block_size > 512 || n.block_size < 32) return GDRR_ERR_INVALID_ARG;
    if (n.hist_per_thread > 4096 || n.batch_min > 32 || n.blocks_per_sm < 0 || n.blocks_per_sm > 64)
        return GDRR_ERR_INVALID_ARG;
    if (!(n.e_cut_kev < 1e6)) return GDRR_ERR_INVALID_ARG;
    if (n.nearest_voxel < 0 || n.nearest_voxel > 1 || n.scatter_filter < 0 || n.scatter_filter > 3)
        return GDRR_ERR_INVALID_ARG;
    if (n.rayleigh_form_factor < 0 || n.rayleigh_form_factor > 1 || (n.rayleigh_form_factor && !ctx->n_ff))
        return GDRR_ERR_INVALID_ARG;
    if (n.photon_pool < -1 || n.photon_pool > 3) return GDRR_ERR_INVALID_ARG;
    if (n.local_majorant < 0 || n.local_majorant > 1) return GDRR_ERR_INVALID_ARG;
    if (n.cell_shift == 0) n.cell_shift = default_cell_shift(ctx, n.local_majorant != 0);
    if (n.cell_shift < -1 || n.cell_shift > 6) return GDRR_ERR_INVALID_ARG;
    if (n.local_majorant && n.cell_shift < 0) return GDRR_ERR_INVALID_ARG;   // the cells are the majorant
    if (n.cell_shift != ctx->cell_shift) {
        if (ctx->n_scans > 0) return GDRR_ERR_INVALID_ARG;     // scans hold the old table pointer
        const int rc = build_cells(ctx, n.cell_shift, true);
        if (rc) {
            ctx->opt.cell_shift = ctx->cell_shift;              // -1: the table is gone
            return rc;
        }
    }
    ctx->opt = n;
    return GDRR_OK;
}

GDRR_API int gdrr_set_form_factor(gdrr_ctx* ctx, const gdrr_form_factor* ff) {
    if (!ctx || !ff) return GDRR_ERR_INVALID_ARG;
    if (ctx->n_scans > 0) return GDRR_ERR_INVALID_ARG;     // scans hold the old table pointers
    if (!ff->form_factor) {
        if (ctx->opt.rayleigh_form_factor) return GDRR_ERR_INVALID_ARG;
        dfree(ctx, ctx->d_ff_s); dfree(ctx, ctx->d_ff_a); dfree(ctx, ctx->d_ff_g);
        ctx->d_ff_s = ctx->d_ff_a = ctx->d_ff_g = nullptr;
        ctx->n_ff = 0;
        return GDRR_OK;
    }
    const double hc = 12.398419843320026;   // keV Angstrom (CODATA 2018)
    const int n = ff->n_x;
    const double dx = ff->dx_inv_angstrom;
    if (n < 2 || !(dx > 0.0) || !std::isfinite(dx)) return GDRR_ERR_INVALID_ARG;
    const double e_max = ctx->e0 + (double)(ctx->n_e - 1) * ctx->de;
    if ((double)(n - 1) * dx < e_max / hc) return GDRR_ERR_INVALID_ARG;
    // nodes s_j = (j dx)^2; A_j = trapezoid sum of F^2 over s; G_j = F_j^2 (FP64, stored FP32)
    std::vector<double> sd(n);
    std::vector<float> s(n), A((size_t)ctx->n_mat * n), G((size_t)ctx->n_mat * n);
    for (int j = 0; j < n; ++j) {
        const double x = (double)j * dx;
        sd[j] = x * x;
        s[j] = (float)(x * x);
    }
    for (int m = 0; m < ctx->n_mat; ++m) {
        const float* F = ff->form_factor + (size_t)m * n;
        if (!(F[0] > 0.0f)) return GDRR_ERR_INVALID_ARG;
        double acc = 0.0;
        for (int j = 0; j < n; ++j) {
            if (!(F[j] >= 0.0f) || !std::isfinite(F[j])) return GDRR_ERR_INVALID_ARG;
            if (j > 0) {
                const double f0 = (double)F[j - 1], f1 = (double)F[j];
                acc += 0.5 * (f0 * f0 + f1 * f1) * (sd[j] - sd[j - 1]);
            }
            A[(size_t)m * n + j] = (float)acc;
            const double g = (double)F[j] * (double)F[j];
            G[(size_t)m * n + j] = (float)g;
        }
    }
    float *ds = nullptr, *da = nullptr, *dg = nullptr;
    int rc = GDRR_OK;
    do {
        if ((rc = upload(ctx, &ds, s.data(), s.size()))) break;
        if ((rc = upload(ctx, &da, A.data(), A.size()))) break;
        if ((rc = upload(ctx, &dg, G.data(), G.size()))) break;
        if ((rc = cuda_err(cudaStreamSynchronize(ctx->stream)))) break;
    } while (0);
    if (rc) { dfree(ctx, ds); dfree(ctx, da); dfree(ctx, dg); return rc; }
    dfree(ctx, ctx->d_ff_s); dfree(ctx, ctx->d_ff_a); dfree(ctx, ctx->d_ff_g);
    ctx->d_ff_s = ds; ctx->d_ff_a = da; ctx->d_ff_g = dg;
    ctx->n_ff = n;
    ctx->ff_idx = (float)(1.0 / dx);
    return GDRR_OK;
}

GDRR_API int gdrr_get_options(const gdrr_ctx* ctx, gdrr_mc_options* o) {
    if (!ctx || !o) return GDRR_ERR_INVALID_ARG;
    *o = ctx->opt;
    return GDRR_OK;
}

GDRR_API int gdrr_sync(gdrr_ctx* ctx) {
    if (!ctx) return GDRR_ERR_INVALID_ARG;
    int status = 0;
    TRY_CUDA(cudaMemcpyAsync(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    if (!status) return GDRR_OK;
    TRY_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    return status_code(status);
}

GDRR_API int gdrr_air_scan(gdrr_ctx* ctx, double* I0_dev) {
    if (!ctx || !I0_dev) return GDRR_ERR_INVALID_ARG;
    RtParams p;
    memset(&p, 0, sizeof p);
    p.n_bins = ctx->n_bins;
    p.wr = ctx->d_wr; p.wr_cols = ctx->d_wr_cols; p.wnorm = ctx->d_wnorm;
    p.nu = ctx->geo.nu; p.nv = ctx->geo.nv;
    return cuda_err(launch_air(p, I0_dev, ctx->stream));
}

static int raytrace(gdrr_ctx* ctx, double angle_rad, double* P_dev, bool siddon, cudaStream_t stream) {
    if (!ctx || !P_dev || !std::isfinite(angle_rad)) return GDRR_ERR_INVALID_ARG;
    if (!geometry_ok(ctx, angle_rad)) return GDRR_ERR_INVALID_ARG;
    RtParams p;
    p.nx = ctx->nx; p.ny = ctx->ny; p.nz = ctx->nz;
    fill_box(ctx, p.lo, p.hi, p.ivox);
    p.vox = ctx->d_vox;
    p.bsy = ctx->bsy; p.bsz = ctx->bsz;
    p.n_mat = ctx->n_mat; p.n_bins = ctx->n_bins;
    p.mu_rt = ctx->d_mu_rt; p.wr = ctx->d_wr; p.wr_cols = ctx->d_wr_cols; p.wnorm = ctx->d_wnorm;
    p.nu = ctx->geo.nu; p.nv = ctx->geo.nv;
    p.hu = (float)(0.5 * ctx->geo.nu); p.hv = (float)(0.5 * ctx->geo.nv);
    p.du = (float)ctx->geo.du_mm; p.dv = (float)ctx->geo.dv_mm;
    p.half_step = (float)(0.5 * std::min(ctx->vox[0], std::min(ctx->vox[1], ctx->vox[2])));
    p.f = make_frame(ctx->geo, angle_rad);
    return cuda_err(siddon ? launch_rt_siddon(p, P_dev, stream) : launch_rt(p, P_dev, stream));
}

GDRR_API int gdrr_raytrace_primary(gdrr_ctx* ctx, double angle_rad, double* P_dev) {
    if (!ctx) return GDRR_ERR_INVALID_ARG;
    return raytrace(ctx, angle_rad, P_dev, false, ctx->stream);
}

GDRR_API int gdrr_raytrace_primary_siddon(gdrr_ctx* ctx, double angle_rad, double* P_dev) {
    if (!ctx) return GDRR_ERR_INVALID_ARG;
    return raytrace(ctx, angle_rad, P_dev, true, ctx->stream);
}

static int launch_grid(const gdrr_ctx* ctx, uint64_t total, bool rec) {
    const int block = ctx->opt.block_size;
    const int per_sm = ctx->opt.blocks_per_sm > 0 ? ctx->opt.blocks_per_sm
                                                  : mc_occupancy_blocks(ctx->n_mat, block, rec, ctx->opt.local_majorant != 0);
    int64_t grid = (int64_t)per_sm * ctx->n_sm;
    const int64_t useful = (int64_t)((total + 31) / 32 * 32 + block - 1) / block;
    if (grid > useful) grid = useful;
    return grid < 1 ? 1 : (int)grid;
}

// Histories per segment of the lane form's source pass: MC_SRC_BYTES each,
// at most 2^27 (4 GiB) per buffer.
constexpr uint64_t SRC_MAX = 1ull << 27;

// The source pass serves the lane form with default options and no records.
static bool source_pass_applies(const gdrr_ctx* ctx, bool rec) {
    return !rec && ctx->opt.nearest_voxel == 0 && ctx->opt.scatter_filter == 0 && ctx->opt.rayleigh_form_factor == 0 &&
           (ctx->opt.photon_pool <= 0 || ctx->opt.local_majorant);
}

// Grows a source-record buffer to min(total, SRC_MAX) histories: the
// context's from its device pool (owner given), a scan's with cudaMalloc
// (owner NULL, on stream s).  When the memory is not there the buffer stays
// empty and the transport samples the sources inline (the same arithmetic, so
// the same results).
static void ensure_src(const gdrr_ctx* owner, cudaStream_t s, float4** buf, uint64_t* cap, uint64_t total) {
    const uint64_t want = std::min(total, SRC_MAX);
    if (*cap >= want) return;
    if (*buf) {
        if (owner) {
            dfree(owner, *buf);
        } else {
            cudaStreamSynchronize(s);
            cudaFree(*buf);
        }
        *buf = nullptr;
        *cap = 0;
    }
    const cudaError_t e = owner ? dalloc(owner, buf, want * MC_SRC_BYTES)
                                : cudaMalloc((void**)buf, want * MC_SRC_BYTES);
    if (e == cudaSuccess) {
        *cap = want;
    } else {
        *buf = nullptr;
        cudaGetLastError();   // an allocation failure here is not an error of the call
    }
}

// The transport launch: the pool form for default options without records
// (when its pool fits the SM), else the lane form; the lane form with
// default options and a source buffer runs in segments of at most src_cap
// histories, each a source pass and a transport launch (the caller zeroes
// the work counter for the first).
static cudaError_t launch_transport(const gdrr_ctx* ctx, const McParams& p, uint64_t total, bool rec,
                                    cudaStream_t s, const float4* src = nullptr, uint64_t src_cap = 0) {
    const bool gen = p.nearest_voxel != 0 || p.scatter_filter != 0 || p.ray_ff != 0;
    if (!rec && !gen && !p.lm && ctx->opt.photon_pool > 0) {
        int per_sm = mc_pool_occupancy_blocks(ctx->n_mat, ctx->opt.photon_pool);
        if (ctx->opt.blocks_per_sm > 0 && ctx->opt.blocks_per_sm < per_sm) per_sm = ctx->opt.blocks_per_sm;
        if (per_sm > 0) {
            int64_t grid = (int64_t)per_sm * ctx->n_sm;
            const int64_t useful = (int64_t)((total + 31) / 32 * 32 + pool_threads() - 1) / pool_threads();
            if (grid > useful) grid = useful;
            return launch_mc_pool(p, ctx->opt.photon_pool, grid < 1 ? 1 : (int)grid, s);
        }
    }
    if (!rec && !gen && src && src_cap > 0) {
        for (uint64_t seg0 = 0; seg0 < total; seg0 += src_cap) {
            McParams q = p;
            q.seg0 = seg0;
            q.total = std::min(src_cap, total - seg0);
            q.src = src;
            cudaError_t e = launch_mc_source(q, s);
            if (e == cudaSuccess && seg0 > 0) e = cudaMemsetAsync(p.counter, 0, sizeof(unsigned long long), s);
            if (e == cudaSuccess) e = launch_mc(q, ctx->opt.block_size, launch_grid(ctx, q.total, false), false, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    return launch_mc(p, ctx->opt.block_size, launch_grid(ctx, total, rec), rec, s);
}

// The launch-independent part of the transport parameters.
static McParams static_mc_params(const gdrr_ctx* ctx) {
    McParams p;
    memset(&p, 0, sizeof p);
    p.nx = ctx->nx; p.ny = ctx->ny; p.nz = ctx->nz;
    fill_box(ctx, p.lo, p.hi, p.ivox);
    p.vox = ctx->d_vox;
    p.bsy = ctx->bsy; p.bsz = ctx->bsz;
    p.n_mat = ctx->n_mat; p.n_e = ctx->n_e;
    p.e0 = (float)ctx->e0; p.inv_de = (float)(1.0 / ctx->de);
    p.tab = ctx->d_tab; p.major = ctx->d_major;
    p.n_r = ctx->n_r; p.r0 = (float)ctx->r0; p.inv_dr = (float)(1.0 / ctx->dr); p.resp = ctx->d_resp;
    p.npix = ctx->geo.nu * ctx->geo.nv; p.n_guide_pix = ctx->n_guide_pix;
    p.kcdf_pix = ctx->d_kcdf_pix; p.guide_pix = ctx->d_guide_pix;
    p.n_bins = ctx->n_bins; p.n_guide_e = ctx->n_guide_e;
    p.kcdf_e = ctx->d_kcdf_e; p.guide_e = ctx->d_guide_e; p.e_col = ctx->e_col; p.bin_e = ctx->d_bin_e;
    p.nu = ctx->geo.nu; p.nv = ctx->geo.nv;
    p.hu = (float)(0.5 * ctx->geo.nu); p.hv = (float)(0.5 * ctx->geo.nv);
    p.du = (float)ctx->geo.du_mm; p.dv = (float)ctx->geo.dv_mm;
    p.idu = (float)(1.0 / ctx->geo.du_mm); p.idv = (float)(1.0 / ctx->geo.dv_mm);
    p.e_cut = (float)ctx->opt.e_cut_kev;
    p.max_steps = ctx->opt.max_steps;
    p.n_ff = ctx->n_ff;
    p.ff_s = ctx->d_ff_s; p.ff_a = ctx->d_ff_a; p.ff_g = ctx->d_ff_g;
    p.inv_hc = (float)(1.0 / 12.398419843320026);
    p.cells = ctx->d_cells;
    p.cshift = ctx->cell_shift; p.ncx = ctx->ncx; p.ncy = ctx->ncy; p.ncz = ctx->ncz;
    p.lm = ctx->opt.local_majorant;
    for (int k = 0; k < 3; ++k) p.vox_mm[k] = (float)ctx->vox[k];
    p.status = ctx->d_status;
    p.ff_idx = ctx->ff_idx;
    return p;
}

static int mc_launch(gdrr_ctx* ctx, const std::vector<Job>& jobs, uint64_t total, uint64_t seed,
                     uint64_t* stats_dev, gdrr_history_record* records_dev) {
    if (total == 0) return GDRR_OK;
    const int nj = (int)jobs.size();
    if (nj > ctx->jobs_cap) {
        dfree(ctx, ctx->d_jobs);
        ctx->d_jobs = nullptr;
        ctx->jobs_cap = 0;
        TRY_CUDA(dalloc(ctx, &ctx->d_jobs, sizeof(Job) * nj));
        ctx->jobs_cap = nj;
    }
    // pageable source: staged before the call returns, so the vector may die
    TRY_CUDA(cudaMemcpyAsync(ctx->d_jobs, jobs.data(), sizeof(Job) * nj, cudaMemcpyHostToDevice, ctx->stream));
    TRY_CUDA(cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned long long), ctx->stream));
    McParams p = static_mc_params(ctx);
    p.rk = round_keys(seed);
    p.jobs = ctx->d_jobs; p.n_jobs = nj; p.total = total;
    p.counter = ctx->d_counter;
    if (stats_dev) {
        p.stats = reinterpret_cast<unsigned long long*>(stats_dev);
    } else {
        TRY_CUDA(cudaMemsetAsync(ctx->d_stats, 0, GDRR_NSTATS * sizeof(unsigned long long), ctx->stream));
        p.stats = ctx->d_stats;
    }
    p.records = records_dev;
    p.chunk = 32 * ctx->opt.hist_per_thread;
    p.batch_min = ctx->opt.batch_min;
    p.nearest_voxel = ctx->opt.nearest_voxel;
    p.scatter_filter = ctx->opt.scatter_filter;
    p.ray_ff = ctx->opt.rayleigh_form_factor;
    const bool rec = records_dev != nullptr;
    if (source_pass_applies(ctx, rec)) {
        ensure_src(ctx, ctx->stream, &ctx->d_src, &ctx->src_cap, total);
        return cuda_err(launch_transport(ctx, p, total, rec, ctx->stream, ctx->d_src, ctx->src_cap));
    }
    return cuda_err(launch_transport(ctx, p, total, rec, ctx->stream));
}

GDRR_API int gdrr_mc_project(gdrr_ctx* ctx, double angle_rad, uint32_t angle_index, uint64_t n_photons,
                             uint64_t seed, uint64_t history_offset, int64_t* prim_dev, int64_t* scat_dev,
                             uint64_t* stats_dev, gdrr_history_record* records_dev) {
    if (!ctx || !prim_dev || !scat_dev || !std::isfinite(angle_rad)) return GDRR_ERR_INVALID_ARG;
    if (!geometry_ok(ctx, angle_rad)) return GDRR_ERR_INVALID_ARG;
    if (history_offset + n_photons < history_offset) return GDRR_ERR_INVALID_ARG;
    Job j;
    memset(&j, 0, sizeof j);
    j.f = make_frame(ctx->geo, angle_rad);
    j.angle_index = angle_index;
    j.first = 0;
    j.count = n_photons;
    j.hid_offset = history_offset;
    j.tally_p = prim_dev;
    j.tally_s = scat_dev;
    return mc_launch(ctx, std::vector<Job>(1, j), n_photons, seed, stats_dev, records_dev);
}

// The job table of a multi-angle scan: angle a transports budgets[a]
// histories with angle index a and history ids 0 .. budgets[a] - 1.
static int scan_jobs(const gdrr_ctx* ctx, int32_t n_angles, const double* angles_rad, const uint64_t* budgets,
                     int64_t* prim_dev, int64_t* scat_dev, std::vector<Job>* jobs, uint64_t* total_out) {
    if (!ctx || n_angles <= 0 || !angles_rad || !budgets || !prim_dev || !scat_dev) return GDRR_ERR_INVALID_ARG;
    jobs->clear();
    jobs->reserve(n_angles);
    const size_t npix = (size_t)ctx->geo.nu * ctx->geo.nv;
    uint64_t total = 0;
    for (int a = 0; a < n_angles; ++a) {
        if (!std::isfinite(angles_rad[a]) || !geometry_ok(ctx, angles_rad[a])) return GDRR_ERR_INVALID_ARG;
        if (budgets[a] == 0) continue;
        Job j;
        memset(&j, 0, sizeof j);
        j.f = make_frame(ctx->geo, angles_rad[a]);
        j.angle_index = (uint32_t)a;
        j.first = total;
        j.count = budgets[a];
        j.hid_offset = 0;
        j.tally_p = prim_dev + (size_t)a * npix;
        j.tally_s = scat_dev + (size_t)a * npix;
        if (total + budgets[a] < total) return GDRR_ERR_INVALID_ARG;
        total += budgets[a];
        jobs->push_back(j);
    }
    *total_out = total;
    return GDRR_OK;
}

GDRR_API int gdrr_mc_project_batched(gdrr_ctx* ctx, int32_t n_angles, const double* angles_rad,
                                     const uint64_t* budgets, uint64_t seed, int64_t* prim_dev, int64_t* scat_dev,
                                     uint64_t* stats_dev) {
    std::vector<Job> jobs;
    uint64_t total = 0;
    const int rc = scan_jobs(ctx, n_angles, angles_rad, budgets, prim_dev, scat_dev, &jobs, &total);
    if (rc) return rc;
    if (jobs.empty()) return GDRR_OK;
    return mc_launch(ctx, jobs, total, seed, stats_dev, nullptr);
}

GDRR_API int gdrr_scan_create(gdrr_ctx* ctx, int32_t n_angles, const double* angles_rad, const uint64_t* budgets,
                              uint64_t seed, int64_t* prim_dev, int64_t* scat_dev, uint64_t* stats_dev,
                              int32_t zero_tallies, gdrr_scan** out) {
    if (!out) return GDRR_ERR_INVALID_ARG;
    std::vector<Job> jobs;
    uint64_t total = 0;
    int rc = scan_jobs(ctx, n_angles, angles_rad, budgets, prim_dev, scat_dev, &jobs, &total);
    if (rc) return rc;
    if (jobs.empty()) return GDRR_ERR_INVALID_ARG;
    gdrr_scan* sc = new (std::nothrow) gdrr_scan();
    if (!sc) return GDRR_ERR_OOM;
    sc->ctx = ctx;
    sc->total = total;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMalloc((void**)&sc->d_jobs, sizeof(Job) * jobs.size())) != cudaSuccess) break;
        if ((e = cudaMalloc((void**)&sc->d_counter, sizeof(unsigned long long))) != cudaSuccess) break;
        if (!stats_dev && (e = cudaMalloc((void**)&sc->d_stats, GDRR_NSTATS * sizeof(unsigned long long))) != cudaSuccess)
            break;
        if ((e = cudaMemcpy(sc->d_jobs, jobs.data(), sizeof(Job) * jobs.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            break;
        McParams p = static_mc_params(ctx);
        p.rk = round_keys(seed);
        p.jobs = sc->d_jobs; p.n_jobs = (int)jobs.size(); p.total = total;
        p.counter = sc->d_counter;
        p.stats = stats_dev ? reinterpret_cast<unsigned long long*>(stats_dev) : sc->d_stats;
        p.records = nullptr;
        p.chunk = 32 * ctx->opt.hist_per_thread;
        p.batch_min = ctx->opt.batch_min;
        p.nearest_voxel = ctx->opt.nearest_voxel;
        p.scatter_filter = ctx->opt.scatter_filter;
        p.ray_ff = ctx->opt.rayleigh_form_factor;
        if (source_pass_applies(ctx, false)) ensure_src(nullptr, ctx->stream, &sc->d_src, &sc->src_cap, total);
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
        const size_t tally_bytes = (size_t)n_angles * ctx->geo.nu * ctx->geo.nv * sizeof(int64_t);
        cudaError_t ce = cudaSuccess;
        if (zero_tallies) {
            ce = cudaMemsetAsync(prim_dev, 0, tally_bytes, cs);
            if (ce == cudaSuccess) ce = cudaMemsetAsync(scat_dev, 0, tally_bytes, cs);
        }
        if (ce == cudaSuccess && !stats_dev)
            ce = cudaMemsetAsync(sc->d_stats, 0, GDRR_NSTATS * sizeof(unsigned long long), cs);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(sc->d_counter, 0, sizeof(unsigned long long), cs);
        if (ce == cudaSuccess) ce = launch_transport(ctx, p, total, false, cs, sc->d_src, sc->src_cap);
        e = cudaStreamEndCapture(cs, &sc->graph);
        if (ce != cudaSuccess) { e = ce; break; }
        if (e != cudaSuccess) break;
        e = cudaGraphInstantiate(&sc->exec, sc->graph, 0);
    } while (0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        gdrr_scan_destroy(sc);
        return cuda_err(e);
    }
    sc->counted = true;
    ++ctx->n_scans;
    *out = sc;
    return GDRR_OK;
}

GDRR_API int gdrr_scan_launch(gdrr_scan* scan) {
    if (!scan || !scan->exec) return GDRR_ERR_INVALID_ARG;
    return cuda_err(cudaGraphLaunch(scan->exec, scan->ctx->stream));
}

GDRR_API void gdrr_scan_destroy(gdrr_scan* scan) {
    if (!scan) return;
    if (scan->ctx) cudaStreamSynchronize(scan->ctx->stream);
    if (scan->exec) cudaGraphExecDestroy(scan->exec);
    if (scan->graph) cudaGraphDestroy(scan->graph);
    if (scan->d_jobs) cudaFree(scan->d_jobs);
    if (scan->d_counter) cudaFree(scan->d_counter);
    if (scan->d_stats) cudaFree(scan->d_stats);
    if (scan->d_src) cudaFree(scan->d_src);
    if (scan->counted && scan->ctx) --scan->ctx->n_scans;
    delete scan;
}

GDRR_API int gdrr_autotune(gdrr_ctx* ctx, double angle_rad, uint64_t n_probe, uint64_t seed,
                           gdrr_mc_options* best_out) {
    if (!ctx || n_probe == 0 || !std::isfinite(angle_rad) || !geometry_ok(ctx, angle_rad)) return GDRR_ERR_INVALID_ARG;
    const size_t npix = (size_t)ctx->geo.nu * ctx->geo.nv;
    if (!ctx->d_tune) TRY_CUDA(dalloc(ctx, &ctx->d_tune, 2 * npix * sizeof(int64_t)));
    Job j;
    memset(&j, 0, sizeof j);
    j.f = make_frame(ctx->geo, angle_rad);
    j.count = n_probe;
    j.tally_p = ctx->d_tune;
    j.tally_s = ctx->d_tune + npix;
    const std::vector<Job> jobs(1, j);
    const gdrr_mc_options base = ctx->opt;
    static const int blocks[] = {64, 128, 256, 512};
    static const int batch[] = {8, 12, 16, 20, 24, 28, 32};
    static const int hpt[] = {1, 8, 64};
    static const int pools[] = {1, 2, 3};
    cudaEvent_t e0, e1;
    TRY_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return GDRR_ERR_CUDA; }
    gdrr_mc_options best = base;
    float best_ms = 3.0e38f;
    int rc = mc_launch(ctx, jobs, n_probe, seed, nullptr, nullptr);   // warm-up
    std::vector<gdrr_mc_options> grid;
    for (int b : blocks)
        for (int m : batch)
            for (int h : hpt) {
                gdrr_mc_options o = base;
                o.block_size = b; o.batch_min = m; o.hist_per_thread = h; o.blocks_per_sm = 0; o.photon_pool = -1;
                grid.push_back(o);
            }
    for (int q : pools)
        for (int h : hpt) {
            if (base.local_majorant) break;              // local majorants run the lane form only
            gdrr_mc_options o = base;
            o.hist_per_thread = h; o.blocks_per_sm = 0; o.photon_pool = q;
            grid.push_back(o);
        }
    for (const gdrr_mc_options& o : grid) {
        if (rc) break;
        ctx->opt = o;
        float ms = 0.0f;
        if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) { rc = GDRR_ERR_CUDA; break; }
        rc = mc_launch(ctx, jobs, n_probe, seed, nullptr, nullptr);
        if (rc) break;
        if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess
            || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = GDRR_ERR_CUDA;
            break;
        }
        if (ms < best_ms) { best_ms = ms; best = o; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->opt = rc ? base : best;
    if (!rc && best_out) *best_out = best;
    return rc;
}

GDRR_API int gdrr_finalize(gdrr_ctx* ctx, const int64_t* tally_dev, int64_t n, uint64_t n_photons,
                           double* signal_dev) {
    if (!ctx || !tally_dev || !signal_dev || n < 0 || n_photons == 0) return GDRR_ERR_INVALID_ARG;
    TRY_CUDA(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    const double scale = ldexp(1.0, -GDRR_TALLY_BITS) / (double)n_photons;
    TRY_CUDA(launch_finalize(tally_dev, n, scale, signal_dev, ctx->d_flag, ctx->stream));
    int bad = 0;
    TRY_CUDA(cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    return bad ? GDRR_ERR_TALLY_OVERFLOW : GDRR_OK;
}

GDRR_API int gdrr_bin_tally(gdrr_ctx* ctx, const int64_t* tally_dev, int32_t nu, int32_t nv, int32_t factor,
                            int64_t* out_dev) {
    if (!ctx || !tally_dev || !out_dev || nu <= 0 || nv <= 0 || factor <= 0 || nu % factor || nv % factor)
        return GDRR_ERR_INVALID_ARG;
    return cuda_err(launch_bin(tally_dev, nu, nv, factor, out_dev, ctx->stream));
}

GDRR_API int gdrr_upsample(gdrr_ctx* ctx, const double* coarse_dev, int32_t cu, int32_t cv, int32_t factor,
                           double* fine_dev) {
    if (!ctx || !coarse_dev || !fine_dev || cu <= 0 || cv <= 0 || factor <= 0) return GDRR_ERR_INVALID_ARG;
    if ((int64_t)cu * factor * cv * factor > (1 << 28)) return GDRR_ERR_INVALID_ARG;
    return cuda_err(launch_upsample(coarse_dev, cu, cv, factor, fine_dev, ctx->stream));
}

// The context's denoiser scratch, grown to the larger of the two forms' needs.
static int denoise_scratch(gdrr_ctx* ctx, int nu, int nv) {
    const size_t need = std::max(denoise_scratch_doubles(nu, nv) * sizeof(double), denoise_fused_scratch_bytes(nu, nv));
    if (need > ctx->denoise_cap) {
        dfree(ctx, ctx->d_denoise);
        ctx->d_denoise = nullptr;
        ctx->denoise_cap = 0;
        TRY_CUDA(dalloc(ctx, &ctx->d_denoise, need));
        ctx->denoise_cap = need;
    }
    return GDRR_OK;
}

// Step 3's iteration with the scalars on the host (scal_dev NULL) or on the
// device (scal_dev[0] count scale, [1] beta): one cooperative launch when the
// image fits its bands, else one launch per iteration.
static int denoise_on_ctx(gdrr_ctx* ctx, const double* S_hat_dev, double* S_dev, int nu, int nv, double count_scale,
                          double beta, const double* scal_dev, double omega, int iters, bool* fused) {
    int rc = denoise_scratch(ctx, nu, nv);
    if (rc) return rc;
    if (denoise_fused_fits(nu, nv)) {
        if (fused) *fused = true;
        return cuda_err(launch_denoise_fused(S_hat_dev, S_dev, nu, nv, count_scale, beta, scal_dev, omega, iters,
                                             ctx->d_denoise, ctx->d_status, ctx->stream));
    }
    if (fused) *fused = false;
    return cuda_err(launch_denoise(S_hat_dev, S_dev, nu, nv, count_scale, beta, scal_dev, omega, iters,
                                   ctx->d_denoise, ctx->stream));
}

GDRR_API int gdrr_denoise_scatter(gdrr_ctx* ctx, const double* S_hat_dev, double* S_dev, int32_t nu, int32_t nv,
                                  double count_scale, double beta, double omega, int32_t iters) {
    if (!ctx || !S_hat_dev || !S_dev || nu <= 0 || nv <= 0 || iters < 0) return GDRR_ERR_INVALID_ARG;
    if (!(count_scale > 0) || !(beta > 0) || !(omega > 0 && omega < 2) || !std::isfinite(count_scale)
        || !std::isfinite(beta))
        return GDRR_ERR_INVALID_ARG;
    if ((int64_t)nu * nv > (1 << 28)) return GDRR_ERR_INVALID_ARG;
    return denoise_on_ctx(ctx, S_hat_dev, S_dev, nu, nv, count_scale, beta, nullptr, omega, iters, nullptr);
}

// Waits for a stream when it goes out of scope, once armed: a projection
// that returns early never leaves its side stream's ray trace running.
struct StreamGuard {
    cudaStream_t s = nullptr;
    bool armed = false;
    ~StreamGuard() {
        if (armed) cudaStreamSynchronize(s);
    }
};

GDRR_API int gdrr_project(gdrr_ctx* ctx, const gdrr_projection* pr, const gdrr_projection_out* out,
                          gdrr_projection_info* info) {
    if (!ctx || !pr || !out) return GDRR_ERR_INVALID_ARG;
    if (!out->P || !out->P_hat || !out->S_hat || !out->S || !out->N) return GDRR_ERR_INVALID_ARG;
    const int nu = ctx->geo.nu, nv = ctx->geo.nv, f = pr->bin_factor;
    if (pr->n_photons == 0 || f <= 0 || nu % f || nv % f || pr->iters < 0) return GDRR_ERR_INVALID_ARG;
    if (!std::isfinite(pr->angle_rad) || !geometry_ok(ctx, pr->angle_rad)) return GDRR_ERR_INVALID_ARG;
    if (!(pr->omega > 0 && pr->omega < 2) || !(pr->mAs > 0) || !(pr->zeta > 0) || !std::isfinite(pr->mAs) ||
        !std::isfinite(pr->zeta) || !std::isfinite(pr->smoothing_px))
        return GDRR_ERR_INVALID_ARG;
    if (!(pr->smoothing_px > 0) && !(pr->beta > 0 && std::isfinite(pr->beta))) return GDRR_ERR_INVALID_ARG;
    const size_t npix = (size_t)nu * nv;
    const int cu = nu / f, cv = nv / f;
    const int ncoarse = cu * cv;
    // scratch: prim, scat, coarse tally (int64 [npix] each), coarse S^ and S
    // (double [npix] each: enough for any bin factor), scalars, counters
    const size_t scratch = 5 * npix * 8 + 8 * sizeof(double) + GDRR_NSTATS * sizeof(unsigned long long) + 64;
    if (!ctx->d_proj) TRY_CUDA(dalloc(ctx, &ctx->d_proj, scratch));
    if (!ctx->h_proj) {
        const Pinned hp = take_pinned(sizeof(ProjHost));
        if (!hp.p) return GDRR_ERR_OOM;
        ctx->h_proj = static_cast<ProjHost*>(hp.p);
        ctx->h_proj_cap = hp.cap;
    }
    for (cudaEvent_t& e : ctx->ev_proj)
        if (!e) TRY_CUDA(cudaEventCreate(&e));
    if (!ctx->side) TRY_CUDA(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
    if (!ctx->ev_fork) TRY_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    if (!ctx->ev_join) TRY_CUDA(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    cudaEvent_t* ev = ctx->ev_proj;
    char* base = static_cast<char*>(ctx->d_proj);
    int64_t* prim = out->prim_tally ? out->prim_tally : reinterpret_cast<int64_t*>(base);
    int64_t* scat = out->scat_tally ? out->scat_tally : reinterpret_cast<int64_t*>(base + npix * 8);
    int64_t* coarse = reinterpret_cast<int64_t*>(base + 2 * npix * 8);
    double* shc = out->S_hat_coarse ? out->S_hat_coarse : reinterpret_cast<double*>(base + 3 * npix * 8);
    double* sc = out->S_coarse ? out->S_coarse : reinterpret_cast<double*>(base + 4 * npix * 8);
    double* scal = reinterpret_cast<double*>(base + 5 * npix * 8);
    unsigned long long* stats = out->stats ? reinterpret_cast<unsigned long long*>(out->stats)
                                           : reinterpret_cast<unsigned long long*>(scal + 8);
    cudaStream_t st = ctx->stream;
    const double omega = pr->omega;
    const double floor_ = omega < 1.0 ? omega / (8.0 * (1.0 - omega)) : INFINITY;
    const double t2s = ldexp(1.0, -GDRR_TALLY_BITS) / (double)pr->n_photons;
    bool fused = false;
    int rc = GDRR_OK;
    TRY_CUDA(cudaEventRecord(ev[0], st));
    TRY_CUDA(cudaEventRecord(ctx->ev_fork, st));
    // Step 2: zeroed tallies and counters, transport, signal per source photon
    TRY_CUDA(cudaMemsetAsync(prim, 0, npix * sizeof(int64_t), st));
    TRY_CUDA(cudaMemsetAsync(scat, 0, npix * sizeof(int64_t), st));
    TRY_CUDA(cudaMemsetAsync(stats, 0, GDRR_NSTATS * sizeof(unsigned long long), st));
    TRY_CUDA(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), st));
    TRY_CUDA(cudaEventRecord(ev[2], st));
    if ((rc = gdrr_mc_project(ctx, pr->angle_rad, pr->angle_index, pr->n_photons, pr->seed, 0, prim, scat,
                              reinterpret_cast<uint64_t*>(stats), nullptr)))
        return rc;
    TRY_CUDA(cudaEventRecord(ev[3], st));
    // Step 1 on the side stream, queued behind the transport: the transport's
    // grid holds every SM's registers, so the ray trace's blocks take the SMs
    // its persistent blocks leave at the end of the launch; Step 4 joins it
    TRY_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
    StreamGuard side_done;
    side_done.s = ctx->side;
    side_done.armed = true;
    if ((rc = raytrace(ctx, pr->angle_rad, out->P, false, ctx->side))) return rc;
    TRY_CUDA(cudaEventRecord(ctx->ev_join, ctx->side));
    TRY_CUDA(launch_finalize(prim, (int64_t)npix, t2s, out->P_hat, ctx->d_flag, st));
    TRY_CUDA(launch_finalize(scat, (int64_t)npix, t2s, out->S_hat, ctx->d_flag, st));
    // Step 3: coarse grid, scalars on the device, Eq. 5, upsampling
    TRY_CUDA(launch_bin(scat, nu, nv, f, coarse, st));
    TRY_CUDA(launch_finalize(coarse, ncoarse, t2s, shc, ctx->d_flag, st));
    TRY_CUDA(launch_project_scalars(coarse, ncoarse, stats, t2s, 1.0 / (double)pr->n_photons, pr->beta,
                                    pr->smoothing_px > 0 ? pr->smoothing_px : 0.0, floor_, scal, st));
    TRY_CUDA(cudaEventRecord(ev[4], st));
    if ((rc = denoise_on_ctx(ctx, shc, sc, cu, cv, 0.0, 0.0, scal, omega, pr->iters, &fused))) return rc;
    TRY_CUDA(cudaEventRecord(ev[5], st));
    TRY_CUDA(launch_upsample(sc, cu, cv, f, out->S, st));
    // Step 4 (needs Step 1's primary)
    TRY_CUDA(cudaStreamWaitEvent(st, ctx->ev_join, 0));
    const double alpha = sqrt((double)pr->n_photons / (pr->zeta * pr->mAs));
    TRY_CUDA(launch_noise(out->P_hat, out->P, out->S_hat, out->S, (int64_t)npix, alpha, out->N, st));
    TRY_CUDA(cudaEventRecord(ev[1], st));
    // one read-back of the scalars, counters and flags, one synchronisation
    ProjHost* h = ctx->h_proj;
    TRY_CUDA(cudaMemcpyAsync(h->scal, scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaMemcpyAsync(h->stats, stats, GDRR_NSTATS * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaMemcpyAsync(&h->overflow, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaMemcpyAsync(&h->status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaStreamSynchronize(st));
    if (info) {
        info->count_scale = h->scal[0];
        info->beta = h->scal[1];
        info->mean_count = h->scal[2];
        info->below_floor = h->scal[3] != 0.0 ? 1 : 0;
        info->tally_scatter = h->stats[GDRR_ST_TALLY_SCATTER];
        info->step_limit = h->stats[GDRR_ST_STEP_LIMIT];
        info->denoise_fused = fused ? 1 : 0;
        float ms[3] = {0.0f, 0.0f, 0.0f};
        for (int k = 0; k < 3; ++k) TRY_CUDA(cudaEventElapsedTime(&ms[k], ev[2 * k], ev[2 * k + 1]));
        info->total_ms = ms[0];
        info->transport_ms = ms[1];
        info->denoise_ms = ms[2];
    }
    if (h->status) {
        TRY_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
        TRY_CUDA(cudaStreamSynchronize(st));
        return status_code(h->status);
    }
    if (h->overflow) return GDRR_ERR_TALLY_OVERFLOW;
    if (h->stats[GDRR_ST_STEP_LIMIT]) return GDRR_ERR_STEP_LIMIT;
    return GDRR_OK;
}

GDRR_API int gdrr_noise_calibrate(gdrr_ctx* ctx, const double* P_hat_dev, const double* P_dev,
                                  const double* S_hat_dev, const double* S_dev, int64_t n, uint64_t n_sim,
                                  double mAs, double zeta, double* N_dev) {
    if (!ctx || !P_hat_dev || !P_dev || !S_hat_dev || !S_dev || !N_dev || n < 0 || n_sim == 0) return GDRR_ERR_INVALID_ARG;
    if (!(mAs > 0) || !(zeta > 0) || !std::isfinite(mAs) || !std::isfinite(zeta)) return GDRR_ERR_INVALID_ARG;
    const double alpha = sqrt((double)n_sim / (zeta * mAs));
    return cuda_err(launch_noise(P_hat_dev, P_dev, S_hat_dev, S_dev, n, alpha, N_dev, ctx->stream));
}

GDRR_API int gdrr_fit_zeta(const double* inv_sqrt_mAs, const double* ratio, int32_t n, uint64_t n_sim,
                           double* zeta_out, double* k_out) {
    if (!inv_sqrt_mAs || !ratio || n <= 0 || n_sim == 0 || !zeta_out) return GDRR_ERR_INVALID_ARG;
    double sxy = 0.0, sxx = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(inv_sqrt_mAs[i]) || !std::isfinite(ratio[i])) return GDRR_ERR_INVALID_ARG;
        sxy += inv_sqrt_mAs[i] * ratio[i];
        sxx += inv_sqrt_mAs[i] * inv_sqrt_mAs[i];
    }
    if (!(sxx > 0.0)) return GDRR_ERR_INVALID_ARG;
    const double k = sxy / sxx;
    if (!(k != 0.0)) return GDRR_ERR_INVALID_ARG;
    *zeta_out = (double)n_sim / (k * k);
    if (k_out) *k_out = k;
    return GDRR_OK;
}

GDRR_API int gdrr_scale_to_f32(const double* src_dev, int64_t n, double scale, float* dst_dev, void* cuda_stream) {
    if ((n > 0 && (!src_dev || !dst_dev)) || n < 0 || !std::isfinite(scale)) return GDRR_ERR_INVALID_ARG;
    return cuda_err(launch_scale_to_f32(src_dev, n, scale, dst_dev, (cudaStream_t)cuda_stream));
}

GDRR_API int gdrr_scale_to_f64(const float* src_dev, int64_t n, double scale, double* dst_dev, void* cuda_stream) {
    if ((n > 0 && (!src_dev || !dst_dev)) || n < 0 || !std::isfinite(scale)) return GDRR_ERR_INVALID_ARG;
    return cuda_err(launch_scale_to_f64(src_dev, n, scale, dst_dev, (cudaStream_t)cuda_stream));
}

GDRR_API int gdrr_gather_roofline(gdrr_ctx* ctx, uint64_t n_cells, double* seconds_out) {
    if (!ctx || !seconds_out || n_cells == 0) return GDRR_ERR_INVALID_ARG;
    McParams p = static_mc_params(ctx);
    const int per_sm = 4;
    cudaEvent_t e0, e1;
    TRY_CUDA(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    if (err != cudaSuccess) { cudaEventDestroy(e0); return cuda_err(err); }
    err = cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream);
    if (err == cudaSuccess) err = launch_gather_probe(p, n_cells / 8 + 1, per_sm * ctx->n_sm,
                                                      reinterpret_cast<unsigned int*>(ctx->d_flag), ctx->stream);
    if (err == cudaSuccess) err = cudaEventRecord(e0, ctx->stream);
    if (err == cudaSuccess) err = launch_gather_probe(p, n_cells, per_sm * ctx->n_sm,
                                                      reinterpret_cast<unsigned int*>(ctx->d_flag), ctx->stream);
    if (err == cudaSuccess) err = cudaEventRecord(e1, ctx->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_err(err);
    *seconds_out = 1e-3 * (double)ms;
    return GDRR_OK;
}

GDRR_API int gdrr_stream_words(uint64_t seed, uint32_t angle_index, uint64_t hid0, int32_t n_hist, int32_t n_blocks,
                               uint32_t* out_dev, void* cuda_stream) {
    if (n_hist < 0 || n_blocks <= 0 || n_blocks > (1 << 20) || (n_hist > 0 && !out_dev)) return GDRR_ERR_INVALID_ARG;
    return cuda_err(launch_stream_words(seed, angle_index, hid0, n_hist, n_blocks, out_dev, (cudaStream_t)cuda_stream));
}

}  // extern "C"
