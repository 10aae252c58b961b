// Image-domain steps of the paper on sm_103a, all FP64:
//  * tally -> signal per source photon (Section 2.6 normalisation);
//  * exact integer binning to the coarse scatter grid, bilinear upsampling;
//  * Step 3, Section 2.5: the Eq. 5 relaxation iteration of the Poisson
//    denoiser (Eq. 2-4), in one cooperative launch whose row bands exchange
//    iterates with their neighbours, or one launch per iteration with
//    ping-pong buffers (images too large for the one-launch form, and the
//    allocation-free entry point);
//  * Step 4, Section 2.6: N = ((P^ - P) + (S^ - S)) * alpha.
// These are element-wise or 5-point-stencil passes over at most a detector
// image (196,608 pixels): launch- and latency-bound, not bandwidth-bound.
#include <algorithm>

#include "gdrr_internal.cuh"

namespace gdrr {
namespace {

constexpr int BLOCK = 256;

inline int grid_for(int64_t n) { return (int)((n + BLOCK - 1) / BLOCK); }

__global__ void finalize_kernel(const int64_t* __restrict__ t, int64_t n, double scale, double* __restrict__ out,
                                int* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t v = t[i];
    if (v < 0) atomicOr(bad, 1);
    out[i] = (double)v * scale;
}

__global__ void bin_kernel(const int64_t* __restrict__ t, int nu, int nv, int f, int64_t* __restrict__ out) {
    const int cu = nu / f, cv = nv / f;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cu * cv) return;
    const int I = i % cu, J = i / cu;
    long long s = 0;
    for (int dy = 0; dy < f; ++dy)
        for (int dx = 0; dx < f; ++dx) s += t[(size_t)(J * f + dy) * nu + I * f + dx];
    out[i] = s;
}

__global__ void upsample_kernel(const double* __restrict__ c, int cu, int cv, int f, double* __restrict__ out) {
    const int nu = cu * f, nv = cv * f;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nu * nv) return;
    const int iu = i % nu, iv = i / nu;
    const double xu = (iu + 0.5) / f - 0.5, xv = (iv + 0.5) / f - 0.5;
    const int u0f = (int)floor(xu), v0f = (int)floor(xv);
    const double tu = xu - u0f, tv = xv - v0f;
    const int u0 = min(max(u0f, 0), cu - 1), u1 = min(max(u0f + 1, 0), cu - 1);
    const int v0 = min(max(v0f, 0), cv - 1), v1 = min(max(v0f + 1, 0), cv - 1);
    const double top = c[v0 * cu + u0] * (1.0 - tu) + c[v0 * cu + u1] * tu;
    const double bot = c[v1 * cu + u0] * (1.0 - tu) + c[v1 * cu + u1] * tu;
    out[i] = (top * (1.0 - tv) + bot * tv) / (double)(f * f);
}

__global__ void noise_kernel(const double* __restrict__ ph, const double* __restrict__ p,
                             const double* __restrict__ sh, const double* __restrict__ s, int64_t n,
                             double alpha, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = ((ph[i] - p[i]) + (sh[i] - s[i])) * alpha;
}

constexpr double DENOISE_EPS = 1e-3;   // counts

// The scalars come from the host (scal NULL) or from the device: count scale
// scal[0], beta scal[1] (gdrr_project derives them on the device).
__global__ void denoise_init(const double* __restrict__ s_hat, int n, double count_scale_h,
                             const double* __restrict__ scal, double* __restrict__ sc, double* __restrict__ s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double inv_scale = 1.0 / (scal ? scal[0] : count_scale_h);
    const double v = s_hat[i] * inv_scale;
    sc[i] = v;
    s[i] = fmax(v, DENOISE_EPS);
}

// One Eq. 5 update: S' = (1 - w) S + w/4 [ Sigma S - (1/beta)(1 - S^/S) ],
// Sigma S = S(i+1,j) + S(i,j+1) + S(i-1,j) + S(i,j-1), replicate edges.
__global__ void denoise_step(const double* __restrict__ sc, const double* __restrict__ s, int nu, int nv,
                             double omega, double beta_h, const double* __restrict__ scal,
                             double* __restrict__ s_next) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nu * nv) return;
    const double inv_beta = 1.0 / (scal ? scal[1] : beta_h);
    const int iu = i % nu, iv = i / nu;
    const double c = s[i];
    const double right = s[iv * nu + min(iu + 1, nu - 1)];
    const double down = s[min(iv + 1, nv - 1) * nu + iu];
    const double left = s[iv * nu + max(iu - 1, 0)];
    const double up = s[max(iv - 1, 0) * nu + iu];
    const double sigma = ((right + down) + left) + up;
    const double v = (1.0 - omega) * c + (omega / 4.0) * (sigma - inv_beta * (1.0 - sc[i] / c));
    s_next[i] = fmax(v, DENOISE_EPS);
}

__global__ void scale_kernel(const double* __restrict__ a, int n, double scale_h, const double* __restrict__ scal,
                             double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] * (scal ? scal[0] : scale_h);
}

}  // namespace

cudaError_t launch_finalize(const int64_t* t, int64_t n, double scale, double* out, int* bad, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    finalize_kernel<<<grid_for(n), BLOCK, 0, s>>>(t, n, scale, out, bad);
    return cudaGetLastError();
}

cudaError_t launch_bin(const int64_t* t, int nu, int nv, int f, int64_t* out, cudaStream_t s) {
    const int n = (nu / f) * (nv / f);
    if (n <= 0) return cudaSuccess;
    bin_kernel<<<grid_for(n), BLOCK, 0, s>>>(t, nu, nv, f, out);
    return cudaGetLastError();
}

cudaError_t launch_upsample(const double* c, int cu, int cv, int f, double* out, cudaStream_t s) {
    const int n = cu * f * cv * f;
    if (n <= 0) return cudaSuccess;
    upsample_kernel<<<grid_for(n), BLOCK, 0, s>>>(c, cu, cv, f, out);
    return cudaGetLastError();
}

cudaError_t launch_noise(const double* ph, const double* p, const double* sh, const double* sc, int64_t n,
                         double alpha, double* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    noise_kernel<<<grid_for(n), BLOCK, 0, s>>>(ph, p, sh, sc, n, alpha, out);
    return cudaGetLastError();
}

namespace {

__global__ void scale_to_f32_kernel(const double* __restrict__ a, int64_t n, double scale, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)(a[i] * scale);
}

__global__ void scale_to_f64_kernel(const float* __restrict__ a, int64_t n, double scale, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)a[i] * scale;
}

}  // namespace

cudaError_t launch_scale_to_f32(const double* a, int64_t n, double scale, float* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    scale_to_f32_kernel<<<grid_for(n), BLOCK, 0, s>>>(a, n, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_scale_to_f64(const float* a, int64_t n, double scale, double* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    scale_to_f64_kernel<<<grid_for(n), BLOCK, 0, s>>>(a, n, scale, out);
    return cudaGetLastError();
}

size_t denoise_scratch_doubles(int nu, int nv) { return 2 * (size_t)nu * nv; }

// ---------------------------------------------------------------------------
// The Eq. 5 iteration in one launch.
//
// Each CTA owns a band of whole image rows and keeps, per owned pixel, the
// count-scale data S^ and the current iterate in registers.  Iterates travel
// through two ping-pong images in global memory (L2-resident: 2 x 96 KB at
// 128 x 96); after writing its rows of iterate k + 1 a CTA publishes k + 2 in
// its flag, and before reading iterate k it waits until the CTAs of the rows
// above and below have published k + 1.  That one wait also shows that those
// neighbours have finished reading the buffer the CTA is about to overwrite
// (they read it before publishing), so no grid-wide barrier is needed.  The
// launch is cooperative, which guarantees that every CTA is resident, and
// every wait is bounded (about a second of %globaltimer): on expiry the CTA
// records a timeout in *status and stops.  The arithmetic per pixel is that
// of denoise_step, in the same order, so both forms give the same result.
namespace {

constexpr int FUSED_MAX_PPT = 4;                    // owned pixels per thread
constexpr unsigned long long WAIT_NS = 1000000000ull;

__global__ void __launch_bounds__(1024) denoise_fused_kernel(
    const double* __restrict__ s_hat, double* __restrict__ s_out, int nu, int nv, int rows_per_cta,
    double count_scale_h, double beta_h, const double* __restrict__ scal, double omega, int iters,
    double* buf0, double* buf1, unsigned* flags, int* status) {
    __shared__ int s_abort;
    const int b = blockIdx.x, G = gridDim.x;
    const int r0 = b * rows_per_cta;
    const int r1 = min(nv, r0 + rows_per_cta);
    const int npx = (r1 - r0) * nu;
    const double count_scale = scal ? scal[0] : count_scale_h;
    const double beta = scal ? scal[1] : beta_h;
    const double inv_scale = 1.0 / count_scale, inv_beta = 1.0 / beta;
    double sc[FUSED_MAX_PPT], cur[FUSED_MAX_PPT];
#pragma unroll
    for (int p = 0; p < FUSED_MAX_PPT; ++p) {
        const int i = threadIdx.x + p * blockDim.x;
        sc[p] = 0.0;
        cur[p] = DENOISE_EPS;
        if (i < npx) {
            const int g = r0 * nu + i;
            const double v = s_hat[g] * inv_scale;
            sc[p] = v;
            cur[p] = fmax(v, DENOISE_EPS);
            buf0[g] = cur[p];
        }
    }
    if (threadIdx.x == 0) s_abort = 0;
    __syncwarp();                                 // converged warps at every block barrier
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release_u32(flags + b, 1u);
    }
    for (int k = 0; k < iters; ++k) {
        if (threadIdx.x == 0) {
            if (!wait_band_neighbours(flags, b, G, (unsigned)k + 1u, WAIT_NS)) {
                atomicOr(status, 1);
                s_abort = 1;
            }
            __threadfence();
        }
        __syncwarp();
        __syncthreads();
        if (s_abort) return;
        const double* src = (k & 1) ? buf1 : buf0;
        double* dst = (k & 1) ? buf0 : buf1;
#pragma unroll
        for (int p = 0; p < FUSED_MAX_PPT; ++p) {
            const int i = threadIdx.x + p * blockDim.x;
            if (i < npx) {
                const int iv = r0 + i / nu, iu = i % nu;
                const double c = cur[p];
                const double right = __ldcg(src + iv * nu + min(iu + 1, nu - 1));
                const double down = __ldcg(src + min(iv + 1, nv - 1) * nu + iu);
                const double left = __ldcg(src + iv * nu + max(iu - 1, 0));
                const double up = __ldcg(src + max(iv - 1, 0) * nu + iu);
                const double sigma = ((right + down) + left) + up;
                const double v = (1.0 - omega) * c + (omega / 4.0) * (sigma - inv_beta * (1.0 - sc[p] / c));
                cur[p] = fmax(v, DENOISE_EPS);
                dst[iv * nu + iu] = cur[p];
            }
        }
        __syncwarp();
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_u32(flags + b, (unsigned)k + 2u);
        }
    }
#pragma unroll
    for (int p = 0; p < FUSED_MAX_PPT; ++p) {
        const int i = threadIdx.x + p * blockDim.x;
        if (i < npx) s_out[r0 * nu + i] = cur[p] * count_scale;
    }
}

struct FusedShape {
    int rows, grid, block;
};

// The band shape of the one-launch form on this device, or grid = 0 when the
// image does not fit it (more owned pixels per thread than the registers
// hold, or more bands than can be resident at once).
FusedShape fused_shape(int nu, int nv) {
    FusedShape f{0, 0, 0};
    int dev = 0, n_sm = 0, coop = 0, per_sm = 0;
    if (nu <= 0 || nv <= 0) return f;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, denoise_fused_kernel, 1024, 0) != cudaSuccess)
        return f;
    if (!coop || n_sm <= 0 || per_sm <= 0) return f;
    const int rows = (nv + n_sm - 1) / n_sm;
    const int64_t band = (int64_t)rows * nu;
    int block = (int)std::min<int64_t>(1024, (band + 31) / 32 * 32);
    if ((band + block - 1) / block > FUSED_MAX_PPT) return f;
    const int grid = (nv + rows - 1) / rows;
    if (grid > n_sm * per_sm) return f;
    f.rows = rows;
    f.grid = grid;
    f.block = block;
    return f;
}

}  // namespace

// scratch of the one-launch form: two ping-pong images, then one flag per band
size_t denoise_fused_scratch_bytes(int nu, int nv) {
    return 2 * (size_t)nu * nv * sizeof(double) + (size_t)(nv + 1) * sizeof(unsigned);
}

bool denoise_fused_fits(int nu, int nv) { return fused_shape(nu, nv).grid > 0; }

cudaError_t launch_denoise_fused(const double* s_hat, double* s_out, int nu, int nv, double count_scale,
                                 double beta, const double* scal_dev, double omega, int iters, void* scratch,
                                 int* status, cudaStream_t stream) {
    const FusedShape f = fused_shape(nu, nv);
    if (!f.grid) return cudaErrorInvalidConfiguration;
    double* buf0 = static_cast<double*>(scratch);
    double* buf1 = buf0 + (size_t)nu * nv;
    unsigned* flags = reinterpret_cast<unsigned*>(buf1 + (size_t)nu * nv);
    cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)f.grid * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    int rows = f.rows;
    void* args[] = {(void*)&s_hat, (void*)&s_out, (void*)&nu, (void*)&nv, (void*)&rows, (void*)&count_scale,
                    (void*)&beta, (void*)&scal_dev, (void*)&omega, (void*)&iters, (void*)&buf0, (void*)&buf1,
                    (void*)&flags, (void*)&status};
    return cudaLaunchCooperativeKernel((const void*)denoise_fused_kernel, dim3(f.grid), dim3(f.block), args, 0,
                                       stream);
}

namespace {

// Step 3's scalars of a whole projection (gdrr_project), on the device: the
// count scale (the scatter tally's exact integer sum, as signal per source
// photon, over the scattered photons tallied; 1 / n_photons when none was)
// and beta (given, or smoothing_px^2 over the mean coarse count).  One block;
// scal[0..4] = count scale, beta, mean count, below-floor flag, scattered
// photons.
__global__ void __launch_bounds__(1024) project_scalars_kernel(const int64_t* __restrict__ coarse, int n,
                                                               const unsigned long long* __restrict__ stats,
                                                               double tally_to_signal, double inv_n_photons,
                                                               double beta, double smoothing_px, double floor_,
                                                               double* __restrict__ scal) {
    __shared__ unsigned long long part[32];
    unsigned long long sum = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) sum += (unsigned long long)coarse[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long total = 0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) total += part[w];
        const unsigned long long n_scat = stats[GDRR_ST_TALLY_SCATTER];
        const double n_det = n_scat > 0 ? (double)n_scat : 1.0;
        double cs = (double)total * tally_to_signal / n_det;
        if (!(cs > 0.0)) cs = inv_n_photons;
        const double mean = n_det / (double)n;
        const double b = smoothing_px > 0.0 ? smoothing_px * smoothing_px / fmax(mean, 1e-6) : beta;
        scal[0] = cs;
        scal[1] = b;
        scal[2] = mean;
        scal[3] = (n_scat > 0 && smoothing_px <= 0.0 && b * mean < floor_) ? 1.0 : 0.0;
        scal[4] = (double)n_scat;
    }
}

}  // namespace

cudaError_t launch_project_scalars(const int64_t* coarse, int n, const unsigned long long* stats,
                                   double tally_to_signal, double inv_n_photons, double beta, double smoothing_px,
                                   double floor_, double* scal, cudaStream_t s) {
    project_scalars_kernel<<<1, 1024, 0, s>>>(coarse, n, stats, tally_to_signal, inv_n_photons, beta, smoothing_px,
                                              floor_, scal);
    return cudaGetLastError();
}

// scratch: 2 * nu * nv doubles (count-scale data, one ping-pong buffer); the
// other ping-pong buffer is the output.
cudaError_t launch_denoise(const double* s_hat, double* s_out, int nu, int nv, double count_scale, double beta,
                           const double* scal_dev, double omega, int iters, double* scratch, cudaStream_t stream) {
    const int n = nu * nv;
    if (n <= 0) return cudaSuccess;
    double* sc = scratch;
    double* buf[2] = {s_out, scratch + n};
    denoise_init<<<grid_for(n), BLOCK, 0, stream>>>(s_hat, n, count_scale, scal_dev, sc, buf[0]);
    for (int k = 0; k < iters; ++k)
        denoise_step<<<grid_for(n), BLOCK, 0, stream>>>(sc, buf[k & 1], nu, nv, omega, beta, scal_dev,
                                                        buf[(k + 1) & 1]);
    // result (count scale) sits in buf[iters & 1]; return it on the input scale
    scale_kernel<<<grid_for(n), BLOCK, 0, stream>>>(buf[iters & 1], n, count_scale, scal_dev, s_out);
    return cudaGetLastError();
}

}  // namespace gdrr

// ---------------------------------------------------------------------------
// Allocation-free variant of the scatter denoiser.
//
// Some callers cannot allocate device memory: host applications that hand a
// plug-in a fixed device-memory budget and own the allocator, or code that
// must not call cudaMalloc / cudaFree because those calls can synchronise the
// device and stall other work.  gdrr_denoise_scatter_static serves them: it
// takes no context and allocates nothing; its ping-pong scratch is the
// file-scope device array below, which every GPU that loads this library
// holds until the process exits.
namespace gdrr {
namespace {

constexpr int STATIC_DENOISE_MAX_PIXELS = GDRR_STATIC_DENOISE_MAX_PIXELS;
static __device__ __align__(256) double g_denoise_scratch[2 * (size_t)STATIC_DENOISE_MAX_PIXELS];

// The device address of g_denoise_scratch in the current context.  In host
// code the array's name is only a host-side stand-in, so the address is looked
// up on every call: it moves when the module is loaded again (a device reset,
// a primary context released and created again), and the lookup allocates
// nothing.
cudaError_t static_scratch(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_denoise_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

}  // namespace
}  // namespace gdrr

extern "C" GDRR_API int gdrr_denoise_scatter_static(const double* S_hat_dev, double* S_dev, int32_t nu, int32_t nv,
                                                   double count_scale, double beta, double omega, int32_t iters,
                                                   void* cuda_stream) {
    if (!S_hat_dev || !S_dev || nu <= 0 || nv <= 0 || iters < 0) return GDRR_ERR_INVALID_ARG;
    if (!(count_scale > 0) || !(beta > 0) || !(omega > 0 && omega < 2) || !isfinite(count_scale) || !isfinite(beta))
        return GDRR_ERR_INVALID_ARG;
    if ((int64_t)nu * nv > gdrr::STATIC_DENOISE_MAX_PIXELS) return GDRR_ERR_INVALID_ARG;
    double* scratch = nullptr;
    cudaError_t e = gdrr::static_scratch(&scratch);
    if (e == cudaSuccess)
        e = gdrr::launch_denoise(S_hat_dev, S_dev, nu, nv, count_scale, beta, nullptr, omega, iters, scratch,
                                 (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? GDRR_OK : GDRR_ERR_CUDA;
}
