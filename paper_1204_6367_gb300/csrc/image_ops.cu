// Image-domain steps of the paper on sm_103a, all FP64:
//  * tally -> signal per source photon (Section 2.6 normalisation);
//  * exact integer binning to the coarse scatter grid, bilinear upsampling;
//  * Step 3, Section 2.5: the Eq. 5 relaxation iteration of the Poisson
//    denoiser (Eq. 2-4), one launch per iteration with ping-pong buffers;
//  * Step 4, Section 2.6: N = ((P^ - P) + (S^ - S)) * alpha.
// These are element-wise or 5-point-stencil passes over at most a detector
// image (196,608 pixels): launch- and latency-bound, not bandwidth-bound.
#include <mutex>

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

__global__ void denoise_init(const double* __restrict__ s_hat, int n, double inv_scale, double* __restrict__ sc,
                             double* __restrict__ s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = s_hat[i] * inv_scale;
    sc[i] = v;
    s[i] = fmax(v, DENOISE_EPS);
}

// One Eq. 5 update: S' = (1 - w) S + w/4 [ Sigma S - (1/beta)(1 - S^/S) ],
// Sigma S = S(i+1,j) + S(i,j+1) + S(i-1,j) + S(i,j-1), replicate edges.
__global__ void denoise_step(const double* __restrict__ sc, const double* __restrict__ s, int nu, int nv,
                             double omega, double inv_beta, double* __restrict__ s_next) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nu * nv) return;
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

__global__ void scale_kernel(const double* __restrict__ a, int n, double scale, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] * scale;
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

// scratch: 2 * nu * nv doubles (count-scale data, one ping-pong buffer); the
// other ping-pong buffer is the output.
cudaError_t launch_denoise(const double* s_hat, double* s_out, int nu, int nv, double count_scale, double beta,
                           double omega, int iters, double* scratch, cudaStream_t stream) {
    const int n = nu * nv;
    if (n <= 0) return cudaSuccess;
    double* sc = scratch;
    double* buf[2] = {s_out, scratch + n};
    denoise_init<<<grid_for(n), BLOCK, 0, stream>>>(s_hat, n, 1.0 / count_scale, sc, buf[0]);
    for (int k = 0; k < iters; ++k)
        denoise_step<<<grid_for(n), BLOCK, 0, stream>>>(sc, buf[k & 1], nu, nv, omega, 1.0 / beta, buf[(k + 1) & 1]);
    // result (count scale) sits in buf[iters & 1]; return it on the input scale
    scale_kernel<<<grid_for(n), BLOCK, 0, stream>>>(buf[iters & 1], n, count_scale, s_out);
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
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_denoise_scratch[2 * (size_t)STATIC_DENOISE_MAX_PIXELS];

std::mutex g_scratch_mutex;
double* g_scratch_addr[MAX_DEVICES] = {nullptr};

// The device address of g_denoise_scratch on the current device.  In host
// code the array's name is only a host-side stand-in, so the address is
// looked up with cudaGetSymbolAddress once per device, with that device
// current, and cached.
cudaError_t static_scratch(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_denoise_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
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
        e = gdrr::launch_denoise(S_hat_dev, S_dev, nu, nv, count_scale, beta, omega, iters, scratch,
                                 (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? GDRR_OK : GDRR_ERR_CUDA;
}
