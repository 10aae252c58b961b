// Cone-beam reconstruction of simulated scans (Section 3.5 reconstructs the
// simulated projections with an FDK algorithm).  Feldkamp-Davis-Kress for the
// circular orbit of Section 2.1 with the imager opposite the source, in the
// textbook form (Kak & Slaney, equally spaced fan beam, Feldkamp's cone
// weighting):
//   * line integrals g = -ln(I / I0) against the air scan I0;
//   * virtual detector at the isocentre (a = u SAD / SDD, b = v SAD / SDD,
//     spacing tau = du SAD / SDD), cosine weight SAD / sqrt(SAD^2 + a^2 + b^2);
//   * Ram-Lak ramp along each row as a linear convolution with zeros outside
//     the row, times the 1/2 of the full-scan fan-beam formula:
//     Qf(n) = (1 / (2 tau)) (q(n) / 4 - sum_{odd d} q(n - d) / (pi d)^2);
//   * voxel-driven backprojection f(x) = sum_beta dbeta (SAD / depth)^2
//     Qf(a(x), b(x)), depth = SAD + x.n, bilinear on the pixel-centre grid,
//     zero outside the detector.
// The filter is a short dense row convolution (nu^2 / 2 FMAs per row) done
// in shared memory with register tiling; the backprojection gathers 4 detector samples per voxel
// and view from L1 / L2 and keeps 8 voxels of a column in registers, so the
// per-view geometry (depth, u, weight) is computed once per column.
#include <cmath>

#include "gdrr_internal.cuh"

namespace gdrr {
namespace {

constexpr int FILTER_BLOCK = 256;
constexpr int FILTER_MAX_NU = 4096;
constexpr int BP_MAX_ANGLES = 128;     // views per backprojection launch (kernel parameters)
constexpr int BP_ZT = 8;               // voxels of a column per thread
constexpr int BP_BX = 32, BP_BY = 8;

struct FilterParams {
    int nu, nv;
    float mag_du, mag_dv;   // virtual-detector spacings tau_u, tau_v (mm)
    float sad;
    float scale;            // 1 / (2 tau_u)
};

// Register tiling: a thread owns FJ outputs of one parity, n_j = n0 + 2j.
// Only sources k of the other parity contribute (odd offsets), and as k
// advances by 2 the offsets |n_j - k| all move by 2 in the same direction, so
// the FJ coefficients in use form a window that slides by one slot per
// source: one shared-memory load of q(k) and one of the entering coefficient
// serve FJ FMAs.  Sources between n_0 and n_{FJ-1} are taken directly.
constexpr int FJ = 4;

__global__ void __launch_bounds__(FILTER_BLOCK) fdk_filter_kernel(const FilterParams p, const float* __restrict__ g,
                                                                 float* __restrict__ out) {
    extern __shared__ float sm[];
    float* q = sm;                // weighted row [nu]
    float* c = sm + p.nu;         // offset |d| -> kernel coefficient [nu + 2 FJ]
    const int nu = p.nu;
    const int row = blockIdx.x;
    const size_t base = ((size_t)blockIdx.y * p.nv + row) * nu;
    const float b = ((float)row + 0.5f - 0.5f * (float)p.nv) * p.mag_dv;
    const float sad2b2 = p.sad * p.sad + b * b;
    for (int k = threadIdx.x; k < nu; k += blockDim.x) {
        const float a = ((float)k + 0.5f - 0.5f * (float)nu) * p.mag_du;
        q[k] = g[base + k] * (p.sad / sqrtf(sad2b2 + a * a));
    }
    for (int k = threadIdx.x; k < nu + 2 * FJ; k += blockDim.x) {
        float ck = 0.0f;
        if (k == 0) {
            ck = 0.25f;
        } else if (k & 1) {
            const float pd = 3.14159265358979f * (float)k;
            ck = -1.0f / (pd * pd);
        }
        c[k] = ck;
    }
    __syncthreads();
    const int n_groups = 2 * ((nu + 2 * FJ - 1) / (2 * FJ));
    for (int grp = threadIdx.x; grp < n_groups; grp += blockDim.x) {
        const int par = grp & 1;
        const int n0 = 2 * FJ * (grp >> 1) + par;
        float acc[FJ], w[FJ];
#pragma unroll
        for (int j = 0; j < FJ; ++j) acc[j] = (n0 + 2 * j < nu) ? c[0] * q[n0 + 2 * j] : 0.0f;
        // sources below n0: offsets n_j - k, shrinking by 2 per source
        int k = 1 - par;
        if (k < n0) {
#pragma unroll
            for (int j = 0; j < FJ; ++j) w[j] = c[n0 - k + 2 * j];
            for (; k < n0; k += 2) {
                const float qk = q[k];
#pragma unroll
                for (int j = 0; j < FJ; ++j) acc[j] += w[j] * qk;
#pragma unroll
                for (int j = FJ - 1; j > 0; --j) w[j] = w[j - 1];
                w[0] = c[max(n0 - k - 2, 0)];
            }
        }
        // sources between n_0 and n_{FJ-1}
        for (k = n0 + 1; k < n0 + 2 * (FJ - 1) && k < nu; k += 2) {
            const float qk = q[k];
#pragma unroll
            for (int j = 0; j < FJ; ++j) acc[j] += c[abs(n0 + 2 * j - k)] * qk;
        }
        // sources above n_{FJ-1}: offsets k - n_j, growing by 2 per source
        k = n0 + 2 * FJ - 1;
        if (k < nu) {
#pragma unroll
            for (int j = 0; j < FJ; ++j) w[j] = c[k - n0 - 2 * j];
            for (; k < nu; k += 2) {
                const float qk = q[k];
#pragma unroll
                for (int j = 0; j < FJ; ++j) acc[j] += w[j] * qk;
#pragma unroll
                for (int j = FJ - 1; j > 0; --j) w[j] = w[j - 1];
                w[0] = c[min(k + 2 - n0, nu + 2 * FJ - 1)];
            }
        }
#pragma unroll
        for (int j = 0; j < FJ; ++j)
            if (n0 + 2 * j < nu) out[base + n0 + 2 * j] = p.scale * acc[j];
    }
}

struct BpParams {
    int nx, ny, nz, nu, nv;
    float x0, y0, z0;        // first voxel centre (mm)
    float dx, dy, dz;
    float sad;
    float inv_tau_u, inv_tau_v;
    float hu, hv;            // nu / 2 - 1/2, nv / 2 - 1/2
    float d_beta;
    int n_ang;
    int accumulate;          // 1: add to the volume, 0: overwrite it
    float2 cs[BP_MAX_ANGLES];   // (cos phi, sin phi) of each view
    int first_view;          // index of cs[0] in the filtered stack
};

__device__ __forceinline__ float tap(const float* __restrict__ img, int nu, int nv, int iu, int iv) {
    return (iu >= 0 && iu < nu && iv >= 0 && iv < nv) ? __ldg(img + (size_t)iv * nu + iu) : 0.0f;
}

__global__ void __launch_bounds__(BP_BX * BP_BY) fdk_backproject_kernel(const BpParams p, const float* __restrict__ q,
                                                                       float* __restrict__ vol) {
    const int ix = blockIdx.x * BP_BX + threadIdx.x;
    const int iy = blockIdx.y * BP_BY + threadIdx.y;
    const int iz0 = blockIdx.z * BP_ZT;
    if (ix >= p.nx || iy >= p.ny) return;
    const float x = p.x0 + (float)ix * p.dx;
    const float y = p.y0 + (float)iy * p.dy;
    float acc[BP_ZT];
#pragma unroll
    for (int k = 0; k < BP_ZT; ++k) acc[k] = 0.0f;
    const size_t view = (size_t)p.nu * p.nv;
    for (int i = 0; i < p.n_ang; ++i) {
        const float cph = p.cs[i].x, sph = p.cs[i].y;
        const float depth = p.sad + x * cph + y * sph;
        const float inv = 1.0f / depth;
        const float fu = p.sad * (x * sph - y * cph) * inv * p.inv_tau_u + p.hu;
        const float fiu = floorf(fu);
        if (fiu < -1.0f || fiu > (float)(p.nu - 1)) continue;   // the column misses the detector
        const int iu = (int)fiu;
        const float wu = fu - fiu;
        const float m = p.sad * inv;
        const float w2 = p.d_beta * (m * m);
        const float sv = m * p.inv_tau_v;                           // dv-index per mm of z
        const float* img = q + (size_t)(p.first_view + i) * view;
#pragma unroll
        for (int k = 0; k < BP_ZT; ++k) {
            const float z = p.z0 + (float)(iz0 + k) * p.dz;
            // clamped two samples beyond the edges (those taps read zero)
            const float fv = fminf(fmaxf(z * sv + p.hv, -2.0f), (float)p.nv + 1.0f);
            const float fiv = floorf(fv);
            const int iv = (int)fiv;
            const float wv = fv - fiv;
            const float v00 = tap(img, p.nu, p.nv, iu, iv), v10 = tap(img, p.nu, p.nv, iu + 1, iv);
            const float v01 = tap(img, p.nu, p.nv, iu, iv + 1), v11 = tap(img, p.nu, p.nv, iu + 1, iv + 1);
            const float val = (1.0f - wv) * ((1.0f - wu) * v00 + wu * v10) + wv * ((1.0f - wu) * v01 + wu * v11);
            acc[k] += w2 * val;
        }
    }
#pragma unroll
    for (int k = 0; k < BP_ZT; ++k) {
        const int iz = iz0 + k;
        if (iz < p.nz) {
            const size_t o = ((size_t)iz * p.ny + iy) * p.nx + ix;
            vol[o] = p.accumulate ? vol[o] + acc[k] : acc[k];
        }
    }
}

__global__ void line_integral_kernel(const double* __restrict__ s, const double* __restrict__ a, int64_t n,
                                     double floor_rel, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double i0 = a[i];
    const double v = fmax(s[i], floor_rel * i0);
    out[i] = (float)(-log(v / i0));
}

bool geometry_valid(const gdrr_fdk_geometry* g) {
    return g && g->sad_mm > 0 && g->sdd_mm > g->sad_mm && g->nu > 0 && g->nv > 0 && g->du_mm > 0 && g->dv_mm > 0
           && g->nx > 0 && g->ny > 0 && g->nz > 0 && g->dx_mm > 0 && g->dy_mm > 0 && g->dz_mm > 0
           && std::isfinite(g->sad_mm) && std::isfinite(g->sdd_mm);
}

}  // namespace
}  // namespace gdrr

extern "C" GDRR_API int gdrr_line_integrals(const double* signal_dev, const double* air_dev, int64_t n,
                                            double floor_rel, float* out_dev, void* cuda_stream) {
    if (n < 0 || (n > 0 && (!signal_dev || !air_dev || !out_dev)) || !(floor_rel > 0.0) || !(floor_rel < 1.0))
        return GDRR_ERR_INVALID_ARG;
    if (n == 0) return GDRR_OK;
    const int block = 256;
    gdrr::line_integral_kernel<<<(unsigned)((n + block - 1) / block), block, 0, (cudaStream_t)cuda_stream>>>(
        signal_dev, air_dev, n, floor_rel, out_dev);
    return cudaGetLastError() == cudaSuccess ? GDRR_OK : GDRR_ERR_CUDA;
}

extern "C" GDRR_API int gdrr_fdk_filter(const gdrr_fdk_geometry* g, int32_t n_proj, const float* proj_dev,
                                        float* filtered_dev, void* cuda_stream) {
    if (!gdrr::geometry_valid(g) || n_proj < 0 || (n_proj > 0 && (!proj_dev || !filtered_dev)))
        return GDRR_ERR_INVALID_ARG;
    if (g->nu > gdrr::FILTER_MAX_NU || g->nv > 65535 || n_proj > 65535) return GDRR_ERR_UNSUPPORTED;
    if (n_proj == 0) return GDRR_OK;
    gdrr::FilterParams p;
    const double mag = g->sad_mm / g->sdd_mm;
    p.nu = g->nu; p.nv = g->nv;
    p.mag_du = (float)(g->du_mm * mag);
    p.mag_dv = (float)(g->dv_mm * mag);
    p.sad = (float)g->sad_mm;
    p.scale = (float)(0.5 / (g->du_mm * mag));
    const dim3 grid((unsigned)g->nv, (unsigned)n_proj);
    const size_t smem = sizeof(float) * (2 * (size_t)g->nu + 2 * gdrr::FJ);
    gdrr::fdk_filter_kernel<<<grid, gdrr::FILTER_BLOCK, smem, (cudaStream_t)cuda_stream>>>(p, proj_dev, filtered_dev);
    return cudaGetLastError() == cudaSuccess ? GDRR_OK : GDRR_ERR_CUDA;
}

extern "C" GDRR_API int gdrr_fdk_backproject(const gdrr_fdk_geometry* g, int32_t n_proj, const double* angles_rad,
                                             double d_beta, const float* filtered_dev, float* volume_dev,
                                             int32_t accumulate, void* cuda_stream) {
    if (!gdrr::geometry_valid(g) || n_proj < 0 || !volume_dev || (n_proj > 0 && (!angles_rad || !filtered_dev))
        || !std::isfinite(d_beta) || (accumulate != 0 && accumulate != 1))
        return GDRR_ERR_INVALID_ARG;
    for (int i = 0; i < n_proj; ++i)
        if (!std::isfinite(angles_rad[i])) return GDRR_ERR_INVALID_ARG;
    // every voxel must lie on the source's side of the isocentre plane at
    // every angle (depth > 0): the grid's half-diagonal stays below SAD
    const double hx = 0.5 * g->nx * g->dx_mm, hy = 0.5 * g->ny * g->dy_mm;
    if (!(std::sqrt(hx * hx + hy * hy) < g->sad_mm)) return GDRR_ERR_INVALID_ARG;
    if ((int64_t)g->ny > 65535 * (int64_t)gdrr::BP_BY) return GDRR_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const double mag = g->sad_mm / g->sdd_mm;
    gdrr::BpParams p;
    p.nx = g->nx; p.ny = g->ny; p.nz = g->nz; p.nu = g->nu; p.nv = g->nv;
    p.x0 = (float)((0.5 - 0.5 * g->nx) * g->dx_mm);
    p.y0 = (float)((0.5 - 0.5 * g->ny) * g->dy_mm);
    p.z0 = (float)((0.5 - 0.5 * g->nz) * g->dz_mm);
    p.dx = (float)g->dx_mm; p.dy = (float)g->dy_mm; p.dz = (float)g->dz_mm;
    p.sad = (float)g->sad_mm;
    p.inv_tau_u = (float)(1.0 / (g->du_mm * mag));
    p.inv_tau_v = (float)(1.0 / (g->dv_mm * mag));
    p.hu = (float)(0.5 * g->nu - 0.5);
    p.hv = (float)(0.5 * g->nv - 0.5);
    p.d_beta = (float)d_beta;
    const dim3 block(gdrr::BP_BX, gdrr::BP_BY);
    const dim3 grid((unsigned)((g->nx + gdrr::BP_BX - 1) / gdrr::BP_BX), (unsigned)((g->ny + gdrr::BP_BY - 1) / gdrr::BP_BY),
                    (unsigned)((g->nz + gdrr::BP_ZT - 1) / gdrr::BP_ZT));
    if (n_proj == 0 && !accumulate) {
        if (cudaMemsetAsync(volume_dev, 0, sizeof(float) * (size_t)g->nx * g->ny * g->nz, s) != cudaSuccess)
            return GDRR_ERR_CUDA;
        return GDRR_OK;
    }
    for (int first = 0; first < n_proj; first += gdrr::BP_MAX_ANGLES) {
        const int n = std::min(gdrr::BP_MAX_ANGLES, n_proj - first);
        p.n_ang = n;
        p.first_view = first;
        p.accumulate = (first > 0 || accumulate) ? 1 : 0;
        for (int i = 0; i < n; ++i)
            p.cs[i] = make_float2((float)std::cos(angles_rad[first + i]), (float)std::sin(angles_rad[first + i]));
        gdrr::fdk_backproject_kernel<<<grid, block, 0, s>>>(p, filtered_dev, volume_dev);
        if (cudaGetLastError() != cudaSuccess) return GDRR_ERR_CUDA;
    }
    return GDRR_OK;
}
