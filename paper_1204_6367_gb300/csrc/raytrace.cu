// Tri-linear ray-traced primary, Section 2.3 / Eq. 1, for sm_103a.
//
// One thread per detector pixel (as in the paper).  The ray from the source
// to the pixel centre is cut, inside the phantom box, into n equal intervals
// of length dl <= half the smallest voxel size; the field is evaluated at the
// interval midpoints with trilinear interpolation (clamp to edge).
//
// Difference from the paper's implementation: the paper repeats the trace for
// every energy channel (~100) with hardware texture interpolation of mu.
// Here mu(x, E) = sum_m mu_hat(m, E) rho_m(x) is linear in the per-material
// trilinear partial densities rho_m, so one trace accumulates the path
// integrals l_m = sum_j dl rho_m(x_j) and the channel sum
//   P = w(u) sum_b phi_b r(E_b) exp(-sum_m mu_hat(m, E_b) l_m)
// follows from them: the same discretised quantity with one trace instead of
// ~100.  Software FP32 interpolation replaces the texture unit's 8-bit
// fixed-point weights.
#include "gdrr_internal.cuh"

namespace gdrr {
namespace {

constexpr int RT_MAX_BINS = 512;

template <int NM>
__global__ void __launch_bounds__(128) rt_kernel(const RtParams P, double* __restrict__ out) {
    __shared__ float s_mu[RT_MAX_BINS * NM];
    __shared__ float s_wr[RT_MAX_BINS];
    for (int i = threadIdx.x; i < P.n_bins * NM; i += blockDim.x) {
        const int b = i / NM, m = i % NM;
        s_mu[i] = m < P.n_mat ? P.mu_rt[b * P.n_mat + m] : 0.0f;
    }
    for (int i = threadIdx.x; i < P.n_bins; i += blockDim.x) s_wr[i] = P.wr[i];
    __syncthreads();

    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.nu * P.nv) return;
    const int iu = j % P.nu, iv = j / P.nu;
    const float au = ((float)iu + 0.5f - P.hu) * P.du;
    const float av = ((float)iv + 0.5f - P.hv) * P.dv;
    float d[3], S[3];
    float L2 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        S[a] = P.f.S[a];
        d[a] = P.f.P[a] + au * P.f.eu[a] + av * P.f.ev[a] - S[a];
        L2 += d[a] * d[a];
    }
    const float L = sqrtf(L2);
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] /= L;
    float tmin = 0.0f, tmax = L;
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0f) {
            float t1 = (P.lo[a] - S[a]) / d[a], t2 = (P.hi[a] - S[a]) / d[a];
            if (t1 > t2) { const float t = t1; t1 = t2; t2 = t; }
            tmin = fmaxf(tmin, t1);
            tmax = fminf(tmax, t2);
        } else if (S[a] < P.lo[a] || S[a] > P.hi[a]) {
            hit = false;
        }
    }
    float ell[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) ell[m] = 0.0f;
    if (hit && tmax > tmin) {
        const float chord = tmax - tmin;
        const int n = (int)ceilf(chord / P.half_step);
        const float dl = chord / (float)n;
        const int dims[3] = {P.nx, P.ny, P.nz};
        // voxel-coordinate start and increment of the midpoints
        float f0[3], df[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float x0 = S[a] + (tmin + 0.5f * dl) * d[a];
            f0[a] = (x0 - P.lo[a]) * P.ivox[a] - 0.5f;
            df[a] = dl * d[a] * P.ivox[a];
        }
        for (int s = 0; s < n; ++s) {
            int i0[3], i1[3];
            float w1[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float fa = f0[a] + (float)s * df[a];
                int g0 = (int)floorf(fa);
                w1[a] = fa - (float)g0;
                int g1 = g0 + 1;
                g0 = min(max(g0, 0), dims[a] - 1);
                g1 = min(max(g1, 0), dims[a] - 1);
                i0[a] = g0; i1[a] = g1;
            }
#pragma unroll
            for (int corner = 0; corner < 8; ++corner) {
                const int cx = corner & 1, cy = (corner >> 1) & 1, cz = corner >> 2;
                const int v = brick_x(cx ? i1[0] : i0[0]) + brick_y(cy ? i1[1] : i0[1], P.bsy)
                            + brick_z(cz ? i1[2] : i0[2], P.bsz);
                const float w = (cx ? w1[0] : 1.0f - w1[0]) * (cy ? w1[1] : 1.0f - w1[1])
                              * (cz ? w1[2] : 1.0f - w1[2]);
                const uint2 vx = __ldg(P.vox + v);
                const float a = w * __uint_as_float(vx.x);
                const int mc = (int)vx.y;
#pragma unroll
                for (int m = 0; m < NM; ++m) ell[m] += (mc == m ? a : 0.0f);
            }
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) ell[m] *= dl;
    }
    // channel weights: the shared separable spectrum, or this column's own
    const float* wcol = P.wr_cols ? P.wr_cols + (size_t)iu * P.n_bins : nullptr;
    float sig = 0.0f;
    for (int b = 0; b < P.n_bins; ++b) {
        float rad = 0.0f;
#pragma unroll
        for (int m = 0; m < NM; ++m) rad += s_mu[b * NM + m] * ell[m];
        sig += (wcol ? __ldg(wcol + b) : s_wr[b]) * expf(-rad);
    }
    out[j] = P.wnorm[j] * (double)sig;
}

// Siddon's algorithm as a 3-D digital differential analyser: the ray visits
// the voxels it crosses in order, each for the exact length between its entry
// and exit planes (Siddon, Med. Phys. 12, 1985; voxel stepping after Amanatides
// and Woo, 1987).  Parametric distances in FP64 (they reach ~1500 mm while
// the segments are ~1 mm), per-material path integrals in FP32.
template <int NM>
__global__ void __launch_bounds__(128) rt_siddon_kernel(const RtParams P, double* __restrict__ out) {
    __shared__ float s_mu[RT_MAX_BINS * NM];
    __shared__ float s_wr[RT_MAX_BINS];
    for (int i = threadIdx.x; i < P.n_bins * NM; i += blockDim.x) {
        const int b = i / NM, m = i % NM;
        s_mu[i] = m < P.n_mat ? P.mu_rt[b * P.n_mat + m] : 0.0f;
    }
    for (int i = threadIdx.x; i < P.n_bins; i += blockDim.x) s_wr[i] = P.wr[i];
    __syncthreads();

    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.nu * P.nv) return;
    const int iu = j % P.nu, iv = j / P.nu;
    const double au = ((double)iu + 0.5 - (double)P.hu) * (double)P.du;
    const double av = ((double)iv + 0.5 - (double)P.hv) * (double)P.dv;
    double d[3], S[3], L2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        S[a] = P.f.S[a];
        d[a] = (double)P.f.P[a] + au * (double)P.f.eu[a] + av * (double)P.f.ev[a] - S[a];
        L2 += d[a] * d[a];
    }
    const double L = sqrt(L2);
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] /= L;
    double tmin = 0.0, tmax = L;
    bool hit = true;
    const double lo[3] = {P.lo[0], P.lo[1], P.lo[2]};
    const double hi[3] = {P.hi[0], P.hi[1], P.hi[2]};
    const double vox[3] = {1.0 / (double)P.ivox[0], 1.0 / (double)P.ivox[1], 1.0 / (double)P.ivox[2]};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0) {
            double t1 = (lo[a] - S[a]) / d[a], t2 = (hi[a] - S[a]) / d[a];
            if (t1 > t2) { const double t = t1; t1 = t2; t2 = t; }
            tmin = fmax(tmin, t1);
            tmax = fmin(tmax, t2);
        } else if (S[a] < lo[a] || S[a] > hi[a]) {
            hit = false;
        }
    }
    float ell[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) ell[m] = 0.0f;
    if (hit && tmax > tmin) {
        const int dims[3] = {P.nx, P.ny, P.nz};
        int idx[3], stp[3];
        double tnext[3], tdelta[3];
        const double tm = 0.5 * (tmin + fmin(tmax, tmin + 1e-3));   // a point just inside the box
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double x = S[a] + tm * d[a];
            idx[a] = min(max((int)floor((x - lo[a]) / vox[a]), 0), dims[a] - 1);
            if (d[a] > 0.0) {
                stp[a] = 1;
                tnext[a] = (lo[a] + (idx[a] + 1) * vox[a] - S[a]) / d[a];
                tdelta[a] = vox[a] / d[a];
            } else if (d[a] < 0.0) {
                stp[a] = -1;
                tnext[a] = (lo[a] + idx[a] * vox[a] - S[a]) / d[a];
                tdelta[a] = -vox[a] / d[a];
            } else {
                stp[a] = 0;
                tnext[a] = 1e300;
                tdelta[a] = 1e300;
            }
        }
        double t = tmin;
        const int max_cross = P.nx + P.ny + P.nz + 3;
        for (int it = 0; it < max_cross && t < tmax; ++it) {
            const int ax = tnext[0] < tnext[1] ? (tnext[0] < tnext[2] ? 0 : 2) : (tnext[1] < tnext[2] ? 1 : 2);
            const double t1 = fmin(tnext[ax], tmax);
            const float len = (float)(t1 - t);
            const uint2 vx = __ldg(P.vox + brick_x(idx[0]) + brick_y(idx[1], P.bsy) + brick_z(idx[2], P.bsz));
            const float a = len * __uint_as_float(vx.x);
            const int mc = (int)vx.y;
#pragma unroll
            for (int m = 0; m < NM; ++m) ell[m] += (mc == m ? a : 0.0f);
            t = t1;
            idx[ax] += stp[ax];
            tnext[ax] += tdelta[ax];
            if (idx[ax] < 0 || idx[ax] >= dims[ax]) break;
        }
    }
    // channel weights: the shared separable spectrum, or this column's own
    const float* wcol = P.wr_cols ? P.wr_cols + (size_t)iu * P.n_bins : nullptr;
    float sig = 0.0f;
    for (int b = 0; b < P.n_bins; ++b) {
        float rad = 0.0f;
#pragma unroll
        for (int m = 0; m < NM; ++m) rad += s_mu[b * NM + m] * ell[m];
        sig += (wcol ? __ldg(wcol + b) : s_wr[b]) * expf(-rad);
    }
    out[j] = P.wnorm[j] * (double)sig;
}

// The unattenuated signal of each pixel: w(u) sum_b phi_u(b) r(E_b).
__global__ void air_kernel(const RtParams P, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.nu * P.nv) return;
    const int iu = j % P.nu;
    const float* w = P.wr_cols ? P.wr_cols + (size_t)iu * P.n_bins : P.wr;
    float sig = 0.0f;
    for (int b = 0; b < P.n_bins; ++b) sig += __ldg(w + b);
    out[j] = P.wnorm[j] * (double)sig;
}

}  // namespace

cudaError_t launch_air(const RtParams& p, double* out, cudaStream_t s) {
    const int npix = p.nu * p.nv;
    const int block = 128, grid = (npix + block - 1) / block;
    air_kernel<<<grid, block, 0, s>>>(p, out);
    return cudaGetLastError();
}

cudaError_t launch_rt_siddon(const RtParams& p, double* out, cudaStream_t s) {
    if (p.n_bins > RT_MAX_BINS) return cudaErrorInvalidValue;
    const int npix = p.nu * p.nv;
    const int block = 128, grid = (npix + block - 1) / block;
    if (p.n_mat <= 2) rt_siddon_kernel<2><<<grid, block, 0, s>>>(p, out);
    else if (p.n_mat <= 4) rt_siddon_kernel<4><<<grid, block, 0, s>>>(p, out);
    else rt_siddon_kernel<8><<<grid, block, 0, s>>>(p, out);
    return cudaGetLastError();
}

cudaError_t launch_rt(const RtParams& p, double* out, cudaStream_t s) {
    if (p.n_bins > RT_MAX_BINS) return cudaErrorInvalidValue;
    const int npix = p.nu * p.nv;
    const int block = 128, grid = (npix + block - 1) / block;
    if (p.n_mat <= 2) rt_kernel<2><<<grid, block, 0, s>>>(p, out);
    else if (p.n_mat <= 4) rt_kernel<4><<<grid, block, 0, s>>>(p, out);
    else rt_kernel<8><<<grid, block, 0, s>>>(p, out);
    return cudaGetLastError();
}

}  // namespace gdrr
