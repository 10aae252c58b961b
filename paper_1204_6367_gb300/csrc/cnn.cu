// Learned scatter estimator: a 4-level convolutional encoder-decoder trained
// and run on the GPU with the library's own kernels (BF16 weights and
// activations, FP32 accumulation on the tcgen05 tensor cores, FP32 master
// weights, gradients and Adam state).
//
// Architecture (base channels c = 32, input 2 x H x W, H and W multiples of 8):
//   e1 = relu(conv3x3(x,   2 -> c))          H   x W
//   e2 = relu(conv3x3(pool(e1), c -> 2c))    H/2 x W/2
//   e3 = relu(conv3x3(pool(e2), 2c -> 4c))   H/4 x W/4
//   e4 = relu(conv3x3(pool(e3), 4c -> 8c))   H/8 x W/8
//   d3 = relu(conv3x3([up(e4), e3], 12c -> 4c))
//   d2 = relu(conv3x3([up(d3), e2],  6c -> 2c))
//   d1 = relu(conv3x3([up(d2), e1],  3c -> c))
//   y  = conv1x1(d1, c -> 1) + x[channel 0]   (residual: a correction to input 0)
// pool = 2 x 2 average, up = nearest 2x, [a, b] = channel concatenation.
// Loss: mean squared error against the target.
//
// Layout.  Activations are NHWC BF16.  Each decoder input [up(prev), skip]
// is one buffer cat_k (H_k x W_k pixels, pitch C_prev + C_skip): the
// encoder convolution that makes the skip writes it in place (channels
// C_prev ..), and the convolution one level down writes its output there
// upsampled (channels 0 .. C_prev - 1, each pixel to its 2 x 2 block).  The
// encoder output e4 and the decoder outputs d3, d2 exist only in that form.
//
// Convolutions.  A 3 x 3 convolution is a GEMM with K = (tap, channel):
//   forward   Y[P x Co]   = cols(x)[P x 9Ci] . W[Co x 9Ci]^T
//   data grad dX[P x Ci]  = cols(dZ)[P x 9Co] . Wf[Ci x 9Co]^T   (Wf: taps flipped)
//   weight    dW[Co x 9Ci] = dZ^T[Co x P] . cols(x)[P x 9Ci]
// The forward and data-gradient products run as implicit GEMMs
// (launch_conv_implicit: the tensor-core kernel loads each tap's shifted input
// tile by TMA, no column matrix) where the layer's grid tiles into 128-pixel
// rows; otherwise, and for the weight gradient (whose K runs over pixels),
// a column matrix is built and multiplied by launch_gemm_bf16.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "cnn_epi.cuh"
#include "gdrr_internal.cuh"

namespace gdrr {

cudaError_t launch_gemm_bf16(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M, int N, int K,
                             int splits, int* err, cudaStream_t s, int64_t partial_stride = 0,
                             int* splits_used = nullptr);

namespace {

typedef __nv_bfloat16 bf16;
constexpr int TB = 256;
inline int nblk(int64_t n) { return (int)((n + TB - 1) / TB); }
inline int pad64(int64_t n) { return (int)((n + 63) / 64 * 64); }

// A BF16 NHWC tensor on a grid H x W: pixel (b, y, x) channel c at
// p[q ld + off + c] with q = (b H s + y s) (W s) + x s; s = up = 2 when the
// tensor is stored upsampled on a 2H x 2W grid (it reads pixel (2y, 2x)).
struct View {
    const bf16* p;
    int ld, off, up;
};

View plain(const bf16* p, int ld, int off = 0) { return View{p, ld, off, 1}; }

__device__ __forceinline__ int64_t view_pixel(const View& v, int64_t p, int H, int W) {
    const int64_t hw = (int64_t)H * W;
    const int64_t b = p / hw;
    const int r = (int)(p - b * hw);
    const int y = r / W, x = r - y * W;
    const int s = v.up;
    return (b * H * s + (int64_t)y * s) * ((int64_t)W * s) + (int64_t)x * s;
}

// x[b][2][H][W] (FP32 NCHW) -> BF16 NHWC [b][H][W][2]
__global__ void to_nhwc2_kernel(const float* __restrict__ x, int64_t P, int HW, bf16* __restrict__ y) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int64_t b = p / HW, r = p % HW;
    __nv_bfloat162 v;
    v.x = __float2bfloat16_rn(x[(b * 2) * HW + r]);
    v.y = __float2bfloat16_rn(x[(b * 2 + 1) * HW + r]);
    reinterpret_cast<__nv_bfloat162*>(y)[p] = v;
}

// Column matrix rows: cols[p][k] (row K9p), k = tap C + c (tap = ky ks +
// kx), zero for k >= ks^2 C and outside the image.  One thread per 8
// consecutive k of a row: one 16-byte load and store when C is a multiple of
// 8 (the 8 channels lie in one tap), else element by element.
__global__ void im2col_nhwc_kernel(const View X, int C, int B, int H, int W, int ks, int K9p,
                                   bf16* __restrict__ out) {
    const int kc_per_row = K9p / 8;
    const int64_t P = (int64_t)B * H * W;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * kc_per_row) return;
    const int64_t p = i / kc_per_row;
    const int k0 = (int)(i - p * kc_per_row) * 8;
    const int HW = H * W;
    const int b = (int)(p / HW), r = (int)(p % HW), y = r / W, x = r % W;
    const int K9 = ks * ks * C, half = ks / 2;
    __align__(16) bf16 v[8];
    if (C % 8 == 0 && X.up == 1) {
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if (k0 < K9) {
            const int tap = k0 / C, c = k0 - tap * C;
            const int ky = tap / ks, kx = tap - ky * ks;
            const int yy = y + ky - half, xx = x + kx - half;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                val = *reinterpret_cast<const uint4*>(X.p + (((int64_t)b * H + yy) * W + xx) * X.ld + X.off + c);
        }
        *reinterpret_cast<uint4*>(out + p * K9p + k0) = val;
        return;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = k0 + j;
        v[j] = __float2bfloat16_rn(0.0f);
        if (k < K9) {
            const int tap = k / C, c = k - tap * C;
            const int ky = tap / ks, kx = tap - ky * ks;
            const int yy = y + ky - half, xx = x + kx - half;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                const int s = X.up;
                const int64_t q = ((int64_t)b * H * s + (int64_t)yy * s) * ((int64_t)W * s) + (int64_t)xx * s;
                v[j] = X.p[q * X.ld + X.off + c];
            }
        }
    }
    *reinterpret_cast<uint4*>(out + p * K9p + k0) = *reinterpret_cast<const uint4*>(v);
}

// Transposed column matrix for the weight gradient: colsT[k][p] (row ldp),
// k = tap C + c, zero for p >= P.  A block takes 64 pixels and 32 channels:
// it loads the 9 taps' shifted 32-channel pixel rows (64-byte pieces along
// the NHWC rows) into shared memory as [tap][c][pixel] and writes the 288
// rows of 64 pixels with 16-byte stores.  C a multiple of 32, ks = 3.
constexpr int CT_PIX = 64, CT_PITCH = 72;

__global__ void __launch_bounds__(256) im2col_t_kernel(const View X, int C, int B, int H, int W, int ldp,
                                                       bf16* __restrict__ out) {
    __shared__ __align__(16) bf16 tile[9 * 32 * CT_PITCH];
    const int64_t P = (int64_t)B * H * W;
    const int64_t p0 = (int64_t)blockIdx.x * CT_PIX;
    const int c0 = blockIdx.y * 32;
    const int HW = H * W;
    // loads: 9 taps x 64 pixels x 4 chunks of 8 channels
    for (int idx = threadIdx.x; idx < 9 * CT_PIX * 4; idx += blockDim.x) {
        const int tap = idx / (CT_PIX * 4), rem = idx - tap * CT_PIX * 4;
        const int px = rem >> 2, ch = rem & 3;
        const int64_t p = p0 + px;
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if (p < P) {
            const int b = (int)(p / HW), r = (int)(p % HW), y = r / W, x = r % W;
            const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                val = *reinterpret_cast<const uint4*>(X.p + (((int64_t)b * H + yy) * W + xx) * X.ld + X.off + c0 +
                                                      ch * 8);
        }
        const bf16* e = reinterpret_cast<const bf16*>(&val);
#pragma unroll
        for (int j = 0; j < 8; ++j) tile[(tap * 32 + ch * 8 + j) * CT_PITCH + px] = e[j];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 9 * 32 * (CT_PIX / 8); idx += blockDim.x) {
        const int row = idx >> 3, seg = idx & 7;          // row = tap * 32 + c
        const int tap = row >> 5, c = row & 31;
        const int64_t k = (int64_t)tap * C + c0 + c;
        *reinterpret_cast<uint4*>(out + k * ldp + p0 + seg * 8) =
            *reinterpret_cast<const uint4*>(tile + row * CT_PITCH + seg * 8);
    }
}

// The same, element by element, for any C and kernel size; rows k >=
// ks^2 C are not written (they reach only product columns that are dropped).
__global__ void im2col_t_any_kernel(const View X, int C, int B, int H, int W, int ks, int ldp,
                                    bf16* __restrict__ out) {
    const int64_t P = (int64_t)B * H * W;
    const int K9 = ks * ks * C;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)K9 * ldp) return;
    const int k = (int)(i / ldp);
    const int64_t p = i - (int64_t)k * ldp;
    bf16 v = __float2bfloat16_rn(0.0f);
    if (p < P) {
        const int HW = H * W;
        const int b = (int)(p / HW), r = (int)(p - (int64_t)b * HW), y = r / W, x = r - y * W;
        const int tap = k / C, c = k - tap * C, half = ks / 2;
        const int yy = y + tap / ks - half, xx = x + tap % ks - half;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
            const int s = X.up;
            const int64_t q = ((int64_t)b * H * s + (int64_t)yy * s) * ((int64_t)W * s) + (int64_t)xx * s;
            v = X.p[q * X.ld + X.off + c];
        }
    }
    out[i] = v;
}

// A 3 x 3 convolution of an input with few channels (CI <= 4), computed
// directly: one thread per output pixel loads its 9 CI input values once and
// accumulates 16 output channels at a time in FP32 over k = tap CI + c in
// order, with the weights w[co][k] (row ldw) from shared memory transposed
// to [k][co] (16-byte loads of four channels).
template <int CI>
__global__ void __launch_bounds__(128) conv_small_kernel(const View X, int B, int H, int W,
                                                         const bf16* __restrict__ w, int ldw, int N,
                                                         const ConvEpi epi) {
    constexpr int K = 9 * CI;
    __shared__ __align__(16) float sw[K * 64];
    const int Np = (N + 15) / 16 * 16;
    for (int i = threadIdx.x; i < K * Np; i += blockDim.x) {
        const int k = i / Np, co = i - k * Np;
        sw[i] = co < N ? __bfloat162float(w[co * ldw + k]) : 0.0f;
    }
    __syncthreads();
    const int64_t P = (int64_t)B * H * W;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int HW = H * W;
    const int b = (int)(p / HW), r = (int)(p - (int64_t)b * HW), y = r / W, x = r - y * W;
    float xin[K];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
        const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
        const bf16* src = X.p + (((int64_t)b * H + yy) * W + xx) * X.ld + X.off;
#pragma unroll
        for (int c = 0; c < CI; ++c) xin[tap * CI + c] = in ? __bfloat162float(src[c]) : 0.0f;
    }
    for (int c0 = 0; c0 < N; c0 += 16) {
        float acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = 0.0f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float4* wk = reinterpret_cast<const float4*>(sw + k * Np + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 w4 = wk[q];
                acc[4 * q] += xin[k] * w4.x;
                acc[4 * q + 1] += xin[k] * w4.y;
                acc[4 * q + 2] += xin[k] * w4.z;
                acc[4 * q + 3] += xin[k] * w4.w;
            }
        }
        epi_store(epi, p, c0, min(16, N - c0), acc);
    }
}

// Epilogue of the column-matrix path: G[p][c] (row ldg) through epi, one
// thread per 16 columns of a pixel.
__global__ void bias_act_kernel(const float* __restrict__ G, int ldg, int64_t P, int N, const ConvEpi epi) {
    const int chunks = (N + 15) / 16;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * chunks) return;
    const int64_t p = i / chunks;
    const int c0 = (int)(i - p * chunks) * 16;
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = c0 + j < N ? G[p * ldg + c0 + j] : 0.0f;
    epi_store(epi, p, c0, min(16, N - c0), v);
}

// 2 x 2 average of an NHWC view on the grid H x W into a plain [B][H/2][W/2][C]
// tensor, one thread per 8 channels of an output pixel: (a + b) + (c + d) in
// FP32 (exact for BF16 inputs), times 1/4, rounded to BF16.
__global__ void pool_kernel(const View X, int C, int B, int H, int W, bf16* __restrict__ y) {
    const int h = H / 2, w = W / 2, cc = C / 8;
    const int64_t n = (int64_t)B * h * w * cc;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t q = i / cc;
    const int c = (int)(i - q * cc) * 8;
    const int64_t b = q / ((int64_t)h * w);
    const int r = (int)(q - b * h * w), yy = r / w, xx = r % w;
    const bf16* s = X.p + ((b * H + 2 * yy) * W + 2 * xx) * X.ld + X.off + c;
    const int64_t row = (int64_t)W * X.ld;
    const uint4 a4 = *reinterpret_cast<const uint4*>(s), b4 = *reinterpret_cast<const uint4*>(s + X.ld);
    const uint4 c4 = *reinterpret_cast<const uint4*>(s + row), d4 = *reinterpret_cast<const uint4*>(s + row + X.ld);
    const bf16 *pa = reinterpret_cast<const bf16*>(&a4), *pb = reinterpret_cast<const bf16*>(&b4);
    const bf16 *pc = reinterpret_cast<const bf16*>(&c4), *pd = reinterpret_cast<const bf16*>(&d4);
    __align__(16) bf16 o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        o[j] = __float2bfloat16_rn(0.25f * ((__bfloat162float(pa[j]) + __bfloat162float(pb[j])) +
                                            (__bfloat162float(pc[j]) + __bfloat162float(pd[j]))));
    *reinterpret_cast<uint4*>(y + q * C + c) = *reinterpret_cast<const uint4*>(o);
}

// Pixels per block of the activation backward: the block holds pt x Co
// values, at most 4096 for wide layers.
inline int act_tile(int co) { return co >= 256 ? 16 : (co >= 128 ? 32 : 64); }

// dZ = dY * (Y > 0) (or dY when relu == 0) for a block of pt pixels (a
// multiple of 16, at most 64) and all Co channels: BF16 NHWC dz16[p][c] (the
// data gradient's convolution input), BF16 channel-major dz_cp[c][p] (row
// ldp; the weight gradient's operand, zero for P <= p < ldp) through a
// shared-memory transpose, and the block's FP32 bias-gradient part
// part[block][c] (its pt pixels added in order).
__global__ void __launch_bounds__(256) act_back_kernel(const float* __restrict__ dy, const View Y, int H, int W,
                                                       int64_t P, int Co, int relu, int pt, bf16* __restrict__ dz16,
                                                       bf16* __restrict__ dz_cp, int ldp, float* __restrict__ part) {
    extern __shared__ __align__(16) uint8_t sm[];
    float* sf = reinterpret_cast<float*>(sm);                          // [pt][Co + 1]
    bf16* sb = reinterpret_cast<bf16*>(sm + (size_t)pt * (Co + 1) * 4); // [Co][pt + 8]
    const int sp = pt + 8;
    __shared__ int64_t ybase[64];
    const int64_t p0 = (int64_t)blockIdx.x * pt;
    if ((int)threadIdx.x < pt) {
        const int64_t p = p0 + threadIdx.x;
        ybase[threadIdx.x] = p < P ? view_pixel(Y, p, H, W) * Y.ld + Y.off : 0;
    }
    __syncthreads();
    const int n = pt * Co;
    for (int base = 0; base < n; base += 4 * 256) {
        float g[4], yv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = base + u * 256 + threadIdx.x;
            g[u] = 0.0f;
            yv[u] = 1.0f;
            if (i < n) {
                const int px = i / Co, c = i - px * Co;
                if (p0 + px < P) {
                    g[u] = dy[p0 * Co + i];
                    if (relu) yv[u] = __bfloat162float(Y.p[ybase[px] + c]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = base + u * 256 + threadIdx.x;
            if (i < n) {
                const int px = i / Co, c = i - px * Co;
                const float gg = (relu && !(yv[u] > 0.0f)) ? 0.0f : g[u];
                if (p0 + px < P) dz16[p0 * Co + i] = __float2bfloat16_rn(gg);
                sf[px * (Co + 1) + c] = gg;
                sb[c * sp + px] = __float2bfloat16_rn(gg);
            }
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < Co; c += blockDim.x) {
        float s = 0.0f;
        for (int px = 0; px < pt; ++px) s += sf[px * (Co + 1) + c];
        part[(int64_t)blockIdx.x * Co + c] = s;
    }
    const int segs = pt / 8;
    for (int i = threadIdx.x; i < Co * segs; i += blockDim.x) {
        const int c = i / segs, seg = i - c * segs;
        if (p0 + seg * 8 < ldp)
            *reinterpret_cast<uint4*>(dz_cp + (int64_t)c * ldp + p0 + seg * 8) =
                *reinterpret_cast<const uint4*>(sb + c * sp + seg * 8);
    }
}

// out[c] = the sum over k of part[k][c] in a fixed order: one block per
// channel, thread t adds parts t, t + 256, ... in turn, then a fixed tree
// over the threads.
__global__ void __launch_bounds__(256) parts_sum_kernel(const float* __restrict__ part, int n_part, int Co,
                                                        float* __restrict__ out) {
    __shared__ float red[256];
    const int c = blockIdx.x;
    float s = 0.0f;
    for (int k = threadIdx.x; k < n_part; k += 256) s += part[(int64_t)k * Co + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

// Gradient of the upsampled part of a decoder input: g[b][y][x][c] = the sum
// over the 2 x 2 block of dcat[b][2y + i][2x + j][c] (row pitch ldc; order
// (0,0), (0,1), (1,0), (1,1)), c < C, on the low grid h x w.  Four channels
// per thread (C and ldc multiples of 4).
__global__ void place_back_kernel(const float* __restrict__ dcat, int ldc, int B, int C, int h, int w,
                                  float* __restrict__ g) {
    const int c4 = C / 4;
    const int64_t n = (int64_t)B * h * w * c4;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t q = i / c4;
    const int c = (int)(i - q * c4) * 4;
    const int64_t b = q / ((int64_t)h * w);
    const int r = (int)(q - b * h * w), y = r / w, x = r - y * w;
    const int W = 2 * w;
    const float* d = dcat + ((b * 2 * h + 2 * y) * W + 2 * x) * ldc + c;
    const float4 a0 = *reinterpret_cast<const float4*>(d);
    const float4 a1 = *reinterpret_cast<const float4*>(d + ldc);
    const float4 a2 = *reinterpret_cast<const float4*>(d + (int64_t)W * ldc);
    const float4 a3 = *reinterpret_cast<const float4*>(d + (int64_t)W * ldc + ldc);
    float4 o;
    o.x = ((0.0f + a0.x) + a1.x + a2.x) + a3.x;
    o.y = ((0.0f + a0.y) + a1.y + a2.y) + a3.y;
    o.z = ((0.0f + a0.z) + a1.z + a2.z) + a3.z;
    o.w = ((0.0f + a0.w) + a1.w + a2.w) + a3.w;
    *reinterpret_cast<float4*>(g + q * C + c) = o;
}

// Gradient of an encoder output that feeds both a skip and a pool:
// g[b][y][x][c] = dcat[b][y][x][off + c] (row pitch ldc) + dp[b][y/2][x/2][c] / 4.
// Four channels per thread (C, ldc and off multiples of 4).
__global__ void pool_back_kernel(const float* __restrict__ dcat, int ldc, int off, const float* __restrict__ dp, int B,
                                 int C, int H, int W, float* __restrict__ g) {
    const int c4 = C / 4;
    const int64_t n = (int64_t)B * H * W * c4;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t q = i / c4;
    const int c = (int)(i - q * c4) * 4;
    const int64_t b = q / ((int64_t)H * W);
    const int r = (int)(q - b * H * W), y = r / W, x = r - y * W;
    const float4 s = *reinterpret_cast<const float4*>(dcat + q * ldc + off + c);
    const float4 d = *reinterpret_cast<const float4*>(dp + ((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c);
    *reinterpret_cast<float4*>(g + q * C + c) =
        make_float4(s.x + 0.25f * d.x, s.y + 0.25f * d.y, s.z + 0.25f * d.z, s.w + 0.25f * d.w);
}

// The 1 x 1 output layer with the residual: out[p] = (sum over c of w[c]
// d1[p][c] + bias) + x[b][0][y][x].
__global__ void head_kernel(const bf16* __restrict__ d1, int C, const bf16* __restrict__ w, const float* __restrict__ bias,
                            const float* __restrict__ x, int64_t P, int HW, float* __restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    float acc = 0.0f;
    for (int c = 0; c < C; ++c) acc += __bfloat162float(w[c]) * __bfloat162float(d1[p * C + c]);
    out[p] = (acc + bias[0]) + x[(p / HW) * 2 * HW + p % HW];
}

// Backward of the 1 x 1 layer for a block of 256 pixels: with g = dL/dout
// and gr = BF16(g), the input gradient gd1[p][c] = gr[p] w[c], and the
// block's parts of the weight gradient (sum of gr[p] d1[p][c]) and of the
// bias gradient (sum of g[p]), each added over the block's pixels in order.
__global__ void __launch_bounds__(256) head_back_kernel(const float* __restrict__ g, const bf16* __restrict__ d1, int C,
                                                        const bf16* __restrict__ w, int64_t P, float* __restrict__ gd1,
                                                        float* __restrict__ part_w, float* __restrict__ part_b) {
    __shared__ float sg[256], sgr[256];
    const int64_t p0 = (int64_t)blockIdx.x * 256;
    const int np = (int)min((int64_t)256, P - p0);
    const float gv = (int)threadIdx.x < np ? g[p0 + threadIdx.x] : 0.0f;
    sg[threadIdx.x] = gv;
    sgr[threadIdx.x] = __bfloat162float(__float2bfloat16_rn(gv));
    __syncthreads();
    for (int i = threadIdx.x; i < np * C; i += 256) {
        const int px = i / C, c = i - px * C;
        gd1[p0 * C + i] = sgr[px] * __bfloat162float(w[c]);
    }
    if ((int)threadIdx.x < C) {
        float s = 0.0f;
        for (int px = 0; px < np; ++px) s += sgr[px] * __bfloat162float(d1[(p0 + px) * C + threadIdx.x]);
        part_w[(int64_t)blockIdx.x * C + threadIdx.x] = s;
    }
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int px = 0; px < np; ++px) s += sg[px];
        part_b[blockIdx.x] = s;
    }
}

__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, int64_t n, float* __restrict__ dy,
                           double* __restrict__ loss) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.0f;
    if (i < n) {
        e = y[i] - t[i];
        dy[i] = 2.0f * e / (float)n;
    }
    float s = e * e;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0f) atomicAdd(loss, (double)s / (double)n);
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of a conv's weights w[co][ci][tap] (tap = ky ks + kx) in the
// products' K order: w16[co][tap Ci + ci] (row K9p) for the column path's
// forward, and wf16[ci][tap Co + co] = w[co][ci][kk - 1 - tap] (row K9dp),
// the weights with the taps flipped for the data gradient (a convolution of
// dZ: dX(y, x) = sum over co, ky, kx of dZ(y + ky - h, x + kx - h)
// w[co][ci][ks - 1 - ky][ks - 1 - kx]); zero beyond the K extent.  For 3 x 3
// layers also the implicit GEMM's ky-major copies w3[ky][co][kx Ci + ci] and
// wf3[ky][ci][kx Co + co] (flipped).
__global__ void weight_copies_kernel(const float* __restrict__ w, int Co, int Ci, int kk, int K9p, int K9dp,
                                     bf16* __restrict__ w16, bf16* __restrict__ wf16, bf16* __restrict__ w3,
                                     bf16* __restrict__ wf3) {
    const int K9 = Ci * kk;
    const int64_t n1 = (int64_t)Co * K9p, n2 = (int64_t)Ci * K9dp;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) {
        const int co = (int)(i / K9p), k = (int)(i % K9p);
        float v = 0.0f;
        if (k < K9) {
            const int tap = k / Ci, ci = k - tap * Ci;
            v = w[(int64_t)co * K9 + (int64_t)ci * kk + tap];
        }
        w16[i] = __float2bfloat16_rn(v);
    }
    if (i < n2) {
        const int ci = (int)(i / K9dp), k = (int)(i % K9dp);
        float v = 0.0f;
        if (k < Co * kk) {
            const int tap = k / Co, co = k - tap * Co;
            v = w[(int64_t)co * K9 + (int64_t)ci * kk + (kk - 1 - tap)];
        }
        wf16[i] = __float2bfloat16_rn(v);
    }
    if (w3 && i < (int64_t)Co * K9) {
        // w3[ky][co][kx Ci + ci] and wf3[ky][ci][kx Co + co], ky, kx < 3
        const int ky = (int)(i / ((int64_t)Co * 3 * Ci));
        const int r = (int)(i - (int64_t)ky * Co * 3 * Ci);
        const int co = r / (3 * Ci), q = r - co * 3 * Ci, kx = q / Ci, ci = q - kx * Ci;
        w3[i] = __float2bfloat16_rn(w[(int64_t)co * K9 + (int64_t)ci * kk + ky * 3 + kx]);
        const int ci2 = r / (3 * Co), q2 = r - ci2 * 3 * Co, kx2 = q2 / Co, co2 = q2 - kx2 * Co;
        wf3[i] = __float2bfloat16_rn(w[(int64_t)co2 * K9 + (int64_t)ci2 * kk + (8 - (ky * 3 + kx2))]);
    }
}

// dW[co][ci][tap] from the transposed weight-gradient product
// GT[tap Ci + ci][co] (row Co)
__global__ void unpad_kernel(const float* __restrict__ GT, int Co, int Ci, int kk, float* __restrict__ dw) {
    const int64_t n = (int64_t)Co * Ci * kk;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int co = (int)(i / ((int64_t)Ci * kk));
    const int r = (int)(i - (int64_t)co * Ci * kk), ci = r / kk, tap = r - ci * kk;
    dw[i] = GT[((int64_t)tap * Ci + ci) * Co + co];
}

// out[i] = sum over z of p[z * stride + i], in the order z = 0, 1, ...
__global__ void splits_sum_kernel(const float* __restrict__ p, int n_splits, int64_t stride, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= stride) return;
    float s = 0.0f;
    for (int z = 0; z < n_splits; ++z) s += p[(int64_t)z * stride + i];
    out[i] = s;
}

struct Conv {
    int ci, co, ks, H, W, relu;
    int K9, K9p, K9dp;     // ci ks^2, padded to 64; co ks^2 padded to 64 (data gradient)
    // parameters (FP32 master), gradients, Adam moments; offsets into the flat arrays
    int64_t w_off, b_off;
    bf16* w16 = nullptr;   // [co][K9p], K = (tap, ci)
    bf16* wf16 = nullptr;  // [ci][K9dp], K = (tap, co), taps flipped
    bf16* w3 = nullptr;    // 3 x 3 layers: [ky][co][kx ci + c], the implicit GEMM's weights
    bf16* wf3 = nullptr;   // 3 x 3 layers: [ky][ci][kx co + c], flipped
};

// K splits of a weight-gradient product over P pixels (a function of P alone,
// so the workspace for the largest batch bounds every call).
int wgrad_splits(int64_t P) {
    const int Pp = pad64(P);
    return std::max(1, std::min(Pp / 64, (int)(P / 4096) + 1));
}

}  // namespace
}  // namespace gdrr

using namespace gdrr;

struct gdrr_cnn {
    cudaStream_t stream = nullptr;
    int max_batch = 0, H = 0, W = 0, c = 0;
    std::vector<Conv> conv;
    int64_t n_params = 0;
    float* params = nullptr;   // FP32 master weights, flat
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int adam_t = 0;
    // activations (BF16 NHWC) of the last forward
    bf16 *x16 = nullptr, *cat1 = nullptr, *cat2 = nullptr, *cat3 = nullptr;
    bf16 *p1 = nullptr, *p2 = nullptr, *p3 = nullptr, *d1 = nullptr;
    float* out = nullptr;
    // gradients (FP32 NHWC)
    float *g_out = nullptr, *g_d1 = nullptr, *g_cat1 = nullptr, *g_d2 = nullptr, *g_cat2 = nullptr;
    float *g_d3 = nullptr, *g_cat3 = nullptr, *g_e4 = nullptr, *g_p3 = nullptr, *g_e3 = nullptr, *g_p2 = nullptr;
    float *g_e2 = nullptr, *g_p1 = nullptr, *g_e1 = nullptr;
    // workspaces
    bf16* cols = nullptr;      // column matrix, either layout
    float* gemm = nullptr;     // column-path GEMM output
    float* partials = nullptr; // per-split partial products of the weight gradients; bias-gradient parts
    bf16* dz16 = nullptr;      // dZ, NHWC
    bf16* dz_cp = nullptr;     // dZ, channel-major
    double* dloss = nullptr;
    int* err = nullptr;
    int last_batch = 0;
    std::vector<void*> allocs;
};

namespace {

template <typename T>
cudaError_t dalloc(gdrr_cnn* n, T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) n->allocs.push_back(*p);
    return e;
}

// splitmix64 + Box-Muller: a platform-independent normal generator for the
// initial weights.
struct InitRng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return sqrt(-2.0 * log(uniform())) * cos(6.283185307179586 * uniform()); }
};

int err_code(cudaError_t e) {
    if (e == cudaSuccess) return GDRR_OK;
    return e == cudaErrorMemoryAllocation ? GDRR_ERR_OOM : GDRR_ERR_CUDA;
}

#define CK(x)                                \
    do {                                     \
        cudaError_t _e = (x);                \
        if (_e != cudaSuccess) return _e;    \
    } while (0)

cudaError_t refresh_weights(gdrr_cnn* n) {
    for (Conv& L : n->conv) {
        const int64_t cnt = std::max({(int64_t)L.co * L.K9p, (int64_t)L.ci * L.K9dp, (int64_t)L.co * L.K9});
        weight_copies_kernel<<<nblk(cnt), TB, 0, n->stream>>>(n->params + L.w_off, L.co, L.ci, L.ks * L.ks, L.K9p,
                                                              L.K9dp, L.w16, L.wf16, L.w3, L.wf3);
        CK(cudaGetLastError());
    }
    return cudaSuccess;
}

ConvEpi epi_bf16(const float* bias, int relu, bf16* y, int ldy, int off, int up, int H, int W) {
    ConvEpi e;
    memset(&e, 0, sizeof e);
    e.bias = bias; e.relu = relu; e.y16 = y; e.ldy = ldy; e.off = off; e.up = up; e.H = H; e.W = W;
    return e;
}

ConvEpi epi_f32(float* y, int ld, int H, int W) {
    ConvEpi e;
    memset(&e, 0, sizeof e);
    e.yf = y; e.ldf = ld; e.up = 1; e.H = H; e.W = W;
    return e;
}

// One convolution on the grid H x W of the plain NHWC input X (C channels)
// into N output columns through epi: the implicit GEMM (ky-major weights w3)
// where the grid tiles, a direct kernel for inputs of at most 4 channels,
// else a column matrix (row K9p), the column-path GEMM with w (row ldw, K =
// (tap, c)) into n->gemm and the elementwise epilogue.
cudaError_t conv_product(gdrr_cnn* n, const View& X, int C, int B, int H, int W, int ks, const bf16* w, int ldw,
                         const bf16* w3, int N, const ConvEpi& epi) {
    const int64_t P = (int64_t)B * H * W;
    if (ks == 3 && w3 && X.up == 1 && conv_implicit_ok(C, H, W) && X.ld % 8 == 0 && X.off % 8 == 0) {
        ConvArgs a;
        a.x = X.p + X.off; a.C = C; a.ldx = X.ld;
        a.B = B; a.H = H; a.W = W;
        a.w3 = w3; a.N = N;
        a.epi = epi;
        return launch_conv_implicit(a, n->err, n->stream);
    }
    if (ks == 3 && C <= 4 && N <= 64) {
        const unsigned g = (unsigned)((P + 127) / 128);
        switch (C) {
            case 1: conv_small_kernel<1><<<g, 128, 0, n->stream>>>(X, B, H, W, w, ldw, N, epi); break;
            case 2: conv_small_kernel<2><<<g, 128, 0, n->stream>>>(X, B, H, W, w, ldw, N, epi); break;
            case 3: conv_small_kernel<3><<<g, 128, 0, n->stream>>>(X, B, H, W, w, ldw, N, epi); break;
            default: conv_small_kernel<4><<<g, 128, 0, n->stream>>>(X, B, H, W, w, ldw, N, epi); break;
        }
        return cudaGetLastError();
    }
    const int K9p = pad64((int64_t)ks * ks * C);
    im2col_nhwc_kernel<<<nblk(P * (K9p / 8)), TB, 0, n->stream>>>(X, C, B, H, W, ks, K9p, n->cols);
    CK(cudaGetLastError());
    if (epi.yf && !epi.bias && epi.ldf >= N && !epi.y16) {
        // FP32 output without bias: the GEMM writes it in place
        return launch_gemm_bf16(n->cols, K9p, w, ldw, epi.yf, epi.ldf, (int)P, N, K9p, 1, n->err, n->stream);
    }
    CK(launch_gemm_bf16(n->cols, K9p, w, ldw, n->gemm, N, (int)P, N, K9p, 1, n->err, n->stream));
    bias_act_kernel<<<nblk(P * ((N + 15) / 16)), TB, 0, n->stream>>>(n->gemm, N, P, N, epi);
    return cudaGetLastError();
}

// Backward of one 3 x 3 convolution L on the grid H x W: dy (FP32 [P][co],
// gradient of the layer output), Y (view of its BF16 output, for the ReLU
// mask), X (its plain NHWC input, ci channels).  Writes the parameter
// gradients and, when dx != NULL, dx (FP32 [P][ci]).
cudaError_t conv_backward(gdrr_cnn* n, const Conv& L, int B, const float* dy, const View& Y, const View& X,
                          float* dx) {
    const int64_t P = (int64_t)B * L.H * L.W;
    const int Pp = pad64(P);
    cudaStream_t st = n->stream;
    const int pt = act_tile(L.co);
    const int n_blk = (int)((P + pt - 1) / pt);
    const size_t smem = (size_t)pt * (L.co + 1) * 4 + (size_t)L.co * (pt + 8) * 2;
    CK(cudaFuncSetAttribute(act_back_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    act_back_kernel<<<n_blk, TB, smem, st>>>(dy, Y, L.H, L.W, P, L.co, L.relu, pt, n->dz16, n->dz_cp, Pp,
                                             n->partials);
    CK(cudaGetLastError());
    parts_sum_kernel<<<L.co, 256, 0, st>>>(n->partials, n_blk, L.co, n->grads + L.b_off);
    CK(cudaGetLastError());
    // weight gradient: dW[co][k] = sum_p dZ[p][co] cols[p][k]
    if (L.ci % 32 == 0 && L.ks == 3 && X.up == 1 && X.ld % 8 == 0 && X.off % 8 == 0) {
        im2col_t_kernel<<<dim3((unsigned)(Pp / CT_PIX), (unsigned)(L.ci / 32)), TB, 0, st>>>(X, L.ci, B, L.H, L.W, Pp,
                                                                                            n->cols);
    } else {
        im2col_t_any_kernel<<<nblk((int64_t)L.K9 * Pp), TB, 0, st>>>(X, L.ci, B, L.H, L.W, L.ks, Pp, n->cols);
    }
    CK(cudaGetLastError());
    // dW^T[k][co] = sum_p cols[p][k] dZ[p][co]: M runs over k (no tile
    // wasted on narrow layers), N over the output channels.  The pixel sum is
    // split across CTAs; each split writes its own partial product and one
    // ordered pass adds them, so training is bit-reproducible.
    const int splits = wgrad_splits(P);
    if (splits > 1) {
        const int64_t slice = (int64_t)L.co * L.K9p;
        int used = 1;
        CK(launch_gemm_bf16(n->cols, Pp, n->dz_cp, Pp, n->partials, L.co, L.K9p, L.co, Pp, splits, n->err, st, slice,
                            &used));
        splits_sum_kernel<<<nblk(slice), TB, 0, st>>>(n->partials, used, slice, n->gemm);
        CK(cudaGetLastError());
    } else {
        CK(launch_gemm_bf16(n->cols, Pp, n->dz_cp, Pp, n->gemm, L.co, L.K9p, L.co, Pp, 1, n->err, st));
    }
    unpad_kernel<<<nblk((int64_t)L.co * L.K9), TB, 0, st>>>(n->gemm, L.co, L.ci, L.ks * L.ks, n->grads + L.w_off);
    CK(cudaGetLastError());
    if (dx) {
        // data gradient: the convolution of dZ with the flipped weights
        CK(conv_product(n, plain(n->dz16, L.co), L.co, B, L.H, L.W, L.ks, L.wf16, L.K9dp, L.wf3, L.ci,
                        epi_f32(dx, L.ci, L.H, L.W)));
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

GDRR_API int gdrr_cnn_create(int32_t max_batch, int32_t height, int32_t width, int32_t base_channels, uint64_t seed,
                             void* cuda_stream, gdrr_cnn** out) {
    if (!out || max_batch <= 0 || height <= 0 || width <= 0 || height % 8 || width % 8 || base_channels <= 0 ||
        base_channels > 64 || base_channels % 8)
        return GDRR_ERR_INVALID_ARG;
    gdrr_cnn* n = new (std::nothrow) gdrr_cnn();
    if (!n) return GDRR_ERR_OOM;
    n->stream = (cudaStream_t)cuda_stream;
    n->max_batch = max_batch;
    n->H = height;
    n->W = width;
    n->c = base_channels;
    const int c = base_channels, H = height, W = width;
    struct Spec { int ci, co, ks, h, w, relu; };
    const Spec specs[] = {{2, c, 3, H, W, 1},           {c, 2 * c, 3, H / 2, W / 2, 1},
                          {2 * c, 4 * c, 3, H / 4, W / 4, 1}, {4 * c, 8 * c, 3, H / 8, W / 8, 1},
                          {12 * c, 4 * c, 3, H / 4, W / 4, 1}, {6 * c, 2 * c, 3, H / 2, W / 2, 1},
                          {3 * c, c, 3, H, W, 1},       {c, 1, 1, H, W, 0}};
    int64_t off = 0;
    for (const Spec& s : specs) {
        Conv L;
        L.ci = s.ci; L.co = s.co; L.ks = s.ks; L.H = s.h; L.W = s.w; L.relu = s.relu;
        L.K9 = s.ci * s.ks * s.ks;
        L.K9p = pad64(L.K9);
        L.K9dp = pad64((int64_t)s.co * s.ks * s.ks);
        L.w_off = off;
        off += (int64_t)L.co * L.K9;
        L.b_off = off;
        off += L.co;
        n->conv.push_back(L);
    }
    n->n_params = off;
    const int64_t B = max_batch, HW = (int64_t)H * W;
    int64_t max_cols = 0, max_gemm = 0, max_dz = 0, max_part = 0;
    for (const Conv& L : n->conv) {
        const int64_t P = B * L.H * L.W, Pp = pad64(P);
        max_cols = std::max({max_cols, Pp * L.K9p, P * L.K9dp});
        max_gemm = std::max({max_gemm, P * L.ci, (int64_t)L.co * L.K9p, P * L.co});
        max_dz = std::max({max_dz, P * L.co, (int64_t)L.co * Pp});
        max_part = std::max({max_part, (int64_t)wgrad_splits(P) * L.co * L.K9p, (Pp / act_tile(L.co) + 1) * L.co,
                             (Pp / 256 + 1) * (L.ci + 1)});
    }
    cudaError_t e = cudaSuccess;
    do {
        if ((e = dalloc(n, &n->params, off)) || (e = dalloc(n, &n->grads, off)) || (e = dalloc(n, &n->adam_m, off)) ||
            (e = dalloc(n, &n->adam_v, off)))
            break;
        bool bad = false;
        for (Conv& L : n->conv) {
            if (dalloc(n, &L.w16, (size_t)L.co * L.K9p) || dalloc(n, &L.wf16, (size_t)L.ci * L.K9dp)) bad = true;
            if (L.ks == 3 && (dalloc(n, &L.w3, (size_t)L.co * L.K9) || dalloc(n, &L.wf3, (size_t)L.co * L.K9))) bad = true;
        }
        if (bad) { e = cudaErrorMemoryAllocation; break; }
        const int64_t s1 = B * HW, s2 = s1 / 4, s3 = s1 / 16, s4 = s1 / 64;
        if ((e = dalloc(n, &n->x16, 2 * s1)) || (e = dalloc(n, &n->cat1, 3 * c * s1)) ||
            (e = dalloc(n, &n->p1, c * s2)) || (e = dalloc(n, &n->cat2, 6 * c * s2)) ||
            (e = dalloc(n, &n->p2, 2 * c * s3)) || (e = dalloc(n, &n->cat3, 12 * c * s3)) ||
            (e = dalloc(n, &n->p3, 4 * c * s4)) || (e = dalloc(n, &n->d1, c * s1)) || (e = dalloc(n, &n->out, s1)))
            break;
        if ((e = dalloc(n, &n->g_out, s1)) || (e = dalloc(n, &n->g_d1, c * s1)) ||
            (e = dalloc(n, &n->g_cat1, 3 * c * s1)) || (e = dalloc(n, &n->g_d2, 2 * c * s2)) ||
            (e = dalloc(n, &n->g_cat2, 6 * c * s2)) || (e = dalloc(n, &n->g_d3, 4 * c * s3)) ||
            (e = dalloc(n, &n->g_cat3, 12 * c * s3)) || (e = dalloc(n, &n->g_e4, 8 * c * s4)) ||
            (e = dalloc(n, &n->g_p3, 4 * c * s4)) || (e = dalloc(n, &n->g_e3, 4 * c * s3)) ||
            (e = dalloc(n, &n->g_p2, 2 * c * s3)) || (e = dalloc(n, &n->g_e2, 2 * c * s2)) ||
            (e = dalloc(n, &n->g_p1, c * s2)) || (e = dalloc(n, &n->g_e1, c * s1)))
            break;
        if ((e = dalloc(n, &n->cols, max_cols)) || (e = dalloc(n, &n->gemm, max_gemm)) ||
            (e = dalloc(n, &n->dz16, max_dz)) || (e = dalloc(n, &n->dz_cp, max_dz)) ||
            (e = dalloc(n, &n->partials, max_part)) || (e = dalloc(n, &n->dloss, 1)) || (e = dalloc(n, &n->err, 1)))
            break;
        // He-normal initial weights, zero biases
        std::vector<float> h(off, 0.0f);
        InitRng rng{seed};
        for (const Conv& L : n->conv) {
            const double sd = sqrt(2.0 / (double)L.K9);
            for (int64_t i = 0; i < (int64_t)L.co * L.K9; ++i) h[L.w_off + i] = (float)(sd * rng.normal());
        }
        if ((e = cudaMemcpy(n->params, h.data(), off * sizeof(float), cudaMemcpyHostToDevice))) break;
        if ((e = cudaMemset(n->adam_m, 0, off * sizeof(float))) || (e = cudaMemset(n->adam_v, 0, off * sizeof(float))) ||
            (e = cudaMemset(n->grads, 0, off * sizeof(float))) || (e = cudaMemset(n->err, 0, sizeof(int))))
            break;
        if ((e = refresh_weights(n))) break;
        e = cudaStreamSynchronize(n->stream);
    } while (0);
    if (e != cudaSuccess) {
        gdrr_cnn_destroy(n);
        return err_code(e);
    }
    *out = n;
    return GDRR_OK;
}

GDRR_API void gdrr_cnn_destroy(gdrr_cnn* n) {
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    for (void* p : n->allocs) cudaFree(p);
    delete n;
}

GDRR_API int gdrr_cnn_num_params(const gdrr_cnn* n, int64_t* count) {
    if (!n || !count) return GDRR_ERR_INVALID_ARG;
    *count = n->n_params;
    return GDRR_OK;
}

GDRR_API int gdrr_cnn_get_params(gdrr_cnn* n, float* host) {
    if (!n || !host) return GDRR_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(host, n->params, n->n_params * sizeof(float), cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return err_code(e);
}

GDRR_API int gdrr_cnn_set_params(gdrr_cnn* n, const float* host) {
    if (!n || !host) return GDRR_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(n->params, host, n->n_params * sizeof(float), cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = refresh_weights(n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    n->adam_t = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_m, 0, n->n_params * sizeof(float), n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_v, 0, n->n_params * sizeof(float), n->stream);
    return err_code(e);
}

GDRR_API int gdrr_cnn_get_grads(gdrr_cnn* n, float* host) {
    if (!n || !host) return GDRR_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(host, n->grads, n->n_params * sizeof(float), cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return err_code(e);
}

GDRR_API int gdrr_cnn_forward(gdrr_cnn* n, int32_t batch, const float* in_dev, float* out_dev) {
    if (!n || !in_dev || batch <= 0 || batch > n->max_batch) return GDRR_ERR_INVALID_ARG;
    const int B = batch, c = n->c, H = n->H, W = n->W;
    const int64_t s1 = (int64_t)B * H * W;
    cudaStream_t st = n->stream;
    const std::vector<Conv>& L = n->conv;
    cudaError_t e = cudaSuccess;
    n->last_batch = B;
    auto conv = [&](int i, const View& X, const ConvEpi& epi) {
        const Conv& l = L[i];
        return conv_product(n, X, l.ci, B, l.H, l.W, l.ks, l.w16, l.K9p, l.w3, l.co, epi);
    };
    auto pool = [&](const View& X, int C, int h, int w, bf16* y) {
        pool_kernel<<<nblk((int64_t)B * (h / 2) * (w / 2) * (C / 8)), TB, 0, st>>>(X, C, B, h, w, y);
        return cudaGetLastError();
    };
    const float* P = n->params;
    do {
        to_nhwc2_kernel<<<nblk(s1), TB, 0, st>>>(in_dev, s1, H * W, n->x16);
        if ((e = cudaGetLastError())) break;
        // encoder: e1 -> cat1[2c..3c), e2 -> cat2[4c..6c), e3 -> cat3[8c..12c), e4 -> cat3[0..8c) upsampled
        if ((e = conv(0, plain(n->x16, 2), epi_bf16(P + L[0].b_off, 1, n->cat1, 3 * c, 2 * c, 1, H, W)))) break;
        if ((e = pool(plain(n->cat1, 3 * c, 2 * c), c, H, W, n->p1))) break;
        if ((e = conv(1, plain(n->p1, c), epi_bf16(P + L[1].b_off, 1, n->cat2, 6 * c, 4 * c, 1, H / 2, W / 2)))) break;
        if ((e = pool(plain(n->cat2, 6 * c, 4 * c), 2 * c, H / 2, W / 2, n->p2))) break;
        if ((e = conv(2, plain(n->p2, 2 * c), epi_bf16(P + L[2].b_off, 1, n->cat3, 12 * c, 8 * c, 1, H / 4, W / 4))))
            break;
        if ((e = pool(plain(n->cat3, 12 * c, 8 * c), 4 * c, H / 4, W / 4, n->p3))) break;
        if ((e = conv(3, plain(n->p3, 4 * c), epi_bf16(P + L[3].b_off, 1, n->cat3, 12 * c, 0, 2, H / 8, W / 8))))
            break;
        // decoder: d3 -> cat2[0..4c) upsampled, d2 -> cat1[0..2c) upsampled, d1
        if ((e = conv(4, plain(n->cat3, 12 * c), epi_bf16(P + L[4].b_off, 1, n->cat2, 6 * c, 0, 2, H / 4, W / 4))))
            break;
        if ((e = conv(5, plain(n->cat2, 6 * c), epi_bf16(P + L[5].b_off, 1, n->cat1, 3 * c, 0, 2, H / 2, W / 2))))
            break;
        // d1 and the 1 x 1 output layer: fused into the implicit GEMM's
        // epilogue when d1's grid tiles, else a separate pass
        ConvEpi e6 = epi_bf16(P + L[6].b_off, 1, n->d1, c, 0, 1, H, W);
        const bool fuse_head = conv_implicit_ok(3 * c, H, W) && c <= 256;
        if (fuse_head) {
            e6.head_w = L[7].w16;
            e6.head_b = P + L[7].b_off;
            e6.head_x = in_dev;
            e6.head_out = n->out;
        }
        if ((e = conv(6, plain(n->cat1, 3 * c), e6))) break;
        if (!fuse_head) {
            head_kernel<<<nblk(s1), TB, 0, st>>>(n->d1, c, L[7].w16, P + L[7].b_off, in_dev, s1, H * W, n->out);
            if ((e = cudaGetLastError())) break;
        }
        if (out_dev) e = cudaMemcpyAsync(out_dev, n->out, s1 * sizeof(float), cudaMemcpyDeviceToDevice, st);
    } while (0);
    return err_code(e);
}

GDRR_API int gdrr_cnn_backward(gdrr_cnn* n, const float* target_dev, double* loss_out) {
    if (!n || !target_dev || n->last_batch <= 0) return GDRR_ERR_INVALID_ARG;
    const int B = n->last_batch, c = n->c, H = n->H, W = n->W;
    const int64_t s1 = (int64_t)B * H * W;
    cudaStream_t st = n->stream;
    const std::vector<Conv>& L = n->conv;
    cudaError_t e = cudaSuccess;
    double loss = 0.0;
    do {
        if ((e = cudaMemsetAsync(n->dloss, 0, sizeof(double), st))) break;
        mse_kernel<<<nblk(s1), TB, 0, st>>>(n->out, target_dev, s1, n->g_out, n->dloss);
        if ((e = cudaMemcpyAsync(&loss, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, st))) break;
        // the 1 x 1 output layer
        {
            const int nb = (int)((s1 + 255) / 256);
            float* pw = n->partials;
            float* pb = n->partials + (int64_t)nb * c;
            head_back_kernel<<<nb, 256, 0, st>>>(n->g_out, n->d1, c, L[7].w16, s1, n->g_d1, pw, pb);
            parts_sum_kernel<<<c, 256, 0, st>>>(pw, nb, c, n->grads + L[7].w_off);
            parts_sum_kernel<<<1, 256, 0, st>>>(pb, nb, 1, n->grads + L[7].b_off);
            if ((e = cudaGetLastError())) break;
        }
        // decoder: each input gradient g_cat splits into the upsampled part
        // (summed over 2 x 2 blocks) and the skip's part
        if ((e = conv_backward(n, L[6], B, n->g_d1, plain(n->d1, c), plain(n->cat1, 3 * c), n->g_cat1))) break;
        place_back_kernel<<<nblk(2 * c * s1 / 16), TB, 0, st>>>(n->g_cat1, 3 * c, B, 2 * c, H / 2, W / 2, n->g_d2);
        if ((e = conv_backward(n, L[5], B, n->g_d2, View{n->cat1, 3 * c, 0, 2}, plain(n->cat2, 6 * c), n->g_cat2)))
            break;
        place_back_kernel<<<nblk(4 * c * s1 / 64), TB, 0, st>>>(n->g_cat2, 6 * c, B, 4 * c, H / 4, W / 4, n->g_d3);
        if ((e = conv_backward(n, L[4], B, n->g_d3, View{n->cat2, 6 * c, 0, 2}, plain(n->cat3, 12 * c), n->g_cat3)))
            break;
        place_back_kernel<<<nblk(8 * c * s1 / 256), TB, 0, st>>>(n->g_cat3, 12 * c, B, 8 * c, H / 8, W / 8, n->g_e4);
        // encoder: an output's gradient is its skip's part plus its pool's
        if ((e = conv_backward(n, L[3], B, n->g_e4, View{n->cat3, 12 * c, 0, 2}, plain(n->p3, 4 * c), n->g_p3))) break;
        pool_back_kernel<<<nblk(4 * c * s1 / 64), TB, 0, st>>>(n->g_cat3, 12 * c, 8 * c, n->g_p3, B, 4 * c, H / 4,
                                                              W / 4, n->g_e3);
        if ((e = conv_backward(n, L[2], B, n->g_e3, plain(n->cat3, 12 * c, 8 * c), plain(n->p2, 2 * c), n->g_p2)))
            break;
        pool_back_kernel<<<nblk(2 * c * s1 / 16), TB, 0, st>>>(n->g_cat2, 6 * c, 4 * c, n->g_p2, B, 2 * c, H / 2, W / 2,
                                                             n->g_e2);
        if ((e = conv_backward(n, L[1], B, n->g_e2, plain(n->cat2, 6 * c, 4 * c), plain(n->p1, c), n->g_p1))) break;
        pool_back_kernel<<<nblk(c * s1 / 4), TB, 0, st>>>(n->g_cat1, 3 * c, 2 * c, n->g_p1, B, c, H, W, n->g_e1);
        if ((e = conv_backward(n, L[0], B, n->g_e1, plain(n->cat1, 3 * c, 2 * c), plain(n->x16, 2), nullptr))) break;
        int bad = 0;
        if ((e = cudaMemcpyAsync(&bad, n->err, sizeof(int), cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaStreamSynchronize(st))) break;
        if (bad) return GDRR_ERR_TIMEOUT;
    } while (0);
    if (e == cudaSuccess && loss_out) *loss_out = loss;
    return err_code(e);
}

GDRR_API int gdrr_cnn_adam_step(gdrr_cnn* n, float lr, float beta1, float beta2, float eps) {
    if (!n || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return GDRR_ERR_INVALID_ARG;
    n->adam_t += 1;
    const float c1 = 1.0f - powf(beta1, (float)n->adam_t), c2 = 1.0f - powf(beta2, (float)n->adam_t);
    adam_kernel<<<nblk(n->n_params), TB, 0, n->stream>>>(n->params, n->grads, n->adam_m, n->adam_v, n->n_params, lr,
                                                         beta1, beta2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = refresh_weights(n);
    return err_code(e);
}

}  // extern "C"
