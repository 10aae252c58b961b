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
// A 3x3 convolution is a GEMM over im2col columns:
//   forward   Y[P x Co]   = cols(x)[P x K9] . W[Co x K9]^T
//   data grad dX[P x Ci]  = cols(dZ)[P x K9d] . Wf[Ci x K9d]^T  (Wf: taps flipped)
//   weight    dW[Co x K9] = dZ^T[Co x P] . colsT(x)[K9 x P]^T   (split over P)
// with P = batch * H * W pixels, K9 = Ci * 9 and K9d = Co * 9 rounded up to
// 64.  The decoder's inputs [up(prev), skip] are read in place by the column
// builders (Src), not copied.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

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

__global__ void to_bf16_kernel(const float* __restrict__ x, int64_t n, bf16* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// The input of a convolution as the channel concatenation of two BF16
// tensors [a, s]: channel c < Ca reads a at resolution (H / up) x (W / up)
// (up = 2: nearest upsampling), channel c >= Ca reads s at H x W.  Element
// (b, c, y, x) of a tensor sits at base + b * batch_stride + c * chan_stride +
// y * width + x (NCHW: batch_stride = C H W, chan_stride = H W; the
// channel-major gradient rows [c][b H W] of the backward: batch_stride = H W,
// chan_stride = padded pixel count).  The decoder's concatenations and
// upsamplings are read in place instead of being copied.
struct Src {
    const bf16* a;
    int Ca, up;
    int64_t a_bs, a_cs;
    const bf16* s;
    int64_t s_bs, s_cs;
    int C, H, W;                        // total channels and the output resolution
};

// UP is the kernel's compile-time copy of S.up (1 or 2), so the upsampling
// index arithmetic is shifts.
template <int UP>
__device__ __forceinline__ bf16 src_at(const Src& S, int b, int c, int y, int x) {
    if (y < 0 || y >= S.H || x < 0 || x >= S.W) return __float2bfloat16_rn(0.0f);
    if (c < S.Ca) {
        const int wa = S.W / UP;
        return S.a[(int64_t)b * S.a_bs + (int64_t)c * S.a_cs + (int64_t)(y / UP) * wa + x / UP];
    }
    return S.s[(int64_t)b * S.s_bs + (int64_t)(c - S.Ca) * S.s_cs + (int64_t)y * S.W + x];
}

// cols[p][k] (row length K9p), p = (b, y, x), k = ci * ks * ks + ky * ks + kx,
// zero beyond C * ks * ks.  One block builds a tile of 32 pixels x 64 k:
// the reads go along pixels (coalesced on the input rows), the tile is
// transposed in shared memory, and each row segment of 64 k (128 bytes) is
// written with 16-byte stores.
constexpr int I2C_PIX = 32, I2C_K = 64;

template <int KS, int UP>
__global__ void __launch_bounds__(256) im2col_rows_kernel(const Src S, int B, int K9p, bf16* __restrict__ out) {
    __shared__ bf16 tile[I2C_K][I2C_PIX + 2];
    const int64_t P = (int64_t)B * S.H * S.W;
    const int64_t p0 = (int64_t)blockIdx.x * I2C_PIX;
    const int k0 = blockIdx.y * I2C_K;
    constexpr int kk = KS * KS, half = KS / 2;
    const int HW = S.H * S.W;
    {
        // the thread's 8 loads go out together, then land in the tile
        const int pl = threadIdx.x & (I2C_PIX - 1), w = threadIdx.x >> 5;
        const int64_t p = p0 + pl;
        const int b = (int)(p / HW), yx = (int)(p % HW), y = yx / S.W, x = yx % S.W;
        bf16 vals[I2C_K / 8];
#pragma unroll
        for (int j = 0; j < I2C_K / 8; ++j) {
            const int k = k0 + w + 8 * j;
            vals[j] = __float2bfloat16_rn(0.0f);
            if (p < P && k < S.C * kk) {
                const int ci = k / kk, r = k - ci * kk, ky = r / KS, kx = r - ky * KS;
                vals[j] = src_at<UP>(S, b, ci, y + ky - half, x + kx - half);
            }
        }
#pragma unroll
        for (int j = 0; j < I2C_K / 8; ++j) tile[w + 8 * j][pl] = vals[j];
    }
    __syncthreads();
    const int pix = threadIdx.x >> 3, chunk = threadIdx.x & 7;
    const int64_t p = p0 + pix;
    if (p < P) {
        __align__(16) bf16 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = tile[chunk * 8 + j][pix];
        *reinterpret_cast<uint4*>(out + p * K9p + k0 + chunk * 8) = *reinterpret_cast<const uint4*>(v);
    }
}

// 3x3 columns of a 32-pixel row segment, all k at once: warp w builds the 9
// taps of channels w, w + 8, ...; for each of the 3 source rows a lane loads
// its own pixel's value and the segment's two halo values come from lanes 0
// and 31, so the left and right taps are warp shuffles instead of loads.  The
// whole row segment [32][K9p] is assembled in shared memory (row pitch
// K9p + 8 elements) and written out with 16-byte stores.
template <int UP>
__global__ void __launch_bounds__(256) im2col_rows_shfl_kernel(const Src S, int K9p, bf16* __restrict__ out) {
    extern __shared__ __align__(16) bf16 seg[];
    const int pitch = K9p + 8;
    const int64_t p0 = (int64_t)blockIdx.x * 32;
    const int HW = S.H * S.W;
    const int b = (int)(p0 / HW), yx0 = (int)(p0 % HW), y = yx0 / S.W, x0 = yx0 % S.W;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = x0 + lane;
    const bf16 zero = __float2bfloat16_rn(0.0f);
    for (int ci = w; ci < S.C; ci += 8) {
        bf16 taps[9];
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const int yy = y + ky - 1;
            bf16 c = zero, edge = zero;
            if (yy >= 0 && yy < S.H) {
                const bf16* row;
                int up = 1;
                if (ci < S.Ca) {
                    row = S.a + (int64_t)b * S.a_bs + (int64_t)ci * S.a_cs + (int64_t)(yy / UP) * (S.W / UP);
                    up = UP;
                } else {
                    row = S.s + (int64_t)b * S.s_bs + (int64_t)(ci - S.Ca) * S.s_cs + (int64_t)yy * S.W;
                }
                c = row[up == 2 ? (x >> 1) : x];
                const int xe = lane == 0 ? x0 - 1 : x0 + 32;          // halo: lane 0 left, lane 31 right
                if ((lane == 0 || lane == 31) && xe >= 0 && xe < S.W) edge = row[up == 2 ? (xe >> 1) : xe];
            }
            bf16 left = __shfl_up_sync(0xffffffffu, c, 1);
            bf16 right = __shfl_down_sync(0xffffffffu, c, 1);
            if (lane == 0) left = edge;
            if (lane == 31) right = edge;
            taps[ky * 3 + 0] = left;
            taps[ky * 3 + 1] = c;
            taps[ky * 3 + 2] = right;
        }
        bf16* dst = seg + lane * pitch + ci * 9;
#pragma unroll
        for (int t = 0; t < 9; ++t) dst[t] = taps[t];
    }
    // zero the padded k columns of each row
    for (int i = threadIdx.x; i < 32 * (K9p - S.C * 9); i += blockDim.x) {
        const int r = i / (K9p - S.C * 9), k = S.C * 9 + i % (K9p - S.C * 9);
        seg[r * pitch + k] = zero;
    }
    __syncthreads();
    const int chunks = K9p / 8;
    for (int i = threadIdx.x; i < 32 * chunks; i += blockDim.x) {
        const int r = i / chunks, ck = i % chunks;
        *reinterpret_cast<uint4*>(out + (p0 + r) * K9p + ck * 8) =
            *reinterpret_cast<const uint4*>(seg + r * pitch + ck * 8);
    }
}

// colsT[k][p] (row length ldp >= P, padding pixels zero): each thread writes
// 8 consecutive pixels of one k (16 bytes).  Where the width is a multiple of
// 8 the 8 pixels share an image row and read consecutive input elements; the
// coarse levels of small images may wrap rows, so each pixel finds its own
// coordinates.
template <int KS, int UP>
__global__ void __launch_bounds__(256) im2col_cols_kernel(const Src S, int B, int K9p, int ldp,
                                                        bf16* __restrict__ out) {
    const int64_t P = (int64_t)B * S.H * S.W;
    const int64_t groups = ldp / 8;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= groups * K9p) return;
    const int k = (int)(i / groups);
    const int64_t p0 = (i - (int64_t)k * groups) * 8;
    constexpr int kk = KS * KS, half = KS / 2;
    const int HW = S.H * S.W;
    __align__(16) bf16 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __float2bfloat16_rn(0.0f);
    if (k < S.C * kk && p0 < P) {
        const int ci = k / kk, r = k - ci * kk, ky = r / KS, kx = r - ky * KS;
        int b = (int)(p0 / HW), yx = (int)(p0 % HW), y = yx / S.W, x = yx % S.W;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (p0 + j < P) v[j] = src_at<UP>(S, b, ci, y + ky - half, x + kx - half);
            if (++x == S.W) {                           // next pixel: wrap to the next row / image
                x = 0;
                if (++y == S.H) { y = 0; ++b; }
            }
        }
    }
    *reinterpret_cast<uint4*>(out + (int64_t)k * ldp + p0) = *reinterpret_cast<const uint4*>(v);
}

// Y[b][co][y][x] (BF16, channel offset in a wider tensor) = act(G[p][co] +
// bias[co]); also the FP32 value when yf != NULL (bias NULL: no bias, no
// activation).  A 32-pixel x 32-channel tile goes through shared memory, so
// both the reads of G's rows and the writes of the NCHW rows are coalesced.
__global__ void __launch_bounds__(256) bias_act_kernel(const float* __restrict__ G, int ldg,
                                                     const float* __restrict__ bias, int B, int Co, int HW, int relu,
                                                     bf16* __restrict__ y, int y_channels, float* __restrict__ yf) {
    __shared__ float t[32][33];
    const int64_t P = (int64_t)B * HW;
    const int64_t p0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32, lane = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < 32; r += 8) {
        const int64_t p = p0 + r;
        const int c = c0 + lane;
        float v = 0.0f;
        if (p < P && c < Co) {
            v = G[p * ldg + c];
            if (bias) v = v + bias[c];
            if (relu) v = fmaxf(v, 0.0f);
        }
        t[r][lane] = v;
    }
    __syncthreads();
    for (int r = threadIdx.x >> 5; r < 32; r += 8) {
        const int c = c0 + r;
        const int64_t p = p0 + lane;
        if (p < P && c < Co) {
            const int64_t b = p / HW, yx = p % HW;
            const float v = t[lane][r];
            if (y) y[(b * y_channels + c) * HW + yx] = __float2bfloat16_rn(v);
            if (yf) yf[(b * Co + c) * HW + yx] = v;
        }
    }
}

// dZ = dY * (Y > 0) (or dY when relu == 0), as BF16 channel-major rows
// dz_cp[co][p] (row length ldp; the weight gradient's operand and the data
// gradient's convolution input) and as FP32 NCHW (the bias gradient).
__global__ void act_back_kernel(const float* __restrict__ dy, const bf16* __restrict__ y, int y_channels, int B,
                                int Co, int H, int W, int relu, bf16* __restrict__ dz_cp, int ldp,
                                float* __restrict__ dz_f) {
    const int64_t n = (int64_t)B * Co * H * W;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % W);
    const int yy = (int)((i / W) % H);
    const int co = (int)((i / ((int64_t)W * H)) % Co);
    const int b = (int)(i / ((int64_t)W * H * Co));
    float g = dy[i];
    if (relu) {
        const float yv = __bfloat162float(y[(((int64_t)b * y_channels + co) * H + yy) * W + x]);
        if (!(yv > 0.0f)) g = 0.0f;
    }
    const int64_t p = ((int64_t)b * H + yy) * W + x;
    dz_cp[(int64_t)co * ldp + p] = __float2bfloat16_rn(g);
    dz_f[i] = g;
}

// db[co] = sum over pixels of dZ (FP32) in two ordered stages: block (co,
// s) reduces the s-th of n_part equal pixel ranges of channel co into
// part[co][s]; then one thread per channel adds its parts in order.  The
// partition and both orders are fixed, so the sum is bit-reproducible.
__global__ void bias_grad_part_kernel(const float* __restrict__ dz, int B, int Co, int HW, int n_part,
                                      float* __restrict__ part) {
    const int co = blockIdx.x, sp = blockIdx.y;
    const int64_t n = (int64_t)B * HW;
    const int64_t per = (n + n_part - 1) / n_part;
    const int64_t i0 = (int64_t)sp * per, i1 = min(n, i0 + per);
    float s = 0.0f;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int64_t b = i / HW, r = i % HW;
        s += dz[(b * Co + co) * HW + r];
    }
    __shared__ float red[TB];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)co * n_part + sp] = red[0];
}

__global__ void bias_grad_sum_kernel(const float* __restrict__ part, int Co, int n_part, float* __restrict__ db) {
    const int co = blockIdx.x * blockDim.x + threadIdx.x;
    if (co >= Co) return;
    float s = 0.0f;
    for (int k = 0; k < n_part; ++k) s += part[(int64_t)co * n_part + k];
    db[co] = s;
}

__global__ void pool_kernel(const bf16* __restrict__ x, int B, int C, int H, int W, bf16* __restrict__ y) {
    const int h = H / 2, w = W / 2;
    const int64_t n = (int64_t)B * C * h * w;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int xx = (int)(i % w), yy = (int)((i / w) % h);
    const int64_t bc = i / ((int64_t)w * h);
    const bf16* s = x + bc * H * W + (int64_t)(2 * yy) * W + 2 * xx;
    const float v = 0.25f * ((__bfloat162float(s[0]) + __bfloat162float(s[1])) +
                             (__bfloat162float(s[W]) + __bfloat162float(s[W + 1])));
    y[i] = __float2bfloat16_rn(v);
}

// dX += up(dY) / 4 (adjoint of the 2 x 2 average)
__global__ void pool_back_kernel(const float* __restrict__ dy, int B, int C, int H, int W, float* __restrict__ dx) {
    const int64_t n = (int64_t)B * C * H * W;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % W), y = (int)((i / W) % H);
    const int64_t bc = i / ((int64_t)W * H);
    dx[i] += 0.25f * dy[bc * (H / 2) * (W / 2) + (int64_t)(y / 2) * (W / 2) + x / 2];
}

// gradient of a channel range of a concatenated input: dsrc[b][c][y][x] (+)=
// the sum over the s x s block of dcat[b][off + c] (s = 2: nearest upsampling)
__global__ void place_back_kernel(const float* __restrict__ dcat, int cat_channels, int off, int B, int C, int h,
                                  int w, int s, int accumulate, float* __restrict__ dsrc) {
    const int64_t n = (int64_t)B * C * h * w;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % w), y = (int)((i / w) % h);
    const int c = (int)((i / ((int64_t)w * h)) % C);
    const int b = (int)(i / ((int64_t)w * h * C));
    const int H = h * s, W = w * s;
    const float* d = dcat + (((int64_t)b * cat_channels + off + c) * H + y * s) * W + x * s;
    float acc = 0.0f;
    for (int dy = 0; dy < s; ++dy)
        for (int dx = 0; dx < s; ++dx) acc += d[(int64_t)dy * W + dx];
    if (accumulate) dsrc[i] += acc; else dsrc[i] = acc;
}

// out[b][0][y][x] += in[b][0][y][x] (in has two channels)
__global__ void residual_kernel(const float* __restrict__ in, int B, int HW, float* __restrict__ out) {
    const int64_t n = (int64_t)B * HW;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += in[(i / HW) * 2 * HW + i % HW];
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

// BF16 copies of a conv's weights w[co][ci][tap] (tap = ky ks + kx):
// w16[co][k] (row K9p) for the forward, and wf16[ci][co kk + t] = w[co][ci][kk -
// 1 - t] (row K9dp), the weights with the taps flipped for the data gradient
// (a convolution of dZ: dX(y, x) = sum over co, ky, kx of dZ(y + ky - h,
// x + kx - h) w[co][ci][ks - 1 - ky][ks - 1 - kx]).
__global__ void weight_copies_kernel(const float* __restrict__ w, int Co, int Ci, int kk, int K9p, int K9dp,
                                     bf16* __restrict__ w16, bf16* __restrict__ wf16) {
    const int K9 = Ci * kk;
    const int64_t n1 = (int64_t)Co * K9p, n2 = (int64_t)Ci * K9dp;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) {
        const int co = (int)(i / K9p), k = (int)(i % K9p);
        w16[i] = __float2bfloat16_rn(k < K9 ? w[(int64_t)co * K9 + k] : 0.0f);
    }
    if (i < n2) {
        const int ci = (int)(i / K9dp), k = (int)(i % K9dp);
        float v = 0.0f;
        if (k < Co * kk) {
            const int co = k / kk, t = k % kk;
            v = w[(int64_t)co * K9 + (int64_t)ci * kk + (kk - 1 - t)];
        }
        wf16[i] = __float2bfloat16_rn(v);
    }
}

// dW[co][k] for k < K9 from the padded GEMM output (row K9p)
__global__ void unpad_kernel(const float* __restrict__ src, int rows, int cols, int ld, float* __restrict__ dst) {
    const int64_t n = (int64_t)rows * cols;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[(i / cols) * ld + i % cols];
}

// colsT for widths that are multiples of 8: a thread's 8 pixels are one row
// segment, read through one source row pointer.
template <int KS, int UP>
__global__ void __launch_bounds__(256) im2col_cols_w8_kernel(const Src S, int B, int K9p, int ldp,
                                                           bf16* __restrict__ out) {
    const int64_t P = (int64_t)B * S.H * S.W;
    const int64_t groups = ldp / 8;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= groups * K9p) return;
    const int k = (int)(i / groups);
    const int64_t p0 = (i - (int64_t)k * groups) * 8;
    constexpr int kk = KS * KS, half = KS / 2;
    const int HW = S.H * S.W;
    __align__(16) bf16 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __float2bfloat16_rn(0.0f);
    if (k < S.C * kk && p0 < P) {
        const int ci = k / kk, r = k - ci * kk, ky = r / KS, kx = r - ky * KS;
        const int b = (int)(p0 / HW), yx = (int)(p0 % HW), y = yx / S.W, x = yx % S.W;
        const int yy = y + ky - half;
        if (yy >= 0 && yy < S.H) {
            const bf16* row;
            if (ci < S.Ca) row = S.a + (int64_t)b * S.a_bs + (int64_t)ci * S.a_cs + (int64_t)(yy / UP) * (S.W / UP);
            else row = S.s + (int64_t)b * S.s_bs + (int64_t)(ci - S.Ca) * S.s_cs + (int64_t)yy * S.W;
            const int up = ci < S.Ca ? UP : 1;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int xx = x + j + kx - half;
                if (xx >= 0 && xx < S.W) v[j] = row[up == 2 ? (xx >> 1) : xx];
            }
        }
    }
    *reinterpret_cast<uint4*>(out + (int64_t)k * ldp + p0) = *reinterpret_cast<const uint4*>(v);
}

struct Conv {
    int ci, co, ks, H, W, relu;
    int K9, K9p, K9dp;     // ci ks^2, padded to 64; co ks^2 padded to 64 (data gradient)
    // parameters (FP32 master), gradients, Adam moments; offsets into the flat arrays
    int64_t w_off, b_off;
    bf16* w16 = nullptr;   // [co][K9p]
    bf16* wf16 = nullptr;  // [ci][K9dp], taps flipped
};

// K splits of a weight-gradient product over P pixels (a function of P alone,
// so the workspace for the largest batch bounds every call).
int wgrad_splits(int64_t P) {
    const int Pp = pad64(P);
    return std::max(1, std::min(Pp / 64, (int)(P / 4096) + 1));
}

// out[i] = sum over z of p[z * stride + i], in the order z = 0, 1, ...
__global__ void splits_sum_kernel(const float* __restrict__ p, int n_splits, int64_t stride, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= stride) return;
    float s = 0.0f;
    for (int z = 0; z < n_splits; ++z) s += p[(int64_t)z * stride + i];
    out[i] = s;
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
    // activations (BF16) for the last forward
    bf16 *x16 = nullptr, *e1 = nullptr, *e2 = nullptr, *e3 = nullptr, *e4 = nullptr;
    bf16 *p1 = nullptr, *p2 = nullptr, *p3 = nullptr;
    bf16 *d3 = nullptr, *d2 = nullptr, *d1 = nullptr;
    float* out = nullptr;
    // gradients of activations (FP32)
    float *g_out = nullptr, *g_d1 = nullptr, *g_c1 = nullptr, *g_d2 = nullptr, *g_c2 = nullptr, *g_d3 = nullptr;
    float *g_c3 = nullptr, *g_e4 = nullptr, *g_p3 = nullptr, *g_e3 = nullptr, *g_p2 = nullptr, *g_e2 = nullptr;
    float *g_p1 = nullptr, *g_e1 = nullptr, *g_x = nullptr;
    // workspaces
    bf16* cols = nullptr;      // im2col, either layout
    float* gemm = nullptr;     // GEMM output
    float* partials = nullptr; // per-split partial products of the weight gradients; bias-gradient parts
    bf16* dz_cp = nullptr;
    float* dz_f = nullptr;
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
        const int64_t cnt = std::max((int64_t)L.co * L.K9p, (int64_t)L.ci * L.K9dp);
        weight_copies_kernel<<<nblk(cnt), TB, 0, n->stream>>>(n->params + L.w_off, L.co, L.ci, L.ks * L.ks, L.K9p,
                                                              L.K9dp, L.w16, L.wf16);
        CK(cudaGetLastError());
    }
    return cudaSuccess;
}

// A tensor [B][C][H][W] (NCHW) as a convolution input.
Src nchw(const bf16* t, int C, int H, int W) {
    Src S;
    memset(&S, 0, sizeof S);
    S.up = 1;
    S.s = t;
    S.s_bs = (int64_t)C * H * W;
    S.s_cs = (int64_t)H * W;
    S.C = C; S.H = H; S.W = W;
    return S;
}

// [up(a), s]: a with Ca channels at H/2 x W/2, upsampled, then s (Cs channels).
Src concat_up(const bf16* a, int Ca, const bf16* s, int Cs, int H, int W) {
    Src S = nchw(s, Cs, H, W);
    S.a = a;
    S.Ca = Ca;
    S.up = 2;
    S.a_bs = (int64_t)Ca * (H / 2) * (W / 2);
    S.a_cs = (int64_t)(H / 2) * (W / 2);
    S.C = Ca + Cs;
    return S;
}

// Channel-major rows t[c][p] (row length ldp, p = b H W + y W + x) as a
// convolution input.
Src chan_major(const bf16* t, int C, int H, int W, int64_t ldp) {
    Src S = nchw(t, C, H, W);
    S.s_bs = (int64_t)H * W;
    S.s_cs = ldp;
    return S;
}

cudaError_t im2col_rows(gdrr_cnn* n, const Src& X, int B, int ks, int K9p) {
    const int64_t P = (int64_t)B * X.H * X.W;
    const dim3 grid((unsigned)((P + I2C_PIX - 1) / I2C_PIX), (unsigned)(K9p / I2C_K));
    const size_t seg_bytes = (size_t)32 * (K9p + 8) * sizeof(bf16);
    if (X.W % 32 == 0 && ks == 3 && seg_bytes <= 200 * 1024) {
        const unsigned blocks = (unsigned)(P / 32);
        if (X.up == 2) {
            CK(cudaFuncSetAttribute(im2col_rows_shfl_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)seg_bytes));
            im2col_rows_shfl_kernel<2><<<blocks, 256, seg_bytes, n->stream>>>(X, K9p, n->cols);
        } else {
            CK(cudaFuncSetAttribute(im2col_rows_shfl_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)seg_bytes));
            im2col_rows_shfl_kernel<1><<<blocks, 256, seg_bytes, n->stream>>>(X, K9p, n->cols);
        }
    } else if (ks == 1) {
        im2col_rows_kernel<1, 1><<<grid, 256, 0, n->stream>>>(X, B, K9p, n->cols);
    } else if (X.up == 2) {
        im2col_rows_kernel<3, 2><<<grid, 256, 0, n->stream>>>(X, B, K9p, n->cols);
    } else {
        im2col_rows_kernel<3, 1><<<grid, 256, 0, n->stream>>>(X, B, K9p, n->cols);
    }
    return cudaGetLastError();
}

cudaError_t im2col_cols(gdrr_cnn* n, const Src& X, int B, int ks, int K9p, int ldp) {
    const int blocks = nblk((int64_t)(ldp / 8) * K9p);
    if (X.W % 8 == 0 && ks == 3) {
        if (X.up == 2) im2col_cols_w8_kernel<3, 2><<<blocks, TB, 0, n->stream>>>(X, B, K9p, ldp, n->cols);
        else im2col_cols_w8_kernel<3, 1><<<blocks, TB, 0, n->stream>>>(X, B, K9p, ldp, n->cols);
        return cudaGetLastError();
    }
    if (ks == 1) im2col_cols_kernel<1, 1><<<blocks, TB, 0, n->stream>>>(X, B, K9p, ldp, n->cols);
    else if (X.up == 2) im2col_cols_kernel<3, 2><<<blocks, TB, 0, n->stream>>>(X, B, K9p, ldp, n->cols);
    else im2col_cols_kernel<3, 1><<<blocks, TB, 0, n->stream>>>(X, B, K9p, ldp, n->cols);
    return cudaGetLastError();
}

// Y = act(conv(X) + bias): BF16 y (channel count y_channels, written at
// channels 0 .. co-1) and/or FP32 yf.
cudaError_t conv_forward(gdrr_cnn* n, const Conv& L, int B, const Src& X, bf16* y, int y_channels, float* yf) {
    const int64_t P = (int64_t)B * L.H * L.W;
    CK(im2col_rows(n, X, B, L.ks, L.K9p));
    CK(launch_gemm_bf16(n->cols, L.K9p, L.w16, L.K9p, n->gemm, L.co, (int)P, L.co, L.K9p, 1, n->err, n->stream));
    const dim3 grid((unsigned)((P + 31) / 32), (unsigned)((L.co + 31) / 32));
    bias_act_kernel<<<grid, 256, 0, n->stream>>>(n->gemm, L.co, n->params + L.b_off, B, L.co, L.H * L.W, L.relu, y,
                                                 y_channels, yf);
    return cudaGetLastError();
}

int bias_parts(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, (n + 8191) / 8192)); }

// Backward of one convolution: dy (FP32 [B][co][H][W], gradient of the
// layer output), y (its BF16 output, for the ReLU mask), X (its input).
// Writes the parameter gradients and, when dx != NULL, dx (FP32 NCHW input
// gradient).
cudaError_t conv_backward(gdrr_cnn* n, const Conv& L, int B, const float* dy, const bf16* y, int y_channels,
                          const Src& X, float* dx) {
    const int64_t P = (int64_t)B * L.H * L.W;
    const int Pp = pad64(P);
    const int HW = L.H * L.W;
    CK(cudaMemsetAsync(n->dz_cp, 0, (size_t)L.co * Pp * sizeof(bf16), n->stream));
    act_back_kernel<<<nblk(P * L.co), TB, 0, n->stream>>>(dy, y, y_channels, B, L.co, L.H, L.W, L.relu, n->dz_cp, Pp,
                                                          n->dz_f);
    CK(cudaGetLastError());
    const int parts = bias_parts(P);
    bias_grad_part_kernel<<<dim3((unsigned)L.co, (unsigned)parts), TB, 0, n->stream>>>(n->dz_f, B, L.co, HW, parts,
                                                                                       n->partials);
    bias_grad_sum_kernel<<<(L.co + 127) / 128, 128, 0, n->stream>>>(n->partials, L.co, parts, n->grads + L.b_off);
    CK(cudaGetLastError());
    // weight gradient: dW[co][k] = sum_p dZ[p][co] cols[p][k]
    CK(im2col_cols(n, X, B, L.ks, L.K9p, Pp));
    // the pixel sum is split across CTAs; each split writes its own partial
    // product and one ordered pass adds them, so training is bit-reproducible
    const int splits = wgrad_splits(P);
    if (splits > 1) {
        const int64_t slice = (int64_t)L.co * L.K9p;
        int used = 1;
        CK(launch_gemm_bf16(n->dz_cp, Pp, n->cols, Pp, n->partials, L.K9p, L.co, L.K9p, Pp, splits, n->err, n->stream,
                            slice, &used));
        splits_sum_kernel<<<nblk(slice), TB, 0, n->stream>>>(n->partials, used, slice, n->gemm);
        CK(cudaGetLastError());
    } else {
        CK(launch_gemm_bf16(n->dz_cp, Pp, n->cols, Pp, n->gemm, L.K9p, L.co, L.K9p, Pp, 1, n->err, n->stream));
    }
    unpad_kernel<<<nblk((int64_t)L.co * L.K9), TB, 0, n->stream>>>(n->gemm, L.co, L.K9, L.K9p, n->grads + L.w_off);
    CK(cudaGetLastError());
    if (dx) {
        // data gradient: the convolution of dZ with the flipped weights,
        // dX[p][ci] = sum_k cols(dZ)[p][k] Wf[ci][k], then to NCHW
        CK(im2col_rows(n, chan_major(n->dz_cp, L.co, L.H, L.W, Pp), B, L.ks, L.K9dp));
        CK(launch_gemm_bf16(n->cols, L.K9dp, L.wf16, L.K9dp, n->gemm, L.ci, (int)P, L.ci, L.K9dp, 1, n->err,
                            n->stream));
        const dim3 grid((unsigned)((P + 31) / 32), (unsigned)((L.ci + 31) / 32));
        bias_act_kernel<<<grid, 256, 0, n->stream>>>(n->gemm, L.ci, nullptr, B, L.ci, HW, 0, nullptr, 0, dx);
        CK(cudaGetLastError());
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

GDRR_API int gdrr_cnn_create(int32_t max_batch, int32_t height, int32_t width, int32_t base_channels, uint64_t seed,
                             void* cuda_stream, gdrr_cnn** out) {
    if (!out || max_batch <= 0 || height <= 0 || width <= 0 || height % 8 || width % 8 || base_channels <= 0 ||
        base_channels > 64)
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
        max_part = std::max({max_part, (int64_t)wgrad_splits(P) * L.co * L.K9p, (int64_t)L.co * bias_parts(P)});
    }
    cudaError_t e = cudaSuccess;
    do {
        if ((e = dalloc(n, &n->params, off)) || (e = dalloc(n, &n->grads, off)) || (e = dalloc(n, &n->adam_m, off)) ||
            (e = dalloc(n, &n->adam_v, off)))
            break;
        bool bad = false;
        for (Conv& L : n->conv) {
            if (dalloc(n, &L.w16, (size_t)L.co * L.K9p) || dalloc(n, &L.wf16, (size_t)L.ci * L.K9dp)) bad = true;
        }
        if (bad) { e = cudaErrorMemoryAllocation; break; }
        const int64_t s1 = B * HW, s2 = s1 / 4, s3 = s1 / 16, s4 = s1 / 64;
        if ((e = dalloc(n, &n->x16, 2 * s1)) || (e = dalloc(n, &n->e1, c * s1)) || (e = dalloc(n, &n->p1, c * s2)) ||
            (e = dalloc(n, &n->e2, 2 * c * s2)) || (e = dalloc(n, &n->p2, 2 * c * s3)) ||
            (e = dalloc(n, &n->e3, 4 * c * s3)) || (e = dalloc(n, &n->p3, 4 * c * s4)) ||
            (e = dalloc(n, &n->e4, 8 * c * s4)) || (e = dalloc(n, &n->d3, 4 * c * s3)) ||
            (e = dalloc(n, &n->d2, 2 * c * s2)) || (e = dalloc(n, &n->d1, c * s1)) || (e = dalloc(n, &n->out, s1)))
            break;
        if ((e = dalloc(n, &n->g_out, s1)) || (e = dalloc(n, &n->g_d1, c * s1)) || (e = dalloc(n, &n->g_c1, 3 * c * s1)) ||
            (e = dalloc(n, &n->g_d2, 2 * c * s2)) || (e = dalloc(n, &n->g_c2, 6 * c * s2)) ||
            (e = dalloc(n, &n->g_d3, 4 * c * s3)) || (e = dalloc(n, &n->g_c3, 12 * c * s3)) ||
            (e = dalloc(n, &n->g_e4, 8 * c * s4)) || (e = dalloc(n, &n->g_p3, 4 * c * s4)) ||
            (e = dalloc(n, &n->g_e3, 4 * c * s3)) || (e = dalloc(n, &n->g_p2, 2 * c * s3)) ||
            (e = dalloc(n, &n->g_e2, 2 * c * s2)) || (e = dalloc(n, &n->g_p1, c * s2)) ||
            (e = dalloc(n, &n->g_e1, c * s1)) || (e = dalloc(n, &n->g_x, 2 * s1)))
            break;
        if ((e = dalloc(n, &n->cols, max_cols)) || (e = dalloc(n, &n->gemm, max_gemm)) ||
            (e = dalloc(n, &n->dz_cp, max_dz)) ||
            (e = dalloc(n, &n->dz_f, max_dz)) || (e = dalloc(n, &n->partials, max_part)) ||
            (e = dalloc(n, &n->err, 1)))
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
    cudaError_t e = cudaSuccess;
    n->last_batch = B;
    do {
        to_bf16_kernel<<<nblk(2 * s1), TB, 0, st>>>(in_dev, 2 * s1, n->x16);
        if ((e = cudaGetLastError())) break;
        const std::vector<Conv>& L = n->conv;
        if ((e = conv_forward(n, L[0], B, nchw(n->x16, 2, H, W), n->e1, c, nullptr))) break;
        pool_kernel<<<nblk(c * s1 / 4), TB, 0, st>>>(n->e1, B, c, H, W, n->p1);
        if ((e = conv_forward(n, L[1], B, nchw(n->p1, c, H / 2, W / 2), n->e2, 2 * c, nullptr))) break;
        pool_kernel<<<nblk(2 * c * s1 / 16), TB, 0, st>>>(n->e2, B, 2 * c, H / 2, W / 2, n->p2);
        if ((e = conv_forward(n, L[2], B, nchw(n->p2, 2 * c, H / 4, W / 4), n->e3, 4 * c, nullptr))) break;
        pool_kernel<<<nblk(4 * c * s1 / 64), TB, 0, st>>>(n->e3, B, 4 * c, H / 4, W / 4, n->p3);
        if ((e = conv_forward(n, L[3], B, nchw(n->p3, 4 * c, H / 8, W / 8), n->e4, 8 * c, nullptr))) break;
        // decoder: [up(prev), skip], read in place
        if ((e = conv_forward(n, L[4], B, concat_up(n->e4, 8 * c, n->e3, 4 * c, H / 4, W / 4), n->d3, 4 * c,
                              nullptr)))
            break;
        if ((e = conv_forward(n, L[5], B, concat_up(n->d3, 4 * c, n->e2, 2 * c, H / 2, W / 2), n->d2, 2 * c,
                              nullptr)))
            break;
        if ((e = conv_forward(n, L[6], B, concat_up(n->d2, 2 * c, n->e1, c, H, W), n->d1, c, nullptr))) break;
        if ((e = conv_forward(n, L[7], B, nchw(n->d1, c, H, W), nullptr, 1, n->out))) break;
        residual_kernel<<<nblk(s1), TB, 0, st>>>(in_dev, B, H * W, n->out);
        if ((e = cudaGetLastError())) break;
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
    double* dloss = reinterpret_cast<double*>(n->dz_f);   // scratch for the loss sum before dz_f is used
    cudaError_t e = cudaSuccess;
    double loss = 0.0;
    do {
        if ((e = cudaMemsetAsync(dloss, 0, sizeof(double), st))) break;
        mse_kernel<<<nblk(s1), TB, 0, st>>>(n->out, target_dev, s1, n->g_out, dloss);
        if ((e = cudaMemcpyAsync(&loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaStreamSynchronize(st))) break;
        if ((e = conv_backward(n, L[7], B, n->g_out, nullptr, 1, nchw(n->d1, c, H, W), n->g_d1))) break;
        if ((e = conv_backward(n, L[6], B, n->g_d1, n->d1, c, concat_up(n->d2, 2 * c, n->e1, c, H, W), n->g_c1)))
            break;
        // c1 = [up(d2), e1]
        place_back_kernel<<<nblk(2 * c * s1 / 4), TB, 0, st>>>(n->g_c1, 3 * c, 0, B, 2 * c, H / 2, W / 2, 2, 0, n->g_d2);
        place_back_kernel<<<nblk(c * s1), TB, 0, st>>>(n->g_c1, 3 * c, 2 * c, B, c, H, W, 1, 0, n->g_e1);
        if ((e = conv_backward(n, L[5], B, n->g_d2, n->d2, 2 * c, concat_up(n->d3, 4 * c, n->e2, 2 * c, H / 2, W / 2),
                               n->g_c2)))
            break;
        place_back_kernel<<<nblk(4 * c * s1 / 16), TB, 0, st>>>(n->g_c2, 6 * c, 0, B, 4 * c, H / 4, W / 4, 2, 0, n->g_d3);
        place_back_kernel<<<nblk(2 * c * s1 / 4), TB, 0, st>>>(n->g_c2, 6 * c, 4 * c, B, 2 * c, H / 2, W / 2, 1, 0,
                                                              n->g_e2);
        if ((e = conv_backward(n, L[4], B, n->g_d3, n->d3, 4 * c, concat_up(n->e4, 8 * c, n->e3, 4 * c, H / 4, W / 4),
                               n->g_c3)))
            break;
        place_back_kernel<<<nblk(8 * c * s1 / 64), TB, 0, st>>>(n->g_c3, 12 * c, 0, B, 8 * c, H / 8, W / 8, 2, 0,
                                                               n->g_e4);
        place_back_kernel<<<nblk(4 * c * s1 / 16), TB, 0, st>>>(n->g_c3, 12 * c, 8 * c, B, 4 * c, H / 4, W / 4, 1, 0,
                                                               n->g_e3);
        // encoder
        if ((e = conv_backward(n, L[3], B, n->g_e4, n->e4, 8 * c, nchw(n->p3, 4 * c, H / 8, W / 8), n->g_p3))) break;
        pool_back_kernel<<<nblk(4 * c * s1 / 16), TB, 0, st>>>(n->g_p3, B, 4 * c, H / 4, W / 4, n->g_e3);
        if ((e = conv_backward(n, L[2], B, n->g_e3, n->e3, 4 * c, nchw(n->p2, 2 * c, H / 4, W / 4), n->g_p2))) break;
        pool_back_kernel<<<nblk(2 * c * s1 / 4), TB, 0, st>>>(n->g_p2, B, 2 * c, H / 2, W / 2, n->g_e2);
        if ((e = conv_backward(n, L[1], B, n->g_e2, n->e2, 2 * c, nchw(n->p1, c, H / 2, W / 2), n->g_p1))) break;
        pool_back_kernel<<<nblk(c * s1), TB, 0, st>>>(n->g_p1, B, c, H, W, n->g_e1);
        if ((e = conv_backward(n, L[0], B, n->g_e1, n->e1, c, nchw(n->x16, 2, H, W), nullptr))) break;
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
