// Convolution outputs of the learned estimator, shared by the tcgen05
// kernels' epilogues and the elementwise epilogue of the column-matrix path.
//
// Activations are NHWC BF16: element (b, y, x, c) of a tensor with pixel
// pitch ld sits at base + ((b H + y) W + x) ld + c.  The decoder's inputs
// [up(prev), skip] are single NHWC buffers: the skip's producer writes its
// channel range in place and the previous decoder level's producer writes its
// output there upsampled (each pixel to its 2 x 2 block), so a decoder
// convolution reads one plain tensor.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace gdrr {

// Where a convolution's accumulator goes.  Pixel p = (b H + y) W + x of the
// output grid (H x W) and column c (output channel):
//   y16 != NULL: BF16 act(acc + bias[c]) at pixel pitch ldy, channel off + c;
//                up == 2 writes the value to the four pixels (2y + i, 2x + j)
//                of a 2H x 2W grid (nearest upsampling);
//   yf  != NULL: FP32 acc (+ bias when given) at yf[p ldf + c].
// head_out != NULL (BF16 output, one column tile holding every column): a
// 1 x 1 convolution to one channel follows, fused: head_out[p] = (sum over c
// in order of head_w[c] y16[p][c] + head_b[0]) + head_x[b][0][y][x] (head_x
// FP32 [b][2][H][W]).
struct ConvEpi {
    const float* bias;          // NULL: no bias
    int relu;
    __nv_bfloat16* y16;
    int ldy, off, up;
    float* yf;
    int ldf;
    int H, W;                   // output grid of the convolution
    const __nv_bfloat16* head_w;
    const float* head_b;
    const float* head_x;
    float* head_out;
};

// Stores columns [c0, c0 + n) (n <= 16) of pixel p from v[0 .. n).  The
// 16-column BF16 store is two 16-byte stores when the address allows it.
// With head != NULL, adds head_w[c] times the stored BF16 value of each
// column c to *head, in column order.
__device__ __forceinline__ void epi_store(const ConvEpi& e, int64_t p, int c0, int n, const float* v,
                                          float* head = nullptr) {
    if (e.y16) {
        __align__(16) __nv_bfloat16 o[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float a = v[j];
            if (j < n) {
                if (e.bias) a = a + e.bias[c0 + j];
                if (e.relu) a = fmaxf(a, 0.0f);
            }
            o[j] = __float2bfloat16_rn(a);
        }
        if (head) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j < n) *head += __bfloat162float(e.head_w[c0 + j]) * __bfloat162float(o[j]);
        }
        const int64_t hw = (int64_t)e.H * e.W;
        const int64_t b = p / hw;
        const int r = (int)(p - b * hw);
        const int yy = r / e.W, xx = r - yy * e.W;
        const int s = e.up;
        for (int i = 0; i < s; ++i)
            for (int j = 0; j < s; ++j) {
                const int64_t q = (b * e.H * s + (int64_t)(yy * s + i)) * ((int64_t)e.W * s) + xx * s + j;
                __nv_bfloat16* d = e.y16 + q * e.ldy + e.off + c0;
                if (n == 16 && (reinterpret_cast<uintptr_t>(d) & 15u) == 0) {
                    reinterpret_cast<uint4*>(d)[0] = reinterpret_cast<const uint4*>(o)[0];
                    reinterpret_cast<uint4*>(d)[1] = reinterpret_cast<const uint4*>(o)[1];
                } else {
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (k < n) d[k] = o[k];
                }
            }
    }
    if (e.yf) {
        float* d = e.yf + p * e.ldf + c0;
        if (n == 16 && !e.bias && (reinterpret_cast<uintptr_t>(d) & 15u) == 0) {
#pragma unroll
            for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4*>(d + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < n) d[k] = e.bias ? v[k] + e.bias[c0 + k] : v[k];
        }
    }
}

// The fused 1 x 1 head of pixel p once every column has been added to acc.
__device__ __forceinline__ void epi_head(const ConvEpi& e, int64_t p, float acc) {
    const int64_t hw = (int64_t)e.H * e.W;
    const int64_t b = p / hw;
    e.head_out[p] = (acc + e.head_b[0]) + e.head_x[b * 2 * hw + (p - b * hw)];
}

// A 3 x 3 convolution with zero padding over an NHWC BF16 tensor x (C
// channels read, pixel pitch ldx; batch B, grid H x W, output on the same
// grid) into N output columns through epi, with the weights stored ky-major:
// w3[ky][n][kx C + c] for tap (ky, kx).
struct ConvArgs {
    const __nv_bfloat16* x;
    int C, ldx;
    int B, H, W;
    const __nv_bfloat16* w3;
    int N;
    ConvEpi epi;
};

// The implicit-GEMM form applies when C is a multiple of 32 and a tile of
// 128 output pixels is whole rows of one image (W divides 128 and the rows
// of an image split into whole tiles) or part of one row (W a multiple of
// 128).
inline bool conv_implicit_ok(int C, int H, int W) {
    if (C % 32 || C <= 0) return false;
    if (W % 128 == 0) return true;
    return W > 0 && 128 % W == 0 && H % (128 / W) == 0;
}

cudaError_t launch_conv_implicit(const ConvArgs& a, int* err, cudaStream_t s);

}  // namespace gdrr
