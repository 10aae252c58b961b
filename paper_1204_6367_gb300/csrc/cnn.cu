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
//   forward   Y[P x Co]   = cols[P x K9] . W[Co x K9]^T
//   data grad dcols[P x K9] = dZ[P x Co] . Wt[K9 x Co]^T, then col2im
//   weight    dW[Co x K9] = dZ^T[Co x P] . colsT[K9 x P]^T   (split over P)
// with P = batch * H * W pixels and K9 = Cin * 9 rounded up to 64.
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

// cols[p][k], p = (b, y, x), k = ci * ks * ks + ky * ks + kx (zero beyond C * ks * ks);
// transposed = colsT[k][p] with row length ldp.
__global__ void im2col_kernel(const bf16* __restrict__ x, int B, int C, int H, int W, int ks, int K9p, int ldp,
                              int transposed, bf16* __restrict__ out) {
    const int64_t P = (int64_t)B * H * W;
    const int64_t cols = transposed ? (int64_t)ldp : P;       // pixel columns written, padding included
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cols * K9p) return;
    int64_t p;
    int k;
    if (transposed) { k = (int)(i / ldp); p = i % ldp; }
    else { p = i / K9p; k = (int)(i % K9p); }
    bf16 v = __float2bfloat16_rn(0.0f);
    const int kk = ks * ks;
    if (k < C * kk && p < P) {
        const int ci = k / kk, r = k % kk, ky = r / ks, kx = r % ks;
        const int b = (int)(p / ((int64_t)H * W));
        const int yx = (int)(p % ((int64_t)H * W));
        const int yy = yx / W + ky - ks / 2, xx = yx % W + kx - ks / 2;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = x[(((int64_t)b * C + ci) * H + yy) * W + xx];
    }
    if (transposed) out[(int64_t)k * ldp + p] = v;
    else out[p * K9p + k] = v;
}

// Y[b][co][y][x] (BF16, channel offset in a wider tensor) = act(G[p][co] + bias[co]);
// also the FP32 value when yf != NULL.
__global__ void bias_act_kernel(const float* __restrict__ G, int ldg, const float* __restrict__ bias, int B, int Co,
                                int H, int W, int relu, bf16* __restrict__ y, int y_channels, float* __restrict__ yf) {
    const int64_t n = (int64_t)B * Co * H * W;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % W);
    const int yy = (int)((i / W) % H);
    const int co = (int)((i / ((int64_t)W * H)) % Co);
    const int b = (int)(i / ((int64_t)W * H * Co));
    const int64_t p = ((int64_t)b * H + yy) * W + x;
    float v = G[p * ldg + co] + bias[co];
    if (relu) v = fmaxf(v, 0.0f);
    if (y) y[(((int64_t)b * y_channels + co) * H + yy) * W + x] = __float2bfloat16_rn(v);
    if (yf) yf[i] = v;
}

// dZ = dY * (Y > 0) (or dY when relu == 0), written as BF16 in two layouts:
// dz_pc[p][co] (row length ldc_pad) and dz_cp[co][p] (row length ldp).
__global__ void act_back_kernel(const float* __restrict__ dy, const bf16* __restrict__ y, int y_channels, int B,
                                int Co, int H, int W, int relu, bf16* __restrict__ dz_pc, int ldc_pad,
                                bf16* __restrict__ dz_cp, int ldp, float* __restrict__ dz_f) {
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
    const bf16 gb = __float2bfloat16_rn(g);
    dz_pc[p * ldc_pad + co] = gb;
    dz_cp[(int64_t)co * ldp + p] = gb;
    dz_f[i] = g;
}

// db[co] = sum over pixels of dZ (FP32), one block per channel.
__global__ void bias_grad_kernel(const float* __restrict__ dz, int B, int Co, int HW, float* __restrict__ db) {
    const int co = blockIdx.x;
    float s = 0.0f;
    for (int64_t i = threadIdx.x; i < (int64_t)B * HW; i += blockDim.x) {
        const int b = (int)(i / HW), r = (int)(i % HW);
        s += dz[((int64_t)b * Co + co) * HW + r];
    }
    __shared__ float red[TB];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[co] = red[0];
}

// dX[b][ci][y][x] = sum over (ky, kx) of dcols[p(b, y - ky + h, x - kx + h)][ci * kk + ky * ks + kx].
__global__ void col2im_kernel(const float* __restrict__ dcols, int K9p, int B, int C, int H, int W, int ks,
                              float* __restrict__ dx) {
    const int64_t n = (int64_t)B * C * H * W;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % W);
    const int y = (int)((i / W) % H);
    const int ci = (int)((i / ((int64_t)W * H)) % C);
    const int b = (int)(i / ((int64_t)W * H * C));
    const int kk = ks * ks, h = ks / 2;
    float s = 0.0f;
    for (int ky = 0; ky < ks; ++ky)
        for (int kx = 0; kx < ks; ++kx) {
            const int yo = y - ky + h, xo = x - kx + h;
            if (yo < 0 || yo >= H || xo < 0 || xo >= W) continue;
            const int64_t p = ((int64_t)b * H + yo) * W + xo;
            s += dcols[p * K9p + ci * kk + ky * ks + kx];
        }
    dx[i] = s;
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

// dst[b][off + c][y][x] = src[b][c][y / s][x / s], s = 2 (upsample) or 1 (copy)
__global__ void place_kernel(const bf16* __restrict__ src, int B, int C, int H, int W, int s, bf16* __restrict__ dst,
                             int dst_channels, int off) {
    const int64_t n = (int64_t)B * C * H * W;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % W), y = (int)((i / W) % H);
    const int c = (int)((i / ((int64_t)W * H)) % C);
    const int b = (int)(i / ((int64_t)W * H * C));
    dst[(((int64_t)b * dst_channels + off + c) * H + y) * W + x] =
        src[(((int64_t)b * C + c) * (H / s) + y / s) * (W / s) + x / s];
}

// adjoint of place: dsrc[b][c][y][x] (+)= sum over the s x s block of dcat[b][off + c]
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

// BF16 copies of a conv's weights: w16[co][k] (row K9p) and wt16[k][co] (row Co_p)
__global__ void weight_copies_kernel(const float* __restrict__ w, int Co, int K9, int K9p, int Cop,
                                     bf16* __restrict__ w16, bf16* __restrict__ wt16) {
    const int64_t n = (int64_t)Co * K9p;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int co = (int)(i / K9p), k = (int)(i % K9p);
    const bf16 v = __float2bfloat16_rn(k < K9 ? w[(int64_t)co * K9 + k] : 0.0f);
    w16[i] = v;
    wt16[(int64_t)k * Cop + co] = v;
}

// dW[co][k] for k < K9 from the padded GEMM output (row K9p)
__global__ void unpad_kernel(const float* __restrict__ src, int rows, int cols, int ld, float* __restrict__ dst) {
    const int64_t n = (int64_t)rows * cols;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[(i / cols) * ld + i % cols];
}

struct Conv {
    int ci, co, ks, H, W, relu;
    int K9, K9p, Cop;
    // parameters (FP32 master), gradients, Adam moments; offsets into the flat arrays
    int64_t w_off, b_off;
    bf16* w16 = nullptr;   // [co][K9p]
    bf16* wt16 = nullptr;  // [K9p][Cop]
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
    bf16 *p1 = nullptr, *p2 = nullptr, *p3 = nullptr, *c3 = nullptr, *c2 = nullptr, *c1 = nullptr;
    bf16 *d3 = nullptr, *d2 = nullptr, *d1 = nullptr;
    float* out = nullptr;
    // gradients of activations (FP32)
    float *g_out = nullptr, *g_d1 = nullptr, *g_c1 = nullptr, *g_d2 = nullptr, *g_c2 = nullptr, *g_d3 = nullptr;
    float *g_c3 = nullptr, *g_e4 = nullptr, *g_p3 = nullptr, *g_e3 = nullptr, *g_p2 = nullptr, *g_e2 = nullptr;
    float *g_p1 = nullptr, *g_e1 = nullptr, *g_x = nullptr;
    // workspaces
    bf16* cols = nullptr;      // im2col, either layout
    float* gemm = nullptr;     // GEMM output
    float* partials = nullptr; // per-split partial products of the weight gradients
    bf16* dz_pc = nullptr;
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
        const int64_t cnt = (int64_t)L.co * L.K9p;
        weight_copies_kernel<<<nblk(cnt), TB, 0, n->stream>>>(n->params + L.w_off, L.co, L.K9, L.K9p, L.Cop, L.w16,
                                                              L.wt16);
        CK(cudaGetLastError());
    }
    return cudaSuccess;
}

// Forward of one convolution from x (BF16 [B][ci][H][W]) into y (BF16, channel
// count y_channels, written at channels 0 .. co-1) and/or yf (FP32).
cudaError_t conv_forward(gdrr_cnn* n, const Conv& L, int B, const bf16* x, bf16* y, int y_channels, float* yf) {
    const int64_t P = (int64_t)B * L.H * L.W;
    im2col_kernel<<<nblk(P * L.K9p), TB, 0, n->stream>>>(x, B, L.ci, L.H, L.W, L.ks, L.K9p, 0, 0, n->cols);
    CK(cudaGetLastError());
    CK(launch_gemm_bf16(n->cols, L.K9p, L.w16, L.K9p, n->gemm, L.co, (int)P, L.co, L.K9p, 1, n->err, n->stream));
    bias_act_kernel<<<nblk(P * L.co), TB, 0, n->stream>>>(n->gemm, L.co, n->params + L.b_off, B, L.co, L.H, L.W,
                                                          L.relu, y, y_channels, yf);
    return cudaGetLastError();
}

// Backward of one convolution: dy (FP32 [B][co][H][W], gradient of the
// layer output), y (its BF16 output, for the ReLU mask), x (its BF16 input).
// Writes the parameter gradients and, when dx != NULL, dx (FP32 input grad).
cudaError_t conv_backward(gdrr_cnn* n, const Conv& L, int B, const float* dy, const bf16* y, int y_channels,
                          const bf16* x, float* dx) {
    const int64_t P = (int64_t)B * L.H * L.W;
    const int Pp = pad64(P);
    CK(cudaMemsetAsync(n->dz_pc, 0, (size_t)P * L.Cop * sizeof(bf16), n->stream));
    CK(cudaMemsetAsync(n->dz_cp, 0, (size_t)L.co * Pp * sizeof(bf16), n->stream));
    act_back_kernel<<<nblk(P * L.co), TB, 0, n->stream>>>(dy, y, y_channels, B, L.co, L.H, L.W, L.relu, n->dz_pc,
                                                          L.Cop, n->dz_cp, Pp, n->dz_f);
    CK(cudaGetLastError());
    bias_grad_kernel<<<L.co, TB, 0, n->stream>>>(n->dz_f, B, L.co, L.H * L.W, n->grads + L.b_off);
    CK(cudaGetLastError());
    // weight gradient: dW[co][k] = sum_p dZ[p][co] cols[p][k]
    im2col_kernel<<<nblk((int64_t)Pp * L.K9p), TB, 0, n->stream>>>(x, B, L.ci, L.H, L.W, L.ks, L.K9p, Pp, 1, n->cols);
    CK(cudaGetLastError());
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
        // data gradient: dcols[p][k] = sum_co dZ[p][co] W[co][k]; then col2im
        CK(launch_gemm_bf16(n->dz_pc, L.Cop, L.wt16, L.Cop, n->gemm, L.K9p, (int)P, L.K9p, L.Cop, 1, n->err,
                            n->stream));
        col2im_kernel<<<nblk(P * L.ci), TB, 0, n->stream>>>(n->gemm, L.K9p, B, L.ci, L.H, L.W, L.ks, dx);
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
        L.Cop = pad64(s.co);
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
        max_cols = std::max(max_cols, Pp * L.K9p);
        max_gemm = std::max({max_gemm, P * L.K9p, (int64_t)L.co * L.K9p, P * L.co});
        max_dz = std::max({max_dz, P * L.Cop, (int64_t)L.co * Pp});
        max_part = std::max(max_part, (int64_t)wgrad_splits(P) * L.co * L.K9p);
    }
    cudaError_t e = cudaSuccess;
    do {
        if ((e = dalloc(n, &n->params, off)) || (e = dalloc(n, &n->grads, off)) || (e = dalloc(n, &n->adam_m, off)) ||
            (e = dalloc(n, &n->adam_v, off)))
            break;
        bool bad = false;
        for (Conv& L : n->conv) {
            if (dalloc(n, &L.w16, (size_t)L.co * L.K9p) || dalloc(n, &L.wt16, (size_t)L.K9p * L.Cop)) bad = true;
            // padded output-channel columns of wt16 stay zero (weight copies write co < Co only)
            else if (cudaMemset(L.wt16, 0, (size_t)L.K9p * L.Cop * sizeof(bf16)) != cudaSuccess) bad = true;
        }
        if (bad) { e = cudaErrorMemoryAllocation; break; }
        const int64_t s1 = B * HW, s2 = s1 / 4, s3 = s1 / 16, s4 = s1 / 64;
        if ((e = dalloc(n, &n->x16, 2 * s1)) || (e = dalloc(n, &n->e1, c * s1)) || (e = dalloc(n, &n->p1, c * s2)) ||
            (e = dalloc(n, &n->e2, 2 * c * s2)) || (e = dalloc(n, &n->p2, 2 * c * s3)) ||
            (e = dalloc(n, &n->e3, 4 * c * s3)) || (e = dalloc(n, &n->p3, 4 * c * s4)) ||
            (e = dalloc(n, &n->e4, 8 * c * s4)) || (e = dalloc(n, &n->c3, 12 * c * s3)) ||
            (e = dalloc(n, &n->d3, 4 * c * s3)) || (e = dalloc(n, &n->c2, 6 * c * s2)) ||
            (e = dalloc(n, &n->d2, 2 * c * s2)) || (e = dalloc(n, &n->c1, 3 * c * s1)) ||
            (e = dalloc(n, &n->d1, c * s1)) || (e = dalloc(n, &n->out, s1)))
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
            (e = dalloc(n, &n->dz_pc, max_dz)) || (e = dalloc(n, &n->dz_cp, max_dz)) ||
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
        if ((e = conv_forward(n, L[0], B, n->x16, n->e1, c, nullptr))) break;
        pool_kernel<<<nblk(c * s1 / 4), TB, 0, st>>>(n->e1, B, c, H, W, n->p1);
        if ((e = conv_forward(n, L[1], B, n->p1, n->e2, 2 * c, nullptr))) break;
        pool_kernel<<<nblk(2 * c * s1 / 16), TB, 0, st>>>(n->e2, B, 2 * c, H / 2, W / 2, n->p2);
        if ((e = conv_forward(n, L[2], B, n->p2, n->e3, 4 * c, nullptr))) break;
        pool_kernel<<<nblk(4 * c * s1 / 64), TB, 0, st>>>(n->e3, B, 4 * c, H / 4, W / 4, n->p3);
        if ((e = conv_forward(n, L[3], B, n->p3, n->e4, 8 * c, nullptr))) break;
        // decoder: [up(prev), skip]
        place_kernel<<<nblk(8 * c * s1 / 16), TB, 0, st>>>(n->e4, B, 8 * c, H / 4, W / 4, 2, n->c3, 12 * c, 0);
        place_kernel<<<nblk(4 * c * s1 / 16), TB, 0, st>>>(n->e3, B, 4 * c, H / 4, W / 4, 1, n->c3, 12 * c, 8 * c);
        if ((e = conv_forward(n, L[4], B, n->c3, n->d3, 4 * c, nullptr))) break;
        place_kernel<<<nblk(4 * c * s1 / 4), TB, 0, st>>>(n->d3, B, 4 * c, H / 2, W / 2, 2, n->c2, 6 * c, 0);
        place_kernel<<<nblk(2 * c * s1 / 4), TB, 0, st>>>(n->e2, B, 2 * c, H / 2, W / 2, 1, n->c2, 6 * c, 4 * c);
        if ((e = conv_forward(n, L[5], B, n->c2, n->d2, 2 * c, nullptr))) break;
        place_kernel<<<nblk(2 * c * s1), TB, 0, st>>>(n->d2, B, 2 * c, H, W, 2, n->c1, 3 * c, 0);
        place_kernel<<<nblk(c * s1), TB, 0, st>>>(n->e1, B, c, H, W, 1, n->c1, 3 * c, 2 * c);
        if ((e = conv_forward(n, L[6], B, n->c1, n->d1, c, nullptr))) break;
        if ((e = conv_forward(n, L[7], B, n->d1, nullptr, 1, n->out))) break;
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
        if ((e = conv_backward(n, L[7], B, n->g_out, nullptr, 1, n->d1, n->g_d1))) break;
        if ((e = conv_backward(n, L[6], B, n->g_d1, n->d1, c, n->c1, n->g_c1))) break;
        // c1 = [up(d2), e1]
        place_back_kernel<<<nblk(2 * c * s1 / 4), TB, 0, st>>>(n->g_c1, 3 * c, 0, B, 2 * c, H / 2, W / 2, 2, 0, n->g_d2);
        place_back_kernel<<<nblk(c * s1), TB, 0, st>>>(n->g_c1, 3 * c, 2 * c, B, c, H, W, 1, 0, n->g_e1);
        if ((e = conv_backward(n, L[5], B, n->g_d2, n->d2, 2 * c, n->c2, n->g_c2))) break;
        place_back_kernel<<<nblk(4 * c * s1 / 16), TB, 0, st>>>(n->g_c2, 6 * c, 0, B, 4 * c, H / 4, W / 4, 2, 0, n->g_d3);
        place_back_kernel<<<nblk(2 * c * s1 / 4), TB, 0, st>>>(n->g_c2, 6 * c, 4 * c, B, 2 * c, H / 2, W / 2, 1, 0,
                                                              n->g_e2);
        if ((e = conv_backward(n, L[4], B, n->g_d3, n->d3, 4 * c, n->c3, n->g_c3))) break;
        place_back_kernel<<<nblk(8 * c * s1 / 64), TB, 0, st>>>(n->g_c3, 12 * c, 0, B, 8 * c, H / 8, W / 8, 2, 0,
                                                               n->g_e4);
        place_back_kernel<<<nblk(4 * c * s1 / 16), TB, 0, st>>>(n->g_c3, 12 * c, 8 * c, B, 4 * c, H / 4, W / 4, 1, 0,
                                                               n->g_e3);
        // encoder
        if ((e = conv_backward(n, L[3], B, n->g_e4, n->e4, 8 * c, n->p3, n->g_p3))) break;
        pool_back_kernel<<<nblk(4 * c * s1 / 16), TB, 0, st>>>(n->g_p3, B, 4 * c, H / 4, W / 4, n->g_e3);
        if ((e = conv_backward(n, L[2], B, n->g_e3, n->e3, 4 * c, n->p2, n->g_p2))) break;
        pool_back_kernel<<<nblk(2 * c * s1 / 4), TB, 0, st>>>(n->g_p2, B, 2 * c, H / 2, W / 2, n->g_e2);
        if ((e = conv_backward(n, L[1], B, n->g_e2, n->e2, 2 * c, n->p1, n->g_p1))) break;
        pool_back_kernel<<<nblk(c * s1), TB, 0, st>>>(n->g_p1, B, c, H, W, n->g_e1);
        if ((e = conv_backward(n, L[0], B, n->g_e1, n->e1, c, n->x16, nullptr))) break;
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
