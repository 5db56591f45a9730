// Learned correction network (not in the paper): a 4-layer 3x3 convolutional
// net, channels 6 -> 32 -> 32 -> 32 -> 1, ReLU after layers 1..3, trained on
// the GPU by these kernels (forward, backpropagation, half-MSE loss, Adam).
//
//   conv3x3(a; W, b)[o, i, j] = b[o] + sum_c sum_{p,q} W[o, c, p, q] a[c, i+p-1, j+q-1]
//   (zero outside the image), images NCHW in FP32.
//
// With BF16 operands the 32-output-channel convolutions (the forward layers
// 1-3 and the backward-data convolutions) run on the tensor cores (mma.sync
// BF16, FP32 accumulation); the one-channel output layer and the weight
// gradient round their operands to BF16 and accumulate in FP32 on the FMA
// pipes.  With BF16 off every kernel is plain FP32 on the FMA pipes.
#include "asdsm.h"
#include "asdsm_internal.h"
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace {

constexpr int CNN_LAYERS = 4;
constexpr int CNN_CH[CNN_LAYERS + 1] = {6, 32, 32, 32, 1};
constexpr int TILE = 16;                 // output pixels per CTA side
constexpr int CONV_THREADS = TILE * TILE;

constexpr int layer_w(int l) { return CNN_CH[l + 1] * CNN_CH[l] * 9; }
constexpr int layer_off(int l) {
    int off = 0;
    for (int q = 0; q < l; ++q) off += layer_w(q) + CNN_CH[q + 1];
    return off;
}
constexpr int CNN_PARAMS = layer_off(CNN_LAYERS);

__device__ __forceinline__ float round_bf16(float x, bool on) {
    return on ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}

// out[b, o, i, j] = (bias[o]) + sum_c sum_taps W[o, c, p, q] in[b, c, i+p-1, j+q-1];
// then relu (relu_out) or times (mask > 0) (mask: same shape as out).
template <int COUT>
__global__ void __launch_bounds__(CONV_THREADS)
conv3x3_kernel(const float* __restrict__ in, int cin, const float* __restrict__ W, const float* __restrict__ bias,
               float* __restrict__ out, int H, int Wd, int relu_out, const float* __restrict__ mask, int bf16) {
    __shared__ float tile[TILE + 2][TILE + 2];
    __shared__ float wsm[COUT * 9];
    const int b = blockIdx.z;
    const int i0 = blockIdx.y * TILE, j0 = blockIdx.x * TILE;
    const int ty = threadIdx.x / TILE, tx = threadIdx.x % TILE;
    const int i = i0 + ty, j = j0 + tx;
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = bias ? bias[o] : 0.0f;
    const size_t plane = (size_t)H * Wd;
    for (int c = 0; c < cin; ++c) {
        const float* src = in + ((size_t)b * cin + c) * plane;
        for (int e = threadIdx.x; e < (TILE + 2) * (TILE + 2); e += CONV_THREADS) {
            const int r = e / (TILE + 2), q = e % (TILE + 2);
            const int ii = i0 + r - 1, jj = j0 + q - 1;
            const float v = (ii >= 0 && ii < H && jj >= 0 && jj < Wd) ? src[(size_t)ii * Wd + jj] : 0.0f;
            tile[r][q] = round_bf16(v, bf16);
        }
        for (int e = threadIdx.x; e < COUT * 9; e += CONV_THREADS) {
            const int o = e / 9, t = e % 9;
            wsm[e] = round_bf16(W[((size_t)o * cin + c) * 9 + t], bf16);
        }
        __syncthreads();
        float v[9];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) v[p * 3 + q] = tile[ty + p][tx + q];
#pragma unroll
        for (int o = 0; o < COUT; ++o) {
            float s = acc[o];
#pragma unroll
            for (int t = 0; t < 9; ++t) s = fmaf(wsm[o * 9 + t], v[t], s);
            acc[o] = s;
        }
        __syncthreads();
    }
    if (i >= H || j >= Wd) return;
#pragma unroll
    for (int o = 0; o < COUT; ++o) {
        const size_t idx = ((size_t)b * COUT + o) * plane + (size_t)i * Wd + j;
        float r = acc[o];
        if (relu_out) r = fmaxf(r, 0.0f);
        if (mask) r = mask[idx] > 0.0f ? r : 0.0f;
        out[idx] = r;
    }
}

// The same convolution for 32 output channels on the tensor cores (BF16
// operands, FP32 accumulation): an implicit GEMM out[pixel][o] =
// sum_k A[pixel][k] W[o][k] with k = c*9 + 3p + q (zero beyond 9 cin, padded
// to a multiple of 16), mma.sync m16n8k16.  A CTA owns 16 x 16 pixels; warp w
// computes tile rows 2w, 2w+1 (one m16 fragment each: the 16 pixels of the
// row) x 32 channels (4 n8 fragments).  The input tile of every channel (with
// its halo) and the weights, as [o][k] rows padded to keep the B-fragment
// loads conflict-free, are staged once in shared memory as BF16.
__device__ __forceinline__ unsigned pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

__global__ void __launch_bounds__(CONV_THREADS)
conv3x3_tc_kernel(const float* __restrict__ in, int cin, const float* __restrict__ W, const float* __restrict__ bias,
                  float* __restrict__ out, int H, int Wd, int relu_out, const float* __restrict__ mask) {
    extern __shared__ __align__(16) unsigned char tc_smem[];
    constexpr int TP = TILE + 2;                        // 18
    const int K = cin * 9;
    const int Kp = (K + 15) / 16 * 16;
    const int KS = Kp + 8;                              // row stride of the weight rows
    __nv_bfloat16* tin = reinterpret_cast<__nv_bfloat16*>(tc_smem);        // [cin][18][18]
    __nv_bfloat16* ws = tin + ((cin * TP * TP + 7) / 8) * 8;               // [32][KS]
    const int b = blockIdx.z;
    const int i0 = blockIdx.y * TILE, j0 = blockIdx.x * TILE;
    const size_t plane = (size_t)H * Wd;
    for (int e = threadIdx.x; e < cin * TP * TP; e += CONV_THREADS) {
        const int c = e / (TP * TP), rq = e % (TP * TP);
        const int ii = i0 + rq / TP - 1, jj = j0 + rq % TP - 1;
        const float v = (ii >= 0 && ii < H && jj >= 0 && jj < Wd) ? in[((size_t)b * cin + c) * plane + (size_t)ii * Wd + jj] : 0.0f;
        tin[e] = __float2bfloat16_rn(v);
    }
    for (int e = threadIdx.x; e < 32 * KS; e += CONV_THREADS) {
        const int o = e / KS, k = e % KS;
        ws[e] = __float2bfloat16_rn(k < K ? W[(size_t)o * K + k] : 0.0f);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    for (int kb = 0; kb < Kp; kb += 16) {
        // the four reduction indices of this lane: kb + 2q + {0, 1, 8, 9}
        int off[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = kb + 2 * q + (u & 1) + (u >> 1) * 8;
            ok[u] = k < K;
            const int c = ok[u] ? k / 9 : 0, t = ok[u] ? k % 9 : 0;
            off[u] = c * TP * TP + (t / 3) * TP + (t % 3);
        }
        unsigned a[2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int row = (2 * warp + i) * TP;        // tile row of this fragment (pixels along x)
            auto at = [&](int u, int x) { return ok[u] ? tin[off[u] + row + x] : zero; };
            a[i][0] = pack_bf16(at(0, g), at(1, g));
            a[i][1] = pack_bf16(at(0, g + 8), at(1, g + 8));
            a[i][2] = pack_bf16(at(2, g), at(3, g));
            a[i][3] = pack_bf16(at(2, g + 8), at(3, g + 8));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __nv_bfloat16* wr = ws + (size_t)(j * 8 + g) * KS + kb + 2 * q;
            const unsigned b0 = *reinterpret_cast<const unsigned*>(wr);
            const unsigned b1 = *reinterpret_cast<const unsigned*>(wr + 8);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                float* d = acc[i][j];
                asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                             : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                             : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b0), "r"(b1));
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int y = i0 + 2 * warp + i;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int x = j0 + g + ((e >> 1) << 3);
                const int o = j * 8 + 2 * q + (e & 1);
                if (y >= H || x >= Wd) continue;
                const size_t idx = ((size_t)b * 32 + o) * plane + (size_t)y * Wd + x;
                float r = acc[i][j][e] + (bias ? bias[o] : 0.0f);
                if (relu_out) r = fmaxf(r, 0.0f);
                if (mask) r = mask[idx] > 0.0f ? r : 0.0f;
                out[idx] = r;
            }
    }
}

size_t conv_tc_smem(int cin) {
    const int K = cin * 9, Kp = (K + 15) / 16 * 16;
    return sizeof(__nv_bfloat16) * ((size_t)((cin * (TILE + 2) * (TILE + 2) + 7) / 8) * 8 + (size_t)32 * (Kp + 8));
}

// W'[c, o, 2-p, 2-q] = W[o, c, p, q]: the backward-data convolution is a
// forward convolution of dZ with W'.
__global__ void flip_transpose_kernel(const float* __restrict__ W, int cout, int cin, float* __restrict__ Wt) {
    const int n = cout * cin * 9;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int o = e / (cin * 9), c = (e / 9) % cin, t = e % 9;
        const int p = t / 3, q = t % 3;
        Wt[((size_t)c * cout + o) * 9 + (2 - p) * 3 + (2 - q)] = W[e];
    }
}

// Per-tile partial sums of dW[o, c, p, q] = sum dZ[b, o, i, j] a[b, c, i+p-1, j+q-1]
// and db[o] = sum dZ[b, o, i, j]; partials[tile][cout*cin*9 + cout].
__global__ void __launch_bounds__(CONV_THREADS)
conv_wgrad_kernel(const float* __restrict__ dZ, int cout, const float* __restrict__ A, int cin, int H, int Wd,
                  float* __restrict__ partials, int bf16) {
    extern __shared__ float wg_smem[];
    float* dz = wg_smem;                                    // [cout][TILE*TILE]
    float* at = dz + cout * TILE * TILE;                    // [cin][TILE+2][TILE+2]
    const int b = blockIdx.z;
    const int i0 = blockIdx.y * TILE, j0 = blockIdx.x * TILE;
    const size_t plane = (size_t)H * Wd;
    for (int e = threadIdx.x; e < cout * TILE * TILE; e += CONV_THREADS) {
        const int o = e / (TILE * TILE), pix = e % (TILE * TILE);
        const int i = i0 + pix / TILE, j = j0 + pix % TILE;
        const float v = (i < H && j < Wd) ? dZ[((size_t)b * cout + o) * plane + (size_t)i * Wd + j] : 0.0f;
        dz[e] = round_bf16(v, bf16);
    }
    for (int e = threadIdx.x; e < cin * (TILE + 2) * (TILE + 2); e += CONV_THREADS) {
        const int c = e / ((TILE + 2) * (TILE + 2)), rq = e % ((TILE + 2) * (TILE + 2));
        const int ii = i0 + rq / (TILE + 2) - 1, jj = j0 + rq % (TILE + 2) - 1;
        const float v = (ii >= 0 && ii < H && jj >= 0 && jj < Wd) ? A[((size_t)b * cin + c) * plane + (size_t)ii * Wd + jj] : 0.0f;
        at[e] = round_bf16(v, bf16);
    }
    __syncthreads();
    const int nw = cout * cin * 9;
    const long long tile_id = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    float* dst = partials + tile_id * (nw + cout);
    for (int e = threadIdx.x; e < nw + cout; e += CONV_THREADS) {
        float s = 0.0f;
        if (e < nw) {
            const int o = e / (cin * 9), c = (e / 9) % cin, t = e % 9;
            const int p = t / 3, q = t % 3;
            const float* dzo = dz + o * TILE * TILE;
            const float* ac = at + c * (TILE + 2) * (TILE + 2);
            for (int pix = 0; pix < TILE * TILE; ++pix) {
                const int r = pix / TILE, cc = pix % TILE;
                s = fmaf(dzo[pix], ac[(r + p) * (TILE + 2) + cc + q], s);
            }
        } else {
            const float* dzo = dz + (e - nw) * TILE * TILE;
            for (int pix = 0; pix < TILE * TILE; ++pix) s += dzo[pix];
        }
        dst[e] = s;
    }
}

// out[e] = sum over tiles of partials[tile][e] (fixed order, FP64 accumulation).
__global__ void sum_partials_kernel(const float* __restrict__ partials, long long ntiles, int n, float* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (long long t = 0; t < ntiles; ++t) s += partials[t * n + e];
        out[e] = (float)s;
    }
}

// dY = w (y - t) / n; per-block sums of w (y - t)^2 (w = 1 when no weights).
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ wt,
                           long long n, float* __restrict__ dy, double* __restrict__ part) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float d = y[e] - t[e];
        const float we = wt ? wt[e] : 1.0f;
        dy[e] = we * d / (float)n;
        s += (double)we * d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = b1 * m[e] + (1.0f - b1) * ge;
        const float ve = b2 * v[e] + (1.0f - b2) * ge * ge;
        m[e] = me;
        v[e] = ve;
        theta[e] -= lr * (me / c1) / (sqrtf(ve / c2) + eps);
    }
}

thread_local std::string g_cnn_error;

}  // namespace

struct asdsm_cnn {
    float* theta = nullptr;
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* wt = nullptr;               // flipped/transposed weights of one layer
    int step = 0;
    int bf16 = 1;
    // Work space sized for B*H*W pixels.
    long long cap_pix = 0;
    float* act[CNN_LAYERS + 1] = {};   // act[0] unused (the input), act[l]: (B, C_l, H, W)
    float* dz[2] = {nullptr, nullptr};
    float* partials = nullptr;
    long long cap_partials = 0;
    double* dpart = nullptr;
    double* hpart = nullptr;
};

namespace {

int cnn_cuda(cudaError_t e) {
    g_cnn_error = cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ASDSM_ERR_OOM : ASDSM_ERR_CUDA;
}
#define CNN_CK(...)                                   \
    do {                                              \
        cudaError_t e__ = (__VA_ARGS__);              \
        if (e__ != cudaSuccess) return cnn_cuda(e__); \
    } while (0)

int ensure_space(asdsm_cnn* net, long long pix, long long ntiles) {
    if (pix > net->cap_pix) {
        for (int l = 1; l <= CNN_LAYERS; ++l) {
            if (net->act[l]) cudaFree(net->act[l]);
            net->act[l] = nullptr;
        }
        for (int q = 0; q < 2; ++q) {
            if (net->dz[q]) cudaFree(net->dz[q]);
            net->dz[q] = nullptr;
        }
        net->cap_pix = 0;
        for (int l = 1; l <= CNN_LAYERS; ++l) CNN_CK(cudaMalloc(&net->act[l], (size_t)pix * CNN_CH[l] * sizeof(float)));
        for (int q = 0; q < 2; ++q) CNN_CK(cudaMalloc(&net->dz[q], (size_t)pix * 32 * sizeof(float)));
        net->cap_pix = pix;
    }
    const long long need = ntiles * (32LL * 32 * 9 + 32);
    if (need > net->cap_partials) {
        if (net->partials) cudaFree(net->partials);
        net->partials = nullptr;
        net->cap_partials = 0;
        CNN_CK(cudaMalloc(&net->partials, (size_t)need * sizeof(float)));
        net->cap_partials = need;
    }
    return ASDSM_OK;
}

cudaError_t conv(const float* in, int cin, int cout, const float* W, const float* bias, float* out, int B, int H,
                 int Wd, int relu, const float* mask, int bf16, cudaStream_t st) {
    dim3 grid((Wd + TILE - 1) / TILE, (H + TILE - 1) / TILE, B);
    if (cout == 32 && bf16) {
        const size_t smem = conv_tc_smem(cin);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        conv3x3_tc_kernel<<<grid, CONV_THREADS, smem, st>>>(in, cin, W, bias, out, H, Wd, relu, mask);
    } else if (cout == 32) conv3x3_kernel<32><<<grid, CONV_THREADS, 0, st>>>(in, cin, W, bias, out, H, Wd, relu, mask, bf16);
    else if (cout == 1) conv3x3_kernel<1><<<grid, CONV_THREADS, 0, st>>>(in, cin, W, bias, out, H, Wd, relu, mask, bf16);
    else return cudaErrorInvalidValue;
    asdsm::note_launch();
    return cudaGetLastError();
}

int forward_impl(asdsm_cnn* net, const float* x, float* y, int B, int H, int Wd, cudaStream_t st) {
    const long long pix = (long long)B * H * Wd;
    const long long ntiles = (long long)B * ((H + TILE - 1) / TILE) * ((Wd + TILE - 1) / TILE);
    if (int rc = ensure_space(net, pix, ntiles)) return rc;
    const float* a = x;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        const float* W = net->theta + layer_off(l);
        const float* b = W + layer_w(l);
        float* out = l + 1 < CNN_LAYERS ? net->act[l + 1] : (y ? y : net->act[CNN_LAYERS]);
        CNN_CK(conv(a, CNN_CH[l], CNN_CH[l + 1], W, b, out, B, H, Wd, l + 1 < CNN_LAYERS, nullptr, net->bf16, st));
        a = out;
    }
    if (y && y != net->act[CNN_LAYERS])
        CNN_CK(cudaMemcpyAsync(net->act[CNN_LAYERS], y, (size_t)pix * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return ASDSM_OK;
}

}  // namespace

extern "C" {

int asdsm_cnn_param_count(void) { return CNN_PARAMS; }

int asdsm_cnn_create(const float* params, int n, int bf16_operands, asdsm_cnn** out) {
    if (!out) return ASDSM_ERR_INVALID;
    *out = nullptr;
    if (!params || n != CNN_PARAMS) return ASDSM_ERR_INVALID;
    asdsm_cnn* net = new asdsm_cnn();
    net->bf16 = bf16_operands ? 1 : 0;
    auto fail = [&](int rc) { asdsm_cnn_destroy(net); return rc; };
    cudaError_t e;
    float** bufs[4] = {&net->theta, &net->grad, &net->m, &net->v};
    for (auto** b : bufs)
        if ((e = cudaMalloc(b, (size_t)CNN_PARAMS * sizeof(float))) != cudaSuccess) return fail(cnn_cuda(e));
    if ((e = cudaMalloc(&net->wt, (size_t)32 * 32 * 9 * sizeof(float))) != cudaSuccess) return fail(cnn_cuda(e));
    if ((e = cudaMemcpy(net->theta, params, (size_t)CNN_PARAMS * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(cnn_cuda(e));
    for (float* b : {net->grad, net->m, net->v})
        if ((e = cudaMemset(b, 0, (size_t)CNN_PARAMS * sizeof(float))) != cudaSuccess) return fail(cnn_cuda(e));
    if ((e = cudaMalloc(&net->dpart, 1024 * sizeof(double))) != cudaSuccess) return fail(cnn_cuda(e));
    if ((e = cudaMallocHost(&net->hpart, 1024 * sizeof(double))) != cudaSuccess) return fail(cnn_cuda(e));
    *out = net;
    return ASDSM_OK;
}

int asdsm_cnn_get_params(const asdsm_cnn* net, float* params, int n) {
    if (!net || !params || n != CNN_PARAMS) return ASDSM_ERR_INVALID;
    CNN_CK(cudaMemcpy(params, net->theta, (size_t)CNN_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    return ASDSM_OK;
}

int asdsm_cnn_set_params(asdsm_cnn* net, const float* params, int n) {
    if (!net || !params || n != CNN_PARAMS) return ASDSM_ERR_INVALID;
    CNN_CK(cudaMemcpy(net->theta, params, (size_t)CNN_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
    net->step = 0;
    CNN_CK(cudaMemset(net->m, 0, (size_t)CNN_PARAMS * sizeof(float)));
    CNN_CK(cudaMemset(net->v, 0, (size_t)CNN_PARAMS * sizeof(float)));
    return ASDSM_OK;
}

int asdsm_cnn_forward(asdsm_cnn* net, const float* x, float* y, int B, int H, int W, void* stream) {
    if (!net || !x || !y || B < 1 || H < 1 || W < 1) return ASDSM_ERR_INVALID;
    return forward_impl(net, x, y, B, H, W, (cudaStream_t)stream);
}

int asdsm_cnn_backward(asdsm_cnn* net, const float* x, const float* t, const float* weights, int B, int H, int W,
                       double* loss, float* grad_host, void* stream) {
    if (!net || !x || !t || B < 1 || H < 1 || W < 1) return ASDSM_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = forward_impl(net, x, nullptr, B, H, W, st)) return rc;
    const long long pix = (long long)B * H * W;
    const long long ntiles = (long long)B * ((H + TILE - 1) / TILE) * ((W + TILE - 1) / TILE);
    dim3 grid((W + TILE - 1) / TILE, (H + TILE - 1) / TILE, B);
    // dL/dz_4 and the loss.
    const int nb = 512;
    mse_kernel<<<nb, 256, 0, st>>>(net->act[CNN_LAYERS], t, weights, pix, net->dz[0], net->dpart);
    asdsm::note_launch();
    CNN_CK(cudaGetLastError());
    int cur = 0;
    for (int l = CNN_LAYERS - 1; l >= 0; --l) {
        const int cin = CNN_CH[l], cout = CNN_CH[l + 1];
        const float* a_in = l == 0 ? x : net->act[l];
        const size_t smem = sizeof(float) * ((size_t)cout * TILE * TILE + (size_t)cin * (TILE + 2) * (TILE + 2));
        CNN_CK(cudaFuncSetAttribute(conv_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        conv_wgrad_kernel<<<grid, CONV_THREADS, smem, st>>>(net->dz[cur], cout, a_in, cin, H, W, net->partials, net->bf16);
        asdsm::note_launch();
        CNN_CK(cudaGetLastError());
        const int nw = layer_w(l) + cout;
        sum_partials_kernel<<<(nw + 255) / 256, 256, 0, st>>>(net->partials, ntiles, nw, net->grad + layer_off(l));
        asdsm::note_launch();
        CNN_CK(cudaGetLastError());
        if (l == 0) break;
        // dz_l = conv(dz_{l+1}; W_{l+1} flipped and transposed) * (a_l > 0)
        flip_transpose_kernel<<<36, 256, 0, st>>>(net->theta + layer_off(l), cout, cin, net->wt);
        asdsm::note_launch();
        CNN_CK(cudaGetLastError());
        CNN_CK(conv(net->dz[cur], cout, cin, net->wt, nullptr, net->dz[1 - cur], B, H, W, 0, net->act[l], net->bf16, st));
        cur = 1 - cur;
    }
    if (loss) {
        CNN_CK(cudaMemcpyAsync(net->hpart, net->dpart, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        CNN_CK(cudaStreamSynchronize(st));
        double s = 0.0;
        for (int q = 0; q < nb; ++q) s += net->hpart[q];
        *loss = 0.5 * s / (double)pix;
    }
    if (grad_host) {
        CNN_CK(cudaMemcpyAsync(grad_host, net->grad, (size_t)CNN_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, st));
        CNN_CK(cudaStreamSynchronize(st));
    }
    return ASDSM_OK;
}

int asdsm_cnn_adam(asdsm_cnn* net, float lr, void* stream) {
    if (!net || !(lr > 0.0f)) return ASDSM_ERR_INVALID;
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - std::pow(b1, (float)net->step), c2 = 1.0f - std::pow(b2, (float)net->step);
    adam_kernel<<<(CNN_PARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(net->theta, net->grad, net->m, net->v,
                                                                            CNN_PARAMS, lr, b1, b2, eps, c1, c2);
    asdsm::note_launch();
    CNN_CK(cudaGetLastError());
    return ASDSM_OK;
}

const char* asdsm_cnn_last_error(void) { return g_cnn_error.c_str(); }

void asdsm_cnn_destroy(asdsm_cnn* net) {
    if (!net) return;
    auto fr = [](void* p) { if (p) cudaFree(p); };
    fr(net->theta); fr(net->grad); fr(net->m); fr(net->v); fr(net->wt);
    for (int l = 0; l <= CNN_LAYERS; ++l) fr(net->act[l]);
    fr(net->dz[0]); fr(net->dz[1]); fr(net->partials); fr(net->dpart);
    if (net->hpart) cudaFreeHost(net->hpart);
    delete net;
}

}  // extern "C"
