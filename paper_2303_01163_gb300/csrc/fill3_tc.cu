// fill3_tc.cu: the homogeneous cube-hole Filler of the 3D sweeps (Algorithm 3
// with zero source, Section 3.5) on the tensor cores.
//
// For zero source the hole values are a fixed linear map of the hole's face
// values: v = G f with G = -A_hh^{-1} A_hs (C^3 x 6 C^2, C = n - 1), the same
// for every hole.  For all H holes at once this is the GEMM
//     Out[h][p] = sum_k F[h][k] G[p][k],
// M = holes, N = hole points, K = face values, on tcgen05 (kind::tf32) with
// both operands split as x ~ hi + lo (both rounded to nearest TF32,
// |x - hi - lo| <= 2^-22 |x|) and three products per term (lo*hi, hi*lo,
// hi*hi), accumulated in FP32 in tensor memory.
//
// Both operands are stored as images of the shared-memory layout the MMAs
// read (tc_common.cuh: K-major, 128-byte swizzle, 128 rows x 32 values per
// block): G^T once on the host, the faces of every sweep by faces3_tc_kernel,
// which gathers, splits and writes them in place.  The GEMM kernel then only
// bulk-copies blocks through a 3-stage ring (one thread), issues the MMAs (one
// thread) and writes the 128 x 128 tile of hole values into the grid (four
// warps, through shared memory so that each hole's points are written along x).
// Every mbarrier wait is bounded; on a timeout the kernel sets *err and returns.
#include "asdsm_internal.h"
#include "fill3_tc.h"
#include "tc_common.cuh"
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>

namespace asdsm {

namespace {

using namespace tc;

constexpr int F3_ROWS = 128, F3_COLS = 128, F3_STAGES = 3;
constexpr int F3_BLK = 128 * kRowBytes;              // one 128-row x 32-value swizzled block (16 KB)
constexpr int F3_STAGE = 4 * F3_BLK;                 // A hi, A lo, B hi, B lo
constexpr int F3_SMEM = F3_STAGES * F3_STAGE + 1024; // + alignment slack
constexpr int F3_SROW = F3_COLS + 1;                 // epilogue staging row stride (floats)
// Warps: 0 issues the MMAs (and holds the tensor memory), 1 copies the blocks,
// 2..5 run the epilogue (tensor-memory lane quarter = warp mod 4).
constexpr int F3_EPI0 = 2, F3_THREADS = 32 * (F3_EPI0 + 4), F3_EPI = 128;
constexpr uint32_t F3_TMEM_COLS = F3_COLS;
constexpr uint32_t kF3Idesc = idesc_tf32(F3_ROWS, F3_COLS);
static_assert(F3_ROWS * F3_SROW * 4 <= F3_STAGES * F3_STAGE, "the epilogue tile fits the ring");

// Block index of (row tile, K chunk, split) in an operand image.
__host__ __device__ __forceinline__ size_t f3_block(int tile, int kc, int split, int KC) {
    return ((size_t)tile * KC + kc) * 2 + split;
}

__device__ __forceinline__ void f3_epi_barrier() {
    __syncwarp();
    asm volatile("barrier.sync 1, %0;" ::"n"(F3_EPI) : "memory");
    __syncwarp();
}

// Origin (x0, y0, z0) of hole h (holes x fastest, then y, then z).
__device__ __forceinline__ void f3_hole_origin(int h, int mc, int n, int& x0, int& y0, int& z0) {
    x0 = (h % mc) * n;
    y0 = ((h / mc) % mc) * n;
    z0 = (h / (mc * mc)) * n;
}

// Face value k of hole h as the A image: faces west, east (x = 0, C + 1),
// south, north, down, up, each C x C with its second axis slowest; k fastest
// across the threads, so that a 128-byte image row is written by 32 threads.
__global__ void faces3_tc_kernel(Fill3TcArgs a) {
    const int C = a.hc, C2 = C * C, N = a.N, n = a.n;
    const long long total = (long long)a.H * a.K;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int h = (int)(e / a.K), k = (int)(e % a.K);
        const int face = k / C2, r = k % C2, u = r % C + 1, v = r / C + 1;
        int x0, y0, z0;
        f3_hole_origin(h, a.mc, n, x0, y0, z0);
        int x, y, zz;
        if (face < 2) { x = x0 + (face == 0 ? 0 : n); y = y0 + u; zz = z0 + v; }
        else if (face < 4) { y = y0 + (face == 2 ? 0 : n); x = x0 + u; zz = z0 + v; }
        else { zz = z0 + (face == 4 ? 0 : n); x = x0 + u; y = y0 + v; }
        const float val = a.z[((long long)zz * N + y) * N + x];
        float hi, lo;
        tf32_split(val, hi, lo);
        unsigned char* img = reinterpret_cast<unsigned char*>(a.aimg);
        const int off = swz_offset(h % F3_ROWS, k % 32);
        *reinterpret_cast<float*>(img + f3_block(h / F3_ROWS, k / 32, 0, a.KC) * F3_BLK + off) = hi;
        *reinterpret_cast<float*>(img + f3_block(h / F3_ROWS, k / 32, 1, a.KC) * F3_BLK + off) = lo;
    }
}

// One 128-hole x 128-point tile: Out[h][p] = sum over K chunks of the
// A block (holes x 32 face values) times the B block (points x 32 face values).
__global__ void __launch_bounds__(F3_THREADS, 1) fill3_tc_kernel(Fill3TcArgs a) {
    extern __shared__ unsigned char f3_raw[];
    __shared__ __align__(8) uint64_t full[F3_STAGES], mdone[F3_STAGES], tdone;
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    const uint32_t raw = smem_u32(f3_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    unsigned char* pbase = f3_raw + (sbase - raw);
    const int pt = blockIdx.x, ht = blockIdx.y, KC = a.KC;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort_v = &abort_flag;
    if (tid == 0) {
        for (int q = 0; q < F3_STAGES; ++q) {
            mbar_init(smem_u32(&full[q]), 1);
            mbar_init(smem_u32(&mdone[q]), 1);
        }
        mbar_init(smem_u32(&tdone), 1);
        abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_holder), F3_TMEM_COLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = tmem_holder;
    if (warp == 1) {
        // Blocks of chunk q into stage q mod 3, once the MMAs of chunk q - 3 completed.
        if (lane == 0) {
            const unsigned char* A = reinterpret_cast<const unsigned char*>(a.aimg);
            const unsigned char* B = reinterpret_cast<const unsigned char*>(a.gimg);
            for (int q = 0; q < KC; ++q) {
                const int st = q % F3_STAGES;
                if (q >= F3_STAGES &&
                    !mbar_wait_abortable(smem_u32(&mdone[st]), (uint32_t)(q / F3_STAGES - 1) & 1u, abort_v)) {
                    *abort_v = 1;
                    break;
                }
                const uint32_t dst = sbase + (uint32_t)(st * F3_STAGE);
                const uint32_t bar = smem_u32(&full[st]);
                mbar_expect_tx(bar, F3_STAGE);
                bulk_g2s(dst, A + f3_block(ht, q, 0, KC) * F3_BLK, F3_BLK, bar);
                bulk_g2s(dst + F3_BLK, A + f3_block(ht, q, 1, KC) * F3_BLK, F3_BLK, bar);
                bulk_g2s(dst + 2 * F3_BLK, B + f3_block(pt, q, 0, KC) * F3_BLK, F3_BLK, bar);
                bulk_g2s(dst + 3 * F3_BLK, B + f3_block(pt, q, 1, KC) * F3_BLK, F3_BLK, bar);
            }
        }
    } else if (warp == 0) {
        // MMA issuer: 4 K-steps x 3 split products per chunk into tensor memory.
        if (lane == 0) {
            bool ok = true;
            for (int q = 0; q < KC; ++q) {
                const int st = q % F3_STAGES;
                if (!mbar_wait_abortable(smem_u32(&full[st]), (uint32_t)(q / F3_STAGES) & 1u, abort_v)) {
                    *abort_v = 1;
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t a0 = sbase + (uint32_t)(st * F3_STAGE), b0 = a0 + 2 * F3_BLK;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t ko = (uint32_t)(ks * 32);
                    const uint64_t aHi = sw128_desc(a0 + ko), aLo = sw128_desc(a0 + F3_BLK + ko);
                    const uint64_t bHi = sw128_desc(b0 + ko), bLo = sw128_desc(b0 + F3_BLK + ko);
                    tc_mma(tbase, aLo, bHi, kF3Idesc, (q > 0 || ks > 0) ? 1u : 0u);   // small terms first
                    tc_mma(tbase, aHi, bLo, kF3Idesc, 1u);
                    tc_mma(tbase, aHi, bHi, kF3Idesc, 1u);
                }
                tc_commit(smem_u32(&mdone[st]));
            }
            // One more commit on a barrier of its own: it completes when every MMA did.
            if (ok) tc_commit(smem_u32(&tdone));
        }
    } else {
        // Epilogue warps: wait for the tile, stage it in the free ring, write it.
        const int pw = warp & 3;                 // tensor-memory lane quarter: tile rows 32 pw .. + 31
        const bool ok = mbar_wait_abortable(smem_u32(&tdone), 0u, abort_v);
        if (!ok) *abort_v = 1;
        f3_epi_barrier();                        // abort flag final for the epilogue warps
        const bool go = *abort_v == 0;
        float* S = reinterpret_cast<float*>(pbase);
        if (go) {
            fence_after_sync();
            const int r = pw * 32 + lane;
#pragma unroll
            for (int jb = 0; jb < F3_COLS / 32; ++jb) {
                uint32_t v[32];
                tmem_ld32(tbase + ((uint32_t)(pw * 32) << 16) + (uint32_t)(jb * 32), v);
#pragma unroll
                for (int c = 0; c < 32; ++c) S[r * F3_SROW + jb * 32 + c] = __uint_as_float(v[c]);
            }
        }
        f3_epi_barrier();
        if (go) {
            // Warp w writes holes w, w + 4, ...: a hole's points p (x fastest) along the lanes.
            const int C = a.hc, C2 = C * C, N = a.N, n = a.n;
            const int ew = warp - F3_EPI0;
            for (int r = ew; r < F3_ROWS; r += 4) {
                const int h = ht * F3_ROWS + r;
                if (h >= a.H) break;
                int x0, y0, z0;
                f3_hole_origin(h, a.mc, n, x0, y0, z0);
#pragma unroll
                for (int m = 0; m < F3_COLS / 32; ++m) {
                    const int c = m * 32 + lane, p = pt * F3_COLS + c;
                    if (p < a.P) {
                        const int x = x0 + 1 + p % C, y = y0 + 1 + (p / C) % C, zz = z0 + 1 + p / C2;
                        a.zout[((long long)zz * N + y) * N + x] = S[r * F3_SROW + c];
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (tid == 0 && abort_flag && a.err) atomicExch(a.err, 1);
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(tbase, F3_TMEM_COLS);
    }
}

}  // namespace

size_t fill3_tc_image_floats(int rows, int K) {
    const int tiles = (rows + F3_ROWS - 1) / F3_ROWS, KC = (K + 31) / 32;
    return (size_t)tiles * KC * 2 * (F3_BLK / sizeof(float));
}

void fill3_tc_gimage(const std::vector<double>& G, int P, int K, std::vector<float>* img) {
    const int KC = (K + 31) / 32;
    img->assign(fill3_tc_image_floats(P, K), 0.0f);
    unsigned char* base = reinterpret_cast<unsigned char*>(img->data());
    for (int p = 0; p < P; ++p)
        for (int k = 0; k < K; ++k) {
            const double v = G[(size_t)p * K + k];
            const float hi = tf32_rn((float)v);
            const float lo = tf32_rn((float)(v - (double)hi));
            const int off = swz_offset(p % F3_ROWS, k % 32);
            std::memcpy(base + f3_block(p / F3_ROWS, k / 32, 0, KC) * F3_BLK + off, &hi, 4);
            std::memcpy(base + f3_block(p / F3_ROWS, k / 32, 1, KC) * F3_BLK + off, &lo, 4);
        }
}

cudaError_t fill3_tc(const Fill3TcArgs& a, cudaStream_t st) {
    if (!a.z || !a.zout || !a.gimg || !a.aimg || a.hc < 1 || a.KC != (a.K + 31) / 32 ||
        a.PT != (a.P + F3_COLS - 1) / F3_COLS || a.HT != (a.H + F3_ROWS - 1) / F3_ROWS)
        return cudaErrorInvalidValue;
    if (((reinterpret_cast<uintptr_t>(a.gimg) | reinterpret_cast<uintptr_t>(a.aimg)) & 15u) != 0)
        return cudaErrorInvalidValue;
    const long long total = (long long)a.H * a.K;
    const unsigned gb = (unsigned)((total + 255) / 256 < 152LL * 16 ? (total + 255) / 256 : 152LL * 16);
    faces3_tc_kernel<<<gb, 256, 0, st>>>(a);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static bool attr_set = false;            // setting it twice is harmless
    if (!attr_set) {
        e = cudaFuncSetAttribute(fill3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, F3_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    fill3_tc_kernel<<<dim3(a.PT, a.HT), F3_THREADS, F3_SMEM, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace asdsm
