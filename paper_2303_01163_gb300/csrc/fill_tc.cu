// fill_tc.cu: the Filler of Algorithm 3 in its homogeneous form (zero source,
// the form every sweep of Algorithm 4 uses) for holes of 15 x 15 points, as a
// tensor-core GEMM.
//
// The hole values are a fixed linear map of the 60 ring values around the hole
// (Remark 2.4: every hole block A_(ij) is the same matrix): v = G z with
// G = -A_hh^{-1} A_hs, precomputed in FP64 on the host.  For a tile of 128
// holes of one hole row,
//     D[p][h] = sum_k G[p][k] * Z[h][k],   p < 240 output points, k < 64,
// with p = 16 (y - 1) + x (x = 0 is the skeleton column left of the hole and
// its row of G is zero), k the ring index (west, east, south, north, 15 each,
// then 4 zeros).  G (the A operand, 256 x 64) stays resident in shared memory
// for all tiles of a persistent CTA; Z (the B operand, 128 holes x 64) is
// gathered from the grid per tile.  Both are stored K-major in the 128-byte
// swizzled canonical layout; D lives in tensor memory (2 x 128 columns).
//
// Precision: FP32 results from TF32 tensor-core products by splitting both
// operands, x = hi + lo with hi = x with its 13 low mantissa bits cleared:
// G z ~ G_lo z_hi + G_hi z_lo + G_hi z_hi (the G_lo z_lo term is ~2^-22
// relative), accumulated in FP32 in tensor memory.
//
// Every wait on an mbarrier is bounded (1 s by %globaltimer); on a timeout the
// kernel sets *err, stops, and frees its tensor memory.
#include "asdsm_internal.h"
#include "tc_common.cuh"
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>
#include <cmath>

namespace asdsm {

namespace {

constexpr int TC_C = kFillTcN - 1;                     // 15 points per hole side
constexpr int TC_RING = 4 * TC_C;                      // 60 ring values
constexpr int TC_HOLES = 128;                          // MMA N: holes per tile
constexpr int TC_K = 64;                               // ring values padded to 8 K-steps of 8
constexpr int TC_MT = 2;                               // 128-row M tiles over 240 output points
constexpr int TC_P = TC_C * kFillTcN;                  // 240
constexpr int TC_THREADS = 128;
constexpr int TC_BLK = 128 * 128;                      // one 128-row x 128-byte K block
constexpr int TC_A_BYTES = 2 * TC_MT * 2 * TC_BLK;     // [hi/lo][mt][kb] = 128 KB
constexpr int TC_B_BYTES = 2 * 2 * TC_BLK;             // [hi/lo][kb] = 64 KB
constexpr int TC_SMEM = TC_A_BYTES + TC_B_BYTES + 1024;  // + alignment slack
constexpr uint32_t TC_TMEM_COLS = 2 * TC_HOLES;        // 256

// Byte offset of element (row r, k) inside one [mt] image of 2 K blocks:
// rows 128 bytes apart, 16-byte chunks XOR-swizzled by r mod 8.
__host__ __device__ __forceinline__ int tc_offset(int r, int k) {
    return (k >> 5) * TC_BLK + tc::swz_offset(r, k & 31);
}

constexpr uint32_t kTcIdesc128 = tc::idesc_tf32(128, TC_HOLES);

using namespace tc;

__global__ void __launch_bounds__(TC_THREADS, 1) fill_tc_kernel(FillTcArgs a) {
    extern __shared__ unsigned char tc_raw[];
    __shared__ __align__(8) uint64_t bars[2];      // 0: G image landed, 1: MMAs of the tile done
    __shared__ uint32_t tmem_holder;
    const uint32_t raw = smem_u32(tc_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    unsigned char* pB = tc_raw + (sbase - raw) + TC_A_BYTES;
    const uint32_t sA = sbase, sB = sbase + TC_A_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_g = smem_u32(&bars[0]), bar_m = smem_u32(&bars[1]);
    if (tid == 0) {
        mbar_init(bar_g, 1);
        mbar_init(bar_m, 1);
        mbar_init_fence();
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_holder), TC_TMEM_COLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = tmem_holder;
    // The A operand (G, hi and lo) by bulk copies into the swizzled image.
    if (tid == 0) {
        mbar_expect_tx(bar_g, TC_A_BYTES);
        const unsigned char* src = reinterpret_cast<const unsigned char*>(a.gimg);
        for (int c = 0; c < TC_A_BYTES / TC_BLK; ++c) bulk_g2s(sA + c * TC_BLK, src + (size_t)c * TC_BLK, TC_BLK, bar_g);
    }
    bool ok = __syncthreads_and(mbar_wait(bar_g, 0)) != 0;
    const int N = a.N, mc = a.mc;
    const int per_row = (mc + TC_HOLES - 1) / TC_HOLES;
    const int ntiles = mc * per_row;
    uint32_t phase = 0;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int bj = tile / per_row, bi0 = (tile % per_row) * TC_HOLES;
        // B operand: row tid = hole bi0 + tid, its ring values split hi / lo.
        {
            const int bi = bi0 + tid;
            const bool valid = bi < mc;
            const long long x0 = (long long)bi * kFillTcN, y0 = (long long)bj * kFillTcN;
            float zr[TC_RING];
#pragma unroll
            for (int i = 0; i < TC_C; ++i) {
                zr[i] = valid ? a.z[(y0 + 1 + i) * N + x0] : 0.f;                          // west
                zr[TC_C + i] = valid ? a.z[(y0 + 1 + i) * N + x0 + kFillTcN] : 0.f;        // east
                zr[2 * TC_C + i] = valid ? a.z[y0 * N + x0 + 1 + i] : 0.f;                 // south
                zr[3 * TC_C + i] = valid ? a.z[(y0 + kFillTcN) * N + x0 + 1 + i] : 0.f;    // north
            }
#pragma unroll
            for (int k = 0; k < TC_K; ++k) {
                const float v = k < TC_RING ? zr[k] : 0.f;
                const float hi = tc::tf32_hi(v);
                const int off = tc_offset(tid, k);
                *reinterpret_cast<float*>(pB + off) = hi;
                *reinterpret_cast<float*>(pB + 2 * TC_BLK + off) = v - hi;
            }
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
#pragma unroll
            for (int mt = 0; mt < TC_MT; ++mt) {
                const uint32_t d = tbase + (uint32_t)(mt * TC_HOLES);
#pragma unroll
                for (int ks = 0; ks < TC_K / 8; ++ks) {
                    const uint32_t koff = (uint32_t)((ks >> 2) * TC_BLK + (ks & 3) * 32);
                    const uint64_t aHi = sw128_desc(sA + (uint32_t)((0 * TC_MT + mt) * 2 * TC_BLK) + koff);
                    const uint64_t aLo = sw128_desc(sA + (uint32_t)((1 * TC_MT + mt) * 2 * TC_BLK) + koff);
                    const uint64_t bHi = sw128_desc(sB + koff);
                    const uint64_t bLo = sw128_desc(sB + 2 * TC_BLK + koff);
                    tc_mma(d, aLo, bHi, kTcIdesc128, ks > 0 ? 1u : 0u);    // small terms first
                    tc_mma(d, aHi, bLo, kTcIdesc128, 1u);
                    tc_mma(d, aHi, bHi, kTcIdesc128, 1u);
                }
            }
            tc_commit(bar_m);
        }
        const bool done = mbar_wait(bar_m, phase);
        phase ^= 1u;
        if (!__syncthreads_and(done)) { ok = false; break; }
        fence_after_sync();
        // Epilogue: warp w reads TMEM lanes 32w..32w+31 = output points; a
        // store instruction writes one hole's two rows of 16 points.
#pragma unroll
        for (int mt = 0; mt < TC_MT; ++mt) {
            const int p = mt * 128 + warp * 32 + lane;
            const int y = p >> 4, x = p & 15;
            const bool pv = p < TC_P && x != 0;
            const long long rowx = ((long long)bj * kFillTcN + y + 1) * N + x;
#pragma unroll
            for (int j = 0; j < TC_HOLES / 32; ++j) {
                uint32_t v[32];
                tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * TC_HOLES + j * 32), v);
                if (pv) {
                    const int hb = bi0 + j * 32;
                    const int cnt = mc - hb < 32 ? mc - hb : 32;
                    float* zo = a.z + rowx + (long long)hb * kFillTcN;
                    if (a.out_d) {
                        double* od = a.out_d + rowx + (long long)hb * kFillTcN;
#pragma unroll
                        for (int c = 0; c < 32; ++c)
                            if (c < cnt) od[c * kFillTcN] = (double)__uint_as_float(v[c]);
                    } else if (cnt == 32) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) zo[c * kFillTcN] = __uint_as_float(v[c]);
                    } else {
#pragma unroll
                        for (int c = 0; c < 32; ++c)
                            if (c < cnt) zo[c * kFillTcN] = __uint_as_float(v[c]);
                    }
                }
            }
        }
        fence_before_sync();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(tbase, TC_TMEM_COLS);
    }
}

}  // namespace

size_t fill_tc_image_bytes() { return (size_t)TC_A_BYTES; }

void fill_tc_image(const std::vector<double>& G, std::vector<float>* img) {
    img->assign(TC_A_BYTES / sizeof(float), 0.0f);
    unsigned char* base = reinterpret_cast<unsigned char*>(img->data());
    for (int mt = 0; mt < TC_MT; ++mt)
        for (int r = 0; r < 128; ++r) {
            const int p = mt * 128 + r, y = p >> 4, x = p & 15;
            if (p >= TC_P || x == 0) continue;
            const int hp = y * TC_C + (x - 1);         // hole point (y+1, x) in row-major order
            for (int k = 0; k < TC_RING; ++k) {
                const double gv = G[(size_t)hp * TC_RING + k];
                const float hi = tc::tf32_hi((float)gv);
                const float lo = (float)(gv - (double)hi);
                const int off = tc_offset(r, k);
                std::memcpy(base + (size_t)(0 * TC_MT + mt) * 2 * TC_BLK + off, &hi, 4);
                std::memcpy(base + (size_t)(1 * TC_MT + mt) * 2 * TC_BLK + off, &lo, 4);
            }
        }
}

cudaError_t fill_tc(const FillTcArgs& a, int num_sms, cudaStream_t st) {
    if (!a.gimg || !a.z || !a.err || a.mc < 1 || a.N != a.mc * kFillTcN + 1) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(a.gimg) & 15u) != 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fill_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    const int per_row = (a.mc + TC_HOLES - 1) / TC_HOLES;
    const int ntiles = a.mc * per_row;
    const int grid = ntiles < num_sms ? ntiles : num_sms;
    fill_tc_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace asdsm
