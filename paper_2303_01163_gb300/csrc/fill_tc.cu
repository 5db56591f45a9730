// fill_tc.cu: the Filler of Algorithm 3 in its homogeneous form (zero source,
// the form every sweep of Algorithm 4 uses) for holes of 15 x 15 points, as a
// tensor-core GEMM.
//
// The hole values are a fixed linear map of the 60 ring values around the hole
// (Remark 2.4: every hole block A_(ij) is the same matrix): v = G z with
// G = -A_hh^{-1} A_hs, precomputed in FP64 on the host.  For a tile of 64
// holes of one hole row,
//     D[p][h] = sum_k G[p][k] * Z[h][k],   p < 240 output points, k < 64,
// with p = 16 (y - 1) + x (x = 0 is the skeleton column left of the hole and
// its row of G is zero), k the ring index (west, east, south, north, 15 each,
// then 4 zeros).  G (the A operand, 256 x 64) stays resident in shared memory
// for all tiles of a persistent CTA; Z (the B operand, 64 holes x 64) is
// gathered from the grid per tile.  Both are stored K-major in the 128-byte
// swizzled canonical layout; D lives in tensor memory (2 x 64 columns).
//
// Warps: 8..11 gather the ring values of a tile into one of two B stages, one
// thread of warp 12 issues the tile's MMAs into one of two tensor-memory
// buffers, warps 0..7 store the previous tile (warp w reads tensor-memory lane
// quarter w mod 4, holes 32 (w / 4) .. + 31 of the tile): gather, MMA and
// stores of consecutive tiles overlap, handed over by mbarriers.  With the
// line values given apart (FillTcArgs::zv), warp 13 copies them into the grid
// (the skeleton column of every hole row), so that each row is written whole.
//
// Precision: FP32 results from TF32 tensor-core products by splitting both
// operands, x ~ hi + lo with hi and lo = x - hi both rounded to nearest TF32
// (|x - hi - lo| <= 2^-22 |x|): G z ~ G_lo z_hi + G_hi z_lo + G_hi z_hi (the
// G_lo z_lo term is of the same order), accumulated in FP32 in tensor memory.
//
// Every wait on an mbarrier is bounded (1 s by %globaltimer); on a timeout the
// kernel sets *err, stops, and frees its tensor memory.
#include "asdsm_internal.h"
#include "tc_common.cuh"
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>
#include <cmath>
#include <type_traits>

namespace asdsm {

namespace {

constexpr int TC_C = kFillTcN - 1;                     // 15 points per hole side
constexpr int TC_RING = 4 * TC_C;                      // 60 ring values
constexpr int TC_HOLES = 64;                           // MMA N: holes per tile
constexpr int TC_K = 64;                               // ring values padded to 8 K-steps of 8
constexpr int TC_MT = 2;                               // 128-row M tiles over 240 output points
constexpr int TC_P = TC_C * kFillTcN;                  // 240
constexpr int TC_BLK = 128 * 128;                      // one 128-row x 128-byte K block (A)
constexpr int TC_BBLK = TC_HOLES * 128;                // one 64-row x 128-byte K block (B)
constexpr int TC_A_BYTES = 2 * TC_MT * 2 * TC_BLK;     // [hi/lo][mt][kb] = 128 KB
constexpr int TC_B_STAGE = 2 * 2 * TC_BBLK;            // [hi/lo][kb] = 32 KB
constexpr int TC_SMEM = TC_A_BYTES + 2 * TC_B_STAGE + 1024;  // + alignment slack
constexpr int TC_EPI_WARPS = 8, TC_PROD_WARPS = 4;
constexpr int TC_MMA_WARP = TC_EPI_WARPS + TC_PROD_WARPS;
constexpr int TC_COPY_WARP = TC_MMA_WARP + 1;
constexpr int TC_THREADS = 32 * (TC_COPY_WARP + 1);
constexpr uint32_t TC_TMEM_COLS = 2 * TC_MT * TC_HOLES;  // 2 buffers x 2 M tiles x 64 = 256

// Byte offset of element (row r, k) inside one [mt] image of 2 K blocks:
// rows 128 bytes apart, 16-byte chunks XOR-swizzled by r mod 8.
__host__ __device__ __forceinline__ int tc_offset(int r, int k) {
    return (k >> 5) * TC_BLK + tc::swz_offset(r, k & 31);
}

constexpr uint32_t kTcIdesc = tc::idesc_tf32(128, TC_HOLES);

using namespace tc;

__global__ void __launch_bounds__(TC_THREADS, 1) fill_tc_kernel(FillTcArgs a) {
    extern __shared__ unsigned char tc_raw[];
    // bar_g: G landed; bfull/bempty: B stages; tfull/tempty: tensor-memory buffers.
    __shared__ __align__(8) uint64_t bar_g, bfull[2], bempty[2], tfull[2], tempty[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    const uint32_t raw = smem_u32(tc_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    unsigned char* pB = tc_raw + (sbase - raw) + TC_A_BYTES;
    const uint32_t sA = sbase, sB = sbase + TC_A_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort_v = &abort_flag;
    if (tid == 0) {
        mbar_init(smem_u32(&bar_g), 1);
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&bfull[q]), 32 * TC_PROD_WARPS);
            mbar_init(smem_u32(&bempty[q]), 1);
            mbar_init(smem_u32(&tfull[q]), 1);
            mbar_init(smem_u32(&tempty[q]), 32 * TC_EPI_WARPS);
        }
        abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_holder), TC_TMEM_COLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = tmem_holder;
    const int N = a.N, mc = a.mc;
    const int per_row = (mc + TC_HOLES - 1) / TC_HOLES;
    const int ntiles = mc * per_row;
    if (warp == TC_MMA_WARP) {
        if (lane == 0) {
            // The A operand (G, hi and lo) by bulk copies into the swizzled image.
            mbar_expect_tx(smem_u32(&bar_g), TC_A_BYTES);
            const unsigned char* src = reinterpret_cast<const unsigned char*>(a.gimg);
            for (int c = 0; c < TC_A_BYTES / TC_BLK; ++c)
                bulk_g2s(sA + c * TC_BLK, src + (size_t)c * TC_BLK, TC_BLK, smem_u32(&bar_g));
            bool ok = mbar_wait_abortable(smem_u32(&bar_g), 0, abort_v);
            int it = 0;
            for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++it) {
                const int st = it & 1;
                const uint32_t ph = (uint32_t)(it >> 1) & 1u;
                if (!mbar_wait_abortable(smem_u32(&bfull[st]), ph, abort_v) ||
                    (it >= 2 && !mbar_wait_abortable(smem_u32(&tempty[st]), ph ^ 1u, abort_v))) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t sb = sB + (uint32_t)(st * TC_B_STAGE);
#pragma unroll
                for (int mt = 0; mt < TC_MT; ++mt) {
                    const uint32_t d = tbase + (uint32_t)((st * TC_MT + mt) * TC_HOLES);
#pragma unroll
                    for (int ks = 0; ks < TC_K / 8; ++ks) {
                        const uint32_t kb = (uint32_t)(ks >> 2), ko = (uint32_t)((ks & 3) * 32);
                        const uint64_t aHi = sw128_desc(sA + (uint32_t)(((0 * TC_MT + mt) * 2 + kb) * TC_BLK) + ko);
                        const uint64_t aLo = sw128_desc(sA + (uint32_t)(((1 * TC_MT + mt) * 2 + kb) * TC_BLK) + ko);
                        const uint64_t bHi = sw128_desc(sb + kb * TC_BBLK + ko);
                        const uint64_t bLo = sw128_desc(sb + (2 + kb) * TC_BBLK + ko);
                        tc_mma(d, aLo, bHi, kTcIdesc, ks > 0 ? 1u : 0u);    // small terms first
                        tc_mma(d, aHi, bLo, kTcIdesc, 1u);
                        tc_mma(d, aHi, bHi, kTcIdesc, 1u);
                    }
                }
                tc_commit(smem_u32(&tfull[st]));
                tc_commit(smem_u32(&bempty[st]));
            }
            if (!ok) *abort_v = 1;
        }
    } else if (warp == TC_COPY_WARP) {
        // The line values of the tile's hole rows (x = bi n, rows 1..15 of the
        // hole row), zv -> z; lanes run over consecutive holes.
        // All 30 loads of a lane are issued before its stores.
        constexpr int PER_LANE = TC_C * TC_HOLES / 32;
        if (a.zv) {
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
                const int bj = tile / per_row, bi0 = (tile % per_row) * TC_HOLES;
                float vals[PER_LANE];
#pragma unroll
                for (int t = 0; t < PER_LANE; ++t) {
                    const int e = lane + 32 * t;
                    const int i = e / TC_HOLES, bi = bi0 + e % TC_HOLES;
                    const long long row = (long long)bj * kFillTcN + 1 + i;
                    vals[t] = bi < mc ? a.zv[row * (mc + 1) + bi] : 0.0f;
                }
#pragma unroll
                for (int t = 0; t < PER_LANE; ++t) {
                    const int e = lane + 32 * t;
                    const int i = e / TC_HOLES, bi = bi0 + e % TC_HOLES;
                    const long long row = (long long)bj * kFillTcN + 1 + i;
                    if (bi < mc) a.z[row * N + (long long)bi * kFillTcN] = vals[t];
                }
            }
        }
    } else if (warp >= TC_EPI_WARPS) {
        // Producers: thread p gathers half of the ring of hole p mod 64 (k < 32
        // or k >= 32), splits it, stores it swizzled into the tile's B stage.
        const int p = tid - 32 * TC_EPI_WARPS;
        const int h = p & (TC_HOLES - 1), half = p >> 6;
        float zr[32];
        // Ring value k (compile-time per half) of this thread's hole in the
        // given tile: west, east, south, north.
        auto gather = [&](int tile, auto half_c) {
            constexpr int H = decltype(half_c)::value;
            const int bj = tile / per_row, bi = (tile % per_row) * TC_HOLES + h;
            const bool valid = bi < mc;
            const long long x0 = (long long)bi * kFillTcN, y0 = (long long)bj * kFillTcN;
#pragma unroll
            for (int kk = 0; kk < 32; ++kk) {
                const int k = H * 32 + kk;
                float v = 0.f;
                if (valid && k < TC_RING) {
                    const int side = k / TC_C, i = k % TC_C;
                    if (side < 2 && a.zv) {
                        v = a.zv[(y0 + 1 + i) * (mc + 1) + bi + side];               // west, east
                    } else {
                        long long idx;
                        if (side == 0) idx = (y0 + 1 + i) * N + x0;                  // west
                        else if (side == 1) idx = (y0 + 1 + i) * N + x0 + kFillTcN;  // east
                        else if (side == 2) idx = y0 * N + x0 + 1 + i;               // south
                        else idx = (y0 + kFillTcN) * N + x0 + 1 + i;                 // north
                        v = a.z[idx];
                    }
                }
                zr[kk] = v;
            }
        };
        auto load_tile = [&](int tile) {
            if (half == 0) gather(tile, std::integral_constant<int, 0>{});
            else gather(tile, std::integral_constant<int, 1>{});
        };
        int it = 0;
        bool ok = true;
        if ((int)blockIdx.x < ntiles) load_tile(blockIdx.x);
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int st = it & 1;
            if (it >= 2 && !mbar_wait_abortable(smem_u32(&bempty[st]), (uint32_t)((it >> 1) - 1) & 1u, abort_v)) {
                ok = false;
                break;
            }
            unsigned char* pb = pB + st * TC_B_STAGE;
#pragma unroll
            for (int kk = 0; kk < 32; ++kk) {
                float hi, lo;
                tf32_split(zr[kk], hi, lo);
                const int off = half * TC_BBLK + swz_offset(h, kk);
                *reinterpret_cast<float*>(pb + off) = hi;
                *reinterpret_cast<float*>(pb + 2 * TC_BBLK + off) = lo;
            }
            fence_async_smem();
            mbar_arrive(smem_u32(&bfull[st]));
            // The next tile's ring values are in flight while this one is multiplied.
            if (tile + (int)gridDim.x < ntiles) load_tile(tile + gridDim.x);
        }
        if (!ok) *abort_v = 1;
    } else {
        // Epilogue: warp w reads tensor-memory lanes 32 (w mod 4) .. + 31 =
        // output points for holes 32 (w / 4) .. + 31; a store instruction
        // writes one hole's two rows of 16 points.
        int it = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int st = it & 1;
            ok = mbar_wait_abortable(smem_u32(&tfull[st]), (uint32_t)(it >> 1) & 1u, abort_v);
            if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
            fence_after_sync();
            const int bj = tile / per_row, bi0 = (tile % per_row) * TC_HOLES;
            const int q4 = warp & 3, j = warp >> 2;
#pragma unroll
            for (int mt = 0; mt < TC_MT; ++mt) {
                const int pt = mt * 128 + q4 * 32 + lane;
                const int y = pt >> 4, x = pt & 15;
                const bool pv = pt < TC_P && x != 0;     // x = 0: the skeleton column (not a hole point)
                const long long rowx = ((long long)bj * kFillTcN + y + 1) * N + x;
                {
                    uint32_t v[32];
                    tmem_ld32(tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)((st * TC_MT + mt) * TC_HOLES + j * 32), v);
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
            mbar_arrive(smem_u32(&tempty[st]));
        }
        if (!ok) *abort_v = 1;
    }
    fence_before_sync();
    __syncthreads();
    if (tid == 0 && abort_flag) atomicExch(a.err, 1);
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(tbase, TC_TMEM_COLS);
    }
}

// Self-test of the failure path of the tensor-core kernels: one CTA takes
// tensor memory as they do, then thread 0 waits on an mbarrier that no thread
// arrives at, with no bulk copy and no MMA in flight.  The bounded wait gives
// up after limit_ns; the kernel then sets *err and frees its tensor memory,
// which is what a tensor-core kernel does when one of its hand-overs stalls.
__global__ void __launch_bounds__(64) wait_selftest_kernel(int* err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_holder;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        mbar_init_fence();
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_holder), 32);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = tmem_holder;
    if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0, limit_ns)) atomicExch(err, 1);
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(tbase, 32);
    }
}

}  // namespace

cudaError_t wait_selftest(int* err, long long limit_ns, cudaStream_t st) {
    wait_selftest_kernel<<<1, 64, 0, st>>>(err, (unsigned long long)limit_ns);
    note_launch();
    return cudaGetLastError();
}

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
                const float hi = tc::tf32_rn((float)gv);
                const float lo = tc::tf32_rn((float)(gv - (double)hi));
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
