// bcr_tc.cu: one level of the block cyclic reduction of the separable
// submesh systems (eq. 2.4; the factors of every level are shared by all rows,
// host_math.cu) on the tensor cores.
//
// A level is a GEMM over the rows t of the level:
//   forward:   x_i += A_t M_l^T,                A_t = -(wl x_{i-s} + wr x_{i+s}),
//   backward:  y_i  = x_i B_l^{-T} + A_t M_l^T, A_t = -(wl y_{i-s} + wr y_{i+s}),
// with i = 2s(t+1) forward, s(2t+1) backward, s = 2^level (rows outside
// 1..R are zero).  A CTA computes 128 rows x 128 columns of the output in
// tensor memory (FP32), walking the reduction in chunks of 32: per chunk the
// factor block (128 columns x 32, pre-split into TF32 hi / lo and
// pre-swizzled on the host, bulk-copied) and the A block (formed from the
// neighbour rows by four producer warps, split, stored swizzled) pass through
// a 3-stage shared-memory ring, handed over by mbarriers: one thread issues the
// 12 MMAs of a chunk (4 K-steps x the split products lo*hi, hi*lo, hi*hi), one
// thread refills a stage with factor blocks once its MMAs completed.
#include "asdsm_internal.h"
#include "tc_common.cuh"
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>

namespace asdsm {

namespace {

using namespace tc;

constexpr int BT_ROWS = 128, BT_COLS = 128, BT_STAGES = 3;
// Warps: 0 issues the MMAs, 1 loads the factor blocks, 4..7 form the A blocks
// and run the epilogue (tensor-memory lane quarter = warp mod 4).
constexpr int BT_THREADS = 256, BT_PRODUCERS = 128;
constexpr int BT_BLK = 128 * kRowBytes;              // one 128-row x 32-value swizzled block
constexpr int BT_STAGE = 4 * BT_BLK;                 // A hi, A lo, B hi, B lo
constexpr int BT_SMEM = BT_STAGES * BT_STAGE + 1024; // + alignment slack
constexpr uint32_t BT_TMEM_COLS = BT_COLS;
constexpr uint32_t kBtIdesc = idesc_tf32(BT_ROWS, BT_COLS);

// Index of the image block (level, pass, split, column block, K chunk);
// pass 0 = B_l^{-1}, pass 1 = M_l; split 0 = hi, 1 = lo.
__host__ __device__ __forceinline__ size_t bt_block(int level, int pass, int split, int cb, int kc, int CB, int KC) {
    return ((((size_t)level * 2 + pass) * 2 + split) * CB + cb) * KC + kc;
}

template <bool kBackward>
__global__ void __launch_bounds__(BT_THREADS, 1)
bcr_tc_kernel(BcrSys<float> g0, BcrSys<float> g1, int ngroups, int level) {
    extern __shared__ unsigned char bt_raw[];
    __shared__ __align__(8) uint64_t bfull[BT_STAGES], afull[BT_STAGES], mdone[BT_STAGES];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    const uint32_t raw = smem_u32(bt_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    unsigned char* pbase = bt_raw + (sbase - raw);
    int z = blockIdx.z;
    const BcrSys<float>* gp = &g0;
    if (ngroups > 1 && z >= g0.nsys) { gp = &g1; z -= g0.nsys; }
    const BcrSys<float>& g = *gp;
    const bool active = z < g.nsys && level < g.L && g.Ti;
    const int R = g.R, C = g.C, KC = g.TKC, CB = g.TCB;
    const int s = 1 << level;
    const int nrows = active ? (kBackward ? ((R + 1) >> (level + 1)) : (((R + 1) >> (level + 1)) - 1)) : 0;
    const int t0 = blockIdx.y * BT_ROWS;
    const int cb = blockIdx.x, c0 = cb * BT_COLS;
    const bool tile_ok = active && t0 < nrows && cb < CB && c0 < C;
    const int nchunks = (kBackward ? 2 : 1) * KC;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort_v = &abort_flag;
    if (tid == 0) {
        for (int q = 0; q < BT_STAGES; ++q) {
            mbar_init(smem_u32(&bfull[q]), 1);
            mbar_init(smem_u32(&afull[q]), BT_PRODUCERS);
            mbar_init(smem_u32(&mdone[q]), 1);
        }
        abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_holder), BT_TMEM_COLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = tmem_holder;
    asm volatile("griddepcontrol.launch_dependents;");
    if (warp == 1) {
        // Factor blocks (constant data: no wait for the previous level).  Chunk
        // q reuses the stage of chunk q - STAGES once that chunk's MMAs completed.
        if (lane == 0 && tile_ok) {
            const unsigned char* img = reinterpret_cast<const unsigned char*>(g.Ti);
            for (int q = 0; q < nchunks; ++q) {
                const int st = q % BT_STAGES;
                if (q >= BT_STAGES &&
                    !mbar_wait_abortable(smem_u32(&mdone[st]), (uint32_t)((q - BT_STAGES) / BT_STAGES) & 1u, abort_v)) {
                    *abort_v = 1;
                    break;
                }
                const int pass = kBackward ? (q < KC ? 0 : 1) : 1;
                const int kc = q % KC;
                const uint32_t dst = sbase + (uint32_t)(st * BT_STAGE + 2 * BT_BLK);
                const uint32_t bar = smem_u32(&bfull[st]);
                mbar_expect_tx(bar, 2 * BT_BLK);
                bulk_g2s(dst, img + bt_block(level, pass, 0, cb, kc, CB, KC) * BT_BLK, BT_BLK, bar);
                bulk_g2s(dst + BT_BLK, img + bt_block(level, pass, 1, cb, kc, CB, KC) * BT_BLK, BT_BLK, bar);
            }
        }
    } else if (warp == 0) {
        // MMA issuer: 4 K-steps x 3 split products per chunk into tensor memory.
        if (lane == 0 && tile_ok) {
            for (int q = 0; q < nchunks; ++q) {
                const int st = q % BT_STAGES;
                const uint32_t ph = (uint32_t)(q / BT_STAGES) & 1u;
                if (!mbar_wait_abortable(smem_u32(&afull[st]), ph, abort_v) ||
                    !mbar_wait_abortable(smem_u32(&bfull[st]), ph, abort_v)) {
                    *abort_v = 1;
                    break;
                }
                fence_after_sync();
                const uint32_t a0 = sbase + (uint32_t)(st * BT_STAGE), b0 = a0 + 2 * BT_BLK;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t ko = (uint32_t)(ks * 32);
                    const uint64_t aHi = sw128_desc(a0 + ko), aLo = sw128_desc(a0 + BT_BLK + ko);
                    const uint64_t bHi = sw128_desc(b0 + ko), bLo = sw128_desc(b0 + BT_BLK + ko);
                    tc_mma(tbase, aLo, bHi, kBtIdesc, (q > 0 || ks > 0) ? 1u : 0u);   // small terms first
                    tc_mma(tbase, aHi, bLo, kBtIdesc, 1u);
                    tc_mma(tbase, aHi, bHi, kBtIdesc, 1u);
                }
                tc_commit(smem_u32(&mdone[st]));
            }
        }
    } else if (warp >= BT_THREADS / 32 - BT_PRODUCERS / 32) {
        // Producers: A blocks (then the epilogue).  Warp p (0..3) forms rows
        // p, p + 4, ... of the tile, lane = reduction index; the rows of chunk
        // q + 1 are loaded into registers while chunk q is multiplied.
        const int pw = warp - (BT_THREADS / 32 - BT_PRODUCERS / 32);
        asm volatile("griddepcontrol.wait;" ::: "memory");
        const float wl = active ? g.wl[level] : 0.0f, wr = active ? g.wr[level] : 0.0f;
        float* X = g.X + (size_t)(active ? z : 0) * g.stride;
        float* Y = g.Y + (size_t)(active ? z : 0) * g.stride;
        const float* nb = kBackward ? Y : X;
        // Row j of this thread: t_j = tb + 4j, level row i_j = i0 + 8 s j.
        const int tb = t0 + pw;
        const int nj = tb < nrows ? min(BT_ROWS / 4, (nrows - tb + 3) / 4) : 0;
        const int i0 = kBackward ? s * (2 * tb + 1) : 2 * s * (tb + 1);
        const long long rstep = 8LL * s * C;                    // elements between rows j and j + 1
        const int nhi = (nj > 0 && i0 + s <= R) ? min(nj, (R - s - i0) / (8 * s) + 1) : 0;
        const int jlo = (kBackward && tb == 0) ? 1 : 0;         // backward t = 0: no lower neighbour
        const long long off_self = (long long)(i0 - 1) * C, off_lo = (long long)(i0 - s - 1) * C,
                        off_hi = (long long)(i0 + s - 1) * C;
        float pa[BT_ROWS / 4], pb[BT_ROWS / 4];
        auto load_chunk = [&](int q) {
            const int pass = kBackward ? (q < KC ? 0 : 1) : 1;
            const int k = (q % KC) * 32 + lane;
            const bool kok = k < C;
            if (pass == 0) {
                const float* p0 = X + off_self + k;
#pragma unroll
                for (int j = 0; j < BT_ROWS / 4; ++j) {
                    pa[j] = (kok && j < nj) ? p0[j * rstep] : 0.0f;
                    pb[j] = 0.0f;
                }
            } else {
#pragma unroll
                for (int j = 0; j < BT_ROWS / 4; ++j) {
                    pa[j] = (kok && j < nj && j >= jlo) ? nb[off_lo + k + j * rstep] : 0.0f;
                    pb[j] = (kok && j < nhi) ? nb[off_hi + k + j * rstep] : 0.0f;
                }
            }
        };
        if (tile_ok) {
            load_chunk(0);
            bool ok = true;
            for (int q = 0; q < nchunks; ++q) {
                const int st = q % BT_STAGES;
                if (q >= BT_STAGES &&
                    !mbar_wait_abortable(smem_u32(&mdone[st]), (uint32_t)((q - BT_STAGES) / BT_STAGES) & 1u, abort_v)) {
                    ok = false;
                    break;
                }
                unsigned char* pA = pbase + st * BT_STAGE;
                const bool combine = !kBackward || q >= KC;
#pragma unroll
                for (int j = 0; j < BT_ROWS / 4; ++j) {
                    const float v = combine ? -(wl * pa[j] + wr * pb[j]) : pa[j];
                    const float hi = tf32_hi(v);
                    const int off = swz_offset(pw + 4 * j, lane);
                    *reinterpret_cast<float*>(pA + off) = hi;
                    *reinterpret_cast<float*>(pA + BT_BLK + off) = v - hi;
                }
                fence_async_smem();
                mbar_arrive(smem_u32(&afull[st]));
                if (q + 1 < nchunks) load_chunk(q + 1);
            }
            const int ql = nchunks - 1;     // its commit covers every MMA of the tile
            if (ok) ok = mbar_wait_abortable(smem_u32(&mdone[ql % BT_STAGES]), (uint32_t)(ql / BT_STAGES) & 1u, abort_v);
            if (!ok) *abort_v = 1;
            // Epilogue: tensor-memory lanes 32 (warp mod 4) .. + 31 = tile rows.
            if (__all_sync(0xffffffffu, ok)) {
                fence_after_sync();
                const int q4 = warp & 3;
                const int t = t0 + q4 * 32 + lane;
                const bool rok = t < nrows;
                const int i = kBackward ? s * (2 * t + 1) : 2 * s * (t + 1);
                float* orow = (kBackward ? Y : X) + (size_t)(rok ? i - 1 : 0) * C;
#pragma unroll
                for (int j = 0; j < BT_COLS / 32; ++j) {
                    uint32_t v[32];
                    tmem_ld32(tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(j * 32), v);
                    const int cbase = c0 + j * 32;
                    if (rok) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            if (cbase + c < C) {
                                if (kBackward) orow[cbase + c] = __uint_as_float(v[c]);
                                else orow[cbase + c] += __uint_as_float(v[c]);
                            }
                        }
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (tid == 0 && abort_flag && g.tc_err) atomicExch(g.tc_err, 1);
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(tbase, BT_TMEM_COLS);
    }
}

template <bool kBackward>
cudaError_t bcr_tc_launch(const BcrSys<float>& g0, const BcrSys<float>& g1, int ngroups, int level, int maxRows,
                          int nsys, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(bcr_tc_kernel<kBackward>, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g0.TCB, (maxRows + BT_ROWS - 1) / BT_ROWS, nsys);
    cfg.blockDim = dim3(BT_THREADS);
    cfg.dynamicSmemBytes = BT_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, bcr_tc_kernel<kBackward>, g0, g1, ngroups, level);
}

}  // namespace

void bcr_tc_image(const BcrFactors& f, std::vector<float>* img, int* KC_out, int* CB_out) {
    const int C = f.C, L = f.L;
    const int KC = (C + 31) / 32, CB = (C + BT_COLS - 1) / BT_COLS;
    img->assign(bt_block(L, 0, 0, 0, 0, CB, KC) * (BT_BLK / sizeof(float)), 0.0f);
    unsigned char* base = reinterpret_cast<unsigned char*>(img->data());
    const std::vector<double>* F[2] = {&f.Bt, &f.Mt};
    for (int l = 0; l < L; ++l)
        for (int pass = 0; pass < 2; ++pass)
            for (int k = 0; k < C; ++k)
                for (int n = 0; n < C; ++n) {
                    // B[n][k] = F_l[n][k], stored transposed as [k][n].
                    const double v = (*F[pass])[((size_t)l * C + k) * C + n];
                    const float hi = tf32_hi((float)v);
                    const float lo = (float)(v - (double)hi);
                    const int off = swz_offset(n % BT_COLS, k % 32);
                    std::memcpy(base + bt_block(l, pass, 0, n / BT_COLS, k / 32, CB, KC) * BT_BLK + off, &hi, 4);
                    std::memcpy(base + bt_block(l, pass, 1, n / BT_COLS, k / 32, CB, KC) * BT_BLK + off, &lo, 4);
                }
    *KC_out = KC;
    *CB_out = CB;
}

cudaError_t bcr_tc_level(const BcrSys<float>& g0, const BcrSys<float>& g1, int ngroups, int level, bool backward,
                         int maxRows, int nsys, cudaStream_t st) {
    const BcrSys<float>* gs[2] = {&g0, &g1};
    for (int q = 0; q < ngroups; ++q) {
        const BcrSys<float>& g = *gs[q];
        if (!g.Ti || (reinterpret_cast<uintptr_t>(g.Ti) & 15u) || g.TCB != g0.TCB || g.TKC != (g.C + 31) / 32)
            return cudaErrorInvalidValue;
    }
    return backward ? bcr_tc_launch<true>(g0, g1, ngroups, level, maxRows, nsys, st)
                    : bcr_tc_launch<false>(g0, g1, ngroups, level, maxRows, nsys, st);
}

}  // namespace asdsm
