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
// neighbour rows, split, stored swizzled) pass through a 3-stage shared-memory
// ring, handed over by mbarriers.  One thread issues the 12 MMAs of a chunk
// (4 K-steps x the split products lo*hi, hi*lo, hi*hi), one thread refills a
// stage with factor blocks once its MMAs completed.  The A blocks come from
// three groups of four warps, group p filling stage p (chunks p, p + 3, ...):
// each group has its next chunk's rows in flight while the tensor core works,
// so three chunks' global loads overlap.  The epilogue stages the tile in the
// free ring and writes whole row segments (coalesced).
//
// The FP32 operands are split as x = hi + lo, both rounded to nearest TF32
// (|x - hi - lo| <= 2^-22 |x|); the dropped lo*lo term is of the same order.
#include "asdsm_internal.h"
#include "tc_common.cuh"
#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <cstdint>
#include <cstring>

namespace asdsm {

namespace cg = cooperative_groups;

namespace {

using namespace tc;

constexpr int BT_ROWS = 128, BT_COLS = 128, BT_STAGES = 3;
// Warps: 0 issues the MMAs, 1 loads the factor blocks, 2-3 idle, 4..15 form the A blocks (group (w - 4) / 4 owns ring stage
// (w - 4) / 4; tensor-memory lane quarter = w mod 4) and run the epilogue.
constexpr int BT_THREADS = 512, BT_PRODUCERS = 128, BT_PROD0 = 4;
constexpr int BT_EPI = BT_STAGES * BT_PRODUCERS;     // producer / epilogue threads
constexpr int BT_BLK = 128 * kRowBytes;              // one 128-row x 32-value swizzled block
constexpr int BT_STAGE = 4 * BT_BLK;                 // A hi, A lo, B hi, B lo
constexpr int BT_SMEM = BT_STAGES * BT_STAGE + 1024; // + alignment slack
constexpr int BT_SROW = BT_COLS + 1;                 // epilogue staging row stride (floats)
constexpr uint32_t BT_TMEM_COLS = BT_COLS;
constexpr uint32_t kBtIdesc = idesc_tf32(BT_ROWS, BT_COLS);
static_assert(BT_ROWS * BT_SROW * 4 <= BT_STAGES * BT_STAGE, "the epilogue tile fits the ring");
static_assert(BT_THREADS == (BT_PROD0 + BT_EPI / 32) * 32, "warp roles cover the block");

// Named barrier of the producer warps.  Their lanes may arrive diverged (the
// bounded mbarrier waits spin per lane), so the warp reconverges first and the
// barrier is the non-aligned form, which counts threads.
__device__ __forceinline__ void epi_barrier() {
    __syncwarp();
    asm volatile("barrier.sync 1, %0;" ::"n"(BT_EPI) : "memory");
    __syncwarp();
}

// Index of the image block (level, pass, split, column block, K chunk);
// pass 0 = B_l^{-1}, pass 1 = M_l; split 0 = hi, 1 = lo.
__host__ __device__ __forceinline__ size_t bt_block(int level, int pass, int split, int cb, int kc, int CB, int KC) {
    return ((((size_t)level * 2 + pass) * 2 + split) * CB + cb) * KC + kc;
}

// KS > 1: the KS CTAs of a thread-block cluster share one output tile, CTA
// rank r taking the reduction chunks [r n / KS, (r + 1) n / KS); after a
// cluster barrier rank r sums rows [128 r / KS, 128 (r + 1) / KS) of the KS
// partial tiles in rank order (deterministic) through distributed shared
// memory and writes them.
template <bool kBackward, int KS>
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
    const int rank = (int)(blockIdx.x % KS);          // rank in the cluster (clusters span x)
    const int cb = (int)(blockIdx.x / KS), c0 = cb * BT_COLS;
    const bool tile_ok = active && t0 < nrows && cb < CB && c0 < C;
    const int nchunks = (kBackward ? 2 : 1) * KC;
    const int qb = rank * nchunks / KS, nloc = (rank + 1) * nchunks / KS - qb;
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
    // Epilogue ownership: producer thread et writes the elements e = et + BT_EPI k
    // (k < NE) of this rank's BT_ROWS / KS rows x 128 columns: tile row
    // r0 + e / 128, column e mod 128 (consecutive threads, consecutive columns).
    constexpr int RPR = BT_ROWS / KS, NE = (RPR * BT_COLS + BT_EPI - 1) / BT_EPI;
    const int et = tid - BT_PROD0 * 32, r0 = rank * RPR;
    float xv[NE];                            // forward: the current values of the updated rows
    if (warp == 1) {
        // Factor blocks (constant data: no wait for the previous level).  Local
        // chunk u reuses the stage of chunk u - STAGES once its MMAs completed.
        if (lane == 0 && tile_ok) {
            const unsigned char* img = reinterpret_cast<const unsigned char*>(g.Ti);
            for (int u = 0; u < nloc; ++u) {
                const int q = qb + u, st = u % BT_STAGES;
                if (u >= BT_STAGES &&
                    !mbar_wait_abortable(smem_u32(&mdone[st]), (uint32_t)(u / BT_STAGES - 1) & 1u, abort_v)) {
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
            for (int u = 0; u < nloc; ++u) {
                const int st = u % BT_STAGES;
                const uint32_t ph = (uint32_t)(u / BT_STAGES) & 1u;
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
                    tc_mma(tbase, aLo, bHi, kBtIdesc, (u > 0 || ks > 0) ? 1u : 0u);   // small terms first
                    tc_mma(tbase, aHi, bLo, kBtIdesc, 1u);
                    tc_mma(tbase, aHi, bHi, kBtIdesc, 1u);
                }
                tc_commit(smem_u32(&mdone[st]));
            }
        }
    }
    float* const S = reinterpret_cast<float*>(pbase);   // epilogue tile [128][BT_SROW], in the ring
    // Writes this thread's output elements, the value of element (tile row r,
    // column cc) being get(r, cc); a batch's values are all read before any
    // is stored, so that their latencies overlap.
    auto write_out = [&](float* X, float* Y, auto get) {
        constexpr int NB = NE < 16 ? NE : 16;
#pragma unroll
        for (int kb = 0; kb < NE; kb += NB) {
            float val[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int e = et + BT_EPI * (kb + k);
                val[k] = (kb + k < NE && e < RPR * BT_COLS) ? get(r0 + (e >> 7), e & (BT_COLS - 1)) : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int e = et + BT_EPI * (kb + k), t = t0 + r0 + (e >> 7), col = c0 + (e & (BT_COLS - 1));
                if (kb + k < NE && e < RPR * BT_COLS && t < nrows && col < C) {
                    if (kBackward) Y[(size_t)(s * (2 * t + 1) - 1) * C + col] = val[k];
                    else X[(size_t)(2 * s * (t + 1) - 1) * C + col] = xv[kb + k] + val[k];
                }
            }
        }
    };
    if (warp >= BT_PROD0) {
        // Producers: A blocks of the group's chunks, then the epilogue.  Warp
        // quarter pw (0..3) forms rows pw, pw + 4, ... of the tile, lane =
        // reduction index; the rows of the group's next chunk are loaded into
        // registers while the tensor core multiplies the current ones.
        const int pg = (warp - BT_PROD0) >> 2, pw = warp & 3;
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
        bool ok = true;
        if (tile_ok) {
            if (pg < nloc) load_chunk(qb + pg);
            unsigned char* pA = pbase + pg * BT_STAGE;
            for (int u = pg; u < nloc; u += BT_STAGES) {
                // Local chunk u is the (u / STAGES)-th use of stage pg; wait for the previous one's MMAs.
                if (u >= BT_STAGES &&
                    !mbar_wait_abortable(smem_u32(&mdone[pg]), (uint32_t)(u / BT_STAGES - 1) & 1u, abort_v)) {
                    ok = false;
                    break;
                }
                const bool combine = !kBackward || qb + u >= KC;
#pragma unroll
                for (int j = 0; j < BT_ROWS / 4; ++j) {
                    const float v = combine ? -(wl * pa[j] + wr * pb[j]) : pa[j];
                    float hi, lo;
                    tf32_split(v, hi, lo);
                    const int off = swz_offset(pw + 4 * j, lane);
                    *reinterpret_cast<float*>(pA + off) = hi;
                    *reinterpret_cast<float*>(pA + BT_BLK + off) = lo;
                }
                fence_async_smem();
                mbar_arrive(smem_u32(&afull[pg]));
                if (u + BT_STAGES < nloc) load_chunk(qb + u + BT_STAGES);
            }
            if (!kBackward) {
                // The rows this level updates (i = 2s(t+1)) are written by this
                // tile's epilogue only: their values are read while the MMAs run.
#pragma unroll
                for (int k = 0; k < NE; ++k) {
                    const int e = et + BT_EPI * k, t = t0 + r0 + (e >> 7), col = c0 + (e & (BT_COLS - 1));
                    xv[k] = (e < RPR * BT_COLS && t < nrows && col < C)
                                ? X[(size_t)(2 * s * (t + 1) - 1) * C + col] : 0.0f;
                }
            }
            // The last chunk's commit covers every MMA of the tile.  Only the group
            // owning its stage waits (its waits on that barrier run phase by phase;
            // another group could be two phases behind, where a parity wait is
            // ambiguous); the others learn of it at the epilogue barrier.
            const int ul = nloc - 1;
            if (ok && nloc > 0 && pg == ul % BT_STAGES)
                ok = mbar_wait_abortable(smem_u32(&mdone[pg]), (uint32_t)(ul / BT_STAGES) & 1u, abort_v);
            if (!ok) *abort_v = 1;
        }
        // Epilogue.  Every producer thread passes the barriers; after the
        // first, the ring is free (all MMAs completed) and this CTA's abort
        // flag is final.
        epi_barrier();
        const bool go = tile_ok && *abort_v == 0;
        if (go) {
            // Tensor-memory lanes 32 pw .. + 31 = tile rows; group pg reads the
            // 32-column blocks pg, pg + 3, ...  A CTA without chunks holds zeros.
            fence_after_sync();
            const int r = pw * 32 + lane;
            for (int jb = pg; jb < BT_COLS / 32; jb += BT_STAGES) {
                uint32_t v[32];
                if (nloc > 0) {
                    tmem_ld32(tbase + ((uint32_t)(pw * 32) << 16) + (uint32_t)(jb * 32), v);
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] = 0u;
                }
#pragma unroll
                for (int c = 0; c < 32; ++c) S[r * BT_SROW + jb * 32 + c] = __uint_as_float(v[c]);
            }
        }
        if constexpr (KS == 1) {
            epi_barrier();
            if (go) write_out(X, Y, [&](int r, int cc) { return S[r * BT_SROW + cc]; });
        }
    }
    if constexpr (KS > 1) {
        // Every thread of every CTA of the cluster passes both cluster barriers.
        cg::cluster_group cluster = cg::this_cluster();
        __syncwarp();
        cluster.sync();                      // every rank's partial tile is in its shared memory
        if (warp >= BT_PROD0) {
            bool all_ok = tile_ok;
            for (int j = 0; j < KS; ++j) all_ok = all_ok && *cluster.map_shared_rank(&abort_flag, j) == 0;
            if (all_ok) {
                const float* Sr[KS];
#pragma unroll
                for (int j = 0; j < KS; ++j) Sr[j] = cluster.map_shared_rank(S, j);
                // The KS partial tiles summed in rank order.
                write_out(g.X + (size_t)z * g.stride, g.Y + (size_t)z * g.stride, [&](int r, int cc) {
                    float v = 0.0f;
#pragma unroll
                    for (int j = 0; j < KS; ++j) v += Sr[j][r * BT_SROW + cc];
                    return v;
                });
            }
        }
        __syncwarp();
        cluster.sync();                      // no CTA leaves while its tile is read
    }
    fence_before_sync();
    __syncthreads();
    if (tid == 0 && abort_flag && g.tc_err) atomicExch(g.tc_err, 1);
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(tbase, BT_TMEM_COLS);
    }
}

template <bool kBackward, int KS>
cudaError_t bcr_tc_launch(const BcrSys<float>& g0, const BcrSys<float>& g1, int ngroups, int level, int maxRows,
                          int nsys, cudaStream_t st) {
    static bool attr_set = false;           // per instantiation; setting it twice is harmless
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(bcr_tc_kernel<kBackward, KS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g0.TCB * KS, (maxRows + BT_ROWS - 1) / BT_ROWS, nsys);
    cfg.blockDim = dim3(BT_THREADS);
    cfg.dynamicSmemBytes = BT_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = KS;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = KS > 1 ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, bcr_tc_kernel<kBackward, KS>, g0, g1, ngroups, level);
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
                    const float hi = tf32_rn((float)v);
                    const float lo = tf32_rn((float)(v - (double)hi));
                    const int off = swz_offset(n % BT_COLS, k % 32);
                    std::memcpy(base + bt_block(l, pass, 0, n / BT_COLS, k / 32, CB, KC) * BT_BLK + off, &hi, 4);
                    std::memcpy(base + bt_block(l, pass, 1, n / BT_COLS, k / 32, CB, KC) * BT_BLK + off, &lo, 4);
                }
    *KC_out = KC;
    *CB_out = CB;
}

cudaError_t bcr_tc_level(const BcrSys<float>& g0, const BcrSys<float>& g1, int ngroups, int level, bool backward,
                         int ks, int maxRows, int nsys, cudaStream_t st) {
    const BcrSys<float>* gs[2] = {&g0, &g1};
    for (int q = 0; q < ngroups; ++q) {
        const BcrSys<float>& g = *gs[q];
        if (!g.Ti || (reinterpret_cast<uintptr_t>(g.Ti) & 15u) || g.TCB != g0.TCB || g.TKC != (g.C + 31) / 32)
            return cudaErrorInvalidValue;
    }
    switch (ks) {
        case 1: return backward ? bcr_tc_launch<true, 1>(g0, g1, ngroups, level, maxRows, nsys, st)
                                : bcr_tc_launch<false, 1>(g0, g1, ngroups, level, maxRows, nsys, st);
        case 2: return backward ? bcr_tc_launch<true, 2>(g0, g1, ngroups, level, maxRows, nsys, st)
                                : bcr_tc_launch<false, 2>(g0, g1, ngroups, level, maxRows, nsys, st);
        case 4: return backward ? bcr_tc_launch<true, 4>(g0, g1, ngroups, level, maxRows, nsys, st)
                                : bcr_tc_launch<false, 4>(g0, g1, ngroups, level, maxRows, nsys, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace asdsm
