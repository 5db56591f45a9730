// Exact direct solves of the separable submesh systems of ASDSM on sm_103a.
//
// Every system of eq. (2.4) is block tridiagonal Toeplitz along its "row"
// axis (R = 2^L - 1 rows, each a vector of C unknowns along the other axis):
//     a x_{i-1} + (d I + T) x_i + c x_{i+1} = f_i.
// Block cyclic reduction (BCR) with the per-level factors of host_math.cu
// (P_l = wl_l M_l, Q_l = wr_l M_l, B_l^{-1}):
//   forward, level l = 0..L-2 (s = 2^l), rows i = 2s, 4s, ...:
//       f_i <- f_i - M_l (wl_l f_{i-s} + wr_l f_{i+s})
//   backward, level l = L-1..0, rows i = s, 3s, 5s, ...:
//       x_i  = B_l^{-1} f_i - M_l (wl_l x_{i-s} + wr_l x_{i+s})
// (P_l, Q_l, B_l^{-1} are functions of T and commute, so the back-substitution
// reuses the forward factors).  Row 0 and row R+1 are zero.
//
// bcr_level_kernel: one launch per level; the level is a small dense GEMM
// (rows of the level x C outputs x C or 2C reduction) split over the
// reduction dimension among the 8 CTAs of a thread-block cluster, whose
// partial tiles are summed in a fixed order through distributed shared
// memory.  Used for the anisotropic families (R = N_f rows, C = N_c).
// bcr_tail_kernel: the last three levels of both directions of an FP32 solve
// as one dense product with the precomputed map of bcr_tail_map, where the
// system carries it.
// fill_holes_kernel: the Filler of Algorithm 3.  A warp segment of C+1 lanes
// owns one hole (lane c = hole column c); 32/(C+1) holes share a warp.  The
// factors of every level stay resident in shared memory for all holes a
// persistent CTA visits; only warp-level synchronisation is needed.
#include "asdsm_internal.h"
#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <cstdio>
#include <algorithm>

namespace cg = cooperative_groups;

namespace asdsm {

namespace {

#ifndef ASDSM_SPLITK_TC
#define ASDSM_SPLITK_TC 0
#endif
constexpr int GT_N = 64;       // output columns per tile
constexpr int GT_K = 32;       // reduction slice
constexpr int GT_THREADS = 128;

// Tensor-core step for the FP32 level GEMM: mma.sync m16n8k8 on TF32
// operands, each FP32 value split as hi = tf32(x), lo = tf32(x - hi) and the
// product formed as lo*hi + hi*lo + hi*hi (the lo*lo term, ~2^-22 relative, is
// dropped), accumulating in FP32.  Warp w owns rows 32(w/2) .. +32 and columns
// 32(w%2) .. +32 of the 64 x 64 tile: 2 x 4 fragments of 16 x 8.
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
    unsigned h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    const float r = x - __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
    hi = h;
    lo = l;
}

__device__ __forceinline__ void mma_tf32(float* d, const unsigned* a, unsigned b0, unsigned b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// As: [k][row] with row stride AW, Fs: [k][col] with row stride FW; k0 the
// first of the 8 reduction indices of this step.
template <int AW, int FW>
__device__ __forceinline__ void tc_step(const float* As, const float* Fs, int k0, int tid, float (*acc)[4]) {
    const int lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int rb = (warp >> 1) * 32, cb = (warp & 1) * 32;
    unsigned ah[2][4], al[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int r = rb + i * 16 + g;
        // A fragment (16 x 8, row major): (g, q), (g+8, q), (g, q+4), (g+8, q+4)
        split_tf32(As[(k0 + q) * AW + r], ah[i][0], al[i][0]);
        split_tf32(As[(k0 + q) * AW + r + 8], ah[i][1], al[i][1]);
        split_tf32(As[(k0 + q + 4) * AW + r], ah[i][2], al[i][2]);
        split_tf32(As[(k0 + q + 4) * AW + r + 8], ah[i][3], al[i][3]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = cb + j * 8 + g;
        // B fragment (8 x 8, column major): (k = q, n = g), (k = q+4, n = g)
        unsigned bh0, bl0, bh1, bl1;
        split_tf32(Fs[(k0 + q) * FW + c], bh0, bl0);
        split_tf32(Fs[(k0 + q + 4) * FW + c], bh1, bl1);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            float* d = acc[i * 4 + j];
            mma_tf32(d, al[i], bh0, bh1);
            mma_tf32(d, ah[i], bl0, bl1);
            mma_tf32(d, ah[i], bh0, bh1);
        }
    }
}

// One BCR level as a GEMM: out[t][c] = sum_k A[t][k] F[k][c], the reduction
// running over one factor (forward: -M (wl f_{i-s} + wr f_{i+s})) or two
// (backward: B^{-1} f_i, then -M (wl x_{i-s} + wr x_{i+s})), i.e. K' = C or 2C.
// A CTA computes a TM x 64 output tile (FP32, TM = 64: on the tensor cores,
// tc_step; otherwise 8 x 4 or 2 x 4 outputs per thread on the FMA pipes),
// walking 32-wide slices of K' staged in shared memory;
// the next slice is loaded into registers while the current one is used.
// With KS > 1 a thread-block cluster of KS CTAs shares the tile: CTA r takes
// the slices r, r+KS, ..., keeps its partial tile in shared memory and, after
// a cluster barrier, sums 1/KS of the tile over the KS partials in rank order
// (deterministic) and writes it.
template <typename T, bool kBackward, int TM, int KS>
__global__ void __launch_bounds__(GT_THREADS, sizeof(T) == 4 ? (TM == 64 ? 4 : 5) : 2)
bcr_level_kernel(BcrSys<T> g0, BcrSys<T> g1, int ngroups, int level) {
    // The split-K tiles stay on the FMA pipes (full FP32 products); the
    // tensor-core path of tc_step is kept for comparison and off by default.
    constexpr bool kTC = sizeof(T) == 4 && TM == 64 && ASDSM_SPLITK_TC;
    constexpr int RPT = TM / 8;                        // output rows per thread (32 or 8 accumulators)
    constexpr int A_PER_T = TM * GT_K / GT_THREADS;    // A-slice elements per thread
    constexpr int F_PER_T = GT_K * GT_N / GT_THREADS;  // factor-slice elements per thread
    constexpr int FSW = kTC ? GT_N + 8 : GT_N;         // padded factor rows: conflict-free fragment loads
    // The slices As [k][row], Fs [k][col] and, after the reduction loop, the
    // partial tile Part [row][col] share one buffer (Part fits in As + Fs).
    constexpr int AS_ELEMS = GT_K * (TM + 4), FS_ELEMS = GT_K * FSW;
    static_assert(TM * GT_N <= AS_ELEMS + FS_ELEMS, "partial tile must fit in the slice buffers");
    __shared__ __align__(16) T smem_buf[AS_ELEMS + FS_ELEMS];
    T (*As)[TM + 4] = reinterpret_cast<T (*)[TM + 4]>(smem_buf);
    T (*Fs)[FSW] = reinterpret_cast<T (*)[FSW]>(smem_buf + AS_ELEMS);
    T* Part = smem_buf;
    int rank = 0;
    if constexpr (KS > 1) rank = (int)cg::this_cluster().block_rank();
    int z = blockIdx.z;
    const BcrSys<T>* gp = &g0;
    if (ngroups > 1 && z >= g0.nsys) { gp = &g1; z -= g0.nsys; }
    const BcrSys<T>& g = *gp;
    // Every CTA of a cluster takes the same branch below (same z, tile), so the
    // cluster barriers are always reached by all of them.
    const bool active = z < g.nsys && level < g.L;
    const int R = g.R, C = g.C;
    const int s = 1 << level;
    const int nrows = active ? (kBackward ? ((R + 1) >> (level + 1)) : (((R + 1) >> (level + 1)) - 1)) : 0;
    const int t0 = blockIdx.y * TM;
    const int c0 = (blockIdx.x / KS) * GT_N;
    const bool tile_ok = active && t0 < nrows && c0 < C;
    const size_t n2 = (size_t)C * C;
    const T* Mt = g.Mt + (size_t)(active ? level : 0) * n2;
    const T* Bt = g.Bt + (size_t)(active ? level : 0) * n2;
    const T wl = active ? g.wl[level] : T(0), wr = active ? g.wr[level] : T(0);
    T* X = g.X + (size_t)(active ? z : 0) * g.stride;
    T* Y = g.Y + (size_t)(active ? z : 0) * g.stride;
    const T* nb = kBackward ? Y : X;            // neighbour rows: solved (bwd) or reduced (fwd)

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    T acc[RPT][4];
#pragma unroll
    for (int a = 0; a < RPT; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);

    const int nk = (C + GT_K - 1) / GT_K;        // slices per factor pass
    const int total = (kBackward ? 2 : 1) * nk;
    T av[A_PER_T], fv[F_PER_T];
    auto load_factor = [&](int q) {
        const int pass = kBackward ? q / nk : 1;
        const int k0 = (q % nk) * GT_K;
        const T* Fm = pass == 0 ? Bt : Mt;
#pragma unroll
        for (int j = 0; j < F_PER_T; ++j) {
            const int e = tid + j * GT_THREADS;
            const int kk = e / GT_N, cc = e % GT_N;
            const int k = k0 + kk, c = c0 + cc;
            fv[j] = (k < C && c < C) ? __ldg(Fm + (size_t)k * C + c) : T(0);
        }
    };
    auto load_rows = [&](int q) {
        const int pass = kBackward ? q / nk : 1;  // 0: B^{-1} f_i, 1: -M v_i
        const int k0 = (q % nk) * GT_K;
#pragma unroll
        for (int j = 0; j < A_PER_T; ++j) {
            const int e = tid + j * GT_THREADS;
            const int r = e / GT_K, kk = e % GT_K;
            const int t = t0 + r, k = k0 + kk;
            T v = T(0);
            if (t < nrows && k < C) {
                const int i = kBackward ? s * (2 * t + 1) : 2 * s * (t + 1);
                if (pass == 0) {
                    v = X[(size_t)(i - 1) * C + k];
                } else {
                    if (i - s >= 1) v += wl * nb[(size_t)(i - s - 1) * C + k];
                    if (i + s <= R) v += wr * nb[(size_t)(i + s - 1) * C + k];
                    v = -v;
                }
            }
            av[j] = v;
        }
    };
    // Programmatic dependent launch: the next level may start launching now;
    // this one prefetches its first factor slice (constant data) and then
    // waits, in every CTA, for the grids it depends on before reading rows.
    asm volatile("griddepcontrol.launch_dependents;");
    if (tile_ok && rank < total) load_factor(rank);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (tile_ok && rank < total) load_rows(rank);
    for (int q = rank; tile_ok && q < total; q += KS) {
        __syncthreads();                          // the previous slice has been used
#pragma unroll
        for (int j = 0; j < A_PER_T; ++j) {
            const int e = tid + j * GT_THREADS;
            As[e % GT_K][e / GT_K] = av[j];
        }
#pragma unroll
        for (int j = 0; j < F_PER_T; ++j) {
            const int e = tid + j * GT_THREADS;
            Fs[e / GT_N][e % GT_N] = fv[j];
        }
        __syncthreads();
        if (q + KS < total) { load_factor(q + KS); load_rows(q + KS); }
        if constexpr (kTC) {
#pragma unroll
            for (int ks = 0; ks < GT_K / 8; ++ks)
                tc_step<TM + 4, FSW>(&As[0][0], &Fs[0][0], ks * 8, tid, acc);
        } else {
#pragma unroll 8
        for (int kk = 0; kk < GT_K; ++kk) {
            T a_[RPT], b_[4];
            if constexpr (sizeof(T) == 4 && RPT == 8) {
                const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
                const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
                a_[0] = a0.x; a_[1] = a0.y; a_[2] = a0.z; a_[3] = a0.w;
                a_[4] = a1.x; a_[5] = a1.y; a_[6] = a1.z; a_[7] = a1.w;
            } else if constexpr (sizeof(T) == 4 && RPT == 2) {
                const float2 a0 = *reinterpret_cast<const float2*>(&As[kk][ty * 2]);
                a_[0] = a0.x; a_[1] = a0.y;
            } else {
#pragma unroll
                for (int a = 0; a < RPT; ++a) a_[a] = As[kk][ty * RPT + a];
            }
            if constexpr (sizeof(T) == 4) {
                const float4 b4 = *reinterpret_cast<const float4*>(&Fs[kk][tx * 4]);
                b_[0] = b4.x; b_[1] = b4.y; b_[2] = b4.z; b_[3] = b4.w;
            } else {
#pragma unroll
                for (int b = 0; b < 4; ++b) b_[b] = Fs[kk][tx * 4 + b];
            }
#pragma unroll
            for (int a = 0; a < RPT; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += a_[a] * b_[b];
        }
        }
    }
    // Position in the tile of accumulator acc[a][b].
    auto tile_pos = [&](int a, int b, int& r, int& c) {
        if constexpr (kTC) {
            const int lane = tid & 31, warp = tid >> 5;
            r = (warp >> 1) * 32 + (a >> 2) * 16 + (lane >> 2) + ((b >> 1) << 3);
            c = (warp & 1) * 32 + (a & 3) * 8 + 2 * (lane & 3) + (b & 1);
        } else {
            r = ty * RPT + a;
            c = tx * 4 + b;
        }
    };
    if constexpr (KS == 1) {
#pragma unroll
        for (int a = 0; a < RPT; ++a) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                int r, cc;
                tile_pos(a, b, r, cc);
                const int t = t0 + r, c = c0 + cc;
                if (!tile_ok || t >= nrows || c >= C) continue;
                const int i = kBackward ? s * (2 * t + 1) : 2 * s * (t + 1);
                if (kBackward) Y[(size_t)(i - 1) * C + c] = acc[a][b];
                else X[(size_t)(i - 1) * C + c] += acc[a][b];
            }
        }
    } else {
        cg::cluster_group cluster = cg::this_cluster();
        __syncthreads();     // the slice buffers are reused for the partial tile
#pragma unroll
        for (int a = 0; a < RPT; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                int r, cc;
                tile_pos(a, b, r, cc);
                Part[r * GT_N + cc] = acc[a][b];
            }
        cluster.sync();
        // Rank r reduces elements [r*TM*64/KS, (r+1)*TM*64/KS) of the tile over the partials.
        constexpr int SLICE = TM * GT_N / KS;
        for (int e = rank * SLICE + tid; tile_ok && e < (rank + 1) * SLICE; e += GT_THREADS) {
            T sum = T(0);
#pragma unroll
            for (int rr = 0; rr < KS; ++rr) sum += cluster.map_shared_rank(Part, rr)[e];
            const int r = e / GT_N, cc = e % GT_N;
            const int t = t0 + r, c = c0 + cc;
            if (t < nrows && c < C) {
                const int i = kBackward ? s * (2 * t + 1) : 2 * s * (t + 1);
                if (kBackward) Y[(size_t)(i - 1) * C + c] = sum;
                else X[(size_t)(i - 1) * C + c] += sum;
            }
        }
        cluster.sync();          // partial tiles stay alive until every CTA has read them
    }
}

// ---------------------------------------------------------------------------
// Wide tensor-core level kernel (FP32): a CTA of 8 warps owns 32 rows x 256
// columns of a level's output, so one wave covers the big levels without
// splitting the reduction.  Each 32-wide reduction slice - the factor slice
// (32 x 256, from the padded, swizzled copy in BcrSys::Mw/Bw, 16-byte
// copies) and the raw neighbour rows it multiplies (4-byte copies) - streams
// through a 4-stage shared-memory ring by cp.async, three slices ahead: each
// thread waits for its own copies, then a CTA barrier publishes the slice.
// The row combination -(wl x_{i-s} + wr x_{i+s}) is formed when the A
// fragments are read; products by the TF32 split (3 mma.sync per fragment).
// ---------------------------------------------------------------------------
constexpr int WD_ROWS = 32, WD_COLS = 256, WD_THREADS = 256, WD_STAGES = 4;
constexpr int WD_AW = WD_ROWS + 8;     // row stride of the [k][row] slices (= 8 mod 32: conflict-free fragments)
constexpr int WD_STAGE_F = GT_K * WD_COLS;           // floats of a factor slice
constexpr int WD_STAGE_A = GT_K * WD_AW;             // floats of one row slice
constexpr int WD_STAGE = WD_STAGE_F + 2 * WD_STAGE_A;
constexpr size_t wd_smem_bytes() { return sizeof(float) * (size_t)WD_STAGES * WD_STAGE; }

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4f(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit_w() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_w() { asm volatile("cp.async.wait_group %0;\n" ::"n"(WD_STAGES - 1) : "memory"); }

// Column of element (k, c) in the swizzled factor rows.
__device__ __forceinline__ int wd_swz(int k, int c) { return (((c >> 2) ^ (2 * (k & 3))) << 2) | (c & 3); }

// A element (row r, reduction index kk) of the slice: the row itself (pass 0)
// or -(wl x_{i-s} + wr x_{i+s}) (pass 1).
__device__ __forceinline__ float wd_a(const float* R1, const float* R2, int kk, int r, bool combine, float wl, float wr) {
    const float a = R1[kk * WD_AW + r];
    if (!combine) return a;
    return -(wl * a + wr * R2[kk * WD_AW + r]);
}

// 32 rows (2 fragments) x this warp's 32 columns (4 fragments), 8 reduction indices.
__device__ __forceinline__ void tc_step_wide(const float* R1, const float* R2, bool combine, float wl, float wr,
                                             const float* Fs, int k0, int tid, float (*acc)[4]) {
    const int lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int cb = warp * 32;
    unsigned ah[2][4], al[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int r = i * 16 + g;
        split_tf32(wd_a(R1, R2, k0 + q, r, combine, wl, wr), ah[i][0], al[i][0]);
        split_tf32(wd_a(R1, R2, k0 + q, r + 8, combine, wl, wr), ah[i][1], al[i][1]);
        split_tf32(wd_a(R1, R2, k0 + q + 4, r, combine, wl, wr), ah[i][2], al[i][2]);
        split_tf32(wd_a(R1, R2, k0 + q + 4, r + 8, combine, wl, wr), ah[i][3], al[i][3]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = cb + j * 8 + g;
        unsigned bh0, bl0, bh1, bl1;
        split_tf32(Fs[(k0 + q) * WD_COLS + wd_swz(k0 + q, c)], bh0, bl0);
        split_tf32(Fs[(k0 + q + 4) * WD_COLS + wd_swz(k0 + q + 4, c)], bh1, bl1);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            float* d = acc[i * 4 + j];
            mma_tf32(d, al[i], bh0, bh1);
            mma_tf32(d, ah[i], bl0, bl1);
            mma_tf32(d, ah[i], bh0, bh1);
        }
    }
}

template <bool kBackward>
__global__ void __launch_bounds__(WD_THREADS, 1)
bcr_level_wide_kernel(BcrSys<float> g0, BcrSys<float> g1, int ngroups, int level) {
    extern __shared__ __align__(16) float wsm[];
    int z = blockIdx.z;
    const BcrSys<float>* gp = &g0;
    if (ngroups > 1 && z >= g0.nsys) { gp = &g1; z -= g0.nsys; }
    const BcrSys<float>& g = *gp;
    const bool active = z < g.nsys && level < g.L;
    const int R = g.R, C = g.C, KW = g.KW, CW = g.CW;
    const int s = 1 << level;
    const int nrows = active ? (kBackward ? ((R + 1) >> (level + 1)) : (((R + 1) >> (level + 1)) - 1)) : 0;
    const int t0 = blockIdx.y * WD_ROWS;
    const int c0 = blockIdx.x * WD_COLS;
    const bool tile_ok = active && t0 < nrows && c0 < C;
    const size_t lw = (size_t)KW * CW;
    const float* Mw = g.Mw + (size_t)(active ? level : 0) * lw;
    const float* Bw = g.Bw + (size_t)(active ? level : 0) * lw;
    const float wl = active ? g.wl[level] : 0.0f, wr = active ? g.wr[level] : 0.0f;
    float* X = g.X + (size_t)(active ? z : 0) * g.stride;
    float* Y = g.Y + (size_t)(active ? z : 0) * g.stride;
    const float* nb = kBackward ? Y : X;
    const int tid = threadIdx.x;
    const int nk = KW / GT_K;
    const int total = (kBackward ? 2 : 1) * nk;
    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;

    auto stage_of = [&](int q) { return wsm + (size_t)(q % WD_STAGES) * WD_STAGE; };
    auto issue_factor = [&](int q) {
        const int pass = kBackward ? q / nk : 1;
        const int k0 = (q % nk) * GT_K;
        const float* Fm = pass == 0 ? Bw : Mw;
        float* dst = stage_of(q);
#pragma unroll
        for (int j = 0; j < GT_K * WD_COLS / 4 / WD_THREADS; ++j) {      // 8 chunks of 16 B per thread
            const int e = tid + j * WD_THREADS;
            const int kk = e / (WD_COLS / 4), ch = e % (WD_COLS / 4);
            cp_async16(dst + kk * WD_COLS + ch * 4, Fm + (size_t)(k0 + kk) * CW + c0 + ch * 4);
        }
    };
    // Raw rows of slice q: R1 = x_i (pass 0) or x_{i-s} (pass 1), R2 = x_{i+s}; zero where absent.
    auto issue_rows = [&](int q) {
        const int pass = kBackward ? q / nk : 1;
        const int k0 = (q % nk) * GT_K;
        float* R1 = stage_of(q) + WD_STAGE_F;
        float* R2 = R1 + WD_STAGE_A;
#pragma unroll
        for (int j = 0; j < WD_ROWS * GT_K / WD_THREADS; ++j) {          // 4 elements per thread
            const int e = tid + j * WD_THREADS;
            const int r = e / GT_K, kk = e % GT_K;
            const int t = t0 + r, k = k0 + kk;
            float* d1 = R1 + kk * WD_AW + r;
            float* d2 = R2 + kk * WD_AW + r;
            const bool ok = t < nrows && k < C;
            const int i = kBackward ? s * (2 * t + 1) : 2 * s * (t + 1);
            if (pass == 0) {
                if (ok) cp_async4f(d1, X + (size_t)(i - 1) * C + k);
                else *d1 = 0.0f;
            } else {
                if (ok && i - s >= 1) cp_async4f(d1, nb + (size_t)(i - s - 1) * C + k);
                else *d1 = 0.0f;
                if (ok && i + s <= R) cp_async4f(d2, nb + (size_t)(i + s - 1) * C + k);
                else *d2 = 0.0f;
            }
        }
    };
    // Programmatic dependent launch: the first two factor slices (constant
    // data) are requested before waiting for the grids this one depends on.
    // Slices 0 .. WD_STAGES-2 are in flight before the loop (factor slices
    // first, one group; then one group of rows per slice); the loop issues
    // slice q + WD_STAGES - 1 and waits for slice q.
    asm volatile("griddepcontrol.launch_dependents;");
    for (int q = 0; tile_ok && q < WD_STAGES - 1 && q < total; ++q) issue_factor(q);
    cp_commit_w();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int q = 0; q < WD_STAGES - 1; ++q) {
        if (tile_ok && q < total) issue_rows(q);
        cp_commit_w();
    }
    for (int q = 0; tile_ok && q < total; ++q) {
        const int qn = q + WD_STAGES - 1;
        if (qn < total) { issue_factor(qn); issue_rows(qn); }          // its stage was released last iteration
        cp_commit_w();
        cp_wait_w();                                                   // this thread's copies of slice q landed
        __syncthreads();                                               // everyone's copies of slice q visible
        const float* st = stage_of(q);
        const float* R1 = st + WD_STAGE_F;
        const float* R2 = R1 + WD_STAGE_A;
        const bool combine = !(kBackward && q < nk);
#pragma unroll
        for (int ks = 0; ks < GT_K / 8; ++ks) tc_step_wide(R1, R2, combine, wl, wr, st, ks * 8, tid, acc);
        __syncthreads();                                               // slice q's stage is free
    }
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int r = (a >> 2) * 16 + (lane >> 2) + ((b >> 1) << 3);
            const int cc = warp * 32 + (a & 3) * 8 + 2 * (lane & 3) + (b & 1);
            const int t = t0 + r, c = c0 + cc;
            if (!tile_ok || t >= nrows || c >= C) continue;
            const int i = kBackward ? s * (2 * t + 1) : 2 * s * (t + 1);
            if (kBackward) Y[(size_t)(i - 1) * C + c] = acc[a][b];
            else X[(size_t)(i - 1) * C + c] += acc[a][b];
        }
    }
}

template <bool kBackward>
cudaError_t launch_wide(dim3 grid, const BcrSys<float>& g0, const BcrSys<float>& g1, int ngroups, int level,
                        cudaStream_t st) {
    const size_t smem = wd_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(bcr_level_wide_kernel<kBackward>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(WD_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, bcr_level_wide_kernel<kBackward>, g0, g1, ngroups, level);
}

template <typename T, bool kBackward, int TM, int KS>
cudaError_t launch_variant(dim3 grid, const BcrSys<T>& g0, const BcrSys<T>& g1, int ngroups, int level,
                           cudaStream_t st) {
    grid.x *= KS;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(GT_THREADS);
    cfg.dynamicSmemBytes = 0;
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
    return cudaLaunchKernelEx(&cfg, bcr_level_kernel<T, kBackward, TM, KS>, g0, g1, ngroups, level);
}

template <typename T, bool kBackward, int TM>
cudaError_t launch_ks(int ks, dim3 grid, const BcrSys<T>& g0, const BcrSys<T>& g1, int ngroups, int level,
                      cudaStream_t st) {
    switch (ks) {
        case 1: return launch_variant<T, kBackward, TM, 1>(grid, g0, g1, ngroups, level, st);
        case 2: return launch_variant<T, kBackward, TM, 2>(grid, g0, g1, ngroups, level, st);
        case 4: return launch_variant<T, kBackward, TM, 4>(grid, g0, g1, ngroups, level, st);
        case 8: return launch_variant<T, kBackward, TM, 8>(grid, g0, g1, ngroups, level, st);
        default: return cudaErrorInvalidValue;
    }
}

// The tail of the reduction (bcr_tail_map) as one dense matrix-vector
// product per system: y = D x over the rt rows i = k 2^l0, one warp per
// output row, x staged in shared memory, a fixed summation order per row.
// Launched with programmatic dependent launch: the first TL_PF float4 of each
// lane's share of its row of D (constant data) are loaded before the wait for
// the forward level that produced x, the rest in batches of TL_PF afterwards.
constexpr int TL_WARPS = 8, TL_PF = 8;

__global__ void __launch_bounds__(32 * TL_WARPS) bcr_tail_kernel(BcrSys<float> g0, BcrSys<float> g1, int ngroups) {
    extern __shared__ __align__(16) float xs[];
    int z = blockIdx.y;
    const BcrSys<float>* gp = &g0;
    if (ngroups > 1 && z >= g0.nsys) { gp = &g1; z -= g0.nsys; }
    const BcrSys<float>& g = *gp;
    const bool sys_ok = z < g.nsys;
    const int C = g.C, rt = g.tail_rt, ld = g.tail_ld, n = rt * C, n4 = ld >> 2;
    const int s0 = (g.R + 1) / (rt + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * TL_WARPS + warp;
    const bool ok = sys_ok && r < n;
    const float4* Drow = reinterpret_cast<const float4*>(g.Dt) + (size_t)(ok ? r : 0) * n4;
    asm volatile("griddepcontrol.launch_dependents;");
    float4 pf[TL_PF];
#pragma unroll
    for (int u = 0; u < TL_PF; ++u) {
        const int q = lane + 32 * u;
        pf[u] = ok && q < n4 ? __ldg(Drow + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const float* X = g.X + (size_t)(sys_ok ? z : 0) * g.stride;
    float* Y = g.Y + (size_t)(sys_ok ? z : 0) * g.stride;
    for (int q = threadIdx.x; q < ld; q += blockDim.x) {
        float v = 0.f;
        if (sys_ok && q < n) v = X[(size_t)((q / C + 1) * s0 - 1) * C + q % C];
        xs[q] = v;
    }
    __syncthreads();
    if (!ok) return;
    const float4* x4 = reinterpret_cast<const float4*>(xs);
    float acc = 0.f;
    auto dot4 = [&](const float4& d, int q) {
        const float4 xv = x4[q];
        acc = fmaf(d.x, xv.x, acc);
        acc = fmaf(d.y, xv.y, acc);
        acc = fmaf(d.z, xv.z, acc);
        acc = fmaf(d.w, xv.w, acc);
    };
#pragma unroll
    for (int u = 0; u < TL_PF; ++u)
        if (lane + 32 * u < n4) dot4(pf[u], lane + 32 * u);
    for (int base = 32 * TL_PF; base < n4; base += 32 * TL_PF) {
#pragma unroll
        for (int u = 0; u < TL_PF; ++u) {
            const int q = base + lane + 32 * u;
            pf[u] = q < n4 ? __ldg(Drow + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < TL_PF; ++u)
            if (base + lane + 32 * u < n4) dot4(pf[u], base + lane + 32 * u);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) Y[(size_t)((r / C + 1) * s0 - 1) * C + r % C] = acc;
}

cudaError_t launch_tail(const BcrSys<float>* groups, int ngroups, cudaStream_t st) {
    int maxn = 0, maxld = 0, nsys = 0;
    for (int q = 0; q < ngroups; ++q) {
        maxn = std::max(maxn, groups[q].tail_rt * groups[q].C);
        maxld = std::max(maxld, groups[q].tail_ld);
        nsys += groups[q].nsys;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((maxn + TL_WARPS - 1) / TL_WARPS, nsys, 1);
    cfg.blockDim = dim3(32 * TL_WARPS);
    cfg.dynamicSmemBytes = (size_t)maxld * sizeof(float);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const BcrSys<float>& g1 = ngroups > 1 ? groups[1] : groups[0];
    cudaError_t e = cudaLaunchKernelEx(&cfg, bcr_tail_kernel, groups[0], g1, ngroups);
    note_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T, bool kBackward>
cudaError_t launch_level(const BcrSys<T>* groups, int ngroups, int level, const BcrTune* tune, cudaStream_t st) {
    int maxC = 0, maxRows = 0, nsys = 0;
    for (int q = 0; q < ngroups; ++q) {
        const BcrSys<T>& g = groups[q];
        if (level >= g.L) continue;
        maxC = g.C > maxC ? g.C : maxC;
        int rows = kBackward ? ((g.R + 1) >> (level + 1)) : (((g.R + 1) >> (level + 1)) - 1);
        maxRows = rows > maxRows ? rows : maxRows;
        nsys += g.nsys;
    }
    if (maxRows <= 0 || nsys == 0) return cudaSuccess;
    BcrSys<T> g1 = ngroups > 1 ? groups[1] : groups[0];
    const int ctiles = (maxC + GT_N - 1) / GT_N;
    const int chunks = (kBackward ? 2 : 1) * ((maxC + GT_K - 1) / GT_K);
    int tm = 0, ks = 0;
    if (tune) {
        const int v = tune->cfg[kBackward ? 1 : 0][level];
        tm = v >> 8;
        ks = v & 0xFF;
    }
    bool wide_ok = sizeof(T) == 4, tc_ok = sizeof(T) == 4;
    for (int q = 0; q < ngroups; ++q) {
        wide_ok = wide_ok && groups[q].Mw && groups[q].Bw;
        tc_ok = tc_ok && groups[q].Ti;
    }
    if (tm == 128 && tc_ok) {
        cudaError_t e = cudaSuccess;
        if constexpr (sizeof(T) == 4) {
            e = bcr_tc_level(reinterpret_cast<const BcrSys<float>&>(groups[0]), reinterpret_cast<const BcrSys<float>&>(g1),
                             ngroups, level, kBackward, ks == 2 || ks == 4 ? ks : 1, maxRows, nsys, st);
        }
        note_launch();
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    if (tm == 32 && wide_ok) {
        int CW = groups[0].CW;
        dim3 grid(CW / WD_COLS, (maxRows + WD_ROWS - 1) / WD_ROWS, nsys);
        cudaError_t e = cudaSuccess;
        if constexpr (sizeof(T) == 4) {
            e = launch_wide<kBackward>(grid, reinterpret_cast<const BcrSys<float>&>(groups[0]),
                                       reinterpret_cast<const BcrSys<float>&>(g1), ngroups, level, st);
        }
        note_launch();
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    if (tm != 16 && tm != 64) tm = maxRows >= 48 ? 64 : 16;
    if (ks != 1 && ks != 2 && ks != 4 && ks != 8) {
        // Split the reduction until the launch has about three CTAs per SM.
        const long long tiles = (long long)ctiles * ((maxRows + tm - 1) / tm) * nsys;
        const long long target = 3LL * (tune && tune->num_sms > 0 ? tune->num_sms : 152);
        ks = 1;
        while (ks < 8 && tiles * ks < target && 2 * ks <= chunks) ks *= 2;
    }
    if (ks > chunks) ks = 1;
    if (tune && tune->trace)
        std::fprintf(stderr, "asdsm bcr: bwd=%d level=%d rows=%d C=%d tm=%d ks=%d (table %d)\n", kBackward ? 1 : 0, level,
                     maxRows, maxC, tm, ks, tune->cfg[kBackward ? 1 : 0][level]);
    dim3 grid(ctiles, (maxRows + tm - 1) / tm, nsys);
    cudaError_t e = tm == 64 ? launch_ks<T, kBackward, 64>(ks, grid, groups[0], g1, ngroups, level, st)
                             : launch_ks<T, kBackward, 16>(ks, grid, groups[0], g1, ngroups, level, st);
    note_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t bcr_solve(const BcrSys<T>* groups, int ngroups, cudaStream_t st, const BcrTune* tune) {
    if (ngroups < 1 || ngroups > 2) return cudaErrorInvalidValue;
    int L = 0;
    for (int q = 0; q < ngroups; ++q) L = groups[q].L > L ? groups[q].L : L;
    for (int q = 0; q < ngroups; ++q)
        if (groups[q].L != L) return cudaErrorInvalidValue;   // groups in one call share the level count
    // Levels l0..L-1 of both directions become one dense product when every
    // group carries the tail map (FP32 only).
    int l0 = L;
    if constexpr (sizeof(T) == 4) {
        bool tail = true;
        for (int q = 0; q < ngroups; ++q)
            tail = tail && groups[q].Dt && groups[q].tail_rt == groups[0].tail_rt && groups[q].tail_rt > 0;
        if (tail) {
            int lt = 0;
            while ((1 << lt) - 1 < groups[0].tail_rt) ++lt;
            if (lt <= L) l0 = L - lt;
        }
    }
    cudaError_t e;
    for (int l = 0; l + 1 < L && l < l0; ++l)
        if ((e = launch_level<T, false>(groups, ngroups, l, tune, st)) != cudaSuccess) return e;
    if constexpr (sizeof(T) == 4) {
        if (l0 < L && (e = launch_tail(reinterpret_cast<const BcrSys<float>*>(groups), ngroups, st)) != cudaSuccess)
            return e;
    }
    for (int l = (l0 < L ? l0 : L) - 1; l >= 0; --l)
        if ((e = launch_level<T, true>(groups, ngroups, l, tune, st)) != cudaSuccess) return e;
    return cudaSuccess;
}

template <typename T>
cudaError_t bcr_level(const BcrSys<T>* groups, int ngroups, int level, bool backward, const BcrTune* tune,
                      cudaStream_t st) {
    if (ngroups < 1 || ngroups > 2) return cudaErrorInvalidValue;
    return backward ? launch_level<T, true>(groups, ngroups, level, tune, st)
                    : launch_level<T, false>(groups, ngroups, level, tune, st);
}

// ---------------------------------------------------------------------------
// Iterative refinement of the separable systems: r = b - A x in FP64 for
// A = block tridiagonal (a I, d I + T, c I), T = tridiag(tl, td, tu) (the
// systems make_bcr factors), written as FP32 for the next FP32 solve; and
// x += y (FP32 correction into the FP64 solution).
// ---------------------------------------------------------------------------
namespace {
__global__ void bcr_residual_kernel(const double* __restrict__ x, const double* __restrict__ b, float* __restrict__ r32,
                                    int R, int C, double a, double d, double c, double tl, double td, double tu) {
    const long long n = (long long)R * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / C), k = (int)(e % C);
        double ax = (d + td) * x[e];
        if (k > 0) ax += tl * x[e - 1];
        if (k + 1 < C) ax += tu * x[e + 1];
        if (i > 0) ax += a * x[e - C];
        if (i + 1 < R) ax += c * x[e + C];
        r32[e] = (float)(b[e] - ax);
    }
}
__global__ void add_float_kernel(double* __restrict__ x, const float* __restrict__ y, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        x[e] += (double)y[e];
}
unsigned refine_grid(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 152LL * 16 ? 152LL * 16 : b));
}
}  // namespace

cudaError_t bcr_residual(const double* x, const double* b, float* r32, int R, int C, const BcrCoefs& k,
                         cudaStream_t st) {
    bcr_residual_kernel<<<refine_grid((long long)R * C), 256, 0, st>>>(x, b, r32, R, C, k.a, k.d, k.c, k.tl, k.td, k.tu);
    note_launch();
    return cudaGetLastError();
}

cudaError_t add_float(double* x, const float* y, long long n, cudaStream_t st) {
    add_float_kernel<<<refine_grid(n), 256, 0, st>>>(x, y, n);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t bcr_level<float>(const BcrSys<float>*, int, int, bool, const BcrTune*, cudaStream_t);
template cudaError_t bcr_level<double>(const BcrSys<double>*, int, int, bool, const BcrTune*, cudaStream_t);
template cudaError_t bcr_solve<float>(const BcrSys<float>*, int, cudaStream_t, const BcrTune*);
template cudaError_t bcr_solve<double>(const BcrSys<double>*, int, cudaStream_t, const BcrTune*);

// ---------------------------------------------------------------------------
// Fused hole fill (Algorithm 3): one warp segment per hole.
// ---------------------------------------------------------------------------
namespace {

constexpr int FILL_MAX_WARPS = 8;
constexpr int FILL_MAX_THREADS = 32 * FILL_MAX_WARPS;

template <typename T>
__device__ __forceinline__ T load_src(const FillArgs<T>& a, long long idx);

template <>
__device__ __forceinline__ double load_src<double>(const FillArgs<double>& a, long long idx) {
    return a.src_d ? a.src_d[idx] : (a.src_hi ? (double)a.src_hi[idx] : 0.0);
}
template <>
__device__ __forceinline__ float load_src<float>(const FillArgs<float>& a, long long idx) {
    return a.src_hi ? a.src_hi[idx] : (a.src_d ? (float)a.src_d[idx] : 0.0f);
}

// Shared-memory layout (elements of T): factors Mt, Bt of all levels as
// [L][C][CP] with CP = C+1 (padded row), then per hole segment X, Y and a
// staging block V, each [R][CP].
__host__ __device__ constexpr int fill_cp(int C) { return C + 1; }

// acc[t] += sum_k F[k][c] * V[t*vs + k] for t < ROWS (V rows 16-byte aligned, padded column zero).
template <typename T, int C, int ROWS>
__device__ __forceinline__ void fill_matvec(const T* __restrict__ F, const T* __restrict__ V, int vs, int c, T* acc) {
    constexpr int CP = fill_cp(C);
    if constexpr (sizeof(T) == 4 && (C + 1) % 4 == 0) {
#pragma unroll
        for (int k = 0; k < C + 1; k += 4) {
            const T m0 = F[(k + 0) * CP + c];
            const T m1 = F[(k + 1) * CP + c];
            const T m2 = F[(k + 2) * CP + c];
            const T m3 = (k + 3 < C) ? F[(k + 3) * CP + c] : T(0);
#pragma unroll
            for (int t = 0; t < ROWS; ++t) {
                const float4 v = *reinterpret_cast<const float4*>(V + t * vs + k);
                acc[t] += m0 * v.x + m1 * v.y + m2 * v.z + m3 * v.w;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const T m = F[k * CP + c];
#pragma unroll
            for (int t = 0; t < ROWS; ++t) acc[t] += m * V[t * vs + k];
        }
    }
}

// Row counts of a level are 2^q or 2^q - 1: dispatch them to compile-time loops.
template <typename T, int C>
__device__ __forceinline__ void fill_matvec_n(int rows, const T* F, const T* V, int vs, int c, T* acc) {
    switch (rows) {
        case 1: fill_matvec<T, C, 1>(F, V, vs, c, acc); break;
        case 2: if constexpr (C >= 2) fill_matvec<T, C, 2>(F, V, vs, c, acc); break;
        case 3: if constexpr (C >= 3) fill_matvec<T, C, 3>(F, V, vs, c, acc); break;
        case 4: if constexpr (C >= 4) fill_matvec<T, C, 4>(F, V, vs, c, acc); break;
        case 7: if constexpr (C >= 7) fill_matvec<T, C, 7>(F, V, vs, c, acc); break;
        case 8: if constexpr (C >= 8) fill_matvec<T, C, 8>(F, V, vs, c, acc); break;
        case 15: if constexpr (C >= 15) fill_matvec<T, C, 15>(F, V, vs, c, acc); break;
        case 16: if constexpr (C >= 16) fill_matvec<T, C, 16>(F, V, vs, c, acc); break;
        default: break;
    }
}

template <typename T, int C>
__global__ void __launch_bounds__(FILL_MAX_THREADS)
fill_holes_kernel(FillArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    constexpr int R = C;
    constexpr int CP = fill_cp(C);
    constexpr int S = C + 1;                    // lanes per hole segment
    constexpr int SEGS = 32 / S;                // holes per warp
    constexpr int L = (C == 1) ? 1 : (C == 3) ? 2 : (C == 7) ? 3 : (C == 15) ? 4 : 5;
    constexpr int FSZ = C * CP;                 // one padded C x C factor
    constexpr int SEG = 3 * R * CP;             // X, Y, V per segment
    T* sMt = sm;
    T* sBt = sMt + L * FSZ;
    T* work = sBt + L * FSZ;
    __shared__ T sW[2][kMaxLevels];
    for (int e = threadIdx.x; e < L * C * C; e += blockDim.x) {
        const int l = e / (C * C), r = (e / C) % C, c = e % C;
        sMt[l * FSZ + r * CP + c] = a.Mt[e];
        sBt[l * FSZ + r * CP + c] = a.Bt[e];
    }
    if (threadIdx.x < kMaxLevels) {
        sW[0][threadIdx.x] = a.wl[threadIdx.x];
        sW[1][threadIdx.x] = a.wr[threadIdx.x];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = lane / S, c = lane % S;     // c == C: padding lane (keeps the zero column)
    T* X = work + (warp * SEGS + seg) * SEG;
    T* Y = X + R * CP;
    T* V = Y + R * CP;
    // The padding column of X and V stays zero (the float4 mat-vec reads it).
    if (c == C) {
        for (int y = 0; y < R; ++y) { X[y * CP + C] = T(0); V[y * CP + C] = T(0); }
    }
    const Geometry& g = a.g;
    const int N = g.N, n = a.n, mc = g.mc;
    const long long nholes = (long long)mc * mc;
    const T cw = (T)a.sten.cw, ce = (T)a.sten.ce, cs = (T)a.sten.cs, cn = (T)a.sten.cn;
    const int warps_cta = blockDim.x >> 5;
    const long long warps_total = (long long)gridDim.x * warps_cta;
    const long long gwarp = (long long)blockIdx.x * warps_cta + warp;
    // Homogeneous mode: the right-hand side is -A_hs z, i.e. the skeleton values
    // around the hole times the stencil.  Lane c < C fetches four of them (left
    // and right of row c, below and above column c); the next hole's four are
    // loaded while the current hole is solved.
    const bool homog = a.mode == FILL_HOMOGENEOUS;
    const long long hstep = warps_total * SEGS;
    auto load_ring = [&](long long hole, T* v) {
        if (c < C && hole < nholes) {
            const int bi = (int)(hole % mc), bj = (int)(hole / mc);
            const long long row = (long long)(bj * n + c + 1) * N;
            v[0] = a.z[row + bi * n];                                   // left of row c
            v[1] = a.z[row + bi * n + n];                               // right of row c
            v[2] = a.z[(long long)(bj * n) * N + bi * n + c + 1];       // below column c
            v[3] = a.z[(long long)(bj * n + n) * N + bi * n + c + 1];   // above column c
        } else {
            v[0] = v[1] = v[2] = v[3] = T(0);
        }
    };
    T ring_next[4];
    if (homog) load_ring(gwarp * SEGS + seg, ring_next);
    for (long long base = gwarp * SEGS; base < nholes; base += hstep) {
        const long long hole = base + seg;
        const bool hole_ok = c < C && hole < nholes;
        const int bi = hole_ok ? (int)(hole % mc) : 0, bj = hole_ok ? (int)(hole / mc) : 0;
        const int gx = bi * n + c + 1;          // grid x of this lane's column
        // Right-hand side of the hole system: P b - P A (skeleton).
        if (homog) {
            T ring[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) ring[q] = ring_next[q];
            load_ring(hole + hstep, ring_next);
            if (hole_ok) {
#pragma unroll
                for (int y = 0; y < R; ++y) X[y * CP + c] = T(0);
                X[c] = -cs * ring[2];
                X[(R - 1) * CP + c] -= cn * ring[3];
            }
            __syncwarp();
            if (hole_ok) {
                X[c * CP] -= cw * ring[0];
                X[c * CP + C - 1] -= ce * ring[1];
            }
        } else if (hole_ok) {
#pragma unroll
            for (int y = 1; y <= R; ++y) {
                const long long gidx = (long long)(bj * n + y) * N + gx;
                T f = T(0);
                if (a.mode == FILL_WITH_SOURCE || a.mode == FILL_ARRAY || a.mode == FILL_RESIDUAL_TO_U)
                    f = load_src<T>(a, gidx);
                if (a.mode == FILL_WITH_SOURCE || a.mode == FILL_HOMOGENEOUS) {
                    if (c == 0) f -= cw * a.z[gidx - 1];
                    if (c == C - 1) f -= ce * a.z[gidx + 1];
                    if (y == 1) f -= cs * a.z[gidx - N];
                    if (y == R) f -= cn * a.z[gidx + N];
                }
                X[(y - 1) * CP + c] = f;
            }
        }
        __syncwarp();
        // Forward reduction: f_i -= M (wl f_{i-s} + wr f_{i+s}).
#pragma unroll
        for (int l = 0; l + 1 < L; ++l) {
            const int s = 1 << l;
            const int nrows = ((R + 1) >> (l + 1)) - 1;
            const T wl = sW[0][l], wr = sW[1][l];
            if (hole_ok) {
                for (int t = 0; t < nrows; ++t) {
                    const int i = 2 * s * (t + 1);
                    V[t * CP + c] = wl * X[(i - s - 1) * CP + c] + wr * X[(i + s - 1) * CP + c];
                }
            }
            __syncwarp();
            if (hole_ok) {
                T acc[(R + 1) / 2];
#pragma unroll
                for (int t = 0; t < (R + 1) / 2; ++t) acc[t] = T(0);
                fill_matvec_n<T, C>(nrows, sMt + l * FSZ, V, CP, c, acc);
                for (int t = 0; t < nrows; ++t) {
                    const int i = 2 * s * (t + 1);
                    X[(i - 1) * CP + c] -= acc[t];
                }
            }
            __syncwarp();
        }
        // Back substitution: x_i = B^{-1} f_i - M (wl x_{i-s} + wr x_{i+s}).
#pragma unroll
        for (int l = L - 1; l >= 0; --l) {
            const int s = 1 << l;
            const int nrows = (R + 1) >> (l + 1);
            const T wl = sW[0][l], wr = sW[1][l];
            if (hole_ok) {
                for (int t = 0; t < nrows; ++t) {
                    const int i = s * (2 * t + 1);
                    T v = T(0);
                    if (i - s >= 1) v += wl * Y[(i - s - 1) * CP + c];
                    if (i + s <= R) v += wr * Y[(i + s - 1) * CP + c];
                    V[t * CP + c] = v;
                }
            }
            __syncwarp();
            if (hole_ok) {
                // B^{-1} f_i reads rows i = s(2t+1) of X: a strided view (s-1, 3s-1, ...) * CP.
                T acc[(R + 1) / 2];
#pragma unroll
                for (int t = 0; t < (R + 1) / 2; ++t) acc[t] = T(0);
                fill_matvec_n<T, C>(nrows, sBt + l * FSZ, X + (s - 1) * CP, 2 * s * CP, c, acc);
                T acc2[(R + 1) / 2];
#pragma unroll
                for (int t = 0; t < (R + 1) / 2; ++t) acc2[t] = T(0);
                fill_matvec_n<T, C>(nrows, sMt + l * FSZ, V, CP, c, acc2);
                for (int t = 0; t < nrows; ++t) {
                    const int i = s * (2 * t + 1);
                    Y[(i - 1) * CP + c] = acc[t] - acc2[t];
                }
            }
            __syncwarp();
        }
        // Write the hole values.
        if (hole_ok) {
#pragma unroll
            for (int y = 1; y <= R; ++y) {
                const long long gidx = (long long)(bj * n + y) * N + gx;
                const T v = Y[(y - 1) * CP + c];
                if (a.mode == FILL_RESIDUAL_TO_U) {
                    if (a.U) a.U[gidx] += __double2ll_rn((double)v * a.fixed_scale);
                    else a.u_d[gidx] += (double)v;
                } else if (a.out_d) {
                    a.out_d[gidx] = (double)v;
                } else {
                    a.out[gidx] = v;
                }
            }
        }
        __syncwarp();
    }
}

}  // namespace

namespace {
size_t fill_factor_bytes(size_t esz, int n, int L) {
    const size_t C = (size_t)(n - 1), CP = (size_t)fill_cp((int)C);
    return esz * 2 * (size_t)L * C * CP;
}
size_t fill_warp_bytes(size_t esz, int n) {
    const size_t C = (size_t)(n - 1), CP = (size_t)fill_cp((int)C);
    return esz * (32 / (C + 1)) * 3 * C * CP;
}
int fill_warps(size_t esz, int n, int L) {
    const size_t budget = 227 * 1024;
    const size_t f = fill_factor_bytes(esz, n, L), w = fill_warp_bytes(esz, n);
    if (f + w > budget) return 0;
    const size_t k = (budget - f) / w;
    return (int)(k < (size_t)FILL_MAX_WARPS ? k : (size_t)FILL_MAX_WARPS);
}
}  // namespace

// Shared memory of one fill CTA with at least one warp (0-fit test by the caller).
template <typename T>
size_t fill_smem_bytes(int n, int L) {
    return fill_factor_bytes(sizeof(T), n, L) + fill_warp_bytes(sizeof(T), n);
}

template <typename T, int C>
cudaError_t fill_holes_launch(const FillArgs<T>& a, int num_sms, cudaStream_t st) {
    const int max_warps = fill_warps(sizeof(T), a.n, a.L);
    if (max_warps < 1) return cudaErrorInvalidValue;
    const int warps = a.warps > 0 && a.warps < max_warps ? a.warps : max_warps;
    const size_t smem = fill_factor_bytes(sizeof(T), a.n, a.L) + (size_t)warps * fill_warp_bytes(sizeof(T), a.n);
    cudaError_t e = cudaFuncSetAttribute(fill_holes_kernel<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fill_holes_kernel<T, C>, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const long long nholes = (long long)a.g.mc * a.g.mc;
    const long long segs = 32 / a.n;
    const long long per_cta = (long long)warps * segs;
    long long grid = (long long)num_sms * per_sm;
    const long long need = (nholes + per_cta - 1) / per_cta;
    if (grid > need) grid = need;
    fill_holes_kernel<T, C><<<(unsigned)grid, 32 * warps, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t fill_holes(const FillArgs<T>& a, int num_sms, cudaStream_t st) {
    switch (a.n) {
        case 2: return fill_holes_launch<T, 1>(a, num_sms, st);
        case 4: return fill_holes_launch<T, 3>(a, num_sms, st);
        case 8: return fill_holes_launch<T, 7>(a, num_sms, st);
        case 16: return fill_holes_launch<T, 15>(a, num_sms, st);
        case 32: return fill_holes_launch<T, 31>(a, num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}

template size_t fill_smem_bytes<float>(int, int);
template size_t fill_smem_bytes<double>(int, int);
template cudaError_t fill_holes<float>(const FillArgs<float>&, int, cudaStream_t);
template cudaError_t fill_holes<double>(const FillArgs<double>&, int, cudaStream_t);

}  // namespace asdsm
