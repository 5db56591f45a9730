// Exact direct solves of the separable submesh systems of ASDSM on sm_103a.
//
// Every system of eq. (2.4) is block tridiagonal Toeplitz along its "row"
// axis (R = 2^L - 1 rows, each a vector of C unknowns along the other axis):
//     a x_{i-1} + (d I + T) x_i + c x_{i+1} = f_i.
// Block cyclic reduction (BCR) with the per-level factors of host_math.cu:
//   forward, level l = 0..L-2 (s = 2^l), rows i = 2s, 4s, ...:
//       f_i <- f_i - P_l f_{i-s} - Q_l f_{i+s}
//   backward, level l = L-1..0, rows i = s, 3s, 5s, ...:
//       x_i  = B_l^{-1} f_i - P_l x_{i-s} - Q_l x_{i+s}
// (P_l, Q_l, B_l^{-1} are functions of T and commute, so the back-substitution
// reuses the forward factors).  Row 0 and row R+1 are zero.
//
// bcr_level_kernel: one launch per level, a CTA computes a TR x TC tile of
// output rows x columns and streams the C x C factors through shared memory
// in KT-wide slices.  Used for the anisotropic families (R = N_f rows).
// fill_holes_kernel: the Filler of Algorithm 3, all levels of one hole in
// shared memory; persistent CTAs keep every level's factors resident and walk
// over the holes.
#include "asdsm_internal.h"
#include <cuda_runtime.h>

namespace asdsm {

namespace {

constexpr int TR = 8;      // output rows per CTA
constexpr int TC = 32;     // output columns per CTA
constexpr int KT = 32;     // reduction slice

template <typename T, bool kBackward>
__global__ void __launch_bounds__(TR * TC)
bcr_level_kernel(BcrSys<T> g0, BcrSys<T> g1, int ngroups, int level) {
    // blockIdx.z enumerates (group, system); blockIdx.y row tiles; blockIdx.x column tiles.
    int z = blockIdx.z;
    const BcrSys<T>* gp = &g0;
    if (ngroups > 1 && z >= g0.nsys) { gp = &g1; z -= g0.nsys; }
    const BcrSys<T>& g = *gp;
    if (z >= g.nsys) return;
    const int R = g.R, C = g.C;
    const int s = 1 << level;
    // Output rows of this level (1-based): forward i = 2s*t (t = 1..), backward i = s*(2t-1).
    const int nrows = kBackward ? ((R + 1) >> (level + 1)) : (((R + 1) >> (level + 1)) - 1);
    const int t0 = blockIdx.y * TR;
    if (t0 >= nrows) return;
    const int c0 = blockIdx.x * TC;
    const size_t n2 = (size_t)C * C;
    const T* Pt = g.Pt + (size_t)level * n2;
    const T* Qt = g.Qt + (size_t)level * n2;
    const T* Bt = g.Bt + (size_t)level * n2;
    T* X = g.X + (size_t)z * g.stride;
    T* Y = g.Y + (size_t)z * g.stride;

    __shared__ T sP[KT][TC], sQ[KT][TC], sB[kBackward ? KT : 1][TC];
    __shared__ T sL[TR][KT], sR[TR][KT], sM[kBackward ? TR : 1][KT];

    const int tc = threadIdx.x, tr = threadIdx.y;
    const int row_t = t0 + tr;                     // 0-based index into this level's rows
    const bool row_ok = row_t < nrows;
    const int i = kBackward ? s * (2 * row_t + 1) : 2 * s * (row_t + 1);   // 1-based row
    const int col = c0 + tc;
    const T* src = kBackward ? Y : X;              // neighbours: solved rows (bwd) or reduced rhs (fwd)
    T acc = T(0);
    for (int k0 = 0; k0 < C; k0 += KT) {
        // Factor slices: [k][c] layout, threads along c.
        for (int kk = tr; kk < KT; kk += TR) {
            const int k = k0 + kk;
            const bool ok = (k < C) && (col < C);
            sP[kk][tc] = ok ? Pt[(size_t)k * C + col] : T(0);
            sQ[kk][tc] = ok ? Qt[(size_t)k * C + col] : T(0);
            if (kBackward) sB[kk][tc] = ok ? Bt[(size_t)k * C + col] : T(0);
        }
        // Neighbour rows i-s, i+s (and row i for the backward B^{-1} f_i term).
        {
            const int k = k0 + tc;
            const bool kok = row_ok && (k < C);
            const int il = i - s, ir = i + s;
            sL[tr][tc] = (kok && il >= 1) ? src[(size_t)(il - 1) * C + k] : T(0);
            sR[tr][tc] = (kok && ir <= R) ? src[(size_t)(ir - 1) * C + k] : T(0);
            if (kBackward) sM[tr][tc] = kok ? X[(size_t)(i - 1) * C + k] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < KT; ++kk) {
            acc -= sP[kk][tc] * sL[tr][kk];
            acc -= sQ[kk][tc] * sR[tr][kk];
            if (kBackward) acc += sB[kk][tc] * sM[tr][kk];
        }
        __syncthreads();
    }
    if (row_ok && col < C) {
        if (kBackward) {
            Y[(size_t)(i - 1) * C + col] = acc;
        } else {
            X[(size_t)(i - 1) * C + col] += acc;
        }
    }
}

template <typename T, bool kBackward>
cudaError_t launch_level(const BcrSys<T>* groups, int ngroups, int level, cudaStream_t st) {
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
    dim3 grid((maxC + TC - 1) / TC, (maxRows + TR - 1) / TR, nsys);
    dim3 block(TC, TR);
    BcrSys<T> g1 = ngroups > 1 ? groups[1] : groups[0];
    bcr_level_kernel<T, kBackward><<<grid, block, 0, st>>>(groups[0], g1, ngroups, level);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t bcr_solve(const BcrSys<T>* groups, int ngroups, cudaStream_t st) {
    if (ngroups < 1 || ngroups > 2) return cudaErrorInvalidValue;
    int L = 0;
    for (int q = 0; q < ngroups; ++q) L = groups[q].L > L ? groups[q].L : L;
    for (int q = 0; q < ngroups; ++q)
        if (groups[q].L != L) return cudaErrorInvalidValue;   // groups in one call share the level count
    cudaError_t e;
    for (int l = 0; l + 1 < L; ++l)
        if ((e = launch_level<T, false>(groups, ngroups, l, st)) != cudaSuccess) return e;
    for (int l = L - 1; l >= 0; --l)
        if ((e = launch_level<T, true>(groups, ngroups, l, st)) != cudaSuccess) return e;
    return cudaSuccess;
}

template cudaError_t bcr_solve<float>(const BcrSys<float>*, int, cudaStream_t);
template cudaError_t bcr_solve<double>(const BcrSys<double>*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Fused hole fill (Algorithm 3).
// ---------------------------------------------------------------------------
namespace {

constexpr int FILL_THREADS = 256;

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

template <typename T>
__global__ void __launch_bounds__(FILL_THREADS)
fill_holes_kernel(FillArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int C = a.n - 1;          // unknowns per hole row and per hole column
    const int R = C;
    const int L = a.L;
    const size_t n2 = (size_t)C * C;
    T* sPt = sm;
    T* sQt = sPt + L * n2;
    T* sBt = sQt + L * n2;
    T* sX = sBt + L * n2;
    T* sY = sX + (size_t)R * C;
    // Factors of every level stay resident for all holes this CTA visits.
    for (size_t e = threadIdx.x; e < L * n2; e += blockDim.x) {
        sPt[e] = a.Pt[e];
        sQt[e] = a.Qt[e];
        sBt[e] = a.Bt[e];
    }
    const Geometry& g = a.g;
    const int N = g.N, n = a.n, mc = g.mc;
    const long long nholes = (long long)mc * mc;
    const T cw = (T)a.sten.cw, ce = (T)a.sten.ce, cs = (T)a.sten.cs, cn = (T)a.sten.cn;
    __syncthreads();
    for (long long hole = blockIdx.x; hole < nholes; hole += gridDim.x) {
        const int bi = (int)(hole % mc), bj = (int)(hole / mc);
        const int gx0 = bi * n, gy0 = bj * n;     // hole-local (x,y) in 1..n-1 -> grid (gx0+x, gy0+y)
        // Right-hand side of step 2: P b + c with c = -P A (skeleton).
        for (int e = threadIdx.x; e < R * C; e += blockDim.x) {
            const int y = e / C + 1, x = e % C + 1;
            const long long gidx = (long long)(gy0 + y) * N + (gx0 + x);
            T f = T(0);
            if (a.mode == FILL_WITH_SOURCE || a.mode == FILL_ARRAY || a.mode == FILL_RESIDUAL_TO_U)
                f = load_src<T>(a, gidx);
            if (a.mode == FILL_WITH_SOURCE || a.mode == FILL_HOMOGENEOUS) {
                if (x == 1) f -= cw * a.z[gidx - 1];
                if (x == C) f -= ce * a.z[gidx + 1];
                if (y == 1) f -= cs * a.z[gidx - N];
                if (y == C) f -= cn * a.z[gidx + N];
            }
            sX[e] = f;
        }
        __syncthreads();
        // Forward reduction.
        for (int l = 0; l + 1 < L; ++l) {
            const int s = 1 << l;
            const int nrows = ((R + 1) >> (l + 1)) - 1;
            const T* P = sPt + l * n2;
            const T* Q = sQt + l * n2;
            for (int e = threadIdx.x; e < nrows * C; e += blockDim.x) {
                const int t = e / C, c = e % C;
                const int i = 2 * s * (t + 1);
                const T* fl = sX + (size_t)(i - s - 1) * C;
                const T* fr = sX + (size_t)(i + s - 1) * C;   // i + s <= R always at these levels
                T acc = T(0);
                for (int k = 0; k < C; ++k) acc += P[(size_t)k * C + c] * fl[k] + Q[(size_t)k * C + c] * fr[k];
                sY[(size_t)(i - 1) * C + c] = acc;            // stage, rows i are written below
            }
            __syncthreads();
            for (int e = threadIdx.x; e < nrows * C; e += blockDim.x) {
                const int t = e / C, c = e % C;
                const int i = 2 * s * (t + 1);
                sX[(size_t)(i - 1) * C + c] -= sY[(size_t)(i - 1) * C + c];
            }
            __syncthreads();
        }
        // Back substitution.
        for (int l = L - 1; l >= 0; --l) {
            const int s = 1 << l;
            const int nrows = (R + 1) >> (l + 1);
            const T* P = sPt + l * n2;
            const T* Q = sQt + l * n2;
            const T* B = sBt + l * n2;
            for (int e = threadIdx.x; e < nrows * C; e += blockDim.x) {
                const int t = e / C, c = e % C;
                const int i = s * (2 * t + 1);
                const T* f = sX + (size_t)(i - 1) * C;
                T acc = T(0);
                for (int k = 0; k < C; ++k) acc += B[(size_t)k * C + c] * f[k];
                if (i - s >= 1) {
                    const T* xl = sY + (size_t)(i - s - 1) * C;
                    for (int k = 0; k < C; ++k) acc -= P[(size_t)k * C + c] * xl[k];
                }
                if (i + s <= R) {
                    const T* xr = sY + (size_t)(i + s - 1) * C;
                    for (int k = 0; k < C; ++k) acc -= Q[(size_t)k * C + c] * xr[k];
                }
                sY[(size_t)(i - 1) * C + c] = acc;
            }
            __syncthreads();
        }
        // Step 3: write the hole values.
        for (int e = threadIdx.x; e < R * C; e += blockDim.x) {
            const int y = e / C + 1, x = e % C + 1;
            const long long gidx = (long long)(gy0 + y) * N + (gx0 + x);
            const T v = sY[e];
            if (a.mode == FILL_RESIDUAL_TO_U) {
                if (a.U) a.U[gidx] += __double2ll_rn((double)v * a.fixed_scale);
                else a.u_d[gidx] += (double)v;
            } else if (a.mode == FILL_ARRAY && a.out_d) {
                a.out_d[gidx] = (double)v;
            } else {
                a.out[gidx] = v;
            }
        }
        __syncthreads();
    }
}

}  // namespace

template <typename T>
size_t fill_smem_bytes(int n, int L) {
    const size_t C = (size_t)(n - 1);
    return sizeof(T) * (3 * (size_t)L * C * C + 2 * C * C);
}

template <typename T>
cudaError_t fill_holes(const FillArgs<T>& a, int num_sms, cudaStream_t st) {
    const size_t smem = fill_smem_bytes<T>(a.n, a.L);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fill_holes_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fill_holes_kernel<T>, FILL_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const long long nholes = (long long)a.g.mc * a.g.mc;
    long long grid = (long long)num_sms * per_sm;
    if (grid > nholes) grid = nholes;
    fill_holes_kernel<T><<<(unsigned)grid, FILL_THREADS, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template size_t fill_smem_bytes<float>(int, int);
template size_t fill_smem_bytes<double>(int, int);
template cudaError_t fill_holes<float>(const FillArgs<float>&, int, cudaStream_t);
template cudaError_t fill_holes<double>(const FillArgs<double>&, int, cudaStream_t);

}  // namespace asdsm
