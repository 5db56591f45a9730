// Grid-wide kernels of the ASDSM sweep on sm_103a: the fine residual of
// Algorithm 4 (with the previous sweep's update fused in), the right-hand
// sides of eq. (2.4), the merge of Algorithm 2, the skeleton operator for the
// least-squares step length, reductions and conversions.
#include "asdsm_internal.h"
#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <atomic>

namespace asdsm {
namespace cg = cooperative_groups;

static std::atomic<long long> g_launches{0};
void note_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

// Tile of the residual kernels: RX x RY interior points per CTA, halo of one.
constexpr int RX = 64;
constexpr int RY = 16;
constexpr int RTHREADS = 256;

__device__ __forceinline__ int skel_kind(int i, int j, int n) {
    // 0 = hole, 1 = fc line only (y on a coarse line), 2 = cf column only, 3 = cross point
    // (n is a power of two)
    const bool fx = (i & (n - 1)) == 0, fy = (j & (n - 1)) == 0;
    return (fy ? 1 : 0) + (fx ? 2 : 0);
}

// Compact skeleton index of an interior skeleton point (i, j) (grid indices).
// Layout: fc lines [l][x] (l = j/n - 1, x = i - 1), then the cf columns
// without cross points, row by row: [yr][k] with yr the non-cross row rank.
__device__ __forceinline__ long long skel_index(int i, int j, const Geometry& g) {
    if ((j & (g.n - 1)) == 0) return (long long)((j >> g.ln) - 1) * g.Nf + (i - 1);
    const int yr = j - 1 - (j >> g.ln);     // rows y0 before j with (y0+1) % n == 0
    return (long long)g.Nc * g.Nf + (long long)yr * g.Nc + ((i >> g.ln) - 1);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Compensated FP32 sum over a warp of the pairs (hi, lo): the additions of the
// hi parts are exact through TwoSum (Knuth), their errors collect in lo, so the
// warp's sum costs no FP64 work (the FP64 pipe of this part runs at 1/64 of FP32).
__device__ __forceinline__ void warp_sum_pair(float& hi, float& lo) {
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const float s = hi + h2, bp = s - hi;
        const float err = (hi - (s - bp)) + (h2 - bp);
        hi = s;
        lo = lo + l2 + err;
    }
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Two-value block sum into partials[block][2].
__device__ void block_sum2(double a, double b, double* partials) {
    __shared__ double red[2][RTHREADS / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][w] = a; red[1][w] = b; }
    __syncthreads();
    if (w == 0) {
        a = lane < (RTHREADS / 32) ? red[0][lane] : 0.0;
        b = lane < (RTHREADS / 32) ? red[1][lane] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
        if (lane == 0) {
            const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
            partials[2 * blk] = a;
            partials[2 * blk + 1] = b;
        }
    }
}

template <typename T>
__device__ __forceinline__ void store_skeleton(const ResidOut& o, const Geometry& g, int i, int j, int kind, T v) {
    if (kind == 0) return;
    if (kind & 1) {   // on an fc line: BCR layout [x][line]
        reinterpret_cast<T*>(o.rfc)[(long long)(i - 1) * g.Nc + ((j >> g.ln) - 1)] = v;
    }
    if (kind & 2) {   // on a cf column: BCR layout [y][column]
        reinterpret_cast<T*>(o.rcf)[(long long)(j - 1) * g.Nc + ((i >> g.ln) - 1)] = v;
    }
    reinterpret_cast<T*>(o.rskel)[skel_index(i, j, g)] = v;
}

// ---------------------------------------------------------------------------
// FP64 residual (plain path): u_out = u_in + sum c_j z_j ; r = s - A u_out.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RTHREADS)
residual_fp64_kernel(const double* __restrict__ s, const double* u_in, double* u_out,
                     UpdateTerms up, Geometry g, Stencil c, ResidOut o) {
    __shared__ double tile[RY + 2][RX + 2];
    const int N = g.N;
    const int i0 = blockIdx.x * RX + 1, j0 = blockIdx.y * RY + 1;   // first interior point of the tile
    int count = up.count;
    const double* ucur = u_in;
    double* unxt = u_out;
    if (up.dyn) {
        if (!up.dyn->live || up.dyn->skip) return;
        count = up.dyn->count;
        if (up.dyn->par) { ucur = u_out; unxt = const_cast<double*>(u_in); }
    }
    // Load u (+ update) on the tile and its halo.  Ring points keep g (no update).
    for (int e = threadIdx.x; e < (RX + 2) * (RY + 2); e += RTHREADS) {
        const int ty = e / (RX + 2), tx = e % (RX + 2);
        const int i = i0 - 1 + tx, j = j0 - 1 + ty;
        double v = 0.0;
        if (i <= N - 1 && j <= N - 1) {
            const long long idx = (long long)j * N + i;
            v = ucur[idx];
            if (i >= 1 && j >= 1 && i <= N - 2 && j <= N - 2) {
                for (int q = 0; q < count; ++q)
                    v += (up.dyn ? up.dyn->coef[q] : up.coef[q]) * reinterpret_cast<const double*>(up.z[q])[idx];
            }
        }
        tile[ty][tx] = v;
    }
    __syncthreads();
    double sr = 0.0, sh = 0.0;
    for (int e = threadIdx.x; e < RX * RY; e += RTHREADS) {
        const int ty = e / RX, tx = e % RX;
        const int i = i0 + tx, j = j0 + ty;
        if (i > N - 2 || j > N - 2) continue;
        const long long idx = (long long)j * N + i;
        const double uc = tile[ty + 1][tx + 1];
        if (up.dyn ? count > 0 : (u_out != u_in || count > 0)) unxt[idx] = uc;
        const double Au = c.cc * uc + c.cw * tile[ty + 1][tx] + c.ce * tile[ty + 1][tx + 2]
                        + c.cs * tile[ty][tx + 1] + c.cn * tile[ty + 2][tx + 1];
        const double r = s[idx] - Au;
        const int kind = skel_kind(i, j, g.n);
        sr += r * r;
        if (kind == 0) sh += r * r;
        if (o.rfull) reinterpret_cast<double*>(o.rfull)[idx] = r;
        if (o.rskel) store_skeleton<double>(o, g, i, j, kind, r);
    }
    block_sum2(sr, sh, o.partials);
}

// ---------------------------------------------------------------------------
// Exact integer <-> FP32 conversions that stay off the FP64 pipe.  On GB300
// the 64-bit integer conversions (I2F.S64 / F2I.S64) run on the FP64 unit,
// which is 1/70 of the FP32 rate; these use only integer and FP32 ops.
// ---------------------------------------------------------------------------
// D = f2 * 2^44 + f1 * 2^22 + f0 exactly, f0, f1 in [0, 2^22), f2 in (-2^19, 2^19).
// Each piece becomes a float through the exponent-bias trick (x | 2^23 bits, minus 2^23).
__device__ __forceinline__ void split3(long long D, float& f2, float& f1, float& f0) {
    const unsigned lo = (unsigned)(unsigned long long)D;
    const unsigned hi = (unsigned)((unsigned long long)D >> 32);
    const unsigned p0 = lo & 0x3FFFFFu;
    const unsigned p1 = __funnelshift_r(lo, hi, 22) & 0x3FFFFFu;
    const int p2 = (int)hi >> 12;
    f0 = __fsub_rn(__uint_as_float(0x4B000000u | p0), 8388608.0f);
    f1 = __fsub_rn(__uint_as_float(0x4B000000u | p1), 8388608.0f);
    f2 = __fsub_rn(__int_as_float(0x4B400000 + p2), 12582912.0f);
}
// Nearest 64-bit integer of a float (|d| < 2^62): round to an integral float,
// then shift its significand into place.
__device__ __forceinline__ long long f2ll_rn(float d) {
    const float r = rintf(d);
    const unsigned b = __float_as_uint(r);
    const int E = (int)((b >> 23) & 0xFFu);
    if (E == 0) return 0;
    const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = E - 150;
    const long long v = sh >= 0 ? (m << sh) : (m >> (-sh));
    return (b >> 31) ? -v : v;
}

// ---------------------------------------------------------------------------
// Mixed residual: U (64-bit fixed point, u = U 2^-S) is the accumulator.
//   U_out = U_in + round(sum_j c_j z_j)              (the previous sweep's update, c_j carry 2^S)
//   A u   = kxx (2U_c - U_w - U_e) + kyy (2U_c - U_s - U_n) + kx (U_e - U_w) + ky (U_n - U_s)
// The integer differences are exact; each splits exactly into 22-bit pieces
// whose products with FP32 pairs of the coefficients (carrying 2^-S and the
// piece weight) are error-free (TwoProd) and summed with TwoSum, so
// r = s - A u keeps FP64-level accuracy with FP32/INT32 instructions only.
// Layout: a warp owns 30 output columns (lanes 1..30; lanes 0 and 31 carry the
// halo columns) and marches down MS_ROWS rows keeping rows j-1, j, j+1 in
// registers; x neighbours come from warp shuffles.
// ---------------------------------------------------------------------------
constexpr int MS_OUT = 30;
constexpr int MS_WARPS = 8;
constexpr int MS_ROWS = 32;
// Register budget: 4 resident CTAs per SM (64 registers); measured fastest of
// 1..6 and of 16/32/64 rows per warp at 4097^2.

struct UpdateF {
    const float* z[16];
    float c[16];
    int count;
    const DynUpdate* dyn;   // non-null: count and c come from the device, U_in/U_out are buffers 0/1
};

// Balanced two-digit split of a difference with |D| < 2^43:
// D = f1 2^22 + f0 exactly, f0, f1 integers in [-2^21, 2^21].
__device__ __forceinline__ void split2(long long D, float& f1, float& f0) {
    const unsigned lo = (unsigned)(unsigned long long)D;
    const int d0 = ((int)(lo << 10)) >> 10;                 // low 22 bits, sign-extended
    const unsigned long long R = (unsigned long long)(D - (long long)d0);   // low 22 bits zero
    const int d1 = (int)__funnelshift_r((unsigned)R, (unsigned)(R >> 32), 22);
    f0 = __fsub_rn(__int_as_float(0x4B400000 + d0), 12582912.0f);
    f1 = __fsub_rn(__int_as_float(0x4B400000 + d1), 12582912.0f);
}

// Raw loads of row j at column x (U and the pending directions), issued one
// row ahead of their use; finish_row applies the update (interior only: the
// direction values are zero elsewhere).
template <int CNT>
struct RowLoads {
    long long U;
    float z[CNT > 0 ? CNT : 1];
};

template <int CNT>
__device__ __forceinline__ void load_row(const long long* __restrict__ U_in, const UpdateF& up, int N, int x, int j,
                                         bool xin, bool xint, RowLoads<CNT>& r) {
    const long long idx = (long long)j * N + x;
    r.U = xin ? U_in[idx] : 0;
    const bool upd = xint && j >= 1 && j <= N - 2;
#pragma unroll
    for (int q = 0; q < CNT; ++q) r.z[q] = upd ? __ldg(up.z[q] + idx) : 0.0f;
}

template <int CNT>
__device__ __forceinline__ long long finish_row(const RowLoads<CNT>& r, const UpdateF& up) {
    if (CNT == 0) return r.U;
    float d = 0.0f;
#pragma unroll
    for (int q = 0; q < CNT; ++q) d = __fmaf_rn(up.c[q], r.z[q], d);
    return r.U + f2ll_rn(d);
}

__device__ __forceinline__ void acc_prod(float khi, float klo, float f, float& hi, float& err) {
    const float p = __fmul_rn(khi, f);
    float e = __fmaf_rn(khi, f, -p);
    e = __fmaf_rn(klo, f, e);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    err = __fadd_rn(err, __fadd_rn(t, e));
}

// The row march of one warp with CNT pending directions (a compile-time count,
// so the update loop has no per-point control flow).
template <int CNT>
__device__ __forceinline__ void resid_rows(const float* __restrict__ s_hi, const float* __restrict__ s_lo,
                                           const long long* __restrict__ U_in, long long* __restrict__ U_out,
                                           const UpdateF& up, const Geometry& g, const MixedCoefs& k,
                                           const ResidOut& o, int x, int j0, int j1, bool out_col,
                                           float& srf, float& shf, bool& ovf) {
    const int N = g.N;
    const bool xin = x >= 0 && x <= N - 1, xint = x >= 1 && x <= N - 2;
    RowLoads<CNT> ra;
    load_row<CNT>(U_in, up, N, x, j0 - 1, xin, xint, ra);
    long long um = finish_row<CNT>(ra, up);
    load_row<CNT>(U_in, up, N, x, j0, xin, xint, ra);
    long long uc = finish_row<CNT>(ra, up);
    load_row<CNT>(U_in, up, N, x, j0 + 1, xin, xint, ra);     // rows j0+1 .. j1+1 <= N-1 exist
    const long long lim = 1LL << 60;
    for (int j = j0; j <= j1; ++j) {
        const long long un = finish_row<CNT>(ra, up);
        if (j + 2 <= j1 + 1) load_row<CNT>(U_in, up, N, x, j + 2, xin, xint, ra);
        const long long idx = (long long)j * N + x;
        const float sh = out_col ? __ldg(s_hi + idx) : 0.0f, sl = out_col ? __ldg(s_lo + idx) : 0.0f;
        const long long uw = __shfl_up_sync(0xffffffffu, uc, 1);
        const long long ue = __shfl_down_sync(0xffffffffu, uc, 1);
        const long long D[4] = {2 * uc - uw - ue, 2 * uc - um - un, ue - uw, un - um};
        // Differences below 2^43 in modulus (the usual case: u is smooth on the
        // fine scale) need two 22-bit digits; otherwise the warp takes three.
        bool wide = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) wide |= (unsigned long long)(D[q] + (1LL << 43)) >= (1ULL << 44);
        float hi = 0.0f, err = 0.0f;
        if (__any_sync(0xffffffffu, out_col && wide)) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float f2, f1, f0;
                split3(D[q], f2, f1, f0);
                acc_prod(k.k2[q][0], k.k2[q][1], f2, hi, err);
                acc_prod(k.k1[q][0], k.k1[q][1], f1, hi, err);
                err = __fmaf_rn(k.k0[q], f0, err);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float f1, f0;
                split2(D[q], f1, f0);
                acc_prod(k.k1[q][0], k.k1[q][1], f1, hi, err);
                err = __fmaf_rn(k.k0[q], f0, err);
            }
        }
        if (out_col) {
            ovf |= (uc > lim) || (uc < -lim);
            if (CNT > 0) U_out[idx] = uc;
            // r = s - A u: TwoSum of the leading parts, then the small terms.
            const float a = sh, b = -hi;
            const float s = __fadd_rn(a, b);
            const float bb = __fsub_rn(s, a);
            const float t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
            const float rf = __fadd_rn(s, __fsub_rn(__fadd_rn(t, sl), err));
            const int kind = skel_kind(x, j, g.n);
            srf = __fmaf_rn(rf, rf, srf);
            if (kind == 0) shf = __fmaf_rn(rf, rf, shf);
            if (o.rfull) reinterpret_cast<float*>(o.rfull)[idx] = rf;
            if (o.rskel) store_skeleton<float>(o, g, x, j, kind, rf);
        }
        um = uc;
        uc = un;
    }
}

__global__ void __launch_bounds__(32 * MS_WARPS, 4)
residual_mixed_kernel(const float* __restrict__ s_hi, const float* __restrict__ s_lo,
                      const long long* U_in0, long long* U_out0,
                      UpdateF up, Geometry g, MixedCoefs k, ResidOut o, int* overflow) {
    const int N = g.N;
    const long long* U_in = U_in0;
    long long* U_out = U_out0;
    if (up.dyn) {
        if (!up.dyn->live || up.dyn->skip) return;
        up.count = up.dyn->count;
#pragma unroll
        for (int q = 0; q < 16; ++q) up.c[q] = up.dyn->cf[q];
        if (up.dyn->par) { U_in = U_out0; U_out = const_cast<long long*>(U_in0); }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = 1 + (blockIdx.x * MS_WARPS + warp) * MS_OUT + lane - 1;   // lane 0: west halo
    const bool out_col = lane >= 1 && lane <= MS_OUT && x <= N - 2;
    const int j0 = 1 + blockIdx.y * MS_ROWS;
    const int j1 = min(j0 + MS_ROWS - 1, N - 2);
    float srf = 0.0f, shf = 0.0f;
    bool ovf = false;
    switch (up.count) {
#define RESID_CASE(C) case C: resid_rows<C>(s_hi, s_lo, U_in, U_out, up, g, k, o, x, j0, j1, out_col, srf, shf, ovf); break;
        RESID_CASE(0) RESID_CASE(1) RESID_CASE(2) RESID_CASE(3) RESID_CASE(4) RESID_CASE(5) RESID_CASE(6)
        RESID_CASE(7) RESID_CASE(8) RESID_CASE(9) RESID_CASE(10) RESID_CASE(11) RESID_CASE(12)
        RESID_CASE(13) RESID_CASE(14) RESID_CASE(15) RESID_CASE(16)
#undef RESID_CASE
        default: break;
    }
    if (ovf) atomicOr(overflow, 1);
    // Block reduction of the two norms (8 warps).
    // Warp sums as compensated FP32 pairs; the block's sum in FP64 by one thread.
    __shared__ double red[2][MS_WARPS];
    float ah = srf, al = 0.0f, bh = shf, bl = 0.0f;
    warp_sum_pair(ah, al);
    warp_sum_pair(bh, bl);
    if (lane == 0) { red[0][warp] = (double)ah + (double)al; red[1][warp] = (double)bh + (double)bl; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < MS_WARPS; ++w) { a += red[0][w]; b += red[1][w]; }
        const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
        o.partials[2 * blk] = a;
        o.partials[2 * blk + 1] = b;
    }
}

// ---------------------------------------------------------------------------
// Right-hand sides on Omega^{h,H}, Omega^{H,h}, Omega^{H,H} with lifting.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void submesh_rhs_kernel(const double* __restrict__ s, const double* __restrict__ u, Geometry g,
                                   double ax, double ay, double bx, double by,
                                   T* bfc, T* bcf, T* bcc) {
    const int N = g.N, M = g.M, n = g.n, Nf = g.Nf, Nc = g.Nc;
    const double h = 1.0 / M, H = 1.0 / g.mc;
    const long long total = 2LL * Nf * Nc + (long long)Nc * Nc;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        int i, j;        // grid indices of the point
        double hx, hy;
        T* dst;
        long long di;
        if (e < (long long)Nf * Nc) {                 // fc: BCR layout [x][line]
            const int x = (int)(e / Nc), l = (int)(e % Nc);
            i = x + 1; j = (l + 1) * n; hx = h; hy = H; dst = bfc; di = e;
        } else if (e < 2LL * Nf * Nc) {               // cf: [y][column]
            const long long f = e - (long long)Nf * Nc;
            const int y = (int)(f / Nc), kcol = (int)(f % Nc);
            i = (kcol + 1) * n; j = y + 1; hx = H; hy = h; dst = bcf; di = f;
        } else {                                      // cc: [y][x]
            const long long f = e - 2LL * Nf * Nc;
            const int ly = (int)(f / Nc), kx = (int)(f % Nc);
            i = (kx + 1) * n; j = (ly + 1) * n; hx = H; hy = H; dst = bcc; di = f;
        }
        const int sx = (int)(hx * M + 0.5), sy = (int)(hy * M + 0.5);
        double v = s[(long long)j * N + i];
        if (i - sx == 0) v += (ax / (hx * hx) + bx / (2 * hx)) * u[(long long)j * N + 0];
        if (i + sx == M) v += (ax / (hx * hx) - bx / (2 * hx)) * u[(long long)j * N + M];
        if (j - sy == 0) v += (ay / (hy * hy) + by / (2 * hy)) * u[i];
        if (j + sy == M) v += (ay / (hy * hy) - by / (2 * hy)) * u[(long long)M * N + i];
        dst[di] = (T)v;
    }
}

// ---------------------------------------------------------------------------
// Algorithm 2.  merge_knots: the cross-point values of both anisotropic
// solutions, the chosen/extrapolated u_hat, the errors e and the spline
// moments of the correction along every coarse line.
// merge_write: every skeleton point gets its anisotropic value plus the spline
// correction and the merged skeleton is stored.
// ---------------------------------------------------------------------------
// 1/||u|| of the normalisation of Algorithm 1 (FP32 reciprocal square root on the mixed path:
// a single scale factor, and FP64 division and square root are slow on this part).
template <typename T>
__device__ __forceinline__ void inv_norms(const MergeArgs<T>& a, T* inv1, T* inv2) {
    if (a.re_mode) { *inv1 = T(1); *inv2 = T(1); return; }
    const double n1 = a.norms2[0], n2 = a.norms2[1];
    if constexpr (sizeof(T) == 4) {
        *inv1 = n1 > 0.0 ? rsqrtf((float)n1) : 1.0f;
        *inv2 = n2 > 0.0 ? rsqrtf((float)n2) : 1.0f;
    } else {
        *inv1 = n1 > 0.0 ? (T)(1.0 / sqrt(n1)) : T(1);
        *inv2 = n2 > 0.0 ? (T)(1.0 / sqrt(n2)) : T(1);
    }
}

// Knot errors and spline moments as one small GEMM per family:
//   M[line][r] = sum_q Sm[r][q] e[line][q]
// with the cross-point errors of Algorithm 2 formed from the cross points.  A
// cluster of MK_KS CTAs owns MK_L lines x MK_R moments; CTA rank k takes the
// k-th quarter of the knots, in chunks of MK_Q (half that for FP64).  Per chunk the cross values
// t1 (u_fc, [x][line] in Yfc) and t2 (u_cf, [y][column] in Ycf) are read as two
// tiles, each along its contiguous index, the errors formed in shared memory,
// and Sm (stored transposed, [knot q][moment r]) staged beside them; a thread
// accumulates 2 lines x 4 moments.  The partial tiles are summed in rank order
// through distributed shared memory.  The CTAs of the first moment block also
// store e.  One cluster wave covers the 4097^2 case (320 CTAs).
constexpr int MK_L = 32, MK_R = 64, MK_Q = 64, MK_KS = 4, MK_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(MK_THREADS) merge_knots_kernel(MergeArgs<T> a) {
    constexpr int MQ = sizeof(T) == 4 ? MK_Q : MK_Q / 2;   // knots per chunk (static shared memory <= 48 KB)
    cg::cluster_group cluster = cg::this_cluster();
    const int Nc = a.g.Nc, K = a.g.mc + 1, n = a.g.n;
    const int nlb = (Nc + MK_L - 1) / MK_L;
    const int rank = (int)(blockIdx.x % MK_KS), tile = (int)(blockIdx.x / MK_KS);
    const int fam = tile / nlb;                  // 0: fc lines, 1: cf columns
    const int l0 = (tile % nlb) * MK_L;
    const int r0 = blockIdx.y * MK_R;
    const bool store_e = blockIdx.y == 0;
    const int qs = (Nc + MK_KS - 1) / MK_KS;     // knots per rank
    const int qb = rank * qs, qe = min(Nc, qb + qs);
    // Ta: the cross value contiguous along the lines (fam 0: t1, fam 1: t2), then the
    // errors; Tb: the one contiguous along the knots; Tc: u_cc (Richardson mode only).
    // After the knot loop the buffer of Tb, Tc holds the partial tile.
    __shared__ T Ta[MQ][MK_L + 1];
    __shared__ __align__(16) T Tbc[2 * MQ * (MK_L + 1)];
    __shared__ __align__(16) T Ss[MQ][MK_R];
    __shared__ T inv_s[2];                       // the families' norm scales, once per block
    static_assert(MK_L * MK_R <= 2 * MQ * (MK_L + 1), "the partial tile fits the Tb, Tc buffer");
    T (*Tb)[MK_L + 1] = reinterpret_cast<T (*)[MK_L + 1]>(Tbc);
    T (*Tc)[MK_L + 1] = reinterpret_cast<T (*)[MK_L + 1]>(Tbc + MQ * (MK_L + 1));
    T (*Part)[MK_R] = reinterpret_cast<T (*)[MK_R]>(Tbc);
    const int tid = threadIdx.x;
    if (tid == 0) inv_norms(a, &inv_s[0], &inv_s[1]);
    const int choice = a.choice_dev ? *a.choice_dev : a.choice;
    const T* along_lines = fam == 0 ? a.Yfc : a.Ycf;   // [(q+1)n-1][line]
    const T* along_knots = fam == 0 ? a.Ycf : a.Yfc;   // [(line+1)n-1][q]
    const int tl = tid / (MK_R / 4), tr = tid % (MK_R / 4);   // lines 2 tl, 2 tl + 1; moments 4 tr .. + 3
    T acc[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = T(0);
    for (int q0 = qb; q0 < qe; q0 += MQ) {
        __syncthreads();                         // previous chunk consumed (and inv_s written)
        for (int e = tid; e < MQ * MK_L; e += MK_THREADS) {
            {
                const int qq = e / MK_L, li = e % MK_L, q = q0 + qq, line = l0 + li;
                const bool ok = q < qe && line < Nc;
                Ta[qq][li] = ok ? along_lines[((long long)(q + 1) * n - 1) * Nc + line] : T(0);
                // u_cc at (l, k): fam 0 (l = line, k = q) along the knots, fam 1 (l = q, k = line) here
                if (a.re_mode && fam == 1) Tc[qq][li] = ok ? a.Ycc[(long long)q * Nc + line] : T(0);
            }
            {
                const int li = e / MQ, qq = e % MQ, q = q0 + qq, line = l0 + li;
                const bool ok = q < qe && line < Nc;
                Tb[qq][li] = ok ? along_knots[((long long)(line + 1) * n - 1) * Nc + q] : T(0);
                if (a.re_mode && fam == 0) Tc[qq][li] = ok ? a.Ycc[(long long)line * Nc + q] : T(0);
            }
        }
        for (int e = tid; e < MQ * MK_R; e += MK_THREADS) {
            const int qq = e / MK_R, rr = e % MK_R, q = q0 + qq, r = r0 + rr;
            Ss[qq][rr] = (q < qe && r < K) ? __ldg(a.Sm + (long long)q * K + r) : T(0);
        }
        __syncthreads();
        const T inv1 = inv_s[0], inv2 = inv_s[1];
        for (int e = tid; e < MQ * MK_L; e += MK_THREADS) {
            const int qq = e / MK_L, li = e % MK_L, q = q0 + qq, line = l0 + li;
            const T A = Ta[qq][li], B = Tb[qq][li];
            const T t1 = (fam == 0 ? A : B) * inv1, t2 = (fam == 0 ? B : A) * inv2;
            T uh;
            if (a.re_mode) uh = t1 + t2 - Tc[qq][li];   // Richardson extrapolation (combination)
            else uh = choice ? t2 : t1;                 // random choice
            const T ev = fam == 0 ? uh - t1 : uh - t2;  // cross-point error (0 outside the ranges)
            Ta[qq][li] = ev;
            if (store_e && q < qe && line < Nc) {
                if (fam == 0) a.E1[(long long)line * Nc + q] = ev;      // E1[l][k]
                else a.E2[(long long)q * Nc + line] = ev;               // E2[l][k]
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int qq = 0; qq < MQ; ++qq) {
            const T e0 = Ta[qq][2 * tl], e1 = Ta[qq][2 * tl + 1];
            T sv4[4];
            if constexpr (sizeof(T) == 4) {
                const float4 v = *reinterpret_cast<const float4*>(&Ss[qq][4 * tr]);
                sv4[0] = v.x; sv4[1] = v.y; sv4[2] = v.z; sv4[3] = v.w;
            } else {
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) sv4[jj] = Ss[qq][4 * tr + jj];
            }
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                acc[0][jj] += sv4[jj] * e0;
                acc[1][jj] += sv4[jj] * e1;
            }
        }
    }
    __syncthreads();                             // the Tb, Tc buffer becomes the partial tile
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) Part[2 * tl + i][4 * tr + jj] = acc[i][jj];
    cluster.sync();                              // every rank's partial tile is complete
    // Rank k sums lines [k MK_L / MK_KS, (k + 1) MK_L / MK_KS) over the ranks, in rank order.
    constexpr int LPR = MK_L / MK_KS;
    const T* P[MK_KS];
#pragma unroll
    for (int j = 0; j < MK_KS; ++j) P[j] = cluster.map_shared_rank(&Part[0][0], j);
    for (int e = tid; e < LPR * MK_R; e += MK_THREADS) {
        const int li = rank * LPR + e / MK_R, rr = e % MK_R;
        T v = T(0);
#pragma unroll
        for (int j = 0; j < MK_KS; ++j) v += P[j][li * MK_R + rr];
        const int line = l0 + li, r = r0 + rr;
        if (line < Nc && r < K) {
            if (fam == 0) a.M1[(long long)line * K + r] = v;
            else a.M2[(long long)r * Nc + line] = v;
        }
    }
    cluster.sync();                              // no CTA leaves while its tile is read
}

// Weights of the not-a-knot spline with moments M and knot values (0, e.., 0) at
// fine offset p (0..n) of a coarse interval: S = w0 M_k + w1 M_{k+1} + w2 y_k + w3 y_{k+1},
// with t = pH/n, u = H - t: w0 = u^3/(6H) - Hu/6, w1 = t^3/(6H) - Ht/6, w2 = u/H, w3 = t/H.
template <typename T>
__device__ __forceinline__ void spline_weights(int p, int n, T H, T* w) {
    const T t = H * (T)p / (T)n;
    const T u = H - t;
    w[0] = u * u * u / (6 * H) - H * u / 6;
    w[1] = t * t * t / (6 * H) - H * t / 6;
    w[2] = u / H;
    w[3] = t / H;
}

// fc lines in tiles of MW_T lines x MW_X MW_T fine x through shared memory (Yfc
// is [x][line]: read along lines, written along x, both coalesced); then blocks
// of MW_Y cf rows (columns along the threads).  A thread's loads are issued
// before the block waits for the spline weights and norm scales, so that about
// one wave of blocks covers the skeleton.
constexpr int MW_T = 32, MW_X = 4, MW_Y = 8, MW_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(MW_THREADS) merge_write_kernel(MergeArgs<T> a, int nft) {
    const Geometry& g = a.g;
    const int Nf = g.Nf, Nc = g.Nc, n = g.n, N = g.N, K = g.mc + 1;
    const T H = T(1) / (T)g.mc;
    __shared__ T sw[33][4];                     // spline weights per fine offset p = 0..n (n <= 32)
    __shared__ T tile[MW_X][MW_T][MW_T + 1];    // [x][line]
    __shared__ T inv_s[2];                      // the families' norm scales, once per block
    for (int p = threadIdx.x; p <= n; p += blockDim.x) spline_weights<T>(p, n, H, sw[p]);
    if (threadIdx.x == 0) inv_norms(a, &inv_s[0], &inv_s[1]);
    const int tx = threadIdx.x % MW_T, ty = threadIdx.x / MW_T;
    if ((int)blockIdx.x < nft) {
        // fc line l, fine x: u_fc/||u_fc|| + Spline(e1); cross points too (written from fc).
        const int nxt = (Nf + MW_T * MW_X - 1) / (MW_T * MW_X);
        const int l0 = ((int)blockIdx.x / nxt) * MW_T, x0 = ((int)blockIdx.x % nxt) * MW_T * MW_X;
#pragma unroll
        for (int c = 0; c < MW_X; ++c)
#pragma unroll
            for (int xx = ty; xx < MW_T; xx += MW_THREADS / MW_T) {
                const int x = x0 + c * MW_T + xx, l = l0 + tx;
                tile[c][xx][tx] = (x < Nf && l < Nc) ? a.Yfc[(long long)x * Nc + l] : T(0);
            }
        __syncthreads();
        const T inv1 = inv_s[0];
#pragma unroll
        for (int c = 0; c < MW_X; ++c)
            for (int ll = ty; ll < MW_T; ll += MW_THREADS / MW_T) {
                const int l = l0 + ll, x = x0 + c * MW_T + tx;
                if (l >= Nc || x >= Nf) continue;
                const int i = x + 1, ki = i >> g.ln, p = i & (n - 1);
                T corr;
                const T yk = ki == 0 ? T(0) : a.E1[(long long)l * Nc + ki - 1];
                if (p == 0) {
                    corr = yk;                   // at a knot the spline interpolates exactly
                } else {
                    const T* Mv = a.M1 + (long long)l * K;
                    const T yk1 = ki + 1 >= g.mc ? T(0) : a.E1[(long long)l * Nc + ki];
                    corr = sw[p][0] * Mv[ki] + sw[p][1] * Mv[ki + 1] + sw[p][2] * yk + sw[p][3] * yk1;
                }
                a.z[(long long)((l + 1) * n) * N + i] = tile[c][tx][ll] * inv1 + corr;
            }
        return;
    }
    // cf points, MW_Y fine rows per block; the cross rows are skipped, their points
    // keep the fc value.  Columns k along the threads, in chunks of MW_THREADS.
    const int y0 = ((int)blockIdx.x - nft) * MW_Y;
    const int nkc = (Nc + MW_THREADS - 1) / MW_THREADS;
    for (int kc = 0; kc < nkc; ++kc) {
        const int k = kc * MW_THREADS + threadIdx.x;
        T yv[MW_Y], e0[MW_Y], e1[MW_Y], m0[MW_Y], m1[MW_Y];
#pragma unroll
        for (int u = 0; u < MW_Y; ++u) {
            const int y = y0 + u, j = y + 1, ki = j >> g.ln;
            const bool ok = y < Nf && k < Nc && (j & (n - 1)) != 0;
            yv[u] = ok ? a.Ycf[(long long)y * Nc + k] : T(0);
            e0[u] = ok && ki > 0 ? a.E2[(ki - 1) * Nc + k] : T(0);
            e1[u] = ok && ki + 1 < g.mc ? a.E2[ki * Nc + k] : T(0);
            m0[u] = ok ? a.M2[ki * Nc + k] : T(0);
            m1[u] = ok ? a.M2[(ki + 1) * Nc + k] : T(0);
        }
        if (kc == 0) __syncthreads();           // spline weights and norm scales ready
        const T inv2 = inv_s[1];
#pragma unroll
        for (int u = 0; u < MW_Y; ++u) {
            const int y = y0 + u, j = y + 1, p = j & (n - 1);
            if (y >= Nf || k >= Nc || p == 0) continue;
            const T corr = sw[p][0] * m0[u] + sw[p][1] * m1[u] + sw[p][2] * e0[u] + sw[p][3] * e1[u];
            const T val = yv[u] * inv2 + corr;
            if (a.zv) a.zv[(long long)j * (g.mc + 1) + k + 1] = val;
            else a.z[(long long)j * N + (k + 1) * n] = val;
        }
    }
}

// Stencil weights in the vectors' precision (rounded on the host: no FP64 work per element).
template <typename T>
struct StencilT { T cc, cw, ce, cs, cn; };

// q = A z at compact skeleton rows (z: full grid, zero ring).  A thread computes
// SA_E points with every load issued before the first use, so that about one
// wave of blocks covers the skeleton: fc lines in chunks of 256 SA_E points
// (consecutive threads, consecutive x), then blocks of SA_E cf rows off the fc
// lines (one row per step, columns along the threads).  Grid offsets fit 32-bit
// integers (N <= 32769).
constexpr int SA_E = 8;

template <typename T>
__global__ void __launch_bounds__(256) skeleton_apply_kernel(const T* __restrict__ z, Geometry g, StencilT<T> c,
                                                            T* __restrict__ q, int nxb) {
    const int N = g.N, n = g.n, Nf = g.Nf, Nc = g.Nc;
    const int b = (int)blockIdx.x, nfb = Nc * nxb;
    T v[SA_E][5];
    int out[SA_E];
    if (b < nfb) {
        const int l = b / nxb, x0 = (b % nxb) * 256 * SA_E + threadIdx.x;
        const int row = ((l + 1) * n) * N + 1;
#pragma unroll
        for (int u = 0; u < SA_E; ++u) {
            const int x = x0 + 256 * u;
            out[u] = x < Nf ? l * Nf + x : -1;
            const int idx = row + (x < Nf ? x : 0);
            v[u][0] = z[idx]; v[u][1] = z[idx - 1]; v[u][2] = z[idx + 1]; v[u][3] = z[idx - N]; v[u][4] = z[idx + N];
        }
    } else {
        const int yr0 = (b - nfb) * SA_E, nyr = Nf - Nc;
#pragma unroll
        for (int u = 0; u < SA_E; ++u) {
            const int yr = yr0 + u, k = threadIdx.x;
            const bool ok = yr < nyr && k < Nc;
            out[u] = ok ? Nc * Nf + yr * Nc + k : -1;
            const int j = ok ? yr + yr / (n - 1) + 1 : n + 1;
            const int idx = j * N + ((ok ? k : 0) + 1) * n;
            v[u][0] = z[idx]; v[u][1] = z[idx - 1]; v[u][2] = z[idx + 1]; v[u][3] = z[idx - N]; v[u][4] = z[idx + N];
        }
    }
#pragma unroll
    for (int u = 0; u < SA_E; ++u)
        if (out[u] >= 0) q[out[u]] = c.cc * v[u][0] + c.cw * v[u][1] + c.ce * v[u][2] + c.cs * v[u][3] + c.cn * v[u][4];
}

// The same for any N_c: one point per thread, grid-strided.
template <typename T>
__global__ void skeleton_apply_generic_kernel(const T* __restrict__ z, Geometry g, StencilT<T> c, T* __restrict__ q) {
    const int N = g.N, n = g.n, Nf = g.Nf, Nc = g.Nc;
    const int nfc = Nc * Nf, skel = (int)g.skel;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < skel; e += gridDim.x * blockDim.x) {
        int i, j;
        if (e < nfc) {
            i = e % Nf + 1;
            j = (e / Nf + 1) * n;
        } else {
            const int f = e - nfc;
            const int yr = f / Nc, k = f % Nc;
            j = yr + yr / (n - 1) + 1;
            i = (k + 1) * n;
        }
        const int idx = j * N + i;
        q[e] = c.cc * z[idx] + c.cw * z[idx - 1] + c.ce * z[idx + 1] + c.cs * z[idx - N] + c.cn * z[idx + N];
    }
}

template <typename T>
struct CombineArgs { const T* Qp[16]; T beta[16]; };

// out = (q - sum_j beta_j Qp_j) * inv_nu on a grid-strided range, in the
// vectors' own precision and in the same order per element; FP32 vectors are
// read and written four at a time (the arrays are 16-byte aligned), the tail
// one by one.  K (the directions, <= 15) is a template parameter: no branch
// per direction and every load of an element issued before the first use.
template <typename T, int K>
__device__ __forceinline__ void combine_range(const T* __restrict__ q, const CombineArgs<T>& c, const T* beta,
                                              T inu, long long n, T* __restrict__ out) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long done = 0;
    if constexpr (sizeof(T) == 4) {
        const long long n4 = n >> 2;
        for (long long e = tid; e < n4; e += stride) {
            float4 v = __ldg(reinterpret_cast<const float4*>(q) + e);
            float4 p[K > 0 ? K : 1];
#pragma unroll
            for (int j = 0; j < K; ++j) p[j] = __ldg(reinterpret_cast<const float4*>(c.Qp[j]) + e);
#pragma unroll
            for (int j = 0; j < K; ++j) {
                v.x -= beta[j] * p[j].x;
                v.y -= beta[j] * p[j].y;
                v.z -= beta[j] * p[j].z;
                v.w -= beta[j] * p[j].w;
            }
            v.x *= inu; v.y *= inu; v.z *= inu; v.w *= inu;
            reinterpret_cast<float4*>(out)[e] = v;
        }
        done = n4 << 2;
    }
    for (long long e = done + tid; e < n; e += stride) {
        T v = q[e];
#pragma unroll
        for (int j = 0; j < K; ++j) v -= beta[j] * __ldg(c.Qp[j] + e);
        out[e] = v * inu;
    }
}

template <typename T, int K>
__global__ void combine_kernel(const T* __restrict__ q, CombineArgs<T> c, T inv_nu, long long n, T* __restrict__ out) {
    T beta[K > 0 ? K : 1];
#pragma unroll
    for (int j = 0; j < K; ++j) beta[j] = c.beta[j];
    combine_range<T, K>(q, c, beta, inv_nu, n, out);
}

template <typename T, int K>
__global__ void combine_dyn_kernel(const T* __restrict__ q, CombineArgs<T> c, const CtlCombine* __restrict__ ctl,
                                   long long n, T* __restrict__ out) {
    if (!ctl->run) return;
    T beta[K > 0 ? K : 1];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int j = 0; j < K; ++j) beta[j] = ctl->beta_f[j];
        combine_range<T, K>(q, c, beta, ctl->inv_nu_f, n, out);
    } else {
#pragma unroll
        for (int j = 0; j < K; ++j) beta[j] = (T)ctl->beta[j];
        combine_range<T, K>(q, c, beta, (T)ctl->inv_nu, n, out);
    }
}

// Multi-dot partials: blockDim 256, partials[block][ndots].
constexpr int DOT_THREADS = 256;
constexpr int MAX_DOTS = kMaxDots;
template <typename T>
struct DotArgs { const T* a[MAX_DOTS]; const T* b[MAX_DOTS]; };

template <typename T>
__global__ void __launch_bounds__(DOT_THREADS)
multi_dot_kernel(DotArgs<T> d, int ndots, long long n, double* partials) {
    __shared__ double red[DOT_THREADS / 32];
    const long long tid = blockIdx.x * (long long)DOT_THREADS + threadIdx.x, stride = (long long)gridDim.x * DOT_THREADS;
    for (int q = 0; q < ndots; ++q) {
        T acct = T(0);
        const T* a = d.a[q];
        const T* b = d.b[q];
        long long done = 0;
        if constexpr (sizeof(T) == 4) {
            // 16-byte aligned vectors: four at a time, the tail one by one.
            if (((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15u) == 0) {
                const long long n4 = n >> 2;
                for (long long e = tid; e < n4; e += stride) {
                    const float4 x = __ldg(reinterpret_cast<const float4*>(a) + e);
                    const float4 y = __ldg(reinterpret_cast<const float4*>(b) + e);
                    acct += x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
                }
                done = n4 << 2;
            }
        }
        for (long long e = done + tid; e < n; e += stride) acct += a[e] * b[e];
        if constexpr (sizeof(T) == 4) {
            // Compensated FP32 warp sums; the block's sum in FP64 by one thread.
            float hi = acct, lo = 0.0f;
            warp_sum_pair(hi, lo);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)hi + (double)lo;
            __syncthreads();
            if (threadIdx.x == 0) {
                double v = 0.0;
                for (int ww = 0; ww < DOT_THREADS / 32; ++ww) v += red[ww];
                partials[(long long)blockIdx.x * ndots + q] = v;
            }
        } else {
            double acc = warp_sum((double)acct);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x < 32) {
                double v = threadIdx.x < DOT_THREADS / 32 ? red[threadIdx.x] : 0.0;
                v = warp_sum(v);
                if (threadIdx.x == 0) partials[(long long)blockIdx.x * ndots + q] = v;
            }
        }
        __syncthreads();
    }
}

// The block's partial sums of ND per-thread accumulators into partials[block][ND]:
// FP32 accumulators as compensated warp sums with FP64 once per dot and block.
template <typename T, int ND>
__device__ __forceinline__ void dots_block_reduce(const T* acc, double* partials) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (sizeof(T) == 4) {
        // Warp sums as compensated FP32 pairs; the block's sum in FP64, once per dot.
        __shared__ float redh[DOT_THREADS / 32][ND], redl[DOT_THREADS / 32][ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            float hi = acc[d], lo = 0.0f;
            warp_sum_pair(hi, lo);
            if (lane == 0) { redh[w][d] = hi; redl[w][d] = lo; }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < ND; d += DOT_THREADS) {
            double v = 0.0;
            for (int ww = 0; ww < DOT_THREADS / 32; ++ww) v += (double)redh[ww][d] + (double)redl[ww][d];
            partials[(long long)blockIdx.x * ND + d] = v;
        }
    } else {
        __shared__ double red[DOT_THREADS / 32][ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const double v = warp_sum((double)acc[d]);
            if (lane == 0) red[w][d] = v;
        }
        __syncthreads();
        for (int d = threadIdx.x; d < ND; d += DOT_THREADS) {
            double v = 0.0;
            for (int ww = 0; ww < DOT_THREADS / 32; ++ww) v += red[ww][d];
            partials[(long long)blockIdx.x * ND + d] = v;
        }
    }
}

// Inner products of the GCR step in one pass over the skeleton vectors:
// out partials [block][2 + 2k]: <q,q>, <q,r>, then <q,p_j>, <r,p_j> for j < k.
template <typename T>
struct GcrDotArgs { const T* p[16]; };

template <typename T, int K>
__global__ void __launch_bounds__(DOT_THREADS)
gcr_dots_kernel(const T* __restrict__ q, const T* __restrict__ r, GcrDotArgs<T> P, long long n, double* partials) {
    constexpr int ND = 2 + 2 * K;
    // Per-thread sums in the vectors' precision (a few dozen terms each), block sums in FP64.
    T acc[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) acc[d] = T(0);
    const long long tid = blockIdx.x * (long long)DOT_THREADS + threadIdx.x, stride = (long long)gridDim.x * DOT_THREADS;
    long long done = 0;
    if constexpr (sizeof(T) == 4) {
        // The skeleton vectors are 16-byte aligned: four elements at a time, every
        // load of an element group issued before the first use; the tail one by one.
        const long long n4 = n >> 2;
        for (long long e = tid; e < n4; e += stride) {
            const float4 qv = __ldg(reinterpret_cast<const float4*>(q) + e);
            const float4 rv = __ldg(reinterpret_cast<const float4*>(r) + e);
            float4 pv[K > 0 ? K : 1];
#pragma unroll
            for (int j = 0; j < K; ++j) pv[j] = __ldg(reinterpret_cast<const float4*>(P.p[j]) + e);
            acc[0] += qv.x * qv.x + qv.y * qv.y + qv.z * qv.z + qv.w * qv.w;
            acc[1] += qv.x * rv.x + qv.y * rv.y + qv.z * rv.z + qv.w * rv.w;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                acc[2 + 2 * j] += qv.x * pv[j].x + qv.y * pv[j].y + qv.z * pv[j].z + qv.w * pv[j].w;
                acc[3 + 2 * j] += rv.x * pv[j].x + rv.y * pv[j].y + rv.z * pv[j].z + rv.w * pv[j].w;
            }
        }
        done = n4 << 2;
    }
    for (long long e = done + tid; e < n; e += stride) {
        const T qv = q[e], rv = r[e];
        acc[0] += qv * qv;
        acc[1] += qv * rv;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const T pv = __ldg(P.p[j] + e);
            acc[2 + 2 * j] += qv * pv;
            acc[3 + 2 * j] += rv * pv;
        }
    }
    dots_block_reduce<T, ND>(acc, partials);
}

// One CTA per column q: out[q] = sum over blocks of partials[b][q], in a fixed
// order (strided per thread, then a fixed tree), so results are reproducible.
__global__ void __launch_bounds__(256) reduce_partials_kernel(const double* partials, int nblocks, int ncols, double* out) {
    __shared__ double red[8];
    const int q = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc += partials[(long long)b * ncols + q];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) out[q] = v;
    }
}

template <typename T>
__global__ void maxabs_kernel(const T* v, long long n, double* partials) {
    __shared__ double red[32];
    double m = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs((double)v[e]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        x = warp_max(x);
        if (threadIdx.x == 0) partials[blockIdx.x] = x;
    }
}

template <typename T>
__global__ void fill_value_kernel(T* p, long long n, T v) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) p[e] = v;
}

template <typename Ts, typename Td>
__global__ void copy_interior_kernel(const Ts* src, Td* dst, Geometry g) {
    const long long n = (long long)g.Nf * g.Nf;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long idx = (e / g.Nf + 1) * g.N + (e % g.Nf + 1);
        dst[idx] = (Td)src[idx];
    }
}

template <typename T>
__global__ void ring_from_kernel(const double* u, T* z, Geometry g, int zero_interior) {
    const long long n = (long long)g.N * g.N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % g.N), j = (int)(e / g.N);
        const bool ring = i == 0 || j == 0 || i == g.N - 1 || j == g.N - 1;
        if (ring) z[e] = u ? (T)u[e] : T(0);
        else if (zero_interior) z[e] = T(0);
    }
}

__global__ void to_fixed_kernel(const float* z, const double* u_ring, long long* U, double scale, Geometry g) {
    const long long n = (long long)g.N * g.N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % g.N), j = (int)(e / g.N);
        const bool ring = i == 0 || j == 0 || i == g.N - 1 || j == g.N - 1;
        const double v = (ring || z == nullptr) ? u_ring[e] : (double)z[e];
        U[e] = __double2ll_rn(v * scale);
    }
}

__global__ void from_fixed_kernel(const long long* U, double inv_scale, double* u, Geometry g) {
    const long long n = (long long)g.Nf * g.Nf;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long idx = (e / g.Nf + 1) * g.N + (e % g.Nf + 1);
        u[idx] = __ll2double_rn(U[idx]) * inv_scale;
    }
}

__global__ void split_kernel(const double* s, float* hi, float* lo, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double v = s[e];
        const float h = __double2float_rn(v);
        hi[e] = h;
        lo[e] = __double2float_rn(v - (double)h);
    }
}

template <typename Ts, typename Td>
__global__ void convert_kernel(const Ts* in, Td* out, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) out[e] = (Td)in[e];
}

inline unsigned grid_for(long long n, int threads = 256, long long cap = 152LL * 16) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
int residual_grid_blocks(const Geometry& g) {
    const int a = ((g.Nf + RX - 1) / RX) * ((g.Nf + RY - 1) / RY);
    const int b = ((g.Nf + MS_OUT * MS_WARPS - 1) / (MS_OUT * MS_WARPS)) * ((g.Nf + MS_ROWS - 1) / MS_ROWS);
    return a > b ? a : b;
}

cudaError_t residual_fp64(const double* s, const double* u_in, double* u_out, const UpdateTerms& up,
                          const Geometry& g, const Stencil& c, ResidOut out, int* nblocks, cudaStream_t st) {
    dim3 grid((g.Nf + RX - 1) / RX, (g.Nf + RY - 1) / RY);
    *nblocks = grid.x * grid.y;
    residual_fp64_kernel<<<grid, RTHREADS, 0, st>>>(s, u_in, u_out, up, g, c, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t residual_mixed(const float* s_hi, const float* s_lo, const long long* U_in, long long* U_out,
                           const UpdateTerms& up, double scale, const Geometry& g, const MixedCoefs& k,
                           ResidOut out, int* nblocks, int* overflow_flag, cudaStream_t st) {
    UpdateF uf{};
    uf.dyn = up.dyn;
    uf.count = up.count;
    for (int q = 0; q < 16; ++q) {
        uf.z[q] = reinterpret_cast<const float*>(up.z[q]);     // every slot given (device-held counts may use them)
        if (q < up.count) uf.c[q] = (float)(up.coef[q] * scale);
    }
    dim3 grid((g.Nf + MS_OUT * MS_WARPS - 1) / (MS_OUT * MS_WARPS), (g.Nf + MS_ROWS - 1) / MS_ROWS);
    *nblocks = grid.x * grid.y;
    residual_mixed_kernel<<<grid, 32 * MS_WARPS, 0, st>>>(s_hi, s_lo, U_in, U_out, uf, g, k, out, overflow_flag);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t build_submesh_rhs(const double* s, const double* u, const Geometry& g,
                              const double alpha[2], const double beta[2],
                              T* bfc, T* bcf, T* bcc, cudaStream_t st) {
    const long long total = 2LL * g.Nf * g.Nc + (long long)g.Nc * g.Nc;
    submesh_rhs_kernel<T><<<grid_for(total), 256, 0, st>>>(s, u, g, alpha[0], alpha[1], beta[0], beta[1], bfc, bcf, bcc);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 check of a returned iterate: per block the sum of r^2 over the
// interior and the largest |r| over the hole points, r = s - A u in FP64
// (A's 5-point stencil of Section 2.3, u's ring carrying g); then one CTA
// folds the blocks in a fixed order into out[0] = ||r||^2, out[1] = max |r|.
// ---------------------------------------------------------------------------
constexpr int FC_THREADS = 256;

__global__ void __launch_bounds__(FC_THREADS)
final_check_kernel(const double* __restrict__ s, const double* __restrict__ u, Geometry g, Stencil c,
                   double* partials) {
    const int N = g.N;
    double sr = 0.0, mh = 0.0;
    for (int j = 1 + blockIdx.x; j <= N - 2; j += gridDim.x) {
        const long long row = (long long)j * N;
        for (int i = 1 + threadIdx.x; i <= N - 2; i += FC_THREADS) {
            const long long idx = row + i;
            const double Au = c.cc * u[idx] + c.cw * u[idx - 1] + c.ce * u[idx + 1]
                            + c.cs * u[idx - N] + c.cn * u[idx + N];
            const double r = s[idx] - Au;
            sr += r * r;
            if (skel_kind(i, j, g.n) == 0) mh = fmax(mh, fabs(r));
        }
    }
    __shared__ double ws[FC_THREADS / 32][2];
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xFFFFFFFFu, sr, o);
        mh = fmax(mh, __shfl_down_sync(0xFFFFFFFFu, mh, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { ws[wid][0] = sr; ws[wid][1] = mh; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, m = 0.0;
        for (int w = 0; w < FC_THREADS / 32; ++w) { a += ws[w][0]; m = fmax(m, ws[w][1]); }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = m;
    }
}

__global__ void __launch_bounds__(32)
fold_sum_max_kernel(const double* __restrict__ partials, int nblocks, double* out) {
    double a = 0.0, m = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 32) { a += partials[2 * b]; m = fmax(m, partials[2 * b + 1]); }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        m = fmax(m, __shfl_down_sync(0xFFFFFFFFu, m, o));
    }
    if (threadIdx.x == 0) { out[0] = a; out[1] = m; }
}

cudaError_t final_check(const double* s, const double* u, const Geometry& g, const Stencil& c, double* partials,
                        int max_blocks, double* out, cudaStream_t st) {
    int nb = g.Nf < max_blocks ? g.Nf : max_blocks;
    if (nb < 1) nb = 1;
    final_check_kernel<<<nb, FC_THREADS, 0, st>>>(s, u, g, c, partials);
    fold_sum_max_kernel<<<1, 32, 0, st>>>(partials, nb, out);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t reduce_partials(const double* partials, int nblocks, int ncols, double* out, cudaStream_t st) {
    if (ncols < 1) return cudaSuccess;
    reduce_partials_kernel<<<ncols, 256, 0, st>>>(partials, nblocks, ncols, out);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t multi_dot(const T* const* a, const T* const* b, int ndots, long long n,
                      double* partials, int* nblocks, cudaStream_t st) {
    if (ndots > MAX_DOTS) return cudaErrorInvalidValue;
    DotArgs<T> d{};
    for (int q = 0; q < ndots; ++q) { d.a[q] = a[q]; d.b[q] = b[q]; }
    unsigned grid = grid_for(n, DOT_THREADS, kDotBlocks);
    *nblocks = (int)grid;
    multi_dot_kernel<T><<<grid, DOT_THREADS, 0, st>>>(d, ndots, n, partials);
    note_launch();
    return cudaGetLastError();
}

template <typename T, int K>
cudaError_t gcr_dots_launch(const T* q, const T* r, const GcrDotArgs<T>& P, long long n, double* partials,
                            unsigned grid, cudaStream_t st) {
    gcr_dots_kernel<T, K><<<grid, DOT_THREADS, 0, st>>>(q, r, P, n, partials);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t gcr_dots(const T* q, const T* r, const T* const* p, int k, long long n,
                     double* partials, int* nblocks, cudaStream_t st) {
    GcrDotArgs<T> P{};
    for (int j = 0; j < k && j < 16; ++j) P.p[j] = p[j];
    const unsigned grid = grid_for(n, DOT_THREADS, kDotBlocks);
    *nblocks = (int)grid;
    switch (k) {
        case 0: return gcr_dots_launch<T, 0>(q, r, P, n, partials, grid, st);
        case 1: return gcr_dots_launch<T, 1>(q, r, P, n, partials, grid, st);
        case 2: return gcr_dots_launch<T, 2>(q, r, P, n, partials, grid, st);
        case 3: return gcr_dots_launch<T, 3>(q, r, P, n, partials, grid, st);
        case 4: return gcr_dots_launch<T, 4>(q, r, P, n, partials, grid, st);
        case 5: return gcr_dots_launch<T, 5>(q, r, P, n, partials, grid, st);
        case 6: return gcr_dots_launch<T, 6>(q, r, P, n, partials, grid, st);
        case 7: return gcr_dots_launch<T, 7>(q, r, P, n, partials, grid, st);
        case 8: return gcr_dots_launch<T, 8>(q, r, P, n, partials, grid, st);
        case 9: return gcr_dots_launch<T, 9>(q, r, P, n, partials, grid, st);
        case 10: return gcr_dots_launch<T, 10>(q, r, P, n, partials, grid, st);
        case 11: return gcr_dots_launch<T, 11>(q, r, P, n, partials, grid, st);
        case 12: return gcr_dots_launch<T, 12>(q, r, P, n, partials, grid, st);
        case 13: return gcr_dots_launch<T, 13>(q, r, P, n, partials, grid, st);
        case 14: return gcr_dots_launch<T, 14>(q, r, P, n, partials, grid, st);
        case 15: return gcr_dots_launch<T, 15>(q, r, P, n, partials, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t merge_knots(const MergeArgs<T>& a, cudaStream_t st) {
    const int nlb = (a.g.Nc + MK_L - 1) / MK_L;
    const int nrb = (a.g.mc + 1 + MK_R - 1) / MK_R;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * nlb * MK_KS, nrb);
    cfg.blockDim = dim3(MK_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = MK_KS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, merge_knots_kernel<T>, a);
    note_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename T>
cudaError_t merge_write(const MergeArgs<T>& a, cudaStream_t st) {
    const int nft = ((a.g.Nc + MW_T - 1) / MW_T) * ((a.g.Nf + MW_T * MW_X - 1) / (MW_T * MW_X));
    merge_write_kernel<T><<<nft + (a.g.Nf + MW_Y - 1) / MW_Y, MW_THREADS, 0, st>>>(a, nft);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t skeleton_apply(const T* z, const Geometry& g, const Stencil& s, T* q, cudaStream_t st) {
    const StencilT<T> c{(T)s.cc, (T)s.cw, (T)s.ce, (T)s.cs, (T)s.cn};
    if (g.Nc > 256) {
        // wider cf rows than one block: the generic per-point kernel
        skeleton_apply_generic_kernel<T><<<grid_for(g.skel), 256, 0, st>>>(z, g, c, q);
        note_launch();
        return cudaGetLastError();
    }
    const int nxb = (g.Nf + 256 * SA_E - 1) / (256 * SA_E);
    const int ncf = (int)((g.skel - (long long)g.Nc * g.Nf) / g.Nc);     // cf rows off the fc lines
    skeleton_apply_kernel<T><<<g.Nc * nxb + (ncf + SA_E - 1) / SA_E, 256, 0, st>>>(z, g, c, q, nxb);
    note_launch();
    return cudaGetLastError();
}

// The tracked residual of a deferred GCR cycle on the compact skeleton, and the
// submesh right-hand sides gathered from it (fc lines [x][line], cf columns [y][column]).
template <typename T>
__global__ void __launch_bounds__(MW_THREADS) track_skeleton_kernel(T* __restrict__ r, const T* __restrict__ qp,
                                                                    T alpha_h, const CtlCombine* __restrict__ ctl,
                                                                    Geometry g, T* __restrict__ rfc,
                                                                    T* __restrict__ rcf, int nft) {
    if (ctl && !ctl->track) return;
    T a = alpha_h;
    if (ctl) {
        if constexpr (sizeof(T) == 4) a = ctl->alpha_f;
        else a = (T)ctl->alpha;
    }
    const int n = g.n, Nf = g.Nf, Nc = g.Nc;
    if ((int)blockIdx.x < nft) {
        // fc line points (cross points included) in tiles of MW_T lines x MW_X MW_T
        // fine x: r updated along x, r_fc ([x][line]) written along lines.
        __shared__ T tile[MW_X][MW_T][MW_T + 1];   // [x][line]
        const int tx = threadIdx.x % MW_T, ty = threadIdx.x / MW_T;
        const int nxt = (Nf + MW_T * MW_X - 1) / (MW_T * MW_X);
        const int l0 = ((int)blockIdx.x / nxt) * MW_T, x0 = ((int)blockIdx.x % nxt) * MW_T * MW_X;
        constexpr int PT = MW_X * MW_T / (MW_THREADS / MW_T);   // points per thread
        T rv[PT], qv[PT];
#pragma unroll
        for (int u = 0; u < PT; ++u) {
            const int c = u / (MW_T / (MW_THREADS / MW_T)), ll = ty + (MW_THREADS / MW_T) * (u % (MW_T / (MW_THREADS / MW_T)));
            const int l = l0 + ll, x = x0 + c * MW_T + tx;
            const bool ok = l < Nc && x < Nf;
            const long long e = ok ? (long long)l * Nf + x : 0;
            rv[u] = ok ? r[e] : T(0);
            qv[u] = ok ? qp[e] : T(0);
        }
#pragma unroll
        for (int u = 0; u < PT; ++u) {
            const int c = u / (MW_T / (MW_THREADS / MW_T)), ll = ty + (MW_THREADS / MW_T) * (u % (MW_T / (MW_THREADS / MW_T)));
            const int l = l0 + ll, x = x0 + c * MW_T + tx;
            if (l >= Nc || x >= Nf) continue;
            const T v = rv[u] - a * qv[u];
            r[(long long)l * Nf + x] = v;
            tile[c][tx][ll] = v;
            const int i = x + 1;
            if ((i & (n - 1)) == 0) rcf[(long long)((l + 1) * n - 1) * Nc + ((i >> g.ln) - 1)] = v;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < MW_X; ++c)
            for (int xx = ty; xx < MW_T; xx += MW_THREADS / MW_T) {
                const int x = x0 + c * MW_T + xx, l = l0 + tx;
                if (x < Nf && l < Nc) rfc[(long long)x * Nc + l] = tile[c][xx][tx];
            }
        return;
    }
    // cf column points off the fc lines: MW_Y such rows yr per block (columns along the threads).
    const int yr0 = ((int)blockIdx.x - nft) * MW_Y, nyr = Nf - Nc;
    for (int k = threadIdx.x; k < Nc; k += blockDim.x) {
        T rv[MW_Y], qv[MW_Y];
#pragma unroll
        for (int u = 0; u < MW_Y; ++u) {
            const int yr = yr0 + u;
            const int e = Nc * Nf + (yr < nyr ? yr : 0) * Nc + k;
            rv[u] = yr < nyr ? r[e] : T(0);
            qv[u] = yr < nyr ? qp[e] : T(0);
        }
#pragma unroll
        for (int u = 0; u < MW_Y; ++u) {
            const int yr = yr0 + u;
            if (yr >= nyr) continue;
            const T v = rv[u] - a * qv[u];
            r[Nc * Nf + yr * Nc + k] = v;
            const int j = yr + yr / (n - 1) + 1;
            rcf[(j - 1) * Nc + k] = v;
        }
    }
}

template <typename T>
cudaError_t track_skeleton(T* rskel, const T* qp, double alpha, const CtlCombine* c, const Geometry& g, T* rfc,
                           T* rcf, cudaStream_t st) {
    const int nft = ((g.Nc + MW_T - 1) / MW_T) * ((g.Nf + MW_T * MW_X - 1) / (MW_T * MW_X));
    const int ncf = (int)((g.skel - (long long)g.Nc * g.Nf) / g.Nc);     // cf rows off the fc lines
    track_skeleton_kernel<T><<<nft + (ncf + MW_Y - 1) / MW_Y, MW_THREADS, 0, st>>>(rskel, qp, (T)alpha, c, g, rfc,
                                                                                  rcf, nft);
    note_launch();
    return cudaGetLastError();
}

// Launch of the combination with K directions as a template argument.
template <typename T, bool kDyn, int K>
cudaError_t combine_launch(const T* q, const CombineArgs<T>& c, T inv_nu, const CtlCombine* ctl, long long n, T* out,
                           cudaStream_t st) {
    const unsigned grid = grid_for(sizeof(T) == 4 ? (n + 3) / 4 : n);
    if constexpr (kDyn) combine_dyn_kernel<T, K><<<grid, 256, 0, st>>>(q, c, ctl, n, out);
    else combine_kernel<T, K><<<grid, 256, 0, st>>>(q, c, inv_nu, n, out);
    note_launch();
    return cudaGetLastError();
}

template <typename T, bool kDyn>
cudaError_t combine_switch(int k, const T* q, const CombineArgs<T>& c, T inv_nu, const CtlCombine* ctl, long long n,
                           T* out, cudaStream_t st) {
    switch (k) {
#define ASDSM_COMBINE_CASE(K) \
        case K: return combine_launch<T, kDyn, K>(q, c, inv_nu, ctl, n, out, st);
        ASDSM_COMBINE_CASE(0) ASDSM_COMBINE_CASE(1) ASDSM_COMBINE_CASE(2) ASDSM_COMBINE_CASE(3)
        ASDSM_COMBINE_CASE(4) ASDSM_COMBINE_CASE(5) ASDSM_COMBINE_CASE(6) ASDSM_COMBINE_CASE(7)
        ASDSM_COMBINE_CASE(8) ASDSM_COMBINE_CASE(9) ASDSM_COMBINE_CASE(10) ASDSM_COMBINE_CASE(11)
        ASDSM_COMBINE_CASE(12) ASDSM_COMBINE_CASE(13) ASDSM_COMBINE_CASE(14) ASDSM_COMBINE_CASE(15)
#undef ASDSM_COMBINE_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t combine_skeleton(const T* q, const T* const* Qp, const double* beta, int k, double inv_nu,
                             long long n, T* out, cudaStream_t st) {
    if (k < 0 || k > 15) return cudaErrorInvalidValue;
    CombineArgs<T> c{};
    for (int j = 0; j < k; ++j) { c.Qp[j] = Qp[j]; c.beta[j] = (T)beta[j]; }
    return combine_switch<T, false>(k, q, c, (T)inv_nu, nullptr, n, out, st);
}

template <typename T>
cudaError_t combine_skeleton_dyn(const T* q, const T* const* Qp, int k, const CtlCombine* ctl,
                                 long long n, T* out, cudaStream_t st) {
    if (k < 0 || k > 15) return cudaErrorInvalidValue;
    CombineArgs<T> c{};
    for (int j = 0; j < k; ++j) c.Qp[j] = Qp[j];
    return combine_switch<T, true>(k, q, c, T(0), ctl, n, out, st);
}

// Input channels of the learned correction on the full N x N grid:
// [r * rs, e * es, c2, c3, c4, c5] (channel-major, x fastest).
__global__ void cnn_features_kernel(const float* __restrict__ r, const float* __restrict__ e, float rs, float es,
                                    float c2, float c3, float c4, float c5, long long nn, float* __restrict__ x) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nn; q += (long long)gridDim.x * blockDim.x) {
        x[q] = r[q] * rs;
        x[nn + q] = e[q] * es;
        x[2 * nn + q] = c2;
        x[3 * nn + q] = c3;
        x[4 * nn + q] = c4;
        x[5 * nn + q] = c5;
    }
}

// z = y on the interior skeleton points (holes and ring untouched).
__global__ void skeleton_from_kernel(const float* __restrict__ y, Geometry g, float* __restrict__ z) {
    const int N = g.N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.skel; e += (long long)gridDim.x * blockDim.x) {
        int i, j;
        if (e < (long long)g.Nc * g.Nf) {
            i = (int)(e % g.Nf) + 1;
            j = ((int)(e / g.Nf) + 1) * g.n;
        } else {
            const long long f = e - (long long)g.Nc * g.Nf;
            const int yr = (int)(f / g.Nc), k = (int)(f % g.Nc);
            j = yr + yr / (g.n - 1) + 1;
            i = (k + 1) * g.n;
        }
        const long long idx = (long long)j * N + i;
        z[idx] = y[idx];
    }
}

cudaError_t cnn_features(const float* r, const float* e, float rs, float es, const float c[4], long long nn, float* x,
                         cudaStream_t st) {
    cnn_features_kernel<<<grid_for(nn), 256, 0, st>>>(r, e, rs, es, c[0], c[1], c[2], c[3], nn, x);
    note_launch();
    return cudaGetLastError();
}

cudaError_t skeleton_from(const float* y, const Geometry& g, float* z, cudaStream_t st) {
    skeleton_from_kernel<<<grid_for(g.skel), 256, 0, st>>>(y, g, z);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t fill_value(T* p, long long n, T v, cudaStream_t st) {
    fill_value_kernel<T><<<grid_for(n), 256, 0, st>>>(p, n, v);
    note_launch();
    return cudaGetLastError();
}

template <typename Ts, typename Td>
cudaError_t copy_interior(const Ts* src, Td* dst, const Geometry& g, cudaStream_t st) {
    copy_interior_kernel<Ts, Td><<<grid_for((long long)g.Nf * g.Nf), 256, 0, st>>>(src, dst, g);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t ring_from(const double* u, T* z, const Geometry& g, int zero_interior, cudaStream_t st) {
    ring_from_kernel<T><<<grid_for((long long)g.N * g.N), 256, 0, st>>>(u, z, g, zero_interior);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t maxabs(const T* v, long long n, double* partials, int* nblocks, cudaStream_t st) {
    unsigned grid = grid_for(n, 256, 152LL * 2);
    *nblocks = (int)grid;
    maxabs_kernel<T><<<grid, 256, 0, st>>>(v, n, partials);
    note_launch();
    return cudaGetLastError();
}

cudaError_t to_fixed(const float* z, const double* u_ring_src, long long* U, double scale, const Geometry& g, cudaStream_t st) {
    to_fixed_kernel<<<grid_for((long long)g.N * g.N), 256, 0, st>>>(z, u_ring_src, U, scale, g);
    note_launch();
    return cudaGetLastError();
}

cudaError_t from_fixed(const long long* U, double inv_scale, double* u, const Geometry& g, cudaStream_t st) {
    from_fixed_kernel<<<grid_for((long long)g.Nf * g.Nf), 256, 0, st>>>(U, inv_scale, u, g);
    note_launch();
    return cudaGetLastError();
}

cudaError_t split_source(const double* s, float* hi, float* lo, long long n, cudaStream_t st) {
    split_kernel<<<grid_for(n), 256, 0, st>>>(s, hi, lo, n);
    note_launch();
    return cudaGetLastError();
}

template <typename Ts, typename Td>
cudaError_t convert_array(const Ts* in, Td* out, long long n, cudaStream_t st) {
    convert_kernel<Ts, Td><<<grid_for(n), 256, 0, st>>>(in, out, n);
    note_launch();
    return cudaGetLastError();
}

// Explicit instantiations.
#define INST(T) \
    template cudaError_t build_submesh_rhs<T>(const double*, const double*, const Geometry&, const double*, const double*, T*, T*, T*, cudaStream_t); \
    template cudaError_t multi_dot<T>(const T* const*, const T* const*, int, long long, double*, int*, cudaStream_t); \
    template cudaError_t gcr_dots<T>(const T*, const T*, const T* const*, int, long long, double*, int*, cudaStream_t); \
    template cudaError_t merge_knots<T>(const MergeArgs<T>&, cudaStream_t); \
    template cudaError_t merge_write<T>(const MergeArgs<T>&, cudaStream_t); \
    template cudaError_t skeleton_apply<T>(const T*, const Geometry&, const Stencil&, T*, cudaStream_t); \
    template cudaError_t combine_skeleton<T>(const T*, const T* const*, const double*, int, double, long long, T*, cudaStream_t); \
    template cudaError_t combine_skeleton_dyn<T>(const T*, const T* const*, int, const CtlCombine*, long long, T*, cudaStream_t); \
    template cudaError_t track_skeleton<T>(T*, const T*, double, const CtlCombine*, const Geometry&, T*, T*, cudaStream_t); \
    template cudaError_t fill_value<T>(T*, long long, T, cudaStream_t); \
    template cudaError_t ring_from<T>(const double*, T*, const Geometry&, int, cudaStream_t); \
    template cudaError_t maxabs<T>(const T*, long long, double*, int*, cudaStream_t);
INST(float)
INST(double)
#undef INST
template cudaError_t fill_value<long long>(long long*, long long, long long, cudaStream_t);
template cudaError_t copy_interior<double, double>(const double*, double*, const Geometry&, cudaStream_t);
template cudaError_t copy_interior<float, double>(const float*, double*, const Geometry&, cudaStream_t);
template cudaError_t copy_interior<double, float>(const double*, float*, const Geometry&, cudaStream_t);
template cudaError_t convert_array<double, float>(const double*, float*, long long, cudaStream_t);
template cudaError_t convert_array<float, double>(const float*, double*, long long, cudaStream_t);
template cudaError_t convert_array<double, double>(const double*, double*, long long, cudaStream_t);

}  // namespace asdsm
