// Grid-wide kernels of the ASDSM sweep on sm_103a: the fine residual of
// Algorithm 4 step 3 (with the previous step-7 update fused in), the
// right-hand sides of eq. (2.4), the merge of Algorithm 2, the skeleton
// operator for the step-6 least squares, reductions and conversions.
#include "asdsm_internal.h"
#include <cuda_runtime.h>
#include <atomic>

namespace asdsm {

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
    const bool fx = (i % n) == 0, fy = (j % n) == 0;
    return (fy ? 1 : 0) + (fx ? 2 : 0);
}

// Compact skeleton index of an interior skeleton point (i, j) (grid indices).
// Layout: fc lines [l][x] (l = j/n - 1, x = i - 1), then the cf columns
// without cross points, row by row: [yr][k] with yr the non-cross row rank.
__device__ __forceinline__ long long skel_index(int i, int j, const Geometry& g) {
    const int n = g.n;
    if (j % n == 0) return (long long)(j / n - 1) * g.Nf + (i - 1);
    const int y0 = j - 1;
    const int yr = y0 - (j / n);            // rows y0 before j with (y0+1) % n == 0
    return (long long)g.Nc * g.Nf + (long long)yr * g.Nc + (i / n - 1);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
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
    const int n = g.n;
    if (kind & 1) {   // on an fc line: BCR layout [x][line]
        reinterpret_cast<T*>(o.rfc)[(long long)(i - 1) * g.Nc + (j / n - 1)] = v;
    }
    if (kind & 2) {   // on a cf column: BCR layout [y][column]
        reinterpret_cast<T*>(o.rcf)[(long long)(j - 1) * g.Nc + (i / n - 1)] = v;
    }
    reinterpret_cast<T*>(o.rskel)[skel_index(i, j, g)] = v;
}

// ---------------------------------------------------------------------------
// FP64 residual (plain path): u_out = u_in + sum c_j z_j ; r = s - A u_out.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RTHREADS)
residual_fp64_kernel(const double* __restrict__ s, const double* __restrict__ u_in, double* __restrict__ u_out,
                     UpdateTerms up, Geometry g, Stencil c, ResidOut o) {
    __shared__ double tile[RY + 2][RX + 2];
    const int N = g.N;
    const int i0 = blockIdx.x * RX + 1, j0 = blockIdx.y * RY + 1;   // first interior point of the tile
    // Load u (+ update) on the tile and its halo.  Ring points keep g (no update).
    for (int e = threadIdx.x; e < (RX + 2) * (RY + 2); e += RTHREADS) {
        const int ty = e / (RX + 2), tx = e % (RX + 2);
        const int i = i0 - 1 + tx, j = j0 - 1 + ty;
        double v = 0.0;
        if (i <= N - 1 && j <= N - 1) {
            const long long idx = (long long)j * N + i;
            v = u_in[idx];
            if (i >= 1 && j >= 1 && i <= N - 2 && j <= N - 2) {
                for (int q = 0; q < up.count; ++q) v += up.coef[q] * reinterpret_cast<const double*>(up.z[q])[idx];
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
        if (u_out != u_in || up.count > 0) u_out[idx] = uc;
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
// FP32-pair ("double-float") primitives: Knuth's TwoSum, FMA-based TwoProd.
// ---------------------------------------------------------------------------
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {   // needs |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b) {                   // accurate sum
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return quick_two_sum(p, e);
}
// Exact split of a 64-bit integer into an FP32 pair (exact while |D| < 2^48).
__device__ __forceinline__ df ll_to_df(long long D) {
    const float hi = __ll2float_rn(D);
    const long long rem = D - __float2ll_rn(hi);
    return {hi, __ll2float_rn(rem)};
}

// ---------------------------------------------------------------------------
// Mixed residual: U (64-bit fixed point, u = U 2^-S) is the accumulator.
//   U_out = U_in + round(sum (coef_j 2^S) z_j)       (step 7 of the previous sweep)
//   A u   = kxx (2U_c - U_w - U_e) + kyy (2U_c - U_s - U_n) + kx (U_e - U_w) + ky (U_n - U_s)
// The integer differences are exact; each k (carrying 2^-S) is an FP32 pair,
// so r = s - A u keeps FP64-level accuracy although only FP32 units are used.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RTHREADS)
residual_mixed_kernel(const float* __restrict__ s_hi, const float* __restrict__ s_lo,
                      const long long* __restrict__ U_in, long long* __restrict__ U_out,
                      UpdateTerms up, Geometry g, MixedCoefs k, ResidOut o, int* overflow) {
    __shared__ long long tile[RY + 2][RX + 2];
    const int N = g.N;
    const int i0 = blockIdx.x * RX + 1, j0 = blockIdx.y * RY + 1;
    float cf[16];
    for (int q = 0; q < 16; ++q) cf[q] = q < up.count ? (float)up.coef[q] : 0.0f;
    for (int e = threadIdx.x; e < (RX + 2) * (RY + 2); e += RTHREADS) {
        const int ty = e / (RX + 2), tx = e % (RX + 2);
        const int i = i0 - 1 + tx, j = j0 - 1 + ty;
        long long v = 0;
        if (i <= N - 1 && j <= N - 1) {
            const long long idx = (long long)j * N + i;
            v = U_in[idx];
            if (up.count > 0 && i >= 1 && j >= 1 && i <= N - 2 && j <= N - 2) {
                float d = 0.0f;
                for (int q = 0; q < up.count; ++q) d = __fmaf_rn(cf[q], reinterpret_cast<const float*>(up.z[q])[idx], d);
                v += __float2ll_rn(d);
            }
        }
        tile[ty][tx] = v;
    }
    __syncthreads();
    double sr = 0.0, sh = 0.0;
    float srf = 0.0f, shf = 0.0f;
    const df kxx{k.kxx[0], k.kxx[1]}, kyy{k.kyy[0], k.kyy[1]}, kx{k.kx[0], k.kx[1]}, ky{k.ky[0], k.ky[1]};
    const long long lim = 1LL << 60;
    bool ovf = false;
    for (int e = threadIdx.x; e < RX * RY; e += RTHREADS) {
        const int ty = e / RX, tx = e % RX;
        const int i = i0 + tx, j = j0 + ty;
        if (i > N - 2 || j > N - 2) continue;
        const long long idx = (long long)j * N + i;
        const long long uc = tile[ty + 1][tx + 1];
        const long long uw = tile[ty + 1][tx], ue = tile[ty + 1][tx + 2];
        const long long us = tile[ty][tx + 1], un = tile[ty + 2][tx + 1];
        ovf |= (uc > lim) || (uc < -lim);
        if (up.count > 0) U_out[idx] = uc;
        const df dxx = ll_to_df(2 * uc - uw - ue);
        const df dyy = ll_to_df(2 * uc - us - un);
        const df dx = ll_to_df(ue - uw);
        const df dy = ll_to_df(un - us);
        df Au = df_add(df_add(df_mul(kxx, dxx), df_mul(kyy, dyy)), df_add(df_mul(kx, dx), df_mul(ky, dy)));
        Au.hi = -Au.hi; Au.lo = -Au.lo;
        const df r = df_add(df{s_hi[idx], s_lo[idx]}, Au);
        const float rf = __fadd_rn(r.hi, r.lo);
        const int kind = skel_kind(i, j, g.n);
        srf = __fmaf_rn(rf, rf, srf);
        if (kind == 0) shf = __fmaf_rn(rf, rf, shf);
        if (o.rfull) reinterpret_cast<float*>(o.rfull)[idx] = rf;
        if (o.rskel) store_skeleton<float>(o, g, i, j, kind, rf);
    }
    sr = srf;
    sh = shf;
    if (ovf) atomicOr(overflow, 1);
    block_sum2(sr, sh, o.partials);
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
// Algorithm 2.  merge_knots: one CTA per (family, coarse line): the cross-point
// values of both anisotropic solutions on that line, the chosen/extrapolated
// u_hat, the errors e and the spline moments of the correction.
// merge_write: every skeleton point gets its anisotropic value plus the spline
// correction (step 5) and the merged skeleton is stored (step 6).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T cross_t1(const MergeArgs<T>& a, T inv1, int l, int k) {
    // t1[l][k] = u_fc at (x = (k+1)n, line l)
    return a.Yfc[(long long)((k + 1) * a.g.n - 1) * a.g.Nc + l] * inv1;
}
template <typename T>
__device__ __forceinline__ T cross_t2(const MergeArgs<T>& a, T inv2, int l, int k) {
    // t2[l][k] = u_cf at (y = (l+1)n, column k)
    return a.Ycf[(long long)((l + 1) * a.g.n - 1) * a.g.Nc + k] * inv2;
}

template <typename T>
__device__ __forceinline__ void inv_norms(const MergeArgs<T>& a, T* inv1, T* inv2) {
    if (a.re_mode) { *inv1 = T(1); *inv2 = T(1); return; }
    const double n1 = a.norms2[0], n2 = a.norms2[1];
    *inv1 = n1 > 0.0 ? (T)(1.0 / sqrt(n1)) : T(1);
    *inv2 = n2 > 0.0 ? (T)(1.0 / sqrt(n2)) : T(1);
}

template <typename T>
__global__ void merge_knots_kernel(MergeArgs<T> a) {
    const int Nc = a.g.Nc, K = a.g.mc + 1;
    const int fam = blockIdx.x / Nc;       // 0: fc line l, 1: cf column k
    const int line = blockIdx.x % Nc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* e = reinterpret_cast<T*>(smem_raw);  // Nc knot errors of this line
    T inv1, inv2;
    inv_norms(a, &inv1, &inv2);
    for (int q = threadIdx.x; q < Nc; q += blockDim.x) {
        // fc line l = line: knots along x (k = q); cf column k = line: knots along y (l = q)
        const int l = fam == 0 ? line : q;
        const int k = fam == 0 ? q : line;
        const T t1 = cross_t1(a, inv1, l, k), t2 = cross_t2(a, inv2, l, k);
        T uh;
        if (a.re_mode) uh = t1 + t2 - a.Ycc[(long long)l * Nc + k];   // step 2: combination RE
        else uh = a.choice ? t2 : t1;                                  // step 3
        const T err = fam == 0 ? uh - t1 : uh - t2;                    // step 4
        e[q] = err;
        if (fam == 0) a.E1[(long long)l * Nc + k] = err;
        else a.E2[(long long)l * Nc + k] = err;
    }
    __syncthreads();
    T* Mout = fam == 0 ? a.M1 + (long long)line * K : a.M2 + (long long)line * K;
    for (int r = threadIdx.x; r < K; r += blockDim.x) {
        T acc = T(0);
        for (int q = 0; q < Nc; ++q) acc += a.Sm[(long long)r * Nc + q] * e[q];
        Mout[r] = acc;
    }
}

// Value of the not-a-knot spline with moments Mv and knot values (0, e.., 0)
// at fine offset t = p (0..n) inside coarse interval ki (0..mc-1).
template <typename T>
__device__ __forceinline__ T spline_eval(const T* Mv, T yk, T yk1, int ki, int p, int n, T H) {
    if (p == 0) return yk;                   // at a knot the spline interpolates exactly
    const T t = H * (T)p / (T)n;
    const T u = H - t;
    const T Mk = Mv[ki], Mk1 = Mv[ki + 1];
    return Mk * (u * u * u / (6 * H) - H * u / 6) + Mk1 * (t * t * t / (6 * H) - H * t / 6) + yk * (u / H) + yk1 * (t / H);
}

template <typename T>
__global__ void merge_write_kernel(MergeArgs<T> a) {
    const Geometry& g = a.g;
    const int Nf = g.Nf, Nc = g.Nc, n = g.n, N = g.N, K = g.mc + 1;
    const T H = T(1) / (T)g.mc;
    T inv1, inv2;
    inv_norms(a, &inv1, &inv2);
    const long long total = 2LL * Nf * Nc;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        if (e < (long long)Nf * Nc) {
            // fc line l, fine x: value u_fc/||u_fc|| + Spline(e1) (step 5.1); cross points too (step 6).
            const int l = (int)(e / Nf), x = (int)(e % Nf);
            const int i = x + 1, ki = i / n, p = i % n;
            const T* Mv = a.M1 + (long long)l * K;
            const T yk = ki == 0 ? T(0) : a.E1[(long long)l * Nc + ki - 1];
            const T yk1 = ki + 1 >= g.mc ? T(0) : a.E1[(long long)l * Nc + ki];
            const T v = a.Yfc[(long long)x * Nc + l] * inv1 + spline_eval(Mv, yk, yk1, ki, p, n, H);
            a.z[(long long)((l + 1) * n) * N + i] = v;
        } else {
            // cf column k, fine y (cross points skipped: they keep the fc value).
            const long long f = e - (long long)Nf * Nc;
            const int k = (int)(f / Nf), y = (int)(f % Nf);
            const int j = y + 1;
            if (j % n == 0) continue;
            const int ki = j / n, p = j % n;
            const T* Mv = a.M2 + (long long)k * K;
            const T yk = ki == 0 ? T(0) : a.E2[(long long)(ki - 1) * Nc + k];
            const T yk1 = ki + 1 >= g.mc ? T(0) : a.E2[(long long)ki * Nc + k];
            const T v = a.Ycf[(long long)y * Nc + k] * inv2 + spline_eval(Mv, yk, yk1, ki, p, n, H);
            a.z[(long long)j * N + (k + 1) * n] = v;
        }
    }
}

// q = A z at compact skeleton rows (z: full grid, zero ring).
template <typename T>
__global__ void skeleton_apply_kernel(const T* __restrict__ z, Geometry g, Stencil c, T* __restrict__ q) {
    const int N = g.N, n = g.n, Nf = g.Nf, Nc = g.Nc;
    const T cc = (T)c.cc, cw = (T)c.cw, ce = (T)c.ce, cs = (T)c.cs, cn = (T)c.cn;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.skel; e += (long long)gridDim.x * blockDim.x) {
        int i, j;
        if (e < (long long)Nc * Nf) {
            i = (int)(e % Nf) + 1;
            j = ((int)(e / Nf) + 1) * n;
        } else {
            const long long f = e - (long long)Nc * Nf;
            const int yr = (int)(f / Nc), k = (int)(f % Nc);
            j = yr + yr / (n - 1) + 1;
            i = (k + 1) * n;
        }
        const long long idx = (long long)j * N + i;
        q[e] = cc * z[idx] + cw * z[idx - 1] + ce * z[idx + 1] + cs * z[idx - N] + cn * z[idx + N];
    }
}

template <typename T>
struct CombineArgs { const T* Qp[16]; double beta[16]; };

template <typename T>
__global__ void combine_kernel(const T* __restrict__ q, CombineArgs<T> c, int k,
                               double inv_nu, long long n, T* __restrict__ out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double v = (double)q[e];
        for (int j = 0; j < k; ++j) v -= c.beta[j] * (double)c.Qp[j][e];
        out[e] = (T)(v * inv_nu);
    }
}

// Multi-dot partials: blockDim 256, partials[block][ndots].
constexpr int DOT_THREADS = 256;
constexpr int MAX_DOTS = 40;
template <typename T>
struct DotArgs { const T* a[MAX_DOTS]; const T* b[MAX_DOTS]; };

template <typename T>
__global__ void __launch_bounds__(DOT_THREADS)
multi_dot_kernel(DotArgs<T> d, int ndots, long long n, double* partials) {
    __shared__ double red[DOT_THREADS / 32];
    for (int q = 0; q < ndots; ++q) {
        double acc = 0.0;
        const T* a = d.a[q];
        const T* b = d.b[q];
        for (long long e = blockIdx.x * (long long)DOT_THREADS + threadIdx.x; e < n; e += (long long)gridDim.x * DOT_THREADS)
            acc += (double)a[e] * (double)b[e];
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < DOT_THREADS / 32 ? red[threadIdx.x] : 0.0;
            v = warp_sum(v);
            if (threadIdx.x == 0) partials[(long long)blockIdx.x * ndots + q] = v;
        }
        __syncthreads();
    }
}

__global__ void reduce_partials_kernel(const double* partials, int nblocks, int ncols, double* out) {
    __shared__ double red[32];
    for (int q = 0; q < ncols; ++q) {
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
        __syncthreads();
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
    return ((g.Nf + RX - 1) / RX) * ((g.Nf + RY - 1) / RY);
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
                           const UpdateTerms& up, double /*scale*/, const Geometry& g, const MixedCoefs& k,
                           ResidOut out, int* nblocks, int* overflow_flag, cudaStream_t st) {
    dim3 grid((g.Nf + RX - 1) / RX, (g.Nf + RY - 1) / RY);
    *nblocks = grid.x * grid.y;
    residual_mixed_kernel<<<grid, RTHREADS, 0, st>>>(s_hi, s_lo, U_in, U_out, up, g, k, out, overflow_flag);
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

cudaError_t reduce_partials(const double* partials, int nblocks, int ncols, double* out, cudaStream_t st) {
    reduce_partials_kernel<<<1, 1024, 0, st>>>(partials, nblocks, ncols, out);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t multi_dot(const T* const* a, const T* const* b, int ndots, long long n,
                      double* partials, int* nblocks, cudaStream_t st) {
    if (ndots > MAX_DOTS) return cudaErrorInvalidValue;
    DotArgs<T> d{};
    for (int q = 0; q < ndots; ++q) { d.a[q] = a[q]; d.b[q] = b[q]; }
    unsigned grid = grid_for(n, DOT_THREADS, 152LL * 2);
    *nblocks = (int)grid;
    multi_dot_kernel<T><<<grid, DOT_THREADS, 0, st>>>(d, ndots, n, partials);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t merge_knots(const MergeArgs<T>& a, cudaStream_t st) {
    const size_t smem = sizeof(T) * (size_t)a.g.Nc;
    merge_knots_kernel<T><<<2 * a.g.Nc, 128, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t merge_write(const MergeArgs<T>& a, cudaStream_t st) {
    merge_write_kernel<T><<<grid_for(2LL * a.g.Nf * a.g.Nc), 256, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t skeleton_apply(const T* z, const Geometry& g, const Stencil& s, T* q, cudaStream_t st) {
    skeleton_apply_kernel<T><<<grid_for(g.skel), 256, 0, st>>>(z, g, s, q);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t combine_skeleton(const T* q, const T* const* Qp, const double* beta, int k, double inv_nu,
                             long long n, T* out, cudaStream_t st) {
    if (k > 16) return cudaErrorInvalidValue;
    CombineArgs<T> c{};
    for (int j = 0; j < k; ++j) { c.Qp[j] = Qp[j]; c.beta[j] = beta[j]; }
    combine_kernel<T><<<grid_for(n), 256, 0, st>>>(q, c, k, inv_nu, n, out);
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
    template cudaError_t merge_knots<T>(const MergeArgs<T>&, cudaStream_t); \
    template cudaError_t merge_write<T>(const MergeArgs<T>&, cudaStream_t); \
    template cudaError_t skeleton_apply<T>(const T*, const Geometry&, const Stencil&, T*, cudaStream_t); \
    template cudaError_t combine_skeleton<T>(const T*, const T* const*, const double*, int, double, long long, T*, cudaStream_t); \
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
