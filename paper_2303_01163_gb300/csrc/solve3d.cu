// The 3D extension of ASDSM (Section 3.5) on the GPU.
//
// Meshes of the unit cube with N points per axis and mc coarse intervals
// (N_f = N - 2 fine and N_c = mc - 1 coarse interior points per axis):
//   plane family P_a (a = x, y, z): coarse in axis a, fine in the other two;
//   line family L_a: fine in axis a only (needed by the extrapolation of the
//   initial guess, R21); the coarse mesh C; the cube holes of n - 1 points
//   per side between the coarse planes.
//
// Every submesh operator is a Kronecker sum of 1D three-point operators
// (Section 2.3 with each axis' own spacing), so every system is solved
// exactly by block cyclic reduction (the kernels of kernels_solve.cu) with
// factors computed once on the host in FP64:
//   * L_a, C and the holes: BCR along one axis with the dense Kronecker-sum
//     block of the two others (N_c^2 or (n-1)^2 columns; all holes at once);
//   * P_a: the coarse-axis operator T_H (N_c x N_c) is brought to real Schur
//     form T_H = Q S Q^T (host).  In the basis of Q the plane system becomes a
//     back-substitution over S's diagonal blocks, each a shifted 2D fine-plane
//     system (A_2D + S_kk I) y_k = g_k - sum_{j>k} S_kj y_j solved by 2D BCR;
//     a 2 x 2 block (a complex eigenvalue pair) is one real system with two
//     components per point (2 N_f columns).
//
// Merge (Algorithm 2 in 3D): the value u_hat on every line point (where two
// or three plane families meet) by the combination technique (R21) or the
// random choice (R22); each plane moved onto u_hat by the Boolean sum of
// not-a-knot splines of its mismatch (R23); the union of the planes, a point
// shared by several families taken from the last of x, y, z.  Filler
// (Algorithm 3): every cube hole solved with Dirichlet data from the
// skeleton.  Sweeps (Algorithm 4): FP64 fine residual with the previous
// update fused in, the correction above, least squares on the skeleton rows
// (the clamped optimal scaling, or GCR(m), R15), the hole-residual pass R18.
//
// Precision: ASDSM_FP64 does everything in FP64.  ASDSM_MIXED solves, merges
// and fills in FP32 and keeps the iterate, the residual and the accumulation
// in FP64.
#include "asdsm.h"
#include "asdsm_internal.h"
#include "solve3d.h"
#include "fill3_tc.h"
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace asdsm {

// ---------------------------------------------------------------------------
// Geometry and stencil
// ---------------------------------------------------------------------------
struct Geo3 {
    int N, M, Nf, mc, Nc, n, hc;     // hc = n - 1 points per hole side
    long long NN;                    // N^3
    long long skel;                  // skeleton points: Nf^3 - (Nf - Nc)^3
    long long plane;                 // Nf^2: points of one plane
};

// 7-point operator: A u = cc u + cw u_{x-1} + ce u_{x+1} + cs u_{y-1} + cn u_{y+1} + cd u_{z-1} + cu u_{z+1}.
struct Sten3 {
    double cc, cw, ce, cs, cn, cd, cu;
};

// Compact skeleton index of interior point (i, j, l) on the skeleton
// (at least one coordinate a multiple of n): z slabs in order; a coarse z
// slab holds its whole N_f x N_f plane, a fine one the 2D skeleton of its
// plane (coarse rows whole, fine rows only at the coarse columns).
__device__ __forceinline__ long long skel3_index(int i, int j, int l, const Geo3& g) {
    const long long P = g.plane;
    const long long S2 = (long long)g.Nc * g.Nf + (long long)(g.Nf - g.Nc) * g.Nc;
    const int cz = (l - 1) / g.n;
    long long off = (long long)cz * P + (long long)(l - 1 - cz) * S2;
    if (l % g.n == 0) return off + (long long)(j - 1) * g.Nf + (i - 1);
    const int cy = (j - 1) / g.n;
    off += (long long)cy * g.Nf + (long long)(j - 1 - cy) * g.Nc;
    if (j % g.n == 0) return off + (i - 1);
    return off + (i / g.n - 1);
}

__device__ __forceinline__ bool on_skel3(int i, int j, int l, int n) {
    return i % n == 0 || j % n == 0 || l % n == 0;
}

namespace {
unsigned grid_rows(long long rows) {
    long long b = rows < 1 ? 1 : rows;
    return (unsigned)(b > 152LL * 32 ? 152LL * 32 : b);
}
}  // namespace

constexpr int T3 = 256;    // threads per CTA of the grid kernels

// Block sums of two values into partials[2 * block].
__device__ __forceinline__ void block_sum_pair(double a, double b, double* partials) {
    __shared__ double red[2][T3 / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        b += __shfl_down_sync(0xFFFFFFFFu, b, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { red[0][w] = a; red[1][w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int q = 0; q < T3 / 32; ++q) { x += red[0][q]; y += red[1][q]; }
        partials[2 * blockIdx.x] = x;
        partials[2 * blockIdx.x + 1] = y;
    }
}

// ---------------------------------------------------------------------------
// The update of Algorithm 4, u_out = u_in + sum_j c_j z_j over the interior
// (FP64 accumulation of the T directions), and the fine residual r = s - A u
// (FP64) with the sums of r^2 over the interior and over the holes and r
// gathered onto the compact skeleton and into the three plane families'
// right-hand sides ([k][q][p], (p, q) the two other axes in increasing order).
// One CTA per (y, z) row, threads along x.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(T3)
update3_kernel(const double* __restrict__ u_in, double* __restrict__ u_out, UpdateTerms up, Geo3 g) {
    const int N = g.N, Nf = g.Nf;
    for (long long row = blockIdx.x; row < (long long)Nf * Nf; row += gridDim.x) {
        const int j = (int)(row % Nf) + 1, l = (int)(row / Nf) + 1;
        const long long base = ((long long)l * N + j) * N;
        for (int i = 1 + threadIdx.x; i <= N - 2; i += T3) {
            const long long idx = base + i;
            double v = u_in[idx];
            for (int t = 0; t < up.count; ++t) v += up.coef[t] * (double)reinterpret_cast<const T*>(up.z[t])[idx];
            u_out[idx] = v;
        }
    }
}

template <typename T>
struct Resid3Out {
    double* rskel;       // [skel], FP64
    T* rp[3];            // plane right-hand sides per family
    double* partials;    // [grid][2]
};

template <typename T>
__global__ void __launch_bounds__(T3)
resid3_kernel(const double* __restrict__ s, const double* __restrict__ u, Geo3 g, Sten3 c, Resid3Out<T> o) {
    const int N = g.N, Nf = g.Nf, n = g.n;
    const long long NN2 = (long long)N * N;
    double sr = 0.0, sh = 0.0;
    for (long long row = blockIdx.x; row < (long long)Nf * Nf; row += gridDim.x) {
        const int j = (int)(row % Nf) + 1, l = (int)(row / Nf) + 1;
        const long long base = ((long long)l * N + j) * N;
        for (int i = 1 + threadIdx.x; i <= N - 2; i += T3) {
            const long long idx = base + i;
            const double Au = c.cc * u[idx] + c.cw * u[idx - 1] + c.ce * u[idx + 1] + c.cs * u[idx - N]
                            + c.cn * u[idx + N] + c.cd * u[idx - NN2] + c.cu * u[idx + NN2];
            const double r = s[idx] - Au;
            sr += r * r;
            const bool ci = i % n == 0, cj = j % n == 0, cl = l % n == 0;
            if (!(ci || cj || cl)) { sh += r * r; continue; }
            const T rt = (T)r;
            if (o.rskel) o.rskel[skel3_index(i, j, l, g)] = r;
            const long long P = g.plane;
            if (ci && o.rp[0]) o.rp[0][(long long)(i / n - 1) * P + (long long)(l - 1) * Nf + (j - 1)] = rt;
            if (cj && o.rp[1]) o.rp[1][(long long)(j / n - 1) * P + (long long)(l - 1) * Nf + (i - 1)] = rt;
            if (cl && o.rp[2]) o.rp[2][(long long)(l / n - 1) * P + (long long)(j - 1) * Nf + (i - 1)] = rt;
        }
    }
    block_sum_pair(sr, sh, o.partials);
}

// ---------------------------------------------------------------------------
// Right-hand sides of the submesh systems with the Dirichlet lifting (R5):
// samples of s plus, along each axis, the moved stencil coefficient (with
// that mesh's spacing on that axis) times g where a neighbour falls on the
// boundary.  kind 0..2: plane family a, [k][q][p]; 3..5: line family a,
// [f][cq][cp]; 6: the coarse mesh, [cz][cy][cx].
// ---------------------------------------------------------------------------
struct Lift3 {
    double lo[3][2], hi[3][2];    // [axis][0: fine step, 1: coarse step]
};

__device__ __forceinline__ void other_axes(int a, int& pa, int& qa) {
    pa = a == 0 ? 1 : 0;
    qa = a == 2 ? 1 : 2;
}

// Grid coordinates (x, y, z) of entry e of a submesh array of the given kind.
__device__ __forceinline__ void submesh_coords(int kind, long long e, const Geo3& g, int c[3], bool coarse[3]) {
    const int Nf = g.Nf, Nc = g.Nc, n = g.n;
    if (kind < 3) {
        const int a = kind;
        int pa, qa;
        other_axes(a, pa, qa);
        const int p = (int)(e % Nf), q = (int)((e / Nf) % Nf), k = (int)(e / ((long long)Nf * Nf));
        c[a] = (k + 1) * n; c[pa] = p + 1; c[qa] = q + 1;
        coarse[a] = true; coarse[pa] = false; coarse[qa] = false;
    } else if (kind < 6) {
        const int a = kind - 3;
        int pa, qa;
        other_axes(a, pa, qa);
        const int cp = (int)(e % Nc), cq = (int)((e / Nc) % Nc), f = (int)(e / ((long long)Nc * Nc));
        c[a] = f + 1; c[pa] = (cp + 1) * n; c[qa] = (cq + 1) * n;
        coarse[a] = false; coarse[pa] = true; coarse[qa] = true;
    } else {
        c[0] = (int)(e % Nc + 1) * n; c[1] = (int)((e / Nc) % Nc + 1) * n; c[2] = (int)(e / ((long long)Nc * Nc) + 1) * n;
        coarse[0] = coarse[1] = coarse[2] = true;
    }
}

template <typename T>
__global__ void __launch_bounds__(T3)
rhs3_kernel(const double* __restrict__ s, const double* __restrict__ u, Geo3 g, int kind, long long count, Lift3 lf,
            T* __restrict__ out) {
    const int N = g.N, M = g.M;
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < count; e += (long long)gridDim.x * T3) {
        int c[3];
        bool co[3];
        submesh_coords(kind, e, g, c, co);
        auto at = [&](int x, int y, int z) { return u[((long long)z * N + y) * N + x]; };
        double b = s[((long long)c[2] * N + c[1]) * N + c[0]];
        for (int a = 0; a < 3; ++a) {
            const int st = co[a] ? g.n : 1;
            int lo[3] = {c[0], c[1], c[2]}, hi[3] = {c[0], c[1], c[2]};
            lo[a] = 0;
            hi[a] = M;
            if (c[a] - st == 0) b += lf.lo[a][co[a] ? 1 : 0] * at(lo[0], lo[1], lo[2]);
            if (c[a] + st == M) b += lf.hi[a][co[a] ? 1 : 0] * at(hi[0], hi[1], hi[2]);
        }
        out[e] = (T)b;
    }
}

// ---------------------------------------------------------------------------
// Plane-family solve in the Schur basis of the coarse-axis operator:
//   right-hand side of block k (size bs = 1 or 2):
//     v_i = sum_j Q[j][k+i] F_j - sum_{j >= k+bs} S[k+i][j] Y_j   (i < bs),
//   written plainly (bs = 1) or interleaved per point (bs = 2, column 2 e + i);
//   back-transform U_j = sum_k Q[j][k] Y_k with the partial sums of U^2.
// ---------------------------------------------------------------------------
constexpr int kMaxNc3 = 31;     // coarse points per axis (mc <= 32)
constexpr int kMaxM3 = 1024;    // directions kept by the 3D GCR (restart length)
constexpr int kCheck3 = 16;     // sweeps between true residuals (hole-residual checks, R18)

struct SchurStep {
    double q[2][kMaxNc3];       // Q[j][k+i]
    double s[2][kMaxNc3];       // S[k+i][j] (zero for j < k + bs)
    int k, bs, Nc;
};

template <typename T>
__global__ void __launch_bounds__(T3)
schur_rhs_kernel(const T* __restrict__ F, const T* __restrict__ Y, long long P, SchurStep ss, T* __restrict__ X) {
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < P; e += (long long)gridDim.x * T3) {
        double v[2] = {0.0, 0.0};
        for (int j = 0; j < ss.Nc; ++j) {
            const double f = (double)F[(long long)j * P + e];
            v[0] += ss.q[0][j] * f;
            if (ss.bs == 2) v[1] += ss.q[1][j] * f;
        }
        for (int j = ss.k + ss.bs; j < ss.Nc; ++j) {
            const double y = (double)Y[(long long)j * P + e];
            v[0] -= ss.s[0][j] * y;
            if (ss.bs == 2) v[1] -= ss.s[1][j] * y;
        }
        if (ss.bs == 1) {
            X[e] = (T)v[0];
        } else {
            X[2 * e] = (T)v[0];
            X[2 * e + 1] = (T)v[1];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(T3)
deinterleave_kernel(const T* __restrict__ Z, long long P, T* __restrict__ Y0, T* __restrict__ Y1) {
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < P; e += (long long)gridDim.x * T3) {
        Y0[e] = Z[2 * e];
        Y1[e] = Z[2 * e + 1];
    }
}

template <typename T>
__global__ void __launch_bounds__(T3)
schur_back_kernel(const T* __restrict__ Y, const T* __restrict__ Q, int Nc, long long P, T* __restrict__ U,
                  double* partials) {
    __shared__ double Qs[kMaxNc3 * kMaxNc3];
    for (int t = threadIdx.x; t < Nc * Nc; t += T3) Qs[t] = (double)Q[t];
    __syncthreads();
    double s2 = 0.0;
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < P; e += (long long)gridDim.x * T3) {
        double y[kMaxNc3];
        for (int k = 0; k < Nc; ++k) y[k] = (double)Y[(long long)k * P + e];
        for (int j = 0; j < Nc; ++j) {
            double v = 0.0;
            for (int k = 0; k < Nc; ++k) v += Qs[j * Nc + k] * y[k];
            const T vt = (T)v;
            U[(long long)j * P + e] = vt;
            s2 += (double)vt * (double)vt;
        }
    }
    block_sum_pair(s2, 0.0, partials);
}

// ---------------------------------------------------------------------------
// Merge, part 1: u_hat on every line point (a point where two or three plane
// families meet).  Enumeration: for each family a the points of L_a that are
// not knots (coordinate a fine and not a multiple of n), then the knots.
//   initial guess (lines and coarse given, R21):
//     on L_a (not a knot):  u_hat = U_pa + U_qa - L_a,
//     knots:                u_hat = U_x + U_y + U_z - L_x - L_y - L_z + C;
//   a sweep's correction (R22): the value of the drawn family if its planes
//   contain the point, else of the next family in the order x -> y -> z -> x.
// Plane values are scaled by 1/||U_a|| when norms are given (R24).
// ---------------------------------------------------------------------------
template <typename T>
struct Merge3Args {
    const T* U[3];          // plane solutions [k][q][p]
    const double* nrm2;     // ||U_a||^2 at nrm2[2 a] (sweep correction) or null
    const T* Lf[3];         // line solutions [f][cq][cp] (initial guess) or null
    const T* Cc;            // coarse solution [cz][cy][cx] (initial guess) or null
    int choice;             // drawn family (sweep correction)
    T* uh;                  // full grid: u_hat on the line points
    const T* W;             // spline values [N_f][N_c]
    T* z;                   // full grid: receives the merged skeleton
};

__device__ __forceinline__ double plane_scale(const double* nrm2, int a) {
    if (!nrm2) return 1.0;
    const double v = nrm2[2 * a];
    return v > 0.0 ? 1.0 / sqrt(v) : 1.0;
}

template <typename T>
__device__ __forceinline__ double plane_at(const Merge3Args<T>& m, const Geo3& g, int a, const int c[3], double sc) {
    int pa, qa;
    other_axes(a, pa, qa);
    const long long e = ((long long)(c[a] / g.n - 1) * g.Nf + (c[qa] - 1)) * g.Nf + (c[pa] - 1);
    return sc * (double)m.U[a][e];
}

template <typename T>
__global__ void __launch_bounds__(T3) uhat3_kernel(Merge3Args<T> m, Geo3 g) {
    const int n = g.n, Nc = g.Nc, N = g.N;
    const long long per = (long long)(g.Nf - Nc) * Nc * Nc, count = 3 * per + (long long)Nc * Nc * Nc;
    double sc[3];
    for (int a = 0; a < 3; ++a) sc[a] = plane_scale(m.nrm2, a);
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < count; e += (long long)gridDim.x * T3) {
        int c[3];
        int a = -1;                       // the line family (fine axis), -1 for a knot
        if (e < 3 * per) {
            a = (int)(e / per);
            const long long r = e % per;
            int pa, qa;
            other_axes(a, pa, qa);
            const int cp = (int)(r % Nc), cq = (int)((r / Nc) % Nc), t = (int)(r / ((long long)Nc * Nc));
            c[a] = t + 1 + t / (n - 1);   // the t-th fine coordinate that is not a multiple of n
            c[pa] = (cp + 1) * n;
            c[qa] = (cq + 1) * n;
        } else {
            const long long r = e - 3 * per;
            c[0] = (int)(r % Nc + 1) * n; c[1] = (int)((r / Nc) % Nc + 1) * n; c[2] = (int)(r / ((long long)Nc * Nc) + 1) * n;
        }
        double v;
        if (m.Lf[0]) {
            auto line_at = [&](int b) {
                int pb, qb;
                other_axes(b, pb, qb);
                return (double)m.Lf[b][((long long)(c[b] - 1) * Nc + (c[qb] / n - 1)) * Nc + (c[pb] / n - 1)];
            };
            if (a >= 0) {
                int pa, qa;
                other_axes(a, pa, qa);
                v = plane_at(m, g, pa, c, sc[pa]) + plane_at(m, g, qa, c, sc[qa]) - line_at(a);
            } else {
                v = plane_at(m, g, 0, c, sc[0]) + plane_at(m, g, 1, c, sc[1]) + plane_at(m, g, 2, c, sc[2])
                  - line_at(0) - line_at(1) - line_at(2)
                  + (double)m.Cc[((long long)(c[2] / n - 1) * Nc + (c[1] / n - 1)) * Nc + (c[0] / n - 1)];
            }
        } else {
            int f = m.choice;
            if (a >= 0 && f == a) f = (f + 1) % 3;          // the drawn family does not contain this line
            v = plane_at(m, g, f, c, sc[f]);
        }
        m.uh[((long long)c[2] * N + c[1]) * N + c[0]] = (T)v;
    }
}

// ---------------------------------------------------------------------------
// Merge, part 2: every plane of every family moved onto u_hat (R23).  On the
// plane of family a at coordinate (k+1) n, with its fine axes p < q and the
// mismatch E = u_hat - U_a on the plane's lines,
//   corr(p, q) = sum_m W[p][m] E(knot m, q) + sum_m W[q][m] E(p, knot m)
//              - sum_m W[p][m] sum_m' W[q][m'] E(knot m, knot m'),
// the Boolean sum S_p E + S_q E - S_p S_q E of the not-a-knot splines.  The
// value U_a + corr is written where family a is the last of x, y, z whose
// planes contain the point.  One CTA per 32 x 8 tile of one plane.
// ---------------------------------------------------------------------------
constexpr int MP = 32, MQ = 8;

template <typename T>
__global__ void __launch_bounds__(MP * MQ) plane_corr_kernel(Merge3Args<T> m, Geo3 g) {
    __shared__ double Wp[MP][kMaxNc3], Wq[MQ][kMaxNc3], Ekk[kMaxNc3][kMaxNc3];
    __shared__ double Eq[kMaxNc3][MQ], Ep[MP][kMaxNc3], Tm[kMaxNc3][MQ];
    const int Nf = g.Nf, Nc = g.Nc, n = g.n, N = g.N;
    const int a = blockIdx.z / Nc, k = blockIdx.z % Nc;
    int pa, qa;
    other_axes(a, pa, qa);
    const int p0 = blockIdx.x * MP, q0 = blockIdx.y * MQ, tid = threadIdx.x;
    const double sc = plane_scale(m.nrm2, a);
    const T* U = m.U[a];
    const long long P = g.plane;
    // E at plane point (pi, qi) (0-based fine indices), a line point of this plane.
    auto E = [&](int pi, int qi) -> double {
        int c[3];
        c[a] = (k + 1) * n; c[pa] = pi + 1; c[qa] = qi + 1;
        return (double)m.uh[((long long)c[2] * N + c[1]) * N + c[0]]
             - sc * (double)U[(long long)k * P + (long long)qi * Nf + pi];
    };
    for (int t = tid; t < MP * Nc; t += MP * MQ) {
        const int r = t / Nc, mm = t % Nc, pi = p0 + r;
        Wp[r][mm] = pi < Nf ? (double)m.W[(long long)pi * Nc + mm] : 0.0;
        Ep[r][mm] = pi < Nf ? E(pi, (mm + 1) * n - 1) : 0.0;
    }
    for (int t = tid; t < MQ * Nc; t += MP * MQ) {
        const int r = t / Nc, mm = t % Nc, qi = q0 + r;
        Wq[r][mm] = qi < Nf ? (double)m.W[(long long)qi * Nc + mm] : 0.0;
        Eq[mm][r] = qi < Nf ? E((mm + 1) * n - 1, qi) : 0.0;
    }
    for (int t = tid; t < Nc * Nc; t += MP * MQ) {
        const int r = t / Nc, mm = t % Nc;
        Ekk[r][mm] = E((r + 1) * n - 1, (mm + 1) * n - 1);
    }
    __syncthreads();
    for (int t = tid; t < Nc * MQ; t += MP * MQ) {
        const int mm = t / MQ, r = t % MQ;
        double v = 0.0;
        for (int m2 = 0; m2 < Nc; ++m2) v += Wq[r][m2] * Ekk[mm][m2];
        Tm[mm][r] = v;
    }
    __syncthreads();
    const int tp = tid % MP, tq = tid / MP, pi = p0 + tp, qi = q0 + tq;
    if (pi >= Nf || qi >= Nf) return;
    double corr = 0.0;
    for (int mm = 0; mm < Nc; ++mm) corr += Wp[tp][mm] * (Eq[mm][tq] - Tm[mm][tq]) + Wq[tq][mm] * Ep[tp][mm];
    int c[3];
    c[a] = (k + 1) * n; c[pa] = pi + 1; c[qa] = qi + 1;
    int owner = a;
    if (c[pa] % n == 0 && pa > owner) owner = pa;
    if (c[qa] % n == 0 && qa > owner) owner = qa;
    if (owner != a) return;
    m.z[((long long)c[2] * N + c[1]) * N + c[0]] = (T)(sc * (double)U[(long long)k * P + (long long)qi * Nf + pi] + corr);
}

// ---------------------------------------------------------------------------
// Filler (Algorithm 3) on the cube holes as one batched block cyclic
// reduction: right-hand sides [hole][lz][ly (n-1) + lx] and the scatter back.
//   mode 0: s - (stencil terms reaching outside the hole) . z   (z: skeleton and g on the ring)
//   mode 1: -(stencil terms reaching outside the hole) . z     (zero source)
//   mode 2: s - A u at the hole point (FP64), the hole part of the residual;
//           the scatter then adds the solution to u (R18);
//   mode 3: the values of the FP64 grid s at the hole points; the scatter
//           writes the solution into the FP64 grid u (single-solve checks).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void hole_point(long long e, const Geo3& g, int& i, int& j, int& l, int& lx, int& ly,
                                           int& lz) {
    const int hc = g.hc, mc = g.mc;
    const long long h3 = (long long)hc * hc * hc;
    const long long hole = e / h3, loc = e % h3;
    lx = (int)(loc % hc); ly = (int)((loc / hc) % hc); lz = (int)(loc / ((long long)hc * hc));
    const int hx = (int)(hole % mc), hy = (int)((hole / mc) % mc), hz = (int)(hole / ((long long)mc * mc));
    i = hx * g.n + 1 + lx; j = hy * g.n + 1 + ly; l = hz * g.n + 1 + lz;
}

template <typename T>
__global__ void __launch_bounds__(T3)
hole_rhs3_kernel(int mode, const T* __restrict__ z, const double* __restrict__ s, const double* __restrict__ u, Geo3 g,
                 Sten3 c, T* __restrict__ X) {
    const long long count = (long long)g.mc * g.mc * g.mc * g.hc * g.hc * g.hc;
    const int N = g.N, hc = g.hc;
    const long long NN2 = (long long)N * N;
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < count; e += (long long)gridDim.x * T3) {
        int i, j, l, lx, ly, lz;
        hole_point(e, g, i, j, l, lx, ly, lz);
        const long long idx = ((long long)l * N + j) * N + i;
        double r;
        if (mode == 3) {
            r = s[idx];
        } else if (mode == 2) {
            r = s[idx] - (c.cc * u[idx] + c.cw * u[idx - 1] + c.ce * u[idx + 1] + c.cs * u[idx - N] + c.cn * u[idx + N]
                          + c.cd * u[idx - NN2] + c.cu * u[idx + NN2]);
        } else {
            r = mode == 0 ? s[idx] : 0.0;
            if (lx == 0) r -= c.cw * (double)z[idx - 1];
            if (lx == hc - 1) r -= c.ce * (double)z[idx + 1];
            if (ly == 0) r -= c.cs * (double)z[idx - N];
            if (ly == hc - 1) r -= c.cn * (double)z[idx + N];
            if (lz == 0) r -= c.cd * (double)z[idx - NN2];
            if (lz == hc - 1) r -= c.cu * (double)z[idx + NN2];
        }
        X[e] = (T)r;
    }
}

template <typename T>
__global__ void __launch_bounds__(T3)
hole_scatter3_kernel(int mode, const T* __restrict__ Y, Geo3 g, T* __restrict__ z, double* __restrict__ u) {
    const long long count = (long long)g.mc * g.mc * g.mc * g.hc * g.hc * g.hc;
    const int N = g.N;
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < count; e += (long long)gridDim.x * T3) {
        int i, j, l, lx, ly, lz;
        hole_point(e, g, i, j, l, lx, ly, lz);
        const long long idx = ((long long)l * N + j) * N + i;
        if (mode == 2) u[idx] += (double)Y[e];
        else if (mode == 3) u[idx] = (double)Y[e];
        else z[idx] = Y[e];
    }
}

// out (FP64 grid) = z at the hole points.
template <typename T>
__global__ void __launch_bounds__(T3) hole_copy3_kernel(const T* __restrict__ z, Geo3 g, double* __restrict__ out) {
    const long long count = (long long)g.mc * g.mc * g.mc * g.hc * g.hc * g.hc;
    const int N = g.N;
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < count; e += (long long)gridDim.x * T3) {
        int i, j, l, lx, ly, lz;
        hole_point(e, g, i, j, l, lx, ly, lz);
        const long long idx = ((long long)l * N + j) * N + i;
        out[idx] = (double)z[idx];
    }
}

// q = A z on the compact skeleton (T arithmetic).
template <typename T>
__global__ void __launch_bounds__(T3)
skel_apply3_kernel(const T* __restrict__ z, Geo3 g, Sten3 c, T* __restrict__ q) {
    const int N = g.N, Nf = g.Nf, n = g.n;
    const long long NN2 = (long long)N * N;
    const T cc = (T)c.cc, cw = (T)c.cw, ce = (T)c.ce, cs = (T)c.cs, cn = (T)c.cn, cd = (T)c.cd, cu = (T)c.cu;
    for (long long row = blockIdx.x; row < (long long)Nf * Nf; row += gridDim.x) {
        const int j = (int)(row % Nf) + 1, l = (int)(row / Nf) + 1;
        const bool row_coarse = j % n == 0 || l % n == 0;
        const long long base = ((long long)l * N + j) * N;
        for (int i = 1 + threadIdx.x; i <= N - 2; i += T3) {
            if (!row_coarse && i % n != 0) continue;
            const long long idx = base + i;
            q[skel3_index(i, j, l, g)] = cc * z[idx] + cw * z[idx - 1] + ce * z[idx + 1] + cs * z[idx - N]
                                        + cn * z[idx + N] + cd * z[idx - NN2] + cu * z[idx + NN2];
        }
    }
}

// z (T grid): its ring from u's ring (g) or zero, its interior zero.
template <typename T>
__global__ void __launch_bounds__(T3) ring3_kernel(const double* __restrict__ u, Geo3 g, T* __restrict__ z) {
    const int N = g.N;
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < g.NN; e += (long long)gridDim.x * T3) {
        const int i = (int)(e % N), j = (int)((e / N) % N), l = (int)(e / ((long long)N * N));
        const bool ring = i == 0 || j == 0 || l == 0 || i == N - 1 || j == N - 1 || l == N - 1;
        z[e] = ring && u ? (T)u[e] : (T)0;
    }
}

// u interior = z interior (converted), ring untouched.
template <typename T>
__global__ void __launch_bounds__(T3) interior3_kernel(const T* __restrict__ z, Geo3 g, double* __restrict__ u) {
    const int N = g.N, Nf = g.Nf;
    for (long long row = blockIdx.x; row < (long long)Nf * Nf; row += gridDim.x) {
        const int j = (int)(row % Nf) + 1, l = (int)(row / Nf) + 1;
        const long long base = ((long long)l * N + j) * N;
        for (int i = 1 + threadIdx.x; i <= N - 2; i += T3) u[base + i] = (double)z[base + i];
    }
}

// Plain copies (FP64 -> T) of submesh arrays, for single-solve checks.
template <typename Ts, typename Td>
__global__ void __launch_bounds__(T3) convert3_kernel(const Ts* __restrict__ a, long long n, Td* __restrict__ b) {
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < n; e += (long long)gridDim.x * T3) b[e] = (Td)a[e];
}

// ---------------------------------------------------------------------------
// GCR with a long memory on the skeleton (R15 with the residual tracked on the
// skeleton rows between true residuals; by Prop. 3.1 A e vanishes in the holes).
//   dots:    for the new image q and the tracked residual r (FP64):
//            out = [<q,q>, <q,r>, <r,r>, <q,V_j> (j < k), <r,V_j> (j < k)]
//            partials [column][chunk], then summed per column in chunk order;
//   combine: V_k = (q - sum_j beta_j V_j) * inv_nu,  r -= alpha V_k, with the
//            partial sums of the new r^2;
//   planes:  the plane families' right-hand sides from the tracked residual;
//   update:  u += sum_j c_j Z_j over the interior (FP64 accumulation).
// ---------------------------------------------------------------------------
constexpr int DK_CHUNKS = 256;     // skeleton chunks of the many-vector dots
constexpr int DK_VEC = 8;          // vectors per CTA

template <typename T>
__global__ void __launch_bounds__(T3)
dots_many_kernel(const T* __restrict__ q, const double* __restrict__ r, const T* __restrict__ V, long long n,
                 long long vstride, int k, double* __restrict__ partials) {
    __shared__ double red[T3 / 32][2 * DK_VEC + 3];
    const int chunk = blockIdx.x, j0 = blockIdx.y * DK_VEC;
    const long long len = (n + DK_CHUNKS - 1) / DK_CHUNKS, e0 = chunk * len, e1 = min(n, e0 + len);
    const int nv = min(DK_VEC, k - j0);
    double acc[2 * DK_VEC + 3];
#pragma unroll
    for (int t = 0; t < 2 * DK_VEC + 3; ++t) acc[t] = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += T3) {
        const double qv = (double)q[e], rv = r[e];
        if (blockIdx.y == 0) { acc[0] += qv * qv; acc[1] += qv * rv; acc[2] += rv * rv; }
#pragma unroll
        for (int t = 0; t < DK_VEC; ++t)
            if (t < nv) {
                const double v = (double)V[(long long)(j0 + t) * vstride + e];
                acc[3 + t] += qv * v;
                acc[3 + DK_VEC + t] += rv * v;
            }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 2 * DK_VEC + 3; ++t) {
        double v = acc[t];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
        if (lane == 0) red[w][t] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * DK_VEC + 3) {
        const int t = threadIdx.x;
        double v = 0.0;
        for (int q2 = 0; q2 < T3 / 32; ++q2) v += red[q2][t];
        // column layout: 0, 1, 2 then <q,V_j> at 3 + j, <r,V_j> at 3 + k + j
        int col = -1;
        if (t < 3) col = blockIdx.y == 0 ? t : -1;
        else if (t < 3 + DK_VEC) col = (t - 3 < nv) ? 3 + j0 + (t - 3) : -1;
        else col = (t - 3 - DK_VEC < nv) ? 3 + k + j0 + (t - 3 - DK_VEC) : -1;
        if (col >= 0) partials[(long long)col * DK_CHUNKS + chunk] = v;
    }
}

__global__ void __launch_bounds__(32) sum_chunks_kernel(const double* __restrict__ partials, int ncols,
                                                        double* __restrict__ out) {
    const int col = blockIdx.x * 32 + threadIdx.x;
    if (col >= ncols) return;
    double v = 0.0;
    for (int c = 0; c < DK_CHUNKS; ++c) v += partials[(long long)col * DK_CHUNKS + c];
    out[col] = v;
}

template <typename T>
__global__ void __launch_bounds__(T3)
combine_many_kernel(const T* __restrict__ q, T* __restrict__ V, long long n, long long vstride, int k,
                    const double* __restrict__ beta, double inv_nu, double alpha, double* __restrict__ r,
                    double* __restrict__ partials) {
    double rr = 0.0;
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < n; e += (long long)gridDim.x * T3) {
        double v = (double)q[e];
        for (int j = 0; j < k; ++j) v -= beta[j] * (double)V[(long long)j * vstride + e];
        const T vk = (T)(v * inv_nu);
        V[(long long)k * vstride + e] = vk;
        const double rn = r[e] - alpha * (double)vk;
        r[e] = rn;
        rr += rn * rn;
    }
    block_sum_pair(rr, 0.0, partials);
}

// rs (FP64) or, when rh is given, the float pairs rh + rl of the FP32 path.
template <typename T>
__global__ void __launch_bounds__(T3) planes_from_skel_kernel(const double* __restrict__ rs, const float* __restrict__ rh,
                                                              const float* __restrict__ rl, Geo3 g, T* F0, T* F1,
                                                              T* F2) {
    const int Nf = g.Nf, n = g.n;
    const long long P = g.plane;
    for (long long row = blockIdx.x; row < (long long)Nf * Nf; row += gridDim.x) {
        const int j = (int)(row % Nf) + 1, l = (int)(row / Nf) + 1;
        const bool row_coarse = j % n == 0 || l % n == 0;
        for (int i = 1 + threadIdx.x; i <= Nf; i += T3) {
            if (!row_coarse && i % n != 0) continue;
            const long long si = skel3_index(i, j, l, g);
            const T rt = rh ? (T)(rh[si] + rl[si]) : (T)rs[si];
            if (i % n == 0) F0[(long long)(i / n - 1) * P + (long long)(l - 1) * Nf + (j - 1)] = rt;
            if (j % n == 0) F1[(long long)(j / n - 1) * P + (long long)(l - 1) * Nf + (i - 1)] = rt;
            if (l % n == 0) F2[(long long)(l / n - 1) * P + (long long)(j - 1) * Nf + (i - 1)] = rt;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(T3)
update_many_kernel(double* __restrict__ u, const T* __restrict__ Z, long long zstride, int k,
                   const double* __restrict__ c, Geo3 g) {
    __shared__ double cs[1024];
    for (int j = threadIdx.x; j < k && j < 1024; j += T3) cs[j] = c[j];
    __syncthreads();
    const int N = g.N, Nf = g.Nf;
    for (long long row = blockIdx.x; row < (long long)Nf * Nf; row += gridDim.x) {
        const int j = (int)(row % Nf) + 1, l = (int)(row / Nf) + 1;
        const long long base = ((long long)l * N + j) * N;
        for (int i = 1 + threadIdx.x; i <= N - 2; i += T3) {
            const long long idx = base + i;
            double v = 0.0;
            for (int t = 0; t < k; ++t) v += cs[t] * (double)Z[(long long)t * zstride + idx];
            u[idx] += v;
        }
    }
}

// ---------------------------------------------------------------------------
// The same three operations for FP32 directions, without the FP64 pipe in the
// inner loops (on GB300 it runs at 1/64 of the FP32 rate): every product is
// made exact by the FMA-based TwoProd and accumulated as an unevaluated pair
// (hi, lo) by TwoSum (Knuth), the compensated dot product "Dot2" of Ogita,
// Rump and Oishi (2005), accurate as if computed in twice the working
// precision.  FP64 coefficients enter as float pairs (hi, lo); an FP64
// operand (the tracked residual) is split into a float pair once per element.
// ---------------------------------------------------------------------------
struct F2 { float h, l; };

__device__ __forceinline__ void acc_prod(F2& s, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);                 // a b = p + e exactly
    const float t = s.h + p;
    const float z = t - s.h;
    s.l += ((s.h - (t - z)) + (p - z)) + e;          // TwoSum error of s.h + p, plus e
    s.h = t;
}

__device__ __forceinline__ double f2_value(const F2& s) { return (double)s.h + (double)s.l; }

__global__ void __launch_bounds__(T3)
dots_many_f32_kernel(const float* __restrict__ q, const float* __restrict__ rhv, const float* __restrict__ rlv,
                     const float* __restrict__ V, long long n, long long vstride, int k, double* __restrict__ partials) {
    __shared__ double red[T3 / 32][2 * DK_VEC + 3];
    const int chunk = blockIdx.x, j0 = blockIdx.y * DK_VEC;
    const long long len = (n + DK_CHUNKS - 1) / DK_CHUNKS, e0 = chunk * len, e1 = min(n, e0 + len);
    const int nv = min(DK_VEC, k - j0);
    F2 aq[DK_VEC], ar[DK_VEC], a0 = {0.f, 0.f}, a1 = {0.f, 0.f}, a2 = {0.f, 0.f};
#pragma unroll
    for (int t = 0; t < DK_VEC; ++t) { aq[t] = {0.f, 0.f}; ar[t] = {0.f, 0.f}; }
    for (long long e = e0 + threadIdx.x; e < e1; e += T3) {
        const float qv = q[e];
        const float rh = rhv[e], rl = rlv[e];    // r's float pair (no FP64 work per element here)
        if (blockIdx.y == 0) {
            acc_prod(a0, qv, qv);
            acc_prod(a1, qv, rh);
            a1.l = fmaf(qv, rl, a1.l);
            acc_prod(a2, rh, rh);
            a2.l = fmaf(2.0f * rh, rl, a2.l);
        }
#pragma unroll
        for (int t = 0; t < DK_VEC; ++t)
            if (t < nv) {
                const float v = V[(long long)(j0 + t) * vstride + e];
                acc_prod(aq[t], qv, v);
                acc_prod(ar[t], rh, v);
                ar[t].l = fmaf(rl, v, ar[t].l);
            }
    }
    // Warp sums of the pairs with TwoSum (FP32 only), FP64 once per warp and value.
    F2 acc[2 * DK_VEC + 3];
    acc[0] = a0; acc[1] = a1; acc[2] = a2;
#pragma unroll
    for (int t = 0; t < DK_VEC; ++t) { acc[3 + t] = aq[t]; acc[3 + DK_VEC + t] = ar[t]; }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 2 * DK_VEC + 3; ++t) {
        float hi = acc[t].h, lo = acc[t].l;
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_down_sync(0xFFFFFFFFu, hi, o), l2 = __shfl_down_sync(0xFFFFFFFFu, lo, o);
            const float sm = hi + h2, bp = sm - hi;
            const float er = (hi - (sm - bp)) + (h2 - bp);
            hi = sm;
            lo = lo + l2 + er;
        }
        if (lane == 0) red[w][t] = (double)hi + (double)lo;
    }
    __syncthreads();
    if (threadIdx.x < 2 * DK_VEC + 3) {
        const int t = threadIdx.x;
        double v = 0.0;
        for (int q2 = 0; q2 < T3 / 32; ++q2) v += red[q2][t];
        int col = -1;
        if (t < 3) col = blockIdx.y == 0 ? t : -1;
        else if (t < 3 + DK_VEC) col = (t - 3 < nv) ? 3 + j0 + (t - 3) : -1;
        else col = (t - 3 - DK_VEC < nv) ? 3 + k + j0 + (t - 3 - DK_VEC) : -1;
        if (col >= 0) partials[(long long)col * DK_CHUNKS + chunk] = v;
    }
}

// r as float pairs (hi, lo): rh = fl(r), rl = fl(r - rh); |r - rh - rl| <= 2^-48 |r|.
__global__ void __launch_bounds__(T3) split_pairs_kernel(const double* __restrict__ r, long long n,
                                                         float* __restrict__ rh, float* __restrict__ rl) {
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < n; e += (long long)gridDim.x * T3) {
        const double v = r[e];
        const float h = (float)v;
        rh[e] = h;
        rl[e] = (float)(v - (double)h);
    }
}

// V_k = (q - sum_j beta_j V_j) * inv_nu (beta as float pairs) and the tracked
// residual, held as float pairs (rh, rl), r -= alpha V_k (alpha as a float pair):
// FP32 operations only (TwoProd, TwoSum, then Fast2Sum to renormalise).
__global__ void __launch_bounds__(T3)
combine_many_f32_kernel(const float* __restrict__ q, float* __restrict__ V, long long n, long long vstride, int k,
                        const float2* __restrict__ beta, float inv_nu, float ah, float al, float* __restrict__ rh,
                        float* __restrict__ rl) {
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < n; e += (long long)gridDim.x * T3) {
        F2 acc = {q[e], 0.f};
        for (int j = 0; j < k; ++j) {
            const float v = V[(long long)j * vstride + e];
            const float2 b = beta[j];
            acc_prod(acc, -b.x, v);
            acc.l = fmaf(-b.y, v, acc.l);
        }
        const float vk = fmaf(acc.h, inv_nu, acc.l * inv_nu);
        V[(long long)k * vstride + e] = vk;
        // (h, l) - (ah + al) vk
        const float p = ah * vk;
        const float pe = fmaf(ah, vk, -p);            // ah vk = p + pe exactly
        const float h = rh[e], l = rl[e];
        const float s = h - p, z = s - h;
        const float t = (h - (s - z)) - (p + z);      // TwoSum error of h - p
        const float lo = ((l + t) - pe) - al * vk;
        const float sh = s + lo;                      // Fast2Sum (|s| >= |lo| in practice)
        rl[e] = lo - (sh - s);
        rh[e] = sh;
    }
}

// u += sum_j c_j Z_j over the interior (c as float pairs), one FP64 add per point.
__global__ void __launch_bounds__(T3)
update_many_f32_kernel(double* __restrict__ u, const float* __restrict__ Z, long long zstride, int k,
                       const float2* __restrict__ c, Geo3 g) {
    __shared__ float2 cs[1024];
    for (int j = threadIdx.x; j < k && j < 1024; j += T3) cs[j] = c[j];
    __syncthreads();
    const int N = g.N, Nf = g.Nf;
    for (long long row = blockIdx.x; row < (long long)Nf * Nf; row += gridDim.x) {
        const int j = (int)(row % Nf) + 1, l = (int)(row / Nf) + 1;
        const long long base = ((long long)l * N + j) * N;
        for (int i = 1 + threadIdx.x; i <= N - 2; i += T3) {
            const long long idx = base + i;
            F2 acc = {0.f, 0.f};
            for (int t = 0; t < k; ++t) {
                const float z = Z[(long long)t * zstride + idx];
                acc_prod(acc, cs[t].x, z);
                acc.l = fmaf(cs[t].y, z, acc.l);
            }
            u[idx] += f2_value(acc);
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

#define CK3(...)                                          \
    do {                                                  \
        cudaError_t e__ = (__VA_ARGS__);                  \
        if (e__ != cudaSuccess) return report_cuda_error(e__); \
    } while (0)

// BCR factors on the device in one precision.
struct Fac {
    void* Mt = nullptr; void* Bt = nullptr;
    void* Dt = nullptr;                 // FP32 plane blocks: the dense tail map (BcrSys::Dt)
    int tail_rt = 0, tail_ld = 0;
    double wl[kMaxLevels] = {}, wr[kMaxLevels] = {};
    int R = 0, C = 0, L = 0;
};

template <typename T>
int upload_fac(const BcrFactors& f, Fac* d) {
    const size_t n = f.Mt.size();
    std::vector<T> tmp(n);
    void** dst[2] = {&d->Mt, &d->Bt};
    const std::vector<double>* src[2] = {&f.Mt, &f.Bt};
    for (int q = 0; q < 2; ++q) {
        CK3(cudaMalloc(dst[q], n * sizeof(T)));
        for (size_t e = 0; e < n; ++e) tmp[e] = (T)(*src[q])[e];
        CK3(cudaMemcpy(*dst[q], tmp.data(), n * sizeof(T), cudaMemcpyHostToDevice));
    }
    for (int l = 0; l < f.L; ++l) { d->wl[l] = f.wl[l]; d->wr[l] = f.wr[l]; }
    d->R = f.R; d->C = f.C; d->L = f.L;
    return ASDSM_OK;
}

void free_fac(Fac& d) {
    if (d.Mt) cudaFree(d.Mt);
    if (d.Bt) cudaFree(d.Bt);
    if (d.Dt) cudaFree(d.Dt);
    d.Mt = d.Bt = d.Dt = nullptr;
}

template <typename T>
BcrSys<T> sys3(const Fac& d, void* X, void* Y, int nsys = 1) {
    BcrSys<T> s{};
    s.X = (T*)X; s.Y = (T*)Y;
    s.Mt = (const T*)d.Mt; s.Bt = (const T*)d.Bt;
    for (int l = 0; l < d.L; ++l) { s.wl[l] = (T)d.wl[l]; s.wr[l] = (T)d.wr[l]; }
    s.R = d.R; s.C = d.C; s.L = d.L; s.nsys = nsys;
    s.stride = (long long)d.R * d.C;
    s.Dt = (const float*)d.Dt; s.tail_rt = d.tail_rt; s.tail_ld = d.tail_ld;
    return s;
}

// 1D three-point operator of axis a on spacing sp: (lower, diagonal, upper).
struct Op1 { double lo, di, up; };
Op1 op1(double alpha, double beta, double sp) {
    return {-alpha / (sp * sp) - beta / (2 * sp), 2 * alpha / (sp * sp), -alpha / (sp * sp) + beta / (2 * sp)};
}

// Dense Kronecker sum  T_q (x) I + I (x) T_p + d I  on a [q][p] grid (p fastest).
std::vector<double> kron_sum2(int nq, Op1 tq, int np, Op1 tp, double d) {
    const int C = nq * np;
    std::vector<double> K((size_t)C * C, 0.0);
    for (int q = 0; q < nq; ++q)
        for (int p = 0; p < np; ++p) {
            const size_t r = (size_t)q * np + p;
            K[r * C + r] = tq.di + tp.di + d;
            if (p > 0) K[r * C + r - 1] = tp.lo;
            if (p + 1 < np) K[r * C + r + 1] = tp.up;
            if (q > 0) K[r * C + r - np] = tq.lo;
            if (q + 1 < nq) K[r * C + r + np] = tq.up;
        }
    return K;
}

struct PlaneFam {
    std::vector<int> bk, bs;             // Schur blocks: first index, size (1 or 2), in back-substitution order
    std::vector<double> Q, S;            // N_c x N_c
    std::vector<Fac> fac[2];             // per precision, per block
    void* Qd[2] = {nullptr, nullptr};    // Q on the device [j][k] (T)
};

template <typename T>
int upload_vec3(const std::vector<double>& v, void** d) {
    std::vector<T> tmp(v.begin(), v.end());
    CK3(cudaMalloc(d, std::max<size_t>(1, tmp.size()) * sizeof(T)));
    if (!tmp.empty()) CK3(cudaMemcpy(*d, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    return ASDSM_OK;
}

}  // namespace

struct Solver3D {
    asdsm_desc desc{};
    asdsm_opts opts{};
    cudaStream_t st = nullptr;
    int num_sms = 152;
    Geo3 g{};
    Sten3 sten{};
    Lift3 lift{};
    PlaneFam plane[3];
    BcrTune ptune[2][2] = {};                // plane-block level shapes [precision][block size - 1]
    bool ptuned[2] = {false, false};
    Fac line[2][3], coarse[2], hole[2];
    void* W[2] = {nullptr, nullptr};       // spline values [N_f][N_c]
    float* g3img = nullptr;                // hole extension operator G^T as the tensor-core operand image
    float* a3img = nullptr;                // the sweeps' face values as the tensor-core operand image
    int* tc3err = nullptr;                 // set by the tensor-core Filler when a wait timed out
    cudaStream_t fork[2] = {nullptr, nullptr};   // the second and third plane family's streams
    cudaStream_t cap = nullptr;                  // capture stream of the plane-solve graph
    cudaEvent_t evf[3] = {nullptr, nullptr, nullptr};
    struct PlaneGraph { cudaGraphExec_t exec = nullptr; long long launches = 0; int runs = 0; } pgraph[2][2];
    struct Work {
        bool ready = false;
        void* F[3] = {}; void* Y[3] = {}; void* U[3] = {};
        void* Xb[3] = {}; void* Yb[3] = {};   // per plane family, so the three can run concurrently
        void* Xl[3] = {}; void* Yl[3] = {};
        void* Xc = nullptr; void* Yc = nullptr;
        void* Xh = nullptr; void* Yh = nullptr;
        void* uh = nullptr;
        void* Z = nullptr;               // m directions, [m][N^3] (ring zero)
        void* V = nullptr;               // their orthonormalised skeleton images, [m][skel]
        void* q = nullptr;               // the new image A e on the skeleton [skel]
        double* rs = nullptr;            // tracked residual on the skeleton [skel], FP64
        float* rsh = nullptr;            // the same as float pairs (hi, lo), for the FP32 GCR products
        float* rsl = nullptr;
        int m = 0;
    } w[2];
    double* dcoef = nullptr;             // [1024] step coefficients / Gram-Schmidt weights
    float2* dcoef2 = nullptr;            // [1024] the same as float pairs (hi, lo) for the FP32 kernels
    double* dsum = nullptr;              // [2*1024 + 3] many-vector dot results
    double* dpart = nullptr;             // many-vector dot partials [(2*1024 + 3)][DK_CHUNKS]
    double* u_work = nullptr;
    double* partials = nullptr;
    int partials_cap = 0;
    // Per-family CUDA-event timing (asdsm_profile) with algorithmic bytes and flops.
    bool prof = false;
    asdsm_kprof pc[8] = {};
    std::vector<cudaEvent_t> evpool;
    struct Mark { int a, b, cat; long long launches; double bytes, flops; };
    std::vector<Mark> marks;
    int evnext = 0;
    double* dsmall = nullptr;
    double* hsmall = nullptr;
    std::vector<double> hist;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
};

namespace {

// Host FP64 factors of every 3D system, computed in parallel threads.
int build_factors(Solver3D* S) {
    const Geo3& g = S->g;
    const double h = 1.0 / g.M, H = 1.0 / g.mc;
    const double* al = S->desc.alpha;
    const double* be = S->desc.beta;
    Op1 fine[3], crs[3];
    for (int a = 0; a < 3; ++a) { fine[a] = op1(al[a], be[a], h); crs[a] = op1(al[a], be[a], H); }
    // Plane blocks with at least 31 columns and 15 rows also get the dense tail of
    // their FP32 reduction (bcr_tail_map: the last three levels of both directions
    // as one product with a (7 C) x (7 C) map, rows padded to a multiple of 4).
    constexpr int kTailRows = 7;
    struct Job { int kind, a, blk; BcrFactors f; bool ok = false; std::vector<float> timg; int tld = 0; };
    std::vector<Job> jobs;
    // Plane families: Schur form of the coarse-axis operator, then one system per block.
    for (int a = 0; a < 3; ++a) {
        PlaneFam& pf = S->plane[a];
        std::vector<double> T((size_t)g.Nc * g.Nc, 0.0);
        for (int k = 0; k < g.Nc; ++k) {
            T[(size_t)k * g.Nc + k] = crs[a].di;
            if (k > 0) T[(size_t)k * g.Nc + k - 1] = crs[a].lo;
            if (k + 1 < g.Nc) T[(size_t)k * g.Nc + k + 1] = crs[a].up;
        }
        if (!real_schur(g.Nc, T, &pf.Q, &pf.S)) { report_error("3D: Schur form of a coarse-axis operator failed"); return ASDSM_ERR_INVALID; }
        std::vector<int> starts, sizes;
        for (int k = 0; k < g.Nc;) {
            const int bs = (k + 1 < g.Nc && pf.S[(size_t)(k + 1) * g.Nc + k] != 0.0) ? 2 : 1;
            starts.push_back(k); sizes.push_back(bs);
            k += bs;
        }
        pf.bk.assign(starts.rbegin(), starts.rend());     // back-substitution: last block first
        pf.bs.assign(sizes.rbegin(), sizes.rend());
        for (size_t b = 0; b < pf.bk.size(); ++b) jobs.push_back({0, a, (int)b, {}, false});
    }
    for (int a = 0; a < 3; ++a) jobs.push_back({1, a, 0, {}, false});
    jobs.push_back({2, 0, 0, {}, false});
    jobs.push_back({3, 0, 0, {}, false});
    auto run = [&](Job& jb) {
        int pa, qa;
        pa = jb.a == 0 ? 1 : 0;
        qa = jb.a == 2 ? 1 : 2;
        if (jb.kind == 0) {
            // Shifted 2D fine-plane system: rows along q, columns along p (and the pair's two components).
            const PlaneFam& pf = S->plane[jb.a];
            const int k = pf.bk[jb.blk], bs = pf.bs[jb.blk], Nc = g.Nc, Nf = g.Nf;
            if (bs == 1) {
                const double sig = pf.S[(size_t)k * Nc + k];
                std::vector<double> K((size_t)Nf * Nf, 0.0);
                for (int p = 0; p < Nf; ++p) {
                    K[(size_t)p * Nf + p] = fine[pa].di + fine[qa].di + sig;
                    if (p > 0) K[(size_t)p * Nf + p - 1] = fine[pa].lo;
                    if (p + 1 < Nf) K[(size_t)p * Nf + p + 1] = fine[pa].up;
                }
                jb.ok = make_bcr_dense(Nf, fine[qa].lo, fine[qa].up, Nf, K, &jb.f);
            } else {
                const int C = 2 * Nf;
                std::vector<double> K((size_t)C * C, 0.0);
                for (int p = 0; p < Nf; ++p)
                    for (int i = 0; i < 2; ++i) {
                        const size_t r = (size_t)p * 2 + i;
                        K[r * C + r] += fine[pa].di + fine[qa].di;
                        if (p > 0) K[r * C + r - 2] = fine[pa].lo;
                        if (p + 1 < Nf) K[r * C + r + 2] = fine[pa].up;
                        for (int j = 0; j < 2; ++j) K[r * C + (size_t)p * 2 + j] += pf.S[(size_t)(k + i) * Nc + k + j];
                    }
                jb.ok = make_bcr_dense(Nf, fine[qa].lo, fine[qa].up, C, K, &jb.f);
            }
            std::vector<double> D;
            if (jb.ok && jb.f.L >= 4 && jb.f.C >= 31 && bcr_tail_map(jb.f, kTailRows, &D)) {
                const int n = kTailRows * jb.f.C;
                jb.tld = (n + 3) / 4 * 4;
                jb.timg.assign((size_t)n * jb.tld, 0.0f);
                for (int r = 0; r < n; ++r)
                    for (int q = 0; q < n; ++q) jb.timg[(size_t)r * jb.tld + q] = (float)D[(size_t)r * n + q];
            }
        } else if (jb.kind == 1) {
            // Line family: rows along the fine axis a, columns (cq, cp) coarse.
            jb.ok = make_bcr_dense(g.Nf, fine[jb.a].lo, fine[jb.a].up, g.Nc * g.Nc,
                                   kron_sum2(g.Nc, crs[qa], g.Nc, crs[pa], fine[jb.a].di), &jb.f);
        } else if (jb.kind == 2) {
            // Coarse mesh: rows along z, columns (y, x).
            jb.ok = make_bcr_dense(g.Nc, crs[2].lo, crs[2].up, g.Nc * g.Nc,
                                   kron_sum2(g.Nc, crs[1], g.Nc, crs[0], crs[2].di), &jb.f);
        } else {
            // Cube holes: rows along z, columns (y, x), all fine.
            jb.ok = make_bcr_dense(g.hc, fine[2].lo, fine[2].up, g.hc * g.hc,
                                   kron_sum2(g.hc, fine[1], g.hc, fine[0], fine[2].di), &jb.f);
        }
    };
    const unsigned nth = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), (unsigned)jobs.size()));
    std::vector<std::thread> pool;
    size_t next = 0;
    std::mutex mu;
    for (unsigned t = 0; t < nth; ++t)
        pool.emplace_back([&] {
            for (;;) {
                size_t i;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    if (next >= jobs.size()) return;
                    i = next++;
                }
                run(jobs[i]);
            }
        });
    for (auto& th : pool) th.join();
    for (auto& jb : jobs)
        if (!jb.ok) { report_error("3D: block cyclic reduction factors could not be formed"); return ASDSM_ERR_INVALID; }
    // Upload in both precisions.
    for (int a = 0; a < 3; ++a)
        for (int pi = 0; pi < 2; ++pi) S->plane[a].fac[pi].assign(S->plane[a].bk.size(), Fac{});
    for (auto& jb : jobs) {
        for (int pi = 0; pi < 2; ++pi) {
            Fac* d = jb.kind == 0 ? &S->plane[jb.a].fac[pi][jb.blk]
                   : jb.kind == 1 ? &S->line[pi][jb.a] : jb.kind == 2 ? &S->coarse[pi] : &S->hole[pi];
            const int rc = pi == 0 ? upload_fac<double>(jb.f, d) : upload_fac<float>(jb.f, d);
            if (rc) return rc;
            if (pi == 1 && !jb.timg.empty()) {
                CK3(cudaMalloc(&d->Dt, jb.timg.size() * sizeof(float)));
                CK3(cudaMemcpy(d->Dt, jb.timg.data(), jb.timg.size() * sizeof(float), cudaMemcpyHostToDevice));
                d->tail_rt = kTailRows;
                d->tail_ld = jb.tld;
            }
        }
        std::vector<float>().swap(jb.timg);
    }
    for (int a = 0; a < 3; ++a) {
        if (int rc = upload_vec3<double>(S->plane[a].Q, &S->plane[a].Qd[0])) return rc;
        if (int rc = upload_vec3<float>(S->plane[a].Q, &S->plane[a].Qd[1])) return rc;
    }
    const std::vector<double> W = spline_value_operator(g.mc, g.n);
    if (int rc = upload_vec3<double>(W, &S->W[0])) return rc;
    if (int rc = upload_vec3<float>(W, &S->W[1])) return rc;
    // The hole extension operator of the sweeps' Filler (FP32 path).
    {
        const double sten7[7] = {S->sten.cc, S->sten.cw, S->sten.ce, S->sten.cs, S->sten.cn, S->sten.cd, S->sten.cu};
        std::vector<double> G;
        if (!hole_extension_operator_3d(g.hc, sten7, &G)) { report_error("3D: hole extension operator failed"); return ASDSM_ERR_INVALID; }
        const int P = g.hc * g.hc * g.hc, K = 6 * g.hc * g.hc, H = g.mc * g.mc * g.mc;
        std::vector<float> img;
        fill3_tc_gimage(G, P, K, &img);
        CK3(cudaMalloc(&S->g3img, img.size() * sizeof(float)));
        CK3(cudaMemcpy(S->g3img, img.data(), img.size() * sizeof(float), cudaMemcpyHostToDevice));
        const size_t an = fill3_tc_image_floats(H, K);
        CK3(cudaMalloc(&S->a3img, an * sizeof(float)));
        CK3(cudaMemset(S->a3img, 0, an * sizeof(float)));   // the padding stays zero
        CK3(cudaMalloc(&S->tc3err, sizeof(int)));
        CK3(cudaMemset(S->tc3err, 0, sizeof(int)));
    }
    return ASDSM_OK;
}

template <typename T>
int ensure_work3(Solver3D* S, int pi) {
    auto& w = S->w[pi];
    if (w.ready) return ASDSM_OK;
    const Geo3& g = S->g;
    const long long PL = (long long)g.Nc * g.plane;
    auto al = [&](void** p, long long n) -> int {
        CK3(cudaMalloc(p, (size_t)std::max(1LL, n) * sizeof(T)));
        CK3(cudaMemset(*p, 0, (size_t)std::max(1LL, n) * sizeof(T)));
        return ASDSM_OK;
    };
    int rc;
    for (int a = 0; a < 3; ++a) {
        if ((rc = al(&w.F[a], PL)) || (rc = al(&w.Y[a], PL)) || (rc = al(&w.U[a], PL))) return rc;
        if ((rc = al(&w.Xl[a], (long long)g.Nf * g.Nc * g.Nc)) || (rc = al(&w.Yl[a], (long long)g.Nf * g.Nc * g.Nc)))
            return rc;
    }
    for (int a = 0; a < 3; ++a)
        if ((rc = al(&w.Xb[a], 2 * g.plane)) || (rc = al(&w.Yb[a], 2 * g.plane))) return rc;
    const long long nc3 = (long long)g.Nc * g.Nc * g.Nc, nh = (long long)g.mc * g.mc * g.mc * g.hc * g.hc * g.hc;
    if ((rc = al(&w.Xc, nc3)) || (rc = al(&w.Yc, nc3)) || (rc = al(&w.Xh, nh)) || (rc = al(&w.Yh, nh))) return rc;
    const int m = std::max(1, std::min(S->opts.accel_m, kMaxM3));
    if ((rc = al(&w.uh, g.NN)) || (rc = al(&w.q, g.skel)) || (rc = al(&w.Z, m * g.NN)) || (rc = al(&w.V, m * g.skel)))
        return rc;
    CK3(cudaMalloc(&w.rs, (size_t)g.skel * sizeof(double)));
    if (sizeof(T) == 4) {
        CK3(cudaMalloc(&w.rsh, (size_t)g.skel * sizeof(float)));
        CK3(cudaMalloc(&w.rsl, (size_t)g.skel * sizeof(float)));
    }
    w.m = m;
    w.ready = true;
    return ASDSM_OK;
}

void free_work3(Solver3D* S, int pi) {
    for (auto& pg : S->pgraph[pi]) {
        if (pg.exec) cudaGraphExecDestroy(pg.exec);
        pg = Solver3D::PlaneGraph{};
    }
    auto& w = S->w[pi];
    auto fr = [](void*& p) { if (p) cudaFree(p); p = nullptr; };
    for (int a = 0; a < 3; ++a) { fr(w.F[a]); fr(w.Y[a]); fr(w.U[a]); fr(w.Xl[a]); fr(w.Yl[a]); }
    for (int a = 0; a < 3; ++a) { fr(w.Xb[a]); fr(w.Yb[a]); }
    fr(w.Xc); fr(w.Yc); fr(w.Xh); fr(w.Yh); fr(w.uh); fr(w.q); fr(w.Z); fr(w.V);
    if (w.rs) cudaFree(w.rs);
    w.rs = nullptr;
    if (w.rsh) cudaFree(w.rsh);
    if (w.rsl) cudaFree(w.rsl);
    w.rsh = w.rsl = nullptr;
    w.ready = false;
}

}  // namespace

// Largest |s - A u| over the hole points (FP64), per block.
__global__ void __launch_bounds__(T3)
hole_max3_kernel(const double* __restrict__ s, const double* __restrict__ u, Geo3 g, Sten3 c, double* partials) {
    const long long count = (long long)g.mc * g.mc * g.mc * g.hc * g.hc * g.hc;
    const int N = g.N;
    const long long NN2 = (long long)N * N;
    double mx = 0.0;
    for (long long e = blockIdx.x * (long long)T3 + threadIdx.x; e < count; e += (long long)gridDim.x * T3) {
        int i, j, l, lx, ly, lz;
        hole_point(e, g, i, j, l, lx, ly, lz);
        const long long idx = ((long long)l * N + j) * N + i;
        const double r = s[idx] - (c.cc * u[idx] + c.cw * u[idx - 1] + c.ce * u[idx + 1] + c.cs * u[idx - N]
                                   + c.cn * u[idx + N] + c.cd * u[idx - NN2] + c.cu * u[idx + NN2]);
        mx = fmax(mx, fabs(r));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xFFFFFFFFu, mx, o));
    __shared__ double red[T3 / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int q = 0; q < T3 / 32; ++q) m = fmax(m, red[q]);
        partials[blockIdx.x] = m;
    }
}

namespace {

// Kernel families of the 3D sweep for asdsm_profile.
enum Prof3 : int { P3_PLANES = 0, P3_MERGE, P3_FILL, P3_RESID, P3_GCR, P3_UPDATE, P3_HOLEFIX, P3_GUESS, P3_COUNT };
const char* const kProf3Names[P3_COUNT] = {"plane_solves", "merge3", "fill3", "residual3", "gcr3", "update3",
                                           "hole_fix3", "initial_guess3"};

struct PMark3 { int ev = -1; long long launches = 0; };

PMark3 prof3_begin(Solver3D* S) {
    PMark3 m;
    if (!S->prof) return m;
    if (S->evnext + 2 > (int)S->evpool.size()) {
        cudaEvent_t e;
        for (int t = 0; t < 64; ++t)
            if (cudaEventCreate(&e) == cudaSuccess) S->evpool.push_back(e);
    }
    if (S->evnext + 2 > (int)S->evpool.size()) return m;
    m.ev = S->evnext;
    S->evnext += 2;
    m.launches = launch_count();
    cudaEventRecord(S->evpool[m.ev], S->st);
    return m;
}

void prof3_end(Solver3D* S, const PMark3& m, int cat, double bytes, double flops) {
    if (m.ev < 0) return;
    cudaEventRecord(S->evpool[m.ev + 1], S->st);
    S->marks.push_back({m.ev, m.ev + 1, cat, launch_count() - m.launches, bytes, flops});
}

void prof3_resolve(Solver3D* S) {
    if (!S->prof) return;
    for (const auto& mk : S->marks) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, S->evpool[mk.a], S->evpool[mk.b]);
        asdsm_kprof& r = S->pc[mk.cat];
        r.launches += mk.launches;
        r.calls += 1;
        r.ms += ms;
        r.bytes += mk.bytes;
        r.flops += mk.flops;
    }
    S->marks.clear();
    S->evnext = 0;
}

// Multiply-adds of one block cyclic reduction: 2 C^2 per reduced row, 3 C^2 per solved row.
double bcr_macs3(int R, int C, int L) {
    const double c2 = (double)C * C;
    double macs = 0.0;
    for (int l = 0; l + 1 < L; ++l) macs += (double)(((R + 1) >> (l + 1)) - 1) * 2.0 * c2;
    for (int l = 0; l < L; ++l) {
        const double rb = (double)((R + 1) >> (l + 1));
        macs += rb * c2 + 2.0 * (rb - 1.0) * c2;
    }
    return macs;
}

unsigned g1d(long long n) {
    long long b = (n + T3 - 1) / T3;
    return (unsigned)(b < 1 ? 1 : (b > 152LL * 16 ? 152LL * 16 : b));
}

// Plane family a: F[a] -> U[a] (Schur back-substitution of shifted 2D solves),
// with the partial sums of U^2 at partials + off (2 values per block).
template <typename T>
int plane_solve3(Solver3D* S, int pi, int a, double* partials, int* nblocks, cudaStream_t st) {
    auto& w = S->w[pi];
    const Geo3& g = S->g;
    const PlaneFam& pf = S->plane[a];
    const long long P = g.plane;
    const T* F = (const T*)w.F[a];
    T* Y = (T*)w.Y[a];
    for (size_t b = 0; b < pf.bk.size(); ++b) {
        const int k = pf.bk[b], bs = pf.bs[b];
        SchurStep ss{};
        ss.k = k; ss.bs = bs; ss.Nc = g.Nc;
        for (int i = 0; i < bs; ++i)
            for (int j = 0; j < g.Nc; ++j) {
                ss.q[i][j] = pf.Q[(size_t)j * g.Nc + k + i];
                ss.s[i][j] = j >= k + bs ? pf.S[(size_t)(k + i) * g.Nc + j] : 0.0;
            }
        schur_rhs_kernel<T><<<g1d(P), T3, 0, st>>>(F, Y, P, ss, (T*)w.Xb[a]);
        note_launch();
        CK3(cudaGetLastError());
        BcrSys<T> sys = sys3<T>(pf.fac[pi][b], w.Xb[a], bs == 1 ? (void*)(Y + (long long)k * P) : w.Yb[a]);
        CK3(bcr_solve<T>(&sys, 1, st, S->ptuned[pi] ? &S->ptune[pi][bs - 1] : nullptr));
        if (bs == 2) {
            deinterleave_kernel<T><<<g1d(P), T3, 0, st>>>((const T*)w.Yb[a], P, Y + (long long)k * P,
                                                         Y + (long long)(k + 1) * P);
            note_launch();
            CK3(cudaGetLastError());
        }
    }
    const unsigned nb = g1d(P);
    schur_back_kernel<T><<<nb, T3, 0, st>>>(Y, (const T*)pf.Qd[pi], g.Nc, P, (T*)w.U[a], partials);
    note_launch();
    CK3(cudaGetLastError());
    *nblocks = (int)nb;
    return ASDSM_OK;
}

// The three plane families, each on its own stream (forked from and joined
// back to the handle's stream); with norms, ||U_a||^2 into dsmall[200 + 2a].
template <typename T>
int planes3_enqueue(Solver3D* S, int pi, bool norms, cudaStream_t st) {
    CK3(cudaEventRecord(S->evf[0], st));
    for (int q = 0; q < 2; ++q) CK3(cudaStreamWaitEvent(S->fork[q], S->evf[0], 0));
    for (int a = 0; a < 3; ++a) {
        cudaStream_t sa = a == 0 ? st : S->fork[a - 1];
        int nb = 0;
        double* part = S->partials + (size_t)a * 2 * 152 * 16;
        if (int rc = plane_solve3<T>(S, pi, a, part, &nb, sa)) return rc;
        if (norms) CK3(reduce_partials(part, nb, 2, S->dsmall + 200 + 2 * a, sa));
    }
    for (int q = 0; q < 2; ++q) {
        CK3(cudaEventRecord(S->evf[1 + q], S->fork[q]));
        CK3(cudaStreamWaitEvent(st, S->evf[1 + q], 0));
    }
    return ASDSM_OK;
}

// Launch shapes of the plane blocks' BCR levels, timed once per precision
// before the plane-solve graph is captured: per level and direction the
// fastest of TM in {16, 64} rows per CTA and KS in {1, 2, 4, 8} CTAs splitting
// the reduction, for the real (C = N_f) and the complex-pair (C = 2 N_f) blocks.
template <typename T>
int tune_planes3(Solver3D* S, int pi) {
    if (S->ptuned[pi]) return ASDSM_OK;
    auto& w = S->w[pi];
    const PlaneFam& pf = S->plane[0];
    cudaEvent_t e0, e1;
    CK3(cudaEventCreate(&e0));
    CK3(cudaEventCreate(&e1));
    int rc = ASDSM_OK;
    for (int bs = 1; bs <= 2 && rc == ASDSM_OK; ++bs) {
        BcrTune& tu = S->ptune[pi][bs - 1];
        tu = BcrTune{};
        tu.num_sms = S->num_sms;
        size_t b = 0;
        while (b < pf.bs.size() && pf.bs[b] != bs) ++b;
        if (b == pf.bs.size()) continue;                // no block of this size
        const Fac& f = pf.fac[pi][b];
        const BcrSys<T> sys = sys3<T>(f, w.Xb[0], w.Yb[0]);
        const int nk = (f.C + 31) / 32;
        for (int dir = 0; dir < 2 && rc == ASDSM_OK; ++dir)
            for (int l = 0; l < (dir ? f.L : f.L - 1); ++l) {
                float best = 1e30f;
                int bestv = 0;
                for (int tm : {16, 64})
                    for (int ks : {1, 2, 4, 8}) {
                        if (ks > (dir ? 2 : 1) * nk) continue;
                        tu.cfg[dir][l] = (tm << 8) | ks;
                        cudaError_t e = bcr_level<T>(&sys, 1, l, dir == 1, &tu, S->st);   // warm-up
                        if (e == cudaSuccess) e = cudaEventRecord(e0, S->st);
                        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = bcr_level<T>(&sys, 1, l, dir == 1, &tu, S->st);
                        if (e == cudaSuccess) e = cudaEventRecord(e1, S->st);
                        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                        float ms = 0.f;
                        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                        if (e != cudaSuccess) { rc = report_cuda_error(e); break; }
                        if (ms < best) { best = ms; bestv = tu.cfg[dir][l]; }
                    }
                tu.cfg[dir][l] = bestv;
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == ASDSM_OK) S->ptuned[pi] = true;
    return rc;
}

// The plane-family solves are the same launches every sweep (fixed buffers),
// so after one plain run they are captured once as a CUDA graph and replayed
// (not while profiling, whose event records would be captured too).
template <typename T>
int planes3(Solver3D* S, int pi, bool norms) {
    if (int rc = tune_planes3<T>(S, pi)) return rc;
    const PMark3 pm = prof3_begin(S);
    double flops = 0.0;
    for (int a = 0; a < 3; ++a)
        for (const Fac& f : S->plane[a].fac[pi]) flops += 2.0 * bcr_macs3(f.R, f.C, f.L);
    const double P = (double)S->g.plane, Nc = S->g.Nc;
    struct End { Solver3D* S; PMark3 pm; double b, f; ~End() { prof3_end(S, pm, P3_PLANES, b, f); } }
        end{S, pm, sizeof(T) * 3.0 * (2.0 * Nc * P), flops + 3.0 * 2.0 * 2.0 * Nc * Nc * P};
    auto& pg = S->pgraph[pi][norms ? 1 : 0];
    if (pg.exec && !S->prof) {
        CK3(cudaGraphLaunch(pg.exec, S->st));
        note_launch(pg.launches);
        return ASDSM_OK;
    }
    if (S->prof || pg.runs == 0) {
        ++pg.runs;
        return planes3_enqueue<T>(S, pi, norms, S->st);
    }
    // Captured on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); replayed on the caller's stream.
    const long long l0 = launch_count();
    cudaGraph_t graph = nullptr;
    CK3(cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal));
    const int rc = planes3_enqueue<T>(S, pi, norms, S->cap);
    const cudaError_t e = cudaStreamEndCapture(S->cap, &graph);
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return report_cuda_error(e);
    const cudaError_t e2 = cudaGraphInstantiate(&pg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) { pg.exec = nullptr; return report_cuda_error(e2); }
    pg.launches = launch_count() - l0;
    CK3(cudaGraphLaunch(pg.exec, S->st));
    return ASDSM_OK;
}

// Algorithm 3 over all cube holes (mode as hole_rhs3_kernel).
template <typename T>
int fill3(Solver3D* S, int pi, int mode, T* z, const double* s, double* u) {
    auto& w = S->w[pi];
    const Geo3& g = S->g;
    const long long nh = (long long)g.mc * g.mc * g.mc * g.hc * g.hc * g.hc;
    const PMark3 pm = prof3_begin(S);
    struct End { Solver3D* S; PMark3 pm; int cat; double b, f; ~End() { prof3_end(S, pm, cat, b, f); } }
        end{S, pm, mode == 2 ? P3_HOLEFIX : P3_FILL, (double)nh * sizeof(T) * 2.0,
            2.0 * (double)g.mc * g.mc * g.mc * bcr_macs3(S->hole[pi].R, S->hole[pi].C, S->hole[pi].L)};
    hole_rhs3_kernel<T><<<g1d(nh), T3, 0, S->st>>>(mode, z, s, u, g, S->sten, (T*)w.Xh);
    note_launch();
    CK3(cudaGetLastError());
    BcrSys<T> sys = sys3<T>(S->hole[pi], w.Xh, w.Yh, g.mc * g.mc * g.mc);
    CK3(bcr_solve<T>(&sys, 1, S->st));
    hole_scatter3_kernel<T><<<g1d(nh), T3, 0, S->st>>>(mode, (const T*)w.Yh, g, z, u);
    note_launch();
    CK3(cudaGetLastError());
    return ASDSM_OK;
}

// Algorithm 3 with zero source on all cube holes of the FP32 grid z: v = G f per
// hole, as one tcgen05 GEMM over all holes (fill3_tc.cu).
int fill_g3(Solver3D* S, float* z) {
    const Geo3& g = S->g;
    const int P = g.hc * g.hc * g.hc, K = 6 * g.hc * g.hc, H = g.mc * g.mc * g.mc;
    const PMark3 pm = prof3_begin(S);
    Fill3TcArgs a{};
    a.z = z; a.zout = z; a.gimg = S->g3img; a.aimg = S->a3img;
    a.N = g.N; a.mc = g.mc; a.n = g.n; a.hc = g.hc;
    a.P = P; a.K = K; a.H = H;
    a.KC = (K + 31) / 32; a.PT = (P + 127) / 128; a.HT = (H + 127) / 128;
    a.err = S->tc3err;
    CK3(fill3_tc(a, S->st));
    prof3_end(S, pm, P3_FILL, 4.0 * ((double)K * H * 2.0 + (double)P * H + (double)P * K), 2.0 * P * (double)K * H);
    return ASDSM_OK;
}

// The tensor-core Filler's timeout flag, read after the stream drained.
int tc3_status(Solver3D* S) {
    int f = 0;
    CK3(cudaMemcpyAsync(&f, S->tc3err, sizeof(int), cudaMemcpyDeviceToHost, S->st));
    CK3(cudaStreamSynchronize(S->st));
    if (f) {
        report_error("3D tensor-core Filler: a wait timed out");
        return ASDSM_ERR_CUDA;
    }
    return ASDSM_OK;
}

// Merge (R21-R23) into z: u_hat on the line points, then every plane moved onto it.
template <typename T>
int merge3(Solver3D* S, int pi, bool initial, int choice, T* z) {
    auto& w = S->w[pi];
    const Geo3& g = S->g;
    Merge3Args<T> m{};
    for (int a = 0; a < 3; ++a) {
        m.U[a] = (const T*)w.U[a];
        m.Lf[a] = initial ? (const T*)w.Yl[a] : nullptr;
    }
    m.Cc = initial ? (const T*)w.Yc : nullptr;
    m.nrm2 = initial ? nullptr : S->dsmall + 200;
    m.choice = choice;
    m.uh = (T*)w.uh;
    m.W = (const T*)S->W[pi];
    m.z = z;
    const long long lines = 3LL * (g.Nf - g.Nc) * g.Nc * g.Nc + (long long)g.Nc * g.Nc * g.Nc;
    const PMark3 pm = prof3_begin(S);
    struct End { Solver3D* S; PMark3 pm; double b, f; ~End() { prof3_end(S, pm, P3_MERGE, b, f); } }
        end{S, pm, sizeof(T) * (3.0 * g.Nc * g.plane + (double)g.skel + 2.0 * lines),
            2.0 * 3.0 * g.Nc * g.plane * 3.0 * g.Nc};
    uhat3_kernel<T><<<g1d(lines), T3, 0, S->st>>>(m, g);
    dim3 grid((g.Nf + MP - 1) / MP, (g.Nf + MQ - 1) / MQ, 3 * g.Nc);
    plane_corr_kernel<T><<<grid, MP * MQ, 0, S->st>>>(m, g);
    note_launch(2);
    CK3(cudaGetLastError());
    return ASDSM_OK;
}

// The ASDSM correction of a sweep into z: plane solves of the residual's
// restrictions (already in F), normalisation, random-choice merge, Filler
// with zero source.
template <typename T>
int correction3(Solver3D* S, int pi, int choice, T* z) {
    if (int rc = planes3<T>(S, pi, true)) return rc;
    if (int rc = merge3<T>(S, pi, false, choice, z)) return rc;
    if constexpr (sizeof(T) == 4) return fill_g3(S, z);
    else return fill3<T>(S, pi, 1, z, nullptr, nullptr);
}

// Algorithm 1 with b_cc in 3D: u's interior receives u^(0) (u's ring = g).
template <typename T>
int initial_guess3(Solver3D* S, int pi, const double* s, double* u) {
    auto& w = S->w[pi];
    const Geo3& g = S->g;
    cudaStream_t st = S->st;
    const long long PL = (long long)g.Nc * g.plane, LN = (long long)g.Nf * g.Nc * g.Nc,
                    C3 = (long long)g.Nc * g.Nc * g.Nc;
    for (int a = 0; a < 3; ++a) {
        rhs3_kernel<T><<<g1d(PL), T3, 0, st>>>(s, u, g, a, PL, S->lift, (T*)w.F[a]);
        rhs3_kernel<T><<<g1d(LN), T3, 0, st>>>(s, u, g, 3 + a, LN, S->lift, (T*)w.Xl[a]);
        note_launch(2);
    }
    rhs3_kernel<T><<<g1d(C3), T3, 0, st>>>(s, u, g, 6, C3, S->lift, (T*)w.Xc);
    note_launch();
    CK3(cudaGetLastError());
    if (int rc = planes3<T>(S, pi, false)) return rc;
    for (int a = 0; a < 3; ++a) {
        BcrSys<T> sys = sys3<T>(S->line[pi][a], w.Xl[a], w.Yl[a]);
        CK3(bcr_solve<T>(&sys, 1, st));
    }
    BcrSys<T> sc = sys3<T>(S->coarse[pi], w.Xc, w.Yc);
    CK3(bcr_solve<T>(&sc, 1, st));
    T* z = (T*)w.Z;
    ring3_kernel<T><<<g1d(g.NN), T3, 0, st>>>(u, g, z);
    note_launch();
    if (int rc = merge3<T>(S, pi, true, 0, z)) return rc;
    if (int rc = fill3<T>(S, pi, 0, z, s, nullptr)) return rc;
    interior3_kernel<T><<<grid_rows((long long)g.Nf * g.Nf), T3, 0, st>>>(z, g, u);
    ring3_kernel<T><<<g1d(g.NN), T3, 0, st>>>(nullptr, g, z);     // a direction slot again: all zero
    note_launch(2);
    CK3(cudaGetLastError());
    return ASDSM_OK;
}

}  // namespace

namespace {

constexpr int kPartials3 = 32768;
constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ull;

uint64_t splitmix64_3(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Family drawn by the random choice of Algorithm 2 at sweep k (R22).
int choice3(uint64_t seed, int k) { return (int)(splitmix64_3(seed + (uint64_t)(k + 1) * kGolden) % 3ull); }

// FP64 coefficients as float pairs (hi, lo = rounding of the remainder) on the device.
int upload_pairs(Solver3D* S, const double* v, int n) {
    static thread_local std::vector<float2> tmp;
    tmp.resize((size_t)n);
    for (int i = 0; i < n; ++i) {
        const float hi = (float)v[i];
        tmp[(size_t)i] = make_float2(hi, (float)(v[i] - (double)hi));
    }
    CK3(cudaMemcpyAsync(S->dcoef2, tmp.data(), (size_t)n * sizeof(float2), cudaMemcpyHostToDevice, S->st));
    return ASDSM_OK;
}

int read3(Solver3D* S, const double* dev, int count) {
    CK3(cudaMemcpyAsync(S->hsmall, dev, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost, S->st));
    CK3(cudaStreamSynchronize(S->st));
    return ASDSM_OK;
}

// FP64 residual of u: ||r||^2 and the hole part into dsmall[0..1]; r also onto
// the skeleton and the plane right-hand sides (when `gather`).
template <typename T>
int residual3(Solver3D* S, int pi, const double* s, const double* u, bool gather) {
    auto& w = S->w[pi];
    const Geo3& g = S->g;
    Resid3Out<T> o{};
    if (gather) {
        o.rskel = w.rs;
        for (int a = 0; a < 3; ++a) o.rp[a] = (T*)w.F[a];
    }
    o.partials = S->partials;
    const unsigned nb = grid_rows((long long)g.Nf * g.Nf);
    resid3_kernel<T><<<nb, T3, 0, S->st>>>(s, u, g, S->sten, o);
    note_launch();
    CK3(cudaGetLastError());
    CK3(reduce_partials(S->partials, (int)nb, 2, S->dsmall, S->st));
    return ASDSM_OK;
}

template <typename T>
int solve3(Solver3D* S, const double* s, double* u, asdsm_stats* stats) {
    const bool mixed = sizeof(T) == 4;
    const int pi = mixed ? 1 : 0;
    if (int rc = ensure_work3<T>(S, pi)) return rc;
    auto& w = S->w[pi];
    const Geo3& g = S->g;
    const asdsm_opts& op = S->opts;
    cudaStream_t st = S->st;
    const int m = w.m;
    const long long launches0 = launch_count();
    S->hist.clear();
    CK3(cudaEventRecord(S->ev0, st));
    // ||b_ff||: the residual of the grid with g on the ring and a zero interior.
    ring3_kernel<double><<<g1d(g.NN), T3, 0, st>>>(u, g, S->u_work);
    note_launch();
    if (int rc = residual3<T>(S, pi, s, S->u_work, false)) return rc;
    if (int rc = read3(S, S->dsmall, 1)) return rc;
    const double bnorm = std::sqrt(S->hsmall[0]);
    if (!std::isfinite(bnorm)) return ASDSM_ERR_NAN;
    if (!op.skip_initial_guess)
        if (int rc = initial_guess3<T>(S, pi, s, u)) return rc;
    CK3(cudaEventRecord(S->ev1, st));
    T* Z = (T*)w.Z;
    T* V = (T*)w.V;
    std::vector<double> Tm((size_t)m * m, 0.0), c(m, 0.0), c_app(m, 0.0), dc(m, 0.0), beta(m, 0.0), rq(m, 0.0);
    auto rel_of = [&](double r2) { return bnorm > 0 ? std::sqrt(std::max(r2, 0.0)) / bnorm : std::sqrt(std::max(r2, 0.0)); };
    int k = 0, kc = 0, status = ASDSM_NOT_CONVERGED, hole_fixes = 0;
    double rel = 0.0, rel0 = 0.0, hole_ref = 0.0, rh2 = 0.0;
    bool hole_ref_pending = false, need_true = true;
    bool last_tracked = false;           // the last history entry is a tracked value of the current iterate
    bool restart = true;                 // the next true residual starts a new cycle
    int since_check = 0;                 // sweeps since the last true residual
    for (;;) {
        if (need_true) {
            // Checkpoint: u receives the part of the cycle's update not applied yet,
            // then the true FP64 residual replaces the tracked one.
            const double nf3 = (double)g.Nf * g.Nf * g.Nf;
            if (kc > 0) {
                for (int i = 0; i < kc; ++i) { dc[i] = c[i] - c_app[i]; c_app[i] = c[i]; }
                const PMark3 pm = prof3_begin(S);
                if constexpr (sizeof(T) == 4) {
                    if (int rc = upload_pairs(S, dc.data(), kc)) return rc;
                    update_many_f32_kernel<<<grid_rows((long long)g.Nf * g.Nf), T3, 0, st>>>(u, Z, g.NN, kc, S->dcoef2, g);
                } else {
                    CK3(cudaMemcpyAsync(S->dcoef, dc.data(), (size_t)kc * sizeof(double), cudaMemcpyHostToDevice, st));
                    update_many_kernel<T><<<grid_rows((long long)g.Nf * g.Nf), T3, 0, st>>>(u, Z, g.NN, kc, S->dcoef, g);
                }
                note_launch();
                CK3(cudaGetLastError());
                prof3_end(S, pm, P3_UPDATE, nf3 * (16.0 + sizeof(T) * kc), 2.0 * kc * nf3);
                CK3(cudaStreamSynchronize(st));      // dcoef is rewritten before the next launch that reads it
            }
            {
                const PMark3 pm = prof3_begin(S);
                if (int rc = residual3<T>(S, pi, s, u, true)) return rc;
                if constexpr (sizeof(T) == 4) {
                    split_pairs_kernel<<<g1d(g.skel), T3, 0, st>>>(w.rs, g.skel, w.rsh, w.rsl);
                    note_launch();
                    CK3(cudaGetLastError());
                }
                prof3_end(S, pm, P3_RESID, nf3 * 16.0 + 8.0 * g.skel + sizeof(T) * 3.0 * g.Nc * g.plane, 14.0 * nf3);
            }
            if (int rc = read3(S, S->dsmall, 2)) return rc;
            const double rr = S->hsmall[0];
            rh2 = S->hsmall[1];
            rel = rel_of(rr);
            if (last_tracked) S->hist.back() = rel;      // replaces the tracked value of this iterate
            else S->hist.push_back(rel);
            last_tracked = false;
            if (restart) {
                kc = 0;
                std::fill(c.begin(), c.end(), 0.0);
                std::fill(c_app.begin(), c_app.end(), 0.0);
                restart = false;
            }
            since_check = 0;
            need_true = false;
            if (!std::isfinite(rel)) { status = ASDSM_ERR_NAN; break; }
            if (k == 0) rel0 = rel;
            if (rel <= op.tol) { status = ASDSM_OK; break; }
            if (k >= op.max_sweeps) { status = ASDSM_NOT_CONVERGED; break; }
            const int win = op.stagnation_window;
            if (win > 0 && (int)S->hist.size() > win &&
                S->hist.back() > (1.0 - op.stagnation_factor) * S->hist[S->hist.size() - 1 - win]) {
                status = ASDSM_STAGNATED;
                break;
            }
            const double hnorm = std::sqrt(rh2), rnorm = std::sqrt(rr);
            if (hole_ref_pending) { hole_ref = hnorm; hole_ref_pending = false; }
            // R18: a Filler pass on the hole part of the residual replaces the sweep.
            if (hnorm > op.hole_fix_ratio * rnorm && hnorm > op.hole_fix_growth * hole_ref) {
                if (int rc = fill3<T>(S, pi, 2, (T*)nullptr, s, u)) return rc;
                hole_ref_pending = true;
                ++hole_fixes;
                ++k;
                need_true = true;
                restart = true;                      // u moved outside the cycle's directions
                continue;
            }
        }
        // The correction: Algorithm 1 without b_cc on the (tracked) residual.
        T* z = Z + (long long)kc * g.NN;
        if (int rc = correction3<T>(S, pi, choice3(op.seed, k), z)) return rc;
        ++k;
        // Least squares on the skeleton rows: A e there and its products with the
        // tracked residual and the cycle's orthonormal images.
        const PMark3 pm_gcr = prof3_begin(S);
        const double gcr_bytes = (double)g.skel * (sizeof(T) * (3.0 + 2.0 * kc) + 16.0);
        const double gcr_flops = (double)g.skel * (14.0 + 6.0 * kc + 6.0);
        skel_apply3_kernel<T><<<grid_rows((long long)g.Nf * g.Nf), T3, 0, st>>>(z, g, S->sten, (T*)w.q);
        const dim3 dgrid(DK_CHUNKS, std::max(1, (kc + DK_VEC - 1) / DK_VEC));
        if constexpr (sizeof(T) == 4)
            dots_many_f32_kernel<<<dgrid, T3, 0, st>>>((const float*)w.q, w.rsh, w.rsl, V, g.skel, g.skel, kc,
                                                       S->dpart);
        else
            dots_many_kernel<T><<<dgrid, T3, 0, st>>>((const T*)w.q, w.rs, V, g.skel, g.skel, kc, S->dpart);
        const int ncol = 3 + 2 * kc;
        sum_chunks_kernel<<<(ncol + 31) / 32, 32, 0, st>>>(S->dpart, ncol, S->dsum);
        note_launch(3);
        CK3(cudaGetLastError());
        if (int rc = read3(S, S->dsum, ncol)) return rc;
        prof3_end(S, pm_gcr, P3_GCR, gcr_bytes, gcr_flops);
        const double qq = S->hsmall[0], qr = S->hsmall[1], rr = S->hsmall[2];
        if (m == 1) {
            // The paper's clamped optimal scaling: s_hat = argmin_{s >= 0} ||r - s A e||.
            const double shat = qq > 0 ? std::max(0.0, qr / qq) : 0.0;
            c[0] = shat;
            kc = 1;
            S->hist.push_back(rel_of(rr - 2 * shat * qr + shat * shat * qq + rh2));
            last_tracked = true;
            need_true = true;
            restart = true;
            continue;
        }
        // GCR (R15): orthogonalise A e against the cycle's earlier images.
        double nu2 = qq;
        for (int j = 0; j < kc; ++j) {
            beta[j] = S->hsmall[3 + j];
            rq[j] = S->hsmall[3 + kc + j];
            nu2 -= beta[j] * beta[j];
        }
        if (!(nu2 > 1e-24 * qq) || !(qq > 0)) {      // a dependent direction ends the cycle
            S->hist.push_back(S->hist.back());
            last_tracked = true;
            need_true = true;
            restart = true;
            continue;
        }
        const double nu = std::sqrt(nu2);
        double alpha_ = qr;
        for (int j = 0; j < kc; ++j) alpha_ -= beta[j] * rq[j];
        alpha_ /= nu;
        // Column kc of T: V_kc = sum_i T[i][kc] Z_i; the cycle's update is sum_i c_i Z_i.
        for (int i = 0; i <= kc; ++i) Tm[(size_t)i * m + kc] = 0.0;
        Tm[(size_t)kc * m + kc] = 1.0 / nu;
        for (int j = 0; j < kc; ++j)
            for (int i = 0; i <= j; ++i) Tm[(size_t)i * m + kc] -= beta[j] * Tm[(size_t)i * m + j] / nu;
        for (int i = 0; i <= kc; ++i) c[i] += alpha_ * Tm[(size_t)i * m + kc];
        {
            const PMark3 pm = prof3_begin(S);
            if constexpr (sizeof(T) == 4) {
                if (kc > 0)
                    if (int rc = upload_pairs(S, beta.data(), kc)) return rc;
                const float ah = (float)alpha_, al = (float)(alpha_ - (double)ah);
                combine_many_f32_kernel<<<g1d(g.skel), T3, 0, st>>>((const float*)w.q, V, g.skel, g.skel, kc, S->dcoef2,
                                                                   (float)(1.0 / nu), ah, al, w.rsh, w.rsl);
            } else {
                if (kc > 0)
                    CK3(cudaMemcpyAsync(S->dcoef, beta.data(), (size_t)kc * sizeof(double), cudaMemcpyHostToDevice, st));
                combine_many_kernel<T><<<g1d(g.skel), T3, 0, st>>>((const T*)w.q, V, g.skel, g.skel, kc, S->dcoef,
                                                                 1.0 / nu, alpha_, w.rs, S->partials);
            }
            note_launch();
            CK3(cudaGetLastError());
            prof3_end(S, pm, P3_GCR, (double)g.skel * (sizeof(T) * (2.0 + kc) + 16.0), (double)g.skel * 2.0 * (kc + 2));
        }
        ++kc;
        // ||r - alpha V_kc||^2 = ||r||^2 - alpha^2 for the orthonormal V_kc with alpha = <r, V_kc>.
        const double rel_t = rel_of(rr - alpha_ * alpha_ + rh2);
        S->hist.push_back(rel_t);
        last_tracked = true;
        ++since_check;
        if (kc >= m) restart = true;
        if (rel_t <= op.tol || kc >= m || k >= op.max_sweeps || since_check >= kCheck3) { need_true = true; continue; }
        const int win = op.stagnation_window;
        if (win > 0 && (int)S->hist.size() > win &&
            S->hist.back() > (1.0 - op.stagnation_factor) * S->hist[S->hist.size() - 1 - win]) {
            need_true = true;
            continue;
        }
        const PMark3 pm_pl = prof3_begin(S);
        // The FP32 path tracks the residual as float pairs between true residuals.
        planes_from_skel_kernel<T><<<grid_rows((long long)g.Nf * g.Nf), T3, 0, st>>>(
            w.rs, sizeof(T) == 4 ? w.rsh : nullptr, sizeof(T) == 4 ? w.rsl : nullptr, g, (T*)w.F[0], (T*)w.F[1],
            (T*)w.F[2]);
        note_launch();
        CK3(cudaGetLastError());
        prof3_end(S, pm_pl, P3_GCR, 8.0 * g.skel + sizeof(T) * 3.0 * g.Nc * g.plane, 0.0);
    }
    // The largest hole residual of the returned iterate.
    const long long nh = (long long)g.mc * g.mc * g.mc * g.hc * g.hc * g.hc;
    const unsigned nbh = g1d(nh);
    hole_max3_kernel<<<nbh, T3, 0, st>>>(s, u, g, S->sten, S->partials);
    note_launch();
    CK3(cudaGetLastError());
    CK3(cudaMemcpyAsync(S->hsmall + 8, S->partials, nbh * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK3(cudaEventRecord(S->ev2, st));
    CK3(cudaEventSynchronize(S->ev2));
    double hmax = 0.0;
    for (unsigned b = 0; b < nbh; ++b) hmax = std::max(hmax, S->hsmall[8 + b]);
    float ms_setup = 0.f, ms_all = 0.f;
    cudaEventElapsedTime(&ms_setup, S->ev0, S->ev1);
    cudaEventElapsedTime(&ms_all, S->ev0, S->ev2);
    prof3_resolve(S);
    if (stats) {
        asdsm_stats stt{};
        stt.sweeps = k;
        stt.status = status;
        stt.hole_fixes = hole_fixes;
        stt.rel_res = rel;
        stt.rel_res0 = rel0;
        stt.setup_ms = ms_setup;
        stt.solve_ms = ms_all;
        stt.launches = launch_count() - launches0;
        stt.rel_res_fp64 = rel;            // the sweep residual is FP64 in 3D
        stt.hole_res_max = hmax;
        *stats = stt;
    }
    return status;
}

}  // namespace

// ---------------------------------------------------------------------------
// Interface to the C ABI
// ---------------------------------------------------------------------------
int s3_create(const asdsm_desc* d, const asdsm_opts* o, cudaStream_t st, Solver3D** out) {
    *out = nullptr;
    const int N = d->n, mc = d->mc;
    auto pow2 = [](long long v) { return v > 0 && (v & (v - 1)) == 0; };
    if (N < 5 || N > 257 || !pow2(N - 1) || !pow2(mc) || mc < 2 || mc > 32 || (N - 1) % mc != 0) {
        report_error("3D sizes: N - 1 and mc powers of two, N <= 257, 2 <= mc <= 32");
        return ASDSM_ERR_INVALID;
    }
    const int n = (N - 1) / mc;
    if (n < 2 || n > 16) { report_error("3D sizes: hole size (N-1)/mc must be 2..16"); return ASDSM_ERR_INVALID; }
    if (o->accel_m < 1 || o->accel_m > kMaxM3 || (o->precision != ASDSM_FP64 && o->precision != ASDSM_MIXED)) {
        report_error("3D options: accel_m in 1..1024, precision ASDSM_FP64 or ASDSM_MIXED");
        return ASDSM_ERR_INVALID;
    }
    for (int a = 0; a < 3; ++a)
        if (!(d->alpha[a] > 0.0) || !std::isfinite(d->alpha[a]) || !std::isfinite(d->beta[a])) {
            report_error("3D: alpha_i must be positive and finite");
            return ASDSM_ERR_INVALID;
        }
    Solver3D* S = new Solver3D();
    S->desc = *d;
    S->opts = *o;
    S->st = st;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, dev);
    Geo3& g = S->g;
    g.N = N; g.M = N - 1; g.Nf = N - 2; g.mc = mc; g.Nc = mc - 1; g.n = n; g.hc = n - 1;
    g.NN = (long long)N * N * N;
    g.plane = (long long)g.Nf * g.Nf;
    const long long nf = g.Nf, nhole = g.Nf - g.Nc;
    g.skel = nf * nf * nf - nhole * nhole * nhole;
    const double h = 1.0 / g.M, H = 1.0 / mc;
    const double* al = d->alpha;
    const double* be = d->beta;
    S->sten.cc = 2 * (al[0] + al[1] + al[2]) / (h * h);
    S->sten.cw = -al[0] / (h * h) - be[0] / (2 * h); S->sten.ce = -al[0] / (h * h) + be[0] / (2 * h);
    S->sten.cs = -al[1] / (h * h) - be[1] / (2 * h); S->sten.cn = -al[1] / (h * h) + be[1] / (2 * h);
    S->sten.cd = -al[2] / (h * h) - be[2] / (2 * h); S->sten.cu = -al[2] / (h * h) + be[2] / (2 * h);
    for (int a = 0; a < 3; ++a)
        for (int q = 0; q < 2; ++q) {
            const double sp = q ? H : h;
            S->lift.lo[a][q] = al[a] / (sp * sp) + be[a] / (2 * sp);
            S->lift.hi[a][q] = al[a] / (sp * sp) - be[a] / (2 * sp);
        }
    auto fail = [&](int rc) { s3_destroy(S); return rc; };
    if (int rc = build_factors(S)) return fail(rc);
    cudaError_t e;
    if ((e = cudaMalloc(&S->u_work, (size_t)g.NN * sizeof(double))) != cudaSuccess) return fail(report_cuda_error(e));
    if ((e = cudaMalloc(&S->partials, (size_t)kPartials3 * sizeof(double))) != cudaSuccess) return fail(report_cuda_error(e));
    if ((e = cudaMalloc(&S->dsmall, 256 * sizeof(double))) != cudaSuccess) return fail(report_cuda_error(e));
    if ((e = cudaMallocHost(&S->hsmall, 4096 * sizeof(double))) != cudaSuccess) return fail(report_cuda_error(e));
    if ((e = cudaMalloc(&S->dcoef, kMaxM3 * sizeof(double))) != cudaSuccess) return fail(report_cuda_error(e));
    if ((e = cudaMalloc(&S->dcoef2, kMaxM3 * sizeof(float2))) != cudaSuccess) return fail(report_cuda_error(e));
    if ((e = cudaMalloc(&S->dsum, (2 * kMaxM3 + 3) * sizeof(double))) != cudaSuccess) return fail(report_cuda_error(e));
    if ((e = cudaMalloc(&S->dpart, (size_t)(2 * kMaxM3 + 3) * DK_CHUNKS * sizeof(double))) != cudaSuccess)
        return fail(report_cuda_error(e));
    for (cudaEvent_t* ev : {&S->ev0, &S->ev1, &S->ev2})
        if ((e = cudaEventCreate(ev)) != cudaSuccess) return fail(report_cuda_error(e));
    for (cudaEvent_t* ev : {&S->evf[0], &S->evf[1], &S->evf[2]})
        if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return fail(report_cuda_error(e));
    for (cudaStream_t* fs : {&S->fork[0], &S->fork[1], &S->cap})
        if ((e = cudaStreamCreateWithFlags(fs, cudaStreamNonBlocking)) != cudaSuccess) return fail(report_cuda_error(e));
    *out = S;
    return ASDSM_OK;
}

int s3_set_opts(Solver3D* S, const asdsm_opts* o) {
    if (o->accel_m < 1 || o->accel_m > kMaxM3) return ASDSM_ERR_INVALID;
    const int m_old = S->opts.accel_m;
    S->opts = *o;
    if (o->accel_m != m_old) { free_work3(S, 0); free_work3(S, 1); }     // direction slots re-allocated on first use
    return ASDSM_OK;
}

int s3_solve(Solver3D* S, const double* s, double* u, asdsm_stats* stats) {
    const int rc = S->opts.precision == ASDSM_FP64 ? solve3<double>(S, s, u, stats) : solve3<float>(S, s, u, stats);
    if (int tc = tc3_status(S)) return tc;
    return rc;
}

int s3_initial_guess(Solver3D* S, const double* s, double* u) {
    const bool fp64 = S->opts.precision == ASDSM_FP64;
    int rc = fp64 ? ensure_work3<double>(S, 0) : ensure_work3<float>(S, 1);
    if (rc) return rc;
    rc = fp64 ? initial_guess3<double>(S, 0, s, u) : initial_guess3<float>(S, 1, s, u);
    if (rc) return rc;
    CK3(cudaStreamSynchronize(S->st));
    return ASDSM_OK;
}

int s3_residual(Solver3D* S, const double* s, const double* u, double* r, double* rel) {
    (void)r;
    if (int rc = ensure_work3<double>(S, 0)) return rc;
    ring3_kernel<double><<<g1d(S->g.NN), T3, 0, S->st>>>(u, S->g, S->u_work);
    note_launch();
    if (int rc = residual3<double>(S, 0, s, S->u_work, false)) return rc;
    if (int rc = read3(S, S->dsmall, 1)) return rc;
    const double b2 = S->hsmall[0];
    if (int rc = residual3<double>(S, 0, s, u, false)) return rc;
    if (int rc = read3(S, S->dsmall, 1)) return rc;
    if (rel) *rel = b2 > 0 ? std::sqrt(S->hsmall[0] / b2) : std::sqrt(S->hsmall[0]);
    return ASDSM_OK;
}

namespace {
template <typename T>
int submesh3(Solver3D* S, int pi, int mesh, const double* in, double* out) {
    if (int rc = ensure_work3<T>(S, pi)) return rc;
    auto& w = S->w[pi];
    const Geo3& g = S->g;
    cudaStream_t st = S->st;
    auto conv_in = [&](void* dst, long long n) {
        convert3_kernel<double, T><<<g1d(n), T3, 0, st>>>(in, n, (T*)dst);
        note_launch();
    };
    auto conv_out = [&](const void* src, long long n) {
        convert3_kernel<T, double><<<g1d(n), T3, 0, st>>>((const T*)src, n, out);
        note_launch();
    };
    if (mesh < 3) {
        const long long n = (long long)g.Nc * g.plane;
        conv_in(w.F[mesh], n);
        int nb = 0;
        if (int rc = plane_solve3<T>(S, pi, mesh, S->partials, &nb, st)) return rc;
        conv_out(w.U[mesh], n);
    } else if (mesh < 6) {
        const int a = mesh - 3;
        const long long n = (long long)g.Nf * g.Nc * g.Nc;
        conv_in(w.Xl[a], n);
        BcrSys<T> sys = sys3<T>(S->line[pi][a], w.Xl[a], w.Yl[a]);
        CK3(bcr_solve<T>(&sys, 1, st));
        conv_out(w.Yl[a], n);
    } else if (mesh == 6) {
        const long long n = (long long)g.Nc * g.Nc * g.Nc;
        conv_in(w.Xc, n);
        BcrSys<T> sys = sys3<T>(S->coarse[pi], w.Xc, w.Yc);
        CK3(bcr_solve<T>(&sys, 1, st));
        conv_out(w.Yc, n);
    } else if (mesh == 7) {
        if (int rc = fill3<T>(S, pi, 3, (T*)nullptr, in, out)) return rc;
    } else {
        // Algorithm 3 with zero source: in's skeleton values as Dirichlet data, out's hole points receive the fill.
        T* z = (T*)w.uh;
        conv_in(z, g.NN);
        if constexpr (sizeof(T) == 4) {
            if (int rc = fill_g3(S, z)) return rc;
        } else {
            if (int rc = fill3<T>(S, pi, 1, z, nullptr, nullptr)) return rc;
        }
        hole_copy3_kernel<T><<<g1d((long long)g.mc * g.mc * g.mc * g.hc * g.hc * g.hc), T3, 0, st>>>(z, g, out);
        note_launch();
    }
    CK3(cudaGetLastError());
    CK3(cudaStreamSynchronize(st));
    return ASDSM_OK;
}
}  // namespace

int s3_submesh_solve(Solver3D* S, int mesh, const double* in, double* out) {
    if (mesh < 0 || mesh > 8) return ASDSM_ERR_INVALID;
    const int rc = S->opts.precision == ASDSM_FP64 ? submesh3<double>(S, 0, mesh, in, out)
                                                   : submesh3<float>(S, 1, mesh, in, out);
    if (int tc = tc3_status(S)) return tc;
    return rc;
}

int s3_profile(Solver3D* S, int enable) {
    S->prof = enable != 0;
    std::memset(S->pc, 0, sizeof(S->pc));
    for (int c = 0; c < P3_COUNT; ++c) std::strncpy(S->pc[c].name, kProf3Names[c], sizeof(S->pc[c].name) - 1);
    S->marks.clear();
    S->evnext = 0;
    return ASDSM_OK;
}

int s3_profile_read(Solver3D* S, asdsm_kprof* out, int cap) {
    const int n = std::min<int>(cap, P3_COUNT);
    for (int c = 0; c < n; ++c) out[c] = S->pc[c];
    return n;
}

int s3_history(Solver3D* S, double* hist, int cap) {
    const int n = std::min<int>(cap, (int)S->hist.size());
    for (int i = 0; i < n; ++i) hist[i] = S->hist[i];
    return n;
}

void s3_destroy(Solver3D* S) {
    if (!S) return;
    if (S->st) cudaStreamSynchronize(S->st);
    for (int pi = 0; pi < 2; ++pi) {
        free_work3(S, pi);
        for (int a = 0; a < 3; ++a) {
            for (Fac& f : S->plane[a].fac[pi]) free_fac(f);
            free_fac(S->line[pi][a]);
            if (S->plane[a].Qd[pi]) cudaFree(S->plane[a].Qd[pi]);
        }
        free_fac(S->coarse[pi]);
        free_fac(S->hole[pi]);
        if (S->W[pi]) cudaFree(S->W[pi]);
    }
    if (S->u_work) cudaFree(S->u_work);
    if (S->partials) cudaFree(S->partials);
    if (S->dsmall) cudaFree(S->dsmall);
    if (S->hsmall) cudaFreeHost(S->hsmall);
    for (double* p : {S->dcoef, S->dsum, S->dpart})
        if (p) cudaFree(p);
    if (S->dcoef2) cudaFree(S->dcoef2);
    for (auto& row : S->pgraph)
        for (auto& pg : row)
            if (pg.exec) cudaGraphExecDestroy(pg.exec);
    for (cudaEvent_t e : S->evf)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t fs : {S->fork[0], S->fork[1], S->cap})
        if (fs) cudaStreamDestroy(fs);
    if (S->g3img) cudaFree(S->g3img);
    if (S->a3img) cudaFree(S->a3img);
    if (S->tc3err) cudaFree(S->tc3err);
    for (cudaEvent_t e : S->evpool) cudaEventDestroy(e);
    for (cudaEvent_t ev : {S->ev0, S->ev1, S->ev2})
        if (ev) cudaEventDestroy(ev);
    delete S;
}

}  // namespace asdsm
