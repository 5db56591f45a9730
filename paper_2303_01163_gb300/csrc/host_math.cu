// Host-side FP64 precomputation for the ASDSM library.
//
// * Block cyclic reduction (BCR) factors of the separable constant-coefficient
//   operators of eq. (2.4): every submesh system of Section 2.3 (A_fc, A_cf,
//   A_cc) and every hole block A_(ij) of Remark 2.4 is
//       (T_row (x) I + I (x) T_col) x = f
//   with T_row, T_col tridiagonal Toeplitz.  Ordered row by row it is block
//   tridiagonal with blocks a I, (d I + T_col), c I.  With R = 2^L - 1 rows,
//   cyclic reduction keeps the Toeplitz structure at every level, so one set
//   of C x C factors per level serves every row (and every hole).
// * The tail of that reduction as one dense map (the last levels, where only
//   a few rows are left, as a single matrix-vector product on the device).
// * The moment operator of the not-a-knot cubic spline used by "Spline" in
//   Algorithm 2 (knot values zero at both ends).
#include "asdsm_internal.h"
#include <cmath>
#include <algorithm>
#include <thread>

namespace asdsm {

namespace {

// C = A B, all n x n row-major.
void matmul(const double* A, const double* B, double* C, int n) {
    std::fill(C, C + (size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        const double* a = A + (size_t)i * n;
        double* c = C + (size_t)i * n;
        for (int k = 0; k < n; ++k) {
            const double aik = a[k];
            if (aik == 0.0) continue;
            const double* b = B + (size_t)k * n;
            for (int j = 0; j < n; ++j) c[j] += aik * b[j];
        }
    }
}

// In-place inverse of an n x n row-major matrix by Gauss-Jordan elimination
// with partial pivoting.  Returns false when a pivot vanishes.
bool invert(std::vector<double>& A, int n) {
    std::vector<double> I((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double best = std::fabs(A[(size_t)col * n + col]);
        for (int r = col + 1; r < n; ++r) {
            double v = std::fabs(A[(size_t)r * n + col]);
            if (v > best) { best = v; piv = r; }
        }
        if (!(best > 0.0) || !std::isfinite(best)) return false;
        if (piv != col) {
            for (int j = 0; j < n; ++j) {
                std::swap(A[(size_t)col * n + j], A[(size_t)piv * n + j]);
                std::swap(I[(size_t)col * n + j], I[(size_t)piv * n + j]);
            }
        }
        const double inv = 1.0 / A[(size_t)col * n + col];
        for (int j = 0; j < n; ++j) {
            A[(size_t)col * n + j] *= inv;
            I[(size_t)col * n + j] *= inv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = A[(size_t)r * n + col];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                A[(size_t)r * n + j] -= f * A[(size_t)col * n + j];
                I[(size_t)r * n + j] -= f * I[(size_t)col * n + j];
            }
        }
    }
    A.swap(I);
    return true;
}

void transpose_into(const double* M, double* out, int n) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) out[(size_t)j * n + i] = M[(size_t)i * n + j];
}

}  // namespace

bool hole_extension_operator(int C, const Stencil& s, std::vector<double>* G) {
    const int n = C * C, K = 4 * C;
    auto id = [C](int y, int x) { return (y - 1) * C + (x - 1); };
    std::vector<double> A((size_t)n * n, 0.0);
    for (int y = 1; y <= C; ++y)
        for (int x = 1; x <= C; ++x) {
            const size_t r = (size_t)id(y, x) * n;
            A[r + id(y, x)] = s.cc;
            if (x > 1) A[r + id(y, x - 1)] = s.cw;
            if (x < C) A[r + id(y, x + 1)] = s.ce;
            if (y > 1) A[r + id(y - 1, x)] = s.cs;
            if (y < C) A[r + id(y + 1, x)] = s.cn;
        }
    if (!invert(A, n)) return false;
    // Ring value k enters the equation of one hole point q with coefficient c:
    // column k of G is -c times column q of A_hh^{-1}.
    G->assign((size_t)n * K, 0.0);
    for (int i = 1; i <= C; ++i) {
        const int ks[4] = {i - 1, C + i - 1, 2 * C + i - 1, 3 * C + i - 1};
        const int qs[4] = {id(i, 1), id(i, C), id(1, i), id(C, i)};
        const double cf[4] = {s.cw, s.ce, s.cs, s.cn};
        for (int t = 0; t < 4; ++t)
            for (int p = 0; p < n; ++p) (*G)[(size_t)p * K + ks[t]] = -cf[t] * A[(size_t)p * n + qs[t]];
    }
    return true;
}

namespace {

// Gaussian elimination with partial pivoting of an n x n band matrix with kl
// sub- and ku super-diagonals, stored by rows with room for the fill-in of the
// row exchanges (ku + kl super-diagonals): row i holds columns i-kl .. i+ku+kl
// at offsets 0 .. 2 kl + ku.  Multipliers overwrite the eliminated entries.
struct BandLU {
    int n = 0, kl = 0, ku2 = 0, W = 0;
    std::vector<double> a;
    std::vector<int> piv;
    double& at(int i, int j) { return a[(size_t)i * W + (j - i + kl)]; }
    bool factor() {
        piv.assign(n, 0);
        for (int k = 0; k < n; ++k) {
            int p = k;
            double best = std::fabs(at(k, k));
            const int last = std::min(n - 1, k + kl);
            for (int i = k + 1; i <= last; ++i)
                if (std::fabs(at(i, k)) > best) { best = std::fabs(at(i, k)); p = i; }
            if (!(best > 0.0) || !std::isfinite(best)) return false;
            piv[k] = p;
            const int jend = std::min(n - 1, k + ku2);
            if (p != k)
                for (int j = k; j <= jend; ++j) std::swap(at(k, j), at(p, j));
            const double inv = 1.0 / at(k, k);
            for (int i = k + 1; i <= last; ++i) {
                const double l = at(i, k) * inv;
                at(i, k) = l;
                if (l == 0.0) continue;
                for (int j = k + 1; j <= jend; ++j) at(i, j) -= l * at(k, j);
            }
        }
        return true;
    }
    void solve(double* b) {
        for (int k = 0; k < n; ++k) {                      // L (unit) with the row exchanges
            if (piv[k] != k) std::swap(b[k], b[piv[k]]);
            const int last = std::min(n - 1, k + kl);
            for (int i = k + 1; i <= last; ++i) b[i] -= at(i, k) * b[k];
        }
        for (int k = n - 1; k >= 0; --k) {                 // U
            const int jend = std::min(n - 1, k + ku2);
            double v = b[k];
            for (int j = k + 1; j <= jend; ++j) v -= at(k, j) * b[j];
            b[k] = v / at(k, k);
        }
    }
};

}  // namespace

bool hole_extension_operator_3d(int C, const double sten7[7], std::vector<double>* G) {
    if (C < 1) return false;
    const int n = C * C * C, F = C * C, K = 6 * F;
    auto id = [C](int x, int y, int z) { return (z * C + y) * C + x; };   // 0-based hole coordinates
    BandLU lu;
    lu.n = n;
    lu.kl = F;
    lu.ku2 = 2 * F;
    lu.W = lu.kl + lu.ku2 + 1;
    lu.a.assign((size_t)n * lu.W, 0.0);
    for (int z = 0; z < C; ++z)
        for (int y = 0; y < C; ++y)
            for (int x = 0; x < C; ++x) {
                const int r = id(x, y, z);
                lu.at(r, r) = sten7[0];
                if (x > 0) lu.at(r, id(x - 1, y, z)) = sten7[1];
                if (x < C - 1) lu.at(r, id(x + 1, y, z)) = sten7[2];
                if (y > 0) lu.at(r, id(x, y - 1, z)) = sten7[3];
                if (y < C - 1) lu.at(r, id(x, y + 1, z)) = sten7[4];
                if (z > 0) lu.at(r, id(x, y, z - 1)) = sten7[5];
                if (z < C - 1) lu.at(r, id(x, y, z + 1)) = sten7[6];
            }
    if (!lu.factor()) return false;
    G->assign((size_t)n * K, 0.0);
    // Face value k touches one hole point q with coefficient c: column k of G is
    // -c times column q of A_hh^{-1}.  Columns are solved once per distinct q.
    std::vector<double> col(n);
    std::vector<int> done(n, 0);
    std::vector<std::vector<std::pair<int, double>>> users(n);
    for (int v = 0; v < C; ++v)
        for (int u = 0; u < C; ++u) {
            const int f = v * C + u;
            users[id(0, u, v)].push_back({0 * F + f, sten7[1]});       // west: (y, z) = (u, v)
            users[id(C - 1, u, v)].push_back({1 * F + f, sten7[2]});   // east
            users[id(u, 0, v)].push_back({2 * F + f, sten7[3]});       // south: (x, z)
            users[id(u, C - 1, v)].push_back({3 * F + f, sten7[4]});   // north
            users[id(u, v, 0)].push_back({4 * F + f, sten7[5]});       // down: (x, y)
            users[id(u, v, C - 1)].push_back({5 * F + f, sten7[6]});   // up
        }
    for (int q = 0; q < n; ++q) {
        if (users[q].empty()) continue;
        std::fill(col.begin(), col.end(), 0.0);
        col[q] = 1.0;
        lu.solve(col.data());
        for (const auto& kc : users[q])
            for (int p = 0; p < n; ++p) (*G)[(size_t)p * K + kc.first] = -kc.second * col[p];
    }
    return true;
}

bool make_bcr(int R, double a, double d, double c, int C, double tl, double td, double tu, BcrFactors* out) {
    int L = 0;
    while (((1 << L) - 1) < R) ++L;
    if (((1 << L) - 1) != R || C < 1 || L > 16) return false;
    const size_t n2 = (size_t)C * C;
    out->R = R; out->C = C; out->L = L;
    out->Mt.assign((size_t)L * n2, 0.0);
    out->Bt.assign((size_t)L * n2, 0.0);
    out->wl.assign(L, 0.0);
    out->wr.assign(L, 0.0);
    // Which neighbour's factor is the larger one: |Q_l| / |P_l| = |c/a|^(2^l).
    const bool left_dominant = std::fabs(a) >= std::fabs(c);
    const double ratio = left_dominant ? c / a : a / c;     // modulus <= 1
    // Level 0: A_0 = a I, C_0 = c I, B_0 = d I + T.
    std::vector<double> A(n2, 0.0), Cm(n2, 0.0), B(n2, 0.0);
    for (int k = 0; k < C; ++k) {
        A[(size_t)k * C + k] = a;
        Cm[(size_t)k * C + k] = c;
        B[(size_t)k * C + k] = d + td;
        if (k > 0) B[(size_t)k * C + k - 1] = tl;
        if (k + 1 < C) B[(size_t)k * C + k + 1] = tu;
    }
    std::vector<double> Binv, P(n2), Q(n2), t1(n2), t2(n2);
    double w = ratio;                                        // ratio^(2^l)
    for (int l = 0; l < L; ++l) {
        Binv = B;
        if (!invert(Binv, C)) return false;
        matmul(A.data(), Binv.data(), P.data(), C);          // P_l = A_l B_l^{-1}
        matmul(Cm.data(), Binv.data(), Q.data(), C);         // Q_l = C_l B_l^{-1}
        transpose_into(left_dominant ? P.data() : Q.data(), out->Mt.data() + (size_t)l * n2, C);
        transpose_into(Binv.data(), out->Bt.data() + (size_t)l * n2, C);
        out->wl[l] = left_dominant ? 1.0 : w;
        out->wr[l] = left_dominant ? w : 1.0;
        w = w * w;
        if (l + 1 == L) break;
        // B_{l+1} = B_l - P_l C_l - Q_l A_l ; A_{l+1} = -P_l A_l ; C_{l+1} = -Q_l C_l
        matmul(P.data(), Cm.data(), t1.data(), C);
        matmul(Q.data(), A.data(), t2.data(), C);
        for (size_t e = 0; e < n2; ++e) B[e] = B[e] - t1[e] - t2[e];
        matmul(P.data(), A.data(), t1.data(), C);
        matmul(Q.data(), Cm.data(), t2.data(), C);
        for (size_t e = 0; e < n2; ++e) { A[e] = -t1[e]; Cm[e] = -t2[e]; }
    }
    for (double v : out->Mt) if (!std::isfinite(v)) return false;
    for (double v : out->Bt) if (!std::isfinite(v)) return false;
    return true;
}

bool bcr_tail_map(const BcrFactors& f, int rt, std::vector<double>* D) {
    int lt = 0;
    while ((1 << lt) - 1 < rt) ++lt;
    if (rt < 1 || (1 << lt) - 1 != rt || lt > f.L) return false;
    const int C = f.C, L = f.L, l0 = L - lt, n = rt * C;
    const size_t n2 = (size_t)C * C;
    D->assign((size_t)n * n, 0.0);
    // The map is linear and its columns are independent: apply the tail levels
    // to the unit vectors, a contiguous range of columns per thread.
    auto work = [&](int col0, int col1) {
        const int w = col1 - col0;
        if (w <= 0) return;
        const size_t rowsz = (size_t)C * w;             // one tail row: [C][w]
        std::vector<double> X((size_t)(rt + 2) * rowsz, 0.0), Y(X.size(), 0.0), v(rowsz);
        auto row = [&](std::vector<double>& A, int k) { return A.data() + (size_t)k * rowsz; };
        for (int col = col0; col < col1; ++col) row(X, col / C + 1)[(size_t)(col % C) * w + (col - col0)] = 1.0;
        // out[c][j] += sum_k in[k][j] F[k][c]  (F: a transposed factor, [k][c] = M[c][k])
        auto apply = [&](const double* F, const double* in, double* out) {
            for (int k = 0; k < C; ++k) {
                const double* ir = in + (size_t)k * w;
                const double* fr = F + (size_t)k * C;
                for (int c = 0; c < C; ++c) {
                    const double fv = fr[c];
                    if (fv == 0.0) continue;
                    double* orow = out + (size_t)c * w;
                    for (int j = 0; j < w; ++j) orow[j] += fv * ir[j];
                }
            }
        };
        auto neighbours = [&](std::vector<double>& A, int k, int step, int l) {
            const double* a = row(A, k - step);
            const double* b = row(A, k + step);
            for (size_t e = 0; e < rowsz; ++e) v[e] = -(f.wl[l] * a[e] + f.wr[l] * b[e]);
        };
        // Forward levels l0..L-2: rows i = 2s(t+1), i.e. tail rows k = 2 step (t+1).
        for (int l = l0; l + 1 < L; ++l) {
            const int step = 1 << (l - l0);
            for (int k = 2 * step; k <= rt + 1 - 2 * step; k += 2 * step) {
                neighbours(X, k, step, l);
                apply(f.Mt.data() + (size_t)l * n2, v.data(), row(X, k));
            }
        }
        // Back substitution L-1..l0: rows i = s(2t+1); tail rows 0 and rt+1 stay zero.
        for (int l = L - 1; l >= l0; --l) {
            const int step = 1 << (l - l0);
            for (int k = step; k <= rt + 1 - step; k += 2 * step) {
                double* y = row(Y, k);
                std::fill(y, y + rowsz, 0.0);
                apply(f.Bt.data() + (size_t)l * n2, row(X, k), y);
                neighbours(Y, k, step, l);
                apply(f.Mt.data() + (size_t)l * n2, v.data(), y);
            }
        }
        for (int k = 1; k <= rt; ++k)
            for (int c = 0; c < C; ++c) {
                const double* y = row(Y, k) + (size_t)c * w;
                double* d = D->data() + ((size_t)(k - 1) * C + c) * n + col0;
                for (int j = 0; j < w; ++j) d[j] = y[j];
            }
    };
    const int nth = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const int chunk = (n + nth - 1) / nth;
    std::vector<std::thread> pool;
    for (int t = 1; t < nth; ++t) pool.emplace_back(work, std::min(n, t * chunk), std::min(n, (t + 1) * chunk));
    work(0, std::min(n, chunk));
    for (auto& th : pool) th.join();
    for (double x : *D)
        if (!std::isfinite(x)) return false;
    return true;
}

std::vector<double> spline_moment_operator(int mc) {
    // Unknowns M_0..M_mc (second derivatives at the knots), H = 1/mc.
    // Interior knots k = 1..mc-1:  M_{k-1} + 4 M_k + M_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1}) / H^2.
    // Not-a-knot (third derivative continuous at x_1 and x_{mc-1}):
    //   M_0 - 2 M_1 + M_2 = 0,   M_{mc-2} - 2 M_{mc-1} + M_mc = 0.
    // Three knots (mc = 2): the interpolant is the parabola, M_0 = M_1 = M_2.
    const int K = mc + 1, Nc = mc - 1;
    const double H = 1.0 / mc;
    std::vector<double> Sm((size_t)K * Nc, 0.0);
    if (mc == 2) {
        for (int r = 0; r < 3; ++r) Sm[(size_t)r * 1 + 0] = -2.0 / (H * H);
        return Sm;
    }
    std::vector<double> Km((size_t)K * K, 0.0);
    Km[0 * K + 0] = 1.0; Km[0 * K + 1] = -2.0; Km[0 * K + 2] = 1.0;
    for (int k = 1; k < mc; ++k) {
        Km[(size_t)k * K + k - 1] = 1.0;
        Km[(size_t)k * K + k] = 4.0;
        Km[(size_t)k * K + k + 1] = 1.0;
    }
    Km[(size_t)mc * K + mc - 2] = 1.0; Km[(size_t)mc * K + mc - 1] = -2.0; Km[(size_t)mc * K + mc] = 1.0;
    std::vector<double> Kinv = Km;
    invert(Kinv, K);
    // rhs for a unit value at interior knot q (1..mc-1): row k gets 6/H^2 * (second difference of e_q at k).
    for (int q = 1; q < mc; ++q) {
        std::vector<double> rhs(K, 0.0);
        for (int k = 1; k < mc; ++k) {
            double v = 0.0;
            if (k + 1 == q) v += 1.0;
            if (k == q) v -= 2.0;
            if (k - 1 == q) v += 1.0;
            rhs[k] = 6.0 * v / (H * H);
        }
        for (int r = 0; r < K; ++r) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += Kinv[(size_t)r * K + k] * rhs[k];
            Sm[(size_t)r * Nc + (q - 1)] = acc;
        }
    }
    return Sm;
}

}  // namespace asdsm

// ---------------------------------------------------------------------------
// Additions for the 3D extension (Section 3.5)
// ---------------------------------------------------------------------------
namespace asdsm {

// Block cyclic reduction factors of  a x_{i-1} + K x_i + c x_{i+1} = f_i  with
// a dense C x C diagonal block K.  Because A_0 = a I and C_0 = c I commute with
// K, every level's blocks are A_l = alpha_l F_l, C_l = gamma_l F_l with one
// matrix F_l commuting with B_l, and
//     B_{l+1} = B_l - 2 alpha_l gamma_l F_l B_l^{-1} F_l,
//     F_{l+1} = F_l B_l^{-1} F_l,  alpha_{l+1} = -alpha_l^2,  gamma_{l+1} = -gamma_l^2,
// so a level costs one inverse and two products.  F absorbs the scale and the
// sign so that the dominant weight is +1 (the layout of BcrFactors).
bool make_bcr_dense(int R, double a, double c, int C, const std::vector<double>& K, BcrFactors* out) {
    int L = 0;
    while (((1 << L) - 1) < R) ++L;
    if (((1 << L) - 1) != R || C < 1 || L > 16 || K.size() != (size_t)C * C) return false;
    const size_t n2 = (size_t)C * C;
    out->R = R; out->C = C; out->L = L;
    out->Mt.assign((size_t)L * n2, 0.0);
    out->Bt.assign((size_t)L * n2, 0.0);
    out->wl.assign(L, 0.0);
    out->wr.assign(L, 0.0);
    std::vector<double> B = K, F(n2, 0.0), Binv, FB(n2), G(n2);
    for (int k = 0; k < C; ++k) F[(size_t)k * C + k] = 1.0;
    double al = a, ga = c;
    for (int l = 0; l < L; ++l) {
        // Normalise: the dominant weight becomes +1, F carries the factor.
        const double mu = std::fabs(al) >= std::fabs(ga) ? al : ga;
        if (mu == 0.0) {
            al = ga = 0.0;
        } else {
            for (double& v : F) v *= mu;
            al /= mu;
            ga /= mu;
        }
        Binv = B;
        if (!invert(Binv, C)) return false;
        matmul(F.data(), Binv.data(), FB.data(), C);                 // M_l = F_l B_l^{-1}
        transpose_into(FB.data(), out->Mt.data() + (size_t)l * n2, C);
        transpose_into(Binv.data(), out->Bt.data() + (size_t)l * n2, C);
        out->wl[l] = al;
        out->wr[l] = ga;
        if (l + 1 == L) break;
        matmul(FB.data(), F.data(), G.data(), C);                     // F B^{-1} F
        for (size_t e = 0; e < n2; ++e) B[e] -= 2.0 * al * ga * G[e];
        F.swap(G);
        al = -al * al;
        ga = -ga * ga;
    }
    for (double v : out->Mt) if (!std::isfinite(v)) return false;
    for (double v : out->Bt) if (!std::isfinite(v)) return false;
    return true;
}

namespace {

// y = P x for the 3 (or 2) rows r0.. of an n x n row-major matrix, P = I - 2 v v^T / (v^T v),
// applied to columns [c0, c1).
void house_left(std::vector<double>& H, int n, int r0, int m, const double* v, int c0, int c1) {
    double vv = 0.0;
    for (int t = 0; t < m; ++t) vv += v[t] * v[t];
    if (vv == 0.0) return;
    for (int j = c0; j < c1; ++j) {
        double d = 0.0;
        for (int t = 0; t < m; ++t) d += v[t] * H[(size_t)(r0 + t) * n + j];
        d *= 2.0 / vv;
        for (int t = 0; t < m; ++t) H[(size_t)(r0 + t) * n + j] -= d * v[t];
    }
}

// The same transformation from the right on columns r0.. of rows [q0, q1).
void house_right(std::vector<double>& H, int n, int r0, int m, const double* v, int q0, int q1) {
    double vv = 0.0;
    for (int t = 0; t < m; ++t) vv += v[t] * v[t];
    if (vv == 0.0) return;
    for (int i = q0; i < q1; ++i) {
        double d = 0.0;
        for (int t = 0; t < m; ++t) d += H[(size_t)i * n + r0 + t] * v[t];
        d *= 2.0 / vv;
        for (int t = 0; t < m; ++t) H[(size_t)i * n + r0 + t] -= d * v[t];
    }
}

// Householder vector v with (I - 2 v v^T / v^T v) x = (-sign(x0) |x|, 0, ..).
void house_vec(const double* x, int m, double* v) {
    double nx = 0.0;
    for (int t = 0; t < m; ++t) nx += x[t] * x[t];
    nx = std::sqrt(nx);
    for (int t = 0; t < m; ++t) v[t] = x[t];
    if (nx == 0.0) return;
    v[0] += x[0] >= 0.0 ? nx : -nx;
}

}  // namespace

// Real Schur form of an upper Hessenberg n x n matrix (row-major):
// A = Q T Q^T with Q orthogonal and T quasi upper triangular, whose 2 x 2
// diagonal blocks carry complex conjugate eigenvalue pairs and whose 1 x 1
// blocks the real eigenvalues.  Francis double-shift QR iteration with
// deflation (Golub and Van Loan, Sections 7.5.5-7.5.6), every transformation
// accumulated into Q and applied to the whole matrix; 2 x 2 blocks with real
// eigenvalues are split by one more rotation.  Returns false when the
// iteration does not converge.
bool real_schur(int n, const std::vector<double>& A, std::vector<double>* Qo, std::vector<double>* To) {
    if (n < 1 || A.size() != (size_t)n * n) return false;
    std::vector<double> H = A, Q((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    for (int i = 2; i < n; ++i)
        for (int j = 0; j < i - 1; ++j) H[(size_t)i * n + j] = 0.0;     // exact Hessenberg form
    auto at = [&](int i, int j) -> double& { return H[(size_t)i * n + j]; };
    const double eps = 2.220446049250313e-16;
    int m = n - 1, iter = 0, total = 0;
    while (m >= 1) {
        int l = m;
        for (; l >= 1; --l) {
            const double s = std::fabs(at(l - 1, l - 1)) + std::fabs(at(l, l));
            if (std::fabs(at(l, l - 1)) <= eps * (s > 0.0 ? s : 1.0)) { at(l, l - 1) = 0.0; break; }
        }
        if (l < 1) l = 0;
        if (l == m) { m -= 1; iter = 0; continue; }
        if (l == m - 1) { m -= 2; iter = 0; continue; }
        if (++total > 60 * n) return false;
        ++iter;
        // Shifts: the eigenvalues of the trailing 2 x 2 block (exceptional ones now and then).
        double s = at(m - 1, m - 1) + at(m, m);
        double t = at(m - 1, m - 1) * at(m, m) - at(m - 1, m) * at(m, m - 1);
        if (iter % 11 == 10) {
            const double w = std::fabs(at(m, m - 1)) + std::fabs(at(m - 1, m - 2));
            s = 1.5 * w + at(m, m);
            t = w * w;
        }
        double x = at(l, l) * at(l, l) + at(l, l + 1) * at(l + 1, l) - s * at(l, l) + t;
        double y = at(l + 1, l) * (at(l, l) + at(l + 1, l + 1) - s);
        double z = at(l + 1, l) * at(l + 2, l + 1);
        for (int k = l - 1; k <= m - 3; ++k) {
            const double xv[3] = {x, y, z};
            double v[3];
            house_vec(xv, 3, v);
            const int c0 = std::max(l, k);
            house_left(H, n, k + 1, 3, v, c0, n);
            house_right(H, n, k + 1, 3, v, 0, std::min(k + 4, m) + 1);
            house_right(Q, n, k + 1, 3, v, 0, n);
            if (k + 1 > l) { at(k + 2, k) = 0.0; at(k + 3, k) = 0.0; }
            x = at(k + 2, k + 1);
            y = at(k + 3, k + 1);
            if (k < m - 3) z = at(k + 4, k + 1);
        }
        const double xv[2] = {x, y};
        double v[2];
        house_vec(xv, 2, v);
        house_left(H, n, m - 1, 2, v, m - 2, n);
        house_right(H, n, m - 1, 2, v, 0, m + 1);
        house_right(Q, n, m - 1, 2, v, 0, n);
        at(m, m - 2) = 0.0;
    }
    // Split the 2 x 2 blocks whose eigenvalues are real.
    for (int i = 0; i + 1 < n; ++i) {
        if (at(i + 1, i) == 0.0) continue;
        const double a = at(i, i), b = at(i, i + 1), c = at(i + 1, i), d = at(i + 1, i + 1);
        const double p = 0.5 * (a - d), disc = p * p + b * c;
        if (disc < 0.0) { ++i; continue; }                            // a complex pair: keep the block
        // An eigenvector (b, lambda - a) of the block for lambda = d + p +/- sqrt(disc).
        const double lam = d + p + (p >= 0.0 ? std::sqrt(disc) : -std::sqrt(disc));
        double e0 = b, e1 = lam - a;
        if (std::fabs(e0) + std::fabs(e1) == 0.0) { e0 = lam - d; e1 = c; }
        const double r = std::hypot(e0, e1);
        const double cs = e0 / r, sn = e1 / r;
        // Rotation G = [[cs, -sn], [sn, cs]] on rows/columns i, i+1: T <- G^T T G, Q <- Q G.
        for (int j = 0; j < n; ++j) {
            const double h0 = at(i, j), h1 = at(i + 1, j);
            at(i, j) = cs * h0 + sn * h1;
            at(i + 1, j) = -sn * h0 + cs * h1;
        }
        for (int j = 0; j < n; ++j) {
            const double h0 = at(j, i), h1 = at(j, i + 1);
            at(j, i) = cs * h0 + sn * h1;
            at(j, i + 1) = -sn * h0 + cs * h1;
            const double q0 = Q[(size_t)j * n + i], q1 = Q[(size_t)j * n + i + 1];
            Q[(size_t)j * n + i] = cs * q0 + sn * q1;
            Q[(size_t)j * n + i + 1] = -sn * q0 + cs * q1;
        }
        at(i + 1, i) = 0.0;
        ++i;
    }
    *Qo = Q;
    *To = H;
    return true;
}

// Values at the fine interior points x = p h (p = 1..M-1) of the not-a-knot
// cubic spline through the knots 0, H, .., 1 with zero end values and value 1
// at interior knot m (R10): W is (M-1) x (mc-1), row-major.
std::vector<double> spline_value_operator(int mc, int n) {
    const int M = mc * n, Nc = mc - 1, Nf = M - 1;
    const double H = 1.0 / mc;
    const std::vector<double> Sm = spline_moment_operator(mc);       // (mc+1) x (mc-1)
    std::vector<double> W((size_t)Nf * Nc, 0.0);
    for (int m = 0; m < Nc; ++m) {
        for (int p = 1; p <= Nf; ++p) {
            const int i = std::min(p / n, mc - 1);                      // knot interval [i H, (i+1) H]
            const double x = (double)p / M, xi = i * H, xj = (i + 1) * H;
            const double yi = (i == m + 1) ? 1.0 : 0.0, yj = (i + 1 == m + 1) ? 1.0 : 0.0;
            const double Mi = Sm[(size_t)i * Nc + m], Mj = Sm[(size_t)(i + 1) * Nc + m];
            const double a = xj - x, b = x - xi;
            W[(size_t)(p - 1) * Nc + m] = Mi * a * a * a / (6.0 * H) + Mj * b * b * b / (6.0 * H)
                                        + (yi - Mi * H * H / 6.0) * a / H + (yj - Mj * H * H / 6.0) * b / H;
        }
    }
    return W;
}

}  // namespace asdsm
