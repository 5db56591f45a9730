// Internal declarations shared by the translation units of the ASDSM library.
// Not part of the public ABI (see include/asdsm.h).
#pragma once
#include <cstdint>
#include <cstddef>
#include <vector>
#include <string>
#include <cuda_runtime.h>

namespace asdsm {

// ---------------------------------------------------------------------------
// Host FP64 precomputation (host_math.cu)
// ---------------------------------------------------------------------------

// Block cyclic reduction factors of the block tridiagonal Toeplitz system
//     a x_{i-1} + (d I + T) x_i + c x_{i+1} = f_i,   i = 1..R,  x_0 = x_{R+1} = 0,
// with R = 2^L - 1 rows and T the C x C tridiagonal Toeplitz matrix
// tridiag(tl, td, tu) (T[k][k-1] = tl, T[k][k+1] = tu).  At level l the
// surviving rows satisfy A_l x_{i-s} + B_l x_i + C_l x_{i+s} = f_i^(l)
// (s = 2^l), with P_l = A_l B_l^{-1} and Q_l = C_l B_l^{-1}.  Because
// A_0 = a I and C_0 = c I, every level keeps C_l = (c/a)^(2^l) A_l, hence
// Q_l = (c/a)^(2^l) P_l: one matrix per level serves both neighbours.
// Stored per level: M_l (the larger of P_l, Q_l) and B_l^{-1}, transposed
// ([k][c] = M[c][k]), and the weights with P_l = wl_l M_l, Q_l = wr_l M_l
// (one of them is 1, the other has modulus <= 1).
struct BcrFactors {
    int R = 0, C = 0, L = 0;
    std::vector<double> Mt, Bt;       // [L][C][C]
    std::vector<double> wl, wr;       // [L]
};
bool make_bcr(int R, double a, double d, double c, int C, double tl, double td, double tu, BcrFactors* out);

// The tail of the reduction as one dense map.  For rt = 2^t - 1 <= R, the
// forward levels l0..L-2 and the back substitution L-1..l0 (l0 = L - t) touch
// only the rt rows i = k 2^l0 (k = 1..rt) and map their reduced right-hand
// sides to their solutions linearly; D is that map, (rt C) x (rt C)
// row-major, entry ((k-1) C + c, (k'-1) C + c') from row k', column c' of the
// input to row k, column c of the output.  False on a non-finite entry.
bool bcr_tail_map(const BcrFactors& f, int rt, std::vector<double>* D);

// The same with a dense C x C diagonal block:  a x_{i-1} + K x_i + c x_{i+1} = f_i
// (K row-major; the 3D extension's submesh systems have Kronecker-sum blocks).
bool make_bcr_dense(int R, double a, double c, int C, const std::vector<double>& K, BcrFactors* out);

// Real Schur form A = Q T Q^T of an upper Hessenberg n x n matrix (row-major):
// Q orthogonal, T quasi upper triangular with 2 x 2 blocks only for complex
// conjugate eigenvalue pairs.  False if the QR iteration does not converge.
bool real_schur(int n, const std::vector<double>& A, std::vector<double>* Q, std::vector<double>* T);

// Values at the fine interior points p h (p = 1..mc n - 1) of the not-a-knot
// spline with zero end values and value 1 at interior knot m: (mc n - 1) x (mc - 1).
std::vector<double> spline_value_operator(int mc, int n);

// Moments of the not-a-knot cubic spline on the uniform knots 0, H, .., 1
// (mc intervals) through values (0, y_1, .., y_{mc-1}, 0): M = Sm y with
// Sm of shape (mc+1) x (mc-1), row-major.
std::vector<double> spline_moment_operator(int mc);

// ---------------------------------------------------------------------------
// Device-side descriptors
// ---------------------------------------------------------------------------
constexpr int kMaxLevels = 16;

template <typename T>
struct BcrSys {
    T* X;              // right-hand sides, [nsys][R][C]; overwritten by the forward reduction
    T* Y;              // solutions, [nsys][R][C]
    const T* Mt;       // [L][C][C]
    const T* Bt;       // [L][C][C]
    T wl[kMaxLevels], wr[kMaxLevels];
    int R, C, L;
    int nsys;          // systems sharing these factors
    long long stride;  // elements between consecutive systems
    // FP32 only: the factors again for the wide tensor-core level kernel,
    // [L][KW][CW] (rows padded to KW = 32-multiple, columns to CW = 256-multiple,
    // zeros outside C x C), 16-byte column chunks XOR-swizzled within groups of
    // 8 by 2*(k mod 4): element (k, c) at column ((c/4) ^ (2 (k mod 4))) * 4 + c mod 4.
    const float* Mw;
    const float* Bw;
    int KW, CW;
    // FP32 only: the factors for the tensor-core level kernel (bcr_tc.cu),
    // B operand blocks [L][pass: B^-1, M][split: hi, lo][TCB][TKC] of 128
    // columns x 32 reduction values, swizzled; null when absent.
    const float* Ti;
    int TKC, TCB;
    int* tc_err;       // set to 1 when a tensor-core kernel's wait timed out
    // FP32 only: bcr_tail_map for tail_rt rows, [tail_rt C][tail_ld] (rows
    // padded with zeros to tail_ld, a multiple of 4); null: every level runs.
    const float* Dt;
    int tail_rt, tail_ld;
};

// Stencil coefficients of A_ff (5-point, Section 2.3): A u = cc u_c + cw u_w + ce u_e + cs u_s + cn u_n.
struct Stencil {
    double cc, cw, ce, cs, cn;
};

struct Geometry {
    int N;      // grid points per axis incl. boundary
    int M;      // N - 1 fine intervals
    int Nf;     // N - 2 interior points per axis
    int mc;     // coarse intervals
    int Nc;     // mc - 1 coarse lines per axis
    int n;      // M / mc (a power of two)
    int ln;     // log2(n)
    long long skel;   // compact skeleton length: Nc*Nf + Nc*(Nf - Nc)
};

// Process-wide count of kernel launches made by the library.
void note_launch(long long n = 1);
long long launch_count();

// ---------------------------------------------------------------------------
// Kernel launchers (kernels_*.cu).  All enqueue on `st`; none synchronise.
// ---------------------------------------------------------------------------
// Launch shape of every BCR level: cfg[dir][level] = (TM << 8) | KS with TM
// in {16, 64} output rows per CTA and KS in {1, 2, 4, 8} CTAs per cluster
// splitting the reduction, or TM = 32: the wide tensor-core kernel (FP32, 32
// rows x 256 columns per CTA, mma.sync, KS = 1), or TM = 128: the tcgen05
// kernel (FP32, 128 x 128 per CTA, KS = 1); 0 (or no table) = the built-in choice.
struct BcrTune {
    int cfg[2][kMaxLevels];    // [0] forward, [1] backward
    int num_sms;
    int trace;                 // print every launch shape (debugging)
};
// Block cyclic reduction of up to 2 factor groups (e.g. the fc and cf families).
template <typename T>
cudaError_t bcr_solve(const BcrSys<T>* groups, int ngroups, cudaStream_t st, const BcrTune* tune = nullptr);
// Coefficients of a system make_bcr factors: a x_{i-1} + (d I + T) x_i + c x_{i+1},
// T = tridiag(tl, td, tu).
struct BcrCoefs { double a, d, c, tl, td, tu; };
// r32 = (float)(b - A x) over the R x C system (FP64 arithmetic).
cudaError_t bcr_residual(const double* x, const double* b, float* r32, int R, int C, const BcrCoefs& k,
                         cudaStream_t st);
// x += (double) y over n elements.
cudaError_t add_float(double* x, const float* y, long long n, cudaStream_t st);
// One level of it (forward reduction or back substitution), for tuning.
template <typename T>
cudaError_t bcr_level(const BcrSys<T>* groups, int ngroups, int level, bool backward, const BcrTune* tune,
                      cudaStream_t st);

// Mode of the hole solve of Algorithm 3.
enum FillMode : int {
    FILL_WITH_SOURCE = 0,   // rhs = s - A_hs z  (inhomogeneous Filler of the initial guess; z carries g on its ring)
    FILL_HOMOGENEOUS = 1,   // rhs = - A_hs z     (Filler with zero source, in the correction of Algorithm 4)
    FILL_RESIDUAL_TO_U = 2, // rhs = r (holes);  u_holes += solution   (hole-residual correction)
    FILL_ARRAY = 3          // rhs = given array (holes), no skeleton term; write solution to out
};

// Fused Algorithm 3 over all holes: each CTA keeps the hole BCR factors in
// shared memory and solves holes one after another.
template <typename T>
struct FillArgs {
    int mode;
    const T* z;               // full grid, skeleton values (and g on the ring for FILL_WITH_SOURCE)
    T* out;                   // full grid, receives hole values (modes 0, 1, 3)
    const double* src_d;      // FP64 source grid (mode 0, FP64 path) / rhs grid (mode 3)
    const float* src_hi;      // FP32 source (mode 0, mixed path) / residual grid (mode 2)
    double* out_d;            // modes 0, 1, 3: if set, hole values written here as FP64 (instead of out)
    double* u_d;              // mode 2, FP64 path: u += v on holes
    long long* U;             // mode 2, mixed path: U += round(v * scale)
    double fixed_scale;       // 2^S for mode 2 mixed
    const T* Mt; const T* Bt;
    T wl[kMaxLevels], wr[kMaxLevels];
    int L, n;                 // hole systems are (n-1) x (n-1)
    Geometry g;
    Stencil sten;
    int warps;                // warps per CTA (0: as many as shared memory allows, at most 8)
};
template <typename T>
cudaError_t fill_holes(const FillArgs<T>& a, int num_sms, cudaStream_t st);
template <typename T>
size_t fill_smem_bytes(int n, int L);

// Tensor-core BCR level kernel (bcr_tc.cu), FP32 systems: the image of the
// factors (BcrSys::Ti, TKC, TCB) and one level for 1 or 2 groups, the
// reduction of each output tile split over ks (1, 2 or 4) CTAs of a cluster.
void bcr_tc_image(const BcrFactors& f, std::vector<float>* img, int* KC, int* CB);
cudaError_t bcr_tc_level(const BcrSys<float>& g0, const BcrSys<float>& g1, int ngroups, int level, bool backward, int ks,
                         int maxRows, int nsys, cudaStream_t st);

// Discrete harmonic extension of a C x C hole (Algorithm 3 with zero source,
// host_math.cu): the hole values v (row by row, y = 1..C, x = 1..C) are G z
// for the 4C ring values z ordered west (y = 1..C), east (y = 1..C), south
// (x = 1..C), north (x = 1..C); G = -A_hh^{-1} A_hs, [C*C][4C] row-major.
bool hole_extension_operator(int C, const Stencil& s, std::vector<double>* G);

// The same for the cube holes of the 3D extension (host_math.cu): the C^3
// hole values (x fastest, then y, then z) are G z for the 6 C^2 face values z
// ordered west (x = 0), east (x = C+1), south (y = 0), north (y = C+1), down
// (z = 0), up (z = C+1), each face's C x C values with its second axis
// slowest (west/east: (y, z); south/north: (x, z); down/up: (x, y)).
// sten7 = {cc, cw, ce, cs, cn, cd, cu} (centre; x-1, x+1; y-1, y+1; z-1, z+1).
// G is [C^3][6 C^2] row-major.
bool hole_extension_operator_3d(int C, const double sten7[7], std::vector<double>* G);

// Tensor-core Filler (fill_tc.cu): the homogeneous fill for holes of
// kFillTcN - 1 = 15 points per side (n = 16), FP32 results.
constexpr int kFillTcN = 16;
struct FillTcArgs {
    const float* gimg;   // fill_tc_image() of G, fill_tc_image_bytes() bytes, 16-byte aligned
    float* z;            // full grid: ring values read, hole values written (unless out_d)
    double* out_d;       // if set, hole values written here in FP64 instead of into z
    const float* zv;     // if set: the values on the lines x = k n, [N][mc+1] (column k; columns 0
                         // and mc zero): west / east ring values are read here, and every hole row
                         // is written whole, its skeleton point x = k n taken from here
    int N, mc;           // N = 16 mc + 1
    int* err;            // set to 1 when a wait timed out (the fill is then incomplete)
};
// One CTA that holds tensor memory and waits, bounded by limit_ns, on an
// mbarrier nothing arrives at; sets *err = 1 when the wait gives up.
cudaError_t wait_selftest(int* err, long long limit_ns, cudaStream_t st);
size_t fill_tc_image_bytes();
void fill_tc_image(const std::vector<double>& G, std::vector<float>* img);
cudaError_t fill_tc(const FillTcArgs& a, int num_sms, cudaStream_t st);

// Right-hand sides of eq. (2.4) on the submeshes (Dirichlet lifting from u's ring).
template <typename T>
cudaError_t build_submesh_rhs(const double* s, const double* u, const Geometry& g,
                              const double alpha[2], const double beta[2],
                              T* bfc, T* bcf, T* bcc, cudaStream_t st);

// Residual kernels -----------------------------------------------------------
struct ResidOut {
    void* rfc;          // T [Nf][Nc]  (BCR layout of Omega^{h,H})
    void* rcf;          // T [Nf][Nc]  (BCR layout of Omega^{H,h})
    void* rskel;        // T [skel]    (compact skeleton)
    void* rfull;        // float or double full grid (optional)
    double* partials;   // [nblocks][2]: sum r^2, sum r^2 over holes
};
// The update of Algorithm 4 as state on the device (sweeps driven from the GPU):
// the residual kernel of the next sweep reads the pending step lengths and
// which of the two iterate buffers is current.
struct DynUpdate {
    int live;           // 0 once the solve has ended: the residual kernel returns at once
    int count;          // pending directions: u += sum_j coef_j z_j, j < count
    int par;            // current iterate: buffer 0 (par = 0) or buffer 1
    int skip;           // 1: a sweep inside a GCR cycle, the residual is tracked on the skeleton
                        //    and the residual kernel returns at once
    double coef[16];    // step lengths (FP64 path)
    float cf[16];       // step lengths times 2^S, rounded to FP32 (mixed path)
};
struct UpdateTerms {
    const void* z[16];  // directions (T full grid)
    double coef[16];    // u += sum coef_j z_j
    int count;
    // Non-null: count, coefficients and the current buffer come from the
    // device; the kernel's input/output pointers are then buffers 0 and 1.
    const DynUpdate* dyn;
};
// FP64 path: u_out = u_in + sum coef z (interior), r = s - A u_out.
cudaError_t residual_fp64(const double* s, const double* u_in, double* u_out, const UpdateTerms& up,
                          const Geometry& g, const Stencil& st_, ResidOut out, int* nblocks, cudaStream_t st);
// Mixed path: U_out = U_in + round(2^S sum coef z), r = s - A U_out 2^-S in FP32-pair arithmetic
// (coef are the unscaled step lengths; `scale` = 2^S).
// Stencil parts q = 0..3 (alpha_x/h^2, alpha_y/h^2, beta_x/(2h), beta_y/(2h)), each times 2^-S,
// pre-multiplied by the weights of the 22-bit pieces of the integer differences.
struct MixedCoefs {
    float k2[4][2];   // (hi, lo) of part * 2^44
    float k1[4][2];   // (hi, lo) of part * 2^22
    float k0[4];      // part (FP32; the low piece needs no more)
};
cudaError_t residual_mixed(const float* s_hi, const float* s_lo, const long long* U_in, long long* U_out,
                           const UpdateTerms& up, double scale, const Geometry& g, const MixedCoefs& k,
                           ResidOut out, int* nblocks, int* overflow_flag, cudaStream_t st);
int residual_grid_blocks(const Geometry& g);

// FP64 check of a returned iterate (s, u: FP64 grids, u's ring = g):
// out[0] = ||s - A u||^2 over the interior, out[1] = max |s - A u| over the
// hole points.  partials: at least 2 * max_blocks doubles.
cudaError_t final_check(const double* s, const double* u, const Geometry& g, const Stencil& c, double* partials,
                        int max_blocks, double* out, cudaStream_t st);

// Reductions ----------------------------------------------------------------
// out[j] = sum over blocks of partials[b][j]  (fixed order, 1 CTA), j < ncols
cudaError_t reduce_partials(const double* partials, int nblocks, int ncols, double* out, cudaStream_t st);
// The dot kernels run at most kDotBlocks CTAs and at most kMaxDots dots, so
// kDotPartials doubles hold their partials; every reduction scratch is at
// least that large.
constexpr int kDotBlocks = 152 * 4, kMaxDots = 40, kDotPartials = kDotBlocks * kMaxDots;
// Multi-dot: out partials for dots <a_i, b_i>, i < ndots <= kMaxDots over length n vectors.
template <typename T>
cudaError_t multi_dot(const T* const* a, const T* const* b, int ndots, long long n,
                      double* partials, int* nblocks, cudaStream_t st);

// GCR inner products in one pass: partials [block][2 + 2k] = <q,q>, <q,r>, then
// <q,p_j>, <r,p_j> for j < k (k <= 15).
template <typename T>
cudaError_t gcr_dots(const T* q, const T* r, const T* const* p, int k, long long n,
                     double* partials, int* nblocks, cudaStream_t st);

// Merge (Algorithm 2) --------------------------------------------------------
template <typename T>
struct MergeArgs {
    const T* Yfc;  const T* Ycf;  const T* Ycc;  // solutions; Ycc used when re_mode
    const double* norms2;     // [2]: ||Yfc||^2, ||Ycf||^2 (normalisation of Algorithm 1)
    int re_mode;              // 1: Richardson (u_cc given), 0: random choice
    int choice;               // 0 or 1 (random choice of Algorithm 2)
    const int* choice_dev;    // non-null: the choice is read from the device instead
    const T* Sm;              // spline moment operator, transposed: [Nc knots][mc+1 moments]
    T* E1; T* E2;             // [Nc][Nc] knot errors (fc lines: E1[l][k]; cf columns: E2[l][k])
    T* M1; T* M2;             // moments: M1[l][mc+1] (fc line l), M2[mc+1][Nc] (moment-major: the
                              // cf points of one row read consecutive columns k)
    T* z;                     // full grid output (skeleton written)
    T* zv;                    // non-null: the points of the lines x = k n (k = 1..mc-1) between knots go
                              // here, [N][mc+1] (column k), instead of into z
    Geometry g;
};
template <typename T> cudaError_t merge_knots(const MergeArgs<T>& a, cudaStream_t st);
template <typename T> cudaError_t merge_write(const MergeArgs<T>& a, cudaStream_t st);

// q = (A z) on the compact skeleton.
template <typename T>
cudaError_t skeleton_apply(const T* z, const Geometry& g, const Stencil& s, T* q, cudaStream_t st);
// qp = (q - sum beta_j Qp_j) * inv_nu   (Qp, beta: host arrays, k <= 16)
template <typename T>
cudaError_t combine_skeleton(const T* q, const T* const* Qp, const double* beta, int k, double inv_nu,
                             long long n, T* out, cudaStream_t st);

// Device-held GCR combination: qp = (q - sum beta_j Qp_j) * inv_nu when run != 0.
struct CtlCombine {
    int run;
    int track;          // 1: then r_skel -= alpha qp (the tracked residual) and the submesh
                        //    right-hand sides are gathered from it for the next sweep
    double beta[16];
    double inv_nu;
    double alpha;
    float beta_f[16];   // the same rounded to FP32, for the FP32 kernels (no FP64 work per element)
    float inv_nu_f;
    float alpha_f;
};
template <typename T>
cudaError_t combine_skeleton_dyn(const T* q, const T* const* Qp, int k, const CtlCombine* c,
                                 long long n, T* out, cudaStream_t st);
// The tracked residual of a deferred GCR cycle: r_skel -= alpha qp on the compact
// skeleton and r_fc, r_cf (the submesh right-hand sides, BCR layouts) gathered
// from it; with track = 0 (from the device control when c is given) nothing is done.
template <typename T>
cudaError_t track_skeleton(T* rskel, const T* qp, double alpha, const CtlCombine* c, const Geometry& g, T* rfc,
                           T* rcf, cudaStream_t st);

// Sweep control on the device (control.cu) ---------------------------------------
// The decisions of Algorithm 4 that the host loop takes between sweeps
// (convergence, stagnation, the hole-residual correction, the GCR(m)
// bookkeeping), kept in device memory so that whole sweeps run as a CUDA graph.
struct SweepCtl {
    // Set by the host before the first sweep.
    double bnorm, tol, hole_fix_ratio, hole_fix_growth, stagnation_factor, scale;
    unsigned long long seed;
    int max_sweeps, window, m, mixed;
    int hist_cap;
    // State.
    int k, status, done, kc, hole_fixes, hole_ref_pending, nhist, branch;
    int runs[20];                 // executions of each branch (sweep bodies 0..m-1, hole fixes m, m+1)
    double hole_ref, rel0, rel;
    double Tm[16][16];
    // GCR cycles with a deferred update (m > 1): the cycle's step coefficients
    // in the basis of its raw directions, applied by the residual kernel of the
    // cycle's next true residual; in between, ||r||^2 is tracked on the skeleton
    // (rr_skel) plus the hole part of the cycle's first residual (rh2).
    double cacc[16];
    double rr_skel, rh2;
    int defer;          // deferred cycles in use (m > 1); cleared for the rest of the solve near the
                        // tolerance or when a cycle's true residual exceeds twice its tracked value
    int cycle_ended;    // the residual about to be computed closes a deferred cycle
    int stag_hold;      // sweeps without the stagnation test (after a tracked value was replaced)
    int pad3;
    DynUpdate upd;
    int choice;
    int pad2;
    CtlCombine comb;
};
// Deferred GCR cycles stop for the rest of a solve once a true residual is
// below kDeferStop * tol: from there each sweep applies its step and takes a
// true residual.  Measured at 4097^2 (three seeds): factor 3 takes 11-13% less
// time than factor 100 with the same or fewer sweeps; without the stop, early
// cycle ends near the tolerance cost more than they save.
constexpr double kDeferStop = 3.0;

// After the residual norms: decide the branch of this sweep and select it in
// the graph's switch node (value m + 2 = nothing: the solve has ended).
cudaError_t ctl_after_residual(SweepCtl* c, const double* sums, int* overflow, double* hist,
                               cudaGraphConditionalHandle sw, cudaStream_t st);
// After the least-squares inner products: the step lengths (clamped optimal scaling / GCR(m)).
cudaError_t ctl_after_dots(SweepCtl* c, const double* dots, cudaStream_t st);

// Learned correction: input channels [r rs, e es, c0..c3] of the full grid,
// and the network output kept on the interior skeleton points of z.
cudaError_t cnn_features(const float* r, const float* e, float rs, float es, const float c[4], long long nn, float* x,
                         cudaStream_t st);
cudaError_t skeleton_from(const float* y, const Geometry& g, float* z, cudaStream_t st);

// Grid utilities -------------------------------------------------------------
template <typename T>
cudaError_t fill_value(T* p, long long n, T v, cudaStream_t st);
// dst interior = src interior (converted), ring untouched
template <typename Ts, typename Td>
cudaError_t copy_interior(const Ts* src, Td* dst, const Geometry& g, cudaStream_t st);
// z (T full grid) = 0 interior, ring = g from u
template <typename T>
cudaError_t ring_from(const double* u, T* z, const Geometry& g, int zero_interior, cudaStream_t st);
// max |v| over a full grid (double partials per block)
template <typename T>
cudaError_t maxabs(const T* v, long long n, double* partials, int* nblocks, cudaStream_t st);
// z == nullptr: convert u_ring_src everywhere (resume from an FP64 iterate)
cudaError_t to_fixed(const float* z, const double* u_ring_src, long long* U, double scale, const Geometry& g, cudaStream_t st);
cudaError_t from_fixed(const long long* U, double inv_scale, double* u, const Geometry& g, cudaStream_t st);
cudaError_t split_source(const double* s, float* hi, float* lo, long long n, cudaStream_t st);
// compact skeleton <-> BCR layouts, for checking: convert FP64 in -> T
template <typename Ts, typename Td>
cudaError_t convert_array(const Ts* in, Td* out, long long n, cudaStream_t st);

}  // namespace asdsm
