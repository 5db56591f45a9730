/*
 * asdsm.h - C ABI of the GB300 (sm_103a) implementation of the Anisotropic
 * Submeshes Domain Splitting Method (ASDSM) of K. Trotti, "A domain splitting
 * strategy for solving PDEs" (arXiv 2303.01163).
 *
 * The library solves the steady advection-diffusion equation (eq. 1.1)
 *     sum_i ( -alpha_i d^2u/dx_i^2 + beta_i du/dx_i ) = s   on the unit square,
 *     u = g                                              on its boundary,
 * discretised by second-order centred finite differences on a uniform grid
 * (Section 2.3), by iterating Algorithm 4 (ASDSM) of Section 3.2 on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid arrays are dense FP64, x fastest (the vector ordering of Section 2.2):
 * element (i, j) of an N x N grid (point x = i/(N-1), y = j/(N-1)) is at
 * offset j*N + i.  Arrays cover the whole grid INCLUDING the boundary ring.
 * All array arguments are DEVICE pointers owned by the caller (for example
 * PyTorch tensors); the library never frees them.  Work is enqueued on the
 * CUDA stream given to asdsm_setup.  Functions that report results to the
 * host (asdsm_solve, asdsm_residual, asdsm_initial_guess) synchronise that
 * stream before returning; the others return once the work is enqueued.
 *
 * Sizes: N - 1 must be a power of two (N = 2^p + 1, p >= 2) and mc (coarse
 * intervals per axis, the N_c + 1 of eq. 2.1) a power of two with
 * 2 <= (N - 1)/mc <= 32, so every line, submesh and hole system has
 * 2^q - 1 unknowns per axis and a hole's factors fit in shared memory, and
 * N <= 32769 (grid offsets fit 32-bit integers).  Other sizes return
 * ASDSM_ERR_INVALID.
 *
 * The 3D extension (Section 3.5; asdsm_desc.d = 3): the unit cube, N x N x N
 * grids (element (i, j, l) at offset (l*N + j)*N + i, boundary included),
 * the 7-point operator with alpha_i, beta_i per axis x, y, z.  Sizes: N - 1
 * and mc powers of two with N <= 257, 2 <= mc <= 32 and
 * 2 <= (N - 1)/mc <= 16.  ASDSM iterates over the three plane families
 * Omega^{H,h,h}, Omega^{h,H,h}, Omega^{h,h,H}; the initial guess also solves
 * the line families and the coarse mesh to extrapolate the intersection
 * points.  asdsm_setup, asdsm_set_opts, asdsm_solve, asdsm_initial_guess,
 * asdsm_residual (rel_norm only; r must be NULL), asdsm_submesh_solve,
 * asdsm_history and asdsm_destroy accept 3D handles; the other entry points
 * that take a handle return ASDSM_ERR_INVALID for them.  The mixed path keeps
 * the iterate, the residual and the accumulation in FP64 (not fixed point).
 *
 * Errors: every int-returning function returns ASDSM_OK (0) or a negative
 * code (see asdsm_strerror).  The library never aborts or traps; after an
 * error the handle stays valid and may be destroyed or reused.
 */
#ifndef ASDSM_H
#define ASDSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define ASDSM_OK                 0
#define ASDSM_ERR_INVALID       -1   /* bad argument: sizes violate eq. 2.1 / powers of two, alpha <= 0, null pointer */
#define ASDSM_ERR_CUDA          -2   /* a CUDA runtime call failed, or a tensor-core kernel's bounded
                                        wait ran out (1 s; sticky for the handle); message in
                                        asdsm_last_error */
#define ASDSM_ERR_OOM           -3   /* device allocation failed */
#define ASDSM_ERR_NAN           -4   /* a NaN/Inf appeared in the residual (bad input data) */
#define ASDSM_NOT_CONVERGED     -5   /* max_sweeps reached above tol; u holds the last iterate */
#define ASDSM_STAGNATED         -6   /* residual stopped decreasing (Remark after Alg. 4); u holds the last iterate */
#define ASDSM_ERR_RANGE         -7   /* mixed path: the fixed-point accumulator would still overflow after
                                        12 restarts with ever smaller shifts (each restart resumes from the
                                        last iterate that fitted, with at least 16x more range); u holds
                                        that iterate.  asdsm_solve_batch does not restart. */

/* ---- precision modes ---------------------------------------------------- */
#define ASDSM_FP64   0   /* every step in FP64 (the plain method) */
#define ASDSM_MIXED  1   /* submesh solves, merge, fill and directions in FP32; residual and
                            accumulation exact to FP64 level (64-bit fixed-point u, FP32-pair
                            arithmetic for the residual) */

/* Problem description: one instance of eq. (1.1) on the unit square (d = 2)
 * or the unit cube (d = 3). */
typedef struct {
    int32_t d;          /* space dimension: 2, or 3 for the 3D extension of Section 3.5 */
    int32_t n;          /* grid points per axis including the boundary (N) */
    int32_t mc;         /* coarse intervals per axis (N_c + 1 in eq. 2.1) */
    int32_t pad_;
    double  alpha[3];   /* diffusion per axis, > 0 (x, y[, z]) */
    double  beta[3];    /* advection per axis (x, y[, z]) */
} asdsm_desc;

/* Iteration options of Algorithm 4. */
typedef struct {
    double   tol;               /* stop when ||b - A u||_2 / ||b||_2 <= tol */
    int32_t  max_sweeps;        /* sweeps of Algorithm 4 (hole corrections count as sweeps) */
    int32_t  precision;         /* ASDSM_FP64 or ASDSM_MIXED */
    int32_t  accel_m;           /* 1: the paper's clamped optimal scaling (s_hat >= 0); m > 1: restarted GCR(m) with the
                                   Algorithm-1 correction as flexible preconditioner */
    int32_t  skip_initial_guess;/* 1: start from the interior of u as given (resume); 0: Algorithm 1 */
    uint64_t seed;              /* SplitMix64 seed of the random choice of Algorithm 2 */
    double   hole_fix_ratio;    /* re-fill holes when ||r_holes|| > ratio*||r|| ... */
    double   hole_fix_growth;   /* ... and > growth * (hole residual after the last fill) */
    int32_t  stagnation_window; /* stagnated if ||r_k|| > (1 - stagnation_factor) ||r_{k-window}|| */
    int32_t  sweep_graph;       /* 1 (default): sweeps replayed as CUDA graphs, every decision between
                                   sweeps taken on the device; 0: the host takes them (two reads per
                                   sweep).  Same arithmetic; profiling (asdsm_profile) uses 0. */
    double   stagnation_factor;
} asdsm_opts;

/* Per-solve statistics. */
typedef struct {
    int32_t sweeps;        /* sweeps performed (including hole corrections) */
    int32_t status;        /* ASDSM_OK, ASDSM_NOT_CONVERGED, ASDSM_STAGNATED, ... */
    int32_t hole_fixes;    /* hole-residual corrections performed */
    int32_t fixed_shift;   /* mixed path: u = U * 2^-fixed_shift; 0 on the FP64 path */
    double  rel_res;       /* final ||b - A u|| / ||b|| */
    double  rel_res0;      /* relative residual of the initial iterate */
    double  setup_ms;      /* right-hand sides + initial guess, GPU time */
    double  solve_ms;      /* whole call, GPU time */
    int64_t launches;      /* kernels this call launched */
    double  rel_res_fp64;  /* ||b - A u||_2 / ||b||_2 of the returned u, recomputed in FP64 arithmetic
                              from the caller's s and u at the end of every solve */
    double  hole_res_max;  /* max |b - A u| over the hole points of the returned u (FP64; zero in exact
                              arithmetic by Prop. 3.1) */
    int32_t rescales;      /* mixed path: restarts with a smaller fixed-point shift after the
                              accumulator would have overflowed (see ASDSM_ERR_RANGE) */
    int32_t pad_;
} asdsm_stats;

/* Per-kernel-family timing of the last asdsm_solve calls (enabled with
 * asdsm_profile).  ms is the sum of CUDA-event durations on the handle's
 * stream around the family's launches; bytes and flops are the ALGORITHMIC
 * traffic and arithmetic of those launches (the minimum the method needs:
 * each grid value read or written once), counted by the library. */
typedef struct {
    char    name[24];
    int64_t launches;
    int64_t calls;         /* timed groups (one group may hold several launches) */
    double  ms;
    double  bytes;
    double  flops;
} asdsm_kprof;

typedef struct asdsm_handle asdsm_handle;

/* Fill *opts with the defaults: tol 1e-10, max_sweeps 500, ASDSM_MIXED,
 * accel_m 8, seed 0, hole_fix_ratio 0.25, hole_fix_growth 4, stagnation
 * window 10 with factor 1e-3, skip_initial_guess 0. */
void asdsm_default_opts(asdsm_opts* opts);

/* Create a solver for one problem (eq. 1.1 with desc's sizes and
 * coefficients).  Precomputes, in FP64 on the host, the block cyclic
 * reduction factors of every submesh operator of eq. (2.4) (A_fc, A_cf, A_cc
 * and the hole blocks A_(ij) of Remark 2.4) and the spline operator of
 * Algorithm 2, uploads them, and allocates all device work space.
 * stream: a cudaStream_t (NULL = legacy default stream).  The handle keeps
 * the stream; opts are copied.  Returns ASDSM_ERR_INVALID for sizes that
 * violate eq. (2.1) or the power-of-two rule, ASDSM_ERR_OOM if allocation
 * fails.  *out is NULL on error. */
int asdsm_setup(const asdsm_desc* desc, const asdsm_opts* opts, void* stream, asdsm_handle** out);

/* Replace the iteration options of an existing handle (e.g. precision). */
int asdsm_set_opts(asdsm_handle* h, const asdsm_opts* opts);

/* Autotune the launch shapes of this handle's kernels for one precision
 * (ASDSM_FP64 or ASDSM_MIXED): for every level of the block cyclic reductions
 * of the submesh systems (eq. 2.4) the rows per CTA and the number of CTAs
 * splitting the reduction, and the Filler's kernel (Algorithm 3: the
 * tensor-core kernel for n = 16 on the mixed path, or the block cyclic
 * reduction kernel at 8, 4, 2 or 1 warps per CTA) are timed with CUDA events
 * on the handle's stream and the fastest kept.
 * Not part of the paper's method; the arithmetic of a solve is the same up
 * to the summation order inside the level products.  Synchronises the
 * stream; takes tens of milliseconds.  Returns ASDSM_OK or an error. */
int asdsm_autotune(asdsm_handle* h, int precision);

/* The handle's launch shapes (as chosen by asdsm_autotune, or 0 = built-in)
 * as 130 integers, to save a tuning and apply it to another handle of the
 * same sizes (asdsm_tune_set; n must be 130).  Layout per precision (FP64
 * first): forward and backward levels of the anisotropic pair (2 x 16), of
 * the coarse system (2 x 16), then the Filler.  A level entry is
 * (TM << 8) | KS: TM = 16 or 64 rows per CTA on the FMA pipes with KS = 1, 2,
 * 4 or 8 CTAs per cluster splitting the reduction; TM = 32 the mma.sync
 * tensor-core kernel (KS = 1), TM = 128 the tcgen05 kernel (FP32 only, KS =
 * 1, 2 or 4 CTAs per cluster splitting the reduction); 0 the built-in choice.  The Filler entry is 16 for the tensor-core kernel, 1..8
 * for the block cyclic reduction kernel's warps per CTA, 0 for the default.  get returns the count written
 * (cap >= 130) or ASDSM_ERR_INVALID. */
int asdsm_tune_get(const asdsm_handle* h, int32_t* out, int cap);
/* set checks the entries as asdsm_tune_check does and returns
 * ASDSM_ERR_INVALID, leaving the handle unchanged, when one does not fit. */
int asdsm_tune_set(asdsm_handle* h, const int32_t* in, int n);

/* Check a saved tuning (n = 130 entries, layout as above) against the
 * encoding without a handle or any device work: every level entry 0,
 * (TM << 8) | KS with TM in {16, 64} and KS in {1, 2, 4, 8}, or - FP32 half
 * only - TM = 32 with KS = 1 or TM = 128 with KS in {1, 2, 4}; every Filler
 * entry 0..8, or 16 in the FP32 half.  Returns ASDSM_OK or ASDSM_ERR_INVALID. */
int asdsm_tune_check(const int32_t* in, int n);

/* Algorithm 4 (ASDSM).  The initial guess (Algorithm 1) has FP64 quality in
 * both precisions (see asdsm_initial_guess); the mixed path then runs its
 * sweeps as described above.
 * s: device N*N source term (boundary entries unused).
 * u: device N*N; its boundary ring carries the Dirichlet data g on input and
 * is never written; its interior is overwritten by the solution (or used as
 * the first iterate when opts.skip_initial_guess is set).  stats may be NULL.
 * Returns ASDSM_OK when tol was reached, ASDSM_NOT_CONVERGED or
 * ASDSM_STAGNATED otherwise (u then holds the last iterate), or an error. */
int asdsm_solve(asdsm_handle* h, const double* s, double* u, asdsm_stats* stats);

/* Algorithm 1 with b_cc given (the initial guess u^(0)) as asdsm_solve
 * computes it: in FP64 for ASDSM_FP64; for ASDSM_MIXED with FP32 solves
 * refined to FP64 quality (each submesh system: FP32 block cyclic reduction
 * plus two refinement steps with its FP64 residual; merge in FP64; holes
 * filled in FP32 and refined once).  Same s/u contract as asdsm_solve;
 * writes the interior of u. */
int asdsm_initial_guess(asdsm_handle* h, const double* s, double* u);

/* Fine residual of Algorithm 4: r = b_ff - A_ff u over the interior,
 * b_ff being s plus the Dirichlet lifting of u's boundary ring.  s, u:
 * device N*N.  r: device N*N or NULL; when given, its interior receives r and
 * its boundary ring zeros.  rel_norm (host, may be NULL) receives
 * ||r||_2/||b_ff||_2.  Always computed in FP64. */
int asdsm_residual(asdsm_handle* h, const double* s, const double* u, double* r, double* rel_norm);

/* Direct solve of one family of the linear systems of eq. (2.4) by the
 * library's block cyclic reduction, in the handle's precision (for checking
 * a single step against a reference).  mesh:
 *   0 = A_fc on Omega^{h,H}: in/out hold N_c*N_f values, layout [line j][x]
 *   1 = A_cf on Omega^{H,h}: layout [y][column i]
 *   2 = A_cc on Omega^{H,H}: layout [y][x]
 *   3 = the holes (P A P^T of Algorithm 3): in/out are N*N grids; only hole
 *       points are read and written (others are left untouched in out).
 *   4 = Algorithm 3 with zero source (the form every sweep uses): out's hole
 *       points receive the hole solutions whose Dirichlet data are in's
 *       skeleton values (in: N*N grid, only skeleton points read); other
 *       points of out are left untouched.  For n = 16 on the mixed path this
 *       is the tensor-core Filler unless the tuned state selects the block
 *       cyclic reduction kernel.
 * in/out: device FP64 arrays; they may not alias.
 * For a 3D handle: mesh 0..2 = the plane family coarse in x, y, z, arrays
 * [k][q][p] (k the coarse plane, (p, q) the two other axes in increasing
 * order, p fastest); 3..5 = the line family fine in x, y, z, arrays
 * [f][cq][cp] (f the fine coordinate, cp/cq the coarse coordinates of the
 * other two axes); 6 = the coarse mesh [cz][cy][cx]; 7 = the cube holes:
 * N^3 grids, only hole points read and written; 8 = Algorithm 3 with zero
 * source as the sweeps apply it (in: N^3 grid whose skeleton values are the
 * Dirichlet data; out: its hole points receive the fill; on the mixed path
 * this is the FP32 product with the hole extension operator). */
int asdsm_submesh_solve(asdsm_handle* h, int mesh, const double* in, double* out);

/* Relative residual after each completed sweep of the last asdsm_solve
 * (entry 0: initial iterate).  Copies min(cap, sweeps+1) values to the host
 * array hist and returns that count (or a negative error). */
int asdsm_history(asdsm_handle* h, double* hist, int cap);

/* The hole extension operator of Algorithm 3 with zero source, as the
 * tensor-core Filler applies it (host FP64, no device work, no handle):
 * for the problem (N, mc, alpha, beta as in asdsm_desc) and holes of
 * C = (N-1)/mc - 1 points per side, G is (C*C) x (4C), row-major, with
 *   hole values (row by row: y = 1..C, x = 1..C) = G * ring values,
 * the ring ordered west (y = 1..C), east (y = 1..C), south (x = 1..C),
 * north (x = 1..C); G = -A_hh^-1 A_hs for the 5-point stencil of Section 2.3.
 * G: host array of C*C*4*C doubles.  Returns ASDSM_OK or ASDSM_ERR_INVALID
 * (sizes as asdsm_setup requires, alpha/beta/G non-null). */
int asdsm_hole_extension_operator(int N, int mc, const double* alpha, const double* beta, double* G);

/* The same for the cube holes of the 3D extension (host FP64, no device work):
 * alpha, beta per axis (x, y, z), C = (N-1)/mc - 1; G is (C^3) x (6 C^2),
 * row-major, with hole values (x fastest, then y, then z) = G * face values,
 * the faces ordered west (x = 0), east (x = C+1), south (y = 0), north
 * (y = C+1), down (z = 0), up (z = C+1), each face's C*C values with its
 * second axis slowest (west/east: y fastest, z; south/north: x, z; down/up:
 * x, y); G = -A_hh^-1 A_hs for the 7-point stencil.  G: host array of
 * C^3 * 6 C^2 doubles.  Returns ASDSM_OK or ASDSM_ERR_INVALID. */
int asdsm_hole_extension_operator_3d(int N, int mc, const double* alpha, const double* beta, double* G);

/* Turn per-kernel-family CUDA-event timing on (1) or off (0) and clear the
 * accumulated counters.  Timing adds two event records per kernel group. */
int asdsm_profile(asdsm_handle* h, int enable);

/* Copy up to cap family records (see asdsm_kprof) to the host array out;
 * returns the number of families or a negative error. */
int asdsm_profile_read(asdsm_handle* h, asdsm_kprof* out, int cap);

/* Real Schur form of an upper Hessenberg n x n matrix A (host FP64, no
 * device work, no handle): A = Q T Q^T with Q orthogonal and T quasi upper
 * triangular, 2 x 2 diagonal blocks only for complex conjugate eigenvalue
 * pairs.  The 3D extension (Section 3.5) uses it on the coarse-axis operator
 * of each plane family: in the basis of Q a plane system becomes a block
 * back-substitution of shifted 2D fine-plane systems.  A, Q, T: host n*n
 * row-major arrays (1 <= n <= 512).  Returns ASDSM_OK, or ASDSM_ERR_INVALID
 * for bad arguments or if the QR iteration does not converge. */
int asdsm_real_schur(int n, const double* A, double* Q, double* T);

/* The tail of the block cyclic reduction that solves the anisotropic
 * systems of eq. (2.4) (host FP64, no device work, no handle), as the FP32
 * solves apply it.  The system is
 *   a x_{i-1} + (d I + T) x_i + c x_{i+1} = f_i,  i = 1..R,  x_0 = x_{R+1} = 0,
 * with x_i, f_i vectors of C values and T = tridiag(tl, td, tu) (C x C);
 * coef = {a, d, c, tl, td, tu}; R = 2^L - 1.  For rt = 2^t - 1 <= R the last
 * t levels of the reduction involve only the rt rows i = k (R+1)/(rt+1),
 * k = 1..rt, and map their reduced right-hand sides to their solutions
 * linearly; D receives that map, (rt C) x (rt C) row-major, entry
 * ((k-1) C + c, (k'-1) C + c') from row k', component c' of the input to
 * row k, component c of the output.  For a right-hand side that vanishes
 * off those rows the reduced right-hand sides are f itself, so D is then
 * the restriction of the system's inverse to them.  D: host array of
 * (rt C)^2 doubles.  Returns ASDSM_OK, or ASDSM_ERR_INVALID for sizes that
 * break these rules (1 <= C <= 512, R <= 32767, rt C <= 8192) or a system the
 * reduction cannot factor. */
int asdsm_bcr_tail_map(int R, int C, const double* coef, int rt, double* D);

/* Failure-path self-test of the tensor-core kernels (no counterpart in the
 * paper): on the handle's stream, one CTA takes tensor memory as the
 * tcgen05 kernels do and waits on an mbarrier that nothing arrives at, with
 * no copy or MMA in flight.  Its wait gives up after limit_ns (0 < limit_ns
 * <= 2e9), it frees its tensor memory and sets the handle's timeout flag, so
 * the call returns ASDSM_ERR_CUDA ("a wait timed out") - the status a solve
 * returns when a tensor-core kernel stalls.  The flag is sticky: later solves
 * on this handle return ASDSM_ERR_CUDA as well; destroy the handle.  The GPU
 * context stays usable. */
int asdsm_selftest_wait_timeout(asdsm_handle* h, long long limit_ns);

/* Kernels launched by this library in this process so far. */
int64_t asdsm_launch_count(void);

/* Fine residual and relative residual norm WITHOUT ANY DEVICE ALLOCATION.
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc when they need the residual - services whose device memory is
 * reserved up front by their own pool allocator, loops where an allocation
 * would stall or synchronise the device.  It needs no handle (creating one
 * allocates).
 * desc: only d, n, alpha and beta are read.  d = 2: N*N grids, 3 <= N <= 8193,
 * the 5-point operator of Section 2.3.  d = 3: N*N*N grids (z slowest, x
 * fastest), 3 <= N <= 2049, the 7-point operator of the 3D extension (alpha,
 * beta per axis x, y, z).
 * s, u: device FP64 grids as for asdsm_residual (u's boundary = g).
 * r: device grid or NULL; its interior receives r = b_ff - A_ff u (the
 * boundary is not written).  rel_norm: host pointer or NULL; receives ||r||/||b_ff||
 * (the call then copies the two norms to the host and synchronises `stream`;
 * with NULL it only enqueues work).  stream: cudaStream_t or NULL.
 * Scratch: statically allocated device arrays of about 1 MiB held by every
 * GPU that loads the library until the process exits.  The first call on a
 * device looks up their device address (cudaGetSymbolAddress) with that
 * device current, so make that first call before any stream capture.  All
 * calls share the scratch; each call rewrites every slot it reads, so nothing
 * carries over, but calls that overlap on the GPU race.  Grids beyond the
 * scratch's size - N > 8193 for d = 2, N > 2049 for d = 3 - return
 * ASDSM_ERR_INVALID before any device work (message in
 * asdsm_noalloc_last_error). */
int asdsm_residual_noalloc(const asdsm_desc* desc, const double* s, const double* u, double* r,
                           double* rel_norm, void* stream);

/* Text of the last error of asdsm_residual_noalloc on this thread ("" if none). */
const char* asdsm_noalloc_last_error(void);

/* Release every device and host resource of the handle (NULL is a no-op). */
void asdsm_destroy(asdsm_handle* h);

/* ---- Batches of independent problems (instances of uneven sizes) ----------
 * Not in the paper: a throughput interface for many problems of eq. (1.1) at
 * once.  Each instance is a full handle (its own factors, work space and
 * sweep graph) on its own internal CUDA stream; asdsm_solve_batch advances
 * all instances stage by stage in turn (their initial guesses, then their
 * graph replays of kSweepsPerGraph sweeps, the host never waiting on one
 * instance while another can be launched), so their kernels overlap on the
 * GPU.  Every instance's arithmetic is exactly that of asdsm_solve on the
 * same inputs. */
typedef struct asdsm_batch asdsm_batch;

/* descs[count]: one description per instance (eq. 2.1 as for asdsm_setup);
 * opts: shared by all instances (NULL = defaults).  stream: the caller's
 * stream; solves are ordered after the work already queued on it and the
 * stream waits for their end.  *out is NULL on error. */
int asdsm_setup_batch(const asdsm_desc* descs, int count, const asdsm_opts* opts, void* stream,
                      asdsm_batch** out);

/* Instances in the batch. */
int asdsm_batch_count(const asdsm_batch* b);

/* Replace the options of every instance. */
int asdsm_set_opts_batch(asdsm_batch* b, const asdsm_opts* opts);

/* asdsm_autotune for every size class (N, mc) of the batch: one instance per
 * class is tuned and the others take its shapes. */
int asdsm_autotune_batch(asdsm_batch* b, int precision);

/* Algorithm 4 for every instance.  s[i], u[i]: device arrays as for
 * asdsm_solve (instance i's N*N).  stats: NULL or count entries; an instance
 * that fails gets its error code in stats[i].status.  Returns ASDSM_OK when
 * every instance reached tol, else the first non-OK status in instance
 * order. */
int asdsm_solve_batch(asdsm_batch* b, const double* const* s, double* const* u, asdsm_stats* stats);

/* Residual history of instance `index` (as asdsm_history). */
int asdsm_batch_history(const asdsm_batch* b, int index, double* hist, int cap);

/* Release the batch and all its instances (NULL is a no-op). */
void asdsm_destroy_batch(asdsm_batch* b);

/* ---- Learned correction network (not in the paper) -------------------------
 * A 4-layer convolutional net, channels 6 -> 32 -> 32 -> 32 -> 1 with 3x3
 * kernels (cross-correlation, zero padding) and ReLU after layers 1..3, with
 * its own forward, backpropagation (half-MSE loss) and Adam kernels.  Images
 * are device FP32 arrays in NCHW order.  Parameters are one flat FP32 vector
 * [W1, b1, W2, b2, W3, b3, W4, b4], W_l of shape (C_out, C_in, 3, 3).  With
 * bf16_operands the factors of every product are rounded to BF16 (FP32
 * accumulation); otherwise the arithmetic is FP32. */
typedef struct asdsm_cnn asdsm_cnn;

/* Parameter count (20545). */
int asdsm_cnn_param_count(void);
/* Create from host parameters (n = asdsm_cnn_param_count()). */
int asdsm_cnn_create(const float* params, int n, int bf16_operands, asdsm_cnn** out);
int asdsm_cnn_get_params(const asdsm_cnn* net, float* params, int n);
/* Replace the parameters; resets the Adam moments. */
int asdsm_cnn_set_params(asdsm_cnn* net, const float* params, int n);
/* y (B,1,H,W) = net(x (B,6,H,W)).  Stream-ordered. */
int asdsm_cnn_forward(asdsm_cnn* net, const float* x, float* y, int B, int H, int W, void* stream);
/* Forward, loss L = sum w (y - t)^2 / (2 B H W) (w: optional per-pixel
 * weights (B,1,H,W), 1 when NULL) and its gradient, kept on the device for
 * asdsm_cnn_adam; loss and grad_host (param_count floats) are filled when
 * non-NULL (the call then synchronises the stream). */
int asdsm_cnn_backward(asdsm_cnn* net, const float* x, const float* t, const float* weights, int B, int H, int W,
                       double* loss, float* grad_host, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradient. */
int asdsm_cnn_adam(asdsm_cnn* net, float lr, void* stream);
const char* asdsm_cnn_last_error(void);
void asdsm_cnn_destroy(asdsm_cnn* net);

/* Use `net` (NULL: none) as a learned correction in the handle's mixed-
 * precision solves: every sweep, after the ASDSM correction e of Algorithm 4
 * (Algorithm 1 on the residual), the network maps [r, e (each scaled to unit RMS over the interior),
 * alpha_x, alpha_y, beta_x h, beta_y h] to a direction; its skeleton values,
 * completed by the homogeneous Filler (Algorithm 3), enter the same GCR(m)
 * cycle as a second direction (least squares over [e, e_cnn]); a dependent
 * direction is dropped, so the plain correction is the fallback.  Needs
 * accel_m > 1; solves with a network run host-driven sweeps.  The handle does
 * not own `net`. */
int asdsm_attach_cnn(asdsm_handle* h, asdsm_cnn* net);
/* Learned directions accepted by the GCR steps of the last solve. */
int asdsm_cnn_directions(const asdsm_handle* h);
/* Training features of an iterate: r_out = s - A u (the fine residual of Algorithm 4)
 * and e_out = the correction of Algorithm 4 (Algorithm 1 without b_cc, choice
 * of sweep k), both FP32 N*N device grids (computed in FP64). */
int asdsm_correction(asdsm_handle* h, const double* s, const double* u, float* r_out, float* e_out, int k);

/* Static description of a status code. */
const char* asdsm_strerror(int code);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char* asdsm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ASDSM_H */
