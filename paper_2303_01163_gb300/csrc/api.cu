// C ABI of the ASDSM library (include/asdsm.h) and the host orchestration of
// Algorithm 4 on one GPU stream.
//
// Per sweep (all on the handle's stream):
//   residual kernel  : the previous sweep's update fused with the fine residual
//                      (u += sum_j delta_j z_j ; r = b - A u ; r on the skeleton
//                      gathered for the submesh right-hand sides and the least squares)
//   bcr_solve        : the anisotropic solves of Algorithm 1 (both families in one batch)
//   multi_dot        : norms of the normalisation of Algorithm 1
//   merge_knots/write: Algorithm 2 (random choice, spline correction, merge)
//   fill_holes       : Algorithm 3 with 0 b
//   skeleton_apply   : A e on the skeleton rows (least squares of the step length)
//   multi_dot        : the least-squares / GCR(m) inner products
// The host reads two small reductions per sweep (the residual norms and the
// least-squares inner products) and keeps the m x m GCR bookkeeping.
#include "asdsm.h"
#include "asdsm_internal.h"
#include <cuda_runtime.h>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <string>
#include <vector>
#include <algorithm>
#include <functional>
#include "solve3d.h"

using namespace asdsm;

namespace {

thread_local std::string g_last_error;

constexpr int kMaxM = 16;

struct DevBcr {
    void* Mt = nullptr; void* Bt = nullptr;
    void* Mw = nullptr; void* Bw = nullptr;      // FP32: wide tensor-core layout (BcrSys)
    int KW = 0, CW = 0;
    void* Ti = nullptr;                          // FP32: tcgen05 level kernel image (BcrSys)
    int TKC = 0, TCB = 0;
    int* tc_err = nullptr;
    void* Dt = nullptr;                          // FP32: the dense tail map (BcrSys::Dt)
    int tail_rt = 0, tail_ld = 0;
    double wl[kMaxLevels] = {}, wr[kMaxLevels] = {};
    int R = 0, C = 0, L = 0;
    BcrCoefs k{};                                // the system itself (refinement residuals)
};

uint64_t splitmix64_out(uint64_t state) {
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// Coin of the random choice of Algorithm 2 at sweep k: top bit of SplitMix64 output k.
int choice_bit(uint64_t seed, int k) {
    const uint64_t state = seed + (uint64_t)(k + 1) * 0x9E3779B97F4A7C15ULL;
    return (int)(splitmix64_out(state) >> 63);
}

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

struct asdsm_handle {
    asdsm_desc desc{};
    asdsm::Solver3D* s3 = nullptr;   // d = 3: the 3D extension's solver; the 2D members stay unused
    asdsm_opts opts{};
    cudaStream_t st = nullptr;
    int num_sms = 152;
    Geometry g{};
    Stencil sten{};
    double alpha[2]{}, beta[2]{};
    // Factors: [0] = FP64, [1] = FP32.
    DevBcr fc[2], cf[2], cc[2], hole[2];
    void* Sm[2] = {nullptr, nullptr};
    // Work buffers, per precision (allocated on first use).
    struct Work {
        bool ready = false;
        void* Xfc = nullptr; void* Xcf = nullptr; void* Yfc = nullptr; void* Ycf = nullptr;
        void* Xcc = nullptr; void* Ycc = nullptr;
        void* E1 = nullptr; void* E2 = nullptr; void* M1 = nullptr; void* M2 = nullptr;
        void* z[kMaxM] = {};
        int nz = 0;
        void* rskel = nullptr; void* q = nullptr;
        void* qp[kMaxM] = {};
        void* rfull = nullptr;   // full-grid residual for hole corrections
        void* zv = nullptr;      // FP32 with the tensor-core Filler: line values [N][mc+1] (MergeArgs::zv)
    } w[2];
    double* u_work = nullptr;       // FP64 ping-pong partner of the caller's u
    long long* U[2] = {nullptr, nullptr};
    float* s_hi = nullptr; float* s_lo = nullptr;
    double* partials = nullptr;     // reduction scratch
    int partials_cap = 0;
    double* dsmall = nullptr;       // small device results (norms, dots)
    int* dflag = nullptr;
    double* hsmall = nullptr;       // pinned host mirror of dsmall
    std::vector<double> hist;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, evA = nullptr;
    // Per-kernel-family profiling (asdsm_profile).
    bool prof = false;
    asdsm_kprof pc[8] = {};
    struct PendingEv { int a, b, cat; long long launches; double bytes, flops; };
    std::vector<cudaEvent_t> evpool;
    int evnext = 0;
    std::vector<PendingEv> pend_ev;
    // Device-driven sweeps (opts.sweep_graph): control block, residual history,
    // capture streams and the instantiated graph of kSweepsPerGraph sweeps.
    SweepCtl* dctl = nullptr;
    SweepCtl* hctl = nullptr;          // pinned
    double* dhist = nullptr;
    int hist_cap = 0;
    int* hdone = nullptr;              // pinned [2]: done flags read between graph launches
    cudaEvent_t evc[2] = {nullptr, nullptr};
    cudaStream_t cap_st = nullptr, body_st = nullptr;
    // Launch shapes (asdsm_autotune): BCR levels of the anisotropic pair and of
    // A_cc, and warps per CTA of the Filler, per precision.
    BcrTune tune_aniso[2] = {}, tune_cc[2] = {};
    int fill_warps[2] = {0, 0};
    // Tensor-core Filler (holes of 15 x 15): the swizzled image of the hole
    // extension operator G and the kernel's timeout flag.
    float* fill_tc_img = nullptr;
    int* dtcerr = nullptr;
    // Learned correction (asdsm_attach_cnn): the network and its input/output grids.
    asdsm_cnn* cnn = nullptr;
    float* cnn_x = nullptr;            // 6 x N x N
    float* cnn_y = nullptr;            // N x N
    int cnn_dirs = 0;                  // learned directions used in the last solve
    struct SweepGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        int prec = -1, m = 0, S = 0;
        const void* s = nullptr; const void* u = nullptr; const void* partials = nullptr;
        long long top_launches = 0;            // kernels per sweep outside the switch node
        long long body_launches[20] = {};      // kernels of each switch body
    } gr;
};

namespace {

int set_cuda_error(cudaError_t e) {
    g_last_error = cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ASDSM_ERR_OOM : ASDSM_ERR_CUDA;
}

#define CK(...)                                         \
    do {                                                \
        cudaError_t e__ = (__VA_ARGS__);                \
        if (e__ != cudaSuccess) return set_cuda_error(e__); \
    } while (0)

// Section 2.3 stencil of A_ff on the fine spacing hh.
Stencil stencil_of(double ax, double ay, double bx, double by, double hh) {
    Stencil s;
    s.cc = 2 * ax / (hh * hh) + 2 * ay / (hh * hh);
    s.cw = -ax / (hh * hh) - bx / (2 * hh);
    s.ce = -ax / (hh * hh) + bx / (2 * hh);
    s.cs = -ay / (hh * hh) - by / (2 * hh);
    s.cn = -ay / (hh * hh) + by / (2 * hh);
    return s;
}

template <typename T>
int upload_bcr(const BcrFactors& f, DevBcr* d) {
    const size_t n = f.Mt.size();
    std::vector<T> tmp(n);
    void** dst[2] = {&d->Mt, &d->Bt};
    const std::vector<double>* src[2] = {&f.Mt, &f.Bt};
    for (int q = 0; q < 2; ++q) {
        CK(cudaMalloc(dst[q], n * sizeof(T)));
        for (size_t e = 0; e < n; ++e) tmp[e] = (T)(*src[q])[e];
        CK(cudaMemcpy(*dst[q], tmp.data(), n * sizeof(T), cudaMemcpyHostToDevice));
    }
    for (int l = 0; l < f.L; ++l) { d->wl[l] = f.wl[l]; d->wr[l] = f.wr[l]; }
    d->R = f.R; d->C = f.C; d->L = f.L;
    if (sizeof(T) == 4) {
        // Padded, chunk-swizzled copies for the wide tensor-core level kernel.
        const int C = f.C, KW = (C + 31) / 32 * 32, CW = (C + 255) / 256 * 256;
        std::vector<float> wide((size_t)f.L * KW * CW);
        void** wdst[2] = {&d->Mw, &d->Bw};
        for (int q = 0; q < 2; ++q) {
            std::fill(wide.begin(), wide.end(), 0.0f);
            for (int l = 0; l < f.L; ++l)
                for (int k = 0; k < C; ++k)
                    for (int c = 0; c < C; ++c) {
                        const int pos = (((c >> 2) ^ (2 * (k & 3))) << 2) | (c & 3);
                        wide[((size_t)l * KW + k) * CW + pos] = (float)(*src[q])[((size_t)l * C + k) * C + c];
                    }
            CK(cudaMalloc(wdst[q], wide.size() * sizeof(float)));
            CK(cudaMemcpy(*wdst[q], wide.data(), wide.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
        d->KW = KW; d->CW = CW;
    }
    return ASDSM_OK;
}

template <typename T>
int upload_vec(const std::vector<double>& v, void** d) {
    std::vector<T> tmp(v.begin(), v.end());
    CK(cudaMalloc(d, std::max<size_t>(1, tmp.size()) * sizeof(T)));
    if (!tmp.empty()) CK(cudaMemcpy(*d, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    return ASDSM_OK;
}

template <typename T>
BcrSys<T> sys_of(const DevBcr& d, void* X, void* Y, int nsys = 1) {
    BcrSys<T> s{};
    s.X = (T*)X; s.Y = (T*)Y;
    s.Mt = (const T*)d.Mt; s.Bt = (const T*)d.Bt;
    for (int l = 0; l < d.L; ++l) { s.wl[l] = (T)d.wl[l]; s.wr[l] = (T)d.wr[l]; }
    s.R = d.R; s.C = d.C; s.L = d.L; s.nsys = nsys;
    s.stride = (long long)d.R * d.C;
    s.Mw = (const float*)d.Mw; s.Bw = (const float*)d.Bw;
    s.KW = d.KW; s.CW = d.CW;
    s.Ti = (const float*)d.Ti; s.TKC = d.TKC; s.TCB = d.TCB; s.tc_err = d.tc_err;
    s.Dt = (const float*)d.Dt; s.tail_rt = d.tail_rt; s.tail_ld = d.tail_ld;
    return s;
}

// The last levels of the FP32 anisotropic solves as one dense map
// (bcr_tail_map): kTailRows rows are left after the forward levels 0..L-4,
// and levels L-3..L-1 of both directions become one product with a
// (7 C) x (7 C) matrix (12.7 MB at C = 255) in place of five launches.
// Systems with fewer than kTailMinC coarse lines keep every level: their
// sweeps are short, and the changed rounding moved a slowly converging
// 65 x 65 instance with mc = 2 from convergence to the stagnation test.
constexpr int kTailRows = 7, kTailMinC = 31;
int upload_tail(const BcrFactors& f, DevBcr* d) {
    if (f.L < 4 || f.C < kTailMinC) return ASDSM_OK;
    std::vector<double> D;
    if (!bcr_tail_map(f, kTailRows, &D)) return ASDSM_OK;      // not finite in FP64: every level runs
    const int n = kTailRows * f.C, ld = (n + 3) / 4 * 4;
    std::vector<float> img((size_t)n * ld, 0.0f);
    for (int r = 0; r < n; ++r)
        for (int q = 0; q < n; ++q) img[(size_t)r * ld + q] = (float)D[(size_t)r * n + q];
    CK(cudaMalloc(&d->Dt, img.size() * sizeof(float)));
    CK(cudaMemcpy(d->Dt, img.data(), img.size() * sizeof(float), cudaMemcpyHostToDevice));
    d->tail_rt = kTailRows;
    d->tail_ld = ld;
    return ASDSM_OK;
}

// Hole factors (and the tuned CTA shape) into a FillArgs.
template <typename T>
void hole_factors(const asdsm_handle* h, int pi, FillArgs<T>* fa) {
    const DevBcr& d = h->hole[pi];
    fa->Mt = (const T*)d.Mt; fa->Bt = (const T*)d.Bt;
    for (int l = 0; l < d.L; ++l) { fa->wl[l] = (T)d.wl[l]; fa->wr[l] = (T)d.wr[l]; }
    fa->L = d.L;
    fa->warps = h->fill_warps[pi];
}

// Factor images of the tcgen05 level kernel for the FP32 systems (A_fc, A_cf,
// A_cc), built on first need from the FP64 factors on the device: when the
// autotuner considers the kernel, or a tune state selects it.
int ensure_tc_images(asdsm_handle* h) {
    DevBcr* fam[3][2] = {{&h->fc[0], &h->fc[1]}, {&h->cf[0], &h->cf[1]}, {&h->cc[0], &h->cc[1]}};
    for (auto& pr : fam) {
        const DevBcr& d64 = *pr[0];
        DevBcr& d32 = *pr[1];
        if (d32.Ti) continue;
        BcrFactors f;
        f.R = d64.R; f.C = d64.C; f.L = d64.L;
        const size_t n = (size_t)d64.L * d64.C * d64.C;
        f.Mt.resize(n);
        f.Bt.resize(n);
        CK(cudaMemcpy(f.Mt.data(), d64.Mt, n * sizeof(double), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(f.Bt.data(), d64.Bt, n * sizeof(double), cudaMemcpyDeviceToHost));
        std::vector<float> img;
        bcr_tc_image(f, &img, &d32.TKC, &d32.TCB);
        CK(cudaMalloc(&d32.Ti, img.size() * sizeof(float)));
        CK(cudaMemcpy(d32.Ti, img.data(), img.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    return ASDSM_OK;
}

bool tune_wants_tc(const BcrTune& t) {
    for (int d = 0; d < 2; ++d)
        for (int l = 0; l < kMaxLevels; ++l)
            if ((t.cfg[d][l] >> 8) == 128) return true;
    return false;
}

// The Filler's kernel for precision pi: fill_warps[pi] == kFillTcCode selects
// the tensor-core kernel, 1..8 the warps per CTA of the block cyclic reduction
// kernel, 0 the default (the tensor-core kernel where it applies).
constexpr int kFillTcCode = 16;
bool use_fill_tc(const asdsm_handle* h, int pi) {
    return pi == 1 && h->fill_tc_img && (h->fill_warps[1] == 0 || h->fill_warps[1] == kFillTcCode);
}

// Algorithm 3 with zero source on the direction z (in place): the hole values
// of z from its skeleton values.
// zv: the line values merge_write stored apart (MergeArgs::zv), or null.
template <typename T>
cudaError_t fill_homogeneous(const asdsm_handle* h, int pi, T* z, cudaStream_t st, const T* zv = nullptr) {
    if constexpr (sizeof(T) == 4) {
        if (use_fill_tc(h, pi)) {
            FillTcArgs ta{h->fill_tc_img, z, nullptr, zv, h->g.N, h->g.mc, h->dtcerr};
            return fill_tc(ta, h->num_sms, st);
        }
    }
    FillArgs<T> fa{};
    fa.mode = FILL_HOMOGENEOUS;
    fa.z = z; fa.out = z;
    hole_factors<T>(h, pi, &fa);
    fa.n = h->g.n; fa.g = h->g; fa.sten = h->sten;
    return fill_holes<T>(fa, h->num_sms, st);
}

template <typename T>
int ensure_work(asdsm_handle* h, int pi, int slots = -1) {
    auto& w = h->w[pi];
    const Geometry& g = h->g;
    const int m = slots > 0 ? slots : std::max(1, std::min(h->opts.accel_m, kMaxM));
    if (!w.ready) {
        const size_t aniso = (size_t)g.Nf * g.Nc * sizeof(T);
        const size_t coarse = (size_t)g.Nc * g.Nc * sizeof(T);
        CK(cudaMalloc(&w.Xfc, aniso)); CK(cudaMalloc(&w.Xcf, aniso));
        CK(cudaMalloc(&w.Yfc, aniso)); CK(cudaMalloc(&w.Ycf, aniso));
        CK(cudaMalloc(&w.Xcc, coarse)); CK(cudaMalloc(&w.Ycc, coarse));
        CK(cudaMalloc(&w.E1, coarse)); CK(cudaMalloc(&w.E2, coarse));
        const size_t mom = (size_t)g.Nc * (g.mc + 1) * sizeof(T);
        CK(cudaMalloc(&w.M1, mom)); CK(cudaMalloc(&w.M2, mom));
        CK(cudaMalloc(&w.rskel, (size_t)g.skel * sizeof(T)));
        CK(cudaMalloc(&w.q, (size_t)g.skel * sizeof(T)));
        CK(cudaMalloc(&w.rfull, (size_t)g.N * g.N * sizeof(T)));
        CK(cudaMemsetAsync(w.rfull, 0, (size_t)g.N * g.N * sizeof(T), h->st));
        if (sizeof(T) == 4 && h->fill_tc_img) {
            const size_t zvb = (size_t)g.N * (g.mc + 1) * sizeof(float);
            CK(cudaMalloc(&w.zv, zvb));
            CK(cudaMemsetAsync(w.zv, 0, zvb, h->st));        // columns 0 and mc (the boundary) stay zero
        }
        w.ready = true;
    }
    while (w.nz < m) {
        const size_t grid = (size_t)g.N * g.N * sizeof(T);
        CK(cudaMalloc(&w.z[w.nz], grid));
        CK(cudaMemsetAsync(w.z[w.nz], 0, grid, h->st));      // ring stays zero for ever
        CK(cudaMalloc(&w.qp[w.nz], (size_t)g.skel * sizeof(T)));
        ++w.nz;
    }
    return ASDSM_OK;
}

int ensure_partials(asdsm_handle* h, int n) {
    if (n <= h->partials_cap) return ASDSM_OK;
    if (h->partials) cudaFree(h->partials);
    CK(cudaMalloc(&h->partials, (size_t)n * sizeof(double)));
    h->partials_cap = n;
    return ASDSM_OK;
}

// The tcgen05 kernels' timeout flag, read after the stream drained.  It is
// sticky: a wait that ran out means the device stopped making progress, and
// every later call on the handle reports it as well.
int tc_status(asdsm_handle* h, cudaStream_t st) {
    int* f = reinterpret_cast<int*>(h->hsmall + 4095);
    *f = 0;
    CK(cudaMemcpyAsync(f, h->dtcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*f) {
        g_last_error = "tensor-core kernel: a wait timed out";
        return ASDSM_ERR_CUDA;
    }
    return ASDSM_OK;
}

// Copy `count` doubles of dsmall to the host and wait.
int read_small(asdsm_handle* h, int count) {
    CK(cudaMemcpyAsync(h->hsmall, h->dsmall, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return ASDSM_OK;
}

// ---------------------------------------------------------------------------
// Profiling: event pairs around kernel groups, resolved after the solve syncs.
// ---------------------------------------------------------------------------
enum ProfCat { PC_RESID = 0, PC_BCR, PC_FILL, PC_MERGE, PC_LSQ, PC_NORM, PC_OTHER, PC_FILL_TC, PC_COUNT };
const char* kProfNames[PC_COUNT] = {"residual", "bcr_aniso", "fill_holes", "merge", "least_squares", "norms", "other",
                                    "fill_tc"};
static_assert(PC_COUNT <= 8, "asdsm_handle::pc holds 8 families");

struct ProfMark { int ev = -1; long long l0 = 0; };

ProfMark prof_begin(asdsm_handle* h) {
    ProfMark m;
    m.l0 = launch_count();
    if (!h->prof) return m;
    if (h->evnext + 2 > (int)h->evpool.size()) {
        for (int q = 0; q < 64; ++q) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return m;
            h->evpool.push_back(e);
        }
    }
    m.ev = h->evnext;
    h->evnext += 2;
    cudaEventRecord(h->evpool[m.ev], h->st);
    return m;
}

void prof_end(asdsm_handle* h, const ProfMark& m, int cat, double bytes, double flops) {
    if (!h->prof || m.ev < 0) return;
    cudaEventRecord(h->evpool[m.ev + 1], h->st);
    h->pend_ev.push_back({m.ev, m.ev + 1, cat, launch_count() - m.l0, bytes, flops});
}

// After a stream synchronisation: fold the recorded pairs into the counters.
void prof_resolve(asdsm_handle* h) {
    for (const auto& p : h->pend_ev) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->evpool[p.a], h->evpool[p.b]) != cudaSuccess) continue;
        asdsm_kprof& c = h->pc[p.cat];
        c.ms += ms;
        c.calls += 1;
        c.launches += p.launches;
        c.bytes += p.bytes;
        c.flops += p.flops;
    }
    h->pend_ev.clear();
    h->evnext = 0;
}

// Multiply-adds of block cyclic reduction for R = 2^L - 1 rows of C unknowns
// (forward: two C x C products per reduced row; backward: B^{-1} f plus one
// product per existing neighbour).
double bcr_macs(int R, int C, int L) {
    const double c2 = (double)C * C;
    double macs = 0.0;
    for (int l = 0; l + 1 < L; ++l) macs += (double)(((R + 1) >> (l + 1)) - 1) * 2.0 * c2;
    for (int l = 0; l < L; ++l) {
        const double rb = (double)((R + 1) >> (l + 1));
        macs += rb * c2 + 2.0 * (rb - 1.0) * c2;
    }
    return macs;
}

// ||b_ff||^2 via the FP64 residual of the zero-interior grid (r = b there).
int bnorm2(asdsm_handle* h, const double* s, const double* u, double* out) {
    const Geometry& g = h->g;
    CK(ring_from<double>(u, h->u_work, g, 1, h->st));
    int nb = 0;
    const int need = std::max(2 * residual_grid_blocks(g), kDotPartials);
    if (int rc = ensure_partials(h, need)) return rc;
    ResidOut o{};
    o.partials = h->partials;
    UpdateTerms up{};
    CK(residual_fp64(s, h->u_work, h->u_work, up, g, h->sten, o, &nb, h->st));
    CK(reduce_partials(h->partials, nb, 2, h->dsmall, h->st));
    if (int rc = read_small(h, 2)) return rc;
    *out = h->hsmall[0];
    return ASDSM_OK;
}

// Mixed-path residual coefficients: FP32 pairs of the stencil parts times 2^-S
// and times the weights 2^44, 2^22 of the integer pieces.
MixedCoefs mixed_coefs(const asdsm_handle* h, int S) {
    const double hh = 1.0 / h->g.M;
    const double sc = std::ldexp(1.0, -S);
    const double v[4] = {h->alpha[0] / (hh * hh) * sc, h->alpha[1] / (hh * hh) * sc,
                         h->beta[0] / (2 * hh) * sc, h->beta[1] / (2 * hh) * sc};
    MixedCoefs k{};
    for (int q = 0; q < 4; ++q) {
        const double w2 = std::ldexp(v[q], 44), w1 = std::ldexp(v[q], 22);
        k.k2[q][0] = (float)w2;
        k.k2[q][1] = (float)(w2 - (double)k.k2[q][0]);
        k.k1[q][0] = (float)w1;
        k.k1[q][1] = (float)(w1 - (double)k.k1[q][0]);
        k.k0[q] = (float)v[q];
    }
    return k;
}

// ---------------------------------------------------------------------------
// Algorithm 1 (initial guess) into the direction slot z[0] (T), ring = g.
// ---------------------------------------------------------------------------
template <typename T>
int initial_guess_to_z(asdsm_handle* h, const double* s, const double* u) {
    const int pi = sizeof(T) == 8 ? 0 : 1;
    auto& w = h->w[pi];
    const Geometry& g = h->g;
    cudaStream_t st = h->st;
    CK(build_submesh_rhs<T>(s, u, g, h->alpha, h->beta, (T*)w.Xfc, (T*)w.Xcf, (T*)w.Xcc, st));
    BcrSys<T> sys[2] = {sys_of<T>(h->fc[pi], w.Xfc, w.Yfc), sys_of<T>(h->cf[pi], w.Xcf, w.Ycf)};
    CK(bcr_solve<T>(sys, 2, st, &h->tune_aniso[pi]));                                       // u_fc, u_cf
    BcrSys<T> scc = sys_of<T>(h->cc[pi], w.Xcc, w.Ycc);
    CK(bcr_solve<T>(&scc, 1, st, &h->tune_cc[pi]));                                      // u_cc
    T* z = (T*)w.z[0];
    CK(ring_from<T>(u, z, g, 0, st));
    MergeArgs<T> ma{};
    ma.Yfc = (T*)w.Yfc; ma.Ycf = (T*)w.Ycf; ma.Ycc = (T*)w.Ycc;
    ma.norms2 = nullptr; ma.re_mode = 1; ma.choice = 0;
    ma.Sm = (const T*)h->Sm[pi];
    ma.E1 = (T*)w.E1; ma.E2 = (T*)w.E2; ma.M1 = (T*)w.M1; ma.M2 = (T*)w.M2;
    ma.z = z; ma.g = g;
    CK(merge_knots<T>(ma, st));                                         // Algorithm 2: cross-point errors
    CK(merge_write<T>(ma, st));                                         // spline corrections, skeleton
    FillArgs<T> fa{};
    fa.mode = FILL_WITH_SOURCE;
    fa.z = z; fa.out = z;
    if (sizeof(T) == 8) fa.src_d = s; else fa.src_hi = h->s_hi;
    hole_factors<T>(h, pi, &fa);
    fa.n = g.n; fa.g = g; fa.sten = h->sten;
    CK(fill_holes<T>(fa, h->num_sms, st));                              // Algorithm 3 with b_ff
    // Restore the ring of z to zero for later use as a direction slot is done by the caller.
    return ASDSM_OK;
}

// Algorithm 1 for the mixed path, to FP64 quality without FP64 solves: each
// submesh system is solved by FP32 block cyclic reduction with two steps of
// iterative refinement (FP64 residual of the system, FP32 solve of the
// correction), the merge of Algorithm 2 runs in FP64, and the holes are
// filled in FP32 (Algorithm 3 with b_ff) straight into the FP64 grid and
// refined once (FP64 residual, FP32 hole solve of it, added in FP64).
// Result in h->w[0].z[0] (ring = g), as initial_guess_to_z.
int initial_guess_refined(asdsm_handle* h, const double* s, const double* u) {
    if (int rc = ensure_work<double>(h, 0, 1)) return rc;
    auto& w64 = h->w[0];
    auto& w32 = h->w[1];
    const Geometry& g = h->g;
    cudaStream_t st = h->st;
    CK(build_submesh_rhs<double>(s, u, g, h->alpha, h->beta, (double*)w64.Xfc, (double*)w64.Xcf, (double*)w64.Xcc, st));
    struct Fam { const DevBcr* d32; void* b64; void* x64; void* r32; void* y32; int R, C; };
    const Fam fam[3] = {
        {&h->fc[1], w64.Xfc, w64.Yfc, w32.Xfc, w32.Yfc, g.Nf, g.Nc},
        {&h->cf[1], w64.Xcf, w64.Ycf, w32.Xcf, w32.Ycf, g.Nf, g.Nc},
        {&h->cc[1], w64.Xcc, w64.Ycc, w32.Xcc, w32.Ycc, g.Nc, g.Nc}};
    for (const Fam& f : fam) {
        const long long n = (long long)f.R * f.C;
        CK(cudaMemsetAsync(f.x64, 0, n * sizeof(double), st));
        CK(convert_array<double, float>((const double*)f.b64, (float*)f.r32, n, st));
    }
    constexpr int kRefine = 2;
    for (int it = 0; it <= kRefine; ++it) {
        BcrSys<float> pair[2] = {sys_of<float>(h->fc[1], w32.Xfc, w32.Yfc), sys_of<float>(h->cf[1], w32.Xcf, w32.Ycf)};
        CK(bcr_solve<float>(pair, 2, st, &h->tune_aniso[1]));                         // u_fc, u_cf
        BcrSys<float> scc = sys_of<float>(h->cc[1], w32.Xcc, w32.Ycc);
        CK(bcr_solve<float>(&scc, 1, st, &h->tune_cc[1]));                            // u_cc
        for (const Fam& f : fam) {
            CK(add_float((double*)f.x64, (const float*)f.y32, (long long)f.R * f.C, st));
            if (it < kRefine)
                CK(bcr_residual((const double*)f.x64, (const double*)f.b64, (float*)f.r32, f.R, f.C, f.d32->k, st));
        }
    }
    double* z = (double*)w64.z[0];
    CK(ring_from<double>(u, z, g, 0, st));
    MergeArgs<double> ma{};
    ma.Yfc = (double*)w64.Yfc; ma.Ycf = (double*)w64.Ycf; ma.Ycc = (double*)w64.Ycc;
    ma.norms2 = nullptr; ma.re_mode = 1; ma.choice = 0;
    ma.Sm = (const double*)h->Sm[0];
    ma.E1 = (double*)w64.E1; ma.E2 = (double*)w64.E2; ma.M1 = (double*)w64.M1; ma.M2 = (double*)w64.M2;
    ma.z = z; ma.g = g;
    CK(merge_knots<double>(ma, st));                                    // Algorithm 2: cross-point errors
    CK(merge_write<double>(ma, st));                                    // spline corrections, skeleton
    float* z32 = (float*)w32.z[0];
    CK(convert_array<double, float>(z, z32, (long long)g.N * g.N, st)); // skeleton and ring for the FP32 fill
    FillArgs<float> fa{};
    fa.mode = FILL_WITH_SOURCE;
    fa.z = z32; fa.out = z32; fa.out_d = z;
    fa.src_hi = h->s_hi;
    hole_factors<float>(h, 1, &fa);
    fa.n = g.n; fa.g = g; fa.sten = h->sten;
    CK(fill_holes<float>(fa, h->num_sms, st));                          // Algorithm 3 with b_ff
    // One refinement of the holes: FP64 residual, FP32 hole solve of it added in FP64.
    ResidOut o{};
    o.rfull = w64.rfull; o.partials = h->partials;
    UpdateTerms none{};
    int nb = 0;
    CK(residual_fp64(s, z, z, none, g, h->sten, o, &nb, st));
    CK(convert_array<double, float>((const double*)w64.rfull, (float*)w32.rfull, (long long)g.N * g.N, st));
    FillArgs<float> fr{};
    fr.mode = FILL_RESIDUAL_TO_U;
    fr.src_hi = (const float*)w32.rfull;
    fr.u_d = z;
    hole_factors<float>(h, 1, &fr);
    fr.n = g.n; fr.g = g; fr.sten = h->sten;
    CK(fill_holes<float>(fr, h->num_sms, st));
    return ASDSM_OK;
}

// ---------------------------------------------------------------------------
// Device-driven sweeps: one CUDA graph replays kSweepsPerGraph sweeps.  Per
// sweep: the residual kernel (pending update read from the device), the norm
// reduction, the controller, and a switch node whose bodies are the sweep for
// direction slot kc (bodies 0..m-1) and the hole correction of the iterate in
// buffer 0 or 1 (bodies m, m+1); value m+2 runs nothing (solve ended).
// ---------------------------------------------------------------------------
constexpr int kSweepsPerGraph = 8;

void destroy_graph(asdsm_handle* h) {
    if (h->gr.exec) cudaGraphExecDestroy(h->gr.exec);
    if (h->gr.graph) cudaGraphDestroy(h->gr.graph);
    h->gr = asdsm_handle::SweepGraph{};
}

template <typename T>
int enqueue_residual_dyn(asdsm_handle* h, const double* s, double* u, double scale, const MixedCoefs& mk,
                         int m, cudaStream_t st) {
    const int pi = sizeof(T) == 8 ? 0 : 1;
    auto& w = h->w[pi];
    const Geometry& g = h->g;
    ResidOut o{};
    o.rfc = w.Xfc; o.rcf = w.Xcf; o.rskel = w.rskel; o.rfull = nullptr; o.partials = h->partials;
    UpdateTerms up{};
    for (int j = 0; j < m; ++j) up.z[j] = w.z[j];
    up.dyn = &h->dctl->upd;
    int nb = 0;
    if (sizeof(T) == 8) CK(residual_fp64(s, u, h->u_work, up, g, h->sten, o, &nb, st));
    else CK(residual_mixed(h->s_hi, h->s_lo, h->U[0], h->U[1], up, scale, g, mk, o, &nb, h->dflag, st));
    CK(reduce_partials(h->partials, nb, 2, h->dsmall, st));
    return ASDSM_OK;
}

// Hole-residual correction of the iterate in buffer par.
template <typename T>
int enqueue_holefix(asdsm_handle* h, const double* s, double* u, int par, double scale, const MixedCoefs& mk,
                    cudaStream_t st) {
    const int pi = sizeof(T) == 8 ? 0 : 1;
    auto& w = h->w[pi];
    const Geometry& g = h->g;
    ResidOut o{};
    o.rfull = w.rfull; o.partials = h->partials;
    UpdateTerms none{};
    FillArgs<T> fa{};
    fa.mode = FILL_RESIDUAL_TO_U;
    int nb = 0;
    if (sizeof(T) == 8) {
        double* ucur = par ? h->u_work : u;
        CK(residual_fp64(s, ucur, ucur, none, g, h->sten, o, &nb, st));
        fa.src_d = (const double*)w.rfull;
        fa.u_d = ucur;
    } else {
        CK(residual_mixed(h->s_hi, h->s_lo, h->U[par], h->U[par], none, scale, g, mk, o, &nb, h->dflag, st));
        fa.src_hi = (const float*)w.rfull;
        fa.U = h->U[par];
        fa.fixed_scale = scale;
    }
    hole_factors<T>(h, pi, &fa);
    fa.n = g.n; fa.g = g; fa.sten = h->sten;
    CK(fill_holes<T>(fa, h->num_sms, st));
    return ASDSM_OK;
}

// The correction of Algorithm 4 into direction slot kc, then the step lengths.
template <typename T>
int enqueue_sweep_body(asdsm_handle* h, int kc, int m, cudaStream_t st) {
    const int pi = sizeof(T) == 8 ? 0 : 1;
    auto& w = h->w[pi];
    const Geometry& g = h->g;
    BcrSys<T> sys[2] = {sys_of<T>(h->fc[pi], w.Xfc, w.Yfc), sys_of<T>(h->cf[pi], w.Xcf, w.Ycf)};
    CK(bcr_solve<T>(sys, 2, st, &h->tune_aniso[pi]));
    const T* av[2] = {(const T*)w.Yfc, (const T*)w.Ycf};
    int nb2 = 0;
    CK(multi_dot<T>(av, av, 2, (long long)g.Nf * g.Nc, h->partials, &nb2, st));
    CK(reduce_partials(h->partials, nb2, 2, h->dsmall + 200, st));
    T* z = (T*)w.z[kc];
    MergeArgs<T> ma{};
    ma.Yfc = (T*)w.Yfc; ma.Ycf = (T*)w.Ycf; ma.Ycc = nullptr;
    ma.norms2 = h->dsmall + 200; ma.re_mode = 0; ma.choice = 0; ma.choice_dev = &h->dctl->choice;
    ma.Sm = (const T*)h->Sm[pi];
    ma.E1 = (T*)w.E1; ma.E2 = (T*)w.E2; ma.M1 = (T*)w.M1; ma.M2 = (T*)w.M2;
    ma.z = z; ma.g = g;
    ma.zv = use_fill_tc(h, pi) ? (T*)w.zv : nullptr;
    CK(merge_knots<T>(ma, st));
    CK(merge_write<T>(ma, st));
    CK(fill_homogeneous<T>(h, pi, z, st, (const T*)ma.zv));
    CK(skeleton_apply<T>(z, g, h->sten, (T*)w.q, st));
    const T* qpv[kMaxM];
    for (int j = 0; j < kc; ++j) qpv[j] = (const T*)w.qp[j];
    int nb3 = 0;
    CK(gcr_dots<T>((const T*)w.q, (const T*)w.rskel, qpv, kc, g.skel, h->partials, &nb3, st));
    CK(reduce_partials(h->partials, nb3, 2 + 2 * kc, h->dsmall, st));
    CK(ctl_after_dots(h->dctl, h->dsmall, st));
    if (m > 1) {
        CK(combine_skeleton_dyn<T>((const T*)w.q, qpv, kc, &h->dctl->comb, g.skel, (T*)w.qp[kc], st));
        // Inside a deferred cycle: the tracked residual and the next sweep's submesh right-hand sides.
        CK(track_skeleton<T>((T*)w.rskel, (const T*)w.qp[kc], 0.0, &h->dctl->comb, g, (T*)w.Xfc, (T*)w.Xcf, st));
    }
    return ASDSM_OK;
}

// Capture and instantiate the graph for this precision, m, fixed-point shift
// and buffers (rebuilt when any of them changes).
template <typename T>
int ensure_graph(asdsm_handle* h, const double* s, double* u, int m, int S, double scale, const MixedCoefs& mk) {
    const int prec = sizeof(T) == 8 ? ASDSM_FP64 : ASDSM_MIXED;
    auto& G = h->gr;
    const bool fp64 = prec == ASDSM_FP64;
    if (G.exec && G.prec == prec && G.m == m && G.S == S && G.partials == h->partials &&
        (!fp64 || (G.s == s && G.u == u)))
        return ASDSM_OK;
    destroy_graph(h);
    if (!h->cap_st) CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
    if (!h->body_st) CK(cudaStreamCreateWithFlags(&h->body_st, cudaStreamNonBlocking));
    const long long lc0 = launch_count();
    int rc = ASDSM_OK;
    cudaError_t e = cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return set_cuda_error(e);
    for (int i = 0; i < kSweepsPerGraph && rc == ASDSM_OK; ++i) {
        const long long t0 = launch_count();
        if ((rc = enqueue_residual_dyn<T>(h, s, u, scale, mk, m, h->cap_st))) break;
        cudaStreamCaptureStatus cst;
        cudaGraph_t cgraph = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        cudaGraphConditionalHandle hc;
        if ((e = cudaStreamGetCaptureInfo(h->cap_st, &cst, nullptr, &cgraph, &deps, nullptr, &ndeps)) != cudaSuccess ||
            (e = cudaGraphConditionalHandleCreate(&hc, cgraph, (unsigned)(m + 2), cudaGraphCondAssignDefault)) != cudaSuccess ||
            (e = ctl_after_residual(h->dctl, h->dsmall, h->dflag, h->dhist, hc, h->cap_st)) != cudaSuccess ||
            (e = cudaStreamGetCaptureInfo(h->cap_st, &cst, nullptr, &cgraph, &deps, nullptr, &ndeps)) != cudaSuccess) {
            rc = set_cuda_error(e);
            break;
        }
        if (i == 0) G.top_launches = launch_count() - t0;
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = hc;
        np.conditional.type = cudaGraphCondTypeSwitch;
        np.conditional.size = (unsigned)(m + 2);
        cudaGraphNode_t node;
        if ((e = cudaGraphAddNode(&node, cgraph, deps, nullptr, ndeps, &np)) != cudaSuccess ||
            (e = cudaStreamUpdateCaptureDependencies(h->cap_st, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess) {
            rc = set_cuda_error(e);
            break;
        }
        for (int b = 0; b < m + 2 && rc == ASDSM_OK; ++b) {
            if ((e = cudaStreamBeginCaptureToGraph(h->body_st, np.conditional.phGraph_out[b], nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
                rc = set_cuda_error(e);
                break;
            }
            const long long b0 = launch_count();
            rc = b < m ? enqueue_sweep_body<T>(h, b, m, h->body_st)
                       : enqueue_holefix<T>(h, s, u, b - m, scale, mk, h->body_st);
            if (i == 0) G.body_launches[b] = launch_count() - b0;
            cudaGraph_t bg = nullptr;
            e = cudaStreamEndCapture(h->body_st, &bg);
            if (rc == ASDSM_OK && e != cudaSuccess) rc = set_cuda_error(e);
        }
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->cap_st, &graph);
    note_launch(-(launch_count() - lc0));           // captured, not launched
    if (rc != ASDSM_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return set_cuda_error(e); }
    G.graph = graph;
    if ((e = cudaGraphInstantiate(&G.exec, graph, 0)) != cudaSuccess) { destroy_graph(h); return set_cuda_error(e); }
    G.prec = prec; G.m = m; G.S = S; G.s = s; G.u = u; G.partials = h->partials;
    return ASDSM_OK;
}

// State of one solve of Algorithm 4, advanced in stages so that a batch can
// interleave its instances on their streams:
//   begin  : everything up to the first value the host must read (||b||, and
//            max |u^(0)| for the fixed-point scale) is enqueued;
//   middle : after those reads, the fixed-point conversion and the first
//            sweeps are enqueued (or, host-driven, all sweeps are run);
//   poll   : graph launches of kSweepsPerGraph sweeps, two in flight, until
//            the device controller reports the end;
//   finish : the iterate is copied out and the statistics filled.
struct SolveRun {
    const double* s = nullptr;
    double* u = nullptr;
    asdsm_stats* stats = nullptr;
    int stage = 0;                   // 1 begun, 2 sweeps in flight, 3 sweeps ended
    long long launches = 0;
    int nb_max = 0;
    double bnorm = 0.0;
    int S = 0;
    double scale = 1.0;
    MixedCoefs mk{};
    const double* u0d = nullptr;
    double* ucur = nullptr;
    double* unxt = nullptr;
    int Ucur = 0;
    int status = ASDSM_NOT_CONVERGED, k = 0, hole_fixes = 0;
    double rel0 = 0.0, rel = 0.0;
    std::vector<double> rhist;
    int q = 0, max_q = 0, in_flight = 0;
    bool done = false;
    bool resume = false;             // start from u as given (a rescaled restart), whatever the options say
    int S_cap = 1 << 20;             // mixed path: largest fixed-point shift allowed
};

// Device controller set up and the graph made ready; no launch yet.
template <typename T>
int graph_start(asdsm_handle* h, SolveRun& r) {
    const asdsm_opts& op = h->opts;
    const int m = std::max(1, std::min(op.accel_m, kMaxM));
    cudaStream_t st = h->st;
    if (h->hist_cap < op.max_sweeps + 2) {
        if (h->dhist) cudaFree(h->dhist);
        h->dhist = nullptr;
        h->hist_cap = 0;
        CK(cudaMalloc(&h->dhist, (size_t)(op.max_sweeps + 2) * sizeof(double)));
        h->hist_cap = op.max_sweeps + 2;
        destroy_graph(h);                                   // the graph holds the old pointer
    }
    if (int rc = ensure_graph<T>(h, r.s, r.u, m, r.S, r.scale, r.mk)) return rc;
    SweepCtl& c = *h->hctl;
    std::memset(&c, 0, sizeof(c));
    c.bnorm = r.bnorm; c.tol = op.tol; c.hole_fix_ratio = op.hole_fix_ratio; c.hole_fix_growth = op.hole_fix_growth;
    c.stagnation_factor = op.stagnation_factor; c.scale = r.scale; c.seed = op.seed;
    c.max_sweeps = op.max_sweeps; c.window = op.stagnation_window; c.m = m; c.mixed = sizeof(T) == 4;
    c.hist_cap = h->hist_cap;
    c.upd.live = 1;
    c.defer = m > 1 && !h->cnn ? 1 : 0;
    CK(cudaMemcpyAsync(h->dctl, &c, sizeof(c), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->dflag, 0, sizeof(int), st));
    // A bounded number of launches: every replayed sweep advances k, ends a
    // deferred GCR cycle early (at most once per cycle, and a cycle holds at
    // least one sweep that advances k) or finds the solve ended, and
    // k = max_sweeps ends it.
    r.max_q = (2 * op.max_sweeps + 2) / kSweepsPerGraph + 3;
    r.q = 0;
    r.in_flight = 0;
    r.done = false;
    return ASDSM_OK;
}

// Read the controller's final state after the last launch.
template <typename T>
int graph_collect(asdsm_handle* h, SolveRun& r) {
    const int m = std::max(1, std::min(h->opts.accel_m, kMaxM));
    CK(cudaMemcpyAsync(h->hctl, h->dctl, sizeof(SweepCtl), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    const SweepCtl& c = *h->hctl;
    r.rhist.resize((size_t)std::min(c.nhist, c.hist_cap));
    if (!r.rhist.empty())
        CK(cudaMemcpy(r.rhist.data(), h->dhist, r.rhist.size() * sizeof(double), cudaMemcpyDeviceToHost));
    if (!c.done) { g_last_error = "device sweep control did not finish"; return ASDSM_ERR_CUDA; }
    r.status = c.status; r.k = c.k; r.hole_fixes = c.hole_fixes;
    r.rel0 = c.rel0; r.rel = c.rel;
    if (sizeof(T) == 8) { if (c.upd.par) r.ucur = h->u_work; }
    else r.Ucur = c.upd.par;
    // Kernels that ran: every replayed sweep's fixed part plus the bodies the switch nodes chose.
    long long ran = (long long)r.q * kSweepsPerGraph * h->gr.top_launches;
    for (int b = 0; b < m + 2 && b < 20; ++b) ran += (long long)c.runs[b] * h->gr.body_launches[b];
    note_launch(ran);
    r.stage = 3;
    return ASDSM_OK;
}

// Keep two graph launches in flight and retire the oldest once it has
// completed (block: wait for it; otherwise return if it is still running).
template <typename T>
int graph_poll(asdsm_handle* h, SolveRun& r, bool block) {
    cudaStream_t st = h->st;
    while (!r.done && r.in_flight < 2 && r.q < r.max_q) {
        const int slot = r.q & 1;
        CK(cudaGraphLaunch(h->gr.exec, st));
        CK(cudaMemcpyAsync(&h->hdone[slot], &h->dctl->done, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(h->evc[slot], st));
        ++r.q;
        ++r.in_flight;
    }
    if (r.in_flight > 0) {
        const int j = r.q - r.in_flight;
        if (block) {
            CK(cudaEventSynchronize(h->evc[j & 1]));
        } else {
            const cudaError_t e = cudaEventQuery(h->evc[j & 1]);
            if (e == cudaErrorNotReady) return ASDSM_OK;
            if (e != cudaSuccess) return set_cuda_error(e);
        }
        --r.in_flight;
        if (h->hdone[j & 1]) r.done = true;
    }
    if (r.done || (r.q >= r.max_q && r.in_flight == 0)) return graph_collect<T>(h, r);
    return ASDSM_OK;
}

// ---------------------------------------------------------------------------
// Autotuning of launch shapes: every BCR level (rows per CTA x cluster split)
// and the Filler's kernel are timed on the handle's own systems (on scratch
// data, in captured CUDA graphs) and the fastest kept.
// ---------------------------------------------------------------------------
// Device time of one launch() as the solves run it: reps launches captured
// into a CUDA graph (no host launch cost between them, programmatic
// dependent launches as in the sweep graphs), replayed once to warm up and
// once between events.  launch() enqueues on h->st, which points at the
// handle's capture stream meanwhile.
template <typename T>
int time_ms(asdsm_handle* h, cudaEvent_t a, cudaEvent_t b, int reps, float* ms, const std::function<int()>& launch) {
    if (int rc = launch()) return rc;                // warm-up (and function attributes) outside the capture
    if (!h->cap_st) CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
    CK(cudaStreamSynchronize(h->st));
    cudaStream_t user = h->st;
    h->st = h->cap_st;
    cudaGraph_t graph = nullptr;
    int rc = ASDSM_OK;
    cudaError_t e = cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        for (int r = 0; r < reps && rc == ASDSM_OK; ++r) rc = launch();
        e = cudaStreamEndCapture(h->cap_st, &graph);
    }
    h->st = user;
    if (rc != ASDSM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    CK(e);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    auto run = [&]() -> cudaError_t {
        cudaError_t r;
        if ((r = cudaGraphLaunch(exec, h->cap_st)) != cudaSuccess) return r;
        if ((r = cudaEventRecord(a, h->cap_st)) != cudaSuccess) return r;
        if ((r = cudaGraphLaunch(exec, h->cap_st)) != cudaSuccess) return r;
        if ((r = cudaEventRecord(b, h->cap_st)) != cudaSuccess) return r;
        return cudaEventSynchronize(b);
    };
    e = run();
    cudaGraphExecDestroy(exec);
    CK(e);
    CK(cudaEventElapsedTime(ms, a, b));
    *ms /= reps;
    return ASDSM_OK;
}

template <typename T>
int tune_bcr(asdsm_handle* h, const BcrSys<T>* sys, int ngroups, BcrTune* tune, cudaEvent_t a, cudaEvent_t b) {
    const int L = sys[0].L;
    for (int dir = 0; dir < 2; ++dir) {
        for (int l = 0; l < (dir ? L : L - 1); ++l) {
            float best = 1e30f;
            int bestv = 0;
            for (int tm : {64, 16, 32, 128}) {
                if (tm == 32 && (sizeof(T) != 4 || !sys[0].Mw)) continue;
                if (tm == 128 && (sizeof(T) != 4 || !sys[0].Ti)) continue;
                for (int ks : {1, 2, 4, 8}) {
                    if ((tm == 32 && ks != 1) || (tm == 128 && ks == 8)) continue;
                    tune->cfg[dir][l] = (tm << 8) | ks;
                    float ms = 0.f;
                    if (int rc = time_ms<T>(h, a, b, 5, &ms, [&]() -> int {
                            CK(bcr_level<T>(sys, ngroups, l, dir == 1, tune, h->st));
                            return ASDSM_OK;
                        })) return rc;
                    if (std::getenv("ASDSM_TRACE"))
                        std::fprintf(stderr, "asdsm tune: C=%d dir=%d level=%d tm=%d ks=%d  %.2f us\n", sys[0].C, dir, l,
                                     tm, ks, ms * 1e3);
                    // The tcgen05 kernel's time is mostly fixed per launch (pipeline
                    // hand-offs between its warps) and it rounds differently: it
                    // replaces the best other shape only when clearly faster.
                    const float margin = tm == 128 ? 0.9f : 1.0f;
                    if (ms < best * margin) { best = ms; bestv = tune->cfg[dir][l]; }
                }
            }
            tune->cfg[dir][l] = bestv;
            if (std::getenv("ASDSM_TRACE"))
                std::fprintf(stderr, "asdsm tune: C=%d dir=%d level=%d chosen tm=%d ks=%d (%.2f us)\n", sys[0].C, dir, l,
                             bestv >> 8, bestv & 0xFF, best * 1e3);
        }
    }
    return ASDSM_OK;
}

template <typename T>
int autotune_impl(asdsm_handle* h) {
    const int pi = sizeof(T) == 8 ? 0 : 1;
    if (int rc = ensure_work<T>(h, pi, 1)) return rc;
    if (sizeof(T) == 4)
        if (int rc = ensure_tc_images(h)) return rc;
    auto& w = h->w[pi];
    const Geometry& g = h->g;
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    auto done = [&](int rc) { cudaEventDestroy(a); cudaEventDestroy(b); return rc; };
    // Scratch right-hand sides (the tuning overwrites them).
    CK(cudaMemsetAsync(w.Xfc, 0, (size_t)g.Nf * g.Nc * sizeof(T), h->st));
    CK(cudaMemsetAsync(w.Xcf, 0, (size_t)g.Nf * g.Nc * sizeof(T), h->st));
    CK(cudaMemsetAsync(w.Xcc, 0, (size_t)g.Nc * g.Nc * sizeof(T), h->st));
    BcrSys<T> sys[2] = {sys_of<T>(h->fc[pi], w.Xfc, w.Yfc), sys_of<T>(h->cf[pi], w.Xcf, w.Ycf)};
    if (int rc = tune_bcr<T>(h, sys, 2, &h->tune_aniso[pi], a, b)) return done(rc);
    BcrSys<T> scc = sys_of<T>(h->cc[pi], w.Xcc, w.Ycc);
    if (int rc = tune_bcr<T>(h, &scc, 1, &h->tune_cc[pi], a, b)) return done(rc);
    // Filler (homogeneous mode): the tensor-core kernel where it applies, and
    // the block cyclic reduction kernel at 8, 4, 2, 1 warps per CTA.
    float best = 1e30f;
    int bestw = 0;
    for (int wv : {kFillTcCode, 8, 4, 2, 1}) {
        if (wv == kFillTcCode && !(pi == 1 && h->fill_tc_img)) continue;
        h->fill_warps[pi] = wv;
        float ms = 0.f;
        if (int rc = time_ms<T>(h, a, b, 3, &ms, [&]() -> int {
                CK(fill_homogeneous<T>(h, pi, (T*)w.z[0], h->st));
                return ASDSM_OK;
            })) return done(rc);
        if (ms < best) { best = ms; bestw = wv; }
    }
    h->fill_warps[pi] = bestw;
    if (int rc = tc_status(h, h->st)) return done(rc);
    destroy_graph(h);                      // recapture with the new shapes
    return done(ASDSM_OK);
}

// Learned correction direction of a mixed sweep into zc (skeleton values; the
// caller fills the holes): the network applied to [r, e normalised to unit
// RMS over the interior, alpha_x, alpha_y, beta_x h, beta_y h].
int cnn_direction(asdsm_handle* h, double r2, const float* e, float* zc) {
    const Geometry& g = h->g;
    cudaStream_t st = h->st;
    const long long NN = (long long)g.N * g.N;
    const float* ev[1] = {e};
    int nb = 0;
    CK(multi_dot<float>(ev, ev, 1, NN, h->partials, &nb, st));
    CK(reduce_partials(h->partials, nb, 1, h->dsmall + 210, st));
    CK(cudaMemcpyAsync(h->hsmall + 210, h->dsmall + 210, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double n = (double)g.Nf * g.Nf;
    const double e2 = h->hsmall[210];
    const float rs = r2 > 0 ? (float)std::sqrt(n / r2) : 0.0f;
    const float es = e2 > 0 ? (float)std::sqrt(n / e2) : 0.0f;
    const double hh = 1.0 / g.M;
    const float c[4] = {(float)h->alpha[0], (float)h->alpha[1], (float)(h->beta[0] * hh), (float)(h->beta[1] * hh)};
    CK(cnn_features((const float*)h->w[1].rfull, e, rs, es, c, NN, h->cnn_x, st));
    if (int rc = asdsm_cnn_forward(h->cnn, h->cnn_x, h->cnn_y, 1, g.N, g.N, st)) return rc;
    CK(skeleton_from(h->cnn_y, g, zc, st));
    return ASDSM_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 4.
// ---------------------------------------------------------------------------
// Host-driven sweeps (opts.sweep_graph = 0, and profiling): the host reads the
// residual norms and the least-squares inner products every sweep.
template <typename T>
int host_sweeps(asdsm_handle* h, SolveRun& r) {
    const bool mixed = sizeof(T) == 4;
    const int pi = mixed ? 1 : 0;
    auto& w = h->w[pi];
    const Geometry& g = h->g;
    cudaStream_t st = h->st;
    const asdsm_opts& op = h->opts;
    const int m = std::max(1, std::min(op.accel_m, kMaxM));
    const double NF2 = (double)g.Nf * g.Nf;
    const double ES = (double)sizeof(T);
    const double* s = r.s;
    double*& ucur = r.ucur;
    double*& unxt = r.unxt;
    int& Ucur = r.Ucur;
    const double scale = r.scale;
    const MixedCoefs& mk = r.mk;
    const double bnorm = r.bnorm;
    int& status = r.status;
    int& k = r.k;
    int& hole_fixes = r.hole_fixes;
    double& rel0 = r.rel0;
    double& rel = r.rel;
    std::vector<double>& rhist = r.rhist;
    // GCR bookkeeping (host, FP64).
    double Tm[kMaxM][kMaxM] = {};
    int kc = 0;                  // directions in the current cycle
    UpdateTerms pend{};          // the update the next residual kernel applies
    double hole_ref = 0.0;       // hole residual right after the last correction (0 before the first)
    bool hole_ref_pending = false;
    const bool trace = std::getenv("ASDSM_TRACE") != nullptr;
    // GCR(m > 1) with a deferred update: a cycle's steps accumulate in cacc (in
    // the basis of its raw directions) and reach u through the residual kernel
    // of the cycle's next true residual; in between the residual is tracked on
    // the skeleton (||r||^2 = rr_skel + rh2, the hole part of the cycle's first
    // residual).  Not with a learned direction, whose features need the full residual.
    // Deferral stops for the rest of the solve near the tolerance, or when a
    // cycle's true residual exceeds twice its tracked value (rounding of the
    // FP32 directions in the holes); the stagnation test then holds for a window.
    bool defer = m > 1 && !h->cnn;
    bool tracked = false, cycle_ended = false;
    int stag_hold = 0;
    double cacc[kMaxM] = {};
    double rr_skel = 0.0, rh2c = 0.0;
    auto end_cycle = [&](int count) {
        pend.count = count;
        for (int i = 0; i < count; ++i) { pend.z[i] = w.z[i]; pend.coef[i] = cacc[i]; cacc[i] = 0.0; }
        tracked = false;
        cycle_ended = count > 0;
        kc = 0;
    };
    for (;;) {
      if (tracked) {
        rel = bnorm > 0 ? std::sqrt(std::max(rr_skel, 0.0) + rh2c) / bnorm : std::sqrt(std::max(rr_skel, 0.0) + rh2c);
        const int win = op.stagnation_window;
        const bool stag = win > 0 && (int)rhist.size() > win &&
                          rel > (1.0 - op.stagnation_factor) * rhist[rhist.size() - 1 - win];
        if (!(rel > op.tol) || k >= op.max_sweeps || stag) {
            end_cycle(kc);               // the next true residual decides
            continue;
        }
        if (!std::isfinite(rel)) { status = ASDSM_ERR_NAN; break; }
        rhist.push_back(rel);
        if (k == 0) rel0 = rel;
      } else {
        // ---- fine residual (with the pending update fused) ----
        ResidOut o{};
        o.rfc = w.Xfc; o.rcf = w.Xcf; o.rskel = w.rskel; o.partials = h->partials;
        o.rfull = (mixed && h->cnn) ? w.rfull : nullptr;    // the learned correction reads r on the full grid
        int nb = 0;
        {
            // Algorithmic bytes: read u and s, read each pending direction, write u when updated,
            // write the skeleton gathers (fc, cf, compact).
            const double ub = mixed ? 8.0 : 8.0;
            const double bytes = NF2 * (ub + 8.0 + ES * pend.count + (pend.count > 0 ? ub : 0.0))
                               + ES * (2.0 * g.Nc * g.Nf + (double)g.skel);
            if (mixed) CK(cudaMemsetAsync(h->dflag, 0, sizeof(int), st));
            const ProfMark pm = prof_begin(h);
            if (!mixed) {
                double* dst = pend.count > 0 ? unxt : ucur;
                CK(residual_fp64(s, ucur, dst, pend, g, h->sten, o, &nb, st));
                if (pend.count > 0) std::swap(ucur, unxt);
            } else {
                CK(residual_mixed(h->s_hi, h->s_lo, h->U[Ucur], h->U[1 - Ucur], pend, scale, g, mk, o, &nb, h->dflag, st));
                if (pend.count > 0) Ucur = 1 - Ucur;
            }
            prof_end(h, pm, PC_RESID, bytes, 0.0);
        }
        pend.count = 0;
        CK(reduce_partials(h->partials, nb, 2, h->dsmall, st));
        if (mixed) CK(cudaMemcpyAsync(h->dsmall + 2, h->dflag, sizeof(int), cudaMemcpyDeviceToDevice, st));
        if (int rc = read_small(h, 3)) return rc;
        const double r2 = h->hsmall[0], rh2 = h->hsmall[1];
        if (mixed) {
            int ovf = 0;
            std::memcpy(&ovf, &h->hsmall[2], sizeof(int));
            if (ovf) { status = ASDSM_ERR_RANGE; break; }
        }
        const double rnorm = std::sqrt(r2), hnorm = std::sqrt(rh2);
        rel = bnorm > 0 ? rnorm / bnorm : rnorm;
        const int win = op.stagnation_window;
        if (defer && cycle_ended) {
            const double p2 = std::max(rr_skel, 0.0) + rh2c;
            const double pred = bnorm > 0 ? std::sqrt(p2) / bnorm : std::sqrt(p2);
            if (rel > 2.0 * pred) { defer = false; stag_hold = win; }
        }
        if (defer && rel < kDeferStop * op.tol) defer = false;
        cycle_ended = false;
        rr_skel = r2 - rh2;
        rh2c = rh2;
        if (!std::isfinite(rel)) { status = ASDSM_ERR_NAN; break; }
        rhist.push_back(rel);
        if (k == 0) rel0 = rel;
        if (rel <= op.tol) { status = ASDSM_OK; break; }
        if (k >= op.max_sweeps) { status = ASDSM_NOT_CONVERGED; break; }
        if (stag_hold > 0) {
            --stag_hold;
        } else if (win > 0 && (int)rhist.size() > win &&
                   rhist.back() > (1.0 - op.stagnation_factor) * rhist[rhist.size() - 1 - win]) {
            status = ASDSM_STAGNATED;
            break;
        }
        if (hole_ref_pending) { hole_ref = hnorm; hole_ref_pending = false; }
        if (trace)
            std::fprintf(stderr, "asdsm: k=%d rel=%.6e hole_rel=%.6e kc=%d\n", k, rel, bnorm > 0 ? hnorm / bnorm : hnorm, kc);
        if (hnorm > op.hole_fix_ratio * rnorm && hnorm > op.hole_fix_growth * hole_ref) {
            // Rounding has left a residual in the holes: Algorithm 3 on the current iterate.
            o.rfc = nullptr; o.rcf = nullptr; o.rskel = nullptr; o.rfull = w.rfull;
            UpdateTerms none{};
            FillArgs<T> fa{};
            fa.mode = FILL_RESIDUAL_TO_U;
            if (!mixed) {
                CK(residual_fp64(s, ucur, ucur, none, g, h->sten, o, &nb, st));
                fa.src_d = (const double*)w.rfull;
                fa.u_d = ucur;
            } else {
                CK(residual_mixed(h->s_hi, h->s_lo, h->U[Ucur], h->U[Ucur], none, scale, g, mk, o, &nb, h->dflag, st));
                fa.src_hi = (const float*)w.rfull;
                fa.U = h->U[Ucur];
                fa.fixed_scale = scale;
            }
            hole_factors<T>(h, pi, &fa);
            fa.n = g.n; fa.g = g; fa.sten = h->sten;
            CK(fill_holes<T>(fa, h->num_sms, st));
            ++hole_fixes;
            kc = 0;
            hole_ref_pending = true;         // re-read from the next residual
            ++k;
            continue;
        }
      }
        // ---- the correction: Algorithm 1 without b_cc on the residual ----
        const int bit = choice_bit(op.seed, k);
        BcrSys<T> sys[2] = {sys_of<T>(h->fc[pi], w.Xfc, w.Yfc), sys_of<T>(h->cf[pi], w.Xcf, w.Ycf)};
        {
            const ProfMark pm = prof_begin(h);
            CK(bcr_solve<T>(sys, 2, st, &h->tune_aniso[pi]));
            const double flops = 2.0 * 2.0 * bcr_macs(g.Nf, g.Nc, h->fc[pi].L);
            const double bytes = ES * (4.0 * g.Nf * g.Nc) + ES * 2.0 * 3.0 * h->fc[pi].L * (double)g.Nc * g.Nc;
            prof_end(h, pm, PC_BCR, bytes, flops);
        }
        {
            const ProfMark pm = prof_begin(h);
            const T* av[2] = {(const T*)w.Yfc, (const T*)w.Ycf};
            int nb2 = 0;
            // Two separate dots over the same length.
            CK(multi_dot<T>(av, av, 2, (long long)g.Nf * g.Nc, h->partials, &nb2, st));
            CK(reduce_partials(h->partials, nb2, 2, h->dsmall + 200, st));
            prof_end(h, pm, PC_NORM, ES * 2.0 * g.Nf * g.Nc, 4.0 * g.Nf * g.Nc);
        }
        T* z = (T*)w.z[kc];
        MergeArgs<T> ma{};
        ma.Yfc = (T*)w.Yfc; ma.Ycf = (T*)w.Ycf; ma.Ycc = nullptr;
        ma.norms2 = h->dsmall + 200; ma.re_mode = 0; ma.choice = bit;
        ma.Sm = (const T*)h->Sm[pi];
        ma.E1 = (T*)w.E1; ma.E2 = (T*)w.E2; ma.M1 = (T*)w.M1; ma.M2 = (T*)w.M2;
        ma.z = z; ma.g = g;
        ma.zv = use_fill_tc(h, pi) ? (T*)w.zv : nullptr;
        {
            const ProfMark pm = prof_begin(h);
            CK(merge_knots<T>(ma, st));
            CK(merge_write<T>(ma, st));
            prof_end(h, pm, PC_MERGE, ES * 4.0 * g.Nf * g.Nc, 0.0);
        }
        {
            const ProfMark pm = prof_begin(h);
            CK(fill_homogeneous<T>(h, pi, z, st, (const T*)ma.zv));
            const double holes = (double)g.mc * g.mc, C = g.n - 1.0;
            const double bytes = ES * (holes * C * C + holes * 4.0 * C);
            if (use_fill_tc(h, pi)) {
                // The map v = G z: 2 (C^2) (4C) flops per hole (the TF32 split products
                // the tensor cores issue are about 3.4 times that).
                prof_end(h, pm, PC_FILL_TC, bytes, 2.0 * holes * C * C * 4.0 * C);
            } else {
                prof_end(h, pm, PC_FILL, bytes, 2.0 * holes * bcr_macs(g.n - 1, g.n - 1, h->hole[pi].L));
            }
        }
        // ---- least squares on the skeleton rows (GCR(m) step for direction zd) ----
        // Returns 1 when the direction is dependent (the cycle restarts), 0 otherwise;
        // with `add` the step's update is added to the pending one (a second
        // direction in the same sweep: by orthogonality its coefficient uses the
        // same residual).
        auto gcr_step = [&](T* zd, bool add) -> int {
            const ProfMark pm_lsq = prof_begin(h);
            CK(skeleton_apply<T>(zd, g, h->sten, (T*)w.q, st));
            const T* qpv[kMaxM];
            for (int j = 0; j < kc; ++j) qpv[j] = (const T*)w.qp[j];
            const int nd = 2 + 2 * kc;      // <q,q>, <q,r>, then <q,q'_j>, <r,q'_j>
            int nb3 = 0;
            CK(gcr_dots<T>((const T*)w.q, (const T*)w.rskel, qpv, kc, g.skel, h->partials, &nb3, st));
            CK(reduce_partials(h->partials, nb3, nd, h->dsmall, st));
            prof_end(h, pm_lsq, PC_LSQ, ES * (double)g.skel * (6.0 + 2.0 + kc), 2.0 * (double)g.skel * nd);
            if (int rc = read_small(h, nd)) return rc;
            const double qq = h->hsmall[0], qr = h->hsmall[1];
            if (m == 1) {
                // The paper's clamped optimal scaling: s_hat = argmin_{s >= 0} ||r - s A e||.
                const double shat = qq > 0 ? std::max(0.0, qr / qq) : 0.0;
                pend.count = 1;
                pend.z[0] = zd;
                pend.coef[0] = shat;
                return 0;
            }
            // GCR(m): orthogonalise A e against the cycle's previous directions.
            double beta_[kMaxM] = {}, rq[kMaxM] = {};
            double nu2 = qq;
            for (int j = 0; j < kc; ++j) {
                beta_[j] = h->hsmall[2 + 2 * j];
                rq[j] = h->hsmall[3 + 2 * j];
                nu2 -= beta_[j] * beta_[j];
            }
            if (!(nu2 > 1e-24 * qq) || !(qq > 0)) return 1;
            const double nu = std::sqrt(nu2);
            double alpha_ = qr;
            for (int j = 0; j < kc; ++j) alpha_ -= beta_[j] * rq[j];
            alpha_ /= nu;
            // Column kc of T: z'_kc = sum_i T[i][kc] z_i.
            for (int i = 0; i <= kc; ++i) Tm[i][kc] = 0.0;
            Tm[kc][kc] = 1.0 / nu;
            for (int j = 0; j < kc; ++j)
                for (int i = 0; i <= j; ++i) Tm[i][kc] -= beta_[j] * Tm[i][j] / nu;
            const T* qps[kMaxM];
            for (int j = 0; j < kc; ++j) qps[j] = (const T*)w.qp[j];
            CK(combine_skeleton<T>((const T*)w.q, qps, beta_, kc, 1.0 / nu, g.skel, (T*)w.qp[kc], st));
            if (defer) {
                for (int i = 0; i <= kc; ++i) cacc[i] += alpha_ * Tm[i][kc];
                rr_skel -= alpha_ * alpha_;
                if (kc + 1 >= m) {
                    end_cycle(kc + 1);
                } else {
                    CK(track_skeleton<T>((T*)w.rskel, (const T*)w.qp[kc], alpha_, nullptr, g, (T*)w.Xfc, (T*)w.Xcf,
                                         st));
                    tracked = true;
                    ++kc;
                }
                return 0;
            }
            for (int i = 0; i <= kc; ++i) {
                pend.z[i] = w.z[i];
                pend.coef[i] = (add && i < pend.count ? pend.coef[i] : 0.0) + alpha_ * Tm[i][kc];
            }
            pend.count = kc + 1;
            ++kc;
            if (kc >= m) kc = 0;
            return 0;
        };
        const int dep = gcr_step(z, false);
        if (dep < 0) return dep;
        if (dep == 1) {
            if (defer) end_cycle(kc);         // dependent direction: restart the cycle
            kc = 0;
            ++k;
            continue;
        }
        // Learned correction: one more direction in the same cycle (not in a new one,
        // whose slots the pending update still reads).
        if (mixed && h->cnn && m > 1 && kc != 0) {
            T* zc = (T*)w.z[kc];
            if (int rc = cnn_direction(h, rr_skel + rh2c, (const float*)z, (float*)zc)) return rc;
            CK(fill_homogeneous<T>(h, pi, zc, st));
            const int dep2 = gcr_step(zc, true);
            if (dep2 < 0) return dep2;
            if (dep2 == 0) ++h->cnn_dirs;
        }
        ++k;
    }
    return ASDSM_OK;
}

template <typename T>
int run_begin(asdsm_handle* h, SolveRun& r) {
    const bool mixed = sizeof(T) == 4;
    const int pi = mixed ? 1 : 0;
    if (int rc = ensure_work<T>(h, pi)) return rc;
    auto& w = h->w[pi];
    const Geometry& g = h->g;
    cudaStream_t st = h->st;
    const asdsm_opts& op = h->opts;
    const long long NN = (long long)g.N * g.N;
    const double* s = r.s;
    double* u = r.u;
    if (int rc = ensure_partials(h, std::max(2 * residual_grid_blocks(g), kDotPartials))) return rc;
    h->hist.clear();
    h->pend_ev.clear();
    h->evnext = 0;
    h->cnn_dirs = 0;
    CK(cudaEventRecord(h->ev0, st));
    // ||b_ff||^2: the FP64 residual of the zero-interior grid (r = b there).
    {
        CK(ring_from<double>(u, h->u_work, g, 1, st));
        int nb = 0;
        ResidOut o{};
        o.partials = h->partials;
        UpdateTerms up{};
        CK(residual_fp64(s, h->u_work, h->u_work, up, g, h->sten, o, &nb, st));
        CK(reduce_partials(h->partials, nb, 2, h->dsmall, st));
        CK(cudaMemcpyAsync(h->hsmall, h->dsmall, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    // Iterate storage.  FP64: ping-pong between the caller's u and u_work (ring = g in both).
    // Mixed: U[0]/U[1] (64-bit fixed point, u = U 2^-S).
    r.ucur = u;
    r.unxt = h->u_work;
    r.Ucur = 0;
    if (mixed) CK(split_source(s, h->s_hi, h->s_lo, NN, st));
    CK(ring_from<double>(u, h->u_work, g, 0, st));
    // Initial guess (or resume from u).  The mixed path computes
    // Algorithm 1 once in FP64: an FP32 u^(0) carries rounding noise whose
    // residual is rough, and ASDSM corrections reduce rough residuals slowly
    // (the irregular-residual stagnation of Section 4, Example 2).
    r.u0d = u;                       // FP64 grid holding u^(0) (ring = g)
    const bool guess = !op.skip_initial_guess && !r.resume;
    if (guess) {
        if (!mixed) {
            if (int rc = initial_guess_to_z<double>(h, s, u)) return rc;
            CK(copy_interior<double, double>((const double*)w.z[0], u, g, st));
        } else {
            if (int rc = initial_guess_refined(h, s, u)) return rc;
            r.u0d = (const double*)h->w[0].z[0];
        }
    }
    if (mixed) {
        // Fixed-point scale from max |u| (interior and ring): block maxima to the host.
        int nb = 0;
        CK(maxabs<double>(r.u0d, NN, h->partials, &nb, st));
        if (nb > 4000) return ASDSM_ERR_INVALID;
        CK(cudaMemcpyAsync(h->hsmall + 8, h->partials, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        r.nb_max = nb;
    }
    CK(cudaEventRecord(h->evA, st));
    r.stage = 1;
    return ASDSM_OK;
}

template <typename T>
int run_middle(asdsm_handle* h, SolveRun& r) {
    const bool mixed = sizeof(T) == 4;
    const int pi = mixed ? 1 : 0;
    auto& w = h->w[pi];
    const Geometry& g = h->g;
    cudaStream_t st = h->st;
    const asdsm_opts& op = h->opts;
    r.bnorm = std::sqrt(h->hsmall[0]);
    if (!std::isfinite(r.bnorm)) return ASDSM_ERR_NAN;
    if (mixed) {
        double mx = 0.0;
        for (int q = 0; q < r.nb_max; ++q) mx = std::max(mx, h->hsmall[8 + q]);
        if (!std::isfinite(mx)) return ASDSM_ERR_NAN;
        if (mx <= 0.0) mx = 1.0;
        int e2 = 0;
        std::frexp(mx, &e2);                // mx < 2^e2
        r.S = std::min(58 - e2, r.S_cap);   // |U| < 2^58: 2^5 headroom below the 2^63 range and the 2^60 check
        r.scale = std::ldexp(1.0, r.S);
        CK(to_fixed(nullptr, r.u0d, h->U[0], r.scale, g, st));
        CK(to_fixed(nullptr, r.u0d, h->U[1], r.scale, g, st));   // ring of the partner
    }
    // Direction slots need a zero ring again (slot 0 carried g).
    if (!op.skip_initial_guess && !r.resume) CK(ring_from<double>(nullptr, (double*)h->w[0].z[0], g, 0, st));
    CK(ring_from<T>(nullptr, (T*)w.z[0], g, 0, st));
    CK(cudaEventRecord(h->ev1, st));
    r.mk = mixed ? mixed_coefs(h, r.S) : MixedCoefs{};
    if (op.sweep_graph && !h->prof && !h->cnn) {
        if (int rc = graph_start<T>(h, r)) return rc;
        r.stage = 2;
    } else {
        if (int rc = host_sweeps<T>(h, r)) return rc;
        r.stage = 3;
    }
    return ASDSM_OK;
}

template <typename T>
int run_finish(asdsm_handle* h, SolveRun& r) {
    const bool mixed = sizeof(T) == 4;
    const Geometry& g = h->g;
    cudaStream_t st = h->st;
    // Final iterate to the caller's buffer.
    if (!mixed) {
        if (r.ucur != r.u) CK(copy_interior<double, double>(r.ucur, r.u, g, st));
    } else {
        // After an overflow the current buffer holds the update that did not
        // fit; the other one holds the last iterate that did.
        const int buf = r.status == ASDSM_ERR_RANGE ? 1 - r.Ucur : r.Ucur;
        CK(from_fixed(h->U[buf], std::ldexp(1.0, -r.S), r.u, g, st));
    }
    // The returned iterate judged in FP64 (residual norm, largest hole residual).
    CK(final_check(r.s, r.u, g, h->sten, h->partials, std::min(8 * h->num_sms, h->partials_cap / 2),
                   h->dsmall + 220, st));
    CK(cudaMemcpyAsync(h->hsmall + 220, h->dsmall + 220, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    int* tcerr = reinterpret_cast<int*>(h->hsmall + 4095);
    *tcerr = 0;
    CK(cudaMemcpyAsync(tcerr, h->dtcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(h->ev2, st));
    CK(cudaEventSynchronize(h->ev2));
    if (*tcerr) {
        g_last_error = "tensor-core kernel: a wait timed out";
        return ASDSM_ERR_CUDA;
    }
    float ms_setup = 0.f, ms_all = 0.f;
    cudaEventElapsedTime(&ms_setup, h->ev0, h->ev1);
    cudaEventElapsedTime(&ms_all, h->ev0, h->ev2);
    h->hist = r.rhist;
    prof_resolve(h);
    asdsm_stats stt{};
    stt.launches = r.launches;
    stt.sweeps = r.k;
    stt.status = r.status;
    stt.hole_fixes = r.hole_fixes;
    stt.fixed_shift = mixed ? r.S : 0;
    stt.rel_res = r.rel;
    stt.rel_res0 = r.rel0;
    stt.setup_ms = ms_setup;
    stt.solve_ms = ms_all;
    stt.rel_res_fp64 = r.bnorm > 0 ? std::sqrt(h->hsmall[220]) / r.bnorm : std::sqrt(h->hsmall[220]);
    stt.hole_res_max = h->hsmall[221];
    if (r.stats) *r.stats = stt;
    return r.status;
}

// Run one stage of a solve, attributing the kernel launches it makes.
template <typename F>
int staged(SolveRun& r, F&& fn) {
    const long long a = launch_count();
    const int rc = fn();
    r.launches += launch_count() - a;
    return rc;
}

template <typename T>
int solve_pass(asdsm_handle* h, SolveRun& r) {
    if (int rc = staged(r, [&] { return run_begin<T>(h, r); })) return rc;
    CK(cudaEventSynchronize(h->evA));
    if (int rc = staged(r, [&] { return run_middle<T>(h, r); })) return rc;
    while (r.stage == 2)
        if (int rc = staged(r, [&] { return graph_poll<T>(h, r, true); })) return rc;
    return staged(r, [&] { return run_finish<T>(h, r); });
}

// A solve, and on the mixed path its restarts after a fixed-point overflow:
// the shift S was chosen from max |u^(0)|, which says little when the
// iterate grows far beyond its start (a resume from a small or zero
// interior).  Each restart resumes from the last iterate that fitted (u,
// now in FP64) with S lowered by at least 4, and at most kMaxRescales times.
constexpr int kMaxRescales = 12;

template <typename T>
int solve_impl(asdsm_handle* h, const double* s, double* u, asdsm_stats* stats) {
    asdsm_stats total{};
    std::vector<double> hist;
    int S_cap = 1 << 20;
    for (int pass = 0;; ++pass) {
        SolveRun r;
        asdsm_stats st{};
        r.s = s; r.u = u; r.stats = &st;
        r.resume = pass > 0;
        r.S_cap = S_cap;
        const int rc = solve_pass<T>(h, r);
        if (r.stage != 3 || (rc != r.status && rc != ASDSM_OK)) return rc;     // an error before any result
        if (pass == 0) {
            total = st;
            hist = h->hist;
        } else {
            total.sweeps += st.sweeps; total.hole_fixes += st.hole_fixes; total.launches += st.launches;
            total.solve_ms += st.solve_ms;
            total.status = st.status; total.fixed_shift = st.fixed_shift; total.rel_res = st.rel_res;
            total.rel_res_fp64 = st.rel_res_fp64; total.hole_res_max = st.hole_res_max;
            hist.insert(hist.end(), h->hist.begin() + (h->hist.empty() ? 0 : 1), h->hist.end());
        }
        total.rescales = pass;
        if (sizeof(T) == 4 && rc == ASDSM_ERR_RANGE && pass < kMaxRescales) {
            S_cap = r.S - 4;
            continue;
        }
        h->hist = hist;
        if (stats) *stats = total;
        return rc;
    }
}

}  // namespace

namespace asdsm {
int report_cuda_error(cudaError_t e) { return set_cuda_error(e); }
void report_error(const std::string& msg) { g_last_error = msg; }
}  // namespace asdsm

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void asdsm_default_opts(asdsm_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-10;
    o->max_sweeps = 500;
    o->precision = ASDSM_MIXED;
    o->accel_m = 8;
    o->skip_initial_guess = 0;
    o->seed = 0;
    o->hole_fix_ratio = 0.25;
    o->hole_fix_growth = 4.0;
    o->stagnation_window = 10;
    o->stagnation_factor = 1e-3;
    o->sweep_graph = 1;
}

const char* asdsm_strerror(int code) {
    switch (code) {
        case ASDSM_OK: return "ok";
        case ASDSM_ERR_INVALID: return "invalid argument (sizes must satisfy eq. 2.1 with N-1 and mc powers of two, 2 <= mc, (N-1)/mc in [2, 32], N <= 32769; alpha > 0)";
        case ASDSM_ERR_CUDA: return "CUDA runtime error";
        case ASDSM_ERR_OOM: return "device allocation failed";
        case ASDSM_ERR_NAN: return "NaN or Inf in the residual";
        case ASDSM_NOT_CONVERGED: return "max_sweeps reached above tol";
        case ASDSM_STAGNATED: return "residual stagnated";
        case ASDSM_ERR_RANGE: return "fixed-point accumulator range exceeded";
        default: return "unknown status";
    }
}

const char* asdsm_last_error(void) { return g_last_error.c_str(); }

int asdsm_setup(const asdsm_desc* desc, const asdsm_opts* opts, void* stream, asdsm_handle** out) {
    if (!out) return ASDSM_ERR_INVALID;
    *out = nullptr;
    if (!desc) return ASDSM_ERR_INVALID;
    if (desc->d == 3) {
        asdsm_opts o3;
        if (opts) o3 = *opts; else asdsm_default_opts(&o3);
        Solver3D* s3 = nullptr;
        if (int rc = s3_create(desc, &o3, (cudaStream_t)stream, &s3)) return rc;
        asdsm_handle* h = new asdsm_handle();
        h->desc = *desc;
        h->opts = o3;
        h->st = (cudaStream_t)stream;
        h->s3 = s3;
        *out = h;
        return ASDSM_OK;
    }
    if (desc->d != 2) return ASDSM_ERR_INVALID;
    const long long N = desc->n, mc = desc->mc;
    if (N < 5 || N > 32769 || !is_pow2(N - 1) || mc < 2 || !is_pow2(mc) || (N - 1) % mc != 0)
        return ASDSM_ERR_INVALID;
    const long long n = (N - 1) / mc;
    if (n < 2 || n > 32) return ASDSM_ERR_INVALID;
    if (!(desc->alpha[0] > 0) || !(desc->alpha[1] > 0)) return ASDSM_ERR_INVALID;
    for (int q = 0; q < 2; ++q)
        if (!std::isfinite(desc->alpha[q]) || !std::isfinite(desc->beta[q])) return ASDSM_ERR_INVALID;

    asdsm_handle* h = new asdsm_handle();
    h->desc = *desc;
    if (opts) h->opts = *opts; else asdsm_default_opts(&h->opts);
    if (h->opts.accel_m < 1 || h->opts.accel_m > kMaxM) { delete h; return ASDSM_ERR_INVALID; }
    h->st = (cudaStream_t)stream;
    auto fail = [&](int rc) { asdsm_destroy(h); return rc; };
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(set_cuda_error(e));
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    for (int q = 0; q < 2; ++q) { h->tune_aniso[q].num_sms = h->num_sms; h->tune_cc[q].num_sms = h->num_sms; }
    if (std::getenv("ASDSM_TRACE_BCR"))
        for (int q = 0; q < 2; ++q) { h->tune_aniso[q].trace = 1; h->tune_cc[q].trace = 1; }
    Geometry& g = h->g;
    g.N = (int)N; g.M = (int)(N - 1); g.Nf = (int)(N - 2); g.mc = (int)mc; g.Nc = (int)(mc - 1); g.n = (int)n;
    g.skel = (long long)g.Nc * g.Nf + (long long)g.Nc * (g.Nf - g.Nc);
    g.ln = 0;
    while ((1 << g.ln) < g.n) ++g.ln;
    for (int q = 0; q < 2; ++q) { h->alpha[q] = desc->alpha[q]; h->beta[q] = desc->beta[q]; }
    const double ax = h->alpha[0], ay = h->alpha[1], bx = h->beta[0], by = h->beta[1];
    const double hh = 1.0 / g.M, HH = 1.0 / g.mc;
    h->sten = stencil_of(ax, ay, bx, by, hh);
    // Block cyclic reduction factors (eq. 2.4 systems; rows = the fine axis of each family).
    auto row = [](double a, double b, double sp, double* lo, double* d, double* up) {
        *lo = -a / (sp * sp) - b / (2 * sp);
        *d = 2 * a / (sp * sp);
        *up = -a / (sp * sp) + b / (2 * sp);
    };
    double xl_h, xd_h, xu_h, yl_h, yd_h, yu_h, xl_H, xd_H, xu_H, yl_H, yd_H, yu_H;
    row(ax, bx, hh, &xl_h, &xd_h, &xu_h);
    row(ay, by, hh, &yl_h, &yd_h, &yu_h);
    row(ax, bx, HH, &xl_H, &xd_H, &xu_H);
    row(ay, by, HH, &yl_H, &yd_H, &yu_H);
    BcrFactors ffc, fcf, fcc, fho;
    // A_fc: rows x (fine), columns the coarse lines in y.
    if (!make_bcr(g.Nf, xl_h, xd_h, xu_h, g.Nc, yl_H, yd_H, yu_H, &ffc)) return fail(ASDSM_ERR_INVALID);
    // A_cf: rows y (fine), columns the coarse lines in x.
    if (!make_bcr(g.Nf, yl_h, yd_h, yu_h, g.Nc, xl_H, xd_H, xu_H, &fcf)) return fail(ASDSM_ERR_INVALID);
    // A_cc: rows y (coarse), columns x (coarse).
    if (!make_bcr(g.Nc, yl_H, yd_H, yu_H, g.Nc, xl_H, xd_H, xu_H, &fcc)) return fail(ASDSM_ERR_INVALID);
    // Hole blocks A_(ij): rows y, columns x, both fine.
    if (!make_bcr(g.n - 1, yl_h, yd_h, yu_h, g.n - 1, xl_h, xd_h, xu_h, &fho)) return fail(ASDSM_ERR_INVALID);
    const BcrCoefs kfc{xl_h, xd_h, xu_h, yl_H, yd_H, yu_H}, kcf{yl_h, yd_h, yu_h, xl_H, xd_H, xu_H},
        kcc{yl_H, yd_H, yu_H, xl_H, xd_H, xu_H};
    for (int q = 0; q < 2; ++q) { h->fc[q].k = kfc; h->cf[q].k = kcf; h->cc[q].k = kcc; }
    int rc;
    if ((rc = upload_bcr<double>(ffc, &h->fc[0])) || (rc = upload_bcr<float>(ffc, &h->fc[1])) ||
        (rc = upload_bcr<double>(fcf, &h->cf[0])) || (rc = upload_bcr<float>(fcf, &h->cf[1])) ||
        (rc = upload_bcr<double>(fcc, &h->cc[0])) || (rc = upload_bcr<float>(fcc, &h->cc[1])) ||
        (rc = upload_bcr<double>(fho, &h->hole[0])) || (rc = upload_bcr<float>(fho, &h->hole[1])) ||
        (rc = upload_tail(ffc, &h->fc[1])) || (rc = upload_tail(fcf, &h->cf[1])))
        return fail(rc);
    // Spline moment operator, stored transposed ([knot][moment]) for the merge kernel.
    const std::vector<double> Sm = spline_moment_operator(g.mc);
    std::vector<double> SmT(Sm.size());
    for (int r = 0; r <= g.mc; ++r)
        for (int q = 0; q < g.Nc; ++q) SmT[(size_t)q * (g.mc + 1) + r] = Sm[(size_t)r * g.Nc + q];
    if ((rc = upload_vec<double>(SmT, &h->Sm[0])) || (rc = upload_vec<float>(SmT, &h->Sm[1]))) return fail(rc);
    if (fill_smem_bytes<double>(g.n, h->hole[0].L) > 227 * 1024) return fail(ASDSM_ERR_INVALID);
    const size_t NN = (size_t)g.N * g.N;
    if ((e = cudaMalloc(&h->u_work, NN * sizeof(double))) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaMalloc(&h->U[0], NN * sizeof(long long))) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaMalloc(&h->U[1], NN * sizeof(long long))) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaMalloc(&h->s_hi, NN * sizeof(float))) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaMalloc(&h->s_lo, NN * sizeof(float))) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaMalloc(&h->dsmall, 256 * sizeof(double))) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaMalloc(&h->dflag, sizeof(int))) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaMalloc(&h->dtcerr, sizeof(int))) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaMemset(h->dtcerr, 0, sizeof(int))) != cudaSuccess) return fail(set_cuda_error(e));
    for (int q = 0; q < 2; ++q)
        for (DevBcr* d : {&h->fc[q], &h->cf[q], &h->cc[q], &h->hole[q]}) d->tc_err = h->dtcerr;
    if (g.n == kFillTcN) {
        std::vector<double> G;
        if (!hole_extension_operator(g.n - 1, h->sten, &G)) return fail(ASDSM_ERR_INVALID);
        std::vector<float> img;
        fill_tc_image(G, &img);
        if ((e = cudaMalloc(&h->fill_tc_img, fill_tc_image_bytes())) != cudaSuccess) return fail(set_cuda_error(e));
        if ((e = cudaMemcpy(h->fill_tc_img, img.data(), fill_tc_image_bytes(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(set_cuda_error(e));
    }
    if ((e = cudaMallocHost(&h->hsmall, 4096 * sizeof(double))) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaEventCreate(&h->ev0)) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaEventCreate(&h->ev1)) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaEventCreate(&h->ev2)) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaEventCreateWithFlags(&h->evA, cudaEventDisableTiming)) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaMalloc(&h->dctl, sizeof(SweepCtl))) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaMallocHost(&h->hctl, sizeof(SweepCtl))) != cudaSuccess) return fail(set_cuda_error(e));
    if ((e = cudaMallocHost(&h->hdone, 2 * sizeof(int))) != cudaSuccess) return fail(set_cuda_error(e));
    for (int q = 0; q < 2; ++q)
        if ((e = cudaEventCreateWithFlags(&h->evc[q], cudaEventDisableTiming)) != cudaSuccess) return fail(set_cuda_error(e));
    if ((rc = ensure_partials(h, std::max(2 * residual_grid_blocks(g), kDotPartials)))) return fail(rc);
    asdsm_profile(h, 0);
    *out = h;
    return ASDSM_OK;
}

int asdsm_autotune(asdsm_handle* h, int precision) {
    if (!h) return ASDSM_ERR_INVALID;
    if (h->s3) { g_last_error = "not available for the 3D extension"; return ASDSM_ERR_INVALID; }
    int rc;
    if (precision == ASDSM_FP64) rc = autotune_impl<double>(h);
    else if (precision == ASDSM_MIXED) rc = autotune_impl<float>(h);
    else return ASDSM_ERR_INVALID;
    return rc;
}

// Tuned launch shapes as plain integers: per precision (FP64 first), the
// forward and backward level shapes of the anisotropic pair (2 x 16), of the
// coarse system (2 x 16), then the Filler's warps per CTA.
constexpr int kTuneInts = 2 * (4 * kMaxLevels + 1);

int asdsm_tune_get(const asdsm_handle* h, int32_t* out, int cap) {
    if (!h || !out || cap < kTuneInts) return ASDSM_ERR_INVALID;
    if (h->s3) { g_last_error = "not available for the 3D extension"; return ASDSM_ERR_INVALID; }
    int q = 0;
    for (int pi = 0; pi < 2; ++pi) {
        for (int d = 0; d < 2; ++d)
            for (int l = 0; l < kMaxLevels; ++l) out[q++] = h->tune_aniso[pi].cfg[d][l];
        for (int d = 0; d < 2; ++d)
            for (int l = 0; l < kMaxLevels; ++l) out[q++] = h->tune_cc[pi].cfg[d][l];
        out[q++] = h->fill_warps[pi];
    }
    return q;
}

int asdsm_tune_check(const int32_t* in, int n) {
    if (!in || n != kTuneInts) return ASDSM_ERR_INVALID;
    int q = 0;
    for (int pi = 0; pi < 2; ++pi) {
        for (int k = 0; k < 4 * kMaxLevels; ++k) {
            const int v = in[q++];
            if (v == 0) continue;
            const int tm = v >> 8, ks = v & 0xFF;
            const bool split_k = (tm == 16 || tm == 64) && (ks == 1 || ks == 2 || ks == 4 || ks == 8);
            const bool tensor = pi == 1 && ((tm == 32 && ks == 1) || (tm == 128 && (ks == 1 || ks == 2 || ks == 4)));
            if (v < 0 || !(split_k || tensor)) return ASDSM_ERR_INVALID;
        }
        const int f = in[q++];
        if (!(f >= 0 && f <= 8) && !(pi == 1 && f == 16)) return ASDSM_ERR_INVALID;
    }
    return ASDSM_OK;
}

int asdsm_tune_set(asdsm_handle* h, const int32_t* in, int n) {
    if (!h) return ASDSM_ERR_INVALID;
    if (h->s3) { g_last_error = "not available for the 3D extension"; return ASDSM_ERR_INVALID; }
    if (int rc = asdsm_tune_check(in, n)) return rc;
    int q = 0;
    for (int pi = 0; pi < 2; ++pi) {
        for (int d = 0; d < 2; ++d)
            for (int l = 0; l < kMaxLevels; ++l) h->tune_aniso[pi].cfg[d][l] = in[q++];
        for (int d = 0; d < 2; ++d)
            for (int l = 0; l < kMaxLevels; ++l) h->tune_cc[pi].cfg[d][l] = in[q++];
        h->fill_warps[pi] = in[q++];
    }
    if (tune_wants_tc(h->tune_aniso[1]) || tune_wants_tc(h->tune_cc[1]))
        if (int rc = ensure_tc_images(h)) return rc;
    destroy_graph(h);
    return ASDSM_OK;
}

int asdsm_attach_cnn(asdsm_handle* h, asdsm_cnn* net) {
    if (!h) return ASDSM_ERR_INVALID;
    if (h->s3) { g_last_error = "not available for the 3D extension"; return ASDSM_ERR_INVALID; }
    if (h->cnn_x) { cudaFree(h->cnn_x); h->cnn_x = nullptr; }
    if (h->cnn_y) { cudaFree(h->cnn_y); h->cnn_y = nullptr; }
    h->cnn = nullptr;
    if (!net) return ASDSM_OK;
    const size_t NN = (size_t)h->g.N * h->g.N;
    CK(cudaMalloc(&h->cnn_x, 6 * NN * sizeof(float)));
    CK(cudaMalloc(&h->cnn_y, NN * sizeof(float)));
    h->cnn = net;
    return ASDSM_OK;
}

int asdsm_cnn_directions(const asdsm_handle* h) { return h ? h->cnn_dirs : ASDSM_ERR_INVALID; }

int asdsm_correction(asdsm_handle* h, const double* s, const double* u, float* r_out, float* e_out, int k) {
    if (!h || !s || !u || !r_out || !e_out || k < 0) return ASDSM_ERR_INVALID;
    if (h->s3) { g_last_error = "not available for the 3D extension"; return ASDSM_ERR_INVALID; }
    if (int rc = ensure_work<double>(h, 0, 1)) return rc;
    if (int rc = ensure_partials(h, std::max(2 * residual_grid_blocks(h->g), kDotPartials))) return rc;
    auto& w = h->w[0];
    const Geometry& g = h->g;
    cudaStream_t st = h->st;
    ResidOut o{};
    o.rfc = w.Xfc; o.rcf = w.Xcf; o.rskel = w.rskel; o.rfull = w.rfull; o.partials = h->partials;
    UpdateTerms none{};
    int nb = 0;
    CK(residual_fp64(s, u, const_cast<double*>(u), none, g, h->sten, o, &nb, st));
    BcrSys<double> sys[2] = {sys_of<double>(h->fc[0], w.Xfc, w.Yfc), sys_of<double>(h->cf[0], w.Xcf, w.Ycf)};
    CK(bcr_solve<double>(sys, 2, st, &h->tune_aniso[0]));
    const double* av[2] = {(const double*)w.Yfc, (const double*)w.Ycf};
    int nb2 = 0;
    CK(multi_dot<double>(av, av, 2, (long long)g.Nf * g.Nc, h->partials, &nb2, st));
    CK(reduce_partials(h->partials, nb2, 2, h->dsmall + 200, st));
    double* z = (double*)w.z[0];
    MergeArgs<double> ma{};
    ma.Yfc = (double*)w.Yfc; ma.Ycf = (double*)w.Ycf; ma.Ycc = nullptr;
    ma.norms2 = h->dsmall + 200; ma.re_mode = 0; ma.choice = choice_bit(h->opts.seed, k);
    ma.Sm = (const double*)h->Sm[0];
    ma.E1 = (double*)w.E1; ma.E2 = (double*)w.E2; ma.M1 = (double*)w.M1; ma.M2 = (double*)w.M2;
    ma.z = z; ma.g = g;
    CK(merge_knots<double>(ma, st));
    CK(merge_write<double>(ma, st));
    FillArgs<double> fa{};
    fa.mode = FILL_HOMOGENEOUS;
    fa.z = z; fa.out = z;
    hole_factors<double>(h, 0, &fa);
    fa.n = g.n; fa.g = g; fa.sten = h->sten;
    CK(fill_holes<double>(fa, h->num_sms, st));
    const long long NN = (long long)g.N * g.N;
    CK(convert_array<double, float>((const double*)w.rfull, r_out, NN, st));
    CK(convert_array<double, float>(z, e_out, NN, st));
    CK(cudaStreamSynchronize(st));
    return ASDSM_OK;
}

int asdsm_set_opts(asdsm_handle* h, const asdsm_opts* opts) {
    if (!h || !opts) return ASDSM_ERR_INVALID;
    if (opts->precision != ASDSM_FP64 && opts->precision != ASDSM_MIXED) return ASDSM_ERR_INVALID;
    if (h->s3) {
        if (int rc = s3_set_opts(h->s3, opts)) return rc;
        h->opts = *opts;
        return ASDSM_OK;
    }
    if (opts->accel_m < 1 || opts->accel_m > kMaxM) return ASDSM_ERR_INVALID;
    h->opts = *opts;
    return ASDSM_OK;
}

int asdsm_solve(asdsm_handle* h, const double* s, double* u, asdsm_stats* stats) {
    if (!h || !s || !u) return ASDSM_ERR_INVALID;
    if (h->s3) return s3_solve(h->s3, s, u, stats);
    if (h->opts.precision == ASDSM_FP64) return solve_impl<double>(h, s, u, stats);
    if (h->opts.precision == ASDSM_MIXED) return solve_impl<float>(h, s, u, stats);
    return ASDSM_ERR_INVALID;
}

int asdsm_initial_guess(asdsm_handle* h, const double* s, double* u) {
    if (!h || !s || !u) return ASDSM_ERR_INVALID;
    if (h->s3) return s3_initial_guess(h->s3, s, u);
    int rc;
    if (h->opts.precision == ASDSM_FP64) {
        if ((rc = ensure_work<double>(h, 0))) return rc;
        if ((rc = initial_guess_to_z<double>(h, s, u))) return rc;
        CK(copy_interior<double, double>((const double*)h->w[0].z[0], u, h->g, h->st));
        CK(ring_from<double>(nullptr, (double*)h->w[0].z[0], h->g, 0, h->st));
    } else {
        // The solver's mixed-path initial guess: FP32 solves refined to FP64 quality.
        CK(split_source(s, h->s_hi, h->s_lo, (long long)h->g.N * h->g.N, h->st));
        if ((rc = ensure_work<float>(h, 1))) return rc;
        if ((rc = ensure_partials(h, std::max(2 * residual_grid_blocks(h->g), kDotPartials)))) return rc;
        if ((rc = initial_guess_refined(h, s, u))) return rc;
        CK(copy_interior<double, double>((const double*)h->w[0].z[0], u, h->g, h->st));
        CK(ring_from<double>(nullptr, (double*)h->w[0].z[0], h->g, 0, h->st));
        CK(ring_from<float>(nullptr, (float*)h->w[1].z[0], h->g, 0, h->st));
    }
    CK(cudaStreamSynchronize(h->st));
    return ASDSM_OK;
}

int asdsm_residual(asdsm_handle* h, const double* s, const double* u, double* r, double* rel_norm) {
    if (!h || !s || !u) return ASDSM_ERR_INVALID;
    if (h->s3) {
        if (r) { g_last_error = "3D: r is not returned (use asdsm_residual_noalloc)"; return ASDSM_ERR_INVALID; }
        return s3_residual(h->s3, s, u, r, rel_norm);
    }
    const Geometry& g = h->g;
    double b2 = 0.0;
    int rc;
    if ((rc = bnorm2(h, s, u, &b2))) return rc;
    ResidOut o{};
    o.partials = h->partials;
    o.rfull = r;
    UpdateTerms up{};
    int nb = 0;
    if (r) CK(ring_from<double>(nullptr, r, g, 0, h->st));
    CK(residual_fp64(s, u, const_cast<double*>(u), up, g, h->sten, o, &nb, h->st));
    CK(reduce_partials(h->partials, nb, 2, h->dsmall, h->st));
    if ((rc = read_small(h, 2))) return rc;
    if (rel_norm) *rel_norm = b2 > 0 ? std::sqrt(h->hsmall[0] / b2) : std::sqrt(h->hsmall[0]);
    return ASDSM_OK;
}

int asdsm_submesh_solve(asdsm_handle* h, int mesh, const double* in, double* out) {
    if (!h || !in || !out || in == out) return ASDSM_ERR_INVALID;
    if (h->s3) return s3_submesh_solve(h->s3, mesh, in, out);
    const Geometry& g = h->g;
    const bool fp64 = h->opts.precision == ASDSM_FP64;
    const int pi = fp64 ? 0 : 1;
    int rc;
    if ((rc = fp64 ? ensure_work<double>(h, 0) : ensure_work<float>(h, 1))) return rc;
    auto& w = h->w[pi];
    cudaStream_t st = h->st;
    if (mesh >= 0 && mesh <= 2) {
        const DevBcr& d = mesh == 0 ? h->fc[pi] : (mesh == 1 ? h->cf[pi] : h->cc[pi]);
        void* X = mesh == 2 ? w.Xcc : w.Xfc;
        void* Y = mesh == 2 ? w.Ycc : w.Yfc;
        const long long n = (long long)d.R * d.C;
        // Layouts: fc in/out are [line][x] on the API, [x][line] inside.
        if (fp64) {
            BcrSys<double> s = sys_of<double>(d, X, Y);
            if (mesh == 0) {
                std::vector<double> hin(n), hx(n);
                CK(cudaMemcpy(hin.data(), in, n * sizeof(double), cudaMemcpyDeviceToHost));
                for (int l = 0; l < g.Nc; ++l)
                    for (int x = 0; x < g.Nf; ++x) hx[(size_t)x * g.Nc + l] = hin[(size_t)l * g.Nf + x];
                CK(cudaMemcpy(X, hx.data(), n * sizeof(double), cudaMemcpyHostToDevice));
            } else {
                CK(cudaMemcpyAsync(X, in, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            }
            CK(bcr_solve<double>(&s, 1, st, mesh == 2 ? &h->tune_cc[0] : &h->tune_aniso[0]));
            if (mesh == 0) {
                std::vector<double> hy(n), hout(n);
                CK(cudaMemcpy(hy.data(), Y, n * sizeof(double), cudaMemcpyDeviceToHost));
                for (int l = 0; l < g.Nc; ++l)
                    for (int x = 0; x < g.Nf; ++x) hout[(size_t)l * g.Nf + x] = hy[(size_t)x * g.Nc + l];
                CK(cudaMemcpy(out, hout.data(), n * sizeof(double), cudaMemcpyHostToDevice));
            } else {
                CK(cudaMemcpyAsync(out, Y, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            }
        } else {
            BcrSys<float> s = sys_of<float>(d, X, Y);
            std::vector<double> hin(n), hx(n);
            CK(cudaMemcpy(hin.data(), in, n * sizeof(double), cudaMemcpyDeviceToHost));
            if (mesh == 0) {
                for (int l = 0; l < g.Nc; ++l)
                    for (int x = 0; x < g.Nf; ++x) hx[(size_t)x * g.Nc + l] = hin[(size_t)l * g.Nf + x];
            } else {
                hx = hin;
            }
            std::vector<float> hf(hx.begin(), hx.end());
            CK(cudaMemcpy(X, hf.data(), n * sizeof(float), cudaMemcpyHostToDevice));
            CK(bcr_solve<float>(&s, 1, st, mesh == 2 ? &h->tune_cc[1] : &h->tune_aniso[1]));
            CK(cudaMemcpy(hf.data(), Y, n * sizeof(float), cudaMemcpyDeviceToHost));
            std::vector<double> hout(n);
            if (mesh == 0) {
                for (int l = 0; l < g.Nc; ++l)
                    for (int x = 0; x < g.Nf; ++x) hout[(size_t)l * g.Nf + x] = hf[(size_t)x * g.Nc + l];
            } else {
                for (long long q = 0; q < n; ++q) hout[q] = hf[q];
            }
            CK(cudaMemcpy(out, hout.data(), n * sizeof(double), cudaMemcpyHostToDevice));
        }
    } else if (mesh == 3) {
        if (fp64) {
            FillArgs<double> fa{};
            fa.mode = FILL_ARRAY; fa.src_d = in; fa.out_d = out;
            hole_factors<double>(h, 0, &fa);
            fa.n = g.n; fa.g = g; fa.sten = h->sten;
            CK(fill_holes<double>(fa, h->num_sms, st));
        } else {
            FillArgs<float> fa{};
            fa.mode = FILL_ARRAY; fa.src_d = in; fa.out_d = out;
            hole_factors<float>(h, 1, &fa);
            fa.n = g.n; fa.g = g; fa.sten = h->sten;
            CK(fill_holes<float>(fa, h->num_sms, st));
        }
    } else if (mesh == 4) {
        if (fp64) {
            FillArgs<double> fa{};
            fa.mode = FILL_HOMOGENEOUS; fa.z = in; fa.out_d = out;
            hole_factors<double>(h, 0, &fa);
            fa.n = g.n; fa.g = g; fa.sten = h->sten;
            CK(fill_holes<double>(fa, h->num_sms, st));
        } else {
            float* z32 = (float*)w.z[0];
            CK(convert_array<double, float>(in, z32, (long long)g.N * g.N, st));
            if (use_fill_tc(h, 1)) {
                FillTcArgs ta{h->fill_tc_img, z32, out, nullptr, g.N, g.mc, h->dtcerr};
                CK(fill_tc(ta, h->num_sms, st));
            } else {
                FillArgs<float> fa{};
                fa.mode = FILL_HOMOGENEOUS; fa.z = z32; fa.out_d = out;
                hole_factors<float>(h, 1, &fa);
                fa.n = g.n; fa.g = g; fa.sten = h->sten;
                CK(fill_holes<float>(fa, h->num_sms, st));
            }
        }
    } else {
        return ASDSM_ERR_INVALID;
    }
    return tc_status(h, st);
}

int asdsm_real_schur(int n, const double* A, double* Q, double* T) {
    if (n < 1 || n > 512 || !A || !Q || !T) return ASDSM_ERR_INVALID;
    std::vector<double> a(A, A + (size_t)n * n), q, t;
    if (!real_schur(n, a, &q, &t)) return ASDSM_ERR_INVALID;
    std::memcpy(Q, q.data(), q.size() * sizeof(double));
    std::memcpy(T, t.data(), t.size() * sizeof(double));
    return ASDSM_OK;
}

int asdsm_bcr_tail_map(int R, int C, const double* coef, int rt, double* D) {
    if (R < 1 || R > 32767 || C < 1 || C > 512 || rt < 1 || rt > R || (long long)rt * C > 8192 || !coef || !D)
        return ASDSM_ERR_INVALID;
    BcrFactors f;
    if (!make_bcr(R, coef[0], coef[1], coef[2], C, coef[3], coef[4], coef[5], &f)) return ASDSM_ERR_INVALID;
    std::vector<double> d;
    if (!bcr_tail_map(f, rt, &d)) return ASDSM_ERR_INVALID;
    std::memcpy(D, d.data(), d.size() * sizeof(double));
    return ASDSM_OK;
}

int asdsm_selftest_wait_timeout(asdsm_handle* h, long long limit_ns) {
    if (!h || limit_ns <= 0 || limit_ns > 2000000000LL) return ASDSM_ERR_INVALID;
    if (h->s3) { g_last_error = "not available for the 3D extension"; return ASDSM_ERR_INVALID; }
    CK(wait_selftest(h->dtcerr, limit_ns, h->st));
    return tc_status(h, h->st);
}

int asdsm_hole_extension_operator(int N, int mc, const double* alpha, const double* beta, double* G) {
    if (N < 3 || mc < 2 || !alpha || !beta || !G || (N - 1) % mc != 0) return ASDSM_ERR_INVALID;
    const int n = (N - 1) / mc;
    if (n < 2 || n > 32) return ASDSM_ERR_INVALID;
    const Stencil st = stencil_of(alpha[0], alpha[1], beta[0], beta[1], 1.0 / (N - 1));
    std::vector<double> g;
    if (!hole_extension_operator(n - 1, st, &g)) return ASDSM_ERR_INVALID;
    std::copy(g.begin(), g.end(), G);
    return ASDSM_OK;
}

int asdsm_hole_extension_operator_3d(int N, int mc, const double* alpha, const double* beta, double* G) {
    if (N < 3 || mc < 2 || !alpha || !beta || !G || (N - 1) % mc != 0) return ASDSM_ERR_INVALID;
    const int n = (N - 1) / mc;
    if (n < 2 || n > 32 || !(alpha[0] > 0) || !(alpha[1] > 0) || !(alpha[2] > 0)) return ASDSM_ERR_INVALID;
    const double hh = 1.0 / (N - 1);
    double s7[7];
    s7[0] = 2 * (alpha[0] + alpha[1] + alpha[2]) / (hh * hh);
    for (int a = 0; a < 3; ++a) {
        s7[1 + 2 * a] = -alpha[a] / (hh * hh) - beta[a] / (2 * hh);
        s7[2 + 2 * a] = -alpha[a] / (hh * hh) + beta[a] / (2 * hh);
    }
    std::vector<double> g;
    if (!hole_extension_operator_3d(n - 1, s7, &g)) return ASDSM_ERR_INVALID;
    std::copy(g.begin(), g.end(), G);
    return ASDSM_OK;
}

int asdsm_history(asdsm_handle* h, double* hist, int cap) {
    if (!h || (!hist && cap > 0)) return ASDSM_ERR_INVALID;
    if (h->s3) return s3_history(h->s3, hist, cap);
    const int n = std::min<int>(cap, (int)h->hist.size());
    for (int q = 0; q < n; ++q) hist[q] = h->hist[q];
    return n;
}

int asdsm_profile(asdsm_handle* h, int enable) {
    if (!h) return ASDSM_ERR_INVALID;
    if (h->s3) return s3_profile(h->s3, enable);
    h->prof = enable != 0;
    std::memset(h->pc, 0, sizeof(h->pc));
    for (int c = 0; c < PC_COUNT; ++c) std::snprintf(h->pc[c].name, sizeof(h->pc[c].name), "%s", kProfNames[c]);
    h->pend_ev.clear();
    h->evnext = 0;
    return ASDSM_OK;
}

int asdsm_profile_read(asdsm_handle* h, asdsm_kprof* out, int cap) {
    if (!h || (!out && cap > 0)) return ASDSM_ERR_INVALID;
    if (h->s3) return s3_profile_read(h->s3, out, cap);
    const int n = std::min<int>(cap, PC_COUNT);
    for (int c = 0; c < n; ++c) out[c] = h->pc[c];
    return n;
}

int64_t asdsm_launch_count(void) { return launch_count(); }

// ---------------------------------------------------------------------------
// Batches: independent instances on their own streams, advanced stage by
// stage in turn so that their kernels overlap on the GPU.
// ---------------------------------------------------------------------------
struct asdsm_batch {
    std::vector<asdsm_handle*> inst;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev_end;
    cudaEvent_t ev_start = nullptr;
    cudaStream_t caller = nullptr;
};

void asdsm_destroy_batch(asdsm_batch* b) {
    if (!b) return;
    for (auto* h : b->inst) asdsm_destroy(h);
    for (auto st : b->streams) if (st) cudaStreamDestroy(st);
    for (auto e : b->ev_end) if (e) cudaEventDestroy(e);
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    delete b;
}

int asdsm_setup_batch(const asdsm_desc* descs, int count, const asdsm_opts* opts, void* stream, asdsm_batch** out) {
    if (!out) return ASDSM_ERR_INVALID;
    *out = nullptr;
    if (!descs || count < 1) return ASDSM_ERR_INVALID;
    asdsm_batch* b = new asdsm_batch();
    b->caller = (cudaStream_t)stream;
    cudaError_t e = cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming);
    if (e != cudaSuccess) { asdsm_destroy_batch(b); return set_cuda_error(e); }
    for (int i = 0; i < count; ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
            asdsm_destroy_batch(b);
            return set_cuda_error(e);
        }
        b->streams.push_back(st);
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            asdsm_destroy_batch(b);
            return set_cuda_error(e);
        }
        b->ev_end.push_back(ev);
        asdsm_handle* h = nullptr;
        const int rc = asdsm_setup(&descs[i], opts, st, &h);
        if (rc != ASDSM_OK) { asdsm_destroy_batch(b); return rc; }
        b->inst.push_back(h);
    }
    *out = b;
    return ASDSM_OK;
}

int asdsm_batch_count(const asdsm_batch* b) { return b ? (int)b->inst.size() : 0; }

int asdsm_set_opts_batch(asdsm_batch* b, const asdsm_opts* opts) {
    if (!b) return ASDSM_ERR_INVALID;
    for (auto* h : b->inst)
        if (int rc = asdsm_set_opts(h, opts)) return rc;
    return ASDSM_OK;
}

int asdsm_autotune_batch(asdsm_batch* b, int precision) {
    if (!b) return ASDSM_ERR_INVALID;
    const int pi = precision == ASDSM_FP64 ? 0 : 1;
    // Launch shapes depend on the sizes only: tune one instance per (N, mc) class.
    for (size_t i = 0; i < b->inst.size(); ++i) {
        asdsm_handle* h = b->inst[i];
        asdsm_handle* src = nullptr;
        for (size_t j = 0; j < i; ++j)
            if (b->inst[j]->g.N == h->g.N && b->inst[j]->g.mc == h->g.mc) { src = b->inst[j]; break; }
        if (!src) {
            if (int rc = asdsm_autotune(h, precision)) return rc;
        } else {
            h->tune_aniso[pi] = src->tune_aniso[pi];
            h->tune_cc[pi] = src->tune_cc[pi];
            h->fill_warps[pi] = src->fill_warps[pi];
            if (pi == 1 && (tune_wants_tc(h->tune_aniso[1]) || tune_wants_tc(h->tune_cc[1])))
                if (int rc = ensure_tc_images(h)) return rc;
            destroy_graph(h);
        }
    }
    return ASDSM_OK;
}

}  // extern "C"
namespace {
template <typename T>
int batch_stage_begin(asdsm_handle* h, SolveRun& r) { return staged(r, [&] { return run_begin<T>(h, r); }); }
template <typename T>
int batch_stage_middle(asdsm_handle* h, SolveRun& r) { return staged(r, [&] { return run_middle<T>(h, r); }); }
template <typename T>
int batch_stage_poll(asdsm_handle* h, SolveRun& r) { return staged(r, [&] { return graph_poll<T>(h, r, false); }); }
template <typename T>
int batch_stage_finish(asdsm_handle* h, SolveRun& r) { return staged(r, [&] { return run_finish<T>(h, r); }); }
}  // namespace
extern "C" {

int asdsm_solve_batch(asdsm_batch* b, const double* const* s, double* const* u, asdsm_stats* stats) {
    if (!b || !s || !u) return ASDSM_ERR_INVALID;
    const size_t n = b->inst.size();
    for (size_t i = 0; i < n; ++i)
        if (!s[i] || !u[i]) return ASDSM_ERR_INVALID;
    CK(cudaEventRecord(b->ev_start, b->caller));
    // From here on every exit goes through the join below, so that the
    // caller's stream never runs ahead of work still queued on the instance
    // streams (which read s and write u), even after a CUDA error.
    int fail = ASDSM_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && fail == ASDSM_OK) fail = set_cuda_error(e);
        return fail == ASDSM_OK;
    };
    for (size_t i = 0; i < n; ++i) ok(cudaStreamWaitEvent(b->streams[i], b->ev_start, 0));
    std::vector<SolveRun> runs(n);
    std::vector<int> rcs(n, fail);
    auto is64 = [&](size_t i) { return b->inst[i]->opts.precision == ASDSM_FP64; };
    for (size_t i = 0; i < n && fail == ASDSM_OK; ++i) {
        runs[i].s = s[i]; runs[i].u = u[i]; runs[i].stats = stats ? &stats[i] : nullptr;
        rcs[i] = is64(i) ? batch_stage_begin<double>(b->inst[i], runs[i]) : batch_stage_begin<float>(b->inst[i], runs[i]);
    }
    for (size_t i = 0; i < n && fail == ASDSM_OK; ++i) {
        if (rcs[i] != ASDSM_OK) continue;
        if (!ok(cudaEventSynchronize(b->inst[i]->evA))) break;
        rcs[i] = is64(i) ? batch_stage_middle<double>(b->inst[i], runs[i]) : batch_stage_middle<float>(b->inst[i], runs[i]);
    }
    if (fail != ASDSM_OK)
        for (size_t i = 0; i < n; ++i)
            if (rcs[i] == ASDSM_OK) rcs[i] = fail;
    // Round-robin over the instances still sweeping; each poll launches up to
    // two graph replays ahead and retires completed ones without blocking.
    for (;;) {
        bool any = false;
        for (size_t i = 0; i < n; ++i) {
            if (rcs[i] != ASDSM_OK || runs[i].stage != 2) continue;
            any = true;
            rcs[i] = is64(i) ? batch_stage_poll<double>(b->inst[i], runs[i]) : batch_stage_poll<float>(b->inst[i], runs[i]);
        }
        if (!any) break;
    }
    int worst = ASDSM_OK;
    for (size_t i = 0; i < n; ++i) {
        int rc = rcs[i];
        if (rc == ASDSM_OK && runs[i].stage == 3)
            rc = is64(i) ? batch_stage_finish<double>(b->inst[i], runs[i]) : batch_stage_finish<float>(b->inst[i], runs[i]);
        else if (stats && rc != ASDSM_OK) { std::memset(&stats[i], 0, sizeof(asdsm_stats)); stats[i].status = rc; }
        if (rc != ASDSM_OK && worst == ASDSM_OK) worst = rc;
        ok(cudaEventRecord(b->ev_end[i], b->streams[i]));
        ok(cudaStreamWaitEvent(b->caller, b->ev_end[i], 0));
    }
    return fail != ASDSM_OK ? fail : worst;
}

int asdsm_batch_history(const asdsm_batch* b, int index, double* out, int cap) {
    if (!b || index < 0 || index >= (int)b->inst.size()) return ASDSM_ERR_INVALID;
    return asdsm_history(b->inst[index], out, cap);
}

void asdsm_destroy(asdsm_handle* h) {
    if (!h) return;
    if (h->s3) {
        s3_destroy(h->s3);
        delete h;
        return;
    }
    for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
    auto fr = [](void* p) { if (p) cudaFree(p); };
    for (int p = 0; p < 2; ++p) {
        DevBcr* ds[4] = {&h->fc[p], &h->cf[p], &h->cc[p], &h->hole[p]};
        for (auto* d : ds) { fr(d->Mt); fr(d->Bt); fr(d->Mw); fr(d->Bw); fr(d->Ti); fr(d->Dt); }
        fr(h->Sm[p]);
        auto& w = h->w[p];
        void* bufs[] = {w.Xfc, w.Xcf, w.Yfc, w.Ycf, w.Xcc, w.Ycc, w.E1, w.E2, w.M1, w.M2, w.rskel, w.q, w.rfull, w.zv};
        for (void* b : bufs) fr(b);
        for (int q = 0; q < w.nz; ++q) { fr(w.z[q]); fr(w.qp[q]); }
    }
    fr(h->u_work); fr(h->U[0]); fr(h->U[1]); fr(h->s_hi); fr(h->s_lo);
    fr(h->partials); fr(h->dsmall); fr(h->dflag); fr(h->dtcerr); fr(h->fill_tc_img);
    if (h->hsmall) cudaFreeHost(h->hsmall);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->ev2) cudaEventDestroy(h->ev2);
    if (h->evA) cudaEventDestroy(h->evA);
    fr(h->cnn_x); fr(h->cnn_y);
    destroy_graph(h);
    fr(h->dctl); fr(h->dhist);
    if (h->hctl) cudaFreeHost(h->hctl);
    if (h->hdone) cudaFreeHost(h->hdone);
    for (int q = 0; q < 2; ++q) if (h->evc[q]) cudaEventDestroy(h->evc[q]);
    if (h->cap_st) cudaStreamDestroy(h->cap_st);
    if (h->body_st) cudaStreamDestroy(h->body_st);
    delete h;
}

}  // extern "C"
