// asdsm_residual_noalloc: the fine residual and its relative norm without any
// device allocation, for callers that cannot call cudaMalloc.
//
// Some callers cannot allocate device memory at the moment they need the
// residual: services whose device memory is reserved up front by their own
// pool allocator (a cudaMalloc beside the pool can fail, or fragment what the
// pool expects to own), and tight loops where an allocation would stall or
// synchronise the device.  This entry point needs no handle (creating one
// allocates) and uses, for its only scratch - the per-block partial sums of
// the norms and their totals - arrays that live in this file as statically
// allocated device memory.  Every GPU that loads the library keeps these
// arrays (about 1 MiB) until the process exits.
//
// The host cannot pass the arrays' names to a kernel: in host code a
// __device__ variable's name is only a host-side stand-in for the symbol, not
// a device address.  The device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, the first
// time the entry point runs on it; that first call should therefore happen
// before any stream capture.
//
// All calls share the arrays and each call overwrites every slot it later
// reads (nothing accumulates across calls, so nothing needs clearing), which
// also means that calls whose work overlaps on the GPU - on two streams, or
// from two host threads - race with each other.
#include "asdsm.h"
#include "asdsm_internal.h"
#include <cuda_runtime.h>
#include <cmath>
#include <mutex>
#include <string>

namespace {

constexpr int NA_RX = 64;
constexpr int NA_RY = 16;
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_N = 8193;   // grid points per axis
constexpr int NA_MAX_BLOCKS = ((NA_MAX_N - 2 + NA_RX - 1) / NA_RX) * ((NA_MAX_N - 2 + NA_RY - 1) / NA_RY);

// The statically allocated scratch: [block][2] partial sums and their totals.
static __device__ __align__(256) double g_noalloc_partials[2 * NA_MAX_BLOCKS];
static __device__ __align__(256) double g_noalloc_totals[2];

struct DeviceScratch {
    double* partials = nullptr;
    double* totals = nullptr;
    bool ready = false;
};
constexpr int kMaxDevices = 64;
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;
thread_local std::string g_na_error;

__device__ __forceinline__ double na_warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// r = s - A u over the interior (u's ring carries g) and b = s - A (ring of u,
// zero interior) = b_ff of Section 2.3; per block: sum r^2 and sum b^2.
__global__ void __launch_bounds__(NA_THREADS)
residual_norms_kernel(const double* __restrict__ s, const double* __restrict__ u, double* __restrict__ r,
                      int N, asdsm::Stencil c, double* __restrict__ partials) {
    __shared__ double tile[NA_RY + 2][NA_RX + 2];
    __shared__ double red[2][NA_THREADS / 32];
    const int i0 = blockIdx.x * NA_RX + 1, j0 = blockIdx.y * NA_RY + 1;
    for (int e = threadIdx.x; e < (NA_RX + 2) * (NA_RY + 2); e += NA_THREADS) {
        const int ty = e / (NA_RX + 2), tx = e % (NA_RX + 2);
        const int i = i0 - 1 + tx, j = j0 - 1 + ty;
        tile[ty][tx] = (i <= N - 1 && j <= N - 1) ? u[(long long)j * N + i] : 0.0;
    }
    __syncthreads();
    double sr = 0.0, sb = 0.0;
    for (int e = threadIdx.x; e < NA_RX * NA_RY; e += NA_THREADS) {
        const int ty = e / NA_RX, tx = e % NA_RX;
        const int i = i0 + tx, j = j0 + ty;
        if (i > N - 2 || j > N - 2) continue;
        const long long idx = (long long)j * N + i;
        const double uc = tile[ty + 1][tx + 1];
        const double uw = tile[ty + 1][tx], ue = tile[ty + 1][tx + 2];
        const double us = tile[ty][tx + 1], un = tile[ty + 2][tx + 1];
        const double Au = c.cc * uc + c.cw * uw + c.ce * ue + c.cs * us + c.cn * un;
        const double rv = s[idx] - Au;
        // Lifting of the Dirichlet data: only neighbours on the ring contribute.
        double lift = 0.0;
        if (i == 1) lift += c.cw * uw;
        if (i == N - 2) lift += c.ce * ue;
        if (j == 1) lift += c.cs * us;
        if (j == N - 2) lift += c.cn * un;
        const double bv = s[idx] - lift;
        sr += rv * rv;
        sb += bv * bv;
        if (r) r[idx] = rv;
    }
    sr = na_warp_sum(sr);
    sb = na_warp_sum(sb);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][w] = sr; red[1][w] = sb; }
    __syncthreads();
    if (w == 0) {
        sr = lane < NA_THREADS / 32 ? red[0][lane] : 0.0;
        sb = lane < NA_THREADS / 32 ? red[1][lane] : 0.0;
        sr = na_warp_sum(sr);
        sb = na_warp_sum(sb);
        if (lane == 0) {
            const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
            partials[2 * blk] = sr;
            partials[2 * blk + 1] = sb;
        }
    }
}

// 3D (the 7-point operator of the 3D extension): the same two quantities,
// one interior point per thread in a grid-strided loop over the N_f^3 points
// (x fastest); neighbours come from L1/L2.
struct Stencil7 {
    double cc, cw, ce, cs, cn, cd, cu;    // centre; x-1, x+1; y-1, y+1; z-1, z+1
};
constexpr int NA3_BLOCKS = 152 * 8;
constexpr int NA3_MAX_N = 2049;
static_assert(NA3_BLOCKS <= NA_MAX_BLOCKS, "3D partials fit the scratch");

__global__ void __launch_bounds__(NA_THREADS)
residual_norms_3d_kernel(const double* __restrict__ s, const double* __restrict__ u, double* __restrict__ r,
                         int N, Stencil7 c, double* __restrict__ partials) {
    __shared__ double red[2][NA_THREADS / 32];
    const long long Nf = N - 2, total = Nf * Nf * Nf;
    const long long sy = N, sz = (long long)N * N;
    double sr = 0.0, sb = 0.0;
    for (long long e = blockIdx.x * (long long)NA_THREADS + threadIdx.x; e < total; e += (long long)gridDim.x * NA_THREADS) {
        const int i = (int)(e % Nf) + 1;
        const long long t = e / Nf;
        const int j = (int)(t % Nf) + 1, l = (int)(t / Nf) + 1;
        const long long idx = (l * sy + j) * (long long)N + i;
        const double uc = u[idx];
        const double uw = u[idx - 1], ue = u[idx + 1];
        const double us = u[idx - sy], un = u[idx + sy];
        const double ud = u[idx - sz], uu = u[idx + sz];
        const double Au = c.cc * uc + c.cw * uw + c.ce * ue + c.cs * us + c.cn * un + c.cd * ud + c.cu * uu;
        const double rv = s[idx] - Au;
        double lift = 0.0;                        // Dirichlet lifting: neighbours on the boundary
        if (i == 1) lift += c.cw * uw;
        if (i == N - 2) lift += c.ce * ue;
        if (j == 1) lift += c.cs * us;
        if (j == N - 2) lift += c.cn * un;
        if (l == 1) lift += c.cd * ud;
        if (l == N - 2) lift += c.cu * uu;
        const double bv = s[idx] - lift;
        sr += rv * rv;
        sb += bv * bv;
        if (r) r[idx] = rv;
    }
    sr = na_warp_sum(sr);
    sb = na_warp_sum(sb);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][w] = sr; red[1][w] = sb; }
    __syncthreads();
    if (w == 0) {
        sr = lane < NA_THREADS / 32 ? red[0][lane] : 0.0;
        sb = lane < NA_THREADS / 32 ? red[1][lane] : 0.0;
        sr = na_warp_sum(sr);
        sb = na_warp_sum(sb);
        if (lane == 0) {
            partials[2 * blockIdx.x] = sr;
            partials[2 * blockIdx.x + 1] = sb;
        }
    }
}

// Fixed-order sum of the block partials into totals[0..1].
__global__ void totals_kernel(const double* __restrict__ partials, int nblocks, double* __restrict__ totals) {
    __shared__ double red[2][32];
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
        a += partials[2 * q];
        b += partials[2 * q + 1];
    }
    a = na_warp_sum(a);
    b = na_warp_sum(b);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][w] = a; red[1][w] = b; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? red[0][lane] : 0.0;
        b = lane < nw ? red[1][lane] : 0.0;
        a = na_warp_sum(a);
        b = na_warp_sum(b);
        if (lane == 0) { totals[0] = a; totals[1] = b; }
    }
}

// Device address of the scratch for the current device (looked up once).
int scratch_for_current_device(DeviceScratch** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { g_na_error = cudaGetErrorString(e); return ASDSM_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) { g_na_error = "device ordinal out of range"; return ASDSM_ERR_INVALID; }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    DeviceScratch& d = g_scratch[dev];
    if (!d.ready) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) { g_na_error = cudaGetErrorString(e); return ASDSM_ERR_CUDA; }
        d.partials = static_cast<double*>(p);
        e = cudaGetSymbolAddress(&p, g_noalloc_totals);
        if (e != cudaSuccess) { g_na_error = cudaGetErrorString(e); return ASDSM_ERR_CUDA; }
        d.totals = static_cast<double*>(p);
        d.ready = true;
    }
    *out = &d;
    return ASDSM_OK;
}

}  // namespace

extern "C" {

int asdsm_residual_noalloc(const asdsm_desc* desc, const double* s, const double* u, double* r,
                           double* rel_norm, void* stream) {
    g_na_error.clear();
    if (!desc || !s || !u) { g_na_error = "null argument"; return ASDSM_ERR_INVALID; }
    if (desc->d != 2 && desc->d != 3) { g_na_error = "d must be 2 or 3"; return ASDSM_ERR_INVALID; }
    const int N = desc->n;
    const bool d3 = desc->d == 3;
    if (N < 3) { g_na_error = "grid needs at least 3 points per axis"; return ASDSM_ERR_INVALID; }
    if (N > (d3 ? NA3_MAX_N : NA_MAX_N)) {
        g_na_error = d3 ? "3D grid larger than 2049 points per axis"
                        : "grid larger than the statically allocated scratch allows (at most 8193 points per axis)";
        return ASDSM_ERR_INVALID;
    }
    if (!(desc->alpha[0] > 0) || !(desc->alpha[1] > 0) || (d3 && !(desc->alpha[2] > 0))) {
        g_na_error = "alpha must be positive";
        return ASDSM_ERR_INVALID;
    }
    DeviceScratch* sc = nullptr;
    int rc = scratch_for_current_device(&sc);
    if (rc != ASDSM_OK) return rc;
    const double h = 1.0 / (N - 1);
    if (d3) {
        const double* al = desc->alpha;
        const double* be = desc->beta;
        Stencil7 c7;
        c7.cc = 2 * (al[0] + al[1] + al[2]) / (h * h);
        c7.cw = -al[0] / (h * h) - be[0] / (2 * h);
        c7.ce = -al[0] / (h * h) + be[0] / (2 * h);
        c7.cs = -al[1] / (h * h) - be[1] / (2 * h);
        c7.cn = -al[1] / (h * h) + be[1] / (2 * h);
        c7.cd = -al[2] / (h * h) - be[2] / (2 * h);
        c7.cu = -al[2] / (h * h) + be[2] / (2 * h);
        cudaStream_t st3 = (cudaStream_t)stream;
        const long long Nf = N - 2, total = Nf * Nf * Nf;
        long long nb = (total + NA_THREADS - 1) / NA_THREADS;
        const int nblocks = (int)(nb < NA3_BLOCKS ? nb : NA3_BLOCKS);
        residual_norms_3d_kernel<<<nblocks, NA_THREADS, 0, st3>>>(s, u, r, N, c7, sc->partials);
        cudaError_t e3 = cudaGetLastError();
        if (e3 != cudaSuccess) { g_na_error = cudaGetErrorString(e3); return ASDSM_ERR_CUDA; }
        totals_kernel<<<1, 1024, 0, st3>>>(sc->partials, nblocks, sc->totals);
        e3 = cudaGetLastError();
        if (e3 != cudaSuccess) { g_na_error = cudaGetErrorString(e3); return ASDSM_ERR_CUDA; }
        if (rel_norm) {
            double tot[2] = {0.0, 0.0};
            e3 = cudaMemcpyAsync(tot, sc->totals, sizeof(tot), cudaMemcpyDeviceToHost, st3);
            if (e3 == cudaSuccess) e3 = cudaStreamSynchronize(st3);
            if (e3 != cudaSuccess) { g_na_error = cudaGetErrorString(e3); return ASDSM_ERR_CUDA; }
            *rel_norm = tot[1] > 0 ? std::sqrt(tot[0] / tot[1]) : std::sqrt(tot[0]);
        }
        return ASDSM_OK;
    }
    const double ax = desc->alpha[0], ay = desc->alpha[1], bx = desc->beta[0], by = desc->beta[1];
    asdsm::Stencil c;
    c.cc = 2 * ax / (h * h) + 2 * ay / (h * h);
    c.cw = -ax / (h * h) - bx / (2 * h);
    c.ce = -ax / (h * h) + bx / (2 * h);
    c.cs = -ay / (h * h) - by / (2 * h);
    c.cn = -ay / (h * h) + by / (2 * h);
    cudaStream_t st = (cudaStream_t)stream;
    const int Nf = N - 2;
    dim3 grid((Nf + NA_RX - 1) / NA_RX, (Nf + NA_RY - 1) / NA_RY);
    const int nblocks = (int)(grid.x * grid.y);
    residual_norms_kernel<<<grid, NA_THREADS, 0, st>>>(s, u, r, N, c, sc->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { g_na_error = cudaGetErrorString(e); return ASDSM_ERR_CUDA; }
    totals_kernel<<<1, 1024, 0, st>>>(sc->partials, nblocks, sc->totals);
    e = cudaGetLastError();
    if (e != cudaSuccess) { g_na_error = cudaGetErrorString(e); return ASDSM_ERR_CUDA; }
    if (rel_norm) {
        double tot[2] = {0.0, 0.0};     // pageable host memory: the copy completes before it returns
        e = cudaMemcpyAsync(tot, sc->totals, sizeof(tot), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { g_na_error = cudaGetErrorString(e); return ASDSM_ERR_CUDA; }
        *rel_norm = tot[1] > 0 ? std::sqrt(tot[0] / tot[1]) : std::sqrt(tot[0]);
    }
    return ASDSM_OK;
}

const char* asdsm_noalloc_last_error(void) { return g_na_error.c_str(); }

}  // extern "C"
