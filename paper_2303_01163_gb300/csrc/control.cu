// Sweep control of Algorithm 4 on the device.
//
// These single-thread kernels take, between the kernels of a sweep, the
// decisions the host loop of api.cu takes between sweeps, in the same order and
// FP64 arithmetic: the stopping tests of Algorithm 4 (tolerance, sweep limit,
// stagnation), the hole-residual correction (Proposition 3.1: after an exact
// Filler the residual vanishes in the holes, so a large hole residual is
// rounding to be removed by one more Filler), and the step lengths of Algorithm 4
// (the clamped s_hat, or the GCR(m) least squares over the cycle's
// directions).  With them a run of sweeps is a fixed sequence of launches that
// a CUDA graph replays; the branch taken by a sweep (new direction in slot kc,
// hole correction, or nothing once the solve has ended) is selected through
// the graph's switch node.
#include "asdsm.h"
#include "asdsm_internal.h"
#include <cuda_runtime.h>

namespace asdsm {

namespace {

__device__ unsigned long long splitmix64_dev(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Coin of the random choice of Algorithm 2 at sweep k: top bit of SplitMix64 output k.
__device__ int choice_bit_dev(unsigned long long seed, int k) {
    const unsigned long long state = seed + (unsigned long long)(k + 1) * 0x9E3779B97F4A7C15ULL;
    return (int)(splitmix64_dev(state) >> 63);
}

__device__ void finish(SweepCtl* c, int status, cudaGraphConditionalHandle sw) {
    c->status = status;
    c->done = 1;
    c->upd.live = 0;
    c->branch = c->m + 2;
    cudaGraphSetConditional(sw, (unsigned)(c->m + 2));
}

__global__ void ctl_after_residual_kernel(SweepCtl* c, const double* __restrict__ sums, int* overflow,
                                          double* hist, cudaGraphConditionalHandle sw) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (c->done) {
        cudaGraphSetConditional(sw, (unsigned)(c->m + 2));
        return;
    }
    c->comb.run = 0;
    c->comb.track = 0;
    const bool tracked = c->upd.skip != 0;
    double rel, rnorm = 0.0, hnorm = 0.0;
    if (!tracked) {
        // The residual kernel has applied the pending update into the other buffer.
        if (c->upd.count > 0) c->upd.par ^= 1;
        c->upd.count = 0;
        if (c->mixed) {
            const int ovf = *overflow;
            *overflow = 0;
            if (ovf) { finish(c, ASDSM_ERR_RANGE, sw); return; }
        }
        rnorm = sqrt(sums[0]);
        hnorm = sqrt(sums[1]);
        rel = c->bnorm > 0 ? rnorm / c->bnorm : rnorm;
        if (c->defer && c->cycle_ended) {
            // The cycle's tracked prediction of this residual against the true one.
            const double p2 = fmax(c->rr_skel, 0.0) + c->rh2;
            const double pred = c->bnorm > 0 ? sqrt(p2) / c->bnorm : sqrt(p2);
            if (rel > 2.0 * pred) { c->defer = 0; c->stag_hold = c->window; }
        }
        if (c->defer && rel < kDeferStop * c->tol) c->defer = 0;
        c->cycle_ended = 0;
        c->rr_skel = sums[0] - sums[1];
        c->rh2 = sums[1];
    } else {
        // Inside a deferred GCR cycle: the residual of the virtual iterate, tracked.
        const double r2 = fmax(c->rr_skel, 0.0) + c->rh2;
        rel = c->bnorm > 0 ? sqrt(r2) / c->bnorm : sqrt(r2);
        const int win = c->window;
        const bool stag = win > 0 && c->nhist > win && c->nhist <= c->hist_cap &&
                          rel > (1.0 - c->stagnation_factor) * hist[c->nhist - 1 - win];
        if (!(rel > c->tol) || c->k >= c->max_sweeps || stag) {
            // End the cycle here: its update is applied by the next residual kernel,
            // whose true residual (replacing this tracked value) takes the decision.
            c->upd.count = c->kc;
            for (int i = 0; i < c->kc; ++i) {
                c->upd.coef[i] = c->cacc[i];
                c->upd.cf[i] = (float)(c->cacc[i] * c->scale);
                c->cacc[i] = 0.0;
            }
            c->upd.skip = 0;
            c->cycle_ended = c->kc > 0;
            c->kc = 0;
            c->branch = c->m + 2;
            cudaGraphSetConditional(sw, (unsigned)(c->m + 2));
            return;
        }
    }
    c->rel = rel;
    if (!isfinite(rel)) { finish(c, ASDSM_ERR_NAN, sw); return; }
    if (c->nhist < c->hist_cap) hist[c->nhist] = rel;
    c->nhist += 1;
    if (c->k == 0) c->rel0 = rel;
    if (!tracked) {
        if (rel <= c->tol) { finish(c, ASDSM_OK, sw); return; }
        if (c->k >= c->max_sweeps) { finish(c, ASDSM_NOT_CONVERGED, sw); return; }
        const int win = c->window;
        if (c->stag_hold > 0) {
            c->stag_hold -= 1;
        } else if (win > 0 && c->nhist > win && c->nhist <= c->hist_cap &&
                   rel > (1.0 - c->stagnation_factor) * hist[c->nhist - 1 - win]) {
            finish(c, ASDSM_STAGNATED, sw);
            return;
        }
        if (c->hole_ref_pending) { c->hole_ref = hnorm; c->hole_ref_pending = 0; }
    }
    int branch;
    if (!tracked && hnorm > c->hole_fix_ratio * rnorm && hnorm > c->hole_fix_growth * c->hole_ref) {
        branch = c->m + c->upd.par;      // hole correction on the current iterate buffer
        c->hole_fixes += 1;
        c->kc = 0;
        c->hole_ref_pending = 1;
        c->k += 1;
    } else {
        branch = c->kc;                  // error guess into direction slot kc
        c->choice = choice_bit_dev(c->seed, c->k);
    }
    c->branch = branch;
    if (branch < 20) c->runs[branch] += 1;
    cudaGraphSetConditional(sw, (unsigned)branch);
}

__global__ void ctl_after_dots_kernel(SweepCtl* c, const double* __restrict__ dots) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || c->done) return;
    const int m = c->m, kc = c->kc;
    const double qq = dots[0], qr = dots[1];
    c->comb.run = 0;
    if (m == 1) {
        // The paper's clamped optimal scaling: s_hat = argmin_{s >= 0} ||r - s A e||.
        const double shat = qq > 0 ? fmax(0.0, qr / qq) : 0.0;
        c->upd.count = 1;
        c->upd.coef[0] = shat;
        c->upd.cf[0] = (float)(shat * c->scale);
        c->k += 1;
        return;
    }
    // GCR(m): orthogonalise A e against the cycle's previous directions.
    double beta[16], rq[16];
    double nu2 = qq;
    for (int j = 0; j < kc; ++j) {
        beta[j] = dots[2 + 2 * j];
        rq[j] = dots[3 + 2 * j];
        nu2 -= beta[j] * beta[j];
    }
    // The cycle's update so far goes to the next residual kernel.
    auto end_cycle = [&](int count) {
        c->upd.count = count;
        for (int i = 0; i < count; ++i) {
            c->upd.coef[i] = c->cacc[i];
            c->upd.cf[i] = (float)(c->cacc[i] * c->scale);
            c->cacc[i] = 0.0;
        }
        c->upd.skip = 0;
        c->cycle_ended = count > 0;
        c->kc = 0;
    };
    if (!(nu2 > 1e-24 * qq) || !(qq > 0)) {
        if (c->defer) end_cycle(kc);     // dependent direction: restart the cycle
        c->kc = 0;
        c->k += 1;
        return;
    }
    const double nu = sqrt(nu2);
    double alpha = qr;
    for (int j = 0; j < kc; ++j) alpha -= beta[j] * rq[j];
    alpha /= nu;
    // Column kc of T: z'_kc = sum_i T[i][kc] z_i; the cycle's update is
    // sum_k alpha_k z'_k = sum_i cacc_i z_i, applied when the cycle ends.
    for (int i = 0; i <= kc; ++i) c->Tm[i][kc] = 0.0;
    c->Tm[kc][kc] = 1.0 / nu;
    for (int j = 0; j < kc; ++j)
        for (int i = 0; i <= j; ++i) c->Tm[i][kc] -= beta[j] * c->Tm[i][j] / nu;
    c->comb.run = 1;
    for (int j = 0; j < kc; ++j) {
        c->comb.beta[j] = beta[j];
        c->comb.beta_f[j] = (float)beta[j];
    }
    c->comb.inv_nu = 1.0 / nu;
    c->comb.alpha = alpha;
    c->comb.inv_nu_f = (float)c->comb.inv_nu;
    c->comb.alpha_f = (float)alpha;
    c->k += 1;
    if (!c->defer) {
        // The step goes to u at the next residual kernel; the cycle continues.
        c->upd.count = kc + 1;
        for (int i = 0; i <= kc; ++i) {
            const double v = alpha * c->Tm[i][kc];
            c->upd.coef[i] = v;
            c->upd.cf[i] = (float)(v * c->scale);
        }
        c->upd.skip = 0;
        c->kc = kc + 1 >= m ? 0 : kc + 1;
        return;
    }
    for (int i = 0; i <= kc; ++i) c->cacc[i] += alpha * c->Tm[i][kc];
    c->rr_skel -= alpha * alpha;         // ||r - alpha z'||^2 for the orthonormal image of z'
    if (kc + 1 >= m) {
        end_cycle(kc + 1);
    } else {
        c->upd.count = 0;
        c->upd.skip = 1;
        c->comb.track = 1;
        c->kc = kc + 1;
    }
}

}  // namespace

cudaError_t ctl_after_residual(SweepCtl* c, const double* sums, int* overflow, double* hist,
                               cudaGraphConditionalHandle sw, cudaStream_t st) {
    ctl_after_residual_kernel<<<1, 32, 0, st>>>(c, sums, overflow, hist, sw);
    note_launch();
    return cudaGetLastError();
}

cudaError_t ctl_after_dots(SweepCtl* c, const double* dots, cudaStream_t st) {
    ctl_after_dots_kernel<<<1, 32, 0, st>>>(c, dots);
    note_launch();
    return cudaGetLastError();
}

}  // namespace asdsm
