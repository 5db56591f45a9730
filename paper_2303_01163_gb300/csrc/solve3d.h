// Internal interface of the 3D extension (solve3d.cu) to the C ABI (api.cu).
#pragma once
#include "asdsm.h"
#include <cuda_runtime.h>
#include <string>

namespace asdsm {

struct Solver3D;

// Sizes accepted in 3D: N - 1 and mc powers of two, 2 <= mc <= 32,
// 2 <= n = (N-1)/mc <= 16, N <= 257.
int s3_create(const asdsm_desc* d, const asdsm_opts* o, cudaStream_t st, Solver3D** out);
int s3_set_opts(Solver3D* S, const asdsm_opts* o);
int s3_solve(Solver3D* S, const double* s, double* u, asdsm_stats* stats);
int s3_initial_guess(Solver3D* S, const double* s, double* u);
int s3_residual(Solver3D* S, const double* s, const double* u, double* r, double* rel);
int s3_submesh_solve(Solver3D* S, int mesh, const double* in, double* out);
int s3_history(Solver3D* S, double* hist, int cap);
int s3_profile(Solver3D* S, int enable);
int s3_profile_read(Solver3D* S, asdsm_kprof* out, int cap);
void s3_destroy(Solver3D* S);

// Error reporting shared with api.cu (asdsm_last_error).
int report_cuda_error(cudaError_t e);
void report_error(const std::string& msg);

}  // namespace asdsm
