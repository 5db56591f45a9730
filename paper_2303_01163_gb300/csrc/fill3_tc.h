// The 3D sweeps' homogeneous cube-hole Filler on the tensor cores (fill3_tc.cu).
#pragma once
#include <cuda_runtime.h>
#include <vector>

namespace asdsm {

struct Fill3TcArgs {
    const float* z;       // FP32 grid (N^3): the faces are read from it
    float* zout;          // the same grid: the hole values are written into it
    const float* gimg;    // G^T image (fill3_tc_gimage), 16-byte aligned
    float* aimg;          // face image scratch, fill3_tc_image_floats(H, K) floats, zeroed once
    int N, mc, n, hc;     // grid points per axis, coarse intervals, hole spacing, C = n - 1
    int P, K, H;          // C^3 hole points, 6 C^2 face values, mc^3 holes
    int KC, PT, HT;       // K chunks of 32, point tiles and hole tiles of 128
    int* err;             // set to 1 when a bounded wait timed out
};

// Floats of an operand image of `rows` rows (points or holes) and K face values.
size_t fill3_tc_image_floats(int rows, int K);
// G (P x K, row-major FP64) as the B image: split, swizzled, padded with zeros.
void fill3_tc_gimage(const std::vector<double>& G, int P, int K, std::vector<float>* img);
// Gather the faces of every hole into the A image and write G f into the holes.
cudaError_t fill3_tc(const Fill3TcArgs& a, cudaStream_t st);

}  // namespace asdsm
