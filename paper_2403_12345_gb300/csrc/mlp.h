// Importance-network kernels (defined in mlp.cu).
#pragma once

#include <cuda_bf16.h>

#include "device.cuh"

namespace gbmc {

constexpr int kMlpHidden = 64;
constexpr int kMlpParams = kMlpHidden * 4 + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden +
                           kMlpHidden + 1;

// Mesh of a geometry's cells x the tally's energy bins, and the affine map
// from (x, y, z, ln E) to the network's features.
struct MeshSpec {
    gbmc_geometry g;
    int32_t n_cells, n_bins;
    const double* edges;   // device, [n_bins + 1]
    double offset[4], scale[4];
};

// Network output for n feature rows (feat [n][4]) with BF16 weights w, on
// the tensor cores; *err (device) is set to 1 if a wait for the tensor cores
// gave up.
cudaError_t mlp_forward(const __nv_bfloat16* w, const float* feat, int64_t n, float* out,
                        int* err, int sms, cudaStream_t s);

// Adds the gradient of the weighted mean squared error to grad and the loss
// to *loss (both device, fp32); scratch_inv receives 1 / sum of weights.
cudaError_t mlp_grad(const __nv_bfloat16* w, const float* feat, const float* y, const float* wt,
                     int64_t n, float* scratch_inv, float* grad, float* loss, int sms,
                     cudaStream_t s);

// One Adam step (step counts from 1); refreshes w, clears grad.
cudaError_t mlp_adam(float* p, float* m, float* v, float* grad, __nv_bfloat16* w, int n, float lr,
                     int step, cudaStream_t s);

// Window lower bounds on the mesh from the network (features and outputs go
// through feat [n][4] and out [n]); src is the source's mesh index.
cudaError_t mesh_windows(const MeshSpec& M, const __nv_bfloat16* w, float* feat, float* out,
                         double survival, int64_t src, double* lower, int* err, int sms,
                         cudaStream_t s);

// Mesh features only.
cudaError_t mesh_features(const MeshSpec& M, float* feat, int sms, cudaStream_t s);

}  // namespace gbmc
