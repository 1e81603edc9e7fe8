// mlp_internal.h -- launchers of the flow-map surrogate (training and inference).
#pragma once

#include "gals_internal.h"
#include "mlp.cuh"

namespace gals {
namespace mlp {

// Inference weights: 16-bit copies (FP16; BF16 in a build with GALS_MLP_F16=0) laid out
// for the tensor-core kernel, and the output de-normalisation.
// Each weight matrix (N units x K inputs) is stored as the tensor core's K-major operand
// in the no-swizzle core-matrix layout (8 x 8 16-bit blocks of 128 bytes).  Biases enter the
// products as one more K-slab: bias column k = 0 of a 16-wide slab times a constant block
// whose column 0 is 1 (layer 1 uses input column 3 = 1 instead).  Hidden layers (weights
// and biases) are pre-scaled by 1/2, exact in FP16 and BF16, so their accumulators hold z/2.
struct InferParams {
    uint16_t *w;        // packed 16-bit operands, W_TOTAL elements (offsets below)
    float scale[OUT];   // output k of the network times scale[k] is the physical target
};
constexpr int64_t W1_OFF = 0,                          // 128 x 16: W1/2 (inputs 0..2), b1/2 (column 3)
                  W2_OFF = W1_OFF + 128 * 16,          // 3 x (128 x 128): W2/2, W3/2, W4/2
                  W5_OFF = W2_OFF + 3 * 128 * 128,     // 16 x 128: W5 (rows 6..15 zero)
                  WB_OFF = W5_OFF + 16 * 128,          // 3 x (128 x 16): b2/2, b3/2, b4/2 in column 0
                  W5B_OFF = WB_OFF + 3 * 128 * 16,     // 16 x 16: b5 in column 0
                  ONES_OFF = W5B_OFF + 16 * 16,        // 128 x 16: 1 in column 0
                  W_TOTAL = ONES_OFF + 128 * 16;

// Residual check of the surrogate trace (per 128-node tile, `samples` nodes against the
// exact RK3 trace): a tile fails when |delta_mlp - delta_rk3|_inf > tol_x cells or
// |J_mlp - J_rk3|_inf > tol_J; failed tiles are recomputed with RK3.
struct Check {
    float tol_x, tol_J;
    int samples;
    unsigned long long *tiles, *fallbacks;  // device counters
    int *err;                               // device error word (bounded waits)
};

__device__ void flowmap_rk4(const VelParams &vp, float x, float y, float t, float dt, int m,
                            float d[2], float J[4]);

cudaError_t launch_targets(const VelParams &vp, const float *X, float *T, int n, float dt, float h,
                           int substeps, cudaStream_t s);
cudaError_t launch_samples(const VelParams &vp, float *Xn, float *T, int n, float dt, float h,
                           int substeps, uint64_t seed, uint64_t step, const float *scale,
                           cudaStream_t s);
// Training products on the tensor cores; a product that does not complete in time sets *err.
cudaError_t forward_train(const float *params, const float *X, int n, float *const *Z,
                          float *const *A, int *err, cudaStream_t s);
// split: kMaxSplit * 128 * 128 floats of split-K partials
constexpr int kMaxSplit = 128;
cudaError_t backward_train(const float *params, const float *X, const float *T, int n,
                           float *const *Z, float *const *A, float *G0, float *G1, float *grad,
                           double *loss, const float *one, float *split, int *err, cudaStream_t s);
cudaError_t adam_step(float *params, const float *grad, float *m, float *v, float lr, float b1,
                      float b2, float eps, int step, cudaStream_t s);
// FP32 master parameters -> inference layout
cudaError_t pack_infer(const float *params, InferParams &ip, cudaStream_t s);
// Network outputs (normalised) for n inputs in [-1,1]^3 with the tensor-core kernel; a
// product that does not complete in time sets *err.
cudaError_t infer_points(const InferParams &ip, const float *Xn, float *Y, int n, int *err,
                         cudaStream_t s);
// Surrogate trace of one step over a 2D grid: planes (dx, dy, J00, J01, J10, J11) with the
// grid's pitch and plane stride, into `trace`; `coef` = this step's stage coefficients.
cudaError_t launch_mlp_trace(const InferParams &ip, const Geom &g, const VelParams &vp,
                             const StageCoef *coef, const double *t_dev, int kstep, double dt,
                             float *trace, const Check &chk, cudaStream_t s);

}  // namespace mlp
}  // namespace gals
