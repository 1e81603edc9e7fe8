// mlp_internal.h -- launchers of the flow-map surrogate (training and inference).
#pragma once

#include "gals_internal.h"
#include "mlp.cuh"

namespace gals {
namespace mlp {

// Inference weights: BF16 copies laid out for the tensor-core kernel, FP32 biases and
// the output de-normalisation.
struct InferParams {
    __nv_bfloat16 *w;   // W1 [128][16] (K padded), W2..W4 [128][128], W5 [8][128] (N padded)
    float *b;           // b1..b4 [128 each], b5 [8]
    float scale[OUT];   // output k of the network times scale[k] is the physical target
};
constexpr int64_t W1_OFF = 0, W2_OFF = 128 * 16, W3_OFF = W2_OFF + 128 * 128,
                  W4_OFF = W3_OFF + 128 * 128, W5_OFF = W4_OFF + 128 * 128,
                  W_TOTAL = W5_OFF + 8 * 128;
constexpr int B_TOTAL = 4 * 128 + 8;

// Residual check of the surrogate trace (per 128-node tile, `samples` nodes against the
// exact RK3 trace): a tile fails when |delta_mlp - delta_rk3|_inf > tol_x cells or
// |J_mlp - J_rk3|_inf > tol_J; failed tiles are recomputed with RK3.
struct Check {
    float tol_x, tol_J;
    int samples;
    unsigned long long *tiles, *fallbacks;  // device counters
};

__device__ void flowmap_rk4(const VelParams &vp, float x, float y, float t, float dt, int m,
                            float d[2], float J[4]);

cudaError_t launch_targets(const VelParams &vp, const float *X, float *T, int n, float dt, float h,
                           int substeps, cudaStream_t s);
cudaError_t launch_samples(const VelParams &vp, float *Xn, float *T, int n, float dt, float h,
                           int substeps, uint64_t seed, uint64_t step, const float *scale,
                           cudaStream_t s);
cudaError_t forward_train(const float *params, const float *X, int n, float *const *Z,
                          float *const *A, cudaStream_t s);
cudaError_t backward_train(const float *params, const float *X, const float *T, int n,
                           float *const *Z, float *const *A, float *G0, float *G1, float *grad,
                           double *loss, const float *one, float *split, cudaStream_t s);
cudaError_t adam_step(float *params, const float *grad, float *m, float *v, float lr, float b1,
                      float b2, float eps, int step, cudaStream_t s);
// FP32 master parameters -> inference layout
cudaError_t pack_infer(const float *params, InferParams &ip, cudaStream_t s);
// Network outputs (normalised) for n inputs in [-1,1]^3 with the tensor-core kernel.
cudaError_t infer_points(const InferParams &ip, const float *Xn, float *Y, int n, cudaStream_t s);
// Surrogate trace of one step over a 2D grid: planes (dx, dy, J00, J01, J10, J11) with the
// grid's pitch and plane stride, into `trace`; `coef` = this step's stage coefficients.
cudaError_t launch_mlp_trace(const InferParams &ip, const Geom &g, const VelParams &vp,
                             const StageCoef *coef, const double *t_dev, int kstep, double dt,
                             float *trace, const Check &chk, cudaStream_t s);

}  // namespace mlp
}  // namespace gals
