// batch_internal.h -- device-side descriptors of the batched 2D mode.
#pragma once

#include "gals_internal.h"

namespace gals {

struct BatchProb {
    Geom g;          // the problem's grid (plane stride, pitch, spacing, origin)
    int64_t off;     // offset of its plane 0 in each state buffer (floats)
    float dt;        // its time step (float for the kernels)
    double dt_d;     // and in FP64 for its clock
};

struct BatchItem {
    int prob;        // problem index
    int x0, y0;      // tile origin (node indices)
};

struct BatchLaunch {
    const float *in;
    float *out;
    const BatchProb *probs;
    const VelParams *vps;    // per-problem velocity parameters
    const StageCoef *coef;   // this step's coefficients, one per problem
    const CUtensorMap *maps; // per-problem TMA maps of `in`
    const BatchItem *items;
    int nitems;
    int grid;                // blocks (0: one per item)
    int variant;             // 0: 128 x 8 tiles, 1: 128 x 16 tiles
    int kind;                // velocity kind shared by all problems
    int compact;             // COMPACT layout (mixed derivatives rebuilt on the fly)
    int *err;
};

// Persistent multi-step launch (all nsteps steps of a call): ctl holds 4 + nitems ints, zero
// before the launch; nbr the 9 neighbour item indices of every item (-1: none).  Feet must
// stay within batch_tile_rows(variant) - 2 rows and 126 columns of their node.
struct BatchRunLaunch {
    float *buf[2];
    int cur;
    const BatchProb *probs;
    const VelParams *vps;
    const StageCoef *coef;       // coefficients of the launch's steps [step][problem]
    const CUtensorMap *maps[2];  // per-problem TMA maps of buf[0], buf[1]
    const BatchItem *items;
    const int *nbr;
    int nitems, nprob, nsteps;
    int variant, kind, compact;
    int *err, *ctl;
};

bool batch_kind_supported(int kind);
cudaError_t launch_batch2d_run(const BatchRunLaunch &a, cudaStream_t s);
int batch_tile_rows(int variant);
void batch_tile_box(int variant, int np, uint32_t box[3]);
int batch_max_blocks_per_sm(int variant, int kind, int compact);
cudaError_t launch_batch2d(const BatchLaunch &a, cudaStream_t s);
cudaError_t launch_batch_coef(StageCoef *table, const VelParams *vps, const double *t_dev,
                              const BatchProb *probs, int nprob, int nsteps, cudaStream_t s);
cudaError_t launch_batch_advance(double *t_dev, const BatchProb *probs, int nprob, int nsteps,
                                 cudaStream_t s);

}  // namespace gals
