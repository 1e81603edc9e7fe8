// gals_internal.h -- host-side interface between the C ABI and the kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gals_device.cuh"

namespace gals {

struct StepLaunch {
    const float *in;     // state at t (all planes, plane stride geom.plane)
    float *out;          // state at t + dt
    Geom geom;
    VelParams vp;
    const StageCoef *coef; // this step's stage coefficients (filled by launch_coef_table)
    double dt;
    int trace;           // TR_EULER / TR_RK3
    int cross_in;        // CROSS_PLANE: read mixed derivatives; CROSS_RECON: rebuild from psi
    int write_cross;     // 1: also write the mixed-derivative planes of the new state
    const CUtensorMap *tmap4; // TMA map of `in` for reading stored mixed derivatives
    const CUtensorMap *tmap3; // TMA map of `in` for rebuilding them (COMPACT)
    const CUtensorMap *tmap_cross; // 3D FULL: TMA map of `out` with the reconstruction box
    int *err;            // device error word (kErrTmaTimeout on a lost tile copy)
    // the band of nodes to update along the last axis (2D rows, 3D z-levels), [lo, hi);
    // hi == 0: all.  lo must be a multiple of band_unit(dim), hi too unless it is n.
    int band_lo, band_hi;
};

// Persistent 2D time loop (FULL layout, approach A): nsteps steps from buffer cur in one
// launch; ctl holds 4 + run2d_tiles(geom) ints, zero before the launch (ticket counter,
// abort word, per-tile step flags).  Feet must stay within run2d_max_cells(axis) cells of
// their node.
struct RunLaunch {
    float *buf[2];
    int cur;
    Geom geom;
    VelParams vp;
    const StageCoef *coef;     // stage coefficients of the launch's steps
    double dt;
    int trace;                 // TR_EULER / TR_RK3 / TR_HEUN
    const CUtensorMap *tmap[2]; // FULL-box TMA maps of buf[0], buf[1]
    int *err;
    int *ctl;
    int nsteps;
};
int run2d_tiles(const Geom &g);
int run2d_max_cells(int axis);
cudaError_t launch_step2d_run(const RunLaunch &a, cudaStream_t s);

// Granularity of StepLaunch bands: the 2D tile height, the 3D tile depth.
int band_unit(int dim);

// Box of the 2D step kernel's staged tile for np planes; its output rows per block.
void tile_box2d(int np, uint32_t box[3]);
int tile_rows2d();
// Box (x, y, z, planes) of the 3D step kernel's staged tile.
void tile_box3d(int cross_recon, uint32_t box[4]);
// Box (x, y, z, planes) of the 3D reconstruction kernel's staged psi_y, psi_z.
void recon_box3d(uint32_t box[4]);
// Encode a tiled TMA map of FP32 data: rank dims (innermost first), byte strides of
// dims 1..rank-1, box extents; zero fill outside the tensor.
cudaError_t make_tile_map(CUtensorMap *map, const float *base, int rank, const uint64_t *dims,
                          const uint64_t *strides_bytes, const uint32_t *box);

// Kernel launchers; return the launch error (cudaSuccess if launched).
cudaError_t launch_step2d(const StepLaunch &a, cudaStream_t s);
cudaError_t launch_step3d(const StepLaunch &a, cudaStream_t s);
// Rebuild the mixed-derivative planes of `buf` from its gradient planes (approach A).
cudaError_t launch_recon(int dim, const Geom &g, float *buf, cudaStream_t s);
// table[s] = stage coefficients of step s (t = t_dev[0] + s*dt), s < nsteps
cudaError_t launch_coef_table(StageCoef *table, const VelParams &vp, const double *t_dev,
                              double dt, int nsteps, cudaStream_t s);
// t_dev[0] += nsteps * dt
cudaError_t launch_advance_time(double *t_dev, int nsteps, double dt, cudaStream_t s);
// the device clock set to t, in stream order (no host staging, the caller does not block)
cudaError_t launch_set_time(double *t_dev, double t, cudaStream_t s);
// Velocity kinds supported per dimension.
bool vel_supported(int dim, int kind);

// Value, unit normal and curvature of the interpolant at npts points (curvature.cu);
// pts: npts * dim FP64 coordinates on the device; any output may be null.
cudaError_t launch_eval_points(int dim, const Geom &g, const double lo[3], const double h[3],
                               const float *state, const double *pts, int64_t npts, bool cell_b,
                               float *H, float *normal, float *kappa, cudaStream_t s);

// Diagnostics (diag.cu)
struct DiagOut {
    unsigned long long n_neg, n_sym, nonfinite;
    unsigned int emax_phi_bits, emax_psi_bits;  // non-negative floats as ordered integers
    double l2_phi_sum;
};
// Scratch: `partials` holds at least diag_partials_needed() doubles; `counters` a DiagOut.
int diag_partials_needed();
// cell_a / cell_b: the interpolant of a / b takes its mixed derivatives by approach B.
cudaError_t launch_diag(int dim, const Geom &g, const float *a, const float *b, int q,
                        DiagOut *counters, double *partials, cudaStream_t s, bool cell_a = false,
                        bool cell_b = false);
// Same kernels with `nparts` node blocks (one FP64 partial each) instead of the default.
cudaError_t launch_diag_with(int dim, const Geom &g, const float *a, const float *b, int q,
                             DiagOut *counters, double *partials, int nparts, cudaStream_t s);

}  // namespace gals
