// capi_internal.h -- helpers shared by the C ABI translation units.
#pragma once

#include <stddef.h>

#include <vector>

#include "../../include/gals.h"
#include "gals_internal.h"
#include "mlp_internal.h"

#include <nvtx3/nvToolsExt.h>

// NVTX range over one ABI call (named after the call), for timeline profilers; free when no
// profiler is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

namespace gals {

// Validate a velocity descriptor for a grid of dimension `dim` and fill the kernels'
// parameters; on error writes a message to msg and returns the status.
gals_status velparams_from(int dim, const gals_velocity *v, VelParams &vp, char *msg, size_t len);

// An upper bound of max_i |v_i| over the box [lo, hi] and all times for a descriptor that
// velparams_from accepted (infinity if none is known).
double speed_bound(const gals_velocity *v, int dim, const double lo[3], const double hi[3]);

// Size limits of the kernels' index arithmetic and launch grids: 2D planes of at most
// 2^31 - 1 elements (row pitch x rows, 32-bit offsets in the tile kernels), at most
// 65535 tile rows of blocks in 2D (n[1] <= 65535 * rows per tile) and at most 65535
// blocks along y and z in 3D (n[1], n[2] <= 262140).  Returns false with a message.
bool grid_size_ok(int dim, const int n[3], char *msg, size_t len);

// Device copy of a WAVES2D mode table (per grid or surrogate): upload() copies the modes
// of v (validated by velparams_from) when they differ from the copy held, after the stream
// has finished earlier work (changed: whether it did); bind() points vp at it.
struct WaveStore {
    void *dev = nullptr;   // 3 M float4, then 3 M doubles (the layout of WaveTab / waves_d)
    int cap = 0, count = 0;
    std::vector<double> host;  // the rows held (6 per mode)
    cudaError_t upload(const gals_velocity *v, cudaStream_t s, bool *changed);
    void bind(VelParams &vp) const;
    void release();
};

// Whether surrogate `s` serves a step with these parameters (v: the step's velocity);
// fills the kernel views.
gals_status surrogate_for_step(const gals_surrogate *s, const gals_velocity *v, const VelParams &vp,
                               double dt, double h0, double h1, mlp::InferParams &ip, mlp::Check &chk,
                               char *msg, size_t len);

}  // namespace gals
