// capi_internal.h -- helpers shared by the C ABI translation units.
#pragma once

#include <stddef.h>

#include "../../include/gals.h"
#include "gals_internal.h"
#include "mlp_internal.h"

namespace gals {

// Validate a velocity descriptor for a grid of dimension `dim` and fill the kernels'
// parameters; on error writes a message to msg and returns the status.
gals_status velparams_from(int dim, const gals_velocity *v, VelParams &vp, char *msg, size_t len);

// Whether surrogate `s` serves a step with these parameters; fills the kernel views.
gals_status surrogate_for_step(const gals_surrogate *s, const VelParams &vp, double dt, double h0,
                               double h1, mlp::InferParams &ip, mlp::Check &chk, char *msg,
                               size_t len);

}  // namespace gals
