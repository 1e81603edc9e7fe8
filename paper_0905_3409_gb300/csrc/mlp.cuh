// mlp.cuh -- the learned flow-map surrogate of the backward trace: shapes, parameter
// layout and the activation shared by the training and inference kernels.
//
// Not in the paper.  The network maps (x, y, t mod 1), scaled to [-1, 1], to the six
// normalised outputs (delta_x/h, delta_y/h, (J - I)/dt) / scale of one backward step of
// fixed dt; layers 3 -> 128 -> 128 -> 128 -> 128 -> 6 with SiLU on the hidden layers.
// Parameters (flat, FP32 master copy): per layer W (out x in, row-major) then b (out).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "gals_device.cuh"

namespace gals {
namespace mlp {

constexpr int IN = 3, HID = 128, OUT = 6, NLAYER = 5;
constexpr int KPAD1 = 16;   // first layer's K padded for the tensor-core tiles
constexpr int NPAD5 = 8;    // last layer's N padded

__host__ __device__ constexpr int lin(int l) { return l == 0 ? IN : HID; }
__host__ __device__ constexpr int lout(int l) { return l == NLAYER - 1 ? OUT : HID; }
__host__ __device__ constexpr int64_t woff(int l)
{
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += (int64_t)lin(i) * lout(i) + lout(i);
    return o;
}
__host__ __device__ constexpr int64_t boff(int l) { return woff(l) + (int64_t)lin(l) * lout(l); }
constexpr int64_t NPARAM = woff(NLAYER);  // 50822

// sigma(z) = (1 + tanh(z/2))/2 with the hardware tanh; silu(z) = z sigma(z)
__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sigm(float z) { return fmaf(0.5f, tanh_fast(0.5f * z), 0.5f); }
__device__ __forceinline__ float silu(float z) { return z * sigm(z); }
__device__ __forceinline__ float silu_prime(float z)
{
    const float s = sigm(z);
    return fmaf(z * s, 1.f - s, s);
}

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16(v)); }

}  // namespace mlp
}  // namespace gals
