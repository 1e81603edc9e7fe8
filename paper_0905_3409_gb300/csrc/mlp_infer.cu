// mlp_infer.cu -- tensor-core (tcgen05 + TMEM) inference of the flow-map surrogate and the
// surrogate trace of one GALS step.
//
// A block holds all 16-bit weights (120 KB with the bias slabs) in shared memory and runs
// NWG = 3 groups of 4 warps, each with its own 128-point tile in flight, so that one tile's
// epilogue overlaps another tile's matrix products.  Per layer and group, one elected
// thread issues tcgen05.mma (M = 128 points, N = 128 units (16 for the output layer),
// K = 16 per instruction, FP16 operands from shared memory, FP32 accumulator in TMEM, 128
// columns per group) and commits them to the group's mbarrier; after a bounded wait each
// thread reads its accumulator row back with tcgen05.ld (the bias is one more K-slab of the
// product), applies SiLU on FP16 pairs and stores the FP16 activations as the next layer's
// A operand.  (GALS_MLP_F16=0 builds the former BF16 operands, SiLU in FP32 with tanh on
// FP16 pairs.)  Operands use the no-swizzle K-major core-matrix layout: 8 rows
// x 16 bytes per core matrix, core matrices adjacent in K `lbo` bytes apart and adjacent
// in M/N 128 bytes apart.  The trace kernel turns the outputs into the foot displacement
// and the Jacobian of the backward map, checks a few nodes of every tile against the exact
// RK3 trace (Sec. 5.1) and recomputes the whole tile with RK3 when the check fails.
#include <cuda_fp16.h>

#include "mlp_internal.h"
#include "tc.cuh"
#include "tma.cuh"

#ifndef GALS_MLP_F16
#define GALS_MLP_F16 1
#endif

namespace gals {
namespace mlp {

using namespace tc;

namespace {

constexpr bool kF16 = GALS_MLP_F16;  // operand type of every inference product

__device__ __forceinline__ uint16_t to_op(float v)
{
    return kF16 ? __half_as_ushort(__float2half_rn(v)) : __bfloat16_as_ushort(__float2bfloat16(v));
}
__device__ __forceinline__ uint32_t pack_op(float a, float b) { return kF16 ? pack_f16(a, b) : pack_bf16(a, b); }
__host__ __device__ constexpr uint32_t idesc_op(int M, int N) { return kF16 ? idesc_f16(M, N) : idesc_bf16(M, N); }

constexpr int NWG = 3;               // tile groups (tiles in flight) per block
constexpr int GT = 128;              // threads per tile group: one per accumulator row
                                     // (four warps, one per TMEM lane quarter)
constexpr int NT = GT * NWG;         // threads per block
constexpr int ROWS = 128;            // points per tile (= M of the products, = TMEM lanes)
constexpr uint32_t TMEM_COLS = NWG <= 2 ? 256 : 512;  // power of two >= NWG * 128
constexpr int kErrMmaTimeout = 2;

struct Smem {
    uint16_t w[W_TOTAL];                 // packed operands (weights, bias slabs, ones block)
    __align__(1024) uint16_t act[NWG][ROWS * HID];  // A operand of each group's tile
    uint64_t bar[NWG];
    uint32_t tmem;                       // TMEM base address from tcgen05.alloc
    int fail[NWG];
};

__device__ __forceinline__ void wg_sync(int g)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(GT) : "memory");
}
// named barrier of the tile group that also ORs a flag over its threads
__device__ __forceinline__ int wg_sync_or(int g, int flag)
{
    int r;
    asm volatile(
        "{\n .reg .pred q, o;\n setp.ne.s32 q, %1, 0;\n bar.red.or.pred o, %2, %3, q;\n"
        " selp.s32 %0, 1, 0, o;\n}\n"
        : "=r"(r)
        : "r"(flag), "r"(1 + g), "n"(GT)
        : "memory");
    return r;
}

// SiLU of two pre-activations given as h = z/2 (FP32): silu(z) = z (1 + tanh(z/2)) / 2
// = h + h tanh(h), returned as an operand pair.  FP16 operands: h rounded to FP16, tanh on
// the FP16 pair (one MUFU operation for two values, relative error about 1e-3) and one
// FP16 fused multiply-add, whose result is the next layer's operand pair as it stands
// (FP16 carries 3 more mantissa bits than BF16).  BF16 operands: the multiply-add in FP32
// and the result rounded to BF16.
__device__ __forceinline__ uint32_t silu2_op(float2 h)
{
    const __half2 hh = __floats2half2_rn(h.x, h.y);
    uint32_t tr;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(tr) : "r"(*reinterpret_cast<const uint32_t *>(&hh)));
    if (kF16) {
        const __half2 y = __hfma2(hh, *reinterpret_cast<const __half2 *>(&tr), hh);
        return *reinterpret_cast<const uint32_t *>(&y);
    }
    const float2 t = __half22float2(*reinterpret_cast<const __half2 *>(&tr));
    const float2 y = __ffma2_rn(h, t, h);
    return pack_bf16(y.x, y.y);
}

// ---- block setup / teardown ----

// Weights and biases into shared memory, barriers, TMEM allocation (warp 0).
__device__ void block_setup(Smem &sm, const InferParams &ip)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(ip.w);
    uint4 *dst = reinterpret_cast<uint4 *>(sm.w);
    for (int e = threadIdx.x; e < (int)(W_TOTAL * 2 / 16); e += NT) dst[e] = src[e];
    if (threadIdx.x < NWG) {
        mbar_init(&sm.bar[threadIdx.x], 1);
        sm.fail[threadIdx.x] = 0;
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sm.tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ void block_teardown(Smem &sm)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem), "r"(TMEM_COLS)
                     : "memory");
}

// Per-thread state of the tile engine.  Tile group g owns TMEM columns 128g..128g+127;
// warp q of the group reads TMEM lane quarter q (rows 32q..32q+31).
struct Wg {
    int g;            // tile group
    int r;            // thread's row = TMEM lane
    uint32_t tcol;    // TMEM address of the group's accumulator, lane 0
    uint32_t tlane;   // this warp's TMEM lane base, in address units
    uint32_t phase;   // parity of the group's mbarrier
};

__device__ __forceinline__ Wg make_wg(const Smem &sm)
{
    Wg w;
    w.g = threadIdx.x / GT;
    w.r = threadIdx.x % GT;
    w.tcol = sm.tmem + (uint32_t)(128 * w.g);
    w.tlane = (uint32_t)((w.r & ~31) << 16);
    w.phase = 0u;
    return w;
}

// Row r's network input (x, y, phase in [-1, 1], then 1 for the bias, K padded to 16 with
// zeros) as the first layer's A operand; then the group barrier that publishes it to the
// tensor core.
__device__ __forceinline__ void stage_input(Smem &sm, const Wg &w, float a, float b, float c)
{
    char *base = reinterpret_cast<char *>(sm.act[w.g]) + (w.r >> 3) * 128 + (w.r & 7) * 16;
    *reinterpret_cast<uint4 *>(base) = make_uint4(pack_op(a, b), pack_op(c, 1.f), 0u, 0u);
    *reinterpret_cast<uint4 *>(base + 2048) = make_uint4(0u, 0u, 0u, 0u);
    fence_async_smem();
    wg_sync(w.g);
}

// The network on the warpgroup's staged tile: out[0..5] = outputs of row r (+ 2 padding).
// Returns false (after recording the error) if a product did not complete in time.
__device__ bool run_tile(Smem &sm, Wg &w, int *err, float out[8])
{
    const int g = w.g;
    const char *act = reinterpret_cast<const char *>(sm.act[g]);
    const char *wts = reinterpret_cast<const char *>(sm.w);
    const bool leader = threadIdx.x % GT == 0;
    for (int L = 0; L < NLAYER; ++L) {
        if (leader) {
            tc_fence_after();
            if (L == 0) {
                umma(w.tcol, sdesc(act, 2048, 128), sdesc(wts + 2 * W1_OFF, 2048, 128),
                     idesc_op(128, 128), 0u);
            } else if (L < NLAYER - 1) {
                const char *W = wts + 2 * (W2_OFF + (int64_t)(L - 1) * 128 * 128);
#pragma unroll
                for (int s = 0; s < 8; ++s)
                    umma(w.tcol, sdesc(act + s * 4096, 2048, 128), sdesc(W + s * 4096, 2048, 128),
                         idesc_op(128, 128), s > 0 ? 1u : 0u);
                umma(w.tcol, sdesc(wts + 2 * ONES_OFF, 2048, 128),
                     sdesc(wts + 2 * (WB_OFF + (int64_t)(L - 1) * 128 * 16), 2048, 128), idesc_op(128, 128), 1u);
            } else {
#pragma unroll
                for (int s = 0; s < 8; ++s)
                    umma(w.tcol, sdesc(act + s * 4096, 2048, 128), sdesc(wts + 2 * W5_OFF + s * 512, 256, 128),
                         idesc_op(128, 16), s > 0 ? 1u : 0u);
                umma(w.tcol, sdesc(wts + 2 * ONES_OFF, 2048, 128), sdesc(wts + 2 * W5B_OFF, 256, 128),
                     idesc_op(128, 16), 1u);
            }
            umma_commit(&sm.bar[g]);
        }
        // one warp polls the barrier; the others sleep in the group barrier below
        const bool ok = (threadIdx.x % GT) < 32 ? mbar_wait_bounded(&sm.bar[g], w.phase) : true;
        w.phase ^= 1u;
        if (wg_sync_or(g, !ok)) {
            if (leader) atomicExch(err, kErrMmaTimeout);
            return false;
        }
        tc_fence_after();
        const uint32_t ta = w.tcol + w.tlane;
        if (L < NLAYER - 1) {
            // SiLU of h = z/2 (the accumulator), BF16 activations of row r as the next
            // layer's A operand (K = 128)
            char *arow = reinterpret_cast<char *>(sm.act[g]) + (w.r >> 3) * 128 + (w.r & 7) * 16;
            // one 32-column TMEM load per wait: two per wait held 64 accumulator values live
            // and pushed the trace kernel past its 168-register cap (spills)
            constexpr int NU = 1;
#pragma unroll 1
            for (int c = 0; c < 4; c += NU) {
                uint32_t v[NU][32];
#pragma unroll
                for (int u = 0; u < NU; ++u) tmem_ld32_nowait(ta + 32 * (c + u), v[u]);
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < NU; ++u)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t p[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int k = 8 * q + 2 * e;
                            p[e] = silu2_op(make_float2(__uint_as_float(v[u][k]), __uint_as_float(v[u][k + 1])));
                        }
                        *reinterpret_cast<uint4 *>(arow + (4 * (c + u) + q) * 2048) =
                            make_uint4(p[0], p[1], p[2], p[3]);
                    }
            }
            tc_fence_before();
            fence_async_smem();
            wg_sync(g);
        } else {
            uint32_t v[8];
            tmem_ld8(ta, v);
#pragma unroll
            for (int k = 0; k < 8; ++k) out[k] = __uint_as_float(v[k]);
            tc_fence_before();
        }
    }
    return true;
}

// After an abort: bounded wait for the products still in flight, before TMEM is freed.
__device__ void drain(Smem &sm, const Wg &w, bool aborted)
{
    if (aborted) mbar_wait_bounded(&sm.bar[w.g], w.phase ^ 1u);
}

__global__ void __launch_bounds__(NT, 1)
k_infer_points(InferParams ip, const float *__restrict__ Xn, float *__restrict__ Y, int n, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    block_setup(sm, ip);
    Wg w = make_wg(sm);
    bool aborted = false;
    const int ntiles = (n + ROWS - 1) / ROWS;
    for (int tile = blockIdx.x * NWG + w.g; tile < ntiles; tile += gridDim.x * NWG) {
        const int p = tile * ROWS + w.r;
        const int64_t pc = min(p, n - 1);
        stage_input(sm, w, Xn[3 * pc], Xn[3 * pc + 1], Xn[3 * pc + 2]);
        float o[8];
        if (!run_tile(sm, w, err, o)) { aborted = true; break; }
        if (p < n)
            for (int c = 0; c < OUT; ++c) Y[6 * (int64_t)p + c] = o[c];
        wg_sync(w.g);  // act[g] is rewritten by the next tile's inputs
    }
    drain(sm, w, aborted);
    block_teardown(sm);
}

__device__ __forceinline__ uint32_t tile_hash(uint32_t a, uint32_t b)
{
    uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 15;
    h *= 0xC2B2AE3Du;
    return h ^ (h >> 13);
}

// Surrogate trace of one step over the grid: tile = 128 consecutive nodes of a row; VK
// is the field of the exact trace the residual check and the fallback run.
template <int VK>
__global__ void __launch_bounds__(NT, 1)
k_mlp_trace(InferParams ip, Geom g, VelParams vp, const StageCoef *__restrict__ coef,
            const double *__restrict__ t_dev, int kstep, double dt, float *__restrict__ trace,
            Check chk)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    block_setup(sm, ip);
    Wg w = make_wg(sm);
    bool aborted = false;
    const double t = t_dev[0] + (double)kstep * dt;
    const float phase = (float)(t - floor(t));
    const float dtf = (float)dt;
    const int tiles_x = (g.n0 + ROWS - 1) / ROWS;
    const int ntiles = tiles_x * g.n1;
    // outputs of the tile's rows for the residual check (act[g] is free after the products)
    float *outs = reinterpret_cast<float *>(sm.act[w.g]);
    for (int tile = blockIdx.x * NWG + w.g; tile < ntiles; tile += gridDim.x * NWG) {
        const int j = tile / tiles_x, x0 = (tile % tiles_x) * ROWS;
        const int i = x0 + w.r;
        if (w.r == 0) sm.fail[w.g] = 0;
        {
            const float x = g.lo0 + (float)min(i, g.n0 - 1) * g.h0, y = g.lo1 + (float)j * g.h1;
            stage_input(sm, w, 2.f * x - 1.f, 2.f * y - 1.f, 2.f * phase - 1.f);
        }
        float y[8];
        if (!run_tile(sm, w, chk.err, y)) { aborted = true; break; }
        for (int c = 0; c < OUT; ++c) outs[w.r * 8 + c] = y[c];
        float d[2], J[4];
        d[0] = y[0] * ip.scale[0] * g.h0;
        d[1] = y[1] * ip.scale[1] * g.h1;
        J[0] = 1.f + dtf * y[2] * ip.scale[2];
        J[1] = dtf * y[3] * ip.scale[3];
        J[2] = dtf * y[4] * ip.scale[4];
        J[3] = 1.f + dtf * y[5] * ip.scale[5];
        wg_sync(w.g);
        // residual check of `samples` nodes of the tile against the exact RK3 trace
        const int width = min(ROWS, g.n0 - x0);
        if (VK == VK_WAVES2D) {
            // a costly field: each sampled node's trace by a whole warp of the group
            // (modes split over the lanes), sample j on warp j mod 4
            for (int jj = w.r >> 5; jj < chk.samples; jj += GT / 32) {
                const int q = (int)(tile_hash((uint32_t)tile, (uint32_t)kstep + 977u * jj) % (uint32_t)width);
                const float *yq = &outs[q * 8];
                const float xq = g.lo0 + (float)(x0 + q) * g.h0, yy = g.lo1 + (float)j * g.h1;
                float dr[2], Jr[4];
                trace2d_waves_warp(vp, *coef, xq, yy, dtf, dr[0], dr[1], Jr);
                const float ex = fmaxf(fabsf(yq[0] * ip.scale[0] * g.h0 - dr[0]) * g.ih0,
                                       fabsf(yq[1] * ip.scale[1] * g.h1 - dr[1]) * g.ih1);
                const float mJ[4] = {1.f + dtf * yq[2] * ip.scale[2], dtf * yq[3] * ip.scale[3],
                                     dtf * yq[4] * ip.scale[4], 1.f + dtf * yq[5] * ip.scale[5]};
                float eJ = 0.f;
                for (int e = 0; e < 4; ++e) eJ = fmaxf(eJ, fabsf(mJ[e] - Jr[e]));
                if ((w.r & 31) == 0 && (!(ex <= chk.tol_x) || !(eJ <= chk.tol_J))) atomicOr(&sm.fail[w.g], 1);
            }
        } else if (w.r < chk.samples) {
            const int q = (int)(tile_hash((uint32_t)tile, (uint32_t)kstep + 977u * w.r) % (uint32_t)width);
            const float *yq = &outs[q * 8];
            const float xq = g.lo0 + (float)(x0 + q) * g.h0, yy = g.lo1 + (float)j * g.h1;
            float dr[2], Jr[4];
            trace2d<TR_RK3, VK>(vp, *coef, xq, yy, dtf, dr[0], dr[1], Jr);
            const float ex = fmaxf(fabsf(yq[0] * ip.scale[0] * g.h0 - dr[0]) * g.ih0,
                                   fabsf(yq[1] * ip.scale[1] * g.h1 - dr[1]) * g.ih1);
            const float mJ[4] = {1.f + dtf * yq[2] * ip.scale[2], dtf * yq[3] * ip.scale[3],
                                 dtf * yq[4] * ip.scale[4], 1.f + dtf * yq[5] * ip.scale[5]};
            float eJ = 0.f;
            for (int e = 0; e < 4; ++e) eJ = fmaxf(eJ, fabsf(mJ[e] - Jr[e]));
            if (!(ex <= chk.tol_x) || !(eJ <= chk.tol_J)) atomicOr(&sm.fail[w.g], 1);
        }
        wg_sync(w.g);
        const bool fail = sm.fail[w.g] != 0;
        if (fail && i < g.n0) {
            const float x = g.lo0 + (float)i * g.h0, yy = g.lo1 + (float)j * g.h1;
            trace2d<TR_RK3, VK>(vp, *coef, x, yy, dtf, d[0], d[1], J);
        }
        if (i < g.n0) {
            const int64_t o = (int64_t)j * g.pitch + i;
            trace[o] = d[0];
            trace[g.plane + o] = d[1];
            trace[2 * g.plane + o] = J[0];
            trace[3 * g.plane + o] = J[1];
            trace[4 * g.plane + o] = J[2];
            trace[5 * g.plane + o] = J[3];
        }
        if (w.r == 0) {
            atomicAdd(chk.tiles, 1ull);
            if (fail) atomicAdd(chk.fallbacks, 1ull);
        }
        wg_sync(w.g);  // outs, fail and act[g] are reused by the next tile
    }
    drain(sm, w, aborted);
    block_teardown(sm);
}

// FP32 master parameters -> packed 16-bit operands in the core-matrix layout (see
// mlp_internal.h): hidden layers and their biases halved, biases as K-slab columns.
__global__ void k_pack(const float *__restrict__ p, uint16_t *__restrict__ w)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < 128 * 16) {  // W1/2 (inputs 0..2), b1/2 (column 3), zeros
        const int r = e / 16, c = e % 16;
        const float v = c < IN ? p[woff(0) + r * IN + c] : (c == IN ? p[boff(0) + r] : 0.f);
        w[W1_OFF + cm_off(128, r, c) / 2] = to_op(0.5f * v);
    }
    if (e < 3 * 128 * 128) {  // W2/2..W4/2: 128 x 128
        const int L = e / (128 * 128), rem = e % (128 * 128), r = rem / 128, c = rem % 128;
        w[W2_OFF + (int64_t)L * 128 * 128 + cm_off(128, r, c) / 2] = to_op(0.5f * p[woff(1 + L) + rem]);
    }
    if (e < 16 * 128) {  // W5: 16 x 128, rows 6..15 zero
        const int r = e / 128, c = e % 128;
        w[W5_OFF + cm_off(16, r, c) / 2] = to_op(r < OUT ? p[woff(4) + r * 128 + c] : 0.f);
    }
    if (e < 3 * 128 * 16) {  // hidden bias slabs: b/2 in column 0
        const int L = e / (128 * 16), rem = e % (128 * 16), r = rem / 16, c = rem % 16;
        w[WB_OFF + (int64_t)L * 128 * 16 + cm_off(128, r, c) / 2] =
            to_op(c == 0 ? 0.5f * p[boff(1 + L) + r] : 0.f);
    }
    if (e < 16 * 16) {  // output bias slab: b5 in column 0
        const int r = e / 16, c = e % 16;
        w[W5B_OFF + cm_off(16, r, c) / 2] = to_op(c == 0 && r < OUT ? p[boff(4) + r] : 0.f);
    }
    if (e < 128 * 16) {  // ones block
        const int r = e / 16, c = e % 16;
        w[ONES_OFF + cm_off(128, r, c) / 2] = to_op(c == 0 ? 1.f : 0.f);
    }
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <class K>
cudaError_t set_smem(K fn)
{
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
}

static_assert(sizeof(Smem) <= 227 * 1024, "shared memory budget");
static_assert(W_TOTAL * 2 % 16 == 0, "weights are copied in 16-byte chunks");
static_assert(W2_OFF * 2 % 16 == 0 && W5_OFF * 2 % 16 == 0 && WB_OFF * 2 % 16 == 0 &&
                  W5B_OFF * 2 % 16 == 0 && ONES_OFF * 2 % 16 == 0,
              "operands start on 16-byte boundaries");

}  // namespace

cudaError_t pack_infer(const float *params, InferParams &ip, cudaStream_t s)
{
    k_pack<<<(3 * 128 * 128 + 255) / 256, 256, 0, s>>>(params, ip.w);
    return cudaGetLastError();
}

cudaError_t infer_points(const InferParams &ip, const float *Xn, float *Y, int n, int *err, cudaStream_t s)
{
    static bool set = false;
    if (!set) {
        cudaError_t e = set_smem(k_infer_points);
        if (e != cudaSuccess) return e;
        set = true;
    }
    const int tiles = (n + ROWS - 1) / ROWS, sms = sm_count();
    const int blocks = (tiles + NWG - 1) / NWG;
    k_infer_points<<<blocks < sms ? blocks : sms, NT, sizeof(Smem), s>>>(ip, Xn, Y, n, err);
    return cudaGetLastError();
}

cudaError_t launch_mlp_trace(const InferParams &ip, const Geom &g, const VelParams &vp,
                             const StageCoef *coef, const double *t_dev, int kstep, double dt,
                             float *trace, const Check &chk, cudaStream_t s)
{
    static bool set = false;
    if (!set) {
        cudaError_t e = set_smem(k_mlp_trace<VK_FOURIER2D>);
        if (e == cudaSuccess) e = set_smem(k_mlp_trace<VK_WAVES2D>);
        if (e != cudaSuccess) return e;
        set = true;
    }
    const int ntiles = ((g.n0 + ROWS - 1) / ROWS) * g.n1, sms = sm_count();
    const int blocks = (ntiles + NWG - 1) / NWG;
    auto kern = vp.kind == VK_WAVES2D ? k_mlp_trace<VK_WAVES2D> : k_mlp_trace<VK_FOURIER2D>;
    kern<<<blocks < sms ? blocks : sms, NT, sizeof(Smem), s>>>(ip, g, vp, coef, t_dev, kstep, dt, trace, chk);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace gals
