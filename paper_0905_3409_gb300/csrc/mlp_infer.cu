// mlp_infer.cu -- tensor-core inference of the flow-map surrogate and the surrogate trace
// of one GALS step.
//
// A block of 8 warps keeps all weights (BF16, about 115 KB) in shared memory and runs the
// network on tiles of 128 points: warp w owns rows 16w..16w+15 of the 128 x 128 activation
// matrix; every layer is mma.sync.m16n8k16 (BF16 operands, FP32 accumulation) with
// operands fetched by ldmatrix from padded shared rows, then bias + SiLU in FP32 and a BF16
// store for the next layer.  Blocks are persistent (one per SM) so the weights are loaded
// once.  The trace kernel turns the outputs into the foot displacement and the Jacobian of
// the backward map, checks a few nodes of every tile against the exact RK3 trace
// (Sec. 5.1) and recomputes the whole tile with RK3 when the check fails.
#include "mlp_internal.h"

namespace gals {
namespace mlp {

namespace {

constexpr int NT = 256;          // threads per block (8 warps x 16 rows)

__device__ __forceinline__ uint32_t smem_u32_(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
constexpr int ROWS = 128;        // points per tile
constexpr int LDA = 136;         // padded row length (bf16) of activations and weights
constexpr int LD1 = 24;          // padded row length of the first layer (K = 16)

struct Smem {
    __nv_bfloat16 w1[128 * LD1];
    __nv_bfloat16 w[3][128 * LDA];
    __nv_bfloat16 w5[8 * LDA];
    float b[B_TOTAL];
    __nv_bfloat16 in[ROWS * LD1];
    __nv_bfloat16 act[2][ROWS * LDA];
    float out[ROWS * 8];
};

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32_(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t r[2], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(smem_u32_(p)));
}
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Load the inference weights into shared memory (all threads).
__device__ void load_weights(Smem &sm, const InferParams &ip)
{
    for (int e = threadIdx.x; e < 128 * 16; e += NT) sm.w1[(e / 16) * LD1 + e % 16] = ip.w[W1_OFF + e];
    for (int L = 0; L < 3; ++L) {
        const __nv_bfloat16 *src = ip.w + W2_OFF + (int64_t)L * 128 * 128;
        for (int e = threadIdx.x; e < 128 * 128 / 8; e += NT) {  // 16-byte chunks
            const int r = e / 16, c = (e % 16) * 8;
            *reinterpret_cast<uint4 *>(&sm.w[L][r * LDA + c]) =
                *reinterpret_cast<const uint4 *>(src + r * 128 + c);
        }
    }
    for (int e = threadIdx.x; e < 8 * 128; e += NT) sm.w5[(e / 128) * LDA + e % 128] = ip.w[W5_OFF + e];
    for (int e = threadIdx.x; e < B_TOTAL; e += NT) sm.b[e] = ip.b[e];
    for (int e = threadIdx.x; e < ROWS * LD1; e += NT) sm.in[e] = __float2bfloat16(0.f);
}

// out[128][8] = network(in[128][16]) ; must be called by all threads (warp w: rows 16w..)
__device__ void run_tile(Smem &sm)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = warp * 16;
    const int arow = r0 + (lane & 15), acol = (lane >> 4) * 8;          // A (x4) lane address
    const int brow = (lane & 7) + ((lane >> 4) << 3), bcol = ((lane >> 3) & 1) * 8;  // B (x4)
    const int crow = r0 + (lane >> 2), ccol = 2 * (lane & 3);            // accumulator
    float acc[16][4];

    // layer 1: K = 16
    {
        uint32_t a[4];
        ldsm_x4(a, &sm.in[arow * LD1 + acol]);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            uint32_t b[4];
            ldsm_x4(b, &sm.w1[(8 * j + brow) * LD1 + bcol]);
            mma_bf16(acc[j], a, b[0], b[1]);
            mma_bf16(acc[j + 1], a, b[2], b[3]);
        }
    }
    int cur = 0;
#pragma unroll 1
    for (int L = 0; L < 4; ++L) {
        // epilogue of the previous layer: bias + SiLU -> BF16 activations (own rows only)
        const float *bias = sm.b + 128 * L;
        __nv_bfloat16 *dst = sm.act[cur];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int c = 8 * j + ccol;
            const float b0 = bias[c], b1 = bias[c + 1];
            *reinterpret_cast<__nv_bfloat162 *>(&dst[crow * LDA + c]) =
                __floats2bfloat162_rn(silu(acc[j][0] + b0), silu(acc[j][1] + b1));
            *reinterpret_cast<__nv_bfloat162 *>(&dst[(crow + 8) * LDA + c]) =
                __floats2bfloat162_rn(silu(acc[j][2] + b0), silu(acc[j][3] + b1));
        }
        __syncwarp();
        const __nv_bfloat16 *A = sm.act[cur];
        if (L < 3) {
            const __nv_bfloat16 *W = sm.w[L];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                uint32_t a[4];
                ldsm_x4(a, &A[arow * LDA + 16 * kk + acol]);
#pragma unroll
                for (int j = 0; j < 16; j += 2) {
                    uint32_t b[4];
                    ldsm_x4(b, &W[(8 * j + brow) * LDA + 16 * kk + bcol]);
                    mma_bf16(acc[j], a, b[0], b[1]);
                    mma_bf16(acc[j + 1], a, b[2], b[3]);
                }
            }
            cur ^= 1;
        } else {
            // output layer: N = 8 (6 used)
            float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                uint32_t a[4], b[2];
                ldsm_x4(a, &A[arow * LDA + 16 * kk + acol]);
                ldsm_x2(b, &sm.w5[(lane & 7) * LDA + 16 * kk + ((lane >> 3) & 1) * 8]);
                mma_bf16(o, a, b[0], b[1]);
            }
            const float *b5 = sm.b + 512;
            sm.out[crow * 8 + ccol] = o[0] + b5[ccol];
            sm.out[crow * 8 + ccol + 1] = o[1] + b5[ccol + 1];
            sm.out[(crow + 8) * 8 + ccol] = o[2] + b5[ccol];
            sm.out[(crow + 8) * 8 + ccol + 1] = o[3] + b5[ccol + 1];
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(NT, 1)
k_infer_points(InferParams ip, const float *__restrict__ Xn, float *__restrict__ Y, int n)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    load_weights(sm, ip);
    __syncthreads();
    for (int t0 = blockIdx.x * ROWS; t0 < n; t0 += gridDim.x * ROWS) {
        if (threadIdx.x < ROWS) {
            const int p = t0 + threadIdx.x;
            for (int c = 0; c < 3; ++c)
                sm.in[threadIdx.x * LD1 + c] = __float2bfloat16(p < n ? Xn[3 * p + c] : 0.f);
        }
        __syncthreads();
        run_tile(sm);
        __syncthreads();
        if (threadIdx.x < ROWS && t0 + threadIdx.x < n)
            for (int c = 0; c < OUT; ++c) Y[6 * (t0 + threadIdx.x) + c] = sm.out[threadIdx.x * 8 + c];
        __syncthreads();
    }
}

__device__ __forceinline__ uint32_t tile_hash(uint32_t a, uint32_t b)
{
    uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 15;
    h *= 0xC2B2AE3Du;
    return h ^ (h >> 13);
}

// Surrogate trace of one step over the grid: tile = 128 consecutive nodes of a row.
__global__ void __launch_bounds__(NT, 1)
k_mlp_trace(InferParams ip, Geom g, VelParams vp, const StageCoef *__restrict__ coef,
            const double *__restrict__ t_dev, int kstep, double dt, float *__restrict__ trace,
            Check chk)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    __shared__ int fail;
    load_weights(sm, ip);
    const double t = t_dev[0] + (double)kstep * dt;
    const float phase = (float)(t - floor(t));
    const float dtf = (float)dt;
    const int tiles_x = (g.n0 + ROWS - 1) / ROWS;
    const int ntiles = tiles_x * g.n1;
    __syncthreads();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int j = tile / tiles_x, x0 = (tile % tiles_x) * ROWS;
        const int tid = threadIdx.x;
        const int i = x0 + tid;
        if (tid < ROWS) {
            const float x = g.lo0 + (float)min(i, g.n0 - 1) * g.h0, y = g.lo1 + (float)j * g.h1;
            sm.in[tid * LD1 + 0] = __float2bfloat16(2.f * x - 1.f);
            sm.in[tid * LD1 + 1] = __float2bfloat16(2.f * y - 1.f);
            sm.in[tid * LD1 + 2] = __float2bfloat16(2.f * phase - 1.f);
        }
        if (tid == 0) fail = 0;
        __syncthreads();
        run_tile(sm);
        __syncthreads();
        const int64_t o = (int64_t)j * g.pitch + i;
        float d[2], J[4];
        if (tid < ROWS) {
            const float *y = &sm.out[tid * 8];
            d[0] = y[0] * ip.scale[0] * g.h0;
            d[1] = y[1] * ip.scale[1] * g.h1;
            J[0] = 1.f + dtf * y[2] * ip.scale[2];
            J[1] = dtf * y[3] * ip.scale[3];
            J[2] = dtf * y[4] * ip.scale[4];
            J[3] = 1.f + dtf * y[5] * ip.scale[5];
        }
        // residual check of `samples` nodes of the tile against the exact RK3 trace
        const int width = min(ROWS, g.n0 - x0);
        if (tid < chk.samples) {
            const int q = (int)(tile_hash((uint32_t)tile, (uint32_t)kstep + 977u * tid) % (uint32_t)width);
            const float *y = &sm.out[q * 8];
            const float xq = g.lo0 + (float)(x0 + q) * g.h0, yq = g.lo1 + (float)j * g.h1;
            float dr[2], Jr[4];
            trace2d<TR_RK3, VK_FOURIER2D>(vp, *coef, xq, yq, dtf, dr[0], dr[1], Jr);
            const float ex = fmaxf(fabsf(y[0] * ip.scale[0] * g.h0 - dr[0]) * g.ih0,
                                   fabsf(y[1] * ip.scale[1] * g.h1 - dr[1]) * g.ih1);
            const float mJ[4] = {1.f + dtf * y[2] * ip.scale[2], dtf * y[3] * ip.scale[3],
                                 dtf * y[4] * ip.scale[4], 1.f + dtf * y[5] * ip.scale[5]};
            float eJ = 0.f;
            for (int e = 0; e < 4; ++e) eJ = fmaxf(eJ, fabsf(mJ[e] - Jr[e]));
            if (!(ex <= chk.tol_x) || !(eJ <= chk.tol_J)) atomicOr(&fail, 1);
        }
        __syncthreads();
        if (fail && tid < ROWS && i < g.n0) {
            const float x = g.lo0 + (float)i * g.h0, y = g.lo1 + (float)j * g.h1;
            trace2d<TR_RK3, VK_FOURIER2D>(vp, *coef, x, y, dtf, d[0], d[1], J);
        }
        if (tid < ROWS && i < g.n0) {
            trace[o] = d[0];
            trace[g.plane + o] = d[1];
            trace[2 * g.plane + o] = J[0];
            trace[3 * g.plane + o] = J[1];
            trace[4 * g.plane + o] = J[2];
            trace[5 * g.plane + o] = J[3];
        }
        if (tid == 0) {
            atomicAdd(chk.tiles, 1ull);
            if (fail) atomicAdd(chk.fallbacks, 1ull);
        }
        __syncthreads();
    }
}

__global__ void k_pack(const float *__restrict__ p, __nv_bfloat16 *__restrict__ w, float *__restrict__ b)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < 128 * 16) {  // W1 [128][16], K padded with zeros
        const int r = e / 16, c = e % 16;
        w[W1_OFF + e] = __float2bfloat16(c < IN ? p[woff(0) + r * IN + c] : 0.f);
    }
    if (e < 3 * 128 * 128) {
        const int L = e / (128 * 128), rem = e % (128 * 128);
        w[W2_OFF + e] = __float2bfloat16(p[woff(1 + L) + rem]);
    }
    if (e < 8 * 128) {  // W5 [8][128], N padded with zeros
        const int r = e / 128;
        w[W5_OFF + e] = __float2bfloat16(r < OUT ? p[woff(4) + e] : 0.f);
    }
    if (e < 4 * 128) b[e] = p[boff(e / 128) + e % 128];
    if (e < 8) b[512 + e] = e < OUT ? p[boff(4) + e] : 0.f;
}

}  // namespace

cudaError_t pack_infer(const float *params, InferParams &ip, cudaStream_t s)
{
    k_pack<<<(3 * 128 * 128 + 255) / 256, 256, 0, s>>>(params, ip.w, ip.b);
    return cudaGetLastError();
}

static cudaError_t set_smem(const void *fn)
{
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
}

cudaError_t infer_points(const InferParams &ip, const float *Xn, float *Y, int n, cudaStream_t s)
{
    static bool set = false;
    if (!set) {
        cudaError_t e = set_smem((const void *)k_infer_points);
        if (e != cudaSuccess) return e;
        set = true;
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (n + ROWS - 1) / ROWS;
    k_infer_points<<<tiles < sms ? tiles : sms, NT, sizeof(Smem), s>>>(ip, Xn, Y, n);
    return cudaGetLastError();
}

cudaError_t launch_mlp_trace(const InferParams &ip, const Geom &g, const VelParams &vp,
                             const StageCoef *coef, const double *t_dev, int kstep, double dt,
                             float *trace, const Check &chk, cudaStream_t s)
{
    static bool set = false;
    if (!set) {
        cudaError_t e = set_smem((const void *)k_mlp_trace);
        if (e != cudaSuccess) return e;
        set = true;
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = ((g.n0 + ROWS - 1) / ROWS) * g.n1;
    k_mlp_trace<<<ntiles < sms ? ntiles : sms, NT, sizeof(Smem), s>>>(ip, g, vp, coef, t_dev, kstep,
                                                                     dt, trace, chk);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace gals
