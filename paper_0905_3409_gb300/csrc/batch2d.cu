// batch2d.cu -- many independent 2D GALS problems of uneven size advanced by one launch
// per step.
//
// The problems' states live in one allocation per ping-pong buffer; a device work list
// holds one (problem, tile origin) item per 128 x TY tile of every problem, largest
// problems first.  A block processes items blockIdx.x, blockIdx.x + gridDim.x, ... with
// the same per-tile code as the single-grid kernel (step2d_tile.cuh), so a batched
// problem evolves bit for bit like the same problem on its own grid.  With gridDim.x equal
// to the number of items every block does one tile; with a smaller grid (a multiple of
// the SM count) the blocks are persistent and re-use their shared memory and barrier
// (one mbarrier phase per tile).
#include "batch_internal.h"
#include "step2d_tile.cuh"

namespace gals {

namespace {

using namespace t2;

template <int TY, int VK, int CR, int WC>
__global__ void __launch_bounds__(TX, 4)
k_batch2d(const float *__restrict__ in_base, float *__restrict__ out_base,
          const BatchProb *__restrict__ probs, const VelParams *__restrict__ vps,
          const StageCoef *__restrict__ coef, const CUtensorMap *__restrict__ maps,
          const BatchItem *__restrict__ items, int nitems, int *__restrict__ err)
{
    extern __shared__ __align__(128) float tile[];
    __shared__ __align__(16) Smem<TY, WC> sm;
    if (threadIdx.x == 0) mbar_init(&sm.bar, 1);
    __syncthreads();
    uint32_t parity = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        const BatchProb &P = probs[w.prob];
        const Geom g = P.g;
        const bool ok = tile_step2d<TY, TR_RK3, VK, CR, WC>(
            in_base + P.off, out_base + P.off, g, vps[w.prob], coef + w.prob, P.dt,
            maps + w.prob, err, w.x0, w.y0, tile, sm, parity);
        if (!ok) return;  // block-uniform
        parity ^= 1u;
        __syncthreads();  // tile and psi_y buffers are free before the next copy
    }
}

// Persistent multi-step launch over the work list: items (step, tile) numbered step-major
// from a ticket counter; a tile of step st waits until the 3 x 3 tiles of its own problem
// around it (nbr, 9 item indices per item, -1 where the problem has none) have finished
// step st - 1 (see k_step2d_run in step2d.cu for the argument that these are all the
// dependences while feet stay within TY - 2 rows and 126 columns of their node, and that
// the launch always finishes).  Every wait is bounded.
constexpr int kErrRunTimeout = 3;
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int TY, int VK, int CR, int WC>
__global__ void __launch_bounds__(TX, 4)
k_batch2d_run(float *__restrict__ buf0, float *__restrict__ buf1, const BatchProb *__restrict__ probs,
              const VelParams *__restrict__ vps, const StageCoef *__restrict__ coef,
              const CUtensorMap *__restrict__ maps0, const CUtensorMap *__restrict__ maps1,
              const BatchItem *__restrict__ items, const int *__restrict__ nbr, int nitems, int nprob,
              int nsteps, int cur, int *__restrict__ err, int *__restrict__ ctl)
{
    extern __shared__ __align__(128) float tile[];
    __shared__ __align__(16) Smem<TY, WC> sm;
    __shared__ int s_item;
    const int tid = threadIdx.x;
    if (tid == 0) mbar_init(&sm.bar, 1);
    const int total = nitems * nsteps;  // < 2^31 - 2^20 (host)
    int *ticket = ctl, *abort_word = ctl + 1, *flags = ctl + 4;
    int next = 0;
    if (tid == 0) next = atomicAdd(ticket, 1);
    uint32_t parity = 0;
    for (;;) {
        if (tid == 0) s_item = next;
        __syncthreads();
        const int t = s_item;
        if (t >= total) break;
        const int st = t / nitems, it = t - st * nitems;
        bool lost = false;
        if (st > 0 && tid < 9) {
            const int nb = __ldg(nbr + (int64_t)it * 9 + tid);
            if (nb >= 0)
                for (uint32_t k = 0; ld_acquire_gpu(flags + nb) < st; ++k) {
                    if (k >= kSpinLimit || *(volatile int *)abort_word) {
                        lost = true;
                        break;
                    }
                    __nanosleep(64);
                }
        }
        if (__syncthreads_or(lost)) {
            if (tid == 0 && atomicExch(abort_word, 1) == 0) atomicExch(err, kErrRunTimeout);
            break;
        }
        if (tid == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
        const BatchItem w = items[it];
        const BatchProb &P = probs[w.prob];
        const Geom g = P.g;
        const int b = (cur + st) & 1;
        const bool ok = tile_step2d<TY, TR_RK3, VK, CR, WC, HY, true>(
            (b ? buf1 : buf0) + P.off, (b ? buf0 : buf1) + P.off, g, vps[w.prob],
            coef + (int64_t)st * nprob + w.prob, P.dt, (b ? maps1 : maps0) + w.prob, err, w.x0, w.y0,
            tile, sm, parity, [&]() { next = atomicAdd(ticket, 1); });
        parity ^= 1u;
        if (!ok) {
            if (tid == 0) atomicExch(abort_word, 1);
            break;
        }
        __syncthreads();  // every store of the tile is issued before thread 0 publishes it
        if (tid == 0) {
            __threadfence();
            st_release_gpu(flags + it, st + 1);
        }
    }
}

__global__ void k_batch_coef(StageCoef *table, const VelParams *__restrict__ vps,
                             const double *__restrict__ t_dev, const BatchProb *__restrict__ probs,
                             int nprob, int nsteps)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nprob * nsteps) return;
    const int p = e % nprob, s = e / nprob;
    const double dt = probs[p].dt_d;
    stage_coef_one(vps[p], t_dev[p] + (double)s * dt, dt, table[e]);
}

__global__ void k_batch_advance(double *t_dev, const BatchProb *__restrict__ probs, int nprob,
                                int nsteps)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nprob) t_dev[p] = t_dev[p] + (double)nsteps * probs[p].dt_d;
}

template <int TY, int VK, int CR, int WC>
cudaError_t launch_t(const BatchLaunch &a, cudaStream_t s)
{
    constexpr int NP = CR == CROSS_PLANE ? 4 : 3;
    auto kern = k_batch2d<TY, VK, CR, WC>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Geo<TY>::bytes(NP));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int grid = a.grid > 0 ? a.grid : a.nitems;
    kern<<<grid, TX, Geo<TY>::bytes(NP), s>>>(a.in, a.out, a.probs, a.vps, a.coef, a.maps,
                                              a.items, a.nitems, a.err);
    return cudaGetLastError();
}

template <int TY, int VK, int CR, int WC>
cudaError_t launch_run_t(const BatchRunLaunch &a, cudaStream_t s)
{
    constexpr int NP = CR == CROSS_PLANE ? 4 : 3;
    auto kern = k_batch2d_run<TY, VK, CR, WC>;
    static int blocks_per_sm = 0;  // per instantiation
    if (blocks_per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Geo<TY>::bytes(NP));
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, TX, Geo<TY>::bytes(NP));
        if (e != cudaSuccess) return e;
        blocks_per_sm = nb > 0 ? nb : 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t items = (int64_t)a.nitems * a.nsteps;
    const int64_t want = (int64_t)blocks_per_sm * (sms > 0 ? sms : 1);
    const int grid = (int)(want < items ? want : items);
    kern<<<grid, TX, Geo<TY>::bytes(NP), s>>>(a.buf[0], a.buf[1], a.probs, a.vps, a.coef, a.maps[0], a.maps[1],
                                              a.items, a.nbr, a.nitems, a.nprob, a.nsteps, a.cur, a.err,
                                              a.ctl);
    return cudaGetLastError();
}

template <int TY, int VK>
cudaError_t launch_run_layout(const BatchRunLaunch &a, cudaStream_t s)
{
    return a.compact ? launch_run_t<TY, VK, CROSS_RECON, 0>(a, s) : launch_run_t<TY, VK, CROSS_PLANE, 1>(a, s);
}

template <int TY>
cudaError_t launch_run_kind(const BatchRunLaunch &a, cudaStream_t s)
{
    switch (a.kind) {
    case VK_FOURIER2D: return launch_run_layout<TY, VK_FOURIER2D>(a, s);
    case VK_VORTEX2D: return launch_run_layout<TY, VK_VORTEX2D>(a, s);
    case VK_ROTATION: return launch_run_layout<TY, VK_ROTATION>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int TY, int VK>
cudaError_t launch_layout(const BatchLaunch &a, cudaStream_t s)
{
    return a.compact ? launch_t<TY, VK, CROSS_RECON, 0>(a, s) : launch_t<TY, VK, CROSS_PLANE, 1>(a, s);
}

template <int TY>
cudaError_t launch_kind(const BatchLaunch &a, cudaStream_t s)
{
    switch (a.kind) {
    case VK_FOURIER2D: return launch_layout<TY, VK_FOURIER2D>(a, s);
    case VK_VORTEX2D: return launch_layout<TY, VK_VORTEX2D>(a, s);
    case VK_ROTATION: return launch_layout<TY, VK_ROTATION>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool batch_kind_supported(int kind)
{
    return kind == VK_FOURIER2D || kind == VK_VORTEX2D || kind == VK_ROTATION;
}

int batch_tile_rows(int variant) { return variant == 0 ? 8 : 16; }

void batch_tile_box(int variant, int np, uint32_t box[3])
{
    box[0] = TW;
    box[1] = (variant == 0 ? Geo<8>::TH : Geo<16>::TH);
    box[2] = (uint32_t)np;
}

int batch_max_blocks_per_sm(int variant, int kind, int compact)
{
    // occupancy of the kernel actually launched (registers and shared memory)
    int nb = 0;
    const int np = compact ? 3 : 4;
    const int bytes = variant == 0 ? Geo<8>::bytes(np) : Geo<16>::bytes(np);
    cudaError_t e = cudaSuccess;
#define OCC(TY, VK)                                                                             \
    e = compact ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch2d<TY, VK, CROSS_RECON, 0>, TX, bytes) \
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch2d<TY, VK, CROSS_PLANE, 1>, TX, bytes)
    if (variant == 0) {
        if (kind == VK_FOURIER2D) OCC(8, VK_FOURIER2D); else if (kind == VK_VORTEX2D) OCC(8, VK_VORTEX2D); else OCC(8, VK_ROTATION);
    } else {
        if (kind == VK_FOURIER2D) OCC(16, VK_FOURIER2D); else if (kind == VK_VORTEX2D) OCC(16, VK_VORTEX2D); else OCC(16, VK_ROTATION);
    }
#undef OCC
    return e == cudaSuccess ? nb : 1;
}

cudaError_t launch_batch2d(const BatchLaunch &a, cudaStream_t s)
{
    // the attribute (dynamic shared memory) must be set before occupancy queries matter
    return a.variant == 0 ? launch_kind<8>(a, s) : launch_kind<16>(a, s);
}

cudaError_t launch_batch2d_run(const BatchRunLaunch &a, cudaStream_t s)
{
    return a.variant == 0 ? launch_run_kind<8>(a, s) : launch_run_kind<16>(a, s);
}

cudaError_t launch_batch_coef(StageCoef *table, const VelParams *vps, const double *t_dev,
                              const BatchProb *probs, int nprob, int nsteps, cudaStream_t s)
{
    const int n = nprob * nsteps;
    k_batch_coef<<<(n + 127) / 128, 128, 0, s>>>(table, vps, t_dev, probs, nprob, nsteps);
    return cudaGetLastError();
}

cudaError_t launch_batch_advance(double *t_dev, const BatchProb *probs, int nprob, int nsteps,
                                 cudaStream_t s)
{
    k_batch_advance<<<(nprob + 127) / 128, 128, 0, s>>>(t_dev, probs, nprob, nsteps);
    return cudaGetLastError();
}

}  // namespace gals
