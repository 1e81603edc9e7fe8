// step2d.cu -- the single-grid 2D GALS step kernel and the 2D reconstruction kernel.
//
// The per-tile work (trace, Hermite, write-back, fused phi_xy) is step2d_tile.cuh; this file
// maps one thread block to one tile of the grid.
#include "step2d_tile.cuh"

#ifndef GALS_2D_TY
#define GALS_2D_TY 14
#endif
#ifndef GALS_2D_MINB
#define GALS_2D_MINB 5
#endif
#ifndef GALS_2D_HY
#define GALS_2D_HY 1
#endif
#ifndef GALS_2D_OV
#define GALS_2D_OV 1
#endif

namespace gals {

namespace {

using namespace t2;
constexpr int TY = GALS_2D_TY;  // output tile rows (even)
constexpr int HYT = GALS_2D_HY; // staged halo rows above and below the tile
constexpr bool OVX = GALS_2D_OV; // overlapped tiles where phi_xy is written (see tile_step2d)
constexpr int TWS = OVX ? TW + 4 : TW;  // staged columns of the single-grid kernels
using GT = Geo<TY, HYT, TWS>;

template <int WC> constexpr bool overlapped() { return OVX && WC; }
template <int WC> constexpr int tile_stride() { return overlapped<WC>() ? TX - 2 : TX; }

template <int TR, int VK, int CR, int WC>
__global__ void __launch_bounds__(TX, GALS_2D_MINB)
k_step2d(const float *__restrict__ in, float *__restrict__ out, Geom g, VelParams vp,
         const StageCoef *__restrict__ coef, float dt, const __grid_constant__ CUtensorMap tmap,
         int *__restrict__ err, int yt0)
{
    extern __shared__ __align__(128) float tile[];
    __shared__ __align__(16) Smem<TY, WC> sm;
    if (threadIdx.x == 0) mbar_init(&sm.bar, 1);
    __syncthreads();
    tile_step2d<TY, TR, VK, CR, WC, HYT, false, TWS, overlapped<WC>()>(
        in, out, g, vp, coef, dt, &tmap, err, blockIdx.x * tile_stride<WC>(), (blockIdx.y + yt0) * TY, tile, sm, 0);
}

// ---------------------------------------------------------------- persistent time loop
//
// All steps of one call in one launch (FULL layout, approach A).  Work items are
// (step, tile) pairs numbered step-major; a block takes the next item from a ticket counter
// and, for step s > 0, first waits until the 3 x 3 tiles around its own have finished step
// s - 1 (a per-tile flag holds the number of steps a tile has finished in this launch).
// With feet at most TY - 2 rows and TX - 2 columns from their node those are every tile
// whose output the step reads (the staged tile, global gathers) and every tile that still
// reads the region the step overwrites (the ping-pong buffer of step s - 1's input), so
// the order of the per-step launches is kept where it matters and nowhere else: blocks
// move on to the next step while the last tiles of the previous one drain.  Items are
// handed out in increasing order and a block waits only for smaller items, so the launch
// finishes whatever the number of resident blocks.  Every wait is bounded; a wait that
// runs out sets the launch's abort word and the error word, and every block returns.
constexpr int kErrRunTimeout = 3;
constexpr uint32_t kSpinLimit = 1u << 22;  // flag polls (~0.2 us each) before giving up

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

template <int TR, int VK>
__global__ void __launch_bounds__(TX, GALS_2D_MINB)
k_step2d_run(float *__restrict__ buf0, float *__restrict__ buf1, Geom g, VelParams vp,
             const StageCoef *__restrict__ coef, float dt, const __grid_constant__ CUtensorMap tmap0,
             const __grid_constant__ CUtensorMap tmap1, int *__restrict__ err, int *__restrict__ ctl,
             int nsteps, int cur)
{
    extern __shared__ __align__(128) float tile[];
    __shared__ __align__(16) Smem<TY, 1> sm;
    __shared__ int s_item;
    const int tid = threadIdx.x;
    if (tid == 0) mbar_init(&sm.bar, 1);
    const int ntx = (g.n0 + TX - 1) / TX, nty = (g.n1 + TY - 1) / TY, ntiles = ntx * nty;
    const int total = ntiles * nsteps;  // < 2^31 - 2^20 (host)
    int *ticket = ctl, *abort_word = ctl + 1, *flags = ctl + 4;
    // thread 0 draws the block's next item one item ahead, so that the draw's latency
    // hides behind a tile (a block waits only for items smaller than the one it holds,
    // and it finishes its current item before the drawn one: no cycle of waits)
    int next = 0;
    if (tid == 0) next = atomicAdd(ticket, 1);
    uint32_t parity = 0;
    for (;;) {
        if (tid == 0) s_item = next;
        __syncthreads();
        const int t = s_item;
        if (t >= total) break;
        const int st = t / ntiles, tt = t - st * ntiles, bx = tt % ntx, by = tt / ntx;
        // wait until the 3 x 3 tiles around this one have finished step st - 1: one flag
        // per thread of the first warp, in parallel
        bool lost = false;
        if (st > 0 && tid < 9) {
            const int nx = bx + tid % 3 - 1, ny = by + tid / 3 - 1;
            if (nx >= 0 && nx < ntx && ny >= 0 && ny < nty) {
                const int *f = flags + ny * ntx + nx;
                for (uint32_t it = 0; ld_acquire_gpu(f) < st; ++it) {
                    if (it >= kSpinLimit || *(volatile int *)abort_word) {
                        lost = true;
                        break;
                    }
                    __nanosleep(64);
                }
            }
        }
        if (__syncthreads_or(lost)) {
            if (tid == 0 && atomicExch(abort_word, 1) == 0) atomicExch(err, kErrRunTimeout);
            break;
        }
        const int b = (cur + st) & 1;
        if (tid == 0) {
            // the tile copy is an async-proxy read of data other blocks wrote through the
            // generic proxy (acquired above, ordered before this thread by the barrier)
            asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        const bool ok = tile_step2d<TY, TR, VK, CROSS_PLANE, 1, HYT, true, TWS>(
            b ? buf1 : buf0, b ? buf0 : buf1, g, vp, coef + st, dt, b ? &tmap1 : &tmap0, err,
            bx * TX, by * TY, tile, sm, parity, [&]() { next = atomicAdd(ticket, 1); });
        parity ^= 1u;
        if (!ok) {  // block-uniform: the staged copy was lost
            if (tid == 0) atomicExch(abort_word, 1);
            break;
        }
        __syncthreads();  // every store of the tile is issued before thread 0 publishes it
        if (tid == 0) {
            __threadfence();
            st_release_gpu(flags + tt, st + 1);
        }
    }
}

// phi_xy = d/dx psi_y at every node (approach A with one-sided ends); used after
// set_state and for the COMPACT layout's read-out.  Blocks of 32 x 8 nodes; the grid's
// y dimension is capped at 65535 and its blocks stride over the rows beyond.
__global__ void __launch_bounds__(256) k_recon2d(float *__restrict__ buf, Geom g)
{
    const int i = blockIdx.x * 32 + threadIdx.x;
    if (i >= g.n0) return;
    for (int j = blockIdx.y * 8 + threadIdx.y; j < g.n1; j += gridDim.y * 8) {
        const float *py = buf + 2 * g.plane + (size_t)j * g.pitch;
        float v = dline(i, g.n0, g.i2h0, [&](int q) { return py[q]; });
        buf[3 * g.plane + (size_t)j * g.pitch + i] = v;
    }
}

template <int TR, int VK, int CR, int WC>
cudaError_t launch_t(const StepLaunch &a, cudaStream_t s)
{
    constexpr int NP = CR == CROSS_PLANE ? 4 : 3;
    static bool attr_set = false;  // one attribute call per instantiation (not a stream op)
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_step2d<TR, VK, CR, WC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             GT::bytes(NP));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    // tile rows of the band (all by default)
    const int yt0 = a.band_lo / TY;
    const int yt1 = ((a.band_hi > 0 ? a.band_hi : a.geom.n1) + TY - 1) / TY;
    if (yt1 <= yt0) return cudaSuccess;
    dim3 grid((a.geom.n0 + tile_stride<WC>() - 1) / tile_stride<WC>(), yt1 - yt0);
    const CUtensorMap &map = NP == 4 ? *a.tmap4 : *a.tmap3;
    k_step2d<TR, VK, CR, WC><<<grid, TX, GT::bytes(NP), s>>>(a.in, a.out, a.geom, a.vp, a.coef,
                                                            (float)a.dt, map, a.err, yt0);
    return cudaGetLastError();
}

template <int TR, int VK>
cudaError_t launch_cr(const StepLaunch &a, cudaStream_t s)
{
    if (a.cross_in == CROSS_CELL) return launch_t<TR, VK, CROSS_CELL, 0>(a, s);  // approach B
    if (a.write_cross)
        return a.cross_in == CROSS_PLANE ? launch_t<TR, VK, CROSS_PLANE, 1>(a, s)
                                         : launch_t<TR, VK, CROSS_RECON, 1>(a, s);
    return a.cross_in == CROSS_PLANE ? launch_t<TR, VK, CROSS_PLANE, 0>(a, s)
                                     : launch_t<TR, VK, CROSS_RECON, 0>(a, s);
}

template <int VK>
cudaError_t launch_tr(const StepLaunch &a, cudaStream_t s)
{
    if (a.trace == TR_HEUN) return launch_cr<TR_HEUN, VK>(a, s);
    return a.trace == TR_EULER ? launch_cr<TR_EULER, VK>(a, s) : launch_cr<TR_RK3, VK>(a, s);
}

}  // namespace

cudaError_t launch_step2d(const StepLaunch &a, cudaStream_t s)
{
    if (a.trace == TR_GIVEN) return launch_cr<TR_GIVEN, VK_CONST>(a, s);  // velocity unused
    switch (a.vp.kind) {
    case VK_CONST: return launch_tr<VK_CONST>(a, s);
    case VK_ROTATION: return launch_tr<VK_ROTATION>(a, s);
    case VK_VORTEX2D: return launch_tr<VK_VORTEX2D>(a, s);
    case VK_PSEUDO1D: return launch_tr<VK_PSEUDO1D>(a, s);
    case VK_FOURIER2D: return launch_tr<VK_FOURIER2D>(a, s);
    case VK_WAVES2D: return launch_tr<VK_WAVES2D>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int TR, int VK>
cudaError_t launch_run_t(const RunLaunch &a, cudaStream_t s)
{
    auto kern = k_step2d_run<TR, VK>;
    static int blocks_per_sm = 0;  // per instantiation
    if (blocks_per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, GT::bytes(4));
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, TX, GT::bytes(4));
        if (e != cudaSuccess) return e;
        blocks_per_sm = nb > 0 ? nb : 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t items = (int64_t)run2d_tiles(a.geom) * a.nsteps;
    const int64_t want = (int64_t)blocks_per_sm * (sms > 0 ? sms : 1);
    const int grid = (int)(want < items ? want : items);
    kern<<<grid, TX, GT::bytes(4), s>>>(a.buf[0], a.buf[1], a.geom, a.vp, a.coef, (float)a.dt, *a.tmap[0],
                                        *a.tmap[1], a.err, a.ctl, a.nsteps, a.cur);
    return cudaGetLastError();
}

template <int VK>
cudaError_t launch_run_tr(const RunLaunch &a, cudaStream_t s)
{
    if (a.trace == TR_HEUN) return launch_run_t<TR_HEUN, VK>(a, s);
    return a.trace == TR_EULER ? launch_run_t<TR_EULER, VK>(a, s) : launch_run_t<TR_RK3, VK>(a, s);
}

int tile_rows2d() { return TY; }

int run2d_tiles(const Geom &g) { return ((g.n0 + TX - 1) / TX) * ((g.n1 + TY - 1) / TY); }

int run2d_max_cells(int axis) { return axis == 0 ? TX - 2 : TY - 2; }

cudaError_t launch_step2d_run(const RunLaunch &a, cudaStream_t s)
{
    switch (a.vp.kind) {
    case VK_CONST: return launch_run_tr<VK_CONST>(a, s);
    case VK_ROTATION: return launch_run_tr<VK_ROTATION>(a, s);
    case VK_VORTEX2D: return launch_run_tr<VK_VORTEX2D>(a, s);
    case VK_PSEUDO1D: return launch_run_tr<VK_PSEUDO1D>(a, s);
    case VK_FOURIER2D: return launch_run_tr<VK_FOURIER2D>(a, s);
    case VK_WAVES2D: return launch_run_tr<VK_WAVES2D>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

int band_unit(int dim) { return dim == 2 ? TY : 4; }

void tile_box2d(int np, uint32_t box[3])
{
    box[0] = TWS;
    box[1] = GT::TH;
    box[2] = (uint32_t)np;
}

cudaError_t launch_recon2d(const Geom &g, float *buf, cudaStream_t s)
{
    dim3 block(32, 8);
    dim3 grid((g.n0 + 31) / 32, std::min((g.n1 + 7) / 8, 65535));
    k_recon2d<<<grid, block, 0, s>>>(buf, g);
    return cudaGetLastError();
}

}  // namespace gals
