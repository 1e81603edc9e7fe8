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

namespace gals {

namespace {

using namespace t2;
constexpr int TY = GALS_2D_TY;  // output tile rows (even)
constexpr int HYT = GALS_2D_HY; // staged halo rows above and below the tile
using GT = Geo<TY, HYT>;

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
    tile_step2d<TY, TR, VK, CR, WC, HYT>(in, out, g, vp, coef, dt, &tmap, err, blockIdx.x * TX,
                                    (blockIdx.y + yt0) * TY, tile, sm, 0);
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
    dim3 grid((a.geom.n0 + TX - 1) / TX, yt1 - yt0);
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
    default: return cudaErrorInvalidValue;
    }
}

int tile_rows2d() { return TY; }

int band_unit(int dim) { return dim == 2 ? TY : 4; }

void tile_box2d(int np, uint32_t box[3])
{
    box[0] = TW;
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
