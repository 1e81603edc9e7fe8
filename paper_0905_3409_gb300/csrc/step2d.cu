// step2d.cu -- the 2D GALS step kernel and the mixed-derivative reconstruction.
//
// One thread per grid node (Sec. 4, steps 1-2 in the superconsistent form of Sec. 5.1):
//   trace back with the Jacobian -> locate the foot cell -> gather the 4 corners x 4 data
//   -> bicubic Hermite value and gradient -> phi+ = H, psi+ = J^T grad H.
// The mixed derivative phi_xy of the 4 corners is either read from its plane (the stored
// representation of Sec. 5.2) or rebuilt on the fly from psi_y by the approach-A central
// differences of Sec. 2.3 (COMPACT layout); both round identically.
#include "gals_internal.h"

namespace gals {

namespace {

constexpr int BX = 32, BY = 8;

// phi_xy at corner column q (q = k + o, o in {0,1}) from the psi_y row window
// w[0..3] = psi_y[k-1 .. k+2]: the same stencils as the reconstruction kernel.
template <int O>
__device__ __forceinline__ float cross_from_window(const float w[4], int q, int n, float i2h)
{
    constexpr int c = 1 + O;  // position of column q in the window
    if (O == 0) {
        if (q == 0) return dfirst(w[c], w[c + 1], w[c + 2], i2h);
    } else {
        if (q == n - 1) return dlast(w[c], w[c - 1], w[c - 2], i2h);
    }
    return dcentral(w[c + 1], w[c - 1], i2h);
}

template <int TR, int VK, int CR>
__global__ void __launch_bounds__(BX *BY)
k_step2d(const float *__restrict__ in, float *__restrict__ out, Geom g, VelParams vp,
         const double *__restrict__ t_dev, int kstep, double dt)
{
    __shared__ StageCoef sc;
    const double t = t_dev[0] + (double)kstep * dt;
    fill_stage_coef(vp, t, dt, sc);
    __syncthreads();

    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.n0 || j >= g.n1) return;

    const float x = g.lo0 + (float)i * g.h0;
    const float y = g.lo1 + (float)j * g.h1;
    float dx, dy, J[4];
    trace2d<TR, VK>(vp, sc, x, y, (float)dt, dx, dy, J);

    int k, l;
    float xi, eta;
    locate(i, dx * g.ih0, g.n0, k, xi);
    locate(j, dy * g.ih1, g.n1, l, eta);

    const float *Pphi = in, *Ppx = in + g.plane, *Ppy = in + 2 * g.plane;
    float c[4][4];
#pragma unroll
    for (int B = 0; B < 2; ++B) {
        const int row = (l + B) * g.pitch;
#pragma unroll
        for (int A = 0; A < 2; ++A) {
            const int id = row + k + A;
            const int v = A + 2 * B;
            c[v][0] = __ldg(Pphi + id);
            c[v][1] = __ldg(Ppx + id);
            c[v][2] = __ldg(Ppy + id);
        }
        if (CR == CROSS_PLANE) {
            const float *Pxy = in + 3 * g.plane;
            c[2 * B][3] = __ldg(Pxy + row + k);
            c[2 * B + 1][3] = __ldg(Pxy + row + k + 1);
        } else {
            float w[4];
            w[1] = c[2 * B][2];
            w[2] = c[2 * B + 1][2];
            w[0] = __ldg(Ppy + row + max(k - 1, 0));
            w[3] = __ldg(Ppy + row + min(k + 2, g.n0 - 1));
            c[2 * B][3] = cross_from_window<0>(w, k, g.n0, g.i2h0);
            c[2 * B + 1][3] = cross_from_window<1>(w, k + 1, g.n0, g.i2h0);
        }
    }

    const Basis1 bx = basis1(xi, g.h0, g.ih0);
    const Basis1 by = basis1(eta, g.h1, g.ih1);
    float H, Hx, Hy;
    hermite2d(c, bx, by, H, Hx, Hy);

    const int o = j * g.pitch + i;
    out[o] = H;
    out[g.plane + o] = fmaf(J[0], Hx, J[2] * Hy);      // (J^T grad H)_x
    out[2 * g.plane + o] = fmaf(J[1], Hx, J[3] * Hy);  // (J^T grad H)_y
}

// phi_xy = d/dx psi_y at every node (approach A with one-sided ends).
__global__ void __launch_bounds__(BX *BY) k_recon2d(float *__restrict__ buf, Geom g)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.n0 || j >= g.n1) return;
    const float *py = buf + 2 * g.plane + (size_t)j * g.pitch;
    float v = dline(i, g.n0, g.i2h0, [&](int q) { return py[q]; });
    buf[3 * g.plane + (size_t)j * g.pitch + i] = v;
}

template <int TR, int VK, int CR>
cudaError_t launch_t(const StepLaunch &a, cudaStream_t s)
{
    dim3 block(BX, BY);
    dim3 grid((a.geom.n0 + BX - 1) / BX, (a.geom.n1 + BY - 1) / BY);
    k_step2d<TR, VK, CR><<<grid, block, 0, s>>>(a.in, a.out, a.geom, a.vp, a.t_dev, a.kstep, a.dt);
    return cudaGetLastError();
}

template <int TR, int VK>
cudaError_t launch_cr(const StepLaunch &a, cudaStream_t s)
{
    return a.cross_in == CROSS_PLANE ? launch_t<TR, VK, CROSS_PLANE>(a, s)
                                     : launch_t<TR, VK, CROSS_RECON>(a, s);
}

template <int VK>
cudaError_t launch_tr(const StepLaunch &a, cudaStream_t s)
{
    return a.trace == TR_EULER ? launch_cr<TR_EULER, VK>(a, s) : launch_cr<TR_RK3, VK>(a, s);
}

}  // namespace

cudaError_t launch_step2d(const StepLaunch &a, cudaStream_t s)
{
    cudaError_t e;
    switch (a.vp.kind) {
    case VK_CONST: e = launch_tr<VK_CONST>(a, s); break;
    case VK_ROTATION: e = launch_tr<VK_ROTATION>(a, s); break;
    case VK_VORTEX2D: e = launch_tr<VK_VORTEX2D>(a, s); break;
    case VK_PSEUDO1D: e = launch_tr<VK_PSEUDO1D>(a, s); break;
    case VK_FOURIER2D: e = launch_tr<VK_FOURIER2D>(a, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess || !a.write_cross) return e;
    return launch_recon(2, a.geom, a.out, s);
}

cudaError_t launch_recon2d(const Geom &g, float *buf, cudaStream_t s)
{
    dim3 block(BX, BY);
    dim3 grid((g.n0 + BX - 1) / BX, (g.n1 + BY - 1) / BY);
    k_recon2d<<<grid, block, 0, s>>>(buf, g);
    return cudaGetLastError();
}

}  // namespace gals
