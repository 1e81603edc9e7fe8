// step3d.cu -- the 3D GALS step kernel and the 3D mixed-derivative reconstruction.
//
// One thread per grid node: trace back with the 3x3 Jacobian (Sec. 5.1, Ex.
// superconsistent Shu-Osher) -> locate the foot cell -> gather 8 corners x 8 data ->
// tricubic Hermite value and gradient (Sec. 2.3) -> phi+ = H, psi+ = J^T grad H.
// Mixed derivatives (Sec. 2.3, approach A): phi_xy = Dx psi_y, phi_xz = Dx psi_z,
// phi_yz = Dy psi_z, phi_xyz = Dx Dy psi_z, read from their planes (FULL) or rebuilt
// from psi windows around the cell (COMPACT) with the same stencils.
#include "gals_internal.h"

namespace gals {

namespace {

constexpr int BX = 32, BY = 4, BZ = 2;

template <int O>
__device__ __forceinline__ float dwin(const float w[4], int q, int n, float i2h)
{
    constexpr int c = 1 + O;
    if (O == 0) {
        if (q == 0) return dfirst(w[c], w[c + 1], w[c + 2], i2h);
    } else {
        if (q == n - 1) return dlast(w[c], w[c - 1], w[c - 2], i2h);
    }
    return dcentral(w[c + 1], w[c - 1], i2h);
}

template <int TR, int VK, int CR>
__global__ void __launch_bounds__(BX *BY *BZ)
k_step3d(const float *__restrict__ in, float *__restrict__ out, Geom g, VelParams vp,
         const StageCoef *__restrict__ coef, float dt)
{
    const StageCoef &sc = *coef;

    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int kz = blockIdx.z * BZ + threadIdx.z;
    if (i >= g.n0 || j >= g.n1 || kz >= g.n2) return;

    const float x = g.lo0 + (float)i * g.h0;
    const float y = g.lo1 + (float)j * g.h1;
    const float z = g.lo2 + (float)kz * g.h2;
    float d[3], J[9];
    trace3d<TR, VK>(vp, sc, x, y, z, dt, d, J);

    int k, l, m;
    float xi, eta, zeta;
    locate(i, d[0] * g.ih0, g.n0, k, xi);
    locate(j, d[1] * g.ih1, g.n1, l, eta);
    locate(kz, d[2] * g.ih2, g.n2, m, zeta);

    const int64_t P = g.plane;
    float c[8][8];
    if (CR == CROSS_PLANE) {
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int64_t id = ((int64_t)(m + (v >> 2)) * g.n1 + (l + ((v >> 1) & 1))) * g.pitch + k + (v & 1);
#pragma unroll
            for (int a = 0; a < 8; ++a) c[v][a] = __ldg(in + a * P + id);
        }
    } else {
        // psi_y on x-window [k-1, k+2] of the 4 corner lines; psi_z on the
        // x-window [k-1, k+2] x y-window [l-1, l+2] of both corner z-planes
        const int xs[4] = {max(k - 1, 0), k, k + 1, min(k + 2, g.n0 - 1)};
        const int ys[4] = {max(l - 1, 0), l, l + 1, min(l + 2, g.n1 - 1)};
        float wy[2][2][4], wz[2][4][4];
#pragma unroll
        for (int C = 0; C < 2; ++C) {
            const int64_t zoff = (int64_t)(m + C) * g.n1;
#pragma unroll
            for (int B = 0; B < 2; ++B) {
                const int64_t row = (zoff + l + B) * g.pitch;
#pragma unroll
                for (int p = 0; p < 4; ++p) wy[C][B][p] = __ldg(in + 2 * P + row + xs[p]);
#pragma unroll
                for (int A = 0; A < 2; ++A) {
                    const int v = A + 2 * B + 4 * C;
                    c[v][0] = __ldg(in + row + k + A);
                    c[v][1] = __ldg(in + P + row + k + A);
                    c[v][2] = wy[C][B][1 + A];
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t row = (zoff + ys[q]) * g.pitch;
#pragma unroll
                for (int p = 0; p < 4; ++p) wz[C][q][p] = __ldg(in + 3 * P + row + xs[p]);
            }
        }
#pragma unroll
        for (int C = 0; C < 2; ++C) {
#pragma unroll
            for (int B = 0; B < 2; ++B) {
                // Dy psi_z at every x-window position for row l+B
                float dyw[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    float col[4] = {wz[C][0][p], wz[C][1][p], wz[C][2][p], wz[C][3][p]};
                    dyw[p] = (B == 0) ? dwin<0>(col, l, g.n1, g.i2h1) : dwin<1>(col, l + 1, g.n1, g.i2h1);
                }
                float zrow[4] = {wz[C][B + 1][0], wz[C][B + 1][1], wz[C][B + 1][2], wz[C][B + 1][3]};
#pragma unroll
                for (int A = 0; A < 2; ++A) {
                    const int v = A + 2 * B + 4 * C;
                    c[v][3] = zrow[1 + A];
                    if (A == 0) {
                        c[v][4] = dwin<0>(wy[C][B], k, g.n0, g.i2h0);
                        c[v][5] = dwin<0>(zrow, k, g.n0, g.i2h0);
                        c[v][7] = dwin<0>(dyw, k, g.n0, g.i2h0);
                    } else {
                        c[v][4] = dwin<1>(wy[C][B], k + 1, g.n0, g.i2h0);
                        c[v][5] = dwin<1>(zrow, k + 1, g.n0, g.i2h0);
                        c[v][7] = dwin<1>(dyw, k + 1, g.n0, g.i2h0);
                    }
                    c[v][6] = dyw[1 + A];
                }
            }
        }
    }

    const Basis1 bx = basis1(xi, g.h0, g.ih0);
    const Basis1 by = basis1(eta, g.h1, g.ih1);
    const Basis1 bz = basis1(zeta, g.h2, g.ih2);
    float H, gr[3];
    hermite3d(c, bx, by, bz, H, gr);

    const int64_t o = ((int64_t)kz * g.n1 + j) * g.pitch + i;
    out[o] = H;
#pragma unroll
    for (int a = 0; a < 3; ++a)  // (J^T grad H)_a = sum_b J[b][a] dH/dx_b
        out[(a + 1) * P + o] = fmaf(J[a], gr[0], fmaf(J[3 + a], gr[1], J[6 + a] * gr[2]));
}

// Mixed derivatives at every node from psi_y, psi_z (approach A, one-sided ends).
__global__ void __launch_bounds__(BX *BY *BZ) k_recon3d(float *__restrict__ buf, Geom g)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int kz = blockIdx.z * BZ + threadIdx.z;
    if (i >= g.n0 || j >= g.n1 || kz >= g.n2) return;
    const int64_t P = g.plane;
    const float *py = buf + 2 * P, *pz = buf + 3 * P;
    auto at = [&](int ii, int jj) { return ((int64_t)kz * g.n1 + jj) * g.pitch + ii; };
    const int64_t o = at(i, j);
    buf[4 * P + o] = dline(i, g.n0, g.i2h0, [&](int q) { return py[at(q, j)]; });
    buf[5 * P + o] = dline(i, g.n0, g.i2h0, [&](int q) { return pz[at(q, j)]; });
    buf[6 * P + o] = dline(j, g.n1, g.i2h1, [&](int q) { return pz[at(i, q)]; });
    buf[7 * P + o] = dline(i, g.n0, g.i2h0, [&](int q) {
        return dline(j, g.n1, g.i2h1, [&](int r) { return pz[at(q, r)]; });
    });
}

template <int TR, int VK, int CR>
cudaError_t launch_t(const StepLaunch &a, cudaStream_t s)
{
    dim3 block(BX, BY, BZ);
    dim3 grid((a.geom.n0 + BX - 1) / BX, (a.geom.n1 + BY - 1) / BY, (a.geom.n2 + BZ - 1) / BZ);
    k_step3d<TR, VK, CR><<<grid, block, 0, s>>>(a.in, a.out, a.geom, a.vp, a.coef, (float)a.dt);
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

cudaError_t launch_step3d(const StepLaunch &a, cudaStream_t s)
{
    cudaError_t e;
    switch (a.vp.kind) {
    case VK_CONST: e = launch_tr<VK_CONST>(a, s); break;
    case VK_ROTATION: e = launch_tr<VK_ROTATION>(a, s); break;
    case VK_DEFORM3D: e = launch_tr<VK_DEFORM3D>(a, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess || !a.write_cross) return e;
    return launch_recon(3, a.geom, a.out, s);
}

cudaError_t launch_recon3d(const Geom &g, float *buf, cudaStream_t s)
{
    dim3 block(BX, BY, BZ);
    dim3 grid((g.n0 + BX - 1) / BX, (g.n1 + BY - 1) / BY, (g.n2 + BZ - 1) / BZ);
    k_recon3d<<<grid, block, 0, s>>>(buf, g);
    return cudaGetLastError();
}

}  // namespace gals
