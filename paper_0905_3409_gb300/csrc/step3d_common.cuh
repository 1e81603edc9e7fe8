// step3d_common.cuh -- per-node pieces of the 3D GALS step kernel (step3d.cu): the
// separable stage-1 deformation field and the cell-line reads with approach-A windows.
#pragma once

#include "gals_internal.h"
#include "gals_pair.cuh"
#include "tma.cuh"

namespace gals {
namespace t3 {

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

// v(x, t+dt) and Dv at the two nodes (x, y, z0) and (x, y, z1) of a thread.  For
// DEFORM3D the xy products of every term (P1..P7 of deform_terms) are fixed per thread
// (Pre3), so only the z-factors are evaluated per node.
struct Pre3 { float P1, P2, P3, P4, P5, P6, P7; };

template <int VK>
__device__ __forceinline__ Pre3 pre3(float x, float y)
{
    Pre3 p{};
    if (VK == VK_DEFORM3D) {
        float Axn, Bx, Ay, By;
        __sincosf(__fmaf_rn(x, -2.f * kPi, kPi), &Axn, &Bx);  // -A(x), B(x)
        sincos_turn(y, &Ay, &By);
        const float Sx2 = Bx + 1.f, Bxm = (-2.f * kPi) * Bx;
        const float Sy = __fmaf_rn(By, 0.5f, 0.5f), By2 = (2.f * kPi) * By;
        p.P1 = Sx2 * Ay; p.P2 = Axn * Sy; p.P3 = Axn * Ay; p.P4 = Sx2 * By2;
        p.P5 = Bxm * Sy; p.P6 = Bxm * Ay; p.P7 = Axn * By2;
    }
    return p;
}

template <int VK>
__device__ __forceinline__ V3p stage1_pair(const VelParams &vp, const StageCoef &sc, const Pre3 &p,
                                           F2 x, F2 y, F2 z)
{
    if (VK != VK_DEFORM3D) return vel3d_pair<VK>(vp, sc, 0, x, y, z);
    F2 Az, Bz;
    sincos_turn2(z, Az, Bz);
    const float c = sc.mod[0], h = 0.5f * c;
    V3p r;
    deform_terms(bc(p.P1), bc(p.P2), bc(p.P3), bc(p.P4), bc(p.P5), bc(p.P6), bc(p.P7),
                 mul2(bc(c), Az), fma2(Bz, bc(h), bc(h)), mul2(bc(2.f * kPi * c), Bz), r);
    return r;
}

// One x-line (y corner B, z corner C) of a foot cell with base corner (k, l, m): the data
// of planes 0..7 at x = k (lo) and x = k+1 (hi).  ld(a, z, y, x) reads plane a at a grid
// index.  With CROSS_RECON the mixed derivatives come from psi_y, psi_z windows with the
// approach-A stencils (central, one-sided at the ends), as in the reconstruction kernels.
template <int CR, class Ld>
__device__ __forceinline__ void cell_line(const Ld &ld, const Geom &g, int k, int l, int m, int B,
                                          int C, float lo[8], float hi[8])
{
    const int zz = m + C, yy = l + B;
    if (CR == CROSS_PLANE) {
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            lo[a] = ld(a, zz, yy, k);
            hi[a] = ld(a, zz, yy, k + 1);
        }
        return;
    }
    const int xs[4] = {max(k - 1, 0), k, k + 1, min(k + 2, g.n0 - 1)};
    const int ys[4] = {max(l - 1, 0), l, l + 1, min(l + 2, g.n1 - 1)};
    lo[0] = ld(0, zz, yy, k);
    hi[0] = ld(0, zz, yy, k + 1);
    lo[1] = ld(1, zz, yy, k);
    hi[1] = ld(1, zz, yy, k + 1);
    float wy[4], wz[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p) wy[p] = ld(2, zz, yy, xs[p]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) wz[q][p] = ld(3, zz, ys[q], xs[p]);
    // Dy psi_z on row yy at every x-window position
    float dyw[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float col[4] = {wz[0][p], wz[1][p], wz[2][p], wz[3][p]};
        dyw[p] = B == 0 ? dwin<0>(col, l, g.n1, g.i2h1) : dwin<1>(col, l + 1, g.n1, g.i2h1);
    }
    const float zrow[4] = {wz[B + 1][0], wz[B + 1][1], wz[B + 1][2], wz[B + 1][3]};
    lo[2] = wy[1];
    hi[2] = wy[2];
    lo[3] = zrow[1];
    hi[3] = zrow[2];
    lo[4] = dwin<0>(wy, k, g.n0, g.i2h0);
    hi[4] = dwin<1>(wy, k + 1, g.n0, g.i2h0);
    lo[5] = dwin<0>(zrow, k, g.n0, g.i2h0);
    hi[5] = dwin<1>(zrow, k + 1, g.n0, g.i2h0);
    lo[6] = dyw[1];
    hi[6] = dyw[2];
    lo[7] = dwin<0>(dyw, k, g.n0, g.i2h0);
    hi[7] = dwin<1>(dyw, k + 1, g.n0, g.i2h0);
}

}  // namespace t3
}  // namespace gals
