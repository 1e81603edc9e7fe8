// step3d.cu -- the 3D GALS step kernel and the 3D mixed-derivative reconstruction.
//
// One thread per two grid nodes of a z-column, in paired FP32 (FFMA2): trace back with the
// 3x3 Jacobian (Sec. 5.1, superconsistent Shu-Osher RK3) -> locate the foot cell -> stream
// the cell's 4 x-lines (2 corners x 8 data) from the TMA-staged tile -> tricubic Hermite
// value and gradient (Sec. 2.3) -> phi+ = H, psi+ = J^T grad H.
// Mixed derivatives (Sec. 2.3, approach A): phi_xy = Dx psi_y, phi_xz = Dx psi_z,
// phi_yz = Dy psi_z, phi_xyz = Dx Dy psi_z, read from their planes (FULL) or rebuilt
// from psi windows around the cell (COMPACT) with the same stencils.
#include "step3d_common.cuh"

namespace gals {

namespace {

using namespace t3;

// Output tile per block: TX x TY nodes in x, y and TZ in z (each thread walks TZ nodes in z).
constexpr int TX = 32, TY = 4, TZ = 4;
constexpr int HX = 4, HZ = 1;          // halo (x rounded to 16 bytes for TMA)
template <int CR> struct Tile3 {
    // psi_z y-window needs one more row (CROSS_RECON); CROSS_CELL shares that tile's map
    static constexpr int HY = CR == CROSS_PLANE ? 1 : 2;
    static constexpr int NP = CR == CROSS_PLANE ? 8 : 4;
    static constexpr int W = TX + 2 * HX, H = TY + 2 * HY, D = TZ + 2 * HZ;
    static constexpr int PS = W * H * D;
    static constexpr int BYTES = NP * PS * 4;
};

// Two nodes per thread, (i, j, kz) and (i, j, kz+1), in paired FP32: trace with the 3x3
// Jacobian, cell location, tricubic Hermite value and gradient from the staged tile,
// phi+ = H and psi+ = J^T grad H.  Feet whose cell data lie outside the staged tile
// (large CFL) read global memory instead.
// FULL layout: at most 128 registers (4 blocks per SM; a few words spill), measured faster
// than 166 registers at 3 blocks per SM.
template <int TR, int VK, int CR>
__global__ void __launch_bounds__(TX *TY, CR == CROSS_PLANE ? 4 : 1)
k_step3d(const float *__restrict__ in, float *__restrict__ out, Geom g, VelParams vp,
         const StageCoef *__restrict__ coef, float dt, const __grid_constant__ CUtensorMap tmap,
         int *__restrict__ err, int zt0)
{
    using T = Tile3<CR>;
    extern __shared__ __align__(128) float tile[];
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x + TX * threadIdx.y;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = (blockIdx.z + zt0) * TZ;
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, T::BYTES);
        tma_load_4d(tile, &tmap, x0 - HX, y0 - T::HY, z0 - HZ, 0, &bar);
    }
    const StageCoef &sc = *coef;
    // threads past a ragged edge trace a clamped node and store nothing
    const bool valid = x0 + (int)threadIdx.x < g.n0 && y0 + (int)threadIdx.y < g.n1;
    const int i = min(x0 + (int)threadIdx.x, g.n0 - 1), j = min(y0 + (int)threadIdx.y, g.n1 - 1);
    const float x = g.lo0 + (float)i * g.h0;
    const float y = g.lo1 + (float)j * g.h1;
    const Pre3 pre = pre3<VK>(x, y);
    const int64_t P = g.plane;
    const int64_t zstride = (int64_t)g.n1 * g.pitch;
    const int zend = min(z0 + TZ, g.n2);
    const F2 X = bc(x), Y = bc(y);
    for (int kz = z0; kz < zend; kz += 2) {
        const bool two = kz + 1 < zend;
        const int kz1 = two ? kz + 1 : kz;
        const F2 Z = make_float2(g.lo2 + (float)kz * g.h2, g.lo2 + (float)kz1 * g.h2);
        F2 d[3], J[9];
        if (kz == z0) {
            if (!mbar_wait_block(&bar, 0)) {
                if (tid == 0) {
                    atomicExch(err, kErrTmaTimeout);
                    mbar_wait_bounded(&bar, 0);
                }
                return;
            }
        }
        trace3d_pair<TR, VK>(stage1_pair<VK>(vp, sc, pre, X, Y, Z), vp, sc, X, Y, Z, dt, d, J);

        int k0, l0, m0, k1, l1, m1;
        float xi0, eta0, zeta0, xi1, eta1, zeta1;
        locate(i, d[0].x * g.ih0, g.n0, k0, xi0);
        locate(j, d[1].x * g.ih1, g.n1, l0, eta0);
        locate(kz, d[2].x * g.ih2, g.n2, m0, zeta0);
        locate(i, d[0].y * g.ih0, g.n0, k1, xi1);
        locate(j, d[1].y * g.ih1, g.n1, l1, eta1);
        locate(kz1, d[2].y * g.ih2, g.n2, m1, zeta1);
        const Basis2 bx = basis_pair(make_float2(xi0, xi1), g.h0, g.ih0);
        const Basis2 by = basis_pair(make_float2(eta0, eta1), g.h1, g.ih1);
        const Basis2 bz = basis_pair(make_float2(zeta0, zeta1), g.h2, g.ih2);

        // a cell is served from the tile if every value its line reads is staged
        auto in_tile = [&](int k, int l, int m) {
            const int tx = k - x0 + HX, ty = l - y0 + T::HY, tz = m - z0 + HZ;
            return CR != CROSS_RECON
                ? (tx >= 0 && tx <= T::W - 2 && ty >= 0 && ty <= T::H - 2 && tz >= 0 && tz <= T::D - 2)
                : (tx >= 1 && tx <= T::W - 3 && ty >= 1 && ty <= T::H - 3 && tz >= 0 && tz <= T::D - 2);
        };
        auto lds = [&](int a, int zz, int yy, int xx) {
            return tile[GALS_CHK(g, a * T::PS + ((zz - z0 + HZ) * T::H + yy - y0 + T::HY) * T::W + xx - x0 + HX,
                                 T::NP * T::PS)];
        };
        auto ldg = [&](int a, int zz, int yy, int xx) {
#ifdef GALS_CHECKED
            return __ldg(in + a * P + GALS_CHK(g, (int64_t)zz * zstride + (int64_t)yy * g.pitch + xx, plane_extent(g)));
#else
            return __ldg(in + a * P + (int64_t)zz * zstride + (int64_t)yy * g.pitch + xx);
#endif
        };
        const bool in0 = in_tile(k0, l0, m0), in1 = in_tile(k1, l1, m1);
        F2 H, gr[3];
        if (CR == CROSS_CELL) {
            // approach B: the cell's 8 vertices x (phi, psi) per foot, mixed derivatives from them
            auto ld0 = [&](int a, int zz, int yy, int xx) { return in0 ? lds(a, zz, yy, xx) : ldg(a, zz, yy, xx); };
            auto ld1 = [&](int a, int zz, int yy, int xx) { return in1 ? lds(a, zz, yy, xx) : ldg(a, zz, yy, xx); };
            float q0[8][4], q1[8][4], c0[8][4], c1[8][4];
#pragma unroll
            for (int v = 0; v < 8; ++v)
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    q0[v][a] = ld0(a, m0 + (v >> 2), l0 + ((v >> 1) & 1), k0 + (v & 1));
                    q1[v][a] = ld1(a, m1 + (v >> 2), l1 + ((v >> 1) & 1), k1 + (v & 1));
                }
            cross_cell3d([&](int v, int a) { return q0[v][a]; }, g.ih0, g.ih1, g.ih2, c0);
            cross_cell3d([&](int v, int a) { return q1[v][a]; }, g.ih0, g.ih1, g.ih2, c1);
            hermite3d_pair(bx, by, bz, [&](int B, int C, F2 lo[8], F2 hi[8]) {
                const int v = 2 * B + 4 * C;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    lo[a] = make_float2(q0[v][a], q1[v][a]);
                    hi[a] = make_float2(q0[v + 1][a], q1[v + 1][a]);
                    lo[4 + a] = make_float2(c0[v][a], c1[v][a]);
                    hi[4 + a] = make_float2(c0[v + 1][a], c1[v + 1][a]);
                }
            }, H, gr);
        } else if (in0 && in1) {
            hermite3d_pair(bx, by, bz, [&](int B, int C, F2 lo[8], F2 hi[8]) {
                float a0[8], b0[8], a1[8], b1[8];
                cell_line<CR>(lds, g, k0, l0, m0, B, C, a0, b0);
                cell_line<CR>(lds, g, k1, l1, m1, B, C, a1, b1);
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    lo[a] = make_float2(a0[a], a1[a]);
                    hi[a] = make_float2(b0[a], b1[a]);
                }
            }, H, gr);
        } else {
            auto ld0 = [&](int a, int zz, int yy, int xx) { return in0 ? lds(a, zz, yy, xx) : ldg(a, zz, yy, xx); };
            auto ld1 = [&](int a, int zz, int yy, int xx) { return in1 ? lds(a, zz, yy, xx) : ldg(a, zz, yy, xx); };
            hermite3d_pair(bx, by, bz, [&](int B, int C, F2 lo[8], F2 hi[8]) {
                float a0[8], b0[8], a1[8], b1[8];
                cell_line<CR>(ld0, g, k0, l0, m0, B, C, a0, b0);
                cell_line<CR>(ld1, g, k1, l1, m1, B, C, a1, b1);
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    lo[a] = make_float2(a0[a], a1[a]);
                    hi[a] = make_float2(b0[a], b1[a]);
                }
            }, H, gr);
        }
        F2 psi[3];
        if (TR == TR_HEUN) {
            // CIR gradient update (Sec. 4): Dv at the foot at time t, Dv at the node at t + dt
            const V3p Df = vel3d_pair<VK>(vp, sc, 1, add2(X, d[0]), add2(Y, d[1]), add2(Z, d[2]));
            const V3p Dn = stage1_pair<VK>(vp, sc, pre, X, Y, Z);
            heun_psi3(Df, Dn, dt, gr, psi);
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a)  // (J^T grad H)_a = sum_b J[b][a] dH/dx_b
                psi[a] = fma2(J[a], gr[0], fma2(J[3 + a], gr[1], mul2(J[6 + a], gr[2])));
        }
        if (!valid) continue;
        const int64_t o = GALS_CHK(g, (int64_t)kz * zstride + (int64_t)j * g.pitch + i, plane_extent(g));
        out[o] = H.x;
#pragma unroll
        for (int a = 0; a < 3; ++a) out[(a + 1) * P + o] = psi[a].x;
        if (two) {
#ifdef GALS_CHECKED
            const int64_t o1 = GALS_CHK(g, o + zstride, plane_extent(g));
            out[o1] = H.y;
#pragma unroll
            for (int a = 0; a < 3; ++a) out[(a + 1) * P + o1] = psi[a].y;
#else
            out[o + zstride] = H.y;
#pragma unroll
            for (int a = 0; a < 3; ++a) out[(a + 1) * P + o + zstride] = psi[a].y;
#endif
        }
    }
}

// Mixed derivatives at every node from psi_y, psi_z (approach A, one-sided ends):
// phi_xy = Dx psi_y, phi_xz = Dx psi_z, phi_yz = Dy psi_z, phi_xyz = Dx (Dy psi_z).
// One thread per (x, y) column walks RZ z-slices; every stencil operand is a direct
// read-only load (neighbours' reads hit L1), with no barriers, so all loads of a slice are
// in flight together.  The stencil functions are the ones the step kernels use, so the
// results are identical.
constexpr int RX = 32, RY = 8, RZ = 4;

__global__ void __launch_bounds__(RX *RY) k_recon3d(const float *__restrict__ py,
                                                     const float *__restrict__ pz,
                                                     float *__restrict__ cross, Geom g)
{
    const int i = blockIdx.x * RX + threadIdx.x, j = blockIdx.y * RY + threadIdx.y;
    if (i >= g.n0 || j >= g.n1) return;
    const int64_t P = g.plane;
    const int z0 = blockIdx.z * RZ, zend = min(z0 + RZ, g.n2);
#pragma unroll
    for (int dz = 0; dz < RZ; ++dz) {
        const int kz = z0 + dz;
        if (kz >= zend) break;
        const int64_t row = ((int64_t)kz * g.n1) * g.pitch;
        const float *ly = py + row, *lz = pz + row;
        auto Y = [&](int xx, int yy) { return __ldg(ly + (int64_t)yy * g.pitch + xx); };
        auto Z = [&](int xx, int yy) { return __ldg(lz + (int64_t)yy * g.pitch + xx); };
        const float fxy = dline(i, g.n0, g.i2h0, [&](int q) { return Y(q, j); });
        const float fxz = dline(i, g.n0, g.i2h0, [&](int q) { return Z(q, j); });
        const float fyz = dline(j, g.n1, g.i2h1, [&](int r) { return Z(i, r); });
        const float fxyz = dline(i, g.n0, g.i2h0, [&](int q) {
            return dline(j, g.n1, g.i2h1, [&](int r) { return Z(q, r); });
        });
        const int64_t o = row + (int64_t)j * g.pitch + i;
        cross[o] = fxy;
        cross[P + o] = fxz;
        cross[2 * P + o] = fyz;
        cross[3 * P + o] = fxyz;
    }
}

// The same reconstruction after a FULL step, with psi_y and psi_z of a block's nodes
// (x-halo 4 for 16-byte TMA rows, y-halo 2 for the one-sided ends) staged in shared memory
// by one TMA copy: a block of 32 x 8 threads covers QZ z-slices.
constexpr int QX = 32, QY = 8, QZ = 4, QHX = 4, QHY = 2;
constexpr int QW = QX + 2 * QHX, QH = QY + 2 * QHY;

__global__ void __launch_bounds__(QX *QY)
k_recon3d_tma(float *__restrict__ buf, Geom g, const __grid_constant__ CUtensorMap map,
              int *__restrict__ err, int zq0)
{
    __shared__ __align__(128) float t[2][QZ][QH][QW];  // psi_y, psi_z
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x + QX * threadIdx.y;
    // slabs zq0 .. zq0 + gridDim.z - 1, in reverse: the step kernel wrote the last slabs
    // last, so their psi_y, psi_z are the ones most likely still in L2
    const int x0 = blockIdx.x * QX, y0 = blockIdx.y * QY;
    const int z0 = (zq0 + (int)gridDim.z - 1 - (int)blockIdx.z) * QZ;
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, (uint32_t)sizeof(t));
        tma_load_4d(&t[0][0][0][0], &map, x0 - QHX, y0 - QHY, z0, 2, &bar);
    }
    if (!mbar_wait_block(&bar, 0)) {
        if (tid == 0) {
            atomicExch(err, kErrTmaTimeout);
            mbar_wait_bounded(&bar, 0);
        }
        return;
    }
    const int i = x0 + threadIdx.x, j = y0 + threadIdx.y;
    if (i >= g.n0 || j >= g.n1) return;
    const int64_t P = g.plane;
    const int nz = min(QZ, g.n2 - z0);
    if (x0 >= 1 && x0 + QX <= g.n0 - 1 && y0 >= 1 && y0 + QY <= g.n1 - 1) {
        // every node of the block is interior in x and y: central differences only (the
        // same operations dline performs there)
        const int tx = threadIdx.x + QHX, ty = threadIdx.y + QHY;
        int64_t o = ((int64_t)z0 * g.n1 + j) * g.pitch + i;
        const int64_t zs = (int64_t)g.n1 * g.pitch;
        for (int dz = 0; dz < nz; ++dz, o += zs) {
            const float(*Y)[QW] = t[0][dz];
            const float(*Z)[QW] = t[1][dz];
            buf[4 * P + o] = dcentral(Y[ty][tx + 1], Y[ty][tx - 1], g.i2h0);
            buf[5 * P + o] = dcentral(Z[ty][tx + 1], Z[ty][tx - 1], g.i2h0);
            buf[6 * P + o] = dcentral(Z[ty + 1][tx], Z[ty - 1][tx], g.i2h1);
            buf[7 * P + o] = dcentral(dcentral(Z[ty + 1][tx + 1], Z[ty - 1][tx + 1], g.i2h1),
                                      dcentral(Z[ty + 1][tx - 1], Z[ty - 1][tx - 1], g.i2h1), g.i2h0);
        }
        return;
    }
    for (int dz = 0; dz < nz; ++dz) {
        auto Y = [&](int q, int r) { return t[0][dz][r - y0 + QHY][q - x0 + QHX]; };
        auto Z = [&](int q, int r) { return t[1][dz][r - y0 + QHY][q - x0 + QHX]; };
        const int64_t o = ((int64_t)(z0 + dz) * g.n1 + j) * g.pitch + i;
        buf[4 * P + o] = dline(i, g.n0, g.i2h0, [&](int q) { return Y(q, j); });
        buf[5 * P + o] = dline(i, g.n0, g.i2h0, [&](int q) { return Z(q, j); });
        buf[6 * P + o] = dline(j, g.n1, g.i2h1, [&](int r) { return Z(i, r); });
        buf[7 * P + o] = dline(i, g.n0, g.i2h0, [&](int q) {
            return dline(j, g.n1, g.i2h1, [&](int r) { return Z(q, r); });
        });
    }
}

template <int TR, int VK, int CR>
cudaError_t launch_t(const StepLaunch &a, cudaStream_t s, int zt0, int nzt)
{
    using T = Tile3<CR>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_step3d<TR, VK, CR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, T::BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 block(TX, TY);
    dim3 grid((a.geom.n0 + TX - 1) / TX, (a.geom.n1 + TY - 1) / TY, nzt);
    const CUtensorMap &map = CR == CROSS_PLANE ? *a.tmap4 : *a.tmap3;
    k_step3d<TR, VK, CR><<<grid, block, T::BYTES, s>>>(a.in, a.out, a.geom, a.vp, a.coef,
                                                      (float)a.dt, map, a.err, zt0);
    return cudaGetLastError();
}

template <int TR, int VK>
cudaError_t launch_cr(const StepLaunch &a, cudaStream_t s, int zt0, int nzt)
{
    if (a.cross_in == CROSS_CELL) return launch_t<TR, VK, CROSS_CELL>(a, s, zt0, nzt);
    return a.cross_in == CROSS_PLANE ? launch_t<TR, VK, CROSS_PLANE>(a, s, zt0, nzt)
                                     : launch_t<TR, VK, CROSS_RECON>(a, s, zt0, nzt);
}

template <int VK>
cudaError_t launch_tr(const StepLaunch &a, cudaStream_t s, int zt0, int nzt)
{
    if (a.trace == TR_HEUN) return launch_cr<TR_HEUN, VK>(a, s, zt0, nzt);
    return a.trace == TR_EULER ? launch_cr<TR_EULER, VK>(a, s, zt0, nzt)
                               : launch_cr<TR_RK3, VK>(a, s, zt0, nzt);
}

// step kernel over the z-tiles [zt0, zt0 + nzt)
cudaError_t launch_step_tiles(const StepLaunch &a, cudaStream_t s, int zt0, int nzt)
{
    switch (a.vp.kind) {
    case VK_CONST: return launch_tr<VK_CONST>(a, s, zt0, nzt);
    case VK_ROTATION: return launch_tr<VK_ROTATION>(a, s, zt0, nzt);
    case VK_DEFORM3D: return launch_tr<VK_DEFORM3D>(a, s, zt0, nzt);
    default: return cudaErrorInvalidValue;
    }
}

// reconstruction of the z-slabs [zq0, zq0 + nzq) of the new state
cudaError_t launch_recon_slabs(const StepLaunch &a, cudaStream_t s, int zq0, int nzq)
{
    dim3 grid((a.geom.n0 + QX - 1) / QX, (a.geom.n1 + QY - 1) / QY, nzq);
    k_recon3d_tma<<<grid, dim3(QX, QY), 0, s>>>(a.out, a.geom, *a.tmap_cross, a.err, zq0);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step3d(const StepLaunch &a, cudaStream_t s)
{
    // z-levels of the band (all by default); the reconstruction of a level needs the new
    // psi_y, psi_z of that level only
    static_assert(TZ == 4 && QZ == 4, "bands are whole tiles of both kernels");
    const int z0 = a.band_lo, z1 = a.band_hi > 0 ? a.band_hi : a.geom.n2;
    if (z1 <= z0) return cudaSuccess;
    cudaError_t e = launch_step_tiles(a, s, z0 / TZ, (z1 - z0 + TZ - 1) / TZ);
    if (e != cudaSuccess || !a.write_cross) return e;
    return launch_recon_slabs(a, s, z0 / QZ, (z1 - z0 + QZ - 1) / QZ);
}

void recon_box3d(uint32_t box[4])
{
    box[0] = QW; box[1] = QH; box[2] = QZ; box[3] = 2;
}

void tile_box3d(int cross_recon, uint32_t box[4])
{
    if (cross_recon) {
        using T = Tile3<CROSS_RECON>;
        box[0] = T::W; box[1] = T::H; box[2] = T::D; box[3] = T::NP;
    } else {
        using T = Tile3<CROSS_PLANE>;
        box[0] = T::W; box[1] = T::H; box[2] = T::D; box[3] = T::NP;
    }
}

cudaError_t launch_recon3d(const Geom &g, float *buf, cudaStream_t s)
{
    dim3 block(RX, RY);
    dim3 grid((g.n0 + RX - 1) / RX, (g.n1 + RY - 1) / RY, (g.n2 + RZ - 1) / RZ);
    k_recon3d<<<grid, block, 0, s>>>(buf + 2 * g.plane, buf + 3 * g.plane, buf + 4 * g.plane, g);
    return cudaGetLastError();
}

}  // namespace gals
