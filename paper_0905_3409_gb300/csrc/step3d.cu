// step3d.cu -- the 3D GALS step kernel and the 3D mixed-derivative reconstruction.
//
// One thread per grid node: trace back with the 3x3 Jacobian (Sec. 5.1, Ex.
// superconsistent Shu-Osher) -> locate the foot cell -> gather 8 corners x 8 data ->
// tricubic Hermite value and gradient (Sec. 2.3) -> phi+ = H, psi+ = J^T grad H.
// Mixed derivatives (Sec. 2.3, approach A): phi_xy = Dx psi_y, phi_xz = Dx psi_z,
// phi_yz = Dy psi_z, phi_xyz = Dx Dy psi_z, read from their planes (FULL) or rebuilt
// from psi windows around the cell (COMPACT) with the same stencils.
#include "gals_internal.h"
#include "tma.cuh"

namespace gals {

namespace {

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

// Output tile per block: TX x TY nodes in x, y and TZ in z (each thread walks TZ nodes in z).
constexpr int TX = 32, TY = 4, TZ = 4;
constexpr int HX = 4, HZ = 1;          // halo (x rounded to 16 bytes for TMA)
template <int CR> struct Tile3 {
    static constexpr int HY = CR == CROSS_RECON ? 2 : 1;  // psi_z y-window needs one more
    static constexpr int NP = CR == CROSS_RECON ? 4 : 8;
    static constexpr int W = TX + 2 * HX, H = TY + 2 * HY, D = TZ + 2 * HZ;
    static constexpr int PS = W * H * D;
    static constexpr int BYTES = NP * PS * 4;
};

// Separable factors of the deformation field on a grid line.
struct Sep { float s2, s2x, c2x; };
__device__ __forceinline__ Sep sep3(float s)
{
    float sn, cs;
    sincospi_f(s, &sn, &cs);
    return Sep{sn * sn, 2.f * sn * cs, 1.f - 2.f * sn * sn};
}

// v(x, t+dt) at a node; DEFORM3D from per-axis factors
template <int VK>
__device__ __forceinline__ V3 stage1_3d(const VelParams &vp, const StageCoef &sc, float x,
                                        float y, float z, const Sep &fx, const Sep &fy,
                                        const Sep &fz)
{
    if (VK == VK_DEFORM3D) {
        V3 r;
        const float c = sc.mod[0], cp = c * kPi;
        const float sss = fx.s2x * fy.s2x * fz.s2x;
        r.v[0] = 2.f * c * fx.s2 * fy.s2x * fz.s2x;
        r.v[1] = -c * fx.s2x * fy.s2 * fz.s2x;
        r.v[2] = -c * fx.s2x * fy.s2x * fz.s2;
        r.d[0] = 2.f * cp * sss;
        r.d[1] = 4.f * cp * fx.s2 * fy.c2x * fz.s2x;
        r.d[2] = 4.f * cp * fx.s2 * fy.s2x * fz.c2x;
        r.d[3] = -2.f * cp * fx.c2x * fy.s2 * fz.s2x;
        r.d[4] = -cp * sss;
        r.d[5] = -2.f * cp * fx.s2x * fy.s2 * fz.c2x;
        r.d[6] = -2.f * cp * fx.c2x * fy.s2x * fz.s2;
        r.d[7] = -2.f * cp * fx.s2x * fy.c2x * fz.s2;
        r.d[8] = r.d[4];
        return r;
    }
    return vel3d<VK>(vp, sc, 0, x, y, z);
}

template <int TR, int VK, int CR>
__global__ void __launch_bounds__(TX *TY)
k_step3d(const float *__restrict__ in, float *__restrict__ out, Geom g, VelParams vp,
         const StageCoef *__restrict__ coef, float dt, const __grid_constant__ CUtensorMap tmap,
         int *__restrict__ err)
{
    using T = Tile3<CR>;
    extern __shared__ __align__(128) float tile[];
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x + TX * threadIdx.y;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, T::BYTES);
        tma_load_4d(tile, &tmap, x0 - HX, y0 - T::HY, z0 - HZ, 0, &bar);
    }
    const StageCoef &sc = *coef;
    const int i = x0 + threadIdx.x, j = y0 + threadIdx.y;
    const float x = g.lo0 + (float)i * g.h0;
    const float y = g.lo1 + (float)j * g.h1;
    const Sep fx = VK == VK_DEFORM3D ? sep3(x) : Sep{0.f, 0.f, 0.f};
    const Sep fy = VK == VK_DEFORM3D ? sep3(y) : Sep{0.f, 0.f, 0.f};

    const bool ok = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicExch(err, kErrTmaTimeout);
            mbar_wait_bounded(&bar, 0);
        }
        return;
    }
    if (i >= g.n0 || j >= g.n1) return;
    const int64_t P = g.plane;
    const int zend = min(z0 + TZ, g.n2);
    for (int kz = z0; kz < zend; ++kz) {
        const float z = g.lo2 + (float)kz * g.h2;
        const Sep fz = VK == VK_DEFORM3D ? sep3(z) : Sep{0.f, 0.f, 0.f};
        float d[3], J[9];
        trace3d_from<TR, VK>(stage1_3d<VK>(vp, sc, x, y, z, fx, fy, fz), vp, sc, x, y, z, dt, d, J);

        int k, l, m;
        float xi, eta, zeta;
        locate(i, d[0] * g.ih0, g.n0, k, xi);
        locate(j, d[1] * g.ih1, g.n1, l, eta);
        locate(kz, d[2] * g.ih2, g.n2, m, zeta);

        // staged-tile coordinates of the cell's base corner
        const int tx = k - x0 + HX, ty = l - y0 + T::HY, tz = m - z0 + HZ;
        const bool inside = CR == CROSS_PLANE
            ? (tx >= 0 && tx <= T::W - 2 && ty >= 0 && ty <= T::H - 2 && tz >= 0 && tz <= T::D - 2)
            : (tx >= 1 && tx <= T::W - 3 && ty >= 1 && ty <= T::H - 3 && tz >= 0 && tz <= T::D - 2);
        // element (plane a, corner offsets dz, dy, dx relative to the cell base)
        auto sm = [&](int a, int dz, int dy, int dx) {
            return tile[a * T::PS + ((tz + dz) * T::H + ty + dy) * T::W + tx + dx];
        };
        auto gm = [&](int a, int zz, int yy, int xx) {
            return __ldg(in + a * P + ((int64_t)zz * g.n1 + yy) * g.pitch + xx);
        };
        float c[8][8];
        if (CR == CROSS_PLANE) {
            if (inside) {
#pragma unroll
                for (int v = 0; v < 8; ++v)
#pragma unroll
                    for (int a = 0; a < 8; ++a) c[v][a] = sm(a, v >> 2, (v >> 1) & 1, v & 1);
            } else {
#pragma unroll
                for (int v = 0; v < 8; ++v)
#pragma unroll
                    for (int a = 0; a < 8; ++a)
                        c[v][a] = gm(a, m + (v >> 2), l + ((v >> 1) & 1), k + (v & 1));
            }
        } else {
            // psi_y on the x-window [k-1, k+2] of the 4 corner lines; psi_z on the
            // x-window [k-1, k+2] x y-window [l-1, l+2] of both corner z-planes
            const int xs[4] = {max(k - 1, 0), k, k + 1, min(k + 2, g.n0 - 1)};
            const int ys[4] = {max(l - 1, 0), l, l + 1, min(l + 2, g.n1 - 1)};
            float wy[2][2][4], wz[2][4][4];
#pragma unroll
            for (int C = 0; C < 2; ++C) {
#pragma unroll
                for (int B = 0; B < 2; ++B) {
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        wy[C][B][p] = inside ? sm(2, C, B, p - 1) : gm(2, m + C, l + B, xs[p]);
#pragma unroll
                    for (int A = 0; A < 2; ++A) {
                        const int v = A + 2 * B + 4 * C;
                        c[v][0] = inside ? sm(0, C, B, A) : gm(0, m + C, l + B, k + A);
                        c[v][1] = inside ? sm(1, C, B, A) : gm(1, m + C, l + B, k + A);
                        c[v][2] = wy[C][B][1 + A];
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        wz[C][q][p] = inside ? sm(3, C, q - 1, p - 1) : gm(3, m + C, ys[q], xs[p]);
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
}

// Mixed derivatives at every node from psi_y, psi_z (approach A, one-sided ends):
// phi_xy = Dx psi_y, phi_xz = Dx psi_z, phi_yz = Dy psi_z, phi_xyz = Dx (Dy psi_z).
// A block of 32 x 8 threads walks RZ slices of a 32 x 8 xy-tile; each slice's psi_y,
// psi_z (x-halo 2, y-halo 2 for the one-sided ends) and the y-differences of psi_z are
// staged in shared memory, so every input is read once with coalesced loads.  The
// stencil functions are the ones the step kernels use, so the results are identical.
constexpr int RX = 32, RY = 8, RZ = 8, RW = RX + 4;

__global__ void __launch_bounds__(RX *RY) k_recon3d(float *__restrict__ buf, Geom g)
{
    __shared__ float spy[RY][RW];
    __shared__ float spz[RY + 4][RW];
    __shared__ float sdy[RY][RW];
    const int x0 = blockIdx.x * RX, y0 = blockIdx.y * RY, z0 = blockIdx.z * RZ;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + RX * ty;
    const int64_t P = g.plane;
    const float *py = buf + 2 * P, *pz = buf + 3 * P;
    const int i = x0 + tx, j = y0 + ty;
    const int zend = min(z0 + RZ, g.n2);
    for (int kz = z0; kz < zend; ++kz) {
        const int64_t zoff = (int64_t)kz * g.n1;
        // stage psi_y (rows y0..y0+7) and psi_z (rows y0-2..y0+9), columns x0-2..x0+33
        for (int e = tid; e < (RY + (RY + 4)) * RW; e += RX * RY) {
            const bool isz = e >= RY * RW;
            const int ee = isz ? e - RY * RW : e;
            const int r = ee / RW, c = ee % RW;
            const int gx = x0 - 2 + c, gy = (isz ? y0 - 2 : y0) + r;
            float v = 0.f;
            if (gx >= 0 && gx < g.n0 && gy >= 0 && gy < g.n1)
                v = (isz ? pz : py)[(zoff + gy) * g.pitch + gx];
            if (isz) spz[r][c] = v; else spy[r][c] = v;
        }
        __syncthreads();
        // Dy psi_z on rows y0..y0+7 for every staged column
        for (int e = tid; e < RY * RW; e += RX * RY) {
            const int r = e / RW, c = e % RW;
            const int gy = y0 + r, gx = x0 - 2 + c;
            float v = 0.f;
            if (gy < g.n1 && gx >= 0 && gx < g.n0)
                v = dline(gy, g.n1, g.i2h1, [&](int q) { return spz[q - y0 + 2][c]; });
            sdy[r][c] = v;
        }
        __syncthreads();
        if (i < g.n0 && j < g.n1) {
            const int64_t o = (zoff + j) * g.pitch + i;
            buf[4 * P + o] = dline(i, g.n0, g.i2h0, [&](int q) { return spy[ty][q - x0 + 2]; });
            buf[5 * P + o] = dline(i, g.n0, g.i2h0, [&](int q) { return spz[ty + 2][q - x0 + 2]; });
            buf[6 * P + o] = sdy[ty][tx + 2];
            buf[7 * P + o] = dline(i, g.n0, g.i2h0, [&](int q) { return sdy[ty][q - x0 + 2]; });
        }
        __syncthreads();
    }
}

template <int TR, int VK, int CR>
cudaError_t launch_t(const StepLaunch &a, cudaStream_t s)
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
    dim3 grid((a.geom.n0 + TX - 1) / TX, (a.geom.n1 + TY - 1) / TY, (a.geom.n2 + TZ - 1) / TZ);
    const CUtensorMap &map = CR == CROSS_PLANE ? *a.tmap4 : *a.tmap3;
    k_step3d<TR, VK, CR><<<grid, block, T::BYTES, s>>>(a.in, a.out, a.geom, a.vp, a.coef,
                                                      (float)a.dt, map, a.err);
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
    k_recon3d<<<grid, block, 0, s>>>(buf, g);
    return cudaGetLastError();
}

}  // namespace gals
