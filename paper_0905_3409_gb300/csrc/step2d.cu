// step2d.cu -- the fused 2D GALS step kernel and the mixed-derivative reconstruction.
//
// Per grid node (Sec. 4, steps 1-2 in the superconsistent form of Sec. 5.1):
//   trace back with the Jacobian -> locate the foot cell -> gather the 4 corners x 4 data
//   -> bicubic Hermite value and gradient -> phi+ = H, psi+ = J^T grad H,
// then (Sec. 2.3, approach A) phi_xy+ = d/dx psi_y+ by central differences.
//
// Work decomposition: a block of 128 threads owns a tile of 128 columns x 16 rows; each
// thread walks its column.  The new psi_y of the tile, plus one halo column on each side
// (recomputed by the block: 2 extra node updates per 128), is kept in shared memory, so
// phi_xy+ is written by the same kernel: one launch per step, the state read once and
// written once (32 bytes per node update in the FULL layout).
//
// The mixed derivative of the 4 corners is either read from its plane (the stored
// representation of Sec. 5.2) or rebuilt on the fly from psi_y (COMPACT layout); both use
// the same stencil code and round identically.
#include "gals_internal.h"

namespace gals {

namespace {

constexpr int TX = 128, TY = 16;

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

// Separable factors of the single-vortex field at a grid line: sin^2(pi s),
// sin(2 pi s), cos(2 pi s).
struct Sep { float s2, s2x, c2x; };

__device__ __forceinline__ Sep sep_factors(float s)
{
    float sn, cs;
    sincospi_f(s, &sn, &cs);
    Sep f;
    f.s2 = sn * sn;
    f.s2x = 2.f * sn * cs;
    f.c2x = 1.f - 2.f * sn * sn;
    return f;
}

// v(x, t+dt) at a node; the single vortex uses the separable column/row factors.
template <int VK>
__device__ __forceinline__ V2 stage1(const VelParams &vp, const StageCoef &sc, float x, float y,
                                     const Sep &cx, const Sep &ry)
{
    if (VK == VK_VORTEX2D) {
        V2 r;
        const float c = sc.mod[0], cp = c * kPi;
        r.u = -c * cx.s2 * ry.s2x;
        r.v = c * cx.s2x * ry.s2;
        r.d00 = -cp * cx.s2x * ry.s2x;
        r.d01 = -2.f * cp * cx.s2 * ry.c2x;
        r.d10 = 2.f * cp * cx.c2x * ry.s2;
        r.d11 = -r.d00;
        return r;
    }
    return vel2d<VK>(vp, sc, 0, x, y);
}

// One node update: returns phi+, psi_x+, psi_y+.
template <int TR, int VK, int CR>
__device__ __forceinline__ void node2d(const float *__restrict__ in, const Geom &g,
                                       const VelParams &vp, const StageCoef &sc, float dt, int i,
                                       int j, float x, float y, const Sep &cx, const Sep &ry,
                                       float &phi, float &px, float &py)
{
    float dx, dy, J[4];
    trace2d_from<TR, VK>(stage1<VK>(vp, sc, x, y, cx, ry), vp, sc, x, y, dt, dx, dy, J);

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
    phi = H;
    px = fmaf(J[0], Hx, J[2] * Hy);  // (J^T grad H)_x
    py = fmaf(J[1], Hx, J[3] * Hy);  // (J^T grad H)_y
}

template <int TR, int VK, int CR, int WC>
__global__ void __launch_bounds__(TX)
k_step2d(const float *__restrict__ in, float *__restrict__ out, Geom g, VelParams vp,
         const StageCoef *__restrict__ coef, float dt)
{
    __shared__ float psy[WC ? TY : 1][TX + 3];  // psi_y+ of columns x0-2 .. x0+TX
    __shared__ StageCoef sc_s;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

    // the step's stage coefficients (FOURIER2D reads its 4x4 tables from shared memory)
    const StageCoef *scp = coef;
    if (VK == VK_FOURIER2D) {
        const float *src = reinterpret_cast<const float *>(coef);
        float *dst = reinterpret_cast<float *>(&sc_s);
        for (int e = tid; e < (int)(sizeof(StageCoef) / 4); e += TX) dst[e] = __ldg(src + e);
        __syncthreads();
        scp = &sc_s;
    }
    const StageCoef &sc = *scp;

    const int i = x0 + tid;
    const int rows = min(TY, g.n1 - y0);
    const float x = g.lo0 + (float)i * g.h0;
    const Sep cx = (VK == VK_VORTEX2D) ? sep_factors(x) : Sep{0.f, 0.f, 0.f};

    if (i < g.n0) {
#pragma unroll 2
        for (int r = 0; r < rows; ++r) {
            const int j = y0 + r;
            const float y = g.lo1 + (float)j * g.h1;
            const Sep ry = (VK == VK_VORTEX2D) ? sep_factors(y) : Sep{0.f, 0.f, 0.f};
            float phi, px, py;
            node2d<TR, VK, CR>(in, g, vp, sc, dt, i, j, x, y, cx, ry, phi, px, py);
            const int o = j * g.pitch + i;
            out[o] = phi;
            out[g.plane + o] = px;
            out[2 * g.plane + o] = py;
            if (WC) psy[WC ? r : 0][tid + 2] = py;
        }
    }
    if (WC) {
        // halo columns of psi_y+: x0-1 and x0+TX (x0-2 too when the tile is one column
        // wide, for the one-sided stencil of the last node)
        const int width = min(TX, g.n0 - x0);
        for (int hh = tid; hh < 3 * rows; hh += TX) {
            const int r = hh / 3, which = hh % 3;
            const int ih = which == 0 ? x0 - 2 : (which == 1 ? x0 - 1 : x0 + TX);
            const bool need = which == 0 ? (width == 1 && ih >= 0) : (ih >= 0 && ih < g.n0);
            if (!need) continue;
            const int j = y0 + r;
            const float xh = g.lo0 + (float)ih * g.h0;
            const float y = g.lo1 + (float)j * g.h1;
            const Sep cxh = (VK == VK_VORTEX2D) ? sep_factors(xh) : Sep{0.f, 0.f, 0.f};
            const Sep ry = (VK == VK_VORTEX2D) ? sep_factors(y) : Sep{0.f, 0.f, 0.f};
            float phi, px, py;
            node2d<TR, VK, CR>(in, g, vp, sc, dt, ih, j, xh, y, cxh, ry, phi, px, py);
            psy[WC ? r : 0][ih - x0 + 2] = py;
        }
        __syncthreads();
        if (i < g.n0) {
            for (int r = 0; r < rows; ++r) {
                const float *line = psy[WC ? r : 0];
                const float v = dline(i, g.n0, g.i2h0, [&](int q) { return line[q - x0 + 2]; });
                out[3 * g.plane + (y0 + r) * g.pitch + i] = v;
            }
        }
    }
}

// phi_xy = d/dx psi_y at every node (approach A with one-sided ends); used after
// set_state and for the COMPACT layout's read-out.
__global__ void __launch_bounds__(256) k_recon2d(float *__restrict__ buf, Geom g)
{
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    if (i >= g.n0 || j >= g.n1) return;
    const float *py = buf + 2 * g.plane + (size_t)j * g.pitch;
    float v = dline(i, g.n0, g.i2h0, [&](int q) { return py[q]; });
    buf[3 * g.plane + (size_t)j * g.pitch + i] = v;
}

template <int TR, int VK, int CR, int WC>
cudaError_t launch_t(const StepLaunch &a, cudaStream_t s)
{
    dim3 grid((a.geom.n0 + TX - 1) / TX, (a.geom.n1 + TY - 1) / TY);
    k_step2d<TR, VK, CR, WC><<<grid, TX, 0, s>>>(a.in, a.out, a.geom, a.vp, a.coef, (float)a.dt);
    return cudaGetLastError();
}

template <int TR, int VK>
cudaError_t launch_cr(const StepLaunch &a, cudaStream_t s)
{
    if (a.write_cross)
        return a.cross_in == CROSS_PLANE ? launch_t<TR, VK, CROSS_PLANE, 1>(a, s)
                                         : launch_t<TR, VK, CROSS_RECON, 1>(a, s);
    return a.cross_in == CROSS_PLANE ? launch_t<TR, VK, CROSS_PLANE, 0>(a, s)
                                     : launch_t<TR, VK, CROSS_RECON, 0>(a, s);
}

template <int VK>
cudaError_t launch_tr(const StepLaunch &a, cudaStream_t s)
{
    return a.trace == TR_EULER ? launch_cr<TR_EULER, VK>(a, s) : launch_cr<TR_RK3, VK>(a, s);
}

}  // namespace

cudaError_t launch_step2d(const StepLaunch &a, cudaStream_t s)
{
    switch (a.vp.kind) {
    case VK_CONST: return launch_tr<VK_CONST>(a, s);
    case VK_ROTATION: return launch_tr<VK_ROTATION>(a, s);
    case VK_VORTEX2D: return launch_tr<VK_VORTEX2D>(a, s);
    case VK_PSEUDO1D: return launch_tr<VK_PSEUDO1D>(a, s);
    case VK_FOURIER2D: return launch_tr<VK_FOURIER2D>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_recon2d(const Geom &g, float *buf, cudaStream_t s)
{
    dim3 block(32, 8);
    dim3 grid((g.n0 + 31) / 32, (g.n1 + 7) / 8);
    k_recon2d<<<grid, block, 0, s>>>(buf, g);
    return cudaGetLastError();
}

}  // namespace gals
