// curvature.cu -- value, unit normal and curvature of the Hermite interpolant at arbitrary
// points (Sec. 3.4, "Approximation of derivative quantities": all first and second
// derivatives inside a cell by differentiating the p-cubic interpolant; eq.
// surface_normal, eq. curvature).
//
// One thread per point.  The point's cell is located from its FP64 position (a 4096^2 grid
// needs more than FP32 to place a point within a cell), the cell's 4^p data are gathered
// from the state planes (mixed derivatives from the planes, approach A, or per cell,
// approach B), and the interpolant is reduced axis by axis: along x each edge of the cell
// gives its value, first and second x-derivative, along y (and z) those combine into every
// derivative of total order <= 2.  phi is shifted by its value at the cell's first corner,
// as in the step kernels, so the derivatives, whose weights scale as 1/h and 1/h^2, carry
// no rounding of the O(1) values themselves.
#include "gals_internal.h"

namespace gals {

namespace {

constexpr int kPtThreads = 256;

// Weights of the four end data (p0, p1, s0, s1) of one cell edge for the d-th derivative
// along it, d = 0, 1, 2, at relative coordinate xi (cell length h):
//   H = p0 f(xi) + p1 f(1-xi) + h s0 g(xi) - h s1 g(1-xi),
//   f(x) = 1 - 3x^2 + 2x^3, g(x) = x (1-x)^2 (eq. 1-cubic_basis_functions).
struct EdgeW { float w[3][4]; };

__device__ __forceinline__ EdgeW edge_weights(float xi, float h, float ih)
{
    const float om = 1.f - xi;
    const float f0 = 1.f - xi * xi * (3.f - 2.f * xi), f1 = 1.f - om * om * (3.f - 2.f * om);
    const float g0 = xi * om * om, g1 = om * xi * xi;
    const float fd0 = 6.f * xi * (xi - 1.f);            // f'(xi); f'(1-xi) is the same value
    const float gd0 = 1.f - xi * (4.f - 3.f * xi);      // g'(xi)
    const float gd1 = 1.f - om * (4.f - 3.f * om);      // g'(1-xi)
    EdgeW e;
    e.w[0][0] = f0;            e.w[0][1] = f1;            e.w[0][2] = h * g0;   e.w[0][3] = -h * g1;
    e.w[1][0] = fd0 * ih;      e.w[1][1] = -fd0 * ih;     e.w[1][2] = gd0;      e.w[1][3] = gd1;
    const float fdd0 = 12.f * xi - 6.f, fdd1 = 12.f * om - 6.f;   // f''(xi), f''(1-xi)
    const float gdd0 = 6.f * xi - 4.f, gdd1 = 6.f * om - 4.f;     // g''(xi), g''(1-xi)
    e.w[2][0] = fdd0 * ih * ih; e.w[2][1] = fdd1 * ih * ih; e.w[2][2] = gdd0 * ih; e.w[2][3] = -gdd1 * ih;
    return e;
}

// plane of derivative multi-index a (bit i = d/dx_i) in the state's plane order
__device__ __forceinline__ int plane_of3(int a)
{
    // 0 phi, 1 x, 2 y, 3 xy -> plane 4, 4 z -> plane 3, 5 xz, 6 yz, 7 xyz
    return a == 3 ? 4 : (a == 4 ? 3 : a);
}

// Locate one coordinate: clamp into the box, cell index clamped to [0, n-2], xi in [0, 1].
__device__ __forceinline__ void locate_point(double x, double lo, double h, int n, int &c, float &xi)
{
    const double hi = lo + (double)(n - 1) * h;
    x = fmin(fmax(x, lo), hi);
    const double r = (x - lo) / h;
    int k = (int)floor(r);
    k = min(max(k, 0), n - 2);
    c = k;
    xi = (float)(r - (double)k);
}

__device__ __forceinline__ void normal_curvature(int dim, float H, const float g[3], const float hs[3][3],
                                                 int64_t p, float *oH, float *on, float *ok)
{
    float g2 = 0.f;
    for (int d = 0; d < dim; ++d) g2 = fmaf(g[d], g[d], g2);
    const float gn = sqrtf(g2);
    if (oH) oH[p] = H;
    if (on)
        for (int d = 0; d < dim; ++d) on[p * dim + d] = gn > 0.f ? g[d] / gn : 0.f;
    if (!ok) return;
    if (!(gn > 0.f)) {
        ok[p] = 0.f;
        return;
    }
    float num;
    if (dim == 2) {  // eq. curvature
        num = hs[0][0] * g[1] * g[1] - 2.f * g[0] * g[1] * hs[0][1] + hs[1][1] * g[0] * g[0];
    } else {         // div(grad H / |grad H|)
        float tr = 0.f, ghg = 0.f;
        for (int j = 0; j < 3; ++j) {
            tr += hs[j][j];
            for (int k = 0; k < 3; ++k) ghg = fmaf(g[j] * hs[j][k], g[k], ghg);
        }
        num = g2 * tr - ghg;
    }
    ok[p] = num / (g2 * gn);
}

// 2D: c[v][a], corner v = vx + 2 vy, a = derivative multi-index (0 phi, 1 x, 2 y, 3 xy)
__global__ void __launch_bounds__(kPtThreads)
k_points2d(const float *__restrict__ s, Geom g, double lo0, double lo1, double h0, double h1,
           const double *__restrict__ pts, int64_t npts, int cell_b, float *oH, float *on, float *ok)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts;
         p += (int64_t)gridDim.x * blockDim.x) {
        int k, l;
        float xi, eta;
        locate_point(pts[2 * p], lo0, h0, g.n0, k, xi);
        locate_point(pts[2 * p + 1], lo1, h1, g.n1, l, eta);
        float c[4][4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t id = (int64_t)(l + (v >> 1)) * g.pitch + k + (v & 1);
#pragma unroll
            for (int a = 0; a < 4; ++a) c[v][a] = s[a * g.plane + id];
        }
        if (cell_b) cross_cell2d(c, g.ih0, g.ih1);
        const float base = c[0][0];
        const EdgeW wx = edge_weights(xi, g.h0, g.ih0), wy = edge_weights(eta, g.h1, g.ih1);
        // along x: row B, y-type t (0: phi with phi_x, 1: phi_y with phi_xy), order d
        float X[2][2][3];
#pragma unroll
        for (int B = 0; B < 2; ++B)
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int v0 = 2 * B, v1 = 2 * B + 1, a = 2 * t;
                // phi shifted by the first corner's value (exactly 0 there)
                const float p0 = t == 0 ? (v0 == 0 ? 0.f : c[v0][0] - base) : c[v0][a];
                const float p1 = t == 0 ? c[v1][0] - base : c[v1][a];
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    X[B][t][d] = fmaf(wx.w[d][0], p0, fmaf(wx.w[d][1], p1,
                                      fmaf(wx.w[d][2], c[v0][a + 1], wx.w[d][3] * c[v1][a + 1])));
            }
        // along y: order e; data of edge B are (value type t = 0, slope type t = 1)
        auto Y = [&](int d, int e) {
            return fmaf(wy.w[e][0], X[0][0][d], fmaf(wy.w[e][1], X[1][0][d],
                        fmaf(wy.w[e][2], X[0][1][d], wy.w[e][3] * X[1][1][d])));
        };
        const float gr[3] = {Y(1, 0), Y(0, 1), 0.f};
        const float hxy = Y(1, 1);
        const float hs[3][3] = {{Y(2, 0), hxy, 0.f}, {hxy, Y(0, 2), 0.f}, {0.f, 0.f, 0.f}};
        normal_curvature(2, base + Y(0, 0), gr, hs, p, oH, on, ok);
    }
}

// 3D: c[v][a], corner v = vx + 2 vy + 4 vz, a = derivative multi-index (bit i = d/dx_i)
__global__ void __launch_bounds__(kPtThreads)
k_points3d(const float *__restrict__ s, Geom g, double lo0, double lo1, double lo2, double h0,
           double h1, double h2, const double *__restrict__ pts, int64_t npts, int cell_b,
           float *oH, float *on, float *ok)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts;
         p += (int64_t)gridDim.x * blockDim.x) {
        int k, l, m;
        float xi, eta, zeta;
        locate_point(pts[3 * p], lo0, h0, g.n0, k, xi);
        locate_point(pts[3 * p + 1], lo1, h1, g.n1, l, eta);
        locate_point(pts[3 * p + 2], lo2, h2, g.n2, m, zeta);
        float c[8][8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int64_t id = ((int64_t)(m + (v >> 2)) * g.n1 + l + ((v >> 1) & 1)) * g.pitch + k + (v & 1);
#pragma unroll
            for (int a = 0; a < 8; ++a) c[v][a] = s[plane_of3(a) * g.plane + id];
        }
        if (cell_b) {
            // approach B: mixed derivatives of each vertex from the cell's gradients
            float cr[8][4];
            cross_cell3d([&](int v, int q) { return c[v][q == 0 ? 0 : (q == 1 ? 1 : (q == 2 ? 2 : 4))]; },
                         g.ih0, g.ih1, g.ih2, cr);
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                c[v][3] = cr[v][0];  // xy
                c[v][5] = cr[v][1];  // xz
                c[v][6] = cr[v][2];  // yz
                c[v][7] = cr[v][3];  // xyz
            }
        }
        const float base = c[0][0];
        const EdgeW wx = edge_weights(xi, g.h0, g.ih0), wy = edge_weights(eta, g.h1, g.ih1),
                    wz = edge_weights(zeta, g.h2, g.ih2);
        // along x: edge (B, C), yz-type t (bit 0: d/dy, bit 1: d/dz of the data), order d
        float X[2][2][4][3];
#pragma unroll
        for (int C = 0; C < 2; ++C)
#pragma unroll
            for (int B = 0; B < 2; ++B)
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int v0 = 2 * B + 4 * C, v1 = v0 + 1, a = ((t & 1) << 1) | ((t >> 1) << 2);
                    const float p0 = t == 0 ? (v0 == 0 ? 0.f : c[v0][0] - base) : c[v0][a];
                    const float p1 = t == 0 ? c[v1][0] - base : c[v1][a];
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        X[C][B][t][d] = fmaf(wx.w[d][0], p0, fmaf(wx.w[d][1], p1,
                                             fmaf(wx.w[d][2], c[v0][a + 1], wx.w[d][3] * c[v1][a + 1])));
                }
        // along y: face C, z-type u (0: the data's value in z, 1: its z-slope), orders d, e
        auto Yr = [&](int C, int u, int d, int e) {
            return fmaf(wy.w[e][0], X[C][0][2 * u][d], fmaf(wy.w[e][1], X[C][1][2 * u][d],
                        fmaf(wy.w[e][2], X[C][0][2 * u + 1][d], wy.w[e][3] * X[C][1][2 * u + 1][d])));
        };
        // along z: orders d, e, f
        auto Zr = [&](int d, int e, int f) {
            return fmaf(wz.w[f][0], Yr(0, 0, d, e), fmaf(wz.w[f][1], Yr(1, 0, d, e),
                        fmaf(wz.w[f][2], Yr(0, 1, d, e), wz.w[f][3] * Yr(1, 1, d, e))));
        };
        const float gr[3] = {Zr(1, 0, 0), Zr(0, 1, 0), Zr(0, 0, 1)};
        const float hxy = Zr(1, 1, 0), hxz = Zr(1, 0, 1), hyz = Zr(0, 1, 1);
        const float hs[3][3] = {{Zr(2, 0, 0), hxy, hxz}, {hxy, Zr(0, 2, 0), hyz}, {hxz, hyz, Zr(0, 0, 2)}};
        normal_curvature(3, base + Zr(0, 0, 0), gr, hs, p, oH, on, ok);
    }
}

}  // namespace

cudaError_t launch_eval_points(int dim, const Geom &g, const double lo[3], const double h[3],
                               const float *state, const double *pts, int64_t npts, bool cell_b,
                               float *H, float *normal, float *kappa, cudaStream_t s)
{
    if (npts <= 0) return cudaSuccess;
    const int64_t want = (npts + kPtThreads - 1) / kPtThreads;
    const int blocks = (int)(want < 65536 ? want : 65536);
    if (dim == 2)
        k_points2d<<<blocks, kPtThreads, 0, s>>>(state, g, lo[0], lo[1], h[0], h[1], pts, npts,
                                                 cell_b ? 1 : 0, H, normal, kappa);
    else
        k_points3d<<<blocks, kPtThreads, 0, s>>>(state, g, lo[0], lo[1], lo[2], h[0], h[1], h[2],
                                                 pts, npts, cell_b ? 1 : 0, H, normal, kappa);
    return cudaGetLastError();
}

}  // namespace gals
