// gals_device.cuh -- device-side building blocks of the GALS step (FP32).
//
// The per-node update follows the superconsistent gradient-augmented CIR scheme of
// Nave, Rosales and Seibold (arXiv 0905.3409):
//   * analytic velocity v and Jacobian Dv (Sec. 4 assumes both are known exactly),
//   * backward trace with the Jacobian of the approximate backward map
//     (Sec. 5.1, Ex. "superconsistent forward Euler" and "superconsistent Shu-Osher"),
//   * cell location of the foot point and the p-cubic Hermite interpolant
//     (Sec. 2.3, eq. 1-cubic_basis_functions and eq. p-cubic_interpolant),
//   * phi+ = H(foot), psi+ = J^T grad H(foot)  (eq. superconsistency),
//   * mixed derivatives from central differences of the gradient (Sec. 2.3, approach A).
//
// FP32 design notes (they keep the result within ~1e-7 relative of an exact evaluation):
//   * the trace carries the foot displacement delta = foot - x (small) instead of the
//     absolute foot, and the cell index is node index + floor(delta/h), so xi keeps
//     full precision even on 4096^2 grids;
//   * the Hermite evaluation subtracts the base corner's phi from all corner values
//     first (the interpolant reproduces constants exactly), so the value terms are O(h)
//     and their derivatives divided by h lose no digits to cancellation;
//   * the interpolant is sum-factorised along x, then y (then z); the sum is the same
//     polynomial as the direct 4^p-term form of the paper.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gals {

constexpr int kMaxModes = 64;
constexpr float kPi = 3.14159265358979323846f;

enum VelKind { VK_CONST = 0, VK_ROTATION = 1, VK_VORTEX2D = 2, VK_DEFORM3D = 3,
               VK_PSEUDO1D = 4, VK_FOURIER2D = 5, VK_WAVES2D = 6 };
// GIVEN: precomputed (surrogate); HEUN: RK3 foot, gradients by Heun's method along the
// characteristic (Sec. 4, CIR form)
enum TraceKind { TR_EULER = 0, TR_RK3 = 1, TR_GIVEN = 2, TR_HEUN = 3 };
// Where a cell's mixed derivatives come from: the stored planes (approach A, FULL), the
// psi windows around the cell (approach A, COMPACT), or the cell's own gradients
// (approach B of Sec. 2.3).
enum CrossSrc { CROSS_PLANE = 0, CROSS_RECON = 1, CROSS_CELL = 2 };

// Velocity descriptor as passed to kernels (by value).
struct VelParams {
    int kind;
    float omega, cx, cy, cz;
    float c0, c1, c2;
    float d0, d1;               // PSEUDO1D direction (unit vector)
    double invT;                // 1/T of the cos(pi t/T) modulation
    int nmodes;
    float mode_a[kMaxModes];
    int mode_kl[kMaxModes];     // k | (l << 8), k, l in 1..4
    double mode_n[kMaxModes];   // temporal frequency n (cycles per unit time)
    double mode_chi[kMaxModes]; // phase / (2 pi)
    const float *given;         // TR_GIVEN: planes dx, dy, J00, J01, J10, J11 of the step
    int64_t given_plane;        //   (grid pitch layout) and their plane stride
    // WAVES2D: device table of nwaves modes (see WaveTab) and the call's amplitude table
    // (per step, per stage, per mode: a cos(2 pi n t_s + chi)), owned by the grid / surrogate
    int nwaves;
    const float4 *waves;
    const double *waves_d;
    float *wamp;
};

// WAVES2D device table of M modes: geo[m] = (kx, ky, phase, kx ky), sq[m] = (kx^2, ky^2, 0, 0),
// tim[m] = (a, n, chi / (2 pi), 0) in FP32 at waves[0..3M), and (a, n, chi / (2 pi)) per
// mode in FP64 at waves_d[0..3M).
struct WaveTab {
    const float4 *geo, *sq, *tim;
};
__host__ __device__ __forceinline__ WaveTab wave_tab(const float4 *w, int M)
{
    return WaveTab{w, w + M, w + 2 * M};
}

// Grid geometry for kernels.
struct Geom {
    int n0, n1, n2;
    int pitch;                  // row pitch in floats (multiple of 4)
    int64_t plane;              // plane stride in floats
    float h0, h1, h2;
    float ih0, ih1, ih2;        // 1/h
    float i2h0, i2h1, i2h2;     // 1/(2h)
    float lo0, lo1, lo2;
#ifdef GALS_CHECKED
    int *chk = nullptr;         // device error word of the checked build (see GALS_CHK)
    // test hook of the checked build (gals_checked_wait_test): polls of a staged-tile
    // wait before it counts as lost, and whether the copy that completes it is issued
    uint32_t wait_polls = 1u << 24;
    int skip_copy = 0;
#endif
};

// Checked build (-DGALS_CHECKED, libgals_checked.so): GALS_CHK(g, i, n) tests a
// data-dependent index of the step kernels (staged-tile and global gathers, stores) against
// its buffer [0, n).  The first violation is recorded in *g.chk as kErrBounds with the
// source line above the low byte, and the access is redirected to element 0, so a checked
// run never leaves its buffers.  Without the flag the macro is the index itself and Geom
// has no chk field, so the normal build's kernels are unchanged.
constexpr int kErrBounds = 2;

__device__ __forceinline__ int64_t checked_index(int *word, int64_t i, int64_t n, int line)
{
    if (i >= 0 && i < n) return i;
    if (word) atomicCAS(word, 0, kErrBounds | (line << 8));
    return 0;
}

#ifdef GALS_CHECKED
#define GALS_CHK(g, i, n) \
    ((decltype((i) + 0))::gals::checked_index((g).chk, (int64_t)(i), (int64_t)(n), __LINE__))
#else
#define GALS_CHK(g, i, n) (i)
#endif

// Nodes of one plane in row-major order (rows of `pitch` floats): every node index of a
// plane lies below this.
__device__ __forceinline__ int64_t plane_extent(const Geom &g)
{
    return (int64_t)g.n2 * g.n1 * g.pitch;
}

// Time-dependent scalars of the three RK3 stage times (t+dt, t, t+dt/2) of one step.
// A table of these (one entry per step of a gals_step call) is filled once per call by
// k_coef_table from the device clock, so the step kernels do no FP64 work.  FOURIER2D
// folds the modes into 4x4 tables A_kl(t) = sum_{m: k_m = k, l_m = l} a_m
// cos(2 pi n_m t + chi_m), pre-scaled.
struct StageCoef {
    float mod[3];               // cos(pi t_s / T)
    float pad;
    const float *wamp;          // WAVES2D: this step's amplitudes [stage][mode]
    float A[3][16];             // A_kl
    float Al[3][16];            // A_kl * l pi
    float All[3][16];           // A_kl * (l pi)^2
};

// ---------------------------------------------------------------- stage coefficients

__device__ inline void stage_coef_one(const VelParams &vp, double t, double dt, StageCoef &sc)
{
    for (int s = 0; s < 3; ++s) {
        const double ts = s == 0 ? t + dt : (s == 1 ? t : t + 0.5 * dt);
        // cos(pi t/T): reduce the phase t/T modulo 2 in FP64, then evaluate in FP64
        double ph = ts * vp.invT;
        ph = ph - 2.0 * floor(0.5 * ph);
        sc.mod[s] = (float)cospi(ph);
    }
    sc.pad = 0.f;
    sc.wamp = nullptr;
    if (vp.kind != VK_FOURIER2D) return;
    // each mode once, added to its (k, l) entry: every entry sums its modes in index order
    double acc[3][16];
    for (int s = 0; s < 3; ++s)
        for (int kl = 0; kl < 16; ++kl) acc[s][kl] = 0.0;
    for (int m = 0; m < vp.nmodes; ++m) {
        const int code = vp.mode_kl[m], k = code & 0xff, l = code >> 8;
        if (k < 1 || k > 4 || l < 1 || l > 4) continue;
        const int kl = (k - 1) * 4 + (l - 1);
        const double a = (double)vp.mode_a[m], n = vp.mode_n[m], chi = vp.mode_chi[m];
        for (int s = 0; s < 3; ++s) {
            const double ts = s == 0 ? t + dt : (s == 1 ? t : t + 0.5 * dt);
            double ph = 2.0 * (n * ts + chi);  // in units of pi
            ph = ph - 2.0 * floor(0.5 * ph);
            acc[s][kl] += a * cospi(ph);
        }
    }
    for (int s = 0; s < 3; ++s)
        for (int kl = 0; kl < 16; ++kl) {
            const float a = (float)acc[s][kl], lp = (float)(kl % 4 + 1) * kPi;
            sc.A[s][kl] = a;
            sc.Al[s][kl] = a * lp;
            sc.All[s][kl] = a * lp * lp;
        }
}

// ---------------------------------------------------------------- velocity fields

struct V2 { float u, v, d00, d01, d10, d11; };          // Dv[i][j] = dv_i/dx_j

__device__ __forceinline__ void sincospi_f(float x, float *s, float *c)
{
    __sincosf(x * kPi, s, c);
}

// sin a and cos a for a = 2 pi (s - 1/2) = 2 pi s - pi, one rounding: for s in [0, 1] the
// angle stays in [-pi, pi], where the hardware approximation is most accurate.  Then
// sin a = -sin(2 pi s), cos a = -cos(2 pi s) and sin^2(pi s) = (1 + cos a) / 2; the
// separable fields (single vortex, deformation) are written in these factors.
__device__ __forceinline__ void sincos_turn(float s, float *sn, float *cs)
{
    __sincosf(__fmaf_rn(s, 2.f * kPi, -kPi), sn, cs);
}

template <int VK>
__device__ __forceinline__ V2 vel2d(const VelParams &vp, const StageCoef &sc, int stage,
                                    float x, float y)
{
    V2 r;
    if (VK == VK_CONST) {
        r.u = vp.c0; r.v = vp.c1; r.d00 = r.d01 = r.d10 = r.d11 = 0.f;
    } else if (VK == VK_ROTATION) {
        r.u = -vp.omega * (y - vp.cy);
        r.v = vp.omega * (x - vp.cx);
        r.d00 = 0.f; r.d01 = -vp.omega; r.d10 = vp.omega; r.d11 = 0.f;
    } else if (VK == VK_VORTEX2D) {
        // u = -c sin^2(pi x) sin(2 pi y), v = c sin(2 pi x) sin^2(pi y), in the factors
        // A = sin a, B = cos a of sincos_turn
        float Ax, Bx, Ay, By;
        sincos_turn(x, &Ax, &Bx);
        sincos_turn(y, &Ay, &By);
        const float c = sc.mod[stage], h = 0.5f * c;
        const float cSx = __fmaf_rn(Bx, h, h), mcSy = __fmaf_rn(By, -h, -h);
        r.u = cSx * Ay;
        r.v = Ax * mcSy;
        r.d00 = -(c * kPi) * (Ax * Ay);
        r.d01 = (2.f * kPi) * (cSx * By);
        r.d10 = (2.f * kPi) * (Bx * mcSy);
        r.d11 = -r.d00;
    } else if (VK == VK_PSEUDO1D) {
        float e = __expf(vp.d0 * x + vp.d1 * y);
        r.u = e * vp.d0; r.v = e * vp.d1;
        r.d00 = e * vp.d0 * vp.d0; r.d01 = e * vp.d0 * vp.d1;
        r.d10 = r.d01; r.d11 = e * vp.d1 * vp.d1;
    } else if (VK == VK_WAVES2D) {
        // Psi = sum C_m sin(theta_m), theta_m = kx x + ky y + phase, C_m the stage amplitude
        const WaveTab T = wave_tab(vp.waves, vp.nwaves);
        const float *amp = sc.wamp + stage * vp.nwaves;
        float u = 0.f, v = 0.f, d00 = 0.f, d01 = 0.f, d10 = 0.f;
#pragma unroll 4
        for (int m = 0; m < vp.nwaves; ++m) {
            const float4 g = __ldg(T.geo + m), q = __ldg(T.sq + m);
            const float C = __ldg(amp + m);
            float sn, cs;
            __sincosf(__fmaf_rn(g.x, x, __fmaf_rn(g.y, y, g.z)), &sn, &cs);
            const float cc = C * cs, cn = C * sn;
            u = __fmaf_rn(-g.y, cc, u);
            v = __fmaf_rn(g.x, cc, v);
            d00 = __fmaf_rn(g.w, cn, d00);
            d01 = __fmaf_rn(q.y, cn, d01);
            d10 = __fmaf_rn(-q.x, cn, d10);
        }
        r.u = u; r.v = v; r.d00 = d00; r.d01 = d01; r.d10 = d10; r.d11 = -d00;
    } else {  // VK_FOURIER2D
        float s[5], c[5], sy_[5], cy_[5];
        sincospi_f(x, &s[1], &c[1]);
        sincospi_f(y, &sy_[1], &cy_[1]);
        // multiple angles by the Chebyshev recurrences
        s[2] = 2.f * s[1] * c[1];            c[2] = 1.f - 2.f * s[1] * s[1];
        s[3] = s[2] * c[1] + c[2] * s[1];    c[3] = c[2] * c[1] - s[2] * s[1];
        s[4] = 2.f * s[2] * c[2];            c[4] = 1.f - 2.f * s[2] * s[2];
        sy_[2] = 2.f * sy_[1] * cy_[1];          cy_[2] = 1.f - 2.f * sy_[1] * sy_[1];
        sy_[3] = sy_[2] * cy_[1] + cy_[2] * sy_[1]; cy_[3] = cy_[2] * cy_[1] - sy_[2] * sy_[1];
        sy_[4] = 2.f * sy_[2] * cy_[2];          cy_[4] = 1.f - 2.f * sy_[2] * sy_[2];
        // Psi = sum A_kl s_k(x) s_l(y); u = -Psi_y, v = Psi_x
        float u = 0.f, v = 0.f, d00 = 0.f, d01 = 0.f, d10 = 0.f;
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            float Ux = 0.f, Vx = 0.f, W = 0.f;
#pragma unroll
            for (int l = 1; l <= 4; ++l) {
                int kl = (k - 1) * 4 + (l - 1);
                Ux = fmaf(sc.Al[stage][kl], cy_[l], Ux);   // sum_l A l pi c_l(y)
                Vx = fmaf(sc.A[stage][kl], sy_[l], Vx);    // sum_l A s_l(y)
                W = fmaf(sc.All[stage][kl], sy_[l], W);    // sum_l A (l pi)^2 s_l(y)
            }
            float kp = (float)k * kPi;
            u = fmaf(-s[k], Ux, u);
            v = fmaf(kp * c[k], Vx, v);
            d00 = fmaf(-kp * c[k], Ux, d00);
            d01 = fmaf(s[k], W, d01);
            d10 = fmaf(-kp * kp * s[k], Vx, d10);
        }
        r.u = u; r.v = v; r.d00 = d00; r.d01 = d01; r.d10 = d10; r.d11 = -d00;
    }
    return r;
}

// ---------------------------------------------------------------- backward traces

// 2D trace from node position (x, y) at t+dt back to t: displacement (dx, dy) of the
// foot and J[i][j] = d foot_i / d x_j (row-major J00, J01, J10, J11).
// The superconsistent trace with the velocity evaluated by vel(stage, x, y) -> V2 (stage 1
// at time t, stage 2 at t + dt/2); a = v(x, t+dt) and its Jacobian from the caller.
template <int TR, class Vel>
__device__ __forceinline__ void trace2d_eval(const V2 &a, Vel vel, float x, float y, float dt,
                                             float &dx, float &dy, float J[4])
{
    // a = v(x, t+dt) and its Jacobian, supplied by the caller
    if (TR == TR_EULER) {
        dx = -dt * a.u; dy = -dt * a.v;
        J[0] = 1.f - dt * a.d00; J[1] = -dt * a.d01;
        J[2] = -dt * a.d10;      J[3] = 1.f - dt * a.d11;
        return;
    }
    // stage 1: x1 = x - dt v(x, t+dt), J1 = I - dt Dv(x, t+dt)
    float J1_00 = 1.f - dt * a.d00, J1_01 = -dt * a.d01;
    float J1_10 = -dt * a.d10, J1_11 = 1.f - dt * a.d11;
    V2 b = vel(1, x - dt * a.u, y - dt * a.v);  // v(x1, t)
    // M = Dv(x1, t) J1
    float M00 = b.d00 * J1_00 + b.d01 * J1_10, M01 = b.d00 * J1_01 + b.d01 * J1_11;
    float M10 = b.d10 * J1_00 + b.d11 * J1_10, M11 = b.d10 * J1_01 + b.d11 * J1_11;
    // stage 2: x2 = x - dt (v1 + v2)/4, J2 = I - dt (Dv1 + Dv2 J1)/4
    float q = 0.25f * dt;
    float J2_00 = 1.f - q * (a.d00 + M00), J2_01 = -q * (a.d01 + M01);
    float J2_10 = -q * (a.d10 + M10), J2_11 = 1.f - q * (a.d11 + M11);
    V2 c = vel(2, x - q * (a.u + b.u), y - q * (a.v + b.v));  // v(x2, t+dt/2)
    float N00 = c.d00 * J2_00 + c.d01 * J2_10, N01 = c.d00 * J2_01 + c.d01 * J2_11;
    float N10 = c.d10 * J2_00 + c.d11 * J2_10, N11 = c.d10 * J2_01 + c.d11 * J2_11;
    // stage 3: foot = x - dt (v1/6 + v2/6 + 2 v3/3), written as w3 + (w1 + w2 - 2 w3)/6,
    // exact for constant v; J = I - dt (Dv1 + Dv2 J1)/6 - 2 dt Dv3 J2 / 3 (= I when Dv = 0)
    const float i6 = 1.f / 6.f, m6 = -dt / 6.f, m23 = -2.f * dt / 3.f;
    dx = -dt * fmaf(a.u + b.u - 2.f * c.u, i6, c.u);
    dy = -dt * fmaf(a.v + b.v - 2.f * c.v, i6, c.v);
    J[0] = fmaf(m6, a.d00 + M00, fmaf(m23, N00, 1.f));
    J[1] = fmaf(m6, a.d01 + M01, m23 * N01);
    J[2] = fmaf(m6, a.d10 + M10, m23 * N10);
    J[3] = fmaf(m6, a.d11 + M11, fmaf(m23, N11, 1.f));
}


template <int TR, int VK>
__device__ __forceinline__ void trace2d_from(const V2 &a, const VelParams &vp, const StageCoef &sc,
                                             float x, float y, float dt, float &dx, float &dy,
                                             float J[4])
{
    trace2d_eval<TR>(a, [&](int stage, float px, float py) { return vel2d<VK>(vp, sc, stage, px, py); },
                     x, y, dt, dx, dy, J);
}

template <int TR, int VK>
__device__ __forceinline__ void trace2d(const VelParams &vp, const StageCoef &sc, float x,
                                        float y, float dt, float &dx, float &dy, float J[4])
{
    trace2d_from<TR, VK>(vel2d<VK>(vp, sc, 0, x, y), vp, sc, x, y, dt, dx, dy, J);
}

// WAVES2D velocity at one point evaluated by a whole warp (every lane passes the same
// point): lane l sums modes l, l + 32, ..., then a butterfly reduction gives every lane the
// totals.  The sums run in another order than vel2d's, so the last bits may differ.
__device__ __forceinline__ V2 vel2d_waves_warp(const VelParams &vp, const StageCoef &sc, int stage,
                                               float x, float y)
{
    const WaveTab T = wave_tab(vp.waves, vp.nwaves);
    const float *amp = sc.wamp + stage * vp.nwaves;
    float u = 0.f, v = 0.f, d00 = 0.f, d01 = 0.f, d10 = 0.f;
    for (int m = threadIdx.x & 31; m < vp.nwaves; m += 32) {
        const float4 g = __ldg(T.geo + m), q = __ldg(T.sq + m);
        const float C = __ldg(amp + m);
        float sn, cs;
        __sincosf(__fmaf_rn(g.x, x, __fmaf_rn(g.y, y, g.z)), &sn, &cs);
        const float cc = C * cs, cn = C * sn;
        u = __fmaf_rn(-g.y, cc, u);
        v = __fmaf_rn(g.x, cc, v);
        d00 = __fmaf_rn(g.w, cn, d00);
        d01 = __fmaf_rn(q.y, cn, d01);
        d10 = __fmaf_rn(-q.x, cn, d10);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        u += __shfl_xor_sync(0xffffffffu, u, o);
        v += __shfl_xor_sync(0xffffffffu, v, o);
        d00 += __shfl_xor_sync(0xffffffffu, d00, o);
        d01 += __shfl_xor_sync(0xffffffffu, d01, o);
        d10 += __shfl_xor_sync(0xffffffffu, d10, o);
    }
    V2 r;
    r.u = u; r.v = v; r.d00 = d00; r.d01 = d01; r.d10 = d10; r.d11 = -d00;
    return r;
}

// The RK3 trace of one point by a whole warp (WAVES2D; all lanes get the result).
__device__ __forceinline__ void trace2d_waves_warp(const VelParams &vp, const StageCoef &sc, float x,
                                                   float y, float dt, float &dx, float &dy, float J[4])
{
    trace2d_eval<TR_RK3>(vel2d_waves_warp(vp, sc, 0, x, y),
                         [&](int stage, float px, float py) { return vel2d_waves_warp(vp, sc, stage, px, py); },
                         x, y, dt, dx, dy, J);
}

// ---------------------------------------------------------------- cell location

// Node index i, foot displacement in cells dc, n nodes: cell k in [0, n-2] and xi in
// [0, 1]; feet outside the box are clamped to its faces.
__device__ __forceinline__ void locate(int i, float dc, int n, int &k, float &xi)
{
    float fl = floorf(dc);
    int kk = i + (int)fl;
    float r = dc - fl;
    if (kk < 0) { k = 0; xi = 0.f; }
    else if (kk >= n - 1) { k = n - 2; xi = 1.f; }
    else { k = kk; xi = r; }
}

// ---------------------------------------------------------------- Hermite basis

// 1D basis at xi for a cell of length h, pre-scaled:
//   value part   F0 = 1 - S, F1 = S with S = 3 xi^2 - 2 xi^3  (f(xi), f(1-xi))
//   slope part   hG0 = h g(xi), hG1 = -h g(1-xi)               (g(x) = x (1-x)^2)
//   derivatives  dS = S'(xi)/h, dG0 = g'(xi), dG1 = g'(1-xi)
// The value part is evaluated from the nearer end: p_near + (p1 - p0) (S - near), with
// near = (xi >= 1/2).  At xi = 0 or 1 this returns the end value exactly, so a foot
// that lands on a node reproduces the node's data bit for bit.
struct Basis1 { float Sn, dS, hG0, hG1, dG0, dG1; bool near1; };

__device__ __forceinline__ Basis1 basis1(float xi, float h, float ih)
{
    Basis1 b;
    float om = 1.f - xi;
    float S = xi * xi * (3.f - 2.f * xi);
    b.near1 = xi >= 0.5f;
    b.Sn = b.near1 ? S - 1.f : S;
    b.dS = 6.f * xi * om * ih;
    b.hG0 = h * xi * om * om;
    b.hG1 = -h * om * xi * xi;
    b.dG0 = om * (1.f - 3.f * xi);
    b.dG1 = xi * (3.f * xi - 2.f);
    return b;
}

// 1D Hermite reduction of an end pair (p0, p1) with slopes (s0, s1): value and derivative
__device__ __forceinline__ float hval(const Basis1 &b, float p0, float p1, float s0, float s1)
{
    return fmaf(p1 - p0, b.Sn, fmaf(s0, b.hG0, fmaf(s1, b.hG1, b.near1 ? p1 : p0)));
}
__device__ __forceinline__ float hder(const Basis1 &b, float p0, float p1, float s0, float s1)
{
    return fmaf(p1 - p0, b.dS, fmaf(s0, b.dG0, s1 * b.dG1));
}

// 2D cell data: c[v][a] with corner v = vx + 2 vy and a = 0 phi, 1 phi_x, 2 phi_y, 3 phi_xy.
// Returns H, H_x, H_y.
__device__ __forceinline__ void hermite2d(const float c[4][4], const Basis1 &bx,
                                          const Basis1 &by, float &H, float &Hx, float &Hy)
{
    // subtract phi of the corner nearest to the foot: the value terms become O(h)
    const float b0 = bx.near1 ? c[1][0] : c[0][0];
    const float b1 = bx.near1 ? c[3][0] : c[2][0];
    const float base = by.near1 ? b1 : b0;
    float p00 = c[0][0] - base, p10 = c[1][0] - base, p01 = c[2][0] - base, p11 = c[3][0] - base;
    // along x on rows y0 (B=0) and y1 (B=1)
    float P0 = hval(bx, p00, p10, c[0][1], c[1][1]);
    float P1 = hval(bx, p01, p11, c[2][1], c[3][1]);
    float Pd0 = hder(bx, p00, p10, c[0][1], c[1][1]);
    float Pd1 = hder(bx, p01, p11, c[2][1], c[3][1]);
    float Q0 = hval(bx, c[0][2], c[1][2], c[0][3], c[1][3]);
    float Q1 = hval(bx, c[2][2], c[3][2], c[2][3], c[3][3]);
    float Qd0 = hder(bx, c[0][2], c[1][2], c[0][3], c[1][3]);
    float Qd1 = hder(bx, c[2][2], c[3][2], c[2][3], c[3][3]);
    // along y
    H = base + hval(by, P0, P1, Q0, Q1);
    Hy = hder(by, P0, P1, Q0, Q1);
    Hx = hval(by, Pd0, Pd1, Qd0, Qd1);
}

// 3D cell data: c[v][a], corner v = vx + 2 vy + 4 vz, a = plane index
// (0 phi, 1 x, 2 y, 3 z, 4 xy, 5 xz, 6 yz, 7 xyz).  Returns H and its gradient.
__device__ __forceinline__ void hermite3d(const float c[8][8], const Basis1 &bx,
                                          const Basis1 &by, const Basis1 &bz, float &H,
                                          float g[3])
{
    // subtract phi of the corner nearest to the foot: the value terms become O(h)
    const int vn = (bx.near1 ? 1 : 0) + (by.near1 ? 2 : 0) + (bz.near1 ? 4 : 0);
    float base = c[0][0];
#pragma unroll
    for (int v = 1; v < 8; ++v) base = (v == vn) ? c[v][0] : base;
    float R[2], Rx[2], Ry[2], Rz[2], Rzx[2], Rzy[2];
#pragma unroll
    for (int C = 0; C < 2; ++C) {
        float P[2], Pd[2], Qy[2], Qyd[2], Qz[2], Qzd[2], Qyz[2], Qyzd[2];
#pragma unroll
        for (int B = 0; B < 2; ++B) {
            int v0 = 2 * B + 4 * C, v1 = v0 + 1;
            float p0 = c[v0][0] - base, p1 = c[v1][0] - base;
            P[B] = hval(bx, p0, p1, c[v0][1], c[v1][1]);
            Pd[B] = hder(bx, p0, p1, c[v0][1], c[v1][1]);
            Qy[B] = hval(bx, c[v0][2], c[v1][2], c[v0][4], c[v1][4]);
            Qyd[B] = hder(bx, c[v0][2], c[v1][2], c[v0][4], c[v1][4]);
            Qz[B] = hval(bx, c[v0][3], c[v1][3], c[v0][5], c[v1][5]);
            Qzd[B] = hder(bx, c[v0][3], c[v1][3], c[v0][5], c[v1][5]);
            Qyz[B] = hval(bx, c[v0][6], c[v1][6], c[v0][7], c[v1][7]);
            Qyzd[B] = hder(bx, c[v0][6], c[v1][6], c[v0][7], c[v1][7]);
        }
        R[C] = hval(by, P[0], P[1], Qy[0], Qy[1]);
        Ry[C] = hder(by, P[0], P[1], Qy[0], Qy[1]);
        Rx[C] = hval(by, Pd[0], Pd[1], Qyd[0], Qyd[1]);
        Rz[C] = hval(by, Qz[0], Qz[1], Qyz[0], Qyz[1]);
        Rzy[C] = hder(by, Qz[0], Qz[1], Qyz[0], Qyz[1]);
        Rzx[C] = hval(by, Qzd[0], Qzd[1], Qyzd[0], Qyzd[1]);
    }
    H = base + hval(bz, R[0], R[1], Rz[0], Rz[1]);
    g[2] = hder(bz, R[0], R[1], Rz[0], Rz[1]);
    g[0] = hval(bz, Rx[0], Rx[1], Rzx[0], Rzx[1]);
    g[1] = hval(bz, Ry[0], Ry[1], Rzy[0], Rzy[1]);
}

// ---------------------------------------------------------------- approach B (cell-based)

// Vertex (u, w) of a facet from its edge-centre differences e (along the facet's second
// axis, at first-axis index 0, 1) and f (along the first axis, at second-axis index 0, 1):
// 3/4 of the two edges through the vertex, -1/4 of the two opposite ones (Sec. 2.3 (B)).
__device__ __forceinline__ float cell_vertex(float e0, float e1, float f0, float f1, int u, int w)
{
    const float ne = u ? e1 : e0, fe = u ? e0 : e1, nf = w ? f1 : f0, ff = w ? f0 : f1;
    return 0.75f * (ne + nf) - 0.25f * (fe + ff);
}

// 2D cell, c[v][a] (v = vx + 2 vy; a = 0 phi, 1 phi_x, 2 phi_y, 3 phi_xy): phi_xy at the
// four vertices from psi_x differenced along y and psi_y differenced along x.
__device__ __forceinline__ void cross_cell2d(float c[4][4], float ih0, float ih1)
{
    const float e0 = (c[2][1] - c[0][1]) * ih1, e1 = (c[3][1] - c[1][1]) * ih1;
    const float f0 = (c[1][2] - c[0][2]) * ih0, f1 = (c[3][2] - c[2][2]) * ih0;
#pragma unroll
    for (int v = 0; v < 4; ++v) c[v][3] = cell_vertex(e0, e1, f0, f1, v & 1, v >> 1);
}

// 3D cell: q(v, a) gives phi (a = 0) and psi_x, psi_y, psi_z (a = 1..3) at vertex
// v = vx + 2 vy + 4 vz; cr[v] = (phi_xy, phi_xz, phi_yz, phi_xyz), each pair derivative
// in the vertex's facet spanning its two axes, phi_xyz from the double difference of
// psi_z over the vertex's x-y facet.
template <class Q>
__device__ __forceinline__ void cross_cell3d(const Q &q, float ih0, float ih1, float ih2,
                                             float cr[8][4])
{
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const int a = v & 1, b = (v >> 1) & 1, c = v >> 2;
        auto P = [&](int x, int y, int z, int comp) { return q(x + 2 * y + 4 * z, comp); };
        cr[v][0] = cell_vertex((P(0, 1, c, 1) - P(0, 0, c, 1)) * ih1, (P(1, 1, c, 1) - P(1, 0, c, 1)) * ih1,
                               (P(1, 0, c, 2) - P(0, 0, c, 2)) * ih0, (P(1, 1, c, 2) - P(0, 1, c, 2)) * ih0, a, b);
        cr[v][1] = cell_vertex((P(0, b, 1, 1) - P(0, b, 0, 1)) * ih2, (P(1, b, 1, 1) - P(1, b, 0, 1)) * ih2,
                               (P(1, b, 0, 3) - P(0, b, 0, 3)) * ih0, (P(1, b, 1, 3) - P(0, b, 1, 3)) * ih0, a, c);
        cr[v][2] = cell_vertex((P(a, 0, 1, 2) - P(a, 0, 0, 2)) * ih2, (P(a, 1, 1, 2) - P(a, 1, 0, 2)) * ih2,
                               (P(a, 1, 0, 3) - P(a, 0, 0, 3)) * ih1, (P(a, 1, 1, 3) - P(a, 0, 1, 3)) * ih1, b, c);
        cr[v][3] = (P(1, 1, c, 3) - P(0, 1, c, 3) - P(1, 0, c, 3) + P(0, 0, c, 3)) * ih0 * ih1;
    }
}

// ---------------------------------------------------------------- approach A stencils

// First derivative along one axis from three samples, shared by every kernel that
// rebuilds mixed derivatives so that all paths round identically:
//   interior  (u[i+1] - u[i-1]) / (2h)
//   i = 0     (-3 u0 + 4 u1 - u2) / (2h)
//   i = n-1   (3 u_{n-1} - 4 u_{n-2} + u_{n-3}) / (2h)
__device__ __forceinline__ float dcentral(float up, float um, float i2h)
{
    return __fmul_rn(__fsub_rn(up, um), i2h);
}
__device__ __forceinline__ float dfirst(float u0, float u1, float u2, float i2h)
{
    return __fmul_rn(__fmaf_rn(4.f, u1, __fmaf_rn(-3.f, u0, -u2)), i2h);
}
__device__ __forceinline__ float dlast(float un1, float un2, float un3, float i2h)
{
    return __fmul_rn(__fmaf_rn(-4.f, un2, __fmaf_rn(3.f, un1, un3)), i2h);
}

// Derivative at index i of a line accessed through get(idx) (n >= 3).
template <class Get>
__device__ __forceinline__ float dline(int i, int n, float i2h, Get get)
{
    if (i == 0) return dfirst(get(0), get(1), get(2), i2h);
    if (i == n - 1) return dlast(get(n - 1), get(n - 2), get(n - 3), i2h);
    return dcentral(get(i + 1), get(i - 1), i2h);
}

}  // namespace gals
