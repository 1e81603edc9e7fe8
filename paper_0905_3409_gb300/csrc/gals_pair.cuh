// gals_pair.cuh -- the node update for two nodes at once in paired FP32 arithmetic.
//
// Blackwell executes fma/add/mul on float2 operands as one instruction (FFMA2 and
// friends, __ffma2_rn & co.), so a thread that advances two nodes of the same column
// (2D: rows j and j+1; 3D: z-levels k and k+1) issues about half the floating-point
// instructions of two scalar updates, and has twice the independent loads in flight.
// Lane x of every float2 is the first node, lane y the second.  The arithmetic is the one
// of gals_device.cuh: superconsistent RK3 trace with Jacobian (Sec. 5.1), cell location,
// bi-/tricubic Hermite value and gradient (Sec. 2.3) from the cell's phi shifted by its
// first corner, J^T grad H.
// Each lane rounds exactly like a scalar FMA/ADD/MUL chain of the same expression.
#pragma once

#include "gals_device.cuh"

namespace gals {

typedef float2 F2;

__device__ __forceinline__ F2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ F2 add2(F2 a, F2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ F2 mul2(F2 a, F2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ F2 sub2(F2 a, F2 b) { return __ffma2_rn(b, bc(-1.f), a); }   // a - b
__device__ __forceinline__ F2 neg2(F2 a) { return __fmul2_rn(a, bc(-1.f)); }

struct V2p { F2 u, v, d00, d01, d10, d11; };

// per-lane sin(pi s), cos(pi s)
__device__ __forceinline__ void sincospi2(F2 s, F2 &sn, F2 &cs)
{
    sincospi_f(s.x, &sn.x, &cs.x);
    sincospi_f(s.y, &sn.y, &cs.y);
}

// per-lane sin a, cos a with a = 2 pi (s - 1/2) (see sincos_turn)
__device__ __forceinline__ void sincos_turn2(F2 s, F2 &A, F2 &B)
{
    const F2 a = fma2(s, bc(2.f * kPi), bc(-kPi));
    __sincosf(a.x, &A.x, &B.x);
    __sincosf(a.y, &A.y, &B.y);
}

// the same with the angle negated: An = -sin a, B = cos a
__device__ __forceinline__ void sincos_turn2n(F2 s, F2 &An, F2 &B)
{
    const F2 a = fma2(s, bc(-2.f * kPi), bc(kPi));
    __sincosf(a.x, &An.x, &B.x);
    __sincosf(a.y, &An.y, &B.y);
}

// Fourier tables duplicated into float2 pairs (both lanes use the same coefficient).
struct StageCoefPair {
    F2 A[3][16], Al[3][16], All[3][16];
};

template <int VK>
__device__ __forceinline__ V2p vel2d_pair(const VelParams &vp, const StageCoef &sc,
                                          const StageCoefPair *scp, int stage, F2 x, F2 y)
{
    V2p r;
    if (VK == VK_CONST) {
        r.u = bc(vp.c0); r.v = bc(vp.c1);
        r.d00 = r.d01 = r.d10 = r.d11 = bc(0.f);
    } else if (VK == VK_ROTATION) {
        const F2 w = bc(vp.omega);
        r.u = mul2(bc(-vp.omega), sub2(y, bc(vp.cy)));
        r.v = mul2(w, sub2(x, bc(vp.cx)));
        r.d00 = bc(0.f); r.d01 = bc(-vp.omega); r.d10 = w; r.d11 = bc(0.f);
    } else if (VK == VK_VORTEX2D) {
        // u = -c sin^2(pi x) sin(2 pi y), v = c sin(2 pi x) sin^2(pi y) in the factors
        // A = sin a = -sin(2 pi s), B = cos a = -cos(2 pi s), sin^2(pi s) = (1 + B)/2
        F2 Ax, Bx, Ay, By;
        sincos_turn2(x, Ax, Bx);
        sincos_turn2(y, Ay, By);
        const float c = sc.mod[stage], h = 0.5f * c;
        const F2 cSx = fma2(Bx, bc(h), bc(h)), mcSy = fma2(By, bc(-h), bc(-h));
        r.u = mul2(cSx, Ay);
        r.v = mul2(Ax, mcSy);
        r.d00 = mul2(bc(-c * kPi), mul2(Ax, Ay));
        r.d01 = mul2(bc(2.f * kPi), mul2(cSx, By));
        r.d10 = mul2(bc(2.f * kPi), mul2(Bx, mcSy));
        r.d11 = neg2(r.d00);
    } else if (VK == VK_PSEUDO1D) {
        const F2 arg = fma2(bc(vp.d0), x, mul2(bc(vp.d1), y));
        const F2 e = make_float2(__expf(arg.x), __expf(arg.y));
        r.u = mul2(e, bc(vp.d0)); r.v = mul2(e, bc(vp.d1));
        r.d00 = mul2(e, bc(vp.d0 * vp.d0)); r.d01 = mul2(e, bc(vp.d0 * vp.d1));
        r.d10 = r.d01; r.d11 = mul2(e, bc(vp.d1 * vp.d1));
    } else if (VK == VK_WAVES2D) {
        // Psi = sum C_m sin(theta_m), theta_m = kx x + ky y + phase (the scalar vel2d, lane by lane)
        const WaveTab T = wave_tab(vp.waves, vp.nwaves);
        const float *amp = sc.wamp + stage * vp.nwaves;
        F2 u = bc(0.f), v = bc(0.f), d00 = bc(0.f), d01 = bc(0.f), d10 = bc(0.f);
#pragma unroll 4
        for (int m = 0; m < vp.nwaves; ++m) {
            const float4 g = __ldg(T.geo + m), q = __ldg(T.sq + m);
            const F2 C = bc(__ldg(amp + m));
            const F2 th = fma2(bc(g.x), x, fma2(bc(g.y), y, bc(g.z)));
            F2 sn, cs;
            __sincosf(th.x, &sn.x, &cs.x);
            __sincosf(th.y, &sn.y, &cs.y);
            const F2 cc = mul2(C, cs), cn = mul2(C, sn);
            u = fma2(bc(-g.y), cc, u);
            v = fma2(bc(g.x), cc, v);
            d00 = fma2(bc(g.w), cn, d00);
            d01 = fma2(bc(q.y), cn, d01);
            d10 = fma2(bc(-q.x), cn, d10);
        }
        r.u = u; r.v = v; r.d00 = d00; r.d01 = d01; r.d10 = d10; r.d11 = neg2(d00);
    } else {  // VK_FOURIER2D: Psi = sum A_kl s_k(x) s_l(y), u = -Psi_y, v = Psi_x
        F2 s[5], c[5], sy_[5], cy_[5];
        sincospi2(x, s[1], c[1]);
        sincospi2(y, sy_[1], cy_[1]);
        const F2 two = bc(2.f), one = bc(1.f), mtwo = bc(-2.f);
        s[2] = mul2(two, mul2(s[1], c[1]));            c[2] = fma2(mtwo, mul2(s[1], s[1]), one);
        s[3] = fma2(s[2], c[1], mul2(c[2], s[1]));     c[3] = fma2(c[2], c[1], neg2(mul2(s[2], s[1])));
        s[4] = mul2(two, mul2(s[2], c[2]));            c[4] = fma2(mtwo, mul2(s[2], s[2]), one);
        sy_[2] = mul2(two, mul2(sy_[1], cy_[1]));          cy_[2] = fma2(mtwo, mul2(sy_[1], sy_[1]), one);
        sy_[3] = fma2(sy_[2], cy_[1], mul2(cy_[2], sy_[1])); cy_[3] = fma2(cy_[2], cy_[1], neg2(mul2(sy_[2], sy_[1])));
        sy_[4] = mul2(two, mul2(sy_[2], cy_[2]));          cy_[4] = fma2(mtwo, mul2(sy_[2], sy_[2]), one);
        F2 u = bc(0.f), v = bc(0.f), d00 = bc(0.f), d01 = bc(0.f), d10 = bc(0.f);
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            F2 Ux = bc(0.f), Vx = bc(0.f), W = bc(0.f);
#pragma unroll
            for (int l = 1; l <= 4; ++l) {
                const int kl = (k - 1) * 4 + (l - 1);
                Ux = fma2(scp->Al[stage][kl], cy_[l], Ux);
                Vx = fma2(scp->A[stage][kl], sy_[l], Vx);
                W = fma2(scp->All[stage][kl], sy_[l], W);
            }
            const float kp = (float)k * kPi;
            u = fma2(neg2(s[k]), Ux, u);
            v = fma2(mul2(bc(kp), c[k]), Vx, v);
            d00 = fma2(mul2(bc(-kp), c[k]), Ux, d00);
            d01 = fma2(s[k], W, d01);
            d10 = fma2(mul2(bc(-kp * kp), s[k]), Vx, d10);
        }
        r.u = u; r.v = v; r.d00 = d00; r.d01 = d01; r.d10 = d10; r.d11 = neg2(d00);
    }
    return r;
}

// Gradient update of the CIR form (Sec. 4, step 3) by Heun's method: from psi0 = grad H at
// the foot (time t) to the node (time t + dt) along the characteristic,
// d psi / d tau = -Dv^T psi; Df = Dv at the foot and time t, Dn = Dv at the node, t + dt.
__device__ __forceinline__ void heun_psi2(const V2p &Df, const V2p &Dn, float dt, F2 gx, F2 gy,
                                          F2 &px, F2 &py)
{
    const F2 k1x = neg2(fma2(Df.d00, gx, mul2(Df.d10, gy)));
    const F2 k1y = neg2(fma2(Df.d01, gx, mul2(Df.d11, gy)));
    const F2 sx = fma2(bc(dt), k1x, gx), sy = fma2(bc(dt), k1y, gy);
    const F2 k2x = neg2(fma2(Dn.d00, sx, mul2(Dn.d10, sy)));
    const F2 k2y = neg2(fma2(Dn.d01, sx, mul2(Dn.d11, sy)));
    px = fma2(bc(0.5f * dt), add2(k1x, k2x), gx);
    py = fma2(bc(0.5f * dt), add2(k1y, k2y), gy);
}

// Superconsistent trace of Sec. 5.1 for two nodes; a = v(x, t+dt) supplied by the caller.
template <int TR, int VK>
__device__ __forceinline__ void trace2d_pair(const V2p &a, const VelParams &vp,
                                             const StageCoef &sc, const StageCoefPair *scp,
                                             F2 x, F2 y, float dt, F2 &dx, F2 &dy, F2 J[4])
{
    const F2 mdt = bc(-dt), one = bc(1.f);
    if (TR == TR_EULER) {
        dx = mul2(mdt, a.u); dy = mul2(mdt, a.v);
        J[0] = fma2(mdt, a.d00, one); J[1] = mul2(mdt, a.d01);
        J[2] = mul2(mdt, a.d10);      J[3] = fma2(mdt, a.d11, one);
        return;
    }
    // stage 1: x1 = x - dt v1, J1 = I - dt Dv1
    const F2 J1_00 = fma2(mdt, a.d00, one), J1_01 = mul2(mdt, a.d01);
    const F2 J1_10 = mul2(mdt, a.d10), J1_11 = fma2(mdt, a.d11, one);
    const V2p b = vel2d_pair<VK>(vp, sc, scp, 1, fma2(mdt, a.u, x), fma2(mdt, a.v, y));
    // S = Dv1 + Dv2 J1 (Dv1 is the accumulator of the product)
    const F2 S00 = fma2(b.d00, J1_00, fma2(b.d01, J1_10, a.d00));
    const F2 S01 = fma2(b.d00, J1_01, fma2(b.d01, J1_11, a.d01));
    const F2 S10 = fma2(b.d10, J1_00, fma2(b.d11, J1_10, a.d10));
    const F2 S11 = fma2(b.d10, J1_01, fma2(b.d11, J1_11, a.d11));
    // stage 2: x2 = x - dt (v1 + v2)/4, J2 = I - dt S / 4, kept as G = (-2 dt / 3) J2
    const F2 mq = bc(-0.25f * dt), m23 = bc(-2.f * dt / 3.f), kq = bc((-2.f * dt / 3.f) * (-0.25f * dt));
    const F2 G00 = fma2(kq, S00, m23), G01 = mul2(kq, S01), G10 = mul2(kq, S10), G11 = fma2(kq, S11, m23);
    const V2p c = vel2d_pair<VK>(vp, sc, scp, 2, fma2(mq, add2(a.u, b.u), x),
                                 fma2(mq, add2(a.v, b.v), y));
    // foot = x - dt (w3 + (w1 + w2 - 2 w3)/6): exact for constant v;
    // J = I - dt S / 6 - 2 dt Dv3 J2 / 3 = (I - dt S / 6) + Dv3 G (= I when Dv = 0)
    const F2 i6 = bc(1.f / 6.f), m2 = bc(-2.f), m6 = bc(-dt / 6.f);
    dx = mul2(mdt, fma2(fma2(m2, c.u, add2(a.u, b.u)), i6, c.u));
    dy = mul2(mdt, fma2(fma2(m2, c.v, add2(a.v, b.v)), i6, c.v));
    J[0] = fma2(c.d00, G00, fma2(c.d01, G10, fma2(m6, S00, one)));
    J[1] = fma2(c.d00, G01, fma2(c.d01, G11, mul2(m6, S01)));
    J[2] = fma2(c.d10, G00, fma2(c.d11, G10, mul2(m6, S10)));
    J[3] = fma2(c.d10, G01, fma2(c.d11, G11, fma2(m6, S11, one)));
}

// Foot cells of the two lanes along one axis (the lanes' node indices i0, i1, their
// displacements in cells dc): the same cells and local coordinates as locate(), lane by
// lane.  The clamp acts on the displacement first, so that a foot before the first node
// lands on (cell 0, xi = 0) and one at or past the last node on (cell n - 2, xi = 1):
// floor(dc) then needs one clamp from above, and xi = dc - floor(dc) is one paired
// subtraction.  Every branch of locate() becomes a min/max.  (The 3D step keeps
// locate(): with its higher register pressure the paired form measured slower there.)
__device__ __forceinline__ void locate_pair(int i0, int i1, F2 dc, int n, int &k0, int &k1, F2 &xi)
{
    const float hi0 = (float)(n - 1 - i0), hi1 = (float)(n - 1 - i1);
    const float c0 = fminf(fmaxf(dc.x, (float)(-i0)), hi0);
    const float c1 = fminf(fmaxf(dc.y, (float)(-i1)), hi1);
    const float f0 = fminf(floorf(c0), hi0 - 1.f), f1 = fminf(floorf(c1), hi1 - 1.f);
    k0 = i0 + (int)f0;
    k1 = i1 + (int)f1;
    xi = sub2(make_float2(c0, c1), make_float2(f0, f1));
}

// Paired 1D basis: S = 3 xi^2 - 2 xi^3, dS = S'(xi)/h, hG0 = h g(xi), hG1 = -h g(1 - xi),
// dG0 = g'(xi), dG1 = -g'(1 - xi) (g(x) = x (1 - x)^2; eq. 1-cubic_basis_functions).
struct Basis2 { F2 S, dS, hG0, hG1, dG0, dG1; };

__device__ __forceinline__ Basis2 basis_pair(F2 xi, float h, float ih)
{
    Basis2 b;
    const F2 om = fma2(xi, bc(-1.f), bc(1.f));
    const F2 xx = mul2(xi, xi), xo = mul2(xi, om);
    b.S = mul2(xx, fma2(bc(-2.f), xi, bc(3.f)));
    b.dS = mul2(xo, bc(6.f * ih));
    b.hG0 = mul2(mul2(xo, om), bc(h));
    b.hG1 = mul2(mul2(om, xx), bc(-h));
    b.dG0 = mul2(om, fma2(bc(-3.f), xi, bc(1.f)));
    b.dG1 = mul2(xi, fma2(bc(3.f), xi, bc(-2.f)));
    return b;
}

// 1D cubic Hermite value and derivative along a cell edge from the end values p0, p1 and
// slopes s0, s1, evaluated from the first end: p0 + (p1 - p0) S + s0 h g(xi) - s1 h g(1-xi).
// At xi = 0 the value is p0 and the derivative s0, exactly.
__device__ __forceinline__ F2 hval2(const Basis2 &b, F2 p0, F2 p1, F2 s0, F2 s1)
{
    return fma2(sub2(p1, p0), b.S, fma2(s0, b.hG0, fma2(s1, b.hG1, p0)));
}
__device__ __forceinline__ F2 hder2(const Basis2 &b, F2 p0, F2 p1, F2 s0, F2 s1)
{
    return fma2(sub2(p1, p0), b.dS, fma2(s0, b.dG0, mul2(s1, b.dG1)));
}
// the same with p0 = 0
__device__ __forceinline__ F2 hval2z(const Basis2 &b, F2 p1, F2 s0, F2 s1)
{
    return fma2(p1, b.S, fma2(s0, b.hG0, mul2(s1, b.hG1)));
}
__device__ __forceinline__ F2 hder2z(const Basis2 &b, F2 p1, F2 s0, F2 s1)
{
    return fma2(p1, b.dS, fma2(s0, b.dG0, mul2(s1, b.dG1)));
}

// Bicubic Hermite value and gradient (eq. p-cubic_interpolant, sum-factorised: x, then y).
// c[v][a]: corner v = vx + 2 vy, data a = 0 phi, 1 phi_x, 2 phi_y, 3 phi_xy (both lanes).
// phi is shifted by its value at corner 0 (the interpolant reproduces constants): the
// x-reduced values P0, P1 are then O(h), so the y-derivative (P1 - P0) dS, whose factor is
// O(1/h), carries no rounding error of the O(1) phi itself.  A foot on a node (xi = eta =
// 0) returns that node's data exactly.
__device__ __forceinline__ void hermite2d_pair(const F2 c[4][4], const Basis2 &bx,
                                               const Basis2 &by, F2 &H, F2 &Hx, F2 &Hy)
{
    const F2 base = c[0][0];
    const F2 p10 = sub2(c[1][0], base), p01 = sub2(c[2][0], base), p11 = sub2(c[3][0], base);
    const F2 P0 = hval2z(bx, p10, c[0][1], c[1][1]);
    const F2 P1 = hval2(bx, p01, p11, c[2][1], c[3][1]);
    const F2 Pd0 = hder2z(bx, p10, c[0][1], c[1][1]);
    const F2 Pd1 = hder2(bx, p01, p11, c[2][1], c[3][1]);
    const F2 Q0 = hval2(bx, c[0][2], c[1][2], c[0][3], c[1][3]);
    const F2 Q1 = hval2(bx, c[2][2], c[3][2], c[2][3], c[3][3]);
    const F2 Qd0 = hder2(bx, c[0][2], c[1][2], c[0][3], c[1][3]);
    const F2 Qd1 = hder2(bx, c[2][2], c[3][2], c[2][3], c[3][3]);
    H = add2(base, hval2(by, P0, P1, Q0, Q1));
    Hy = hder2(by, P0, P1, Q0, Q1);
    Hx = hval2(by, Pd0, Pd1, Qd0, Qd1);
}

// ---------------------------------------------------------------- 3D, two nodes per thread

struct V3p { F2 v[3]; F2 d[9]; };

// The deformation field from its folded xy products P1 = 2 Sx Ay, P2 = -Ax Sy,
// P3 = -Ax Ay, P4 = 4 pi Sx By, P5 = -2 pi Bx Sy, P6 = -2 pi Bx Ay, P7 = -2 pi Ax By and
// z factors Azc = c Az, Szc = c Sz, Bzc = 2 pi c Bz (see vel3d_pair).
__device__ __forceinline__ void deform_terms(F2 P1, F2 P2, F2 P3, F2 P4, F2 P5, F2 P6, F2 P7,
                                             F2 Azc, F2 Szc, F2 Bzc, V3p &r)
{
    const F2 T = mul2(P3, Azc);                  // -c Ax Ay Az
    r.v[0] = mul2(P1, Azc);
    r.v[1] = mul2(P2, Azc);
    r.v[2] = mul2(P3, Szc);
    r.d[0] = mul2(bc(2.f * kPi), T);
    r.d[1] = mul2(P4, Azc);
    r.d[2] = mul2(P1, Bzc);
    r.d[3] = mul2(P5, Azc);
    r.d[4] = mul2(bc(-kPi), T);
    r.d[5] = mul2(P2, Bzc);
    r.d[6] = mul2(P6, Szc);
    r.d[7] = mul2(P7, Szc);
    r.d[8] = r.d[4];
}

// v and Dv (Dv[3i+j] = dv_i/dx_j) at two points; DEFORM3D is LeVeque's field
// u = 2 sin^2(pi x) sin(2 pi y) sin(2 pi z) c, v = -sin(2 pi x) sin^2(pi y) sin(2 pi z) c,
// w = -sin(2 pi x) sin(2 pi y) sin^2(pi z) c with c = cos(pi t / T).
template <int VK>
__device__ __forceinline__ V3p vel3d_pair(const VelParams &vp, const StageCoef &sc, int stage,
                                          F2 x, F2 y, F2 z)
{
    V3p r;
#pragma unroll
    for (int a = 0; a < 9; ++a) r.d[a] = bc(0.f);
    if (VK == VK_CONST) {
        r.v[0] = bc(vp.c0); r.v[1] = bc(vp.c1); r.v[2] = bc(vp.c2);
    } else if (VK == VK_ROTATION) {
        r.v[0] = mul2(bc(-vp.omega), sub2(y, bc(vp.cy)));
        r.v[1] = mul2(bc(vp.omega), sub2(x, bc(vp.cx)));
        r.v[2] = bc(0.f);
        r.d[1] = bc(-vp.omega); r.d[3] = bc(vp.omega);
    } else {  // VK_DEFORM3D
        // In the factors A = sin a, B = cos a of a = 2 pi (s - 1/2) and S = sin^2(pi s) =
        // (1 + B)/2 every term is (constant) x (x factor)(y factor)(z factor); the constants
        // are folded into the factors: x with the angle negated (A -> -A), 2S and -2 pi B;
        // y: S and 2 pi B; z: c A, c S and 2 pi c B.
        F2 Axn, Bx, Ay, By, Az, Bz;
        sincos_turn2n(x, Axn, Bx);
        sincos_turn2(y, Ay, By);
        sincos_turn2(z, Az, Bz);
        const float c = sc.mod[stage], h = 0.5f * c;
        const F2 Sx2 = add2(Bx, bc(1.f)), Bxm = mul2(bc(-2.f * kPi), Bx);
        const F2 Sy = fma2(By, bc(0.5f), bc(0.5f)), By2 = mul2(bc(2.f * kPi), By);
        const F2 Azc = mul2(bc(c), Az), Szc = fma2(Bz, bc(h), bc(h)), Bzc = mul2(bc(2.f * kPi * c), Bz);
        deform_terms(mul2(Sx2, Ay), mul2(Axn, Sy), mul2(Axn, Ay), mul2(Sx2, By2), mul2(Bxm, Sy),
                     mul2(Bxm, Ay), mul2(Axn, By2), Azc, Szc, Bzc, r);
    }
    return r;
}

// C = A B + D (3x3, row-major), D the accumulator of each entry's chain
__device__ __forceinline__ void matmul3_acc_pair(const F2 *A, const F2 *B, const F2 *D, F2 *C)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = fma2(A[3 * i], B[j], fma2(A[3 * i + 1], B[3 + j], fma2(A[3 * i + 2], B[6 + j], D[3 * i + j])));
}

// 3D gradient update of the CIR form by Heun's method (see heun_psi2); Df, Dn as there.
__device__ __forceinline__ void heun_psi3(const V3p &Df, const V3p &Dn, float dt, const F2 g[3],
                                          F2 psi[3])
{
    F2 k1[3], s[3], k2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        k1[a] = neg2(fma2(Df.d[a], g[0], fma2(Df.d[3 + a], g[1], mul2(Df.d[6 + a], g[2]))));
#pragma unroll
    for (int a = 0; a < 3; ++a) s[a] = fma2(bc(dt), k1[a], g[a]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        k2[a] = neg2(fma2(Dn.d[a], s[0], fma2(Dn.d[3 + a], s[1], mul2(Dn.d[6 + a], s[2]))));
#pragma unroll
    for (int a = 0; a < 3; ++a) psi[a] = fma2(bc(0.5f * dt), add2(k1[a], k2[a]), g[a]);
}

// Superconsistent RK3 trace of Sec. 5.1 for two nodes (a = v(x, t+dt) from the caller):
// d = foot - x and J[3i+j] = d foot_i / d x_j.
template <int TR, int VK>
__device__ __forceinline__ void trace3d_pair(const V3p &a, const VelParams &vp, const StageCoef &sc,
                                             F2 x, F2 y, F2 z, float dt, F2 d[3], F2 J[9])
{
    const F2 mdt = bc(-dt), one = bc(1.f);
    if (TR == TR_EULER) {
#pragma unroll
        for (int i = 0; i < 3; ++i) d[i] = mul2(mdt, a.v[i]);
#pragma unroll
        for (int e = 0; e < 9; ++e) J[e] = (e % 4) == 0 ? fma2(mdt, a.d[e], one) : mul2(mdt, a.d[e]);
        return;
    }
    F2 J1[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) J1[e] = (e % 4) == 0 ? fma2(mdt, a.d[e], one) : mul2(mdt, a.d[e]);
    const V3p b = vel3d_pair<VK>(vp, sc, 1, fma2(mdt, a.v[0], x), fma2(mdt, a.v[1], y),
                                 fma2(mdt, a.v[2], z));
    // S = Dv1 + Dv2 J1 (Dv1 is the accumulator of the product)
    F2 S[9];
    matmul3_acc_pair(b.d, J1, a.d, S);
    const F2 mq = bc(-0.25f * dt);
    F2 J2[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) J2[e] = (e % 4) == 0 ? fma2(mq, S[e], one) : mul2(mq, S[e]);
    F2 s1[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) s1[i] = add2(a.v[i], b.v[i]);
    const V3p c = vel3d_pair<VK>(vp, sc, 2, fma2(mq, s1[0], x), fma2(mq, s1[1], y), fma2(mq, s1[2], z));
    F2 N[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            N[3 * i + j] = fma2(c.d[3 * i], J2[j], fma2(c.d[3 * i + 1], J2[3 + j], mul2(c.d[3 * i + 2], J2[6 + j])));
    // d = -dt (w3 + (w1 + w2 - 2 w3)/6): exact for constant v;
    // J = I - dt S / 6 - 2 dt N / 3 (= I when Dv = 0)
    const F2 i6 = bc(1.f / 6.f), m2 = bc(-2.f), m6 = bc(-dt / 6.f), m23 = bc(-2.f * dt / 3.f);
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = mul2(mdt, fma2(fma2(m2, c.v[i], s1[i]), i6, c.v[i]));
#pragma unroll
    for (int e = 0; e < 9; ++e)
        J[e] = fma2(m6, S[e], (e % 4) == 0 ? fma2(m23, N[e], one) : mul2(m23, N[e]));
}

// Tricubic Hermite value and gradient for two feet, streamed over the four x-lines of
// the cell (B = y corner, C = z corner).  row(B, C, lo, hi) must fill lo[a], hi[a] with
// plane a (0 phi, 1 x, 2 y, 3 z, 4 xy, 5 xz, 6 yz, 7 xyz) at the line's x = k and x = k+1
// corners, for both lanes.  phi is shifted by its value at the cell's first corner (line
// B = C = 0, x = k), as in hermite2d_pair.  The reduction order is x, then y, then z, as
// in the sum-factorised form of Sec. 2.3.
struct XRed2 { F2 P, Pd, Qy, Qyd, Qz, Qzd, Qyz, Qyzd; };

template <bool FIRST>
__device__ __forceinline__ XRed2 xreduce2(const Basis2 &bx, const F2 lo[8], const F2 hi[8], F2 base)
{
    XRed2 r;
    const F2 p1 = sub2(hi[0], base);
    if (FIRST) {  // lo[0] is the base itself
        r.P = hval2z(bx, p1, lo[1], hi[1]);
        r.Pd = hder2z(bx, p1, lo[1], hi[1]);
    } else {
        const F2 p0 = sub2(lo[0], base);
        r.P = hval2(bx, p0, p1, lo[1], hi[1]);
        r.Pd = hder2(bx, p0, p1, lo[1], hi[1]);
    }
    r.Qy = hval2(bx, lo[2], hi[2], lo[4], hi[4]);
    r.Qyd = hder2(bx, lo[2], hi[2], lo[4], hi[4]);
    r.Qz = hval2(bx, lo[3], hi[3], lo[5], hi[5]);
    r.Qzd = hder2(bx, lo[3], hi[3], lo[5], hi[5]);
    r.Qyz = hval2(bx, lo[6], hi[6], lo[7], hi[7]);
    r.Qyzd = hder2(bx, lo[6], hi[6], lo[7], hi[7]);
    return r;
}

template <class Row>
__device__ __forceinline__ void hermite3d_pair(const Basis2 &bx, const Basis2 &by, const Basis2 &bz,
                                               Row row, F2 &H, F2 g[3])
{
    F2 R[2], Rx[2], Ry[2], Rz[2], Rzx[2], Rzy[2];
    F2 base;
#pragma unroll
    for (int C = 0; C < 2; ++C) {
        XRed2 q[2];
#pragma unroll
        for (int B = 0; B < 2; ++B) {
            F2 lo[8], hi[8];
            row(B, C, lo, hi);
            if (B == 0 && C == 0) {
                base = lo[0];
                q[B] = xreduce2<true>(bx, lo, hi, base);
            } else {
                q[B] = xreduce2<false>(bx, lo, hi, base);
            }
        }
        R[C] = hval2(by, q[0].P, q[1].P, q[0].Qy, q[1].Qy);
        Ry[C] = hder2(by, q[0].P, q[1].P, q[0].Qy, q[1].Qy);
        Rx[C] = hval2(by, q[0].Pd, q[1].Pd, q[0].Qyd, q[1].Qyd);
        Rz[C] = hval2(by, q[0].Qz, q[1].Qz, q[0].Qyz, q[1].Qyz);
        Rzy[C] = hder2(by, q[0].Qz, q[1].Qz, q[0].Qyz, q[1].Qyz);
        Rzx[C] = hval2(by, q[0].Qzd, q[1].Qzd, q[0].Qyzd, q[1].Qyzd);
    }
    H = add2(base, hval2(bz, R[0], R[1], Rz[0], Rz[1]));
    g[2] = hder2(bz, R[0], R[1], Rz[0], Rz[1]);
    g[0] = hval2(bz, Rx[0], Rx[1], Rzx[0], Rzx[1]);
    g[1] = hval2(bz, Ry[0], Ry[1], Rzy[0], Rzy[1]);
}

}  // namespace gals
