// step2d_tile.cuh -- one 2D GALS step over one tile of nodes, shared by the single-grid
// kernel (step2d.cu) and the batched kernels (batch2d.cu).
//
// Per grid node (Sec. 4, steps 1-2 in the superconsistent form of Sec. 5.1):
//   trace back with the Jacobian -> locate the foot cell -> gather the 4 corners x 4 data
//   -> bicubic Hermite value and gradient -> phi+ = H, psi+ = J^T grad H,
// then (Sec. 2.3, approach A) phi_xy+ = d/dx psi_y+ by central differences.
//
// A block of 128 threads owns a tile of 128 columns x TY rows; each thread walks its
// column two rows at a time in paired FP32 arithmetic (gals_pair.cuh).  The input tile
// (all state planes, halo 4 columns x HYV rows: 1 in the single-grid kernel, 2 in the
// batched ones) is staged into shared memory by one TMA copy;
// feet whose cell leaves the staged tile read global memory instead.  With WC the new
// psi_y of the tile plus one halo column on each side (2 extra node updates per 128 per
// row) stays in shared memory and phi_xy+ is written by the same kernel: the halo columns
// are traced after the tile's own, or (overlapped tiles, the single-grid kernel) tiles of
// 126 columns overlap by one column on each side and the halo is traced with the rest.
#pragma once

#include "gals_internal.h"
#include "gals_pair.cuh"
#include "tma.cuh"

namespace gals {
namespace t2 {

constexpr int TX = 128;               // output tile columns (one thread each)
constexpr int HX = 4, HY = 2;         // input halo (x rounded to 16 bytes for TMA)
constexpr int TW = TX + 2 * HX;

template <int TY, int HYV = HY, int W = TW> struct Geo {
    static constexpr int TH = TY + 2 * HYV;
    static constexpr int PS = W * TH;  // floats per staged plane (W columns a row)
    static constexpr int bytes(int np) { return np * PS * 4; }
};

// static shared memory of a tile step (the staged tile itself is dynamic)
template <int TY, int WC> struct Smem {
    float psy[WC ? TY : 1][TX + 3];   // psi_y+ of columns x0-2 .. x0+TX
    StageCoefPair scp;
    float fsum[12][TY];               // FOURIER2D stage 1: row sums of the tile's rows
    uint64_t bar;
};

// FOURIER2D at grid nodes (stage 1, t + dt).  Psi = sum_kl A_kl s_k(x) s_l(y) separates:
// the sums over l depend on the row only, so the block computes them once per tile row
// (FRow, in shared memory), and each thread keeps its column's s_k(x), c_k(x) (FCol); a
// node then costs the four-term sums over k.  The arithmetic (multiple angles by the
// Chebyshev recurrences, the order of every sum) is that of vel2d_pair, lane by lane.
struct FCol { float s[5], c[5]; };

__device__ __forceinline__ void multiple_angles(float s1, float c1, float s[5], float c[5])
{
    s[1] = s1;
    c[1] = c1;
    s[2] = 2.f * __fmul_rn(s1, c1);
    c[2] = __fmaf_rn(-2.f, __fmul_rn(s1, s1), 1.f);
    s[3] = __fmaf_rn(s[2], c1, __fmul_rn(c[2], s1));
    c[3] = __fmaf_rn(c[2], c1, -__fmul_rn(s[2], s1));
    s[4] = 2.f * __fmul_rn(s[2], c[2]);
    c[4] = __fmaf_rn(-2.f, __fmul_rn(s[2], s[2]), 1.f);
}

__device__ __forceinline__ FCol fourier_col(float x)
{
    FCol f;
    float s1, c1;
    sincospi_f(x, &s1, &c1);
    multiple_angles(s1, c1, f.s, f.c);
    return f;
}

// Row sums of row y for stage-1 tables: Ux_k = sum_l Al_kl c_l(y), Vx_k = sum_l A_kl s_l(y),
// W_k = sum_l All_kl s_l(y), into out[k-1], out[4+k-1], out[8+k-1] (k = 1..4).
__device__ __forceinline__ void fourier_row(const StageCoef &sc, float y, int k, float &ux, float &vx,
                                            float &w)
{
    float sy1, cy1, sy[5], cy[5];
    sincospi_f(y, &sy1, &cy1);
    multiple_angles(sy1, cy1, sy, cy);
    ux = 0.f; vx = 0.f; w = 0.f;
#pragma unroll
    for (int l = 1; l <= 4; ++l) {
        const int kl = (k - 1) * 4 + (l - 1);
        ux = __fmaf_rn(sc.Al[0][kl], cy[l], ux);
        vx = __fmaf_rn(sc.A[0][kl], sy[l], vx);
        w = __fmaf_rn(sc.All[0][kl], sy[l], w);
    }
}

// v, Dv at the two nodes (rows r, r+1 of the tile) of a thread's column.
template <int TY>
__device__ __forceinline__ V2p fourier_stage1_pair(const FCol &f, const float (*fsum)[TY], int r)
{
    F2 u = bc(0.f), v = bc(0.f), d00 = bc(0.f), d01 = bc(0.f), d10 = bc(0.f);
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        const F2 Ux = make_float2(fsum[k - 1][r], fsum[k - 1][r + 1]);
        const F2 Vx = make_float2(fsum[4 + k - 1][r], fsum[4 + k - 1][r + 1]);
        const F2 W = make_float2(fsum[8 + k - 1][r], fsum[8 + k - 1][r + 1]);
        const float kp = (float)k * kPi;
        const F2 sk = bc(f.s[k]), ck = bc(f.c[k]);
        u = fma2(neg2(sk), Ux, u);
        v = fma2(mul2(bc(kp), ck), Vx, v);
        d00 = fma2(mul2(bc(-kp), ck), Ux, d00);
        d01 = fma2(sk, W, d01);
        d10 = fma2(mul2(bc(-kp * kp), sk), Vx, d10);
    }
    V2p rr;
    rr.u = u; rr.v = v; rr.d00 = d00; rr.d01 = d01; rr.d10 = d10; rr.d11 = neg2(d00);
    return rr;
}

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

// Separable factors of the single-vortex field on a grid line, per lane: A = sin a,
// B = cos a for a = 2 pi (s - 1/2), and S = sin^2(pi s) = (1 + B)/2 (see sincos_turn).
struct Sep2 { F2 S, A, B; };

__device__ __forceinline__ Sep2 sep_factors2(F2 s)
{
    Sep2 f;
    sincos_turn2(s, f.A, f.B);
    f.S = fma2(f.B, bc(0.5f), bc(0.5f));
    return f;
}

// A column's factors of the single vortex at t + dt (stage coefficient c), constants
// folded in: u = ku Ay, v = kv Sy, du/dx = k00 Ay, du/dy = k01 By, dv/dx = k10 Sy.
struct VCol { float ku, kv, k00, k01, k10; };

__device__ __forceinline__ VCol vortex_col(float x, float c)
{
    float A, B;
    sincos_turn(x, &A, &B);
    const float S = __fmaf_rn(B, 0.5f, 0.5f), cp = c * kPi;
    return VCol{c * S, -c * A, -cp * A, (2.f * cp) * S, (-2.f * cp) * B};
}

// v(x, t+dt) at two nodes of one column; the single vortex uses the column factors cx
// (fixed per thread) and the row factors ry.
template <int VK>
__device__ __forceinline__ V2p stage1_pair(const VelParams &vp, const StageCoef &sc,
                                           const StageCoefPair *scp, F2 x, F2 y, const VCol &cx,
                                           const Sep2 &ry)
{
    if (VK == VK_VORTEX2D) {
        V2p r;
        r.u = mul2(bc(cx.ku), ry.A);
        r.v = mul2(bc(cx.kv), ry.S);
        r.d00 = mul2(bc(cx.k00), ry.A);
        r.d01 = mul2(bc(cx.k01), ry.B);
        r.d10 = mul2(bc(cx.k10), ry.S);
        r.d11 = neg2(r.d00);
        return r;
    }
    return vel2d_pair<VK>(vp, sc, scp, 0, x, y);
}

// A state value read from global memory: through the read-only path, or (COH) through
// L2 only, for a persistent launch whose earlier steps wrote the buffer in the same launch.
template <bool COH>
__device__ __forceinline__ float ld_state(const float *p)
{
    return COH ? __ldcg(p) : __ldg(p);
}

// The 4 corners x 4 data of the cell (k, l) for one node, from the staged tile when the
// cell (and, for COMPACT, its psi_y window k-1..k+2) lies inside it, else from global
// memory (feet farther than the halo: CFL well above 1).  The staged tile is W columns
// wide from column x0 - HX (SX: from column x0), TY + 2 HYV rows from row y0 - HYV.
template <int TY, int CR, int HYV = HY, bool COH = false, int W = TW, bool SX = false>
__device__ __forceinline__ void gather_lane(const float *__restrict__ in, const Geom &g,
                                            const float *__restrict__ tile, int x0, int y0, int k,
                                            int l, float c[4][4])
{
    constexpr int TH = Geo<TY, HYV, W>::TH, PS = Geo<TY, HYV, W>::PS;
    const int tx = SX ? k - x0 : k - x0 + HX, ty = l - y0 + HYV;
    if (tx >= 1 && tx <= W - 3 && ty >= 0 && ty <= TH - 2) {
#ifdef GALS_CHECKED
        // every read below is t[o + a PS] with -1 <= o <= W + 2, a < 4
        const float *t = tile + GALS_CHK(g, ty * W + tx, PS - W - 2);
#else
        const float *t = tile + ty * W + tx;
#endif
#pragma unroll
        for (int B = 0; B < 2; ++B) {
#pragma unroll
            for (int A = 0; A < 2; ++A) {
                const int v = A + 2 * B, o = B * W + A;
                c[v][0] = t[o];
                c[v][1] = t[PS + o];
                c[v][2] = t[2 * PS + o];
                if (CR == CROSS_PLANE) c[v][3] = t[3 * PS + o];
            }
            if (CR == CROSS_RECON) {
                const float w[4] = {t[2 * PS + B * W - 1], c[2 * B][2], c[2 * B + 1][2],
                                    t[2 * PS + B * W + 2]};
                c[2 * B][3] = cross_from_window<0>(w, k, g.n0, g.i2h0);
                c[2 * B + 1][3] = cross_from_window<1>(w, k + 1, g.n0, g.i2h0);
            }
        }
        if (CR == CROSS_CELL) cross_cell2d(c, g.ih0, g.ih1);
        return;
    }
    const float *Pphi = in, *Ppx = in + g.plane, *Ppy = in + 2 * g.plane;
#pragma unroll
    for (int B = 0; B < 2; ++B) {
        // the reads below lie in r - 1 .. r + 2 of a plane, inside row l + B
#ifdef GALS_CHECKED
        // the whole window: the cell's first column k <= n0 - 2 and the row exist (a read
        // past the row's end would wrap into the next row unseen by the index test below)
        (void)GALS_CHK(g, k, g.n0 - 1);
        (void)GALS_CHK(g, l + B, g.n1);
#endif
        const int r = GALS_CHK(g, (l + B) * g.pitch + k, plane_extent(g));
#pragma unroll
        for (int A = 0; A < 2; ++A) {
            const int v = A + 2 * B;
            c[v][0] = ld_state<COH>(Pphi + r + A);
            c[v][1] = ld_state<COH>(Ppx + r + A);
            c[v][2] = ld_state<COH>(Ppy + r + A);
            if (CR == CROSS_PLANE) c[v][3] = ld_state<COH>(in + 3 * g.plane + r + A);
        }
        if (CR == CROSS_RECON) {
            const float w[4] = {ld_state<COH>(Ppy + r - (k > 0 ? 1 : 0)), c[2 * B][2], c[2 * B + 1][2],
                                ld_state<COH>(Ppy + r + (k + 2 < g.n0 ? 2 : 1))};
            c[2 * B][3] = cross_from_window<0>(w, k, g.n0, g.i2h0);
            c[2 * B + 1][3] = cross_from_window<1>(w, k + 1, g.n0, g.i2h0);
        }
    }
    if (CR == CROSS_CELL) cross_cell2d(c, g.ih0, g.ih1);
}

// Update of two nodes (i0, j0) and (i1, j1): phi+, psi_x+, psi_y+ per lane; the staged
// tile (W columns from column x0 - HX; SX: from column x0) has HYV halo rows.
template <int TY, int TR, int VK, int CR, int HYV = HY, bool COH = false, int W = TW, bool SX = false>
__device__ __forceinline__ void node2d_pair(const float *__restrict__ in, const Geom &g,
                                            const float *__restrict__ tile, int x0, int y0,
                                            const VelParams &vp, const StageCoef &sc,
                                            const StageCoefPair *scp, float dt, int i0, int j0,
                                            int i1, int j1, F2 x, F2 y, const VCol &cx,
                                            const Sep2 &ry, F2 &phi, F2 &px, F2 &py,
                                            const V2p *a1 = nullptr)
{
    F2 dx, dy, J[4];
    if (TR == TR_GIVEN) {
        // foot displacement and Jacobian precomputed for this step (learned surrogate)
        const int64_t o0 = (int64_t)j0 * g.pitch + i0, o1 = (int64_t)j1 * g.pitch + i1;
        const float *tb = vp.given;
        const int64_t P = vp.given_plane;
        dx = make_float2(__ldg(tb + o0), __ldg(tb + o1));
        dy = make_float2(__ldg(tb + P + o0), __ldg(tb + P + o1));
#pragma unroll
        for (int e = 0; e < 4; ++e) J[e] = make_float2(__ldg(tb + (2 + e) * P + o0), __ldg(tb + (2 + e) * P + o1));
    } else if (VK == VK_FOURIER2D && a1 != nullptr) {
        trace2d_pair<TR, VK>(*a1, vp, sc, scp, x, y, dt, dx, dy, J);
    } else {
        trace2d_pair<TR, VK>(stage1_pair<VK>(vp, sc, scp, x, y, cx, ry), vp, sc, scp, x, y, dt, dx,
                             dy, J);
    }
    (void)J;
    int k0, l0, k1, l1;
    F2 xi, eta;
    locate_pair(i0, i1, mul2(dx, bc(g.ih0)), g.n0, k0, k1, xi);
    locate_pair(j0, j1, mul2(dy, bc(g.ih1)), g.n1, l0, l1, eta);

    float c0[4][4], c1[4][4];
    gather_lane<TY, CR, HYV, COH, W, SX>(in, g, tile, x0, y0, k0, l0, c0);
    gather_lane<TY, CR, HYV, COH, W, SX>(in, g, tile, x0, y0, k1, l1, c1);
    F2 c[4][4];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int a = 0; a < 4; ++a) c[v][a] = make_float2(c0[v][a], c1[v][a]);

    const Basis2 bx = basis_pair(xi, g.h0, g.ih0);
    const Basis2 by = basis_pair(eta, g.h1, g.ih1);
    F2 H, Hx, Hy;
    hermite2d_pair(c, bx, by, H, Hx, Hy);
    phi = H;
    if (TR == TR_HEUN) {
        // CIR gradient update (Sec. 4): Dv at the foot at time t (stage coefficients 1),
        // Dv at the node at t + dt (the trace's first stage, evaluated again)
        const V2p Df = vel2d_pair<VK>(vp, sc, scp, 1, add2(x, dx), add2(y, dy));
        const V2p Dn = (VK == VK_FOURIER2D && a1 != nullptr) ? *a1 : stage1_pair<VK>(vp, sc, scp, x, y, cx, ry);
        heun_psi2(Df, Dn, dt, Hx, Hy, px, py);
        return;
    }
    px = fma2(J[0], Hx, mul2(J[2], Hy));  // (J^T grad H)_x
    py = fma2(J[1], Hx, mul2(J[3], Hy));  // (J^T grad H)_y
}

// One tile step: origin (x0, y0).  `tile` is the dynamic shared buffer for the staged
// input (W columns), `sm` the static part; the barrier sm.bar must be initialised (count 1)
// and `parity` is the phase this tile's copy completes.  COH: global-memory gathers go
// through L2 (see ld_state).  after_issue() runs on thread 0 right after it issued the copy.  Returns false (after recording
// kErrTmaTimeout) if the staged copy did not arrive within the wait limit.
// Must be called by all TX threads of the block.
//
// OV (overlapped tiles, WC only): the block owns the TX - 2 columns x0 .. x0 + TX - 3 and
// its threads walk the columns x0 - 1 .. x0 + TX - 2, so that the two halo columns of the
// phi_xy stencil are traced in the main loop by the first and last thread instead of in a
// separate pass after it (those two also store their phi+, psi+, identical to the
// neighbouring tiles' own, see st_out; they write no phi_xy+).  The staged tile then starts
// at the 16-byte boundary at or below x0 - 1 - HX, and W = TW + 4 keeps at least HX staged
// columns on both sides of the walked ones.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// Output store of the overlapped tiles: the halo lanes store the same bits as the lanes of
// the neighbouring tile that own the column, so every output store is a strong (relaxed,
// GPU-scope) one and the duplicates do not race.
__device__ __forceinline__ void st_out(float *p, float v)
{
    asm("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v));
}

template <int TY, int TR, int VK, int CR, int WC, int HYV = HY, bool COH = false, int W = TW,
          bool OV = false, class Hook = NoHook>
__device__ __forceinline__ bool tile_step2d(const float *__restrict__ in, float *__restrict__ out,
                                            const Geom &g, const VelParams &vp,
                                            const StageCoef *__restrict__ coef, float dt,
                                            const CUtensorMap *tmap, int *__restrict__ err,
                                            int x0, int y0, float *tile, Smem<TY, WC> &sm,
                                            uint32_t parity, Hook after_issue = Hook())
{
    static_assert(!OV || (WC && W >= TW + 4), "overlapped tiles carry the phi_xy halo");
    auto &psy = sm.psy;
    auto &scp_s = sm.scp;
    const int tid = threadIdx.x;
    constexpr int NP = CR == CROSS_PLANE ? 4 : 3;
    // first staged column (a multiple of 4: TMA rows start on 16-byte boundaries)
    const int sx0 = OV ? ((x0 - 1 - HX) & ~3) : x0 - HX;
    const int gx0 = OV ? sx0 : x0;  // gathers index the staged tile from sx0 (OV) or x0 - HX

    // stage the input tile (all planes, halo HX x HY) with one TMA copy
#ifdef GALS_CHECKED
    const uint32_t polls = g.wait_polls;
    if (tid == 0 && !g.skip_copy) {  // test hook: a copy never issued, a wait that runs out
#else
    constexpr uint32_t polls = kWaitLimit;
    if (tid == 0) {
#endif
        mbar_arrive_expect_tx(&sm.bar, Geo<TY, HYV, W>::bytes(NP));
        tma_load_3d(tile, tmap, sx0, y0 - HYV, 0, &sm.bar);
        after_issue();  // thread 0's own work while the copy is in flight
    }
    const StageCoef &sc = *coef;
    if (VK == VK_FOURIER2D) {
        // duplicate the step's 4x4 tables into float2 pairs in shared memory
        for (int e = tid; e < 3 * 3 * 16; e += TX) {
            const int tab = e / 48, rest = e % 48, st = rest / 16, kl = rest % 16;
            const float v = tab == 0 ? __ldg(&coef->A[st][kl])
                          : (tab == 1 ? __ldg(&coef->Al[st][kl]) : __ldg(&coef->All[st][kl]));
            F2 *dst = tab == 0 ? &scp_s.A[st][kl] : (tab == 1 ? &scp_s.Al[st][kl] : &scp_s.All[st][kl]);
            *dst = bc(v);
        }
        __syncthreads();
    }
    const StageCoefPair *scp = &scp_s;
    (void)psy;
    if (VK == VK_FOURIER2D) {
        // stage-1 row sums of the tile's rows (rows past the grid repeat the last one)
        for (int e = tid; e < TY * 4; e += TX) {
            const int r = e >> 2, k = (e & 3) + 1;
            const float yr = g.lo1 + (float)min(y0 + r, g.n1 - 1) * g.h1;
            float ux, vx, w;
            fourier_row(sc, yr, k, ux, vx, w);
            sm.fsum[k - 1][r] = ux;
            sm.fsum[4 + k - 1][r] = vx;
            sm.fsum[8 + k - 1][r] = w;
        }
    }

    const int i = OV ? x0 - 1 + tid : x0 + tid;
    const bool own = !OV || (tid >= 1 && tid <= TX - 2);  // a column of this tile's output
    constexpr int PQ = OV ? 1 : 2;                          // psy index of column i: i - x0 + 2
    const int rows = min(TY, g.n1 - y0);
    const float xs = g.lo0 + (float)i * g.h0;
    const F2 x = bc(xs);
    const VCol cx = (VK == VK_VORTEX2D) ? vortex_col(xs, sc.mod[0]) : VCol{0.f, 0.f, 0.f, 0.f, 0.f};
    FCol fcol;
    if (VK == VK_FOURIER2D) fcol = fourier_col(xs);

    // bounded wait for the tile; a block-uniform verdict so no thread is left at a barrier
    if (!mbar_wait_block(&sm.bar, parity, polls)) {
        if (tid == 0) {
            atomicExch(err, kErrTmaTimeout);
            mbar_wait_bounded(&sm.bar, parity, polls);  // let a late copy land before giving up
        }
        return false;
    }

    if ((!OV || i >= 0) && i < g.n0) {
        for (int r = 0; r < rows; r += 2) {
            const int j0 = y0 + r, j1 = min(j0 + 1, g.n1 - 1);
            const F2 y = make_float2(g.lo1 + (float)j0 * g.h1, g.lo1 + (float)j1 * g.h1);
            const Sep2 ry = (VK == VK_VORTEX2D) ? sep_factors2(y) : Sep2{bc(0.f), bc(0.f), bc(0.f)};
            F2 phi, px, py;
            if (VK == VK_FOURIER2D && TR != TR_GIVEN) {
                const V2p a1 = fourier_stage1_pair<TY>(fcol, sm.fsum, r);
                node2d_pair<TY, TR, VK, CR, HYV, COH, W, OV>(in, g, tile, gx0, y0, vp, sc, scp, dt, i, j0, i,
                                                   j1, x, y, cx, ry, phi, px, py, &a1);
            } else {
                node2d_pair<TY, TR, VK, CR, HYV, COH, W, OV>(in, g, tile, gx0, y0, vp, sc, scp, dt, i, j0, i,
                                                   j1, x, y, cx, ry, phi, px, py);
            }
            const int o = GALS_CHK(g, j0 * g.pitch + i, plane_extent(g));
            if (OV) {
                st_out(out + o, phi.x);
                st_out(out + g.plane + o, px.x);
                st_out(out + 2 * g.plane + o, py.x);
            } else {
                out[o] = phi.x;
                out[g.plane + o] = px.x;
                out[2 * g.plane + o] = py.x;
            }
            if (WC) psy[WC ? r : 0][tid + PQ] = py.x;
            if (r + 1 < rows) {
                const int o1 = GALS_CHK(g, o + g.pitch, plane_extent(g));
                if (OV) {
                    st_out(out + o1, phi.y);
                    st_out(out + g.plane + o1, px.y);
                    st_out(out + 2 * g.plane + o1, py.y);
                } else {
                    out[o1] = phi.y;
                    out[g.plane + o1] = px.y;
                    out[2 * g.plane + o1] = py.y;
                }
                if (WC) psy[WC ? r + 1 : 0][tid + PQ] = py.y;
            }
        }
    }
    if (WC) {
        // halo columns of psi_y+: x0-1 and x0+TX (x0-2 too when the tile is one column
        // wide, for the one-sided stencil of the last node); two rows per task
        const int width = min(OV ? TX - 2 : TX, g.n0 - x0);
        const int npairs = (rows + 1) / 2;
        for (int hh = tid; hh < 3 * npairs; hh += TX) {
            const int rp = hh / 3, which = hh % 3;
            const int ih = which == 0 ? x0 - 2 : (which == 1 ? x0 - 1 : x0 + TX);
            const bool need = which == 0 ? (width == 1 && ih >= 0) : (!OV && ih >= 0 && ih < g.n0);
            if (!need) continue;
            const int r = 2 * rp, j0 = y0 + r, j1 = min(j0 + 1, g.n1 - 1);
            const F2 xh = bc(g.lo0 + (float)ih * g.h0);
            const F2 y = make_float2(g.lo1 + (float)j0 * g.h1, g.lo1 + (float)j1 * g.h1);
            const VCol cxh = (VK == VK_VORTEX2D) ? vortex_col(xh.x, sc.mod[0]) : VCol{0.f, 0.f, 0.f, 0.f, 0.f};
            const Sep2 ry = (VK == VK_VORTEX2D) ? sep_factors2(y) : Sep2{bc(0.f), bc(0.f), bc(0.f)};
            F2 phi, px, py;
            node2d_pair<TY, TR, VK, CR, HYV, COH, W, OV>(in, g, tile, gx0, y0, vp, sc, scp, dt, ih, j0, ih, j1,
                                               xh, y, cxh, ry, phi, px, py);
            psy[WC ? r : 0][GALS_CHK(g, ih - x0 + 2, TX + 3)] = py.x;
            if (r + 1 < rows) psy[WC ? r + 1 : 0][GALS_CHK(g, ih - x0 + 2, TX + 3)] = py.y;
        }
        __syncthreads();
        if (own && i < g.n0) {
            for (int r = 0; r < rows; ++r) {
                const float *line = psy[WC ? r : 0];
                const float v = dline(i, g.n0, g.i2h0, [&](int q) { return line[q - x0 + 2]; });
                out[GALS_CHK(g, 3 * g.plane + (y0 + r) * g.pitch + i, 4 * g.plane)] = v;
            }
        }
    }
    return true;
}

}  // namespace t2
}  // namespace gals
