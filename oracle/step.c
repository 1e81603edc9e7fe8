/*
 * step.c -- one step of the gradient-augmented CIR scheme, node by node.
 *
 * TEST INFRASTRUCTURE ONLY (the oracle): see gals_oracle.h.
 *
 * One step t -> t+dt (Sec. 4, in the superconsistent form of Sec. 5.1):
 *   1. for every grid node x_j, trace the characteristic back to time t and get
 *      the foot point and the Jacobian J of the approximate backward map (trace.c);
 *   2. evaluate the Hermite interpolant H of the cell the foot falls into
 *      (eq. p-cubic_interpolant), phi+ = H(foot), psi+ = J^T grad H(foot)
 *      (eq. superconsistency; J^T is the paper's grad of the foot map);
 *   3. rebuild the cross derivatives from the new gradients (Sec. 2.3, approach A),
 *      which completes the projection M = P A of Sec. 5.2.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - a foot outside the box is clamped per component into [lo, hi]; J is kept
 *     (Sec. 4.1 leaves outflow free; no configuration here has inflow data);
 *   - the cell is k = floor((foot-lo)/h) clamped to [0, n-2], xi = (foot - x_k)/h;
 *   - approach A at boundary nodes uses second-order one-sided differences;
 *   - the differenced gradient component: phi_xy <- d/dx psi_y, phi_xz <- d/dx psi_z,
 *     phi_yz <- d/dy psi_z, phi_xyz <- d/dx d/dy psi_z (the paper's printed pattern).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "gals_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

static int nplanes_of(int dim) { return dim == 1 ? 2 : (dim == 2 ? 4 : 8); }

/* plane holding derivative multi-index a (bit i = d/dx_i) */
static int plane_of(int dim, int a)
{
    if (dim == 1) return a;            /* phi, phi_x */
    if (dim == 2) return a;            /* phi, phi_x, phi_y, phi_xy */
    static const int map3[8] = {0, 1, 2, 4, 3, 5, 6, 7};
    /* a: 0 phi, 1 x, 2 y, 3 xy, 4 z, 5 xz, 6 yz, 7 xyz */
    return map3[a];
}

static long node_index(const orc_grid *g, int i, int j, int k)
{
    return ((long)k * g->n[1] + j) * g->n[0] + i;
}

static long total_nodes(const orc_grid *g)
{
    long N = 1;
    for (int d = 0; d < g->dim; ++d) N *= g->n[d];
    return N;
}

/* phi_xy-type value at vertex (u, w) of a 2D facet from its four edge-centre differences:
 * eu[0], eu[1] along the second axis at first-axis index 0, 1 and ew[0], ew[1] along the
 * first axis at second-axis index 0, 1 (Sec. 2.3 (B), weights 3/4 near, -1/4 opposite) */
static double cell_vertex(const double eu[2], const double ew[2], int u, int w)
{
    return 0.75 * (eu[u] + ew[w]) - 0.25 * (eu[1 - u] + ew[1 - w]);
}

void orc_cross_cell(int dim, const double *h, double *data)
{
    if (dim == 2) {
        /* psi_x differenced along y at x-index u; psi_y differenced along x at y-index w */
        double eu[2], ew[2];
        for (int u = 0; u < 2; ++u) eu[u] = (data[(u + 2) * 4 + 1] - data[u * 4 + 1]) / h[1];
        for (int w = 0; w < 2; ++w) ew[w] = (data[(1 + 2 * w) * 4 + 2] - data[(2 * w) * 4 + 2]) / h[0];
        for (int v = 0; v < 4; ++v) data[v * 4 + 3] = cell_vertex(eu, ew, v & 1, (v >> 1) & 1);
        return;
    }
    /* 3D: entry of corner (a, b, c) and derivative index d */
#define D3(a, b, c, d) data[((a) + 2 * (b) + 4 * (c)) * 8 + (d)]
    double xy[8], xz[8], yz[8], xyz[8];
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                double eu[2], ew[2];
                /* x-y facet at z-index c: psi_x along y at x = u, psi_y along x at y = w */
                for (int u = 0; u < 2; ++u) eu[u] = (D3(u, 1, c, 1) - D3(u, 0, c, 1)) / h[1];
                for (int w = 0; w < 2; ++w) ew[w] = (D3(1, w, c, 2) - D3(0, w, c, 2)) / h[0];
                xy[a + 2 * b + 4 * c] = cell_vertex(eu, ew, a, b);
                /* x-z facet at y-index b: psi_x along z at x = u, psi_z along x at z = w */
                for (int u = 0; u < 2; ++u) eu[u] = (D3(u, b, 1, 1) - D3(u, b, 0, 1)) / h[2];
                for (int w = 0; w < 2; ++w) ew[w] = (D3(1, b, w, 4) - D3(0, b, w, 4)) / h[0];
                xz[a + 2 * b + 4 * c] = cell_vertex(eu, ew, a, c);
                /* y-z facet at x-index a: psi_y along z at y = u, psi_z along y at z = w */
                for (int u = 0; u < 2; ++u) eu[u] = (D3(a, u, 1, 2) - D3(a, u, 0, 2)) / h[2];
                for (int w = 0; w < 2; ++w) ew[w] = (D3(a, 1, w, 4) - D3(a, 0, w, 4)) / h[1];
                yz[a + 2 * b + 4 * c] = cell_vertex(eu, ew, b, c);
                /* psi_z double difference over the x-y facet at z-index c */
                xyz[a + 2 * b + 4 * c] = (D3(1, 1, c, 4) - D3(0, 1, c, 4) - D3(1, 0, c, 4) + D3(0, 0, c, 4)) /
                                         (h[0] * h[1]);
            }
    for (int v = 0; v < 8; ++v) {
        data[v * 8 + 3] = xy[v];
        data[v * 8 + 5] = xz[v];
        data[v * 8 + 6] = yz[v];
        data[v * 8 + 7] = xyz[v];
    }
#undef D3
}

/* steps 2 of Sec. 4 at one foot point: the cell the foot falls into (clamped into the box,
 * floor, clamped to [0, n-2]), its 4^p data (approach B rebuilds the mixed entries per
 * cell), and the interpolant's value and gradient there (eq. p-cubic_interpolant) */
static void eval_at_foot(const orc_grid *g, int cross, const double *const *in,
                         const double foot[3], double *H, double gradH[3])
{
    int dim = g->dim;
    int cell[3] = {0, 0, 0};
    double xi[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
        double hi = g->lo[d] + (g->n[d] - 1) * g->h[d];
        double f = foot[d];
        if (f < g->lo[d]) f = g->lo[d];
        if (f > hi) f = hi;
        int c = (int)floor((f - g->lo[d]) / g->h[d]);
        if (c < 0) c = 0;
        if (c > g->n[d] - 2) c = g->n[d] - 2;
        cell[d] = c;
        xi[d] = (f - (g->lo[d] + c * g->h[d])) / g->h[d];
    }
    int np = 1 << dim;
    double data[64];
    for (int v = 0; v < np; ++v) {
        int ci = cell[0] + (v & 1);
        int cj = dim > 1 ? cell[1] + ((v >> 1) & 1) : 0;
        int ck = dim > 2 ? cell[2] + ((v >> 2) & 1) : 0;
        long nid = node_index(g, ci, cj, ck);
        for (int a = 0; a < np; ++a) data[v * np + a] = in[plane_of(dim, a)][nid];
    }
    if (cross == ORC_CROSS_CELL && dim >= 2) orc_cross_cell(dim, g->h, data);
    gradH[0] = gradH[1] = gradH[2] = 0.0;
    orc_hermite_cell(dim, data, g->h, xi, H, gradH);
}

/* superconsistent update (eq. superconsistency): psi+ = J^T grad H(foot) */
static void superconsistent_psi(int dim, const double J[9], const double gradH[3], double psi[3])
{
    for (int a = 0; a < dim; ++a) {
        double s = 0.0;
        for (int b = 0; b < dim; ++b) s += J[3 * b + a] * gradH[b];
        psi[a] = s;
    }
}

void orc_node_update(const orc_grid *g, const orc_velocity *vel, int trace, int cross,
                     double t, double dt, const double *const *in,
                     int i, int j, int k, double *phi, double psi[3])
{
    int dim = g->dim;
    int idx[3] = {i, j, k};
    double x[3] = {0, 0, 0}, foot[3], J[9];
    for (int d = 0; d < dim; ++d) x[d] = g->lo[d] + idx[d] * g->h[d];

    /* step 1: backward trace with Jacobian */
    orc_trace(trace, vel, dim, x, t, dt, foot, J);

    /* step 2: the interpolant of the foot's cell */
    double H, gradH[3];
    eval_at_foot(g, cross, in, foot, &H, gradH);

    *phi = H;
    if (trace == ORC_TRACE_HEUN_PSI) {
        /* CIR step 3 (Sec. 4): psi(tau) along the characteristic from (foot, t) to
         * (x, t+dt), d psi/d tau = -(grad v) . psi = -Dv^T psi, by Heun's method:
         * k1 = f(foot, t, psi0), k2 = f(x, t+dt, psi0 + dt k1), psi+ = psi0 + dt (k1+k2)/2.
         * The characteristic passes through the computed foot (not the clamped point). */
        double v0[3], D0[9], v1[3], D1[9], k1[3], ps[3], k2[3];
        orc_vel_eval(vel, dim, foot, t, v0, D0);
        orc_vel_eval(vel, dim, x, t + dt, v1, D1);
        for (int a = 0; a < dim; ++a) {
            double s = 0.0;
            for (int b = 0; b < dim; ++b) s += D0[3 * b + a] * gradH[b];
            k1[a] = -s;
        }
        for (int a = 0; a < dim; ++a) ps[a] = gradH[a] + dt * k1[a];
        for (int a = 0; a < dim; ++a) {
            double s = 0.0;
            for (int b = 0; b < dim; ++b) s += D1[3 * b + a] * ps[b];
            k2[a] = -s;
        }
        for (int a = 0; a < dim; ++a) psi[a] = gradH[a] + 0.5 * dt * (k1[a] + k2[a]);
        return;
    }
    superconsistent_psi(dim, J, gradH, psi);
}

void orc_step_given(const orc_grid *g, int cross, const double *const *in,
                    const double *const *disp, const double *const *jac, double *const *out,
                    int nthreads)
{
    int dim = g->dim;
    int nz = dim == 3 ? g->n[2] : 1, ny = dim >= 2 ? g->n[1] : 1;
    long rows = (long)nz * ny;
    (void)nthreads;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (long r = 0; r < rows; ++r) {
        int k = (int)(r / ny), j = (int)(r % ny);
        int idx[3] = {0, j, k};
        for (int i = 0; i < g->n[0]; ++i) {
            idx[0] = i;
            long id = node_index(g, i, j, k);
            double foot[3] = {0, 0, 0}, J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int d = 0; d < dim; ++d) foot[d] = g->lo[d] + idx[d] * g->h[d] + disp[d][id];
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) J[3 * a + b] = jac[dim * a + b][id];
            double H, gradH[3], psi[3];
            eval_at_foot(g, cross, in, foot, &H, gradH);
            superconsistent_psi(dim, J, gradH, psi);
            out[0][id] = H;
            for (int a = 0; a < dim; ++a) out[1 + a][id] = psi[a];
        }
    }
    if (dim == 1) return;
    if (cross == ORC_CROSS_ZERO || cross == ORC_CROSS_CELL) {
        long N = total_nodes(g);
        int first = dim == 2 ? 3 : 4, nc = dim == 2 ? 1 : 4;
        for (int c = 0; c < nc; ++c) memset(out[first + c], 0, N * sizeof(double));
        return;
    }
    orc_recon_cross(g, out);
}

/* stencil of the first-derivative approximation along one axis at index i:
 * central (u[i+1]-u[i-1])/(2h) inside, (-3u0+4u1-u2)/(2h) and
 * (3u_{n-1}-4u_{n-2}+u_{n-3})/(2h) at the two ends */
static void deriv_stencil(int i, int n, double h, int idx[3], double w[3])
{
    if (i == 0) {
        idx[0] = 0; idx[1] = 1; idx[2] = 2;
        w[0] = -3.0 / (2.0 * h); w[1] = 4.0 / (2.0 * h); w[2] = -1.0 / (2.0 * h);
    } else if (i == n - 1) {
        idx[0] = n - 1; idx[1] = n - 2; idx[2] = n - 3;
        w[0] = 3.0 / (2.0 * h); w[1] = -4.0 / (2.0 * h); w[2] = 1.0 / (2.0 * h);
    } else {
        idx[0] = i + 1; idx[1] = i - 1; idx[2] = i;
        w[0] = 1.0 / (2.0 * h); w[1] = -1.0 / (2.0 * h); w[2] = 0.0;
    }
}

/* cross derivatives of node (i,j,k) from gradient values supplied by `get`
 * (plane index, node) -- shared by the full-grid and the sampled versions */
typedef double (*getter_fn)(void *ctx, int plane, int i, int j, int k);

static void cross_at(const orc_grid *g, getter_fn get, void *ctx, int i, int j, int k,
                     double *cross)
{
    int ix[3], iy[3];
    double wx[3], wy[3];
    deriv_stencil(i, g->n[0], g->h[0], ix, wx);
    deriv_stencil(j, g->n[1], g->h[1], iy, wy);
    if (g->dim == 2) {
        double s = 0.0; /* phi_xy = d/dx psi_y */
        for (int a = 0; a < 3; ++a) s += wx[a] * get(ctx, 2, ix[a], j, 0);
        cross[0] = s;
        return;
    }
    /* 3D: phi_xy = Dx psi_y, phi_xz = Dx psi_z, phi_yz = Dy psi_z, phi_xyz = Dx Dy psi_z */
    double sxy = 0.0, sxz = 0.0, syz = 0.0, sxyz = 0.0;
    for (int a = 0; a < 3; ++a) {
        sxy += wx[a] * get(ctx, 2, ix[a], j, k);
        sxz += wx[a] * get(ctx, 3, ix[a], j, k);
        syz += wy[a] * get(ctx, 3, i, iy[a], k);
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            sxyz += wx[a] * wy[b] * get(ctx, 3, ix[a], iy[b], k);
    cross[0] = sxy; cross[1] = sxz; cross[2] = syz; cross[3] = sxyz;
}

typedef struct { const orc_grid *g; double *const *planes; } plane_ctx;

static double get_plane(void *vctx, int plane, int i, int j, int k)
{
    plane_ctx *c = (plane_ctx *)vctx;
    return c->planes[plane][node_index(c->g, i, j, k)];
}

void orc_recon_cross(const orc_grid *g, double *const *planes)
{
    if (g->dim == 1) return;
    int ncross = g->dim == 2 ? 1 : 4;
    int first = g->dim == 2 ? 3 : 4;
    plane_ctx ctx = {g, planes};
    int nz = g->dim == 3 ? g->n[2] : 1;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                double cr[4];
                cross_at(g, get_plane, &ctx, i, j, k, cr);
                long id = node_index(g, i, j, k);
                for (int c = 0; c < ncross; ++c) planes[first + c][id] = cr[c];
            }
}

void orc_step(const orc_grid *g, const orc_velocity *vel, int trace, int cross,
              double t, double dt, const double *const *in, double *const *out,
              int nthreads)
{
    int dim = g->dim;
    int nz = dim == 3 ? g->n[2] : 1, ny = dim >= 2 ? g->n[1] : 1;
    long rows = (long)nz * ny;
    (void)nthreads;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (long r = 0; r < rows; ++r) {
        int k = (int)(r / ny), j = (int)(r % ny);
        for (int i = 0; i < g->n[0]; ++i) {
            double phi, psi[3];
            orc_node_update(g, vel, trace, cross, t, dt, in, i, j, k, &phi, psi);
            long id = node_index(g, i, j, k);
            out[0][id] = phi;
            for (int a = 0; a < dim; ++a) out[1 + a][id] = psi[a];
        }
    }
    if (dim == 1) return;
    if (cross == ORC_CROSS_ZERO || cross == ORC_CROSS_CELL) {
        long N = total_nodes(g);
        int first = dim == 2 ? 3 : 4, nc = dim == 2 ? 1 : 4;
        for (int c = 0; c < nc; ++c) memset(out[first + c], 0, N * sizeof(double));
        return;
    }
    orc_recon_cross(g, out);
}

/* sampled version: recompute the node updates a node's cross stencil needs */
typedef struct {
    const orc_grid *g; const orc_velocity *vel; int trace; double t, dt;
    const double *const *in;
} upd_ctx;

static double get_updated(void *vctx, int plane, int i, int j, int k)
{
    upd_ctx *c = (upd_ctx *)vctx;
    double phi, psi[3];
    orc_node_update(c->g, c->vel, c->trace, ORC_CROSS_CENTRAL, c->t, c->dt, c->in, i, j, k, &phi, psi);
    return plane == 0 ? phi : psi[plane - 1];
}

void orc_step_nodes(const orc_grid *g, const orc_velocity *vel, int trace, int cross,
                    double t, double dt, const double *const *in, long nsel,
                    const long *sel, double *outv, int nthreads)
{
    int dim = g->dim, np = nplanes_of(dim);
    (void)nthreads;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (long s = 0; s < nsel; ++s) {
        long id = sel[s];
        int i = (int)(id % g->n[0]);
        int j = dim >= 2 ? (int)((id / g->n[0]) % g->n[1]) : 0;
        int k = dim == 3 ? (int)(id / ((long)g->n[0] * g->n[1])) : 0;
        double phi, psi[3];
        orc_node_update(g, vel, trace, cross, t, dt, in, i, j, k, &phi, psi);
        double *o = outv + s * np;
        o[0] = phi;
        for (int a = 0; a < dim; ++a) o[1 + a] = psi[a];
        if (dim == 1) continue;
        int first = dim == 2 ? 3 : 4, nc = dim == 2 ? 1 : 4;
        double cr[4] = {0, 0, 0, 0};
        if (cross == ORC_CROSS_CENTRAL) {
            upd_ctx ctx = {g, vel, trace, t, dt, in};
            cross_at(g, get_updated, &ctx, i, j, k, cr);
        }
        for (int c = 0; c < nc; ++c) o[first + c] = cr[c];
    }
}

void orc_run(const orc_grid *g, const orc_velocity *vel, int trace, int cross,
             double t0, double dt, int nsteps, double *const *state,
             double *const *scratch, int nthreads)
{
    int np = nplanes_of(g->dim);
    long N = total_nodes(g);
    double *a[8], *b[8];
    for (int p = 0; p < np; ++p) { a[p] = state[p]; b[p] = scratch[p]; }
    for (int s = 0; s < nsteps; ++s) {
        orc_step(g, vel, trace, cross, t0 + s * dt, dt, (const double *const *)a, b,
                 nthreads);
        for (int p = 0; p < np; ++p) { double *tmp = a[p]; a[p] = b[p]; b[p] = tmp; }
    }
    if (a[0] != state[0])
        for (int p = 0; p < np; ++p) memcpy(state[p], a[p], N * sizeof(double));
}

/* band of the outermost axis (rows j in [b0,b1) in 2D, slices k in [b0,b1) in 3D): the
 * approach-A stencils difference along x (and y in 3D) only, so a band is updated
 * exactly from the old state alone.  out planes hold the band's nodes contiguously. */
typedef struct { const orc_grid *g; double *const *planes; int b0; } band_ctx;

static double get_band(void *vctx, int plane, int i, int j, int k)
{
    band_ctx *c = (band_ctx *)vctx;
    const orc_grid *g = c->g;
    long id = g->dim == 2 ? (long)(j - c->b0) * g->n[0] + i
                          : ((long)(k - c->b0) * g->n[1] + j) * g->n[0] + i;
    return c->planes[plane][id];
}

void orc_step_band(const orc_grid *g, const orc_velocity *vel, int trace, int cross,
                   double t, double dt, const double *const *in, int b0, int b1,
                   double *const *out, int nthreads)
{
    int dim = g->dim;
    int inner = dim == 2 ? 1 : g->n[1];
    long lines = (long)(b1 - b0) * inner;
    (void)nthreads;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (long r = 0; r < lines; ++r) {
        int outer = b0 + (int)(r / inner), jj = (int)(r % inner);
        int j = dim == 2 ? outer : jj, k = dim == 2 ? 0 : outer;
        for (int i = 0; i < g->n[0]; ++i) {
            double phi, psi[3];
            orc_node_update(g, vel, trace, cross, t, dt, in, i, j, k, &phi, psi);
            long id = r * g->n[0] + i;
            out[0][id] = phi;
            for (int a = 0; a < dim; ++a) out[1 + a][id] = psi[a];
        }
    }
    int first = dim == 2 ? 3 : 4, nc = dim == 2 ? 1 : 4;
    band_ctx ctx = {g, out, b0};
    for (long r = 0; r < lines; ++r) {
        int outer = b0 + (int)(r / inner), jj = (int)(r % inner);
        int j = dim == 2 ? outer : jj, k = dim == 2 ? 0 : outer;
        for (int i = 0; i < g->n[0]; ++i) {
            double cr[4] = {0, 0, 0, 0};
            if (cross == ORC_CROSS_CENTRAL) cross_at(g, get_band, &ctx, i, j, k, cr);
            long id = r * g->n[0] + i;
            for (int c = 0; c < nc; ++c) out[first + c][id] = cr[c];
        }
    }
}
