/*
 * diag.c -- error norms and interface measures, in FP64 plain loops.
 *
 * TEST INFRASTRUCTURE ONLY (the oracle): see gals_oracle.h.
 *
 *   e_max (eq. maximum_norm, Sec. 6.1): max_j |a_j - b_j| over the nodes.
 *   Area / volume of {phi < 0} (the volume-loss tables of Sec. 6.2.6; the paper
 *   does not say how it measured volume): q^p cell-centred sample points per cell,
 *   xi = (s + 1/2)/q, each counted where the cell's Hermite interpolant is negative.
 *   Interface error: the measure of the symmetric difference of {H_a < 0} and
 *   {H_b < 0} with the same samples (an L1 shape error of the zero contours).
 */
#include <math.h>
#include "gals_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

static int plane_of(int dim, int a)
{
    if (dim <= 2) return a;
    static const int map3[8] = {0, 1, 2, 4, 3, 5, 6, 7};
    return map3[a];
}

static long node_index(const orc_grid *g, int i, int j, int k)
{
    return ((long)k * g->n[1] + j) * g->n[0] + i;
}

double orc_emax(long n, const double *a, const double *b)
{
    double m = 0.0;
    for (long i = 0; i < n; ++i) {
        double d = fabs(a[i] - b[i]);
        if (d > m || d != d) m = d;
    }
    return m;
}

static void gather_cell(const orc_grid *g, const double *const *planes, const int *cell,
                        double *data)
{
    int dim = g->dim, np = 1 << dim;
    for (int v = 0; v < np; ++v) {
        int ci = cell[0] + (v & 1);
        int cj = dim > 1 ? cell[1] + ((v >> 1) & 1) : 0;
        int ck = dim > 2 ? cell[2] + ((v >> 2) & 1) : 0;
        long nid = node_index(g, ci, cj, ck);
        for (int a = 0; a < np; ++a) data[v * np + a] = planes[plane_of(dim, a)][nid];
    }
    if (g->cross == ORC_CROSS_CELL && dim >= 2) orc_cross_cell(dim, g->h, data);
}

/* loop over the cells; for each, the q^p samples; accumulate per sample:
 * mode 0 -> count H_a < 0; mode 1 -> count sign(H_a<0) != sign(H_b<0) */
static double sample_cells(const orc_grid *g, const double *const *a,
                           const double *const *b, int q, int mode, double eps,
                           long *n_amb, int nthreads)
{
    int dim = g->dim;
    int nc[3] = {1, 1, 1};
    for (int d = 0; d < dim; ++d) nc[d] = g->n[d] - 1;
    long ncells = (long)nc[0] * nc[1] * nc[2];
    int nsub = 1;
    for (int d = 0; d < dim; ++d) nsub *= q;
    double cellvol = 1.0;
    for (int d = 0; d < dim; ++d) cellvol *= g->h[d];
    long total = 0, amb = 0;
    (void)nthreads;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) reduction(+ : total, amb) num_threads(nthreads)
#endif
    for (long c = 0; c < ncells; ++c) {
        int cell[3];
        cell[0] = (int)(c % nc[0]);
        cell[1] = (int)((c / nc[0]) % nc[1]);
        cell[2] = (int)(c / ((long)nc[0] * nc[1]));
        double da[64], db[64];
        gather_cell(g, a, cell, da);
        if (mode == 1) gather_cell(g, b, cell, db);
        for (int s = 0; s < nsub; ++s) {
            double xi[3] = {0, 0, 0};
            int r = s;
            for (int d = 0; d < dim; ++d) { xi[d] = ((r % q) + 0.5) / q; r /= q; }
            double Ha, ga[3];
            orc_hermite_cell(dim, da, g->h, xi, &Ha, ga);
            if (fabs(Ha) < eps) amb += 1;
            if (mode == 0) {
                if (Ha < 0.0) total += 1;
            } else {
                double Hb, gb[3];
                orc_hermite_cell(dim, db, g->h, xi, &Hb, gb);
                if (fabs(Hb) < eps && !(fabs(Ha) < eps)) amb += 1;
                if ((Ha < 0.0) != (Hb < 0.0)) total += 1;
            }
        }
    }
    if (n_amb) *n_amb = amb;
    return (double)total * cellvol / nsub;
}

double orc_measure_negative(const orc_grid *g, const double *const *planes, int q,
                            int nthreads)
{
    return sample_cells(g, planes, 0, q, 0, 0.0, 0, nthreads);
}

double orc_symdiff(const orc_grid *g, const double *const *a, const double *const *b,
                   int q, double eps, long *n_ambiguous, int nthreads)
{
    return sample_cells(g, a, b, q, 1, eps, n_ambiguous, nthreads);
}

void orc_eval_points(const orc_grid *g, const double *const *planes, long npts,
                     const double *pts, double *H, double *grad)
{
    int dim = g->dim;
    for (long p = 0; p < npts; ++p) {
        int cell[3] = {0, 0, 0};
        double xi[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) {
            double hi = g->lo[d] + (g->n[d] - 1) * g->h[d];
            double f = pts[p * dim + d];
            if (f < g->lo[d]) f = g->lo[d];
            if (f > hi) f = hi;
            int c = (int)floor((f - g->lo[d]) / g->h[d]);
            if (c < 0) c = 0;
            if (c > g->n[d] - 2) c = g->n[d] - 2;
            cell[d] = c;
            xi[d] = (f - (g->lo[d] + c * g->h[d])) / g->h[d];
        }
        double data[64], gr[3];
        gather_cell(g, planes, cell, data);
        orc_hermite_cell(dim, data, g->h, xi, &H[p], gr);
        for (int d = 0; d < dim; ++d) grad[p * dim + d] = gr[d];
    }
}

/* Sec. 3.4, eqs. surface_normal and curvature, with the interpolant's own first and
 * second derivatives inside the cell of each point (cell located as in orc_eval_points) */
void orc_curvature_points(const orc_grid *g, const double *const *planes, long npts,
                          const double *pts, double *H, double *normal, double *kappa)
{
    int dim = g->dim;
    for (long p = 0; p < npts; ++p) {
        int cell[3] = {0, 0, 0};
        double xi[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) {
            double hi = g->lo[d] + (g->n[d] - 1) * g->h[d];
            double f = pts[p * dim + d];
            if (f < g->lo[d]) f = g->lo[d];
            if (f > hi) f = hi;
            int c = (int)floor((f - g->lo[d]) / g->h[d]);
            if (c < 0) c = 0;
            if (c > g->n[d] - 2) c = g->n[d] - 2;
            cell[d] = c;
            xi[d] = (f - (g->lo[d] + c * g->h[d])) / g->h[d];
        }
        double data[64], gr[3], hs[9];
        gather_cell(g, planes, cell, data);
        orc_hermite_cell2(dim, data, g->h, xi, &H[p], gr, hs);
        double g2 = 0.0;
        for (int d = 0; d < dim; ++d) g2 += gr[d] * gr[d];
        double gn = sqrt(g2);
        for (int d = 0; d < dim; ++d) normal[p * dim + d] = gn > 0.0 ? gr[d] / gn : 0.0;
        if (!(gn > 0.0)) {
            kappa[p] = 0.0;
            continue;
        }
        double num;
        if (dim == 2) {
            double px = gr[0], py = gr[1];
            num = hs[0] * py * py - 2.0 * px * py * hs[1] + hs[3] * px * px;
        } else {
            double tr = 0.0, ghg = 0.0;
            for (int j = 0; j < dim; ++j) {
                tr += hs[j * dim + j];
                for (int k = 0; k < dim; ++k) ghg += gr[j] * hs[j * dim + k] * gr[k];
            }
            num = g2 * tr - ghg;
        }
        kappa[p] = num / (g2 * gn);
    }
}
