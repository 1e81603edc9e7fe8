/*
 * hermite.c -- p-cubic Hermite interpolant, written out term by term.
 *
 * TEST INFRASTRUCTURE ONLY (the oracle): see gals_oracle.h.
 *
 * Sec. 2.3 of the paper builds the interpolant on a cell from the 4^p data
 * phi_a^v = d^a phi(x_v), v, a in {0,1}^p (Def. "data for phi on C"), as the
 * tensor-product sum of eq. p-cubic_interpolant:
 *     H(x) = sum_{v,a} phi_a^v h^{|a|} W_a^v(x/h),   W_a^v(x) = prod_i w_{a_i}^{v_i}(x_i)
 * with the 1-cubic basis of eq. 1-cubic_basis_functions built from
 *     f(x) = 1 - 3x^2 + 2x^3,   g(x) = x (1-x)^2 .
 * For rectangular cells h^{|a|} becomes prod_i h_i^{a_i}.  The gradient is the
 * analytic derivative of the same sum: d/dx_j brings 1/h_j and w' in factor j, and the
 * second derivatives (Sec. 3.4, "Approximation of derivative quantities": all first and
 * second derivatives inside a cell by differentiating the interpolant) bring w'' in
 * factor j for d^2/dx_j^2, and w' in factors j and k for d^2/dx_j dx_k.
 * This file evaluates the 4^p-term sum directly; it does not factorise it.
 */
#include "gals_oracle.h"

static double f_(double x) { return 1.0 - 3.0 * x * x + 2.0 * x * x * x; }
static double fp_(double x) { return -6.0 * x + 6.0 * x * x; }
static double g_(double x) { return x * (1.0 - x) * (1.0 - x); }
static double gp_(double x) { return (1.0 - x) * (1.0 - x) - 2.0 * x * (1.0 - x); }
static double fpp_(double x) { return -6.0 + 12.0 * x; }
static double gpp_(double x) { return -4.0 + 6.0 * x; }

/* second xi-derivatives of the four w_a^v, same index order as orc_basis1d */
static void basis1d_dd(double xi, double ddw[4])
{
    ddw[0] = fpp_(xi);
    ddw[1] = gpp_(xi);
    ddw[2] = fpp_(1.0 - xi);     /* d^2/dxi^2 f(1-xi) */
    ddw[3] = -gpp_(1.0 - xi);    /* d^2/dxi^2 (-g(1-xi)) */
}

/* w_a^v(xi) for v, a in {0,1}, index v*2+a, with its xi-derivative:
 *   v=0,a=0: f(xi)      v=1,a=0: f(1-xi)
 *   v=0,a=1: g(xi)      v=1,a=1: -g(1-xi)            (eq. 1-cubic_basis_functions) */
void orc_basis1d(double xi, double w[4], double dw[4])
{
    w[0] = f_(xi);          dw[0] = fp_(xi);
    w[1] = g_(xi);          dw[1] = gp_(xi);
    w[2] = f_(1.0 - xi);    dw[2] = -fp_(1.0 - xi);
    w[3] = -g_(1.0 - xi);   dw[3] = gp_(1.0 - xi);
}

void orc_hermite_cell(int dim, const double *data, const double *h,
                      const double *xi, double *H, double *gradH)
{
    double w[3][4], dw[3][4];
    int np = 1 << dim; /* 2^p corners and 2^p derivative multi-indices */
    for (int i = 0; i < dim; ++i) orc_basis1d(xi[i], w[i], dw[i]);

    double sum = 0.0, grad[3] = {0.0, 0.0, 0.0};
    for (int v = 0; v < np; ++v) {
        for (int a = 0; a < np; ++a) {
            double coef = data[v * np + a];
            /* h^{|a|} for rectangular cells */
            double scale = 1.0;
            for (int i = 0; i < dim; ++i)
                if ((a >> i) & 1) scale *= h[i];
            /* W_a^v(xi) and its xi_j-derivatives */
            double W = 1.0;
            for (int i = 0; i < dim; ++i) {
                int vi = (v >> i) & 1, ai = (a >> i) & 1;
                W *= w[i][vi * 2 + ai];
            }
            sum += coef * scale * W;
            for (int j = 0; j < dim; ++j) {
                double dWj = 1.0;
                for (int i = 0; i < dim; ++i) {
                    int vi = (v >> i) & 1, ai = (a >> i) & 1;
                    dWj *= (i == j) ? dw[i][vi * 2 + ai] : w[i][vi * 2 + ai];
                }
                grad[j] += coef * scale * dWj / h[j];
            }
        }
    }
    *H = sum;
    for (int j = 0; j < dim; ++j) gradH[j] = grad[j];
}

void orc_hermite_cell2(int dim, const double *data, const double *h, const double *xi,
                       double *H, double *gradH, double *hessH)
{
    double w[3][4], dw[3][4], ddw[3][4];
    int np = 1 << dim;
    for (int i = 0; i < dim; ++i) {
        orc_basis1d(xi[i], w[i], dw[i]);
        basis1d_dd(xi[i], ddw[i]);
    }
    double sum = 0.0, grad[3] = {0.0, 0.0, 0.0}, hess[9] = {0.0};
    for (int v = 0; v < np; ++v) {
        for (int a = 0; a < np; ++a) {
            double coef = data[v * np + a];
            double scale = 1.0;
            for (int i = 0; i < dim; ++i)
                if ((a >> i) & 1) scale *= h[i];
            double W = 1.0;
            for (int i = 0; i < dim; ++i) W *= w[i][((v >> i) & 1) * 2 + ((a >> i) & 1)];
            sum += coef * scale * W;
            for (int j = 0; j < dim; ++j) {
                double dWj = 1.0;
                for (int i = 0; i < dim; ++i) {
                    int e = ((v >> i) & 1) * 2 + ((a >> i) & 1);
                    dWj *= (i == j) ? dw[i][e] : w[i][e];
                }
                grad[j] += coef * scale * dWj / h[j];
                for (int k = 0; k < dim; ++k) {
                    double d2 = 1.0;
                    for (int i = 0; i < dim; ++i) {
                        int e = ((v >> i) & 1) * 2 + ((a >> i) & 1);
                        if (i == j && i == k) d2 *= ddw[i][e];
                        else if (i == j || i == k) d2 *= dw[i][e];
                        else d2 *= w[i][e];
                    }
                    hess[j * dim + k] += coef * scale * d2 / (h[j] * h[k]);
                }
            }
        }
    }
    *H = sum;
    for (int j = 0; j < dim; ++j) gradH[j] = grad[j];
    for (int e = 0; e < dim * dim; ++e) hessH[e] = hess[e];
}
