/*
 * mlp.c -- a plain FP64 multilayer perceptron: forward pass, backward pass, Adam.
 *
 * TEST INFRASTRUCTURE ONLY (the oracle): see gals_oracle.h.
 *
 * The paper has no learned component; this is the reference for the learned
 * flow-map surrogate of the backward trace (inputs (x, y, t mod 1), outputs the
 * scaled foot displacement and Jacobian).  Layers l = 0..L-1 map
 *     z_l = W_l a_l + b_l,   a_{l+1} = silu(z_l) for hidden layers, a_L = z_{L-1},
 * with silu(z) = z / (1 + exp(-z)).  Loss: mean squared error over batch and
 * outputs, L = 1/(B*m) sum (y - target)^2.  Backward: the textbook chain rule,
 * dL/dW_l = delta_l a_l^T, dL/db_l = sum delta_l, delta_{l-1} = (W_l^T delta_l) * silu'(z_{l-1}).
 * Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr mhat/(sqrt(vhat)+eps)
 * with bias corrections 1 - b^step.
 * Parameter layout (flat): for each layer, W (out x in, row-major), then b (out).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double silu_prime(double z)
{
    double s = 1.0 / (1.0 + exp(-z));
    return s + z * s * (1.0 - s);
}

static long param_count(int nl, const int *sizes)
{
    long n = 0;
    for (int l = 0; l < nl; ++l) n += (long)sizes[l + 1] * sizes[l] + sizes[l + 1];
    return n;
}

/* forward for one sample; stores pre-activations z and activations a per layer
 * (a[0] = input); widths up to 512 */
static void fwd_one(int nl, const int *sizes, const double *params, const double *x,
                    double z[][512], double a[][512])
{
    for (int i = 0; i < sizes[0]; ++i) a[0][i] = x[i];
    const double *p = params;
    for (int l = 0; l < nl; ++l) {
        int nin = sizes[l], nout = sizes[l + 1];
        const double *W = p, *b = p + (long)nout * nin;
        for (int o = 0; o < nout; ++o) {
            double s = b[o];
            for (int i = 0; i < nin; ++i) s += W[(long)o * nin + i] * a[l][i];
            z[l][o] = s;
            a[l + 1][o] = (l < nl - 1) ? silu(s) : s;
        }
        p += (long)nout * nin + nout;
    }
}

void orc_mlp_forward(int nl, const int *sizes, const double *params, long batch,
                     const double *X, double *Y, double *unused)
{
    (void)unused;
    double (*z)[512] = malloc(sizeof(double[8][512]));
    double (*a)[512] = malloc(sizeof(double[9][512]));
    for (long s = 0; s < batch; ++s) {
        fwd_one(nl, sizes, params, X + s * sizes[0], z, a);
        for (int o = 0; o < sizes[nl]; ++o) Y[s * sizes[nl] + o] = a[nl][o];
    }
    free(z);
    free(a);
}

double orc_mlp_backward(int nl, const int *sizes, const double *params, long batch,
                        const double *X, const double *T, double *grad, double *unused)
{
    (void)unused;
    long np = param_count(nl, sizes);
    memset(grad, 0, np * sizeof(double));
    double (*z)[512] = malloc(sizeof(double[8][512]));
    double (*a)[512] = malloc(sizeof(double[9][512]));
    double *delta = malloc(512 * sizeof(double)), *dprev = malloc(512 * sizeof(double));
    int nout_last = sizes[nl];
    double loss = 0.0, scale = 1.0 / ((double)batch * nout_last);
    /* offsets of each layer's W in the flat parameter vector */
    long off[8];
    long acc = 0;
    for (int l = 0; l < nl; ++l) { off[l] = acc; acc += (long)sizes[l + 1] * sizes[l] + sizes[l + 1]; }

    for (long s = 0; s < batch; ++s) {
        fwd_one(nl, sizes, params, X + s * sizes[0], z, a);
        for (int o = 0; o < nout_last; ++o) {
            double r = a[nl][o] - T[s * nout_last + o];
            loss += r * r;
            delta[o] = 2.0 * r * scale; /* dL/dz_{L-1} (linear output) */
        }
        for (int l = nl - 1; l >= 0; --l) {
            int nin = sizes[l], nout = sizes[l + 1];
            const double *W = params + off[l];
            double *gW = grad + off[l], *gb = grad + off[l] + (long)nout * nin;
            for (int o = 0; o < nout; ++o) {
                gb[o] += delta[o];
                for (int i = 0; i < nin; ++i) gW[(long)o * nin + i] += delta[o] * a[l][i];
            }
            if (l > 0) {
                for (int i = 0; i < nin; ++i) {
                    double sacc = 0.0;
                    for (int o = 0; o < nout; ++o) sacc += W[(long)o * nin + i] * delta[o];
                    dprev[i] = sacc * silu_prime(z[l - 1][i]);
                }
                memcpy(delta, dprev, nin * sizeof(double));
            }
        }
    }
    free(z); free(a); free(delta); free(dprev);
    return loss * scale;
}

void orc_adam_update(long n, double *params, const double *grad, double *m, double *v,
                     double lr, double b1, double b2, double eps, int step)
{
    double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    for (long i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        params[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
