/*
 * trace.c -- backward characteristic traces with their Jacobians.
 *
 * TEST INFRASTRUCTURE ONLY (the oracle): see gals_oracle.h.
 *
 * The characteristic through node x at time t+dt is followed back to time t
 * (eq. cir_characteristics).  A superconsistent scheme carries the Jacobian of the
 * approximate backward map alongside the foot point (Def. superconsistent):
 *   Euler  (Ex. superconsistent forward Euler):
 *       foot = x - dt v(x, t+dt),               J = I - dt Dv(x, t+dt)
 *   RK3    (Ex. superconsistent Shu-Osher):
 *       x1 = x - dt v(x, t+dt)                               J1 = I - dt Dv(x,t+dt)
 *       x2 = x - dt (v(x,t+dt)/4 + v(x1,t)/4)                J2 = I - dt (Dv(x,t+dt)/4 + Dv(x1,t) J1/4)
 *       foot = x - dt (v(x,t+dt)/6 + v(x1,t)/6 + 2 v(x2,t+dt/2)/3)
 *       J    = I - dt (Dv(x,t+dt)/6 + Dv(x1,t) J1/6 + 2 Dv(x2,t+dt/2) J2/3)
 * With Dv the usual Jacobian, the chain rule puts the inner Jacobian on the
 * right (the paper's grad x1 . grad v(x1) is the transpose of Dv(x1) J1).
 * orc_flowmap_rk4 integrates the same backward flow with classical RK4 and the
 * variational equation dJ/dtau = Dv(X,tau) J: an accurate reference for the traces.
 */
#include <string.h>
#include "gals_oracle.h"

static void matmul3(const double *A, const double *B, double *C)
{
    double tmp[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            tmp[3 * i + j] = s;
        }
    memcpy(C, tmp, sizeof(tmp));
}

static void identity3(double *A)
{
    memset(A, 0, 9 * sizeof(double));
    A[0] = A[4] = A[8] = 1.0;
}

void orc_trace(int scheme, const orc_velocity *vel, int dim, const double *x,
               double t, double dt, double foot[3], double J[9])
{
    double xv[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) xv[i] = x[i];
    double v1[3], D1[9];
    orc_vel_eval(vel, dim, xv, t + dt, v1, D1);

    /* HEUN_PSI uses the RK3 foot (its J is not used by that scheme) */
    if (scheme == ORC_TRACE_EULER) {
        identity3(J);
        for (int i = 0; i < 3; ++i) foot[i] = xv[i] - dt * v1[i];
        for (int a = 0; a < 9; ++a) J[a] -= dt * D1[a];
        return;
    }

    /* stage 1 */
    double x1[3], J1[9];
    identity3(J1);
    for (int i = 0; i < 3; ++i) x1[i] = xv[i] - dt * v1[i];
    for (int a = 0; a < 9; ++a) J1[a] -= dt * D1[a];

    /* stage 2 at (x1, t) */
    double v2[3], D2[9], D2J1[9];
    orc_vel_eval(vel, dim, x1, t, v2, D2);
    matmul3(D2, J1, D2J1);
    double x2[3], J2[9];
    identity3(J2);
    for (int i = 0; i < 3; ++i) x2[i] = xv[i] - dt * (0.25 * v1[i] + 0.25 * v2[i]);
    for (int a = 0; a < 9; ++a) J2[a] -= dt * (0.25 * D1[a] + 0.25 * D2J1[a]);

    /* stage 3 at (x2, t + dt/2) */
    double v3[3], D3[9], D3J2[9];
    orc_vel_eval(vel, dim, x2, t + 0.5 * dt, v3, D3);
    matmul3(D3, J2, D3J2);
    identity3(J);
    for (int i = 0; i < 3; ++i)
        foot[i] = xv[i] - dt * (v1[i] / 6.0 + v2[i] / 6.0 + 2.0 * v3[i] / 3.0);
    for (int a = 0; a < 9; ++a)
        J[a] -= dt * (D1[a] / 6.0 + D2J1[a] / 6.0 + 2.0 * D3J2[a] / 3.0);

    for (int i = dim; i < 3; ++i) foot[i] = 0.0;
}

/* right-hand side of the backward flow in reverse time s = t+dt - tau:
 * dX/ds = -v(X, t+dt-s),  dJ/ds = -Dv(X, t+dt-s) J */
static void flow_rhs(const orc_velocity *vel, int dim, const double *X, const double *Jm,
                     double tau, double *dX, double *dJ)
{
    double v[3], Dv[9], DJ[9];
    orc_vel_eval(vel, dim, X, tau, v, Dv);
    matmul3(Dv, Jm, DJ);
    for (int i = 0; i < 3; ++i) dX[i] = -v[i];
    for (int a = 0; a < 9; ++a) dJ[a] = -DJ[a];
}

void orc_flowmap_rk4(const orc_velocity *vel, int dim, const double *x, double t,
                     double dt, int m, double foot[3], double J[9])
{
    double X[3] = {0, 0, 0}, Jm[9];
    for (int i = 0; i < dim; ++i) X[i] = x[i];
    identity3(Jm);
    double hs = dt / m;
    for (int s = 0; s < m; ++s) {
        double tau = t + dt - s * hs; /* physical time at the start of this sub-step */
        double k1x[3], k1J[9], k2x[3], k2J[9], k3x[3], k3J[9], k4x[3], k4J[9];
        double Xt[3], Jt[9];
        flow_rhs(vel, dim, X, Jm, tau, k1x, k1J);
        for (int i = 0; i < 3; ++i) Xt[i] = X[i] + 0.5 * hs * k1x[i];
        for (int a = 0; a < 9; ++a) Jt[a] = Jm[a] + 0.5 * hs * k1J[a];
        flow_rhs(vel, dim, Xt, Jt, tau - 0.5 * hs, k2x, k2J);
        for (int i = 0; i < 3; ++i) Xt[i] = X[i] + 0.5 * hs * k2x[i];
        for (int a = 0; a < 9; ++a) Jt[a] = Jm[a] + 0.5 * hs * k2J[a];
        flow_rhs(vel, dim, Xt, Jt, tau - 0.5 * hs, k3x, k3J);
        for (int i = 0; i < 3; ++i) Xt[i] = X[i] + hs * k3x[i];
        for (int a = 0; a < 9; ++a) Jt[a] = Jm[a] + hs * k3J[a];
        flow_rhs(vel, dim, Xt, Jt, tau - hs, k4x, k4J);
        for (int i = 0; i < 3; ++i)
            X[i] += hs / 6.0 * (k1x[i] + 2.0 * k2x[i] + 2.0 * k3x[i] + k4x[i]);
        for (int a = 0; a < 9; ++a)
            Jm[a] += hs / 6.0 * (k1J[a] + 2.0 * k2J[a] + 2.0 * k3J[a] + k4J[a]);
    }
    for (int i = 0; i < 3; ++i) foot[i] = (i < dim) ? X[i] : 0.0;
    memcpy(J, Jm, sizeof(Jm));
    /* unused dimensions: identity rows/cols stay as integrated (Dv is zero there) */
}
