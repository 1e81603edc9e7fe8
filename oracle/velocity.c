/*
 * velocity.c -- analytic velocity fields v(x,t) and their Jacobians Dv.
 *
 * TEST INFRASTRUCTURE ONLY (the oracle): see gals_oracle.h.
 *
 * Sec. 4 assumes v and its deformation matrix are exactly accessible everywhere.
 * Dv[3*i+j] = d v_i / d x_j (the paper writes the transpose).  Fields:
 *   CONST      v = c.
 *   ROTATION   u = -omega (y - cy), v = omega (x - cx), w = 0 (Zalesak rotation,
 *              Sec. 6.2.1 and 6.2.3, rescaled to the unit box).
 *   VORTEX2D   v = (-dPsi/dy, dPsi/dx) with Psi = (1/pi) cos(pi t/T) sin^2(pi x) sin^2(pi y)
 *              (eq. swirl_2d_velocity_field, Sec. 6.1.2).
 *   DEFORM3D   u = 2 sin^2(pi x) sin(2 pi y) sin(2 pi z), v = -sin(2 pi x) sin^2(pi y) sin(2 pi z),
 *              w = -sin(2 pi x) sin(2 pi y) sin^2(pi z), all times cos(pi t/T) (Sec. 6.2.4;
 *              the printed sin(2 pi x y) in u is read as sin(2 pi y), LeVeque's field).
 *   PSEUDO1D   v = (1/sqrt(2+pi)) exp((sqrt2 x + sqrtpi y)/sqrt(2+pi)) (sqrt2, sqrtpi)
 *              (eq. velocity_1, Sec. 6.1.1).
 *   FOURIER2D  v = (-dPsi/dy, dPsi/dx), Psi = sum_m a_m sin(k_m pi x) sin(l_m pi y) cos(2 pi n_m t + chi_m).
 *   WAVES2D    v = (-dPsi/dy, dPsi/dx), Psi = sum_m a_m sin(kx_m x + ky_m y + phase_m) cos(2 pi n_m t + chi_m)
 *              (a costly field: no separable form, one sine and cosine per mode).
 * Each field is written out from its definition; derivatives by hand.
 */
#include <math.h>
#include <string.h>
#include "gals_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

void orc_vel_eval(const orc_velocity *vel, int dim, const double *x, double t,
                  double v[3], double Dv[9])
{
    memset(v, 0, 3 * sizeof(double));
    memset(Dv, 0, 9 * sizeof(double));
    const double pi = M_PI;
    switch (vel->kind) {
    case ORC_VEL_CONST:
        for (int i = 0; i < dim; ++i) v[i] = vel->c[i];
        break;
    case ORC_VEL_ROTATION: {
        double w = vel->omega;
        v[0] = -w * (x[1] - vel->center[1]);
        v[1] = w * (x[0] - vel->center[0]);
        Dv[0 * 3 + 1] = -w;
        Dv[1 * 3 + 0] = w;
        break;
    }
    case ORC_VEL_VORTEX2D: {
        double c = cos(pi * t / vel->T);
        double X = x[0], Y = x[1];
        double sx = sin(pi * X), sy = sin(pi * Y);
        /* Psi = (c/pi) sin^2(pi x) sin^2(pi y) */
        /* u = -Psi_y = -(c/pi) sin^2(pi x) 2 pi sin(pi y) cos(pi y) = -c sin^2(pi x) sin(2 pi y) */
        v[0] = -c * sx * sx * sin(2.0 * pi * Y);
        /* v = Psi_x = c sin(2 pi x) sin^2(pi y) */
        v[1] = c * sin(2.0 * pi * X) * sy * sy;
        /* du/dx = -c * 2 sin(pi x) cos(pi x) pi * sin(2 pi y) = -c pi sin(2 pi x) sin(2 pi y) */
        Dv[0] = -c * pi * sin(2.0 * pi * X) * sin(2.0 * pi * Y);
        /* du/dy = -c sin^2(pi x) 2 pi cos(2 pi y) */
        Dv[1] = -c * sx * sx * 2.0 * pi * cos(2.0 * pi * Y);
        /* dv/dx = c 2 pi cos(2 pi x) sin^2(pi y) */
        Dv[3] = c * 2.0 * pi * cos(2.0 * pi * X) * sy * sy;
        /* dv/dy = c sin(2 pi x) 2 sin(pi y) cos(pi y) pi = c pi sin(2 pi x) sin(2 pi y) */
        Dv[4] = c * pi * sin(2.0 * pi * X) * sin(2.0 * pi * Y);
        break;
    }
    case ORC_VEL_DEFORM3D: {
        double c = cos(pi * t / vel->T);
        double X = x[0], Y = x[1], Z = x[2];
        double s1x = sin(pi * X), s1y = sin(pi * Y), s1z = sin(pi * Z);
        double s2x = sin(2 * pi * X), s2y = sin(2 * pi * Y), s2z = sin(2 * pi * Z);
        double c2x = cos(2 * pi * X), c2y = cos(2 * pi * Y), c2z = cos(2 * pi * Z);
        /* u = 2 sin^2(pi x) sin(2 pi y) sin(2 pi z) c */
        v[0] = 2.0 * s1x * s1x * s2y * s2z * c;
        /* v = -sin(2 pi x) sin^2(pi y) sin(2 pi z) c */
        v[1] = -s2x * s1y * s1y * s2z * c;
        /* w = -sin(2 pi x) sin(2 pi y) sin^2(pi z) c */
        v[2] = -s2x * s2y * s1z * s1z * c;
        /* d(sin^2(pi s))/ds = pi sin(2 pi s);  d(sin(2 pi s))/ds = 2 pi cos(2 pi s) */
        Dv[0] = 2.0 * pi * s2x * s2y * s2z * c;
        Dv[1] = 2.0 * s1x * s1x * 2.0 * pi * c2y * s2z * c;
        Dv[2] = 2.0 * s1x * s1x * s2y * 2.0 * pi * c2z * c;
        Dv[3] = -2.0 * pi * c2x * s1y * s1y * s2z * c;
        Dv[4] = -s2x * pi * s2y * s2z * c;
        Dv[5] = -s2x * s1y * s1y * 2.0 * pi * c2z * c;
        Dv[6] = -2.0 * pi * c2x * s2y * s1z * s1z * c;
        Dv[7] = -s2x * 2.0 * pi * c2y * s1z * s1z * c;
        Dv[8] = -s2x * s2y * pi * s2z * c;
        break;
    }
    case ORC_VEL_PSEUDO1D: {
        double nrm = sqrt(2.0 + pi);
        double d0 = sqrt(2.0) / nrm, d1 = sqrt(pi) / nrm;
        double e = exp(d0 * x[0] + d1 * x[1]);
        /* v = e^s d with s = d.x (the prefactor 1/sqrt(2+pi) is the normalisation of d) */
        v[0] = e * d0;
        v[1] = e * d1;
        Dv[0] = e * d0 * d0;
        Dv[1] = e * d0 * d1;
        Dv[3] = e * d1 * d0;
        Dv[4] = e * d1 * d1;
        break;
    }
    case ORC_VEL_FOURIER2D: {
        for (int m = 0; m < vel->nmodes; ++m) {
            const double *md = vel->modes + 5 * m;
            double a = md[0], k = md[1], l = md[2], n = md[3], chi = md[4];
            double c = cos(2.0 * pi * n * t + chi);
            double skx = sin(k * pi * x[0]), ckx = cos(k * pi * x[0]);
            double sly = sin(l * pi * x[1]), cly = cos(l * pi * x[1]);
            /* Psi_m = a skx sly c;  u = -Psi_y, v = Psi_x */
            v[0] += -a * skx * l * pi * cly * c;
            v[1] += a * k * pi * ckx * sly * c;
            Dv[0] += -a * k * pi * ckx * l * pi * cly * c;
            Dv[1] += a * skx * l * pi * l * pi * sly * c;
            Dv[3] += -a * k * pi * k * pi * skx * sly * c;
            Dv[4] += a * k * pi * ckx * l * pi * cly * c;
        }
        break;
    }
    case ORC_VEL_WAVES2D: {
        for (int m = 0; m < vel->nmodes; ++m) {
            const double *md = vel->modes + 6 * m;
            double a = md[0], kx = md[1], ky = md[2], phase = md[3], n = md[4], chi = md[5];
            double c = a * cos(2.0 * pi * n * t + chi);
            double th = kx * x[0] + ky * x[1] + phase;
            double s = sin(th), co = cos(th);
            /* Psi_m = c sin(th): Psi_x = c kx cos(th), Psi_y = c ky cos(th);
             * u = -Psi_y, v = Psi_x */
            v[0] += -c * ky * co;
            v[1] += c * kx * co;
            Dv[0] += c * ky * kx * s;     /* du/dx */
            Dv[1] += c * ky * ky * s;     /* du/dy */
            Dv[3] += -c * kx * kx * s;    /* dv/dx */
            Dv[4] += -c * kx * ky * s;    /* dv/dy */
        }
        break;
    }
    default:
        break;
    }
}
