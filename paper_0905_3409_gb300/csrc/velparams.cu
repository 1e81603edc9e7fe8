// velparams.cu -- validation of a gals_velocity descriptor and its conversion to the
// kernels' VelParams (shared by the single-grid and batched C ABI).
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "capi_internal.h"

namespace gals {

namespace {
bool finite3(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

gals_status vfail(char *msg, size_t len, gals_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, len, fmt, ap);
    va_end(ap);
    return st;
}
}  // namespace

gals_status velparams_from(int dim, const gals_velocity *v, VelParams &vp, char *msg, size_t len)
{
    std::memset(&vp, 0, sizeof(vp));
    if (!v) return vfail(msg, len, GALS_ERR_ARG, "velocity descriptor is NULL");
    if (v->trace != GALS_TRACE_EULER && v->trace != GALS_TRACE_RK3 && v->trace != GALS_TRACE_SURROGATE &&
        v->trace != GALS_TRACE_HEUN_PSI)
        return vfail(msg, len, GALS_ERR_ARG, "unknown trace scheme %d", v->trace);
    if (!vel_supported(dim, v->kind))
        return vfail(msg, len, GALS_ERR_UNSUPPORTED, "velocity kind %d not available in %dD", v->kind, dim);
    if (!finite3(v->c, 3) || !finite3(v->center, 3) || !std::isfinite(v->omega) || !std::isfinite(v->T))
        return vfail(msg, len, GALS_ERR_ARG, "non-finite velocity parameter");
    vp.kind = v->kind;
    vp.omega = (float)v->omega;
    vp.cx = (float)v->center[0]; vp.cy = (float)v->center[1]; vp.cz = (float)v->center[2];
    vp.c0 = (float)v->c[0]; vp.c1 = (float)v->c[1]; vp.c2 = (float)v->c[2];
    const double nrm = std::sqrt(2.0 + M_PI);
    vp.d0 = (float)(std::sqrt(2.0) / nrm);
    vp.d1 = (float)(std::sqrt(M_PI) / nrm);
    if (v->kind == GALS_VEL_VORTEX2D || v->kind == GALS_VEL_DEFORM3D) {
        if (!(v->T > 0.0)) return vfail(msg, len, GALS_ERR_ARG, "modulation period T must be > 0");
        vp.invT = 1.0 / v->T;
    }
    if (v->kind == GALS_VEL_FOURIER2D) {
        if (v->nmodes < 1 || v->nmodes > GALS_MAX_MODES || !v->modes)
            return vfail(msg, len, GALS_ERR_ARG, "FOURIER2D needs 1..%d modes", GALS_MAX_MODES);
        vp.nmodes = v->nmodes;
        for (int m = 0; m < v->nmodes; ++m) {
            const double *md = v->modes + 5 * m;
            if (!finite3(md, 5)) return vfail(msg, len, GALS_ERR_ARG, "non-finite mode %d", m);
            int k = (int)md[1], l = (int)md[2];
            if (k != md[1] || l != md[2] || k < 1 || k > 4 || l < 1 || l > 4)
                return vfail(msg, len, GALS_ERR_ARG, "mode %d: k, l must be integers in 1..4", m);
            if (md[3] < 0) return vfail(msg, len, GALS_ERR_ARG, "mode %d: n must be >= 0", m);
            vp.mode_a[m] = (float)md[0];
            vp.mode_kl[m] = k | (l << 8);
            vp.mode_n[m] = md[3];
            vp.mode_chi[m] = md[4] / (2.0 * M_PI);
        }
    }
    return GALS_OK;
}

double speed_bound(const gals_velocity *v, int dim, const double lo[3], const double hi[3])
{
    // the largest |x - c| over the box along one axis
    auto reach = [&](int a, double c) { return std::fmax(std::fabs(lo[a] - c), std::fabs(hi[a] - c)); };
    switch (v->kind) {
    case GALS_VEL_CONST:
        return std::fmax(std::fabs(v->c[0]), std::fmax(std::fabs(v->c[1]), dim == 3 ? std::fabs(v->c[2]) : 0.0));
    case GALS_VEL_ROTATION:  // u = -omega (y - cy), v = omega (x - cx)
        return std::fabs(v->omega) * std::fmax(reach(0, v->center[0]), reach(1, v->center[1]));
    case GALS_VEL_VORTEX2D:  // |sin^2 (pi x) sin(2 pi y) cos(pi t / T)| <= 1
        return 1.0;
    case GALS_VEL_DEFORM3D:  // the u component carries the factor 2
        return 2.0;
    case GALS_VEL_PSEUDO1D: {  // v = exp(d . x) d with d = (sqrt 2, sqrt pi) / sqrt(2 + pi)
        const double nrm = std::sqrt(2.0 + M_PI), d0 = std::sqrt(2.0) / nrm, d1 = std::sqrt(M_PI) / nrm;
        return std::exp(d0 * std::fmax(lo[0], hi[0]) + d1 * std::fmax(lo[1], hi[1]));
    }
    case GALS_VEL_FOURIER2D: {  // |u| <= pi sum |a| l, |v| <= pi sum |a| k
        double b = 0.0;
        for (int m = 0; m < v->nmodes; ++m) {
            const double *md = v->modes + 5 * m;
            b += std::fabs(md[0]) * std::fmax(md[1], md[2]);
        }
        return M_PI * b;
    }
    default:
        return INFINITY;
    }
}

bool grid_size_ok(int dim, const int n[3], char *msg, size_t len)
{
    if (dim == 2) {
        const int64_t pitch = ((int64_t)n[0] + 3) / 4 * 4;
        if (pitch * n[1] > (int64_t)INT32_MAX) {
            snprintf(msg, len, "2D grid %d x %d: more than 2^31 - 1 elements per plane", n[0], n[1]);
            return false;
        }
        const int64_t rows = (int64_t)65535 * tile_rows2d();
        if (n[1] > rows) {
            snprintf(msg, len, "2D grid: n[1] = %d above %lld", n[1], (long long)rows);
            return false;
        }
        return true;
    }
    for (int i = 1; i < 3; ++i)
        if (n[i] > 65535 * 4) {
            snprintf(msg, len, "3D grid: n[%d] = %d above %d", i, n[i], 65535 * 4);
            return false;
        }
    if (n[0] > INT32_MAX - 3) {
        snprintf(msg, len, "3D grid: n[0] = %d too large", n[0]);
        return false;
    }
    return true;
}

}  // namespace gals
