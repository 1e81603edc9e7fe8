// velparams.cu -- validation of a gals_velocity descriptor and its conversion to the
// kernels' VelParams (shared by the single-grid and batched C ABI).
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

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
    if (v->kind == GALS_VEL_WAVES2D) {
        // the mode table itself goes to device memory of the caller (grid or surrogate):
        // upload_waves
        if (v->nmodes < 1 || v->nmodes > GALS_MAX_WAVES || !v->modes)
            return vfail(msg, len, GALS_ERR_ARG, "WAVES2D needs 1..%d modes", GALS_MAX_WAVES);
        for (int m = 0; m < v->nmodes; ++m) {
            const double *md = v->modes + 6 * m;
            if (!finite3(md, 6)) return vfail(msg, len, GALS_ERR_ARG, "non-finite wave %d", m);
            if (md[4] < 0) return vfail(msg, len, GALS_ERR_ARG, "wave %d: n must be >= 0", m);
        }
        vp.nwaves = v->nmodes;
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
    case GALS_VEL_WAVES2D: {  // |u|, |v| <= sum |a| |k|
        double b = 0.0;
        for (int m = 0; m < v->nmodes; ++m) {
            const double *md = v->modes + 6 * m;
            b += std::fabs(md[0]) * std::hypot(md[1], md[2]);
        }
        return b;
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

cudaError_t WaveStore::upload(const gals_velocity *v, cudaStream_t s, bool *changed)
{
    *changed = false;
    const int M = v->nmodes;
    const size_t nd = (size_t)6 * M;
    if (M == count && std::memcmp(host.data(), v->modes, sizeof(double) * nd) == 0) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(s);  // earlier work may still read the table
    if (e != cudaSuccess) return e;
    if (M > cap) {
        cudaFree(dev);
        dev = nullptr;
        cap = 0;
        if ((e = cudaMalloc(&dev, (sizeof(float4) * 3 + sizeof(double) * 3) * (size_t)M)) != cudaSuccess) {
            count = 0;
            return e;
        }
        cap = M;
    }
    std::vector<float4> f((size_t)3 * M);
    std::vector<double> d((size_t)3 * M);
    for (int m = 0; m < M; ++m) {
        const double *md = v->modes + 6 * m;
        const float kx = (float)md[1], ky = (float)md[2];
        f[m] = make_float4(kx, ky, (float)md[3], kx * ky);
        f[M + m] = make_float4(kx * kx, ky * ky, 0.f, 0.f);
        const double chi = md[5] / (2.0 * M_PI);
        f[2 * M + m] = make_float4((float)md[0], (float)md[4], (float)chi, 0.f);
        d[3 * m] = md[0];
        d[3 * m + 1] = md[4];
        d[3 * m + 2] = chi;
    }
    if ((e = cudaMemcpy(dev, f.data(), sizeof(float4) * f.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(reinterpret_cast<char *>(dev) + sizeof(float4) * f.size(), d.data(),
                        sizeof(double) * d.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
        count = 0;
        return e;
    }
    host.assign(v->modes, v->modes + nd);
    count = M;
    *changed = true;
    return cudaSuccess;
}

void WaveStore::bind(VelParams &vp) const
{
    vp.waves = reinterpret_cast<const float4 *>(dev);
    vp.waves_d = reinterpret_cast<const double *>(reinterpret_cast<const char *>(dev) +
                                                  sizeof(float4) * 3 * (size_t)count);
}

void WaveStore::release()
{
    cudaFree(dev);
    dev = nullptr;
    cap = count = 0;
    host.clear();
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
