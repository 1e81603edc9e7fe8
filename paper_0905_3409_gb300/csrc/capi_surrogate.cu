// capi_surrogate.cu -- C ABI of the learned flow-map surrogate (gals_surrogate_*).
//
// Holds the FP32 master parameters, the Adam moments, the BF16 inference copy and the
// training scratch on the device.  Training draws a fresh batch each step (random points
// and phases, RK4 flow-map targets), runs the forward and backward kernels and an Adam
// update with a cosine learning-rate schedule; the output scales (one per output) are the
// standard deviations of a calibration batch, so the network works on O(1) targets.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "capi_internal.h"
#include "mlp_internal.h"

using namespace gals;
using namespace gals::mlp;

struct gals_surrogate {
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    InferParams ip{};
    float *scale_dev = nullptr, *one = nullptr;
    double *loss_dev = nullptr;
    // training scratch (capacity `cap` samples)
    int cap = 0;
    float *Xn = nullptr, *T = nullptr, *Z[NLAYER] = {}, *A[NLAYER] = {}, *G0 = nullptr, *G1 = nullptr;
    float *split = nullptr;
    // bound field
    bool bound = false;
    VelParams vp{};
    WaveStore waves;  // WAVES2D: the bound field's modes on the device
    double dt = 0.0, h = 0.0;
    // residual check
    float tol_x = 0.05f, tol_J = 0.05f;
    int samples = 4;
    unsigned long long *counters = nullptr;  // tiles, fallbacks
    int *err_dev = nullptr;                  // device error word of the inference kernel
    int adam_step = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char err[256] = "";
};

namespace {

char g_sur_err[256] = "";

gals_status sfail(gals_surrogate *s, gals_status st, const char *fmt, ...)
{
    char *dst = s ? s->err : g_sur_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return st;
}

gals_status scuda(gals_surrogate *s, cudaError_t e, const char *what)
{
    // the runtime keeps a failed call's error as the thread's last error; a non-sticky one
    // (a failed allocation) would otherwise fail the next launch check of any handle
    cudaGetLastError();
    return sfail(s, e == cudaErrorMemoryAllocation ? GALS_ERR_NOMEM : GALS_ERR_CUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

// After a synchronisation: report (and clear) a timeout recorded by the inference kernel.
gals_status check_err(gals_surrogate *s)
{
    int code = 0;
    cudaError_t e = cudaMemcpy(&code, s->err_dev, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return scuda(s, e, "error word");
    if (code == 0) return GALS_OK;
    cudaMemset(s->err_dev, 0, sizeof(int));
    return sfail(s, GALS_ERR_TIMEOUT, "a bounded wait of a tensor-core kernel ran out (code %d)", code);
}

uint64_t splitmix64_host(uint64_t &state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

cudaError_t ensure_scratch(gals_surrogate *s, int n)
{
    if (n <= s->cap) return cudaSuccess;
    cudaStreamSynchronize(s->stream);
    cudaFree(s->Xn); cudaFree(s->T); cudaFree(s->G0); cudaFree(s->G1); cudaFree(s->split);
    for (int l = 0; l < NLAYER; ++l) { cudaFree(s->Z[l]); cudaFree(s->A[l]); s->Z[l] = s->A[l] = nullptr; }
    s->Xn = s->T = s->G0 = s->G1 = s->split = nullptr;
    s->cap = 0;
    cudaError_t e;
    if ((e = cudaMalloc(&s->Xn, sizeof(float) * 3 * (size_t)n)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&s->T, sizeof(float) * OUT * (size_t)n)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&s->G0, sizeof(float) * HID * (size_t)n)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&s->G1, sizeof(float) * HID * (size_t)n)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&s->split, sizeof(float) * kMaxSplit * HID * HID)) != cudaSuccess) return e;
    for (int l = 0; l < NLAYER; ++l) {
        if ((e = cudaMalloc(&s->Z[l], sizeof(float) * lout(l) * (size_t)n)) != cudaSuccess) return e;
        if (l > 0 && (e = cudaMalloc(&s->A[l], sizeof(float) * HID * (size_t)n)) != cudaSuccess) return e;
    }
    s->cap = n;
    return cudaSuccess;
}

gals_status check_field(gals_surrogate *s, const gals_velocity *vel, VelParams &vp)
{
    char msg[200];
    gals_status st = velparams_from(2, vel, vp, msg, sizeof(msg));
    if (st != GALS_OK) return sfail(s, st, "%s", msg);
    if (vel->kind != GALS_VEL_FOURIER2D && vel->kind != GALS_VEL_WAVES2D)
        return sfail(s, GALS_ERR_UNSUPPORTED, "the surrogate is built for FOURIER2D and WAVES2D fields");
    if (vel->kind == GALS_VEL_WAVES2D) {
        bool changed = false;
        cudaError_t e = s->waves.upload(vel, s->stream, &changed);
        if (e != cudaSuccess) return scuda(s, e, "wave table");
        s->waves.bind(vp);
    }
    return GALS_OK;
}

cudaError_t repack(gals_surrogate *s)
{
    return pack_infer(s->params, s->ip, s->stream);
}

}  // namespace

namespace gals {

// Used by gals_step: is `s` usable for this call?  On success fills the kernel-side views.
gals_status surrogate_for_step(const gals_surrogate *s, const gals_velocity *v, const VelParams &vp,
                               double dt, double h0, double h1, mlp::InferParams &ip, mlp::Check &chk,
                               char *msg, size_t len)
{
    if (!s) { snprintf(msg, len, "GALS_TRACE_SURROGATE needs vel->surrogate"); return GALS_ERR_ARG; }
    if (!s->bound) { snprintf(msg, len, "the surrogate is not trained or bound"); return GALS_ERR_STATE; }
    const double rel = 1e-9;
    if (std::fabs(dt - s->dt) > rel * s->dt || std::fabs(h0 - s->h) > rel * s->h ||
        std::fabs(h1 - s->h) > rel * s->h) {
        snprintf(msg, len, "the surrogate was trained for dt = %.17g, h = %.17g", s->dt, s->h);
        return GALS_ERR_ARG;
    }
    if (vp.kind == VK_WAVES2D) {
        if (s->vp.kind != VK_WAVES2D || v->nmodes != s->waves.count ||
            std::memcmp(v->modes, s->waves.host.data(), sizeof(double) * 6 * (size_t)v->nmodes)) {
            snprintf(msg, len, "the velocity differs from the one the surrogate was trained for");
            return GALS_ERR_ARG;
        }
    } else if (vp.kind != s->vp.kind || vp.nmodes != s->vp.nmodes ||
        std::memcmp(vp.mode_a, s->vp.mode_a, sizeof(float) * vp.nmodes) ||
        std::memcmp(vp.mode_kl, s->vp.mode_kl, sizeof(int) * vp.nmodes) ||
        std::memcmp(vp.mode_n, s->vp.mode_n, sizeof(double) * vp.nmodes) ||
        std::memcmp(vp.mode_chi, s->vp.mode_chi, sizeof(double) * vp.nmodes)) {
        snprintf(msg, len, "the velocity differs from the one the surrogate was trained for");
        return GALS_ERR_ARG;
    }
    ip = s->ip;
    chk.tol_x = s->tol_x;
    chk.tol_J = s->tol_J;
    chk.samples = s->samples;
    chk.tiles = s->counters;
    chk.fallbacks = s->counters + 1;
    return GALS_OK;
}

}  // namespace gals

extern "C" {

const char *gals_surrogate_last_error(const gals_surrogate *s) { return s ? s->err : g_sur_err; }

gals_status gals_surrogate_create(const gals_mlp_desc *desc, gals_surrogate **out)
{
    if (!out) return sfail(nullptr, GALS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return sfail(nullptr, GALS_ERR_ARG, "desc is NULL");
    gals_surrogate *s = new (std::nothrow) gals_surrogate();
    if (!s) return sfail(nullptr, GALS_ERR_NOMEM, "host allocation failed");
    cudaError_t e;
    auto bail = [&](cudaError_t err, const char *what) {
        gals_status st = scuda(nullptr, err, what);
        gals_surrogate_destroy(s);
        return st;
    };
    if (desc->cuda_stream) {
        s->stream = (cudaStream_t)desc->cuda_stream;
    } else {
        if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(e, "cudaStreamCreate");
        s->own_stream = true;
    }
    const size_t pb = sizeof(float) * NPARAM;
    if ((e = cudaMalloc(&s->params, pb)) != cudaSuccess || (e = cudaMalloc(&s->grad, pb)) != cudaSuccess ||
        (e = cudaMalloc(&s->m, pb)) != cudaSuccess || (e = cudaMalloc(&s->v, pb)) != cudaSuccess ||
        (e = cudaMalloc(&s->ip.w, sizeof(uint16_t) * W_TOTAL)) != cudaSuccess ||
        (e = cudaMalloc(&s->scale_dev, sizeof(float) * OUT)) != cudaSuccess ||
        (e = cudaMalloc(&s->one, sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&s->loss_dev, sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&s->counters, 2 * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&s->err_dev, sizeof(int))) != cudaSuccess)
        return bail(e, "cudaMalloc");
    // Weights uniform in [-a, a]: Glorot for the hidden and output layers; the first layer
    // (and its bias) uniform in [-4, 4], so that the SiLU units of the first layer already
    // vary over the unit box at the frequencies of the field (with Glorot's small first
    // layer the network starts nearly linear and learns them very slowly).  Other biases 0.
    std::vector<float> p(NPARAM, 0.f);
    uint64_t st = desc->seed;
    auto uni = [&]() { return (double)(splitmix64_host(st) >> 11) * (1.0 / 9007199254740992.0); };
    for (int l = 0; l < NLAYER; ++l) {
        const float a = l == 0 ? 4.f : std::sqrt(6.f / (float)(lin(l) + lout(l)));
        for (int64_t i = 0; i < (int64_t)lin(l) * lout(l); ++i) p[woff(l) + i] = (float)((2.0 * uni() - 1.0) * a);
        if (l == 0)
            for (int i = 0; i < lout(0); ++i) p[boff(0) + i] = (float)((2.0 * uni() - 1.0) * 4.0);
    }
    const float one = 1.f;
    std::vector<float> ones(OUT, 1.f);
    for (int k = 0; k < OUT; ++k) s->ip.scale[k] = 1.f;
    if ((e = cudaMemcpy(s->params, p.data(), pb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(s->m, 0, pb)) != cudaSuccess || (e = cudaMemset(s->v, 0, pb)) != cudaSuccess ||
        (e = cudaMemcpy(s->one, &one, sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(s->scale_dev, ones.data(), sizeof(float) * OUT, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(s->counters, 0, 2 * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemset(s->err_dev, 0, sizeof(int))) != cudaSuccess)
        return bail(e, "initial upload");
    if ((e = repack(s)) != cudaSuccess || (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
        return bail(e, "pack");
    *out = s;
    return GALS_OK;
}

gals_status gals_surrogate_destroy(gals_surrogate *s)
{
    if (!s) return GALS_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    s->waves.release();
    cudaFree(s->params); cudaFree(s->grad); cudaFree(s->m); cudaFree(s->v);
    cudaFree(s->ip.w); cudaFree(s->scale_dev); cudaFree(s->one);
    cudaFree(s->loss_dev); cudaFree(s->counters); cudaFree(s->err_dev);
    cudaFree(s->Xn); cudaFree(s->T); cudaFree(s->G0); cudaFree(s->G1); cudaFree(s->split);
    for (int l = 0; l < NLAYER; ++l) { cudaFree(s->Z[l]); cudaFree(s->A[l]); }
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return GALS_OK;
}

gals_status gals_surrogate_train(gals_surrogate *s, const gals_velocity *vel, double dt, double h,
                                 const gals_train_opts *o, gals_train_report *report)
{
    NvtxRange nvtx_range("gals_surrogate_train");
    if (!s) return sfail(nullptr, GALS_ERR_ARG, "surrogate is NULL");
    if (!o) return sfail(s, GALS_ERR_ARG, "opts is NULL");
    if (!(dt > 0.0) || !(h > 0.0) || !std::isfinite(dt) || !std::isfinite(h))
        return sfail(s, GALS_ERR_ARG, "dt and h must be finite and > 0");
    if (o->steps < 1 || o->batch < 128 || o->batch > 65536 || o->substeps < 1 || !(o->lr > 0.0) ||
        !(o->lr_min >= 0.0))
        return sfail(s, GALS_ERR_ARG, "bad training options");
    VelParams vp;
    gals_status st = check_field(s, vel, vp);
    if (st != GALS_OK) return st;
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t e;
    if ((e = ensure_scratch(s, o->batch)) != cudaSuccess) return scuda(s, e, "training scratch");
    // output scales: standard deviations of a calibration batch (scale 1 first)
    const int n = o->batch;
    std::vector<float> ones(OUT, 1.f), Th((size_t)n * OUT);
    if ((e = cudaMemcpyAsync(s->scale_dev, ones.data(), sizeof(float) * OUT, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess ||
        (e = launch_samples(vp, s->Xn, s->T, n, (float)dt, (float)h, o->substeps, o->seed ^ 0xC0FFEEull, 0,
                            s->scale_dev, s->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(Th.data(), s->T, sizeof(float) * Th.size(), cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
        return scuda(s, e, "calibration batch");
    float scale[OUT];
    for (int k = 0; k < OUT; ++k) {
        double m1 = 0.0, m2 = 0.0;
        for (int i = 0; i < n; ++i) { m1 += Th[(size_t)i * OUT + k]; m2 += (double)Th[(size_t)i * OUT + k] * Th[(size_t)i * OUT + k]; }
        m1 /= n;
        const double var = m2 / n;  // second moment: targets are not centred by the network
        scale[k] = (float)std::sqrt(var > 1e-30 ? var : 1.0);
        s->ip.scale[k] = scale[k];
    }
    if ((e = cudaMemcpyAsync(s->scale_dev, scale, sizeof(scale), cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
        return scuda(s, e, "scales");
    double first = -1.0, last = 0.0;
    for (int it = 0; it < o->steps; ++it) {
        if ((e = launch_samples(vp, s->Xn, s->T, n, (float)dt, (float)h, o->substeps, o->seed, (uint64_t)it + 1,
                                s->scale_dev, s->stream)) != cudaSuccess ||
            (e = forward_train(s->params, s->Xn, n, s->Z, s->A, s->err_dev, s->stream)) != cudaSuccess ||
            (e = backward_train(s->params, s->Xn, s->T, n, s->Z, s->A, s->G0, s->G1, s->grad, s->loss_dev,
                                s->one, s->split, s->err_dev, s->stream)) != cudaSuccess)
            return scuda(s, e, "training step");
        const double frac = o->steps > 1 ? (double)it / (o->steps - 1) : 0.0;
        const double lr = o->lr_min + 0.5 * (o->lr - o->lr_min) * (1.0 + std::cos(M_PI * frac));
        if ((e = adam_step(s->params, s->grad, s->m, s->v, (float)lr, 0.9f, 0.999f, 1e-8f, ++s->adam_step,
                           s->stream)) != cudaSuccess)
            return scuda(s, e, "adam");
        if (it == 0 || it == o->steps - 1) {
            double l = 0.0;
            if ((e = cudaMemcpyAsync(&l, s->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess ||
                (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
                return scuda(s, e, "loss");
            if (it == 0) first = l;
            last = l;
        }
    }
    if ((e = repack(s)) != cudaSuccess || (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
        return scuda(s, e, "pack");
    if ((st = check_err(s)) != GALS_OK) return st;  // a training product that timed out
    s->vp = vp;
    s->dt = dt;
    s->h = h;
    s->bound = true;
    if (report) {
        report->initial_loss = first;
        report->final_loss = last;
        report->steps = o->steps;
        report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return GALS_OK;
}

gals_status gals_surrogate_set_check(gals_surrogate *s, double tol_x, double tol_J, int samples)
{
    if (!s) return sfail(nullptr, GALS_ERR_ARG, "surrogate is NULL");
    if (!(tol_x >= 0.0) || !(tol_J >= 0.0) || samples < 0 || samples > 128)
        return sfail(s, GALS_ERR_ARG, "tolerances must be >= 0 and samples in 0..128");
    s->tol_x = (float)tol_x;
    s->tol_J = (float)tol_J;
    s->samples = samples;
    return GALS_OK;
}

gals_status gals_surrogate_stats(gals_surrogate *s, int64_t *tiles, int64_t *fallbacks, int reset)
{
    if (!s) return sfail(nullptr, GALS_ERR_ARG, "surrogate is NULL");
    unsigned long long h[2];
    cudaError_t e;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess ||
        (e = cudaMemcpy(h, s->counters, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return scuda(s, e, "counters");
    if (tiles) *tiles = (int64_t)h[0];
    if (fallbacks) *fallbacks = (int64_t)h[1];
    if (reset && (e = cudaMemset(s->counters, 0, sizeof(h))) != cudaSuccess) return scuda(s, e, "reset");
    return check_err(s);
}

gals_status gals_surrogate_get_params(const gals_surrogate *s, float *params, float *scales)
{
    if (!s) return sfail(nullptr, GALS_ERR_ARG, "surrogate is NULL");
    gals_surrogate *ms = const_cast<gals_surrogate *>(s);
    cudaError_t e;
    if (params) {
        if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess ||
            (e = cudaMemcpy(params, s->params, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return scuda(ms, e, "get params");
    }
    if (scales) std::memcpy(scales, s->ip.scale, sizeof(float) * OUT);
    return GALS_OK;
}

gals_status gals_surrogate_set_params(gals_surrogate *s, const float *params, const float *scales)
{
    if (!s || !params || !scales) return sfail(s, GALS_ERR_ARG, "NULL argument");
    for (int k = 0; k < OUT; ++k)
        if (!(scales[k] > 0.f) || !std::isfinite(scales[k])) return sfail(s, GALS_ERR_ARG, "bad scale %d", k);
    cudaError_t e;
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess ||
        (e = cudaMemcpy(s->params, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(s->scale_dev, scales, sizeof(float) * OUT, cudaMemcpyHostToDevice)) != cudaSuccess)
        return scuda(s, e, "set params");
    std::memcpy(s->ip.scale, scales, sizeof(float) * OUT);
    if ((e = repack(s)) != cudaSuccess || (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
        return scuda(s, e, "pack");
    s->bound = false;
    return GALS_OK;
}

gals_status gals_surrogate_bind(gals_surrogate *s, const gals_velocity *vel, double dt, double h)
{
    if (!s) return sfail(nullptr, GALS_ERR_ARG, "surrogate is NULL");
    if (!(dt > 0.0) || !(h > 0.0)) return sfail(s, GALS_ERR_ARG, "dt and h must be > 0");
    VelParams vp;
    gals_status st = check_field(s, vel, vp);
    if (st != GALS_OK) return st;
    s->vp = vp;
    s->dt = dt;
    s->h = h;
    s->bound = true;
    return GALS_OK;
}

gals_status gals_surrogate_forward(gals_surrogate *s, const float *inputs, int n, float *outputs)
{
    if (!s || !inputs || !outputs || n < 1 || n > 65536) return sfail(s, GALS_ERR_ARG, "bad arguments");
    cudaError_t e;
    if ((e = ensure_scratch(s, n)) != cudaSuccess) return scuda(s, e, "scratch");
    if ((e = cudaMemcpyAsync(s->Xn, inputs, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess ||
        (e = infer_points(s->ip, s->Xn, s->T, n, s->err_dev, s->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(outputs, s->T, sizeof(float) * OUT * n, cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
        return scuda(s, e, "forward");
    return check_err(s);
}

gals_status gals_surrogate_forward_device(gals_surrogate *s, const float *inputs, int64_t n, float *outputs)
{
    if (!s || !inputs || !outputs || n < 1 || n > ((int64_t)1 << 26)) return sfail(s, GALS_ERR_ARG, "bad arguments");
    cudaError_t e = infer_points(s->ip, inputs, outputs, (int)n, s->err_dev, s->stream);
    if (e != cudaSuccess) return scuda(s, e, "forward_device");
    return GALS_OK;
}

gals_status gals_surrogate_gradient(gals_surrogate *s, const float *inputs, const float *targets, int n,
                                    float *grad, double *loss)
{
    if (!s || !inputs || !targets || !grad || n < 1 || n > 65536) return sfail(s, GALS_ERR_ARG, "bad arguments");
    cudaError_t e;
    if ((e = ensure_scratch(s, n)) != cudaSuccess) return scuda(s, e, "scratch");
    double l = 0.0;
    if ((e = cudaMemcpyAsync(s->Xn, inputs, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->T, targets, sizeof(float) * OUT * n, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess ||
        (e = forward_train(s->params, s->Xn, n, s->Z, s->A, s->err_dev, s->stream)) != cudaSuccess ||
        (e = backward_train(s->params, s->Xn, s->T, n, s->Z, s->A, s->G0, s->G1, s->grad, s->loss_dev, s->one,
                            s->split, s->err_dev, s->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(grad, s->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&l, s->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
        return scuda(s, e, "gradient");
    gals_status st = check_err(s);
    if (st != GALS_OK) return st;
    if (loss) *loss = l;
    return GALS_OK;
}

gals_status gals_surrogate_targets(gals_surrogate *s, const gals_velocity *vel, double dt, double h,
                                   int substeps, const float *points, int n, float *targets)
{
    if (!s || !points || !targets || n < 1 || n > 65536 || substeps < 1 || !(dt > 0.0) || !(h > 0.0))
        return sfail(s, GALS_ERR_ARG, "bad arguments");
    VelParams vp;
    gals_status st = check_field(s, vel, vp);
    if (st != GALS_OK) return st;
    cudaError_t e;
    if ((e = ensure_scratch(s, n)) != cudaSuccess) return scuda(s, e, "scratch");
    if ((e = cudaMemcpyAsync(s->Xn, points, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess ||
        (e = launch_targets(vp, s->Xn, s->T, n, (float)dt, (float)h, substeps, s->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(targets, s->T, sizeof(float) * OUT * n, cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
        return scuda(s, e, "targets");
    return GALS_OK;
}

}  // extern "C"

namespace {
const char kMagic[8] = {'G', 'A', 'L', 'S', 'M', 'L', 'P', 1};

struct FileCloser {
    FILE *f;
    ~FileCloser() { if (f) fclose(f); }
};

template <class T>
bool put(FILE *f, const T *v, size_t n) { return fwrite(v, sizeof(T), n, f) == n; }
template <class T>
bool get(FILE *f, T *v, size_t n) { return fread(v, sizeof(T), n, f) == n; }
}  // namespace

gals_status gals_surrogate_save(const gals_surrogate *s, const char *path)
{
    if (!s || !path) return sfail(const_cast<gals_surrogate *>(s), GALS_ERR_ARG, "NULL argument");
    gals_surrogate *ms = const_cast<gals_surrogate *>(s);
    std::vector<float> p(NPARAM);
    float sc[OUT];
    gals_status st = gals_surrogate_get_params(s, p.data(), sc);
    if (st != GALS_OK) return st;
    FileCloser fc{fopen(path, "wb")};
    if (!fc.f) return sfail(ms, GALS_ERR_ARG, "cannot write %s", path);
    // version 2 where the bound field is WAVES2D (its rows follow), else version 1
    const int32_t version = s->bound && s->vp.kind == VK_WAVES2D ? 2 : 1;
    const int32_t hdr[3] = {version, (int32_t)NPARAM, (int32_t)OUT};
    const float tols[2] = {s->tol_x, s->tol_J};
    const int32_t samples = s->samples, bound = s->bound ? 1 : 0;
    bool ok = put(fc.f, kMagic, 8) && put(fc.f, hdr, 3) && put(fc.f, p.data(), NPARAM) && put(fc.f, sc, OUT) &&
              put(fc.f, tols, 2) && put(fc.f, &samples, 1) && put(fc.f, &bound, 1);
    if (ok && bound && s->vp.kind == VK_WAVES2D) {
        const double dh[2] = {s->dt, s->h};
        const int32_t kn[2] = {s->vp.kind, s->waves.count};
        ok = put(fc.f, dh, 2) && put(fc.f, kn, 2) && put(fc.f, s->waves.host.data(), s->waves.host.size());
    } else if (ok && bound) {
        const double dh[2] = {s->dt, s->h};
        const int32_t kn[2] = {s->vp.kind, s->vp.nmodes};
        const size_t m = (size_t)s->vp.nmodes;
        ok = put(fc.f, dh, 2) && put(fc.f, kn, 2) && put(fc.f, s->vp.mode_a, m) &&
             put(fc.f, s->vp.mode_kl, m) && put(fc.f, s->vp.mode_n, m) && put(fc.f, s->vp.mode_chi, m);
    }
    if (!ok) return sfail(ms, GALS_ERR_ARG, "write to %s failed", path);
    return GALS_OK;
}

gals_status gals_surrogate_load(gals_surrogate *s, const char *path)
{
    if (!s || !path) return sfail(s, GALS_ERR_ARG, "NULL argument");
    FileCloser fc{fopen(path, "rb")};
    if (!fc.f) return sfail(s, GALS_ERR_ARG, "cannot read %s", path);
    char magic[8];
    int32_t hdr[3];
    if (!get(fc.f, magic, 8) || std::memcmp(magic, kMagic, 8) != 0)
        return sfail(s, GALS_ERR_ARG, "%s is not a surrogate file", path);
    if (!get(fc.f, hdr, 3) || (hdr[0] != 1 && hdr[0] != 2) || hdr[1] != (int32_t)NPARAM || hdr[2] != (int32_t)OUT)
        return sfail(s, GALS_ERR_ARG, "%s: unsupported version or network shape", path);
    std::vector<float> p(NPARAM);
    float sc[OUT], tols[2];
    int32_t samples = 0, bound = 0;
    if (!get(fc.f, p.data(), NPARAM) || !get(fc.f, sc, OUT) || !get(fc.f, tols, 2) || !get(fc.f, &samples, 1) ||
        !get(fc.f, &bound, 1))
        return sfail(s, GALS_ERR_ARG, "%s is truncated", path);
    VelParams vp{};
    double dh[2] = {0.0, 0.0};
    std::vector<double> rows;
    if (bound && hdr[0] == 2) {
        int32_t kn[2];
        if (!get(fc.f, dh, 2) || !get(fc.f, kn, 2)) return sfail(s, GALS_ERR_ARG, "%s is truncated", path);
        if (kn[0] != VK_WAVES2D || kn[1] < 1 || kn[1] > GALS_MAX_WAVES || !(dh[0] > 0.0) || !(dh[1] > 0.0))
            return sfail(s, GALS_ERR_ARG, "%s: invalid bound field", path);
        rows.resize((size_t)6 * kn[1]);
        if (!get(fc.f, rows.data(), rows.size())) return sfail(s, GALS_ERR_ARG, "%s is truncated", path);
        gals_velocity wv{};
        wv.kind = GALS_VEL_WAVES2D;
        wv.trace = GALS_TRACE_RK3;
        wv.nmodes = kn[1];
        wv.modes = rows.data();
        char msg[200];
        if (velparams_from(2, &wv, vp, msg, sizeof(msg)) != GALS_OK)
            return sfail(s, GALS_ERR_ARG, "%s: invalid bound field (%s)", path, msg);
        bool changed = false;
        cudaError_t e = s->waves.upload(&wv, s->stream, &changed);
        if (e != cudaSuccess) return scuda(s, e, "wave table");
        s->waves.bind(vp);
    } else if (bound) {
        int32_t kn[2];
        if (!get(fc.f, dh, 2) || !get(fc.f, kn, 2)) return sfail(s, GALS_ERR_ARG, "%s is truncated", path);
        if (kn[0] != VK_FOURIER2D || kn[1] < 1 || kn[1] > kMaxModes || !(dh[0] > 0.0) || !(dh[1] > 0.0))
            return sfail(s, GALS_ERR_ARG, "%s: invalid bound field", path);
        vp.kind = kn[0];
        vp.nmodes = kn[1];
        const size_t m = (size_t)kn[1];
        if (!get(fc.f, vp.mode_a, m) || !get(fc.f, vp.mode_kl, m) || !get(fc.f, vp.mode_n, m) ||
            !get(fc.f, vp.mode_chi, m))
            return sfail(s, GALS_ERR_ARG, "%s is truncated", path);
    }
    if (!(tols[0] >= 0.f) || !(tols[1] >= 0.f) || samples < 0)
        return sfail(s, GALS_ERR_ARG, "%s: invalid residual-check settings", path);
    gals_status st = gals_surrogate_set_params(s, p.data(), sc);
    if (st != GALS_OK) return st;
    s->tol_x = tols[0];
    s->tol_J = tols[1];
    s->samples = samples;
    if (bound) {
        s->vp = vp;
        s->dt = dh[0];
        s->h = dh[1];
        s->bound = true;
    }
    return GALS_OK;
}
