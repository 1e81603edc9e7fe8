// capi.cu -- implementation of the C ABI declared in include/gals.h.
//
// A grid owns two device state buffers (A/B ping-pong), each holding all planes of the
// state in SoA form with a row pitch that is a multiple of 4 floats (16-byte rows).
// gals_step issues one kernel launch per step (plus the approach-A reconstruction in the
// FULL layout); runs of more than one step are captured once into a CUDA graph and
// replayed.  The grid time lives on the device too, so a cached graph is valid for any
// start time: step s of a call reads t = t_dev + s*dt, and the graph ends by advancing
// t_dev.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gals.h"
#include "gals_internal.h"
#include "capi_internal.h"

using namespace gals;

namespace {

char g_create_err[256] = "";

struct GraphEntry {
    // key
    int nsteps, cur, first_explicit, trace, layout;
    double dt;
    VelParams vp;
    const void *sur;      // surrogate (its scales and check settings are baked in)
    float sur_key[9];
    // value
    cudaGraphExec_t exec;
    int64_t launches;     // kernel launches the graph holds
};

}  // namespace

// at most this many bands in gals_step_host (rows in 2D, z-levels in 3D)
constexpr int kHostBands = 16;
#ifndef GALS_STEP_BANDS
#define GALS_STEP_BANDS 4
#endif
constexpr int kStepBands = GALS_STEP_BANDS;  // row bands of a captured multi-step 2D call
// Longest run of steps one cached graph holds (even: a whole graph leaves the ping-pong
// buffers as it found them); longer calls replay it.
constexpr int kGraphSteps = 256;

struct gals_grid {
    int dim = 0;
    int n[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, h[3] = {1, 1, 1};
    int layout = GALS_LAYOUT_FULL;
    int cross = GALS_CROSS_CENTRAL;   // mixed derivatives: approach A (planes) or B (per cell)
    int nplanes = 0;
    Geom geom{};
    float *buf[2] = {nullptr, nullptr};
    int cur = 0;
    bool has_state = false;
    bool cross_explicit = false;  // COMPACT: buffer cur holds given mixed derivatives to use once
    double t = 0.0;
    int64_t steps = 0;
    double *t_dev = nullptr;
    CUtensorMap maps[2][3];       // TMA maps per buffer: [b][0] COMPACT box, [b][1] FULL box,
                                  // [b][2] 3D reconstruction box
    float *trace_buf = nullptr;   // surrogate trace of the current step: dx, dy, J (6 planes)
    char *pt_buf = nullptr;       // gals_eval_points: device staging of host points / results
    size_t pt_cap = 0;
    int *err_dev = nullptr;       // device error word written by kernels (bounded waits)
    StageCoef *coef = nullptr;    // per-step stage coefficients of the current call
    int coef_cap = 0;
    DiagOut *diag_dev = nullptr;
    double *diag_partials = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // gals_step_host: copy-in and copy-out streams, one event per band and direction
    cudaStream_t hs_in = nullptr, hs_out = nullptr;
    cudaEvent_t hs_enter = nullptr, hs_in_ev[kHostBands] = {}, hs_step_ev[kHostBands] = {};
    cudaEvent_t hs_out_ev[kHostBands] = {};  // copy-out of each band, of the last host step
    cudaEvent_t hs_done = nullptr;           // its last copy-out
    bool hs_pending = false;      // an asynchronous host step's copies may still run
    std::vector<GraphEntry> graphs;
    // captured multi-step 2D calls: one stream per row band (they carry no work outside a
    // capture) and two generations of per-band events
    cudaStream_t band_s[kStepBands] = {};
    cudaEvent_t band_fork = nullptr, band_ev[2][kStepBands] = {};
    int64_t last_launches = 0;    // kernel launches of the last gals_step call
    WaveStore waves;              // WAVES2D: device copy of the field's modes
    float *wamp = nullptr;        // WAVES2D: amplitudes of a call's steps [step][stage][mode]
    int64_t wamp_cap = 0;
    int loop = GALS_LOOP_LAUNCHES; // time loop of multi-step calls (gals_set_time_loop)
    int *run_ctl = nullptr;       // persistent 2D loop: ticket, abort word, per-tile flags
    char err[256] = "";
};

namespace {

gals_status fail(gals_grid *g, gals_status st, const char *fmt, ...)
{
    char *dst = g ? g->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return st;
}

#ifdef GALS_CHECKED
// test hook of the checked build (gals_checked_wait_test), read by gals_create_grid
uint32_t g_test_wait_polls = 1u << 24;
int g_test_skip_copy = 0;
#endif

gals_status cuda_fail(gals_grid *g, cudaError_t e, const char *what)
{
    // the runtime keeps a failed call's error as the thread's last error; a non-sticky one
    // (a failed allocation) would otherwise fail the next launch check of any handle
    cudaGetLastError();
    return fail(g, e == cudaErrorMemoryAllocation ? GALS_ERR_NOMEM : GALS_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// After gals_step_host_async: the grid stream waits for its last copy-out before any other
// call touches the state buffers (the host streams run on their own until then).
cudaError_t join_host_steps(gals_grid *g)
{
    if (!g->hs_pending) return cudaSuccess;
    g->hs_pending = false;
    return cudaStreamWaitEvent(g->stream, g->hs_done, 0);
}

int full_planes(int dim) { return dim == 2 ? 4 : 8; }

bool finite3(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

gals_status make_velparams(gals_grid *g, const gals_velocity *v, VelParams &vp)
{
    char msg[200];
    gals_status st = gals::velparams_from(g->dim, v, vp, msg, sizeof(msg));
    if (st != GALS_OK) return fail(g, st, "%s", msg);
    return GALS_OK;
}

// Kernel launch descriptor of step s of a call, from buffer cur to buffer cur ^ 1.
StepLaunch step_launch(gals_grid *g, const VelParams &vp, int trace, double dt, int s, int cur,
                       bool first_explicit)
{
    StepLaunch a{};
    a.in = g->buf[cur];
    a.out = g->buf[cur ^ 1];
    a.geom = g->geom;
    a.vp = vp;
    a.coef = g->coef + s;
    a.dt = dt;
    a.tmap3 = &g->maps[cur][0];
    a.tmap4 = &g->maps[cur][1];
    a.tmap_cross = &g->maps[cur ^ 1][2];
    a.err = g->err_dev;
    a.trace = trace == GALS_TRACE_EULER      ? TR_EULER
              : trace == GALS_TRACE_SURROGATE ? TR_GIVEN
              : trace == GALS_TRACE_HEUN_PSI  ? TR_HEUN
                                              : TR_RK3;
    if (g->cross == GALS_CROSS_CELL) {
        a.cross_in = CROSS_CELL;  // approach B: mixed derivatives per cell, none stored
        a.write_cross = 0;
    } else if (g->layout == GALS_LAYOUT_FULL) {
        a.cross_in = CROSS_PLANE;
        a.write_cross = 1;
    } else {
        a.cross_in = (s == 0 && first_explicit) ? CROSS_PLANE : CROSS_RECON;
        a.write_cross = 0;
    }
    return a;
}

// Whether a call of nsteps steps runs as one persistent launch (launch_step2d_run): 2D,
// FULL layout, approach A, an analytic trace, and feet (at most reach[a] cells from their
// node along axis a) within the launch's dependency radius.
bool use_run(const gals_grid *g, int trace, int nsteps, const double reach[2])
{
    return g->loop == GALS_LOOP_PERSISTENT && g->dim == 2 && nsteps >= 2 && g->layout == GALS_LAYOUT_FULL &&
           g->cross == GALS_CROSS_CENTRAL && trace != GALS_TRACE_SURROGATE &&
           reach[0] <= run2d_max_cells(0) && reach[1] <= run2d_max_cells(1);
}

// Row bands of a captured multi-step 2D call.  Step s of band b reads the rows of step
// s - 1 that its feet reach (plus the staged tile's halo row and the cubic cell) and
// overwrites rows that step s - 1 of the neighbouring bands read, so with bands at least
// reach + 4 rows high it depends on bands b - 1, b, b + 1 of step s - 1 only: in the graph a
// band starts as soon as those three are done, and the next step's first bands fill the
// tail of the current one.  Whole tile rows per band; n < 2 means one launch per step.
struct StepBands {
    int n = 0;
    int row[kStepBands + 1] = {};
};

StepBands step_bands(const gals_grid *g, int trace, int nsteps, const double reach[2])
{
    StepBands sb;
    if (g->dim != 2 || nsteps < 2 || trace == GALS_TRACE_SURROGATE || !(reach[1] < 1e6)) return sb;
    const int unit = band_unit(2);
    const int tile_rows = (g->geom.n1 + unit - 1) / unit;
    const int min_rows = (int)std::ceil(reach[1]) + 4;
    const int min_tiles = std::max(2, (min_rows + unit - 1) / unit);
    const int n = std::min(kStepBands, tile_rows / min_tiles);
    if (n < 2) return sb;
    sb.n = n;
    for (int b = 0; b <= n; ++b) sb.row[b] = std::min(g->geom.n1, (int)((int64_t)b * tile_rows / n) * unit);
    sb.row[n] = g->geom.n1;
    return sb;
}

// The band streams and events, made once per grid (all or none).
cudaError_t make_band_streams(gals_grid *g)
{
    if (g->band_fork) return cudaSuccess;
    cudaStream_t st[kStepBands] = {};
    cudaEvent_t ev[2][kStepBands] = {}, fork = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int b = 0; b < kStepBands && e == cudaSuccess; ++b) {
        e = cudaStreamCreateWithFlags(&st[b], cudaStreamNonBlocking);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k][b], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        for (int b = 0; b < kStepBands; ++b) {
            if (st[b]) cudaStreamDestroy(st[b]);
            for (int k = 0; k < 2; ++k)
                if (ev[k][b]) cudaEventDestroy(ev[k][b]);
        }
        if (fork) cudaEventDestroy(fork);
        return e;
    }
    std::memcpy(g->band_s, st, sizeof(st));
    std::memcpy(g->band_ev, ev, sizeof(ev));
    g->band_fork = fork;
    return cudaSuccess;
}

// The kernels of one gals_step call on the grid stream; `launches` counts them (the
// coefficient table and clock kernels included).
cudaError_t issue_steps(gals_grid *g, const VelParams &vp, int trace, double dt, int nsteps,
                        bool first_explicit, int64_t &launches, const mlp::InferParams *ip = nullptr,
                        const mlp::Check *chk = nullptr, bool run = false, const StepBands *bands = nullptr)
{
    int cur = g->cur;
    launches = (vp.kind == VK_WAVES2D ? 2 : 1) + 1;  // coefficients (+ wave amplitudes), clock
    cudaError_t ce = launch_coef_table(g->coef, vp, g->t_dev, dt, nsteps, g->stream);
    if (ce != cudaSuccess) return ce;
    if (bands && bands->n >= 2) {
        // fork the band streams off the grid stream, chain each band on its two neighbours'
        // previous step, join them back before the clock advances
        const int nb = bands->n;
        if ((ce = cudaEventRecord(g->band_fork, g->stream)) != cudaSuccess) return ce;
        for (int b = 0; b < nb; ++b)
            if ((ce = cudaStreamWaitEvent(g->band_s[b], g->band_fork, 0)) != cudaSuccess) return ce;
        for (int s = 0; s < nsteps; ++s) {
            for (int b = 0; b < nb; ++b) {
                cudaStream_t bs = g->band_s[b];
                if (s > 0) {
                    const cudaEvent_t *prev = g->band_ev[(s - 1) & 1];
                    if (b > 0 && (ce = cudaStreamWaitEvent(bs, prev[b - 1], 0)) != cudaSuccess) return ce;
                    if (b + 1 < nb && (ce = cudaStreamWaitEvent(bs, prev[b + 1], 0)) != cudaSuccess) return ce;
                }
                StepLaunch a = step_launch(g, vp, trace, dt, s, cur, first_explicit);
                a.band_lo = bands->row[b];
                a.band_hi = bands->row[b + 1];
                if ((ce = launch_step2d(a, bs)) != cudaSuccess) return ce;
                if ((ce = cudaEventRecord(g->band_ev[s & 1][b], bs)) != cudaSuccess) return ce;
            }
            cur ^= 1;
        }
        for (int b = 0; b < nb; ++b)
            if ((ce = cudaStreamWaitEvent(g->stream, g->band_ev[(nsteps - 1) & 1][b], 0)) != cudaSuccess) return ce;
        launches += (int64_t)nsteps * nb;
        return launch_advance_time(g->t_dev, nsteps, dt, g->stream);
    }
    if (run) {
        // persistent launches of fewer than 2^31 - 2^20 work items (tiles x steps) each:
        // the ticket counter also counts one final draw per block
        const int tiles = run2d_tiles(g->geom);
        const int chunk = (int)((INT32_MAX - (1 << 20)) / tiles);
        for (int s0 = 0; s0 < nsteps; s0 += chunk) {
            StepLaunch a = step_launch(g, vp, trace, dt, 0, cur, first_explicit);
            RunLaunch r{};
            r.buf[0] = g->buf[0];
            r.buf[1] = g->buf[1];
            r.cur = cur;
            r.geom = g->geom;
            r.vp = vp;
            r.coef = g->coef + s0;
            r.dt = dt;
            r.trace = a.trace;
            r.tmap[0] = &g->maps[0][1];
            r.tmap[1] = &g->maps[1][1];
            r.err = g->err_dev;
            r.ctl = g->run_ctl;
            r.nsteps = nsteps - s0 < chunk ? nsteps - s0 : chunk;
            if ((ce = cudaMemsetAsync(g->run_ctl, 0, sizeof(int) * (4 + (size_t)tiles), g->stream)) != cudaSuccess ||
                (ce = launch_step2d_run(r, g->stream)) != cudaSuccess)
                return ce;
            ++launches;
            if (r.nsteps & 1) cur ^= 1;
        }
        return launch_advance_time(g->t_dev, nsteps, dt, g->stream);
    }
    for (int s = 0; s < nsteps; ++s) {
        StepLaunch a = step_launch(g, vp, trace, dt, s, cur, first_explicit);
        if (trace == GALS_TRACE_SURROGATE) {
            // learned trace of this step (with RK3 fallback per tile), then the Hermite stage
            ce = mlp::launch_mlp_trace(*ip, g->geom, vp, g->coef + s, g->t_dev, s, dt, g->trace_buf,
                                       *chk, g->stream);
            if (ce != cudaSuccess) return ce;
            a.vp.given = g->trace_buf;
            a.vp.given_plane = g->geom.plane;
            ++launches;
        }
        cudaError_t e = g->dim == 2 ? launch_step2d(a, g->stream) : launch_step3d(a, g->stream);
        if (e != cudaSuccess) return e;
        launches += (g->dim == 3 && a.write_cross) ? 2 : 1;  // 3D FULL: step + reconstruction
        cur ^= 1;
    }
    return launch_advance_time(g->t_dev, nsteps, dt, g->stream);
}

bool same_key(const GraphEntry &e, int nsteps, int cur, int fe, int trace, int layout, double dt,
              const VelParams &vp, const void *sur, const float *sur_key)
{
    return e.nsteps == nsteps && e.cur == cur && e.first_explicit == fe && e.trace == trace &&
           e.layout == layout && e.dt == dt && std::memcmp(&e.vp, &vp, sizeof(vp)) == 0 &&
           e.sur == sur && std::memcmp(e.sur_key, sur_key, sizeof(e.sur_key)) == 0;
}

}  // namespace

extern "C" {

gals_status gals_set_time_loop(gals_grid *g, int mode)
{
    if (!g) return fail(nullptr, GALS_ERR_ARG, "grid is NULL");
    if (mode != GALS_LOOP_LAUNCHES && mode != GALS_LOOP_PERSISTENT) return fail(g, GALS_ERR_ARG, "unknown time loop");
    if (mode != g->loop) {
        // cached graphs hold the other loop
        cudaError_t e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) return cuda_fail(g, e, "sync");
        for (auto &ge : g->graphs) cudaGraphExecDestroy(ge.exec);
        g->graphs.clear();
        g->loop = mode;
    }
    return GALS_OK;
}

gals_status gals_last_step_launches(const gals_grid *g, int64_t *launches)
{
    if (!g || !launches) return fail(nullptr, GALS_ERR_ARG, "grid or output is NULL");
    *launches = g->last_launches;
    return GALS_OK;
}

gals_status gals_checked_wait_test(uint32_t polls, int skip_copy)
{
#ifdef GALS_CHECKED
    if (polls < 1) return fail(nullptr, GALS_ERR_ARG, "polls must be >= 1");
    g_test_wait_polls = polls;
    g_test_skip_copy = skip_copy != 0;
    return GALS_OK;
#else
    (void)polls;
    (void)skip_copy;
    return fail(nullptr, GALS_ERR_UNSUPPORTED,
                "the wait test hook exists only in the checked build (libgals_checked.so)");
#endif
}

const char *gals_version(void) { return "gals-gb300 0.1 (sm_103a)"; }

const char *gals_last_error(const gals_grid *g) { return g ? g->err : g_create_err; }

double gals_time(const gals_grid *g) { return g ? g->t : 0.0; }

gals_status gals_create_grid(const gals_grid_desc *d, gals_grid **out)
{
    if (!out) return fail(nullptr, GALS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!d) return fail(nullptr, GALS_ERR_ARG, "descriptor is NULL");
    if (d->dim != 2 && d->dim != 3) return fail(nullptr, GALS_ERR_ARG, "dim must be 2 or 3");
    if (d->layout != GALS_LAYOUT_FULL && d->layout != GALS_LAYOUT_COMPACT)
        return fail(nullptr, GALS_ERR_ARG, "unknown layout %d", d->layout);
    if (d->cross_scheme != GALS_CROSS_CENTRAL && d->cross_scheme != GALS_CROSS_CELL)
        return fail(nullptr, GALS_ERR_ARG, "unknown cross scheme %d", d->cross_scheme);
    for (int i = 0; i < d->dim; ++i) {
        if (d->n[i] < 4) return fail(nullptr, GALS_ERR_ARG, "n[%d] = %d < 4", i, d->n[i]);
        if (!std::isfinite(d->lo[i]) || !std::isfinite(d->hi[i]) || !(d->hi[i] > d->lo[i]))
            return fail(nullptr, GALS_ERR_ARG, "axis %d: need finite lo < hi", i);
    }
    {
        char msg[160];
        const int n3[3] = {d->n[0], d->n[1], d->dim == 3 ? d->n[2] : 1};
        if (!gals::grid_size_ok(d->dim, n3, msg, sizeof(msg))) return fail(nullptr, GALS_ERR_ARG, "%s", msg);
    }
    gals_grid *g = new (std::nothrow) gals_grid();
    if (!g) return fail(nullptr, GALS_ERR_NOMEM, "host allocation failed");
    g->dim = d->dim;
    g->layout = d->layout;
    g->cross = d->cross_scheme;
    g->nplanes = full_planes(d->dim);
    for (int i = 0; i < 3; ++i) {
        g->n[i] = i < d->dim ? d->n[i] : 1;
        g->lo[i] = i < d->dim ? d->lo[i] : 0.0;
        g->hi[i] = i < d->dim ? d->hi[i] : 1.0;
        g->h[i] = i < d->dim ? (g->hi[i] - g->lo[i]) / (g->n[i] - 1) : 1.0;
    }
    Geom &G = g->geom;
    G.n0 = g->n[0]; G.n1 = g->n[1]; G.n2 = g->n[2];
    G.pitch = (g->n[0] + 3) / 4 * 4;
    const int64_t plane = (int64_t)G.pitch * G.n1 * G.n2;
    G.plane = (plane + 63) / 64 * 64;  // 256-byte aligned planes
    G.h0 = (float)g->h[0]; G.h1 = (float)g->h[1]; G.h2 = (float)g->h[2];
    G.ih0 = (float)(1.0 / g->h[0]); G.ih1 = (float)(1.0 / g->h[1]); G.ih2 = (float)(1.0 / g->h[2]);
    G.i2h0 = (float)(0.5 / g->h[0]); G.i2h1 = (float)(0.5 / g->h[1]); G.i2h2 = (float)(0.5 / g->h[2]);
    G.lo0 = (float)g->lo[0]; G.lo1 = (float)g->lo[1]; G.lo2 = (float)g->lo[2];
#ifdef GALS_CHECKED
    G.wait_polls = g_test_wait_polls;
    G.skip_copy = g_test_skip_copy;
#endif

    cudaError_t e;
    if (d->cuda_stream) {
        g->stream = (cudaStream_t)d->cuda_stream;
    } else {
        if ((e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking)) != cudaSuccess) {
            gals_status st = cuda_fail(nullptr, e, "cudaStreamCreate");
            delete g;
            return st;
        }
        g->own_stream = true;
    }
    const size_t bytes = (size_t)G.plane * g->nplanes * sizeof(float);
    for (int b = 0; b < 2; ++b) {
        if ((e = cudaMalloc(&g->buf[b], bytes)) != cudaSuccess) {
            gals_status st = cuda_fail(nullptr, e, "cudaMalloc(state)");
            gals_destroy_grid(g);
            return st;
        }
    }
    if ((e = cudaMalloc(&g->t_dev, sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&g->err_dev, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&g->diag_dev, sizeof(DiagOut))) != cudaSuccess ||
        (e = cudaMalloc(&g->diag_partials, sizeof(double) * diag_partials_needed())) != cudaSuccess) {
        gals_status st = cuda_fail(nullptr, e, "cudaMalloc(aux)");
        gals_destroy_grid(g);
        return st;
    }
#ifdef GALS_CHECKED
    g->geom.chk = g->err_dev;  // the checked build's bounds errors land in the error word
#endif
    if ((e = cudaMemsetAsync(g->err_dev, 0, sizeof(int), g->stream)) != cudaSuccess) {
        gals_status st = cuda_fail(nullptr, e, "cudaMemset");
        gals_destroy_grid(g);
        return st;
    }
    // TMA maps of each buffer with the step kernels' tile boxes:
    // 2D (x, y, plane), 3D (x, y, z, plane); 3D also the reconstruction kernel's box
    for (int b = 0; b < 2; ++b)
        for (int v = 0; v < (g->dim == 2 ? 2 : 3); ++v) {
            if (g->dim == 2) {
                const int np = v == 0 ? 3 : 4;
                const uint64_t dims[3] = {(uint64_t)G.n0, (uint64_t)G.n1, (uint64_t)np};
                const uint64_t strides[2] = {(uint64_t)G.pitch * 4, (uint64_t)G.plane * 4};
                uint32_t box[3];
                tile_box2d(np, box);
                e = make_tile_map(&g->maps[b][v], g->buf[b], 3, dims, strides, box);
            } else {
                uint32_t box[4];
                if (v < 2)
                    tile_box3d(v == 0, box);
                else
                    recon_box3d(box);
                const uint64_t np = v == 2 ? 8 : box[3];  // the reconstruction box starts at plane 2
                const uint64_t dims[4] = {(uint64_t)G.n0, (uint64_t)G.n1, (uint64_t)G.n2, np};
                const uint64_t strides[3] = {(uint64_t)G.pitch * 4, (uint64_t)G.pitch * G.n1 * 4,
                                             (uint64_t)G.plane * 4};
                e = make_tile_map(&g->maps[b][v], g->buf[b], 4, dims, strides, box);
            }
            if (e != cudaSuccess) {
                gals_status st = cuda_fail(nullptr, e, "TMA descriptor");
                gals_destroy_grid(g);
                return st;
            }
        }
    // zero both buffers so that pitch padding never holds garbage
    for (int b = 0; b < 2; ++b)
        if ((e = cudaMemsetAsync(g->buf[b], 0, bytes, g->stream)) != cudaSuccess) {
            gals_status st = cuda_fail(nullptr, e, "cudaMemset");
            gals_destroy_grid(g);
            return st;
        }
    *out = g;
    return GALS_OK;
}

gals_status gals_destroy_grid(gals_grid *g)
{
    if (!g) return GALS_OK;
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (auto &ge : g->graphs) cudaGraphExecDestroy(ge.exec);
    for (int b = 0; b < 2; ++b) cudaFree(g->buf[b]);
    cudaFree(g->t_dev);
    cudaFree(g->err_dev);
    cudaFree(g->trace_buf);
    cudaFree(g->pt_buf);
    cudaFree(g->coef);
    cudaFree(g->diag_dev);
    cudaFree(g->diag_partials);
    cudaFree(g->run_ctl);
    cudaFree(g->wamp);
    g->waves.release();
    for (cudaStream_t hs : {g->hs_in, g->hs_out})
        if (hs) {
            cudaStreamSynchronize(hs);
            cudaStreamDestroy(hs);
        }
    if (g->hs_enter) cudaEventDestroy(g->hs_enter);
    for (int b = 0; b < kHostBands; ++b) {
        if (g->hs_in_ev[b]) cudaEventDestroy(g->hs_in_ev[b]);
        if (g->hs_step_ev[b]) cudaEventDestroy(g->hs_step_ev[b]);
        if (g->hs_out_ev[b]) cudaEventDestroy(g->hs_out_ev[b]);
    }
    if (g->hs_done) cudaEventDestroy(g->hs_done);
    for (int b = 0; b < kStepBands; ++b) {
        if (g->band_s[b]) cudaStreamDestroy(g->band_s[b]);
        for (int k = 0; k < 2; ++k)
            if (g->band_ev[k][b]) cudaEventDestroy(g->band_ev[k][b]);
    }
    if (g->band_fork) cudaEventDestroy(g->band_fork);
    if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
    delete g;
    return GALS_OK;
}

gals_status gals_set_state(gals_grid *g, const float *const *fields, int nfields, int memspace,
                           double t0, int flags)
{
    NvtxRange nvtx_range("gals_set_state");
    if (!g) return fail(nullptr, GALS_ERR_ARG, "grid is NULL");
    if (cudaError_t je = join_host_steps(g); je != cudaSuccess) return cuda_fail(g, je, "join host steps");
    if (!fields) return fail(g, GALS_ERR_ARG, "fields is NULL");
    const int core = 1 + g->dim;
    if (nfields != core && nfields != g->nplanes)
        return fail(g, GALS_ERR_ARG, "nfields must be %d or %d", core, g->nplanes);
    if (memspace != GALS_MEM_HOST && memspace != GALS_MEM_DEVICE)
        return fail(g, GALS_ERR_ARG, "bad memspace %d", memspace);
    if (!std::isfinite(t0)) return fail(g, GALS_ERR_ARG, "t0 is not finite");
    for (int p = 0; p < nfields; ++p)
        if (!fields[p]) return fail(g, GALS_ERR_ARG, "fields[%d] is NULL", p);
    const Geom &G = g->geom;
    const size_t row = (size_t)g->n[0] * sizeof(float);
    const size_t rows = (size_t)g->n[1] * g->n[2];
    const cudaMemcpyKind kind = memspace == GALS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    float *dst = g->buf[g->cur];
    cudaError_t e;
    for (int p = 0; p < nfields; ++p) {
        e = cudaMemcpy2DAsync(dst + p * G.plane, (size_t)G.pitch * sizeof(float), fields[p], row, row,
                              rows, kind, g->stream);
        if (e != cudaSuccess) return cuda_fail(g, e, "set_state copy");
    }
    const bool recon = nfields == core || (flags & GALS_SET_RECON_CROSS);
    if (g->cross == GALS_CROSS_CELL) {
        // approach B keeps no node values of the mixed derivatives
        for (int p = core; p < g->nplanes; ++p)
            if ((e = cudaMemsetAsync(dst + p * G.plane, 0, sizeof(float) * (size_t)G.plane, g->stream)) != cudaSuccess)
                return cuda_fail(g, e, "set_state zero");
    } else if (recon) {
        if ((e = launch_recon(g->dim, G, dst, g->stream)) != cudaSuccess) return cuda_fail(g, e, "recon");
    }
    g->cross_explicit = (g->layout == GALS_LAYOUT_COMPACT) && !recon && g->cross != GALS_CROSS_CELL;
    g->t = t0;
    g->steps = 0;
    if ((e = cudaMemcpyAsync(g->t_dev, &g->t, sizeof(double), cudaMemcpyHostToDevice, g->stream)) != cudaSuccess)
        return cuda_fail(g, e, "set time");
    // the sources and the host time word must be consumed before returning
    if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cuda_fail(g, e, "set_state sync");
    g->has_state = true;
    return GALS_OK;
}

gals_status gals_step(gals_grid *g, const gals_velocity *v, double dt, int nsteps)
{
    NvtxRange nvtx_range("gals_step");
    if (!g) return fail(nullptr, GALS_ERR_ARG, "grid is NULL");
    if (cudaError_t je = join_host_steps(g); je != cudaSuccess) return cuda_fail(g, je, "join host steps");
    if (!g->has_state) return fail(g, GALS_ERR_STATE, "no state loaded");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(g, GALS_ERR_ARG, "dt must be finite and > 0");
    if (nsteps < 0) return fail(g, GALS_ERR_ARG, "nsteps must be >= 0");
    VelParams vp;
    gals_status st = make_velparams(g, v, vp);
    if (st != GALS_OK) return st;
    mlp::InferParams ip{};
    mlp::Check chk{};
    const void *sur = nullptr;
    float sur_key[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    cudaError_t e;
    if (v->kind == GALS_VEL_WAVES2D && nsteps > 0) {
        // the modes in device memory, and room for the amplitude table of a run of steps
        bool changed = false;
        if ((e = g->waves.upload(v, g->stream, &changed)) != cudaSuccess) return cuda_fail(g, e, "wave table");
        const int64_t need = (int64_t)std::min(nsteps, kGraphSteps) * 3 * v->nmodes;
        if (need > g->wamp_cap) {
            if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cuda_fail(g, e, "sync");
            for (auto &ge : g->graphs) cudaGraphExecDestroy(ge.exec);  // they use the old table
            g->graphs.clear();
            cudaFree(g->wamp);
            g->wamp = nullptr;
            g->wamp_cap = 0;
            if ((e = cudaMalloc(&g->wamp, sizeof(float) * (size_t)need)) != cudaSuccess)
                return cuda_fail(g, e, "cudaMalloc(wave amplitudes)");
            g->wamp_cap = need;
        }
        g->waves.bind(vp);
        vp.wamp = g->wamp;
    }
    if (v->trace == GALS_TRACE_SURROGATE) {
        if (g->dim != 2) return fail(g, GALS_ERR_UNSUPPORTED, "the surrogate trace is 2D");
        char msg[200];
        st = surrogate_for_step(v->surrogate, v, vp, dt, g->h[0], g->h[1], ip, chk, msg, sizeof(msg));
        if (st != GALS_OK) return fail(g, st, "%s", msg);
        chk.err = g->err_dev;
        sur = v->surrogate;
        for (int k = 0; k < 6; ++k) sur_key[k] = ip.scale[k];
        sur_key[6] = chk.tol_x;
        sur_key[7] = chk.tol_J;
        sur_key[8] = (float)chk.samples;
    }
    if (nsteps == 0) {
        g->last_launches = 0;
        return GALS_OK;
    }
    const bool fe = g->cross_explicit;
    if (sur && !g->trace_buf) {
        if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cuda_fail(g, e, "sync");
        if ((e = cudaMalloc(&g->trace_buf, sizeof(float) * 6 * (size_t)g->geom.plane)) != cudaSuccess)
            return cuda_fail(g, e, "cudaMalloc(trace buffer)");
    }
    if (std::min(nsteps, kGraphSteps) > g->coef_cap) {
        // grow the coefficient table; cached graphs refer to the old one
        if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cuda_fail(g, e, "sync");
        for (auto &ge : g->graphs) cudaGraphExecDestroy(ge.exec);
        g->graphs.clear();
        cudaFree(g->coef);
        g->coef = nullptr;
        g->coef_cap = 0;
        const int cap = std::max(64, std::min(nsteps, kGraphSteps));
        if ((e = cudaMalloc(&g->coef, sizeof(StageCoef) * (size_t)cap)) != cudaSuccess)
            return cuda_fail(g, e, "cudaMalloc(coefficient table)");
        g->coef_cap = cap;
    }
    const double vmax = speed_bound(v, g->dim, g->lo, g->hi);
    const double reach[2] = {dt * vmax / g->h[0], dt * vmax / g->h[1]};
    const bool run = use_run(g, v->trace, std::min(nsteps, kGraphSteps), reach);
    if (run && !g->run_ctl) {
        if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cuda_fail(g, e, "sync");
        if ((e = cudaMalloc(&g->run_ctl, sizeof(int) * (4 + (size_t)run2d_tiles(g->geom)))) != cudaSuccess)
            return cuda_fail(g, e, "cudaMalloc(time-loop control)");
    }
    // runs of up to kGraphSteps steps: one step as launches, more from a cached graph; each
    // graph computes its coefficients from the device clock and advances it, so the graph of
    // one run serves every run of the same length, buffer parity and first-step layout
    int64_t total = 0;
    const char *what = "";
    auto run_one = [&](int cs, bool fe_c) -> cudaError_t {
        cudaError_t ce;
        if (cs == 1) {
            int64_t nl = 0;
            if ((ce = issue_steps(g, vp, v->trace, dt, 1, fe_c, nl, &ip, &chk)) != cudaSuccess) {
                what = "step launch";
                return ce;
            }
            total += nl;
            return cudaSuccess;
        }
        GraphEntry *hit = nullptr;
        for (auto &ge : g->graphs)
            if (same_key(ge, cs, g->cur, fe_c, v->trace, g->layout, dt, vp, sur, sur_key)) { hit = &ge; break; }
        if (!hit) {
            const StepBands bands = run ? StepBands{} : step_bands(g, v->trace, cs, reach);
            if (bands.n >= 2 && (ce = make_band_streams(g)) != cudaSuccess) { what = "band streams"; return ce; }
            cudaGraph_t graph;
            if ((ce = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
                what = "begin capture";
                return ce;
            }
            int64_t nl = 0;
            const cudaError_t le = issue_steps(g, vp, v->trace, dt, cs, fe_c, nl, &ip, &chk, run, &bands);
            ce = cudaStreamEndCapture(g->stream, &graph);
            if (le != cudaSuccess) {
                if (ce == cudaSuccess) cudaGraphDestroy(graph);
                what = "capture launch";
                return le;
            }
            if (ce != cudaSuccess) { what = "end capture"; return ce; }
            cudaGraphExec_t exec;
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) { what = "graph instantiate"; return ce; }
            if (g->graphs.size() >= 8) {
                cudaGraphExecDestroy(g->graphs.front().exec);
                g->graphs.erase(g->graphs.begin());
            }
            GraphEntry ge;
            ge.nsteps = cs; ge.cur = g->cur; ge.first_explicit = fe_c; ge.trace = v->trace;
            ge.layout = g->layout; ge.dt = dt; ge.vp = vp; ge.exec = exec;
            ge.sur = sur;
            ge.launches = nl;
            std::memcpy(ge.sur_key, sur_key, sizeof(sur_key));
            g->graphs.push_back(ge);
            hit = &g->graphs.back();
        }
        if ((ce = cudaGraphLaunch(hit->exec, g->stream)) != cudaSuccess) { what = "graph launch"; return ce; }
        total += hit->launches;
        return cudaSuccess;
    };
    int done = 0;  // steps of the runs already issued
    while (done < nsteps) {
        const int cs = std::min(kGraphSteps, nsteps - done);
        if ((e = run_one(cs, fe && done == 0)) != cudaSuccess) {
            // the runs issued before stand: the host clock follows the device's
            g->last_launches = total;
            g->t = g->t + (double)done * dt;
            g->steps += done;
            if (done > 0) g->cross_explicit = false;
            return cuda_fail(g, e, what);
        }
        if (cs & 1) g->cur ^= 1;
        done += cs;
    }
    g->last_launches = total;
    g->t = g->t + (double)nsteps * dt;
    g->steps += nsteps;
    g->cross_explicit = false;
    return GALS_OK;
}

// After a stream synchronisation: report (and clear) a kernel-side error word.
static gals_status check_device_error(gals_grid *g)
{
    int code = 0;
    cudaError_t e = cudaMemcpy(&code, g->err_dev, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(g, e, "error word");
    if (code == 0) return GALS_OK;
    cudaMemset(g->err_dev, 0, sizeof(int));
    if ((code & 0xff) == kErrBounds)
        return fail(g, GALS_ERR_CUDA, "checked build: an index left its buffer (source line %d)",
                    code >> 8);
    return fail(g, GALS_ERR_TIMEOUT, "a bounded device wait ran out (code %d); results of the "
                "affected steps are invalid", code);
}

gals_status gals_synchronize(gals_grid *g)
{
    if (!g) return fail(nullptr, GALS_ERR_ARG, "grid is NULL");
    if (cudaError_t je = join_host_steps(g); je != cudaSuccess) return cuda_fail(g, je, "join host steps");
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(g, e, "synchronize");
    return check_device_error(g);
}

static gals_status ensure_cross(gals_grid *g)
{
    // COMPACT layout: the mixed derivatives of the current state are not stored by the
    // step; rebuild them (unless set_state just provided them explicitly).
    if (g->layout == GALS_LAYOUT_COMPACT && !g->cross_explicit && g->cross != GALS_CROSS_CELL) {
        cudaError_t e = launch_recon(g->dim, g->geom, g->buf[g->cur], g->stream);
        if (e != cudaSuccess) return cuda_fail(g, e, "recon");
    }
    return GALS_OK;
}

gals_status gals_read_state(gals_grid *g, float *const *fields, int nfields, int memspace)
{
    NvtxRange nvtx_range("gals_read_state");
    if (!g) return fail(nullptr, GALS_ERR_ARG, "grid is NULL");
    if (cudaError_t je = join_host_steps(g); je != cudaSuccess) return cuda_fail(g, je, "join host steps");
    if (!g->has_state) return fail(g, GALS_ERR_STATE, "no state loaded");
    if (!fields || nfields < 1 || nfields > g->nplanes)
        return fail(g, GALS_ERR_ARG, "nfields must be in 1..%d", g->nplanes);
    if (memspace != GALS_MEM_HOST && memspace != GALS_MEM_DEVICE)
        return fail(g, GALS_ERR_ARG, "bad memspace %d", memspace);
    for (int p = 0; p < nfields; ++p)
        if (!fields[p]) return fail(g, GALS_ERR_ARG, "fields[%d] is NULL", p);
    if (nfields > 1 + g->dim) {
        gals_status st = ensure_cross(g);
        if (st != GALS_OK) return st;
    }
    const Geom &G = g->geom;
    const size_t row = (size_t)g->n[0] * sizeof(float);
    const size_t rows = (size_t)g->n[1] * g->n[2];
    const cudaMemcpyKind kind = memspace == GALS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaError_t e;
    for (int p = 0; p < nfields; ++p) {
        e = cudaMemcpy2DAsync(fields[p], row, g->buf[g->cur] + p * G.plane, (size_t)G.pitch * sizeof(float),
                              row, rows, kind, g->stream);
        if (e != cudaSuccess) return cuda_fail(g, e, "read_state copy");
    }
    if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cuda_fail(g, e, "read_state sync");
    return check_device_error(g);
}

// gals_step_host and gals_step_host_async: queue the band pipeline; the synchronous form
// then drains every stream.
static gals_status step_host_impl(gals_grid *g, const gals_velocity *v, double dt, double t0,
                                  const float *const *in, float *const *out, bool async)
{
    if (!g) return fail(nullptr, GALS_ERR_ARG, "grid is NULL");
    if (!in || !out) return fail(g, GALS_ERR_ARG, "in / out is NULL");
    for (int p = 0; p < g->nplanes; ++p)
        if (!in[p] || !out[p]) return fail(g, GALS_ERR_ARG, "in[%d] / out[%d] is NULL", p, p);
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(g, GALS_ERR_ARG, "dt must be finite and > 0");
    if (!std::isfinite(t0)) return fail(g, GALS_ERR_ARG, "t0 is not finite");
    if (g->layout != GALS_LAYOUT_FULL || g->cross != GALS_CROSS_CENTRAL)
        return fail(g, GALS_ERR_UNSUPPORTED, "gals_step_host needs the FULL layout and approach A");
    VelParams vp;
    gals_status st = make_velparams(g, v, vp);
    if (st != GALS_OK) return st;
    if (v->trace == GALS_TRACE_SURROGATE)
        return fail(g, GALS_ERR_UNSUPPORTED, "gals_step_host does not take the surrogate trace");
    if (v->kind == GALS_VEL_WAVES2D)
        return fail(g, GALS_ERR_UNSUPPORTED, "gals_step_host does not take the WAVES2D field");
    cudaError_t e = cudaSuccess;
    if (!g->hs_in) {
        e = cudaStreamCreateWithFlags(&g->hs_in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->hs_out, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->hs_enter, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->hs_done, cudaEventDisableTiming);
        for (int b = 0; b < kHostBands && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&g->hs_in_ev[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->hs_step_ev[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->hs_out_ev[b], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(g, e, "copy streams / events");
    }
    if (g->coef_cap < 1) {
        if ((e = cudaMalloc(&g->coef, sizeof(StageCoef) * 64)) != cudaSuccess)
            return cuda_fail(g, e, "cudaMalloc(coefficient table)");
        g->coef_cap = 64;
    }
    // Bands along the last axis, whole tiles each.  The step of band b reads the input
    // from every band its feet, cells and staged tiles reach: |foot - node| <= dt * vmax
    // along that axis, plus the cell's far corner and the tile halo (3 nodes); it waits
    // for the copy of the last of those bands (all bands if no speed bound is known).
    // About 64 MB of copies per band, 4 to 16 bands: fewer bands cost a longer fill and
    // drain of the pipeline, more cost per-copy overhead (measured on GB300: 8 bands best
    // for a 4096^2 state, 16 for 512^3).
    const int ax = g->dim - 1, nax = g->n[ax], unit = band_unit(g->dim);
    const int64_t copy_bytes = 2 * (int64_t)g->nplanes * sizeof(float) * g->n[0] * g->n[1] * g->n[2];
    const int want = (int)std::min<int64_t>(kHostBands, std::max<int64_t>(4, copy_bytes >> 26));
    const int R = ((nax + want - 1) / want + unit - 1) / unit * unit;
    const int nb = (nax + R - 1) / R;
    const double reach = dt * speed_bound(v, g->dim, g->lo, g->hi) / g->h[ax] + 3.0;
    const int K = reach < (double)nax ? (int)std::ceil(reach / R) : nb;
    const Geom &G = g->geom;
    const size_t row = (size_t)g->n[0] * sizeof(float), dpitch = (size_t)G.pitch * sizeof(float);
    const size_t rows_per = g->dim == 2 ? 1 : (size_t)g->n[1];  // 2D-copy rows per band node
    const int cur = g->cur;
    float *bin = g->buf[cur], *bout = g->buf[cur ^ 1];
    g->t = t0;
    // work already queued on the grid stream (a step reading or writing the buffers)
    // comes first; the copy-in of a band also waits for the copy-out of the same band of
    // the previous host step, which may still be running (it reads the buffer this step
    // fills, and its host rows may be this step's input)
    if ((e = cudaEventRecord(g->hs_enter, g->stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(g->hs_in, g->hs_enter, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(g->hs_out, g->hs_enter, 0)) != cudaSuccess)
        return cuda_fail(g, e, "step_host order");
    if ((e = launch_set_time(g->t_dev, t0, g->stream)) != cudaSuccess ||
        (e = launch_coef_table(g->coef, vp, g->t_dev, dt, 1, g->stream)) != cudaSuccess)
        return cuda_fail(g, e, "step_host coefficients");
    auto copy_in = [&](int b) {
        const size_t r0 = (size_t)b * R * rows_per, nr = (size_t)(std::min(nax, (b + 1) * R) - b * R) * rows_per;
        e = cudaStreamWaitEvent(g->hs_in, g->hs_out_ev[b], 0);
        for (int p = 0; p < g->nplanes && e == cudaSuccess; ++p)
            e = cudaMemcpy2DAsync(bin + p * G.plane + r0 * G.pitch, dpitch, in[p] + r0 * g->n[0], row, row,
                                  nr, cudaMemcpyHostToDevice, g->hs_in);
        if (e == cudaSuccess) e = cudaEventRecord(g->hs_in_ev[b], g->hs_in);
    };
    StepLaunch a = step_launch(g, vp, v->trace, dt, 0, cur, false);
    auto step_out = [&](int b) {
        if ((e = cudaStreamWaitEvent(g->stream, g->hs_in_ev[std::min(nb - 1, b + K)], 0)) != cudaSuccess) return;
        a.band_lo = b * R;
        a.band_hi = std::min(nax, (b + 1) * R);
        e = g->dim == 2 ? launch_step2d(a, g->stream) : launch_step3d(a, g->stream);
        if (e == cudaSuccess) e = cudaEventRecord(g->hs_step_ev[b], g->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g->hs_out, g->hs_step_ev[b], 0);
        const size_t r0 = (size_t)b * R * rows_per, nr = (size_t)(a.band_hi - a.band_lo) * rows_per;
        for (int p = 0; p < g->nplanes && e == cudaSuccess; ++p)
            e = cudaMemcpy2DAsync(out[p] + r0 * g->n[0], row, bout + p * G.plane + r0 * G.pitch, dpitch, row,
                                  nr, cudaMemcpyDeviceToHost, g->hs_out);
        if (e == cudaSuccess) e = cudaEventRecord(g->hs_out_ev[b], g->hs_out);
    };
    // enqueue in pipeline order, so that the first bands are stepped and copied out while
    // the host is still queueing the copies of later ones
    for (int b = 0; b <= std::min(nb - 1, K) && e == cudaSuccess; ++b) copy_in(b);
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
        if (b + K + 1 < nb) copy_in(b + K + 1);
        if (e == cudaSuccess) step_out(b);
    }
    if (e == cudaSuccess) e = launch_advance_time(g->t_dev, 1, dt, g->stream);
    if (e == cudaSuccess) e = cudaEventRecord(g->hs_done, g->hs_out);
    if (async && e == cudaSuccess) {
        // the copies run on; other calls on the grid wait for them (join_host_steps)
        g->hs_pending = true;
        g->cur ^= 1;
        g->t = t0 + dt;
        g->steps = 1;
        g->cross_explicit = false;
        g->has_state = true;
        return GALS_OK;
    }
    // every stream is drained before returning, also after a failed launch
    g->hs_pending = false;
    cudaError_t s1 = cudaStreamSynchronize(g->hs_in), s2 = cudaStreamSynchronize(g->hs_out);
    cudaError_t s3 = cudaStreamSynchronize(g->stream);
    if (e == cudaSuccess) e = s1 != cudaSuccess ? s1 : (s2 != cudaSuccess ? s2 : s3);
    if (e != cudaSuccess) {
        g->has_state = false;
        return cuda_fail(g, e, "step_host");
    }
    g->cur ^= 1;
    g->t = t0 + dt;
    g->steps = 1;
    g->cross_explicit = false;
    g->has_state = true;
    return check_device_error(g);
}

gals_status gals_step_host(gals_grid *g, const gals_velocity *v, double dt, double t0,
                           const float *const *in, float *const *out)
{
    NvtxRange nvtx_range("gals_step_host");
    return step_host_impl(g, v, dt, t0, in, out, false);
}

gals_status gals_step_host_async(gals_grid *g, const gals_velocity *v, double dt, double t0,
                                 const float *const *in, float *const *out)
{
    NvtxRange nvtx_range("gals_step_host_async");
    return step_host_impl(g, v, dt, t0, in, out, true);
}

gals_status gals_eval_points(gals_grid *g, const double *points, int64_t npoints, int memspace,
                             float *H, float *normal, float *kappa)
{
    NvtxRange nvtx_range("gals_eval_points");
    if (!g) return fail(nullptr, GALS_ERR_ARG, "grid is NULL");
    if (cudaError_t je = join_host_steps(g); je != cudaSuccess) return cuda_fail(g, je, "join host steps");
    if (!g->has_state) return fail(g, GALS_ERR_STATE, "no state loaded");
    if (npoints < 0) return fail(g, GALS_ERR_ARG, "npoints must be >= 0");
    if (npoints > 0 && !points) return fail(g, GALS_ERR_ARG, "points is NULL");
    if (memspace != GALS_MEM_HOST && memspace != GALS_MEM_DEVICE)
        return fail(g, GALS_ERR_ARG, "bad memspace %d", memspace);
    if (npoints == 0) return GALS_OK;
    gals_status st = ensure_cross(g);
    if (st != GALS_OK) return st;
    const int dim = g->dim;
    const bool cell_b = g->cross == GALS_CROSS_CELL;
    cudaError_t e;
    if (memspace == GALS_MEM_DEVICE) {
        e = launch_eval_points(dim, g->geom, g->lo, g->h, g->buf[g->cur], points, npoints, cell_b, H,
                               normal, kappa, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        return e == cudaSuccess ? GALS_OK : cuda_fail(g, e, "eval_points");
    }
    // host points and results: stage them through a device buffer kept by the grid
    const size_t pb = sizeof(double) * dim * (size_t)npoints;
    const size_t ob = sizeof(float) * (size_t)npoints;
    const size_t need = pb + ob * (2 + dim);
    if (need > g->pt_cap) {
        if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cuda_fail(g, e, "sync");
        cudaFree(g->pt_buf);
        g->pt_buf = nullptr;
        g->pt_cap = 0;
        if ((e = cudaMalloc(&g->pt_buf, need)) != cudaSuccess) return cuda_fail(g, e, "cudaMalloc(points)");
        g->pt_cap = need;
    }
    double *dp = reinterpret_cast<double *>(g->pt_buf);
    float *dH = reinterpret_cast<float *>(g->pt_buf + pb), *dk = dH + npoints, *dn = dk + npoints;
    if ((e = cudaMemcpyAsync(dp, points, pb, cudaMemcpyHostToDevice, g->stream)) != cudaSuccess)
        return cuda_fail(g, e, "points copy");
    e = launch_eval_points(dim, g->geom, g->lo, g->h, g->buf[g->cur], dp, npoints, cell_b, H ? dH : nullptr,
                           normal ? dn : nullptr, kappa ? dk : nullptr, g->stream);
    if (e == cudaSuccess && H) e = cudaMemcpyAsync(H, dH, ob, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess && kappa) e = cudaMemcpyAsync(kappa, dk, ob, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess && normal) e = cudaMemcpyAsync(normal, dn, ob * dim, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    return e == cudaSuccess ? GALS_OK : cuda_fail(g, e, "eval_points");
}

gals_status gals_state_planes(gals_grid *g, float **planes, int nplanes, int64_t *row_pitch)
{
    if (!g) return fail(nullptr, GALS_ERR_ARG, "grid is NULL");
    if (cudaError_t je = join_host_steps(g); je != cudaSuccess) return cuda_fail(g, je, "join host steps");
    if (!planes || nplanes < 1 || nplanes > g->nplanes)
        return fail(g, GALS_ERR_ARG, "nplanes must be in 1..%d", g->nplanes);
    for (int p = 0; p < nplanes; ++p) planes[p] = g->buf[g->cur] + p * g->geom.plane;
    if (row_pitch) *row_pitch = g->geom.pitch;
    return GALS_OK;
}

gals_status gals_diagnostics(gals_grid *g, const gals_diag_request *req, gals_diag *out)
{
    NvtxRange nvtx_range("gals_diagnostics");
    if (!g) return fail(nullptr, GALS_ERR_ARG, "grid is NULL");
    if (cudaError_t je = join_host_steps(g); je != cudaSuccess) return cuda_fail(g, je, "join host steps");
    if (!req || !out) return fail(g, GALS_ERR_ARG, "request/out is NULL");
    if (!g->has_state) return fail(g, GALS_ERR_STATE, "no state loaded");
    if (req->q < 0 || req->q > 16) return fail(g, GALS_ERR_ARG, "q must be in 0..16");
    const gals_grid *r = req->reference;
    if (r) {
        if (r->dim != g->dim || r->n[0] != g->n[0] || r->n[1] != g->n[1] || r->n[2] != g->n[2])
            return fail(g, GALS_ERR_ARG, "reference grid has another shape");
        if (!r->has_state) return fail(g, GALS_ERR_STATE, "reference has no state");
    }
    gals_status st = ensure_cross(g);
    if (st != GALS_OK) return st;
    cudaError_t e;
    if (r) {
        // the reference is read on this grid's stream: order after its own work
        if ((e = cudaStreamSynchronize(r->stream)) != cudaSuccess) return cuda_fail(g, e, "reference sync");
        if (r->layout == GALS_LAYOUT_COMPACT && !r->cross_explicit && r->cross != GALS_CROSS_CELL) {
            if ((e = launch_recon(r->dim, r->geom, r->buf[r->cur], g->stream)) != cudaSuccess)
                return cuda_fail(g, e, "reference recon");
        }
    }
    e = launch_diag(g->dim, g->geom, g->buf[g->cur], r ? r->buf[r->cur] : nullptr, req->q, g->diag_dev,
                    g->diag_partials, g->stream, g->cross == GALS_CROSS_CELL,
                    r && r->cross == GALS_CROSS_CELL);
    if (e != cudaSuccess) return cuda_fail(g, e, "diagnostics launch");
    DiagOut h;
    if ((e = cudaMemcpyAsync(&h, g->diag_dev, sizeof(h), cudaMemcpyDeviceToHost, g->stream)) != cudaSuccess)
        return cuda_fail(g, e, "diagnostics copy");
    if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cuda_fail(g, e, "diagnostics sync");
    if ((st = check_device_error(g)) != GALS_OK) return st;
    std::memset(out, 0, sizeof(*out));
    double cell = 1.0;
    int64_t ncell = 1;
    for (int i = 0; i < g->dim; ++i) { cell *= g->h[i]; ncell *= g->n[i] - 1; }
    const int q = req->q;
    double qp = 1.0;
    for (int i = 0; i < g->dim; ++i) qp *= q;
    out->t = g->t;
    out->steps = g->steps;
    out->samples = q > 0 ? (int64_t)(ncell * qp) : 0;
    out->n_negative = (int64_t)h.n_neg;
    out->measure_negative = q > 0 ? (double)h.n_neg * cell / qp : 0.0;
    out->n_symdiff = (int64_t)h.n_sym;
    out->measure_symdiff = q > 0 ? (double)h.n_sym * cell / qp : 0.0;
    float fphi, fpsi;
    std::memcpy(&fphi, &h.emax_phi_bits, 4);
    std::memcpy(&fpsi, &h.emax_psi_bits, 4);
    out->emax_phi = r ? (double)fphi : 0.0;
    out->emax_psi = r ? (double)fpsi : 0.0;
    out->l2_phi = r ? std::sqrt(h.l2_phi_sum * cell) : 0.0;
    out->nonfinite = (int64_t)h.nonfinite;
    return GALS_OK;
}

}  // extern "C"
