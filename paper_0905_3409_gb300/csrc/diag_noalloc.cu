// diag_noalloc.cu -- gals_diagnostics_noalloc: the diagnostics of a state held in caller
// memory, computed without allocating any device memory.
//
// Some callers cannot allocate on the device at the moment they want diagnostics: a
// loop whose whole device memory was reserved up front by another allocator (a framework's
// caching allocator, a fixed arena), code that must not let cudaMalloc/cudaFree
// synchronise the device behind its back, or a service that accounts for every byte it
// holds.  This entry point gives them the same results as gals_diagnostics using a fixed
// scratch area that lives in the library image instead: a file-scope __device__ array that
// every device holding the library keeps until the process exits.  The caller passes the
// state (and an optional reference) and receives the results; nothing is allocated.
//
// The scratch holds the result counters and one FP64 partial sum per block of the node
// pass, one block per kNodesPerPartial nodes, so its capacity bounds the grid size.
#include <cmath>
#include <cstring>
#include <mutex>

#include "capi_internal.h"

using namespace gals;

namespace {

constexpr int kMaxPartials = 16384;
constexpr int64_t kNodesPerPartial = 16384;
constexpr int64_t kMaxNodes = (int64_t)kMaxPartials * kNodesPerPartial;  // 268,435,456
constexpr int kMaxDevices = 64;

struct Scratch {
    DiagOut counters;
    double pad[3];
    double partials[kMaxPartials];
};

// The scratch itself (about 128 KB per device).  In host code this name is only a
// stand-in: its device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(Scratch)];

std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up on first use).
cudaError_t scratch_address(Scratch **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<Scratch *>(g_scratch_addr[dev]);
    return cudaSuccess;
}

char g_noalloc_err[256] = "";

gals_status nfail(gals_status st, const char *msg)
{
    std::strncpy(g_noalloc_err, msg, sizeof(g_noalloc_err) - 1);
    return st;
}

}  // namespace

extern "C" {

const char *gals_noalloc_last_error(void) { return g_noalloc_err; }

int64_t gals_noalloc_max_nodes(void) { return kMaxNodes; }

gals_status gals_diagnostics_noalloc(int dim, const int *n, const double *lo, const double *hi,
                                     const float *state, const float *reference,
                                     int64_t row_pitch, int64_t plane_stride, int q,
                                     void *cuda_stream, gals_diag *out)
{
    if (dim != 2 && dim != 3) return nfail(GALS_ERR_ARG, "dim must be 2 or 3");
    if (!n || !lo || !hi || !state || !out) return nfail(GALS_ERR_ARG, "NULL argument");
    if (q < 0 || q > 16) return nfail(GALS_ERR_ARG, "q must be in 0..16");
    int64_t nodes = 1;
    for (int i = 0; i < dim; ++i) {
        if (n[i] < 4) return nfail(GALS_ERR_ARG, "every n[i] must be >= 4");
        if (!std::isfinite(lo[i]) || !std::isfinite(hi[i]) || !(hi[i] > lo[i]))
            return nfail(GALS_ERR_ARG, "need finite lo < hi");
        nodes *= n[i];
    }
    const int64_t rows = (int64_t)n[1] * (dim == 3 ? n[2] : 1);
    if (row_pitch < n[0] || plane_stride < row_pitch * rows)
        return nfail(GALS_ERR_ARG, "row_pitch / plane_stride smaller than the grid");
    if (nodes > kMaxNodes)
        return nfail(GALS_ERR_ARG, "grid larger than the no-allocation scratch allows "
                                   "(gals_noalloc_max_nodes() nodes)");
    Geom G{};
    G.n0 = n[0]; G.n1 = n[1]; G.n2 = dim == 3 ? n[2] : 1;
    G.pitch = (int)row_pitch;
    G.plane = plane_stride;
    double h[3] = {1.0, 1.0, 1.0};
    for (int i = 0; i < dim; ++i) h[i] = (hi[i] - lo[i]) / (n[i] - 1);
    G.h0 = (float)h[0]; G.h1 = (float)h[1]; G.h2 = (float)h[2];
    G.ih0 = (float)(1.0 / h[0]); G.ih1 = (float)(1.0 / h[1]); G.ih2 = (float)(1.0 / h[2]);
    G.i2h0 = (float)(0.5 / h[0]); G.i2h1 = (float)(0.5 / h[1]); G.i2h2 = (float)(0.5 / h[2]);
    G.lo0 = (float)lo[0]; G.lo1 = (float)lo[1]; G.lo2 = dim == 3 ? (float)lo[2] : 0.f;

    Scratch *sc = nullptr;
    cudaError_t e = scratch_address(&sc);
    if (e != cudaSuccess) return nfail(GALS_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nparts = (int)((nodes + kNodesPerPartial - 1) / kNodesPerPartial);
    // launch_diag_with clears the counters first: the scratch keeps the previous call's
    // contents
    e = launch_diag_with(dim, G, state, reference, q, &sc->counters, sc->partials, nparts, s);
    if (e != cudaSuccess) return nfail(GALS_ERR_CUDA, cudaGetErrorString(e));
    DiagOut hcnt;
    if ((e = cudaMemcpyAsync(&hcnt, &sc->counters, sizeof(hcnt), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return nfail(GALS_ERR_CUDA, cudaGetErrorString(e));
    std::memset(out, 0, sizeof(*out));
    double cell = 1.0, qp = 1.0;
    int64_t ncell = 1;
    for (int i = 0; i < dim; ++i) { cell *= h[i]; ncell *= n[i] - 1; qp *= q; }
    out->samples = q > 0 ? (int64_t)(ncell * qp) : 0;
    out->n_negative = (int64_t)hcnt.n_neg;
    out->measure_negative = q > 0 ? (double)hcnt.n_neg * cell / qp : 0.0;
    out->n_symdiff = (int64_t)hcnt.n_sym;
    out->measure_symdiff = q > 0 ? (double)hcnt.n_sym * cell / qp : 0.0;
    float fphi, fpsi;
    std::memcpy(&fphi, &hcnt.emax_phi_bits, 4);
    std::memcpy(&fpsi, &hcnt.emax_psi_bits, 4);
    out->emax_phi = reference ? (double)fphi : 0.0;
    out->emax_psi = reference ? (double)fpsi : 0.0;
    out->l2_phi = reference ? std::sqrt(hcnt.l2_phi_sum * cell) : 0.0;
    out->nonfinite = (int64_t)hcnt.nonfinite;
    return GALS_OK;
}

}  // extern "C"
