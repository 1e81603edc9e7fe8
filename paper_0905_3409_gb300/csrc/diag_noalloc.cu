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
#include <cstdint>
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
// stand-in: its device address comes from cudaGetSymbolAddress, once per device (and
// context).
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(Scratch)];

std::mutex g_mutex;
struct ScratchSlot {
    unsigned long long ctx_id = 0;  // unique id of the context the address belongs to
    void *addr = nullptr;
};
ScratchSlot g_slot[kMaxDevices];

// Unique id of the driver's current context (cuCtxGetCurrent, cuCtxGetId; reached through
// the runtime's driver entry points so that the library links against the runtime only);
// 0 when no context is current or the driver does not offer the calls.  Ids are never
// reused within a process, unlike context handles.
unsigned long long current_context_id()
{
    typedef int (*CtxGetCurrent)(void **);
    typedef int (*CtxGetId)(void *, unsigned long long *);
    auto entry = [](const char *name) -> void * {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return p;
    };
    static CtxGetCurrent get_current = reinterpret_cast<CtxGetCurrent>(entry("cuCtxGetCurrent"));
    static CtxGetId get_id = reinterpret_cast<CtxGetId>(entry("cuCtxGetId"));
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch on the current device.  The lookup
// (cudaGetSymbolAddress) is the set-up: it runs on the first call on a device, and again
// only if that device's context has changed since (after cudaDeviceReset, or when the
// caller made another context current), because the address belongs to one context.
cudaError_t scratch_address(Scratch **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    const unsigned long long id = current_context_id();  // 0 before a context is current
    std::lock_guard<std::mutex> lock(g_mutex);
    ScratchSlot &slot = g_slot[dev];
    if (!slot.addr || id == 0 || slot.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        slot.addr = p;
        slot.ctx_id = current_context_id();
    }
    *out = static_cast<Scratch *>(slot.addr);
    return cudaSuccess;
}

// the message of the calling thread's last failed call
thread_local char g_noalloc_err[256] = "";

gals_status nfail(gals_status st, const char *msg)
{
    std::strncpy(g_noalloc_err, msg, sizeof(g_noalloc_err) - 1);
    g_noalloc_err[sizeof(g_noalloc_err) - 1] = '\0';
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
        nodes *= n[i];  // n[i] < 2^31 and nodes <= kMaxNodes < 2^29 before: no overflow
        if (nodes > kMaxNodes)
            return nfail(GALS_ERR_ARG, "grid larger than the no-allocation scratch allows "
                                       "(gals_noalloc_max_nodes() nodes)");
    }
    const int64_t rows = (int64_t)n[1] * (dim == 3 ? n[2] : 1);
    // the kernels keep the row pitch in an int and index planes as p * plane_stride
    // (p < 8) in 64 bits
    if (row_pitch < n[0] || row_pitch > INT32_MAX)
        return nfail(GALS_ERR_ARG, "row_pitch must be in [n[0], 2^31 - 1]");
    if (plane_stride < row_pitch * rows || plane_stride > INT64_MAX / 8)  // rows < 2^29
        return nfail(GALS_ERR_ARG, "plane_stride smaller than a plane, or too large");
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
