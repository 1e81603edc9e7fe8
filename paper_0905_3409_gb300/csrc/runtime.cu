// runtime.cu -- small launchers shared by the C ABI: approach-A reconstruction dispatch,
// the device clock update and the velocity/dimension support table.
#include "gals_internal.h"

namespace gals {

cudaError_t launch_recon2d(const Geom &g, float *buf, cudaStream_t s);
cudaError_t launch_recon3d(const Geom &g, float *buf, cudaStream_t s);

cudaError_t launch_recon(int dim, const Geom &g, float *buf, cudaStream_t s)
{
    return dim == 2 ? launch_recon2d(g, buf, s) : launch_recon3d(g, buf, s);
}

namespace {
__global__ void k_advance_time(double *t, int nsteps, double dt)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) t[0] = t[0] + (double)nsteps * dt;
}

__global__ void k_set_time(double *t, double value)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) t[0] = value;
}
}  // namespace

namespace {
__global__ void k_coef_table(StageCoef *table, VelParams vp, const double *t_dev, double dt,
                             int nsteps)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsteps) return;
    const double t = t_dev[0] + (double)k * dt;
    stage_coef_one(vp, t, dt, table[k]);
    if (vp.kind == VK_WAVES2D) table[k].wamp = vp.wamp + (size_t)k * 3 * vp.nwaves;
}

// WAVES2D amplitudes of the call's steps: wamp[(k 3 + s) M + m] = a_m cos(2 pi (n_m t_s + chi_m'))
// at the stage times t_s (t + dt, t, t + dt/2) of step k, the phase reduced in FP64.
__global__ void k_wave_amp(VelParams vp, const double *t_dev, double dt, int nsteps)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int M = vp.nwaves;
    if (e >= (int64_t)nsteps * 3 * M) return;
    const int m = (int)(e % M), s = (int)((e / M) % 3), k = (int)(e / (3 * M));
    const double t = t_dev[0] + (double)k * dt;
    const double ts = s == 0 ? t + dt : (s == 1 ? t : t + 0.5 * dt);
    const double a = vp.waves_d[3 * m], n = vp.waves_d[3 * m + 1], chi = vp.waves_d[3 * m + 2];
    double ph = 2.0 * (n * ts + chi);  // in units of pi
    ph = ph - 2.0 * floor(0.5 * ph);
    vp.wamp[e] = (float)(a * cospi(ph));
}
}  // namespace

cudaError_t launch_coef_table(StageCoef *table, const VelParams &vp, const double *t_dev,
                              double dt, int nsteps, cudaStream_t s)
{
    if (vp.kind == VK_WAVES2D) {
        const int64_t n = (int64_t)nsteps * 3 * vp.nwaves;
        k_wave_amp<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(vp, t_dev, dt, nsteps);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_coef_table<<<(nsteps + 63) / 64, 64, 0, s>>>(table, vp, t_dev, dt, nsteps);
    return cudaGetLastError();
}

cudaError_t launch_advance_time(double *t_dev, int nsteps, double dt, cudaStream_t s)
{
    k_advance_time<<<1, 32, 0, s>>>(t_dev, nsteps, dt);
    return cudaGetLastError();
}

cudaError_t launch_set_time(double *t_dev, double t, cudaStream_t s)
{
    k_set_time<<<1, 32, 0, s>>>(t_dev, t);
    return cudaGetLastError();
}

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}
}  // namespace

cudaError_t make_tile_map(CUtensorMap *map, const float *base, int rank, const uint64_t *dims,
                          const uint64_t *strides_bytes, const uint32_t *box)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t d[5], st[4];
    cuuint32_t b[5], es[5];
    for (int i = 0; i < rank; ++i) { d[i] = dims[i]; b[i] = box[i]; es[i] = 1; }
    for (int i = 0; i < rank - 1; ++i) st[i] = strides_bytes[i];
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, (void *)base, d, st, b, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool vel_supported(int dim, int kind)
{
    if (dim == 2)
        return kind == VK_CONST || kind == VK_ROTATION || kind == VK_VORTEX2D ||
               kind == VK_PSEUDO1D || kind == VK_FOURIER2D || kind == VK_WAVES2D;
    return kind == VK_CONST || kind == VK_ROTATION || kind == VK_DEFORM3D;
}

}  // namespace gals
