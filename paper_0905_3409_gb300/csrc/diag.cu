// diag.cu -- diagnostics of a GALS state: sampled area/volume of {H < 0}, the symmetric
// difference against a reference state, e_max norms (eq. maximum_norm, Sec. 6.1), an
// FP64 L2 norm and a non-finite count.
//
// Counts are exact 64-bit integers (order-independent atomics), maxima are taken on
// the ordered bit patterns of non-negative floats, and the FP64 sum is reduced per
// block into a scratch array and then summed in a fixed order by one block, so every
// result is deterministic.
#include "gals_internal.h"

namespace gals {

namespace {

constexpr int kThreads = 256;
constexpr int kNodeBlocks = 1216;  // 8 x 152 SMs; grid-stride over nodes

__device__ __forceinline__ void gather2d(const float *s, const Geom &g, int k, int l, float c[4][4])
{
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int64_t id = (int64_t)(l + (v >> 1)) * g.pitch + k + (v & 1);
#pragma unroll
        for (int a = 0; a < 4; ++a) c[v][a] = s[a * g.plane + id];
    }
}

__device__ __forceinline__ void gather3d(const float *s, const Geom &g, int k, int l, int m,
                                         float c[8][8])
{
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const int64_t id = ((int64_t)(m + (v >> 2)) * g.n1 + l + ((v >> 1) & 1)) * g.pitch + k + (v & 1);
#pragma unroll
        for (int a = 0; a < 8; ++a) c[v][a] = s[a * g.plane + id];
    }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kThreads / 32; ++i) s += red[i];
    return s;  // valid in thread 0
}

__device__ __forceinline__ unsigned block_max(unsigned v, unsigned *red)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, off));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    unsigned s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kThreads / 32; ++i) s = max(s, red[i]);
    return s;
}

// approach B for a gathered 3D cell (planes 0 phi, 1-3 psi, 4-7 mixed derivatives)
__device__ __forceinline__ void cell3d_planes(float c[8][8], const Geom &g)
{
    float cr[8][4];
    cross_cell3d([&](int v, int a) { return c[v][a]; }, g.ih0, g.ih1, g.ih2, cr);
#pragma unroll
    for (int v = 0; v < 8; ++v)
#pragma unroll
        for (int i = 0; i < 4; ++i) c[v][4 + i] = cr[v][i];
}

// One thread per cell: q^p cell-centred samples of H (state a) and of the reference b;
// cell_a / cell_b: that state's interpolant takes its mixed derivatives by approach B.
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_diag_cells(Geom g, const float *__restrict__ a, const float *__restrict__ b, int q,
             DiagOut *out, int cell_a, int cell_b)
{
    __shared__ unsigned long long red[kThreads / 32];
    const int64_t nc0 = g.n0 - 1, nc1 = g.n1 - 1, nc2 = DIM == 3 ? g.n2 - 1 : 1;
    const int64_t ncell = nc0 * nc1 * nc2;
    unsigned long long nneg = 0, nsym = 0;
    const float invq = 1.f / (float)q;
    for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < ncell;
         c += (int64_t)gridDim.x * kThreads) {
        const int k = (int)(c % nc0);
        const int l = (int)((c / nc0) % nc1);
        const int m = (int)(c / (nc0 * nc1));
        if (DIM == 2) {
            float ca[4][4], cb[4][4];
            gather2d(a, g, k, l, ca);
            if (b) gather2d(b, g, k, l, cb);
            // approach B: the cell's mixed derivatives from its vertices' gradients
            if (cell_a) cross_cell2d(ca, g.ih0, g.ih1);
            if (b && cell_b) cross_cell2d(cb, g.ih0, g.ih1);
            for (int sy = 0; sy < q; ++sy) {
                const Basis1 by = basis1(((float)sy + 0.5f) * invq, g.h1, g.ih1);
                for (int sx = 0; sx < q; ++sx) {
                    const Basis1 bx = basis1(((float)sx + 0.5f) * invq, g.h0, g.ih0);
                    float Ha, hx, hy;
                    hermite2d(ca, bx, by, Ha, hx, hy);
                    nneg += (Ha < 0.f);
                    if (b) {
                        float Hb;
                        hermite2d(cb, bx, by, Hb, hx, hy);
                        nsym += ((Ha < 0.f) != (Hb < 0.f));
                    }
                }
            }
        } else {
            float ca[8][8], cb[8][8];
            gather3d(a, g, k, l, m, ca);
            if (b) gather3d(b, g, k, l, m, cb);
            if (cell_a) cell3d_planes(ca, g);
            if (b && cell_b) cell3d_planes(cb, g);
            for (int sz = 0; sz < q; ++sz) {
                const Basis1 bz = basis1(((float)sz + 0.5f) * invq, g.h2, g.ih2);
                for (int sy = 0; sy < q; ++sy) {
                    const Basis1 by = basis1(((float)sy + 0.5f) * invq, g.h1, g.ih1);
                    for (int sx = 0; sx < q; ++sx) {
                        const Basis1 bx = basis1(((float)sx + 0.5f) * invq, g.h0, g.ih0);
                        float Ha, gr[3];
                        hermite3d(ca, bx, by, bz, Ha, gr);
                        nneg += (Ha < 0.f);
                        if (b) {
                            float Hb;
                            hermite3d(cb, bx, by, bz, Hb, gr);
                            nsym += ((Ha < 0.f) != (Hb < 0.f));
                        }
                    }
                }
            }
        }
    }
    unsigned long long s = block_sum(nneg, red);
    if (threadIdx.x == 0 && s) atomicAdd(&out->n_neg, s);
    s = block_sum(nsym, red);
    if (threadIdx.x == 0 && s) atomicAdd(&out->n_sym, s);
}

// One thread per node (grid-stride): non-finite count, e_max of phi and psi against b,
// FP64 sum of (phi - phi_b)^2 into partials[blockIdx.x].
__global__ void __launch_bounds__(kThreads)
k_diag_nodes(Geom g, int dim, const float *__restrict__ a, const float *__restrict__ b,
             DiagOut *out, double *partials)
{
    __shared__ unsigned long long redu[kThreads / 32];
    __shared__ double redd[kThreads / 32];
    __shared__ unsigned redm[kThreads / 32];
    const int np = dim == 2 ? 4 : 8;
    const int64_t n = (int64_t)g.n0 * g.n1 * (dim == 3 ? g.n2 : 1);
    unsigned long long nonfin = 0;
    unsigned mphi = 0, mpsi = 0;
    double l2 = 0.0;
    for (int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * kThreads) {
        const int i = (int)(idx % g.n0);
        const int64_t rest = idx / g.n0;
        const int64_t o = rest * g.pitch + i;
        bool bad = false;
        for (int p = 0; p < np; ++p) bad |= !isfinite(a[p * g.plane + o]);
        nonfin += bad;
        if (b) {
            const float d = fabsf(a[o] - b[o]);
            mphi = max(mphi, __float_as_uint(d));
            for (int p = 1; p <= dim; ++p)
                mpsi = max(mpsi, __float_as_uint(fabsf(a[p * g.plane + o] - b[p * g.plane + o])));
            const double dd = (double)a[o] - (double)b[o];
            l2 += dd * dd;
        }
    }
    unsigned long long s = block_sum(nonfin, redu);
    if (threadIdx.x == 0 && s) atomicAdd(&out->nonfinite, s);
    unsigned m1 = block_max(mphi, redm);
    if (threadIdx.x == 0) atomicMax(&out->emax_phi_bits, m1);
    unsigned m2 = block_max(mpsi, redm);
    if (threadIdx.x == 0) atomicMax(&out->emax_psi_bits, m2);
    double ds = block_sum(l2, redd);
    if (threadIdx.x == 0) partials[blockIdx.x] = ds;
}

// Fixed-order FP64 sum of the per-block partials.
__global__ void k_diag_finish(const double *partials, int nparts, DiagOut *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nparts; ++i) s += partials[i];
        out->l2_phi_sum = s;
    }
}

}  // namespace

int diag_partials_needed() { return kNodeBlocks; }

cudaError_t launch_diag(int dim, const Geom &g, const float *a, const float *b, int q,
                        DiagOut *counters, double *partials, cudaStream_t s, bool cell_a, bool cell_b)
{
    cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(DiagOut), s);
    if (e != cudaSuccess) return e;
    if (q > 0) {
        const int64_t ncell = (int64_t)(g.n0 - 1) * (g.n1 - 1) * (dim == 3 ? g.n2 - 1 : 1);
        int blocks = (int)std::min<int64_t>((ncell + kThreads - 1) / kThreads, 152 * 16);
        if (dim == 2) k_diag_cells<2><<<blocks, kThreads, 0, s>>>(g, a, b, q, counters, cell_a, cell_b);
        else k_diag_cells<3><<<blocks, kThreads, 0, s>>>(g, a, b, q, counters, cell_a, cell_b);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_diag_nodes<<<kNodeBlocks, kThreads, 0, s>>>(g, dim, a, b, counters, partials);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_diag_finish<<<1, 32, 0, s>>>(partials, kNodeBlocks, counters);
    return cudaGetLastError();
}

cudaError_t launch_diag_with(int dim, const Geom &g, const float *a, const float *b, int q,
                             DiagOut *counters, double *partials, int nparts, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(DiagOut), s);
    if (e != cudaSuccess) return e;
    if (q > 0) {
        const int64_t ncell = (int64_t)(g.n0 - 1) * (g.n1 - 1) * (dim == 3 ? g.n2 - 1 : 1);
        int blocks = (int)std::min<int64_t>((ncell + kThreads - 1) / kThreads, 152 * 16);
        if (dim == 2) k_diag_cells<2><<<blocks, kThreads, 0, s>>>(g, a, b, q, counters, 0, 0);
        else k_diag_cells<3><<<blocks, kThreads, 0, s>>>(g, a, b, q, counters, 0, 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_diag_nodes<<<nparts, kThreads, 0, s>>>(g, dim, a, b, counters, partials);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_diag_finish<<<1, 32, 0, s>>>(partials, nparts, counters);
    return cudaGetLastError();
}

}  // namespace gals
