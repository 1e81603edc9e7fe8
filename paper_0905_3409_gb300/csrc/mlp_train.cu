// mlp_train.cu -- training of the flow-map surrogate on the GPU: target generation by a
// 32-sub-step RK4 backward flow map with its variational Jacobian, and the forward pass,
// backward pass and Adam update of the MLP: the products (forward, dX = dZ W, dW = dZ^T X)
// on the tensor cores (tcgen05, BF16 operands, FP32 accumulation in TMEM).
//
// Target generation follows the same backward flow the oracle integrates
// (dX/ds = -v(X, t+dt-s), dJ/ds = -Dv(X, t+dt-s) J, J(0) = I), here with the displacement
// X - x carried instead of X so that FP32 keeps its relative precision.  Samples
// (x, y, phase) come from a counter-based generator (SplitMix64, Steele, Lea and Flood,
// OOPSLA 2014) keyed on (seed, step, sample), so a training run is reproducible.
#include "mlp_internal.h"
#include "tc.cuh"

namespace gals {
namespace mlp {

using namespace tc;

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float uniform01(uint64_t key)
{
    return (float)(splitmix64(key) >> 40) * (1.0f / 16777216.0f);  // 24 random bits
}

// Fourier stream-function field: v and Dv at (x, y) and time t, mode by mode (FP32).
__device__ void fourier_vdv(const VelParams &vp, float x, float y, float t, float v[2], float D[4])
{
    v[0] = v[1] = 0.f;
    D[0] = D[1] = D[2] = D[3] = 0.f;
    for (int m = 0; m < vp.nmodes; ++m) {
        const float a = vp.mode_a[m];
        const float k = (float)(vp.mode_kl[m] & 0xff), l = (float)(vp.mode_kl[m] >> 8);
        const float ph = (float)vp.mode_n[m] * t + (float)vp.mode_chi[m];  // in turns
        const float c = __cosf(2.f * kPi * (ph - floorf(ph)));
        float skx, ckx, sly, cly;
        __sincosf(k * kPi * x, &skx, &ckx);
        __sincosf(l * kPi * y, &sly, &cly);
        const float kp = k * kPi, lp = l * kPi, ac = a * c;
        v[0] -= ac * skx * lp * cly;
        v[1] += ac * kp * ckx * sly;
        D[0] -= ac * kp * ckx * lp * cly;
        D[1] += ac * skx * lp * lp * sly;
        D[2] -= ac * kp * kp * skx * sly;
        D[3] += ac * kp * ckx * lp * cly;
    }
}

// Plane-wave stream-function field (WAVES2D): the same, from the device mode table.
__device__ void waves_vdv(const VelParams &vp, float x, float y, float t, float v[2], float D[4])
{
    v[0] = v[1] = 0.f;
    D[0] = D[1] = D[2] = D[3] = 0.f;
    const WaveTab T = wave_tab(vp.waves, vp.nwaves);
    for (int m = 0; m < vp.nwaves; ++m) {
        const float4 g = __ldg(T.geo + m), q = __ldg(T.sq + m), w = __ldg(T.tim + m);
        const float ph = w.y * t + w.z;  // in turns
        const float C = w.x * __cosf(2.f * kPi * (ph - floorf(ph)));
        float sn, cs;
        __sincosf(g.x * x + g.y * y + g.z, &sn, &cs);
        v[0] -= C * g.y * cs;
        v[1] += C * g.x * cs;
        D[0] += C * g.w * sn;
        D[1] += C * q.y * sn;
        D[2] -= C * q.x * sn;
        D[3] -= C * g.w * sn;
    }
}

__device__ void flow_rhs(const VelParams &vp, float x, float y, const float d[2], const float Jm[4],
                         float tau, float dd[2], float dJ[4])
{
    float v[2], D[4];
    if (vp.kind == VK_WAVES2D)
        waves_vdv(vp, x + d[0], y + d[1], tau, v, D);
    else
        fourier_vdv(vp, x + d[0], y + d[1], tau, v, D);
    dd[0] = -v[0];
    dd[1] = -v[1];
    dJ[0] = -(D[0] * Jm[0] + D[1] * Jm[2]);
    dJ[1] = -(D[0] * Jm[1] + D[1] * Jm[3]);
    dJ[2] = -(D[2] * Jm[0] + D[3] * Jm[2]);
    dJ[3] = -(D[2] * Jm[1] + D[3] * Jm[3]);
}

}  // namespace

// Backward flow map of one step from (x, y) at time t+dt to time t: displacement and J.
__device__ void flowmap_rk4(const VelParams &vp, float x, float y, float t, float dt, int m,
                            float d[2], float J[4])
{
    d[0] = d[1] = 0.f;
    J[0] = 1.f; J[1] = 0.f; J[2] = 0.f; J[3] = 1.f;
    const float hs = dt / (float)m;
    for (int s = 0; s < m; ++s) {
        const float tau = t + dt - (float)s * hs;
        float k1d[2], k1J[4], k2d[2], k2J[4], k3d[2], k3J[4], k4d[2], k4J[4], dt_[2], Jt[4];
        flow_rhs(vp, x, y, d, J, tau, k1d, k1J);
        for (int i = 0; i < 2; ++i) dt_[i] = d[i] + 0.5f * hs * k1d[i];
        for (int i = 0; i < 4; ++i) Jt[i] = J[i] + 0.5f * hs * k1J[i];
        flow_rhs(vp, x, y, dt_, Jt, tau - 0.5f * hs, k2d, k2J);
        for (int i = 0; i < 2; ++i) dt_[i] = d[i] + 0.5f * hs * k2d[i];
        for (int i = 0; i < 4; ++i) Jt[i] = J[i] + 0.5f * hs * k2J[i];
        flow_rhs(vp, x, y, dt_, Jt, tau - 0.5f * hs, k3d, k3J);
        for (int i = 0; i < 2; ++i) dt_[i] = d[i] + hs * k3d[i];
        for (int i = 0; i < 4; ++i) Jt[i] = J[i] + hs * k3J[i];
        flow_rhs(vp, x, y, dt_, Jt, tau - hs, k4d, k4J);
        for (int i = 0; i < 2; ++i) d[i] += hs / 6.f * (k1d[i] + 2.f * k2d[i] + 2.f * k3d[i] + k4d[i]);
        for (int i = 0; i < 4; ++i) J[i] += hs / 6.f * (k1J[i] + 2.f * k2J[i] + 2.f * k3J[i] + k4J[i]);
    }
}

namespace {

// Targets (unnormalised) for given inputs: X rows (x, y, phase) -> T rows (dx/h, dy/h, (J-I)/dt).
__global__ void k_targets(const VelParams vp, const float *__restrict__ X, float *__restrict__ T,
                          int n, float dt, float h, int m)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float d[2], J[4];
    flowmap_rk4(vp, X[3 * i], X[3 * i + 1], X[3 * i + 2], dt, m, d, J);
    float *o = T + 6 * i;
    o[0] = d[0] / h;
    o[1] = d[1] / h;
    o[2] = (J[0] - 1.f) / dt;
    o[3] = J[1] / dt;
    o[4] = J[2] / dt;
    o[5] = (J[3] - 1.f) / dt;
}

// Random training samples: Xn = network inputs in [-1, 1] (x, y, phase), T = normalised
// targets (divided by `scale`).
__global__ void k_samples(const VelParams vp, float *__restrict__ Xn, float *__restrict__ T, int n,
                          float dt, float h, int m, uint64_t seed, uint64_t step,
                          const float *__restrict__ scale)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t key = (seed * 0x100000001B3ull) ^ (step << 24) ^ ((uint64_t)i * 4);
    const float x = uniform01(key), y = uniform01(key + 1), ph = uniform01(key + 2);
    float d[2], J[4];
    flowmap_rk4(vp, x, y, ph, dt, m, d, J);
    Xn[3 * i] = 2.f * x - 1.f;
    Xn[3 * i + 1] = 2.f * y - 1.f;
    Xn[3 * i + 2] = 2.f * ph - 1.f;
    float *o = T + 6 * i;
    o[0] = d[0] / h / scale[0];
    o[1] = d[1] / h / scale[1];
    o[2] = (J[0] - 1.f) / dt / scale[2];
    o[3] = J[1] / dt / scale[3];
    o[4] = J[2] / dt / scale[4];
    o[5] = (J[3] - 1.f) / dt / scale[5];
}

// C[m][n] (+)= sum_k A(m,k) B(k,n) (+ bias[n]) with A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn] on the tensor cores: operands rounded to BF16, FP32
// accumulation in TMEM.  A block owns 128 rows of C (one TMEM lane each) and TN columns
// (16 or 128); the threads stage 64-wide K chunks of both operands from global memory into
// shared memory (any strides: transposed operands cost nothing extra here) in the
// core-matrix layout, and one thread issues the four K = 16 products of a chunk and
// commits them to an mbarrier that the block waits on (bounded) before the next chunk.
// Split-K: blockIdx.z covers K-range [z*kchunk, (z+1)*kchunk) and writes C + z*M*ldc.
constexpr int TM = 128, TKC = 64;
constexpr int kErrGemmTimeout = 4;

template <int R>
__device__ __forceinline__ void stage_operand(char *dst, const float *__restrict__ src, int rows,
                                              int64_t srow, int64_t sk, int r0, int k0, int kend)
{
    // task (r, q): 8 consecutive K values of row r as one 16-byte core-matrix row
    for (int e = threadIdx.x; e < R * (TKC / 8); e += TM) {
        const int r = e % R, q = e / R;
        const int gr = r0 + r, gk = k0 + 8 * q;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            v[j] = (gr < rows && gk + j < kend) ? src[(int64_t)gr * srow + (int64_t)(gk + j) * sk] : 0.f;
        *reinterpret_cast<uint4 *>(dst + cm_off(R, r, 8 * q)) =
            make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    }
}

template <int TN>
__global__ void __launch_bounds__(TM)
k_tc_gemm(int M, int N, int K, const float *__restrict__ A, int64_t sam, int64_t sak,
          const float *__restrict__ B, int64_t sbk, int64_t sbn, float *__restrict__ C, int64_t ldc,
          const float *__restrict__ bias, int kchunk, int *__restrict__ err)
{
    __shared__ __align__(1024) char As[TM * TKC * 2];
    __shared__ __align__(1024) char Bs[TN * TKC * 2];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    constexpr uint32_t TCOLS = TN < 32 ? 32 : TN;  // TMEM allocations are powers of two >= 32
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    C += (int64_t)blockIdx.z * M * ldc;
    if (tid == 0) mbar_init(&bar, 1);
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "n"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base;
    uint32_t phase = 0;
    bool ok = true, any = false;
    for (int k0 = kbeg; k0 < kend; k0 += TKC) {
        stage_operand<TM>(As, A, M, sam, sak, m0, k0, kend);
        stage_operand<TN>(Bs, B, N, sbn, sbk, n0, k0, kend);
        fence_async_smem();  // generic-proxy writes, read by the tensor core (async proxy)
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int q = 0; q < TKC / 16; ++q)
                umma(tbase, sdesc(As + q * 2 * TM * 16, TM * 16, 128), sdesc(Bs + q * 2 * TN * 16, TN * 16, 128),
                     idesc_bf16(TM, TN), (any || q > 0) ? 1u : 0u);
            umma_commit(&bar);
        }
        any = true;
        // the chunk is overwritten next: wait for its products (one warp polls)
        const bool done = tid < 32 ? mbar_wait_bounded(&bar, phase) : true;
        phase ^= 1u;
        if (__syncthreads_or(!done)) {
            ok = false;
            if (tid == 0) {
                atomicExch(err, kErrGemmTimeout);
                mbar_wait_bounded(&bar, phase ^ 1u);  // let the late products land
            }
            break;
        }
        tc_fence_after();
    }
    // epilogue: thread r holds row m0 + r (TMEM lane r); 8 columns per load
    const int gm = m0 + tid;
    const uint32_t ta = tbase + ((uint32_t)(tid & ~31) << 16);
    if (ok) {
#pragma unroll 1
        for (int c0 = 0; c0 < TN; c0 += 8) {
            uint32_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (any) tmem_ld8(ta + (uint32_t)c0, v);
            if (gm < M)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int gn = n0 + c0 + j;
                    if (gn < N) C[(int64_t)gm * ldc + gn] = __uint_as_float(v[j]) + (bias ? bias[gn] : 0.f);
                }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(TCOLS) : "memory");
}

// Column sums of G (n rows x no columns, row-major) over row blocks: P[z*no + o] = sum of
// rows [z*rows, (z+1)*rows) (the bias gradients' split-K partials; a fixed order).
__global__ void k_colsum(const float *__restrict__ G, int n, int no, int rows, float *__restrict__ P)
{
    const int o = threadIdx.x, z = blockIdx.x;
    if (o >= no) return;
    float acc = 0.f;
    const int r1 = min(n, (z + 1) * rows);
    for (int r = z * rows; r < r1; ++r) acc += G[(int64_t)r * no + o];
    P[(int64_t)z * no + o] = acc;
}

__global__ void k_silu(const float *__restrict__ Z, float *__restrict__ A, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) A[i] = silu(Z[i]);
}

// G = dL/dY for the mean squared error over n x OUT outputs; loss partial sums
__global__ void k_out_grad(const float *__restrict__ Y, const float *__restrict__ T,
                           float *__restrict__ G, int64_t n, double *loss)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < n) {
        const float r = Y[i] - T[i];
        G[i] = 2.f * r / (float)n;
        l = (double)r * r;
    }
    for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l / (double)n);
}

__global__ void k_act_bwd(const float *__restrict__ dA, const float *__restrict__ Z,
                          float *__restrict__ G, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) G[i] = dA[i] * silu_prime(Z[i]);
}

// C[i] = sum_z P[z*n + i] in a fixed order (the split-K partials)
__global__ void k_sum_splits(const float *__restrict__ P, int nsplit, int64_t n, float *__restrict__ C)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int z = 0; z < nsplit; ++z) s += P[z * n + i];
    C[i] = s;
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// C (M x N, row stride N) = A B (+ bias) on the tensor cores; K split into `nsplit`
// chunks reduced through `split` (nsplit*M*N floats) when nsplit > 1.
void gemm(int M, int N, int K, const float *A, int64_t sam, int64_t sak, const float *B, int64_t sbk,
          int64_t sbn, float *C, const float *bias, int nsplit, float *split, int *err, cudaStream_t s)
{
    const int kchunk = (K + nsplit - 1) / nsplit;
    float *dst = nsplit > 1 ? split : C;
    const float *bb = nsplit > 1 ? nullptr : bias;
    if (N > 16)
        k_tc_gemm<128><<<dim3(nb(N, 128), nb(M, TM), nsplit), TM, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn,
                                                                          dst, N, bb, kchunk, err);
    else
        k_tc_gemm<16><<<dim3(nb(N, 16), nb(M, TM), nsplit), TM, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn,
                                                                        dst, N, bb, kchunk, err);
    if (nsplit > 1) k_sum_splits<<<nb((int64_t)M * N, 256), 256, 0, s>>>(split, nsplit, (int64_t)M * N, C);
}

}  // namespace

cudaError_t launch_targets(const VelParams &vp, const float *X, float *T, int n, float dt, float h,
                           int substeps, cudaStream_t s)
{
    k_targets<<<nb(n, 128), 128, 0, s>>>(vp, X, T, n, dt, h, substeps);
    return cudaGetLastError();
}

cudaError_t launch_samples(const VelParams &vp, float *Xn, float *T, int n, float dt, float h,
                           int substeps, uint64_t seed, uint64_t step, const float *scale,
                           cudaStream_t s)
{
    k_samples<<<nb(n, 128), 128, 0, s>>>(vp, Xn, T, n, dt, h, substeps, seed, step, scale);
    return cudaGetLastError();
}

// Forward pass keeping pre-activations Z[l] (n x out_l) and activations A[l] (A[0] = X).
cudaError_t forward_train(const float *params, const float *X, int n, float *const *Z,
                          float *const *A, int *err, cudaStream_t s)
{
    const float *in = X;
    for (int l = 0; l < NLAYER; ++l) {
        const int ni = lin(l), no = lout(l);
        // Z = in (n x ni) * W^T (ni x no) + b ; W(k=i, n=o) = W[o*ni + i]
        gemm(n, no, ni, in, ni, 1, params + woff(l), 1, ni, Z[l], params + boff(l), 1, nullptr, err, s);
        if (l < NLAYER - 1) {
            k_silu<<<nb((int64_t)n * no, 256), 256, 0, s>>>(Z[l], A[l + 1], (int64_t)n * no);
            in = A[l + 1];
        }
    }
    return cudaGetLastError();
}

// Backward pass of the mean squared error against T: grad (flat, like params) and the loss.
cudaError_t backward_train(const float *params, const float *X, const float *T, int n,
                           float *const *Z, float *const *A, float *G0, float *G1, float *grad,
                           double *loss, const float *one, float *split, int *err, cudaStream_t s)
{
    (void)one;
    // K = n split into chunks of at least 128 samples, at most kMaxSplit of them
    const int nsplit = (n + 127) / 128 < kMaxSplit ? (n + 127) / 128 : kMaxSplit;
    const int64_t nout = (int64_t)n * OUT;
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    k_out_grad<<<nb(nout, 256), 256, 0, s>>>(Z[NLAYER - 1], T, G0, nout, loss);
    float *G = G0, *Gn = G1;
    for (int l = NLAYER - 1; l >= 0; --l) {
        const int ni = lin(l), no = lout(l);
        const float *Ain = l == 0 ? X : A[l];
        // dW (no x ni) = G^T (no x n) * Ain (n x ni): A(m=o,k=b) = G[b*no + o], B(k=b,n=i) = Ain[b*ni + i]
        gemm(no, ni, n, G, 1, no, Ain, ni, 1, grad + woff(l), nullptr, nsplit, split, err, s);
        // db (no) = column sums of G
        const int rows = (n + nsplit - 1) / nsplit;
        k_colsum<<<nsplit, HID, 0, s>>>(G, n, no, rows, split);
        k_sum_splits<<<nb(no, 256), 256, 0, s>>>(split, nsplit, no, grad + boff(l));
        if (l > 0) {
            // dA (n x ni) = G (n x no) * W (no x ni)
            gemm(n, ni, no, G, no, 1, params + woff(l), ni, 1, Gn, nullptr, 1, nullptr, err, s);
            k_act_bwd<<<nb((int64_t)n * ni, 256), 256, 0, s>>>(Gn, Z[l - 1], Gn, (int64_t)n * ni);
            float *tmp = G;
            G = Gn;
            Gn = tmp;
        }
    }
    return cudaGetLastError();
}

cudaError_t adam_step(float *params, const float *grad, float *m, float *v, float lr, float b1,
                      float b2, float eps, int step, cudaStream_t s)
{
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<nb(NPARAM, 256), 256, 0, s>>>(params, grad, m, v, NPARAM, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace gals
