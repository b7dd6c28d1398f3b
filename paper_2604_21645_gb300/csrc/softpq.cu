// softpq.cu -- differentiable soft-assignment PQ reconstruction loss and its
// gradients, for codebook refinement.
//
// Per row n and subspace m (width Ds), with temperature tau:
//     p_k  = softmax_k( -||x - c_k||^2 / tau )
//     xh   = sum_k p_k c_k
//     L    = (1/N) sum_n sum_m ||xh - x||^2
// The paper fixes hard assignments (Sec. 2.1); this relaxation is the
// refinement objective of the soft form, so everything below follows from
// differentiating L directly.  With r = xh - x, G_k = r.c_k, pg = r.xh and
// q_k = p_k (G_k - pg):
//     dL/dc_k = (2/N) sum_n [ p_k r + (2/tau) q_k (x - c_k) ]
//     dL/dx   = (2/N) [ -r + (2/tau) sum_k q_k c_k ]
// (the x-term of dL/dx drops out because sum_k q_k = 0).
//
// Arithmetic (FP32).  Distances are translation invariant, so each subspace is
// centred on its codeword mean mu: x' = x - mu, c'_k = c_k - mu.  The base-2
// logit of codeword k is t_k = x'.(2a c'_k) - a||c'_k||^2 - a||x'||^2 with
// a = log2(e)/tau, i.e. -a ||x - c_k||^2; e_k = 2^t_k, Z = sum_k e_k and
// p_k = e_k / Z.  t_k <= 0, so no shift is needed unless every codeword is so
// far that Z underflows (Z < 2^-100), in which case the row is recomputed with
// the maximum logit subtracted.  G_k - pg is formed as r.c'_k - r.xh' (the
// shift by mu cancels between the two).
//
// Work split.  The forward pass and the per-row part of the backward pass run
// one thread per (row, subspace), the codebook of the subspace in shared
// memory (every lane of a warp reads the same codeword: broadcast).  The
// codebook gradient needs a sum over rows for every codeword, so after each
// tile of 256 rows the block switches to one thread per codeword, re-derives
// p_k and q_k for the tile's rows from a per-row record in shared memory
// (x', r, the logit offset, 1/Z, r.xh') and adds the tile's contributions in
// FP32; tile sums go into FP64 per-thread totals, and the per-block totals are
// added in a fixed order by a finalise kernel.  Assignments are recomputed,
// never stored.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

constexpr int kTile = 256;  // rows per tile = threads per block

template <int DS>
struct Spq {
    static constexpr int P = 2 * DS + 4;   // codeword record: 2a c' [DS], c' [DS], -a||c'||^2, pad
    static constexpr int RP = 2 * DS + 4;  // row record: x' [DS], r [DS], logit offset, 1/Z, r.xh', pad
};

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// prep[m][k][P]: the scaled and centred codewords; mu[m][DS]: the codeword means
template <int DS>
__global__ void softpq_prep_kernel(const float *__restrict__ C, int Ks, float alpha, float *__restrict__ prep,
                                   float *__restrict__ mu)
{
    constexpr int P = Spq<DS>::P;
    const int m = blockIdx.x;
    __shared__ float smu[DS];
    const float *Cm = C + (size_t)m * Ks * DS;
    if (threadIdx.x < DS) {
        float s = 0.0f;
        for (int k = 0; k < Ks; ++k) s += Cm[k * DS + threadIdx.x];
        smu[threadIdx.x] = s / (float)Ks;
        mu[m * DS + threadIdx.x] = smu[threadIdx.x];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < Ks; k += blockDim.x) {
        float *rec = prep + ((size_t)m * Ks + k) * P;
        float nn = 0.0f;
#pragma unroll
        for (int j = 0; j < DS; ++j) {
            const float c = Cm[k * DS + j] - smu[j];
            nn = fmaf(c, c, nn);
            rec[j] = 2.0f * alpha * c;
            rec[DS + j] = c;
        }
        rec[2 * DS] = -alpha * nn;
#pragma unroll
        for (int j = 2 * DS + 1; j < P; ++j) rec[j] = 0.0f;
    }
}

template <int DS>
__device__ __forceinline__ void load_codebook(float *cb, const float *prep, int m, int Ks)
{
    constexpr int P = Spq<DS>::P;
    const float4 *src = reinterpret_cast<const float4 *>(prep + (size_t)m * Ks * P);
    float4 *dst = reinterpret_cast<float4 *>(cb);
    for (int i = threadIdx.x; i < Ks * P / 4; i += blockDim.x) dst[i] = src[i];
}

template <int DS>
__device__ __forceinline__ void load_row(const float *X, int64_t n, int D, int m, const float *mu, float *xp)
{
    const float4 *src = reinterpret_cast<const float4 *>(X + n * D + (int64_t)m * DS);
#pragma unroll
    for (int i = 0; i < DS / 4; ++i) {
        const float4 v = src[i];
        xp[4 * i + 0] = v.x - mu[4 * i + 0];
        xp[4 * i + 1] = v.y - mu[4 * i + 1];
        xp[4 * i + 2] = v.z - mu[4 * i + 2];
        xp[4 * i + 3] = v.w - mu[4 * i + 3];
    }
}

// logit of codeword record `rec` for the centred row xp with offset gam
template <int DS>
__device__ __forceinline__ float logit(const float *rec, const float *xp, float gam)
{
    float t = rec[2 * DS] + gam;
#pragma unroll
    for (int j = 0; j < DS; ++j) t = fmaf(xp[j], rec[j], t);
    return t;
}

// Z and sum_k e_k c'_k of one row; gam is updated when the row needs the max shift.
template <int DS>
__device__ __forceinline__ float softmax_pass(const float *cb, int Ks, const float *xp, float &gam, float *xa)
{
    constexpr int P = Spq<DS>::P;
    float Z = 0.0f;
#pragma unroll
    for (int j = 0; j < DS; ++j) xa[j] = 0.0f;
    for (int k = 0; k < Ks; ++k) {
        const float *rec = cb + k * P;
        const float e = ex2(logit<DS>(rec, xp, gam));
        Z += e;
#pragma unroll
        for (int j = 0; j < DS; ++j) xa[j] = fmaf(e, rec[DS + j], xa[j]);
    }
    if (Z < 0x1p-100f) {
        // every codeword is far: subtract the largest logit and recompute
        float tm = -INFINITY;
        for (int k = 0; k < Ks; ++k) tm = fmaxf(tm, logit<DS>(cb + k * P, xp, gam));
        gam -= tm;
        Z = 0.0f;
#pragma unroll
        for (int j = 0; j < DS; ++j) xa[j] = 0.0f;
        for (int k = 0; k < Ks; ++k) {
            const float *rec = cb + k * P;
            const float e = ex2(logit<DS>(rec, xp, gam));
            Z += e;
#pragma unroll
            for (int j = 0; j < DS; ++j) xa[j] = fmaf(e, rec[DS + j], xa[j]);
        }
    }
    return Z;
}

template <int DS>
__global__ void __launch_bounds__(kTile) softpq_fwd_kernel(const float *__restrict__ X, int64_t N, int D, int Ks,
                                                            const float *__restrict__ prep,
                                                            const float *__restrict__ mu, float alpha,
                                                            double *__restrict__ loss_acc)
{
    extern __shared__ float4 smem4[];
    float *cb = reinterpret_cast<float *>(smem4);
    const int m = blockIdx.y;
    load_codebook<DS>(cb, prep, m, Ks);
    float mum[DS];
#pragma unroll
    for (int j = 0; j < DS; ++j) mum[j] = mu[m * DS + j];
    __syncthreads();
    float ls = 0.0f, lc = 0.0f;  // Kahan pair
    const int64_t tiles = (N + kTile - 1) / kTile;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t n = tile * kTile + threadIdx.x;
        if (n >= N) continue;
        float xp[DS], xa[DS];
        load_row<DS>(X, n, D, m, mum, xp);
        float xx = 0.0f;
#pragma unroll
        for (int j = 0; j < DS; ++j) xx = fmaf(xp[j], xp[j], xx);
        float gam = -alpha * xx;
        const float Z = softmax_pass<DS>(cb, Ks, xp, gam, xa);
        const float iz = 1.0f / Z;
        float e = 0.0f;
#pragma unroll
        for (int j = 0; j < DS; ++j) {
            const float r = xa[j] * iz - xp[j];
            e = fmaf(r, r, e);
        }
        const float y = e - lc;
        const float t = ls + y;
        lc = (t - ls) - y;
        ls = t;
    }
    double tot = warp_sum((double)ls - (double)lc);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, tot);
}

template <int DS>
__global__ void __launch_bounds__(kTile) softpq_bwd_kernel(const float *__restrict__ X, int64_t N, int D, int M,
                                                            int Ks, const float *__restrict__ prep,
                                                            const float *__restrict__ mu, float alpha, float two_tau,
                                                            const float *__restrict__ grad_loss,
                                                            float *__restrict__ dX, double *__restrict__ part)
{
    constexpr int P = Spq<DS>::P;
    constexpr int RP = Spq<DS>::RP;
    extern __shared__ float4 smem4[];
    float *cb = reinterpret_cast<float *>(smem4);
    float *rows = cb + Ks * P;
    const int m = blockIdx.y;
    const int tid = threadIdx.x;
    load_codebook<DS>(cb, prep, m, Ks);
    float mum[DS];
#pragma unroll
    for (int j = 0; j < DS; ++j) mum[j] = mu[m * DS + j];
    const float coef = (grad_loss ? *grad_loss : 1.0f) * (float)(2.0 / (double)N);
    __syncthreads();

    // codeword owned in the per-codeword phase
    const bool own = tid < Ks;
    float ch[DS], cp[DS], cbeta = 0.0f;
    {
        const float *rec = cb + (own ? tid : 0) * P;
#pragma unroll
        for (int j = 0; j < DS; ++j) {
            ch[j] = rec[j];
            cp[j] = rec[DS + j];
        }
        cbeta = rec[2 * DS];
    }
    double ta[DS], tb[DS];
#pragma unroll
    for (int j = 0; j < DS; ++j) ta[j] = tb[j] = 0.0;

    const int64_t tiles = (N + kTile - 1) / kTile;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        // ---- per-row phase: thread = row ------------------------------------
        const int64_t n = tile * kTile + tid;
        float *rr = rows + tid * RP;
        if (n < N) {
            float xp[DS], xa[DS];
            load_row<DS>(X, n, D, m, mum, xp);
            float xx = 0.0f;
#pragma unroll
            for (int j = 0; j < DS; ++j) xx = fmaf(xp[j], xp[j], xx);
            float gam = -alpha * xx;
            const float Z = softmax_pass<DS>(cb, Ks, xp, gam, xa);
            const float iz = 1.0f / Z;
            float r[DS], pg = 0.0f;
#pragma unroll
            for (int j = 0; j < DS; ++j) {
                const float xh = xa[j] * iz;
                r[j] = xh - xp[j];
                pg = fmaf(r[j], xh, pg);
            }
            float w[DS];
#pragma unroll
            for (int j = 0; j < DS; ++j) w[j] = 0.0f;
            for (int k = 0; k < Ks; ++k) {
                const float *rec = cb + k * P;
                const float e = ex2(logit<DS>(rec, xp, gam));
                float d = -pg;
#pragma unroll
                for (int j = 0; j < DS; ++j) d = fmaf(r[j], rec[DS + j], d);
                const float q = e * d;
#pragma unroll
                for (int j = 0; j < DS; ++j) w[j] = fmaf(q, rec[DS + j], w[j]);
            }
            if (dX) {
                float g[DS];
#pragma unroll
                for (int j = 0; j < DS; ++j) g[j] = coef * fmaf(two_tau * iz, w[j], -r[j]);
                float4 *dst = reinterpret_cast<float4 *>(dX + n * D + (int64_t)m * DS);
#pragma unroll
                for (int i = 0; i < DS / 4; ++i) dst[i] = make_float4(g[4 * i], g[4 * i + 1], g[4 * i + 2], g[4 * i + 3]);
            }
#pragma unroll
            for (int j = 0; j < DS; ++j) {
                rr[j] = xp[j];
                rr[DS + j] = r[j];
            }
            rr[2 * DS] = gam;
            rr[2 * DS + 1] = iz;
            rr[2 * DS + 2] = pg;
        } else {
            // a row past the end contributes nothing (1/Z = 0 gives p = q = 0)
#pragma unroll
            for (int j = 0; j < RP; ++j) rr[j] = 0.0f;
        }
        __syncthreads();
        // ---- per-codeword phase: thread = codeword --------------------------
        if (own) {
            const int nr = (int)std::min<int64_t>(kTile, N - tile * kTile);
            float fa[DS], fb[DS];
#pragma unroll
            for (int j = 0; j < DS; ++j) fa[j] = fb[j] = 0.0f;
            for (int i = 0; i < nr; ++i) {
                const float *ri = rows + i * RP;
                float t = cbeta + ri[2 * DS];
#pragma unroll
                for (int j = 0; j < DS; ++j) t = fmaf(ri[j], ch[j], t);
                const float p = ex2(t) * ri[2 * DS + 1];
                float d = -ri[2 * DS + 2];
#pragma unroll
                for (int j = 0; j < DS; ++j) d = fmaf(ri[DS + j], cp[j], d);
                const float q = p * d;
#pragma unroll
                for (int j = 0; j < DS; ++j) {
                    fa[j] = fmaf(p, ri[DS + j], fa[j]);
                    fb[j] = fmaf(q, ri[j] - cp[j], fb[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < DS; ++j) {
                ta[j] += (double)fa[j];
                tb[j] += (double)fb[j];
            }
        }
        __syncthreads();
    }
    if (own) {
        double *dst = part + (((size_t)blockIdx.x * M + m) * Ks + tid) * (2 * DS);
#pragma unroll
        for (int j = 0; j < DS; ++j) {
            dst[j] = ta[j];
            dst[DS + j] = tb[j];
        }
    }
}

// dC[m][k][j] = (2/N) g sum_b (A + (2/tau) B), blocks added in order
__global__ void softpq_finalize_kernel(const double *__restrict__ part, int gx, int M, int Ks, int ds, double two_tau,
                                       const float *__restrict__ grad_loss, double two_over_n, float *__restrict__ dC)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * Ks * ds) return;
    const int j = idx % ds, mk = idx / ds;
    double a = 0.0, b = 0.0;
    for (int blk = 0; blk < gx; ++blk) {
        const double *src = part + ((size_t)blk * M * Ks + mk) * (2 * ds);
        a += src[j];
        b += src[ds + j];
    }
    const double g = grad_loss ? (double)*grad_loss : 1.0;
    dC[idx] = (float)(g * two_over_n * (a + two_tau * b));
}

__global__ void softpq_loss_kernel(const double *__restrict__ acc, double inv_n, float *__restrict__ loss)
{
    *loss = (float)(*acc * inv_n);
}

template <int DS>
int run_softpq(const float *X, int64_t N, int D, int M, int Ks, const float *C, float tau, float *loss,
               const float *grad_loss, float *dC, float *dX, cudaStream_t s)
{
    constexpr int P = Spq<DS>::P;
    constexpr int RP = Spq<DS>::RP;
    int dev = 0, sms = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    PQ_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const float alpha = (float)(1.4426950408889634 / (double)tau);
    Scratch ws(s);
    float *prep = ws.get<float>((size_t)M * Ks * P);
    float *mu = ws.get<float>((size_t)M * DS);
    if (ws.status) return ws.status;
    {
        ProfScope ps("softpq_prep", s);
        softpq_prep_kernel<DS><<<M, 256, 0, s>>>(C, Ks, alpha, prep, mu);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
    }
    const int64_t tiles = (N + kTile - 1) / kTile;
    if (loss) {
        double *acc = ws.get<double>(1, true);
        if (ws.status) return ws.status;
        const size_t smem = (size_t)Ks * P * sizeof(float);
        int per_sm = 0;
        PQ_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, softpq_fwd_kernel<DS>, kTile, smem));
        const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * std::max(per_sm, 1) / M));
        if (N > 0) {
            ProfScope ps("softpq_fwd", s);
            softpq_fwd_kernel<DS><<<dim3(gx, M), kTile, smem, s>>>(X, N, D, Ks, prep, mu, alpha, acc);
            count_launch();
            PQ_TRY_CUDA(cudaGetLastError());
        }
        softpq_loss_kernel<<<1, 1, 0, s>>>(acc, N > 0 ? 1.0 / (double)N : 0.0, loss);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
        return ws.status;
    }
    if (N == 0) {
        PQ_TRY_CUDA(cudaMemsetAsync(dC, 0, (size_t)M * Ks * DS * sizeof(float), s));
        return PQ_OK;
    }
    const size_t smem = ((size_t)Ks * P + (size_t)kTile * RP) * sizeof(float);
    PQ_TRY_CUDA(cudaFuncSetAttribute(softpq_bwd_kernel<DS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PQ_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, softpq_bwd_kernel<DS>, kTile, smem));
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * std::max(per_sm, 1) / M));
    double *part = ws.get<double>((size_t)gx * M * Ks * 2 * DS);
    if (ws.status) return ws.status;
    {
        ProfScope ps("softpq_bwd", s);
        softpq_bwd_kernel<DS><<<dim3(gx, M), kTile, smem, s>>>(X, N, D, M, Ks, prep, mu, alpha, (float)(2.0 / tau),
                                                               grad_loss, dX, part);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
    }
    {
        const int n = M * Ks * DS;
        ProfScope ps("softpq_finalize", s);
        softpq_finalize_kernel<<<(n + 255) / 256, 256, 0, s>>>(part, gx, M, Ks, DS, 2.0 / (double)tau, grad_loss,
                                                               2.0 / (double)N, dC);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
    }
    return ws.status;
}

}  // namespace

bool softpq_supported(int D, int M) { return M > 0 && D % M == 0 && (D / M == 4 || D / M == 8 || D / M == 16); }

int run_softpq_forward(const float *X, int64_t N, int D, int M, int Ks, const float *C, float tau, float *loss,
                       cudaStream_t s)
{
    switch (D / M) {
    case 4: return run_softpq<4>(X, N, D, M, Ks, C, tau, loss, nullptr, nullptr, nullptr, s);
    case 8: return run_softpq<8>(X, N, D, M, Ks, C, tau, loss, nullptr, nullptr, nullptr, s);
    case 16: return run_softpq<16>(X, N, D, M, Ks, C, tau, loss, nullptr, nullptr, nullptr, s);
    default: return fail(PQ_ENOTSUP, "soft PQ supports D/M in {4, 8, 16}");
    }
}

int run_softpq_backward(const float *X, int64_t N, int D, int M, int Ks, const float *C, float tau,
                        const float *grad_loss, float *dC, float *dX, cudaStream_t s)
{
    switch (D / M) {
    case 4: return run_softpq<4>(X, N, D, M, Ks, C, tau, nullptr, grad_loss, dC, dX, s);
    case 8: return run_softpq<8>(X, N, D, M, Ks, C, tau, nullptr, grad_loss, dC, dX, s);
    case 16: return run_softpq<16>(X, N, D, M, Ks, C, tau, nullptr, grad_loss, dC, dX, s);
    default: return fail(PQ_ENOTSUP, "soft PQ supports D/M in {4, 8, 16}");
    }
}

}  // namespace pqgb
