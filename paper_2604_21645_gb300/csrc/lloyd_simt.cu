// lloyd_simt.cu -- PQ Lloyd pass in the plain FP32 form (Sec. 2.1: k-means
// in every subspace; encode = nearest codeword per subspace), the centroid
// finalisation, and decode + reconstruction error (Sec. 2.1, Sec. 3).
//
// Assignment.  For row x and codeword c_k of subspace m the kernel scores
//     s_k = ||c_k||^2 / 2 - x . c_k        (argmin s_k == argmin ||x - c_k||^2)
// with FP32 fused multiply-adds and keeps the two smallest scores.  The
// rounding error of every score is below
//     delta = 2.2 gamma_{Ds+1} (max_k ||c_k||^2/2 + ||x|| max_k ||c_k||)
//             + 1e-13 (||x|| + max_k ||c_k||)^2
// (the last term covers FP64 rounding of the reference distances).  If the
// second-best score exceeds the best by more than 2 delta the best index is
// the exact argmin.  Otherwise every codeword whose score is within 2 delta
// of the best is re-scored in FP64 by direct differences (the rule of the
// CPU reference) and the lowest-index minimum wins.  Codes are therefore
// exact, not approximate.
//
// Update.  Each member adds its residual x - c_code to its codeword's sums in
// the exact fixed-point format of common.cuh (int32 shared-memory atomics,
// independent of the order of the additions); each block writes its sums as
// int64, and the finalise kernel adds the blocks in int64 and moves every
// codeword by the float-float mean residual of its members.
#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

constexpr int kThreads = 256;

// shared sums: row stride DS + 1 words, so that the atomics of a warp's random codes spread over the banks
template <int DS>
constexpr int acc_stride() { return DS + 1; }

template <int DS>
struct SmemLayout {
    static size_t bytes(int Ks, bool fit)
    {
        size_t b = (size_t)Ks * DS * sizeof(float) + (size_t)Ks * sizeof(float);
        if (fit) b += 3 * (size_t)Ks * acc_stride<DS>() * sizeof(int) + (size_t)Ks * sizeof(int);
        return b;
    }
};

template <int DS>
__device__ __forceinline__ void load_row(const float *__restrict__ src, float (&x)[DS], bool vec)
{
    if constexpr (DS % 4 == 0) {
        if (vec) {
#pragma unroll
            for (int j = 0; j < DS; j += 4) {
                float4 v = __ldg(reinterpret_cast<const float4 *>(src + j));
                x[j] = v.x; x[j + 1] = v.y; x[j + 2] = v.z; x[j + 3] = v.w;
            }
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < DS; ++j) x[j] = __ldg(src + j);
}

// Scores of every codeword (same rounding as the main loop).
template <int DS>
__device__ __forceinline__ float score(const float (&x)[DS], const float *cb, const float *cn, int k)
{
    float s = cn[k];
#pragma unroll
    for (int j = 0; j < DS; ++j) s = fmaf(-x[j], cb[k * DS + j], s);
    return s;
}

// Uncertain case: FP64 direct-difference distances over the candidate window.
template <int DS>
__device__ __noinline__ int fp64_recheck(const float (&x)[DS], const float *cb, const float *cn, int Ks, float m1,
                                         float win)
{
    double best = DBL_MAX;
    int bk = 0;
    for (int k = 0; k < Ks; ++k) {
        if (score<DS>(x, cb, cn, k) <= m1 + win) {
            double d = d2_fp64(x, cb + k * DS, DS);
            if (d < best) { best = d; bk = k; }
        }
    }
    return bk;
}

template <int DS>
__global__ void __launch_bounds__(kThreads) pq_pass_f32_kernel(const PqPass a, const bool vec)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.y, Ks = a.Ks, tid = threadIdx.x;
    const bool fit = a.part.active();
    // chunk of this block (batched form) and its rows
    int chunk = 0, lb = blockIdx.x, gxc = gridDim.x;
    int64_t r0 = 0, r1 = a.N;
    if (a.blk_chunk) {
        chunk = a.blk_chunk[blockIdx.x];
        lb = blockIdx.x - a.chunk_blk[chunk];
        gxc = a.chunk_blk[chunk + 1] - a.chunk_blk[chunk];
        r0 = a.chunk_off[chunk];
        r1 = a.chunk_off[chunk + 1];
    }
    constexpr int AS = acc_stride<DS>();
    float *cb = reinterpret_cast<float *>(smem_raw);
    float *cn = cb + Ks * DS;
    int *acch = reinterpret_cast<int *>(cn + Ks);  // [Ks][AS] high parts, then low parts, FP32 sums, counts
    int *accl = acch + Ks * AS;
    float *accf = reinterpret_cast<float *>(accl + Ks * AS);
    int *cnt = reinterpret_cast<int *>(accf + Ks * AS);
    __shared__ float s_red[kThreads / 32];
    __shared__ double s_sse[kThreads / 32];
    __shared__ float s_mu[DS];
    __shared__ unsigned s_r0;

    const float *Cm = a.C + ((size_t)chunk * a.M + m) * Ks * DS;
    for (int e = tid; e < Ks * DS; e += kThreads) cb[e] = Cm[e];
    if (fit) {
        for (int e = tid; e < Ks * AS; e += kThreads) {
            acch[e] = 0;
            accl[e] = 0;
            accf[e] = 0.0f;
        }
        for (int k = tid; k < Ks; k += kThreads) cnt[k] = 0;
    }
    if (tid == 0) s_r0 = 0u;
    __syncthreads();
    if (fit) {
        // residual scale of the fixed-point sums: twice the largest codeword norm about the codeword mean
        if (tid < DS) {
            float mu = 0.0f;
            for (int k = 0; k < Ks; ++k) mu += cb[k * DS + tid];
            s_mu[tid] = mu / (float)Ks;
        }
        __syncthreads();
        for (int k = tid; k < Ks; k += kThreads) {
            float n = 0.0f;
#pragma unroll
            for (int j = 0; j < DS; ++j) {
                const float t = cb[k * DS + j] - s_mu[j];
                n = fmaf(t, t, n);
            }
            atomicMax(&s_r0, __float_as_uint(sqrtf(n)));
        }
    }
    __syncthreads();
    float lmax = 0.0f;
    for (int k = tid; k < Ks; k += kThreads) {
        float n = 0.0f;
#pragma unroll
        for (int j = 0; j < DS; ++j) n = fmaf(cb[k * DS + j], cb[k * DS + j], n);
        cn[k] = 0.5f * n;
        lmax = fmaxf(lmax, 0.5f * n);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((tid & 31) == 0) s_red[tid >> 5] = lmax;
    __syncthreads();
    float nmax = 0.0f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) nmax = fmaxf(nmax, s_red[w]);
    nmax *= 1.0f + 4.0f * gamma_f32(DS + 1);
    const float cmax = sqrtf(2.0f * nmax) * (1.0f + 1e-6f);
    const float gam = 2.2f * gamma_f32(DS + 1);

    double sse = 0.0;
    unsigned rechecks = 0;
    const int64_t stride = (int64_t)gxc * kThreads;
    // every block of a chunk uses the same format: the row bound is the busiest block's rows
    const FixFmt fx = fix_format(((r1 - r0 + stride - 1) / stride) * kThreads,
                                 2.0f * __uint_as_float(s_r0) * (1.0f + 1e-6f));
    for (int bi = 0;; ++bi) {
        const int64_t base = r0 + (int64_t)bi * stride + (int64_t)lb * kThreads;
        if (base >= r1) break;
        const int64_t row = base + tid;
        if (row < r1) {
            float x[DS];
            load_row<DS>(a.X + row * a.D + (int64_t)m * DS, x, vec);
            float xx = 0.0f;
#pragma unroll
            for (int j = 0; j < DS; ++j) xx = fmaf(x[j], x[j], xx);
            const float xn = sqrtf(xx) * (1.0f + 1e-6f);
            float m1 = FLT_MAX, m2 = FLT_MAX;
            int i1 = 0;
#pragma unroll 4
            for (int k = 0; k < Ks; ++k) {
                const float s = score<DS>(x, cb, cn, k);
                const bool lt = s < m1;
                m2 = lt ? m1 : fminf(m2, s);
                i1 = lt ? k : i1;
                m1 = fminf(m1, s);
            }
            const float t = xn + cmax;
            const float delta = gam * (nmax + xn * cmax) + 1e-13f * t * t;
            int code = i1;
            if (!(m2 - m1 > 2.0f * delta)) {
                code = fp64_recheck<DS>(x, cb, cn, Ks, m1, 2.0f * delta);
                ++rechecks;
            }
            float e = 0.0f;
#pragma unroll
            for (int j = 0; j < DS; ++j) {
                const float d = x[j] - cb[code * DS + j];
                e = fmaf(d, d, e);
            }
            sse += (double)e;
            if (a.codes) a.codes[row * a.M + m] = (uint8_t)code;
            if (fit) {
                bool big = false;
#pragma unroll
                for (int j = 0; j < DS; ++j) big |= !(fabsf(__fmul_rn(x[j] - cb[code * DS + j], fx.scale)) < fx.lim);
                const int o = code * AS;
                if (!big) {
#pragma unroll
                    for (int j = 0; j < DS; ++j) {
                        const int q = __float2int_rn(__fmul_rn(x[j] - cb[code * DS + j], fx.scale));
                        atomicAdd(acch + o + j, q >> fx.L);
                        atomicAdd(accl + o + j, q & ((1 << fx.L) - 1));
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < DS; ++j) atomicAdd(accf + o + j, x[j] - cb[code * DS + j]);
                }
                atomicAdd(cnt + code, 1);
            }
        }
    }
    if (fit) {
        __syncthreads();
        const size_t base = ((size_t)blockIdx.x * a.M + m) * Ks;
        for (int e = tid; e < Ks * DS; e += kThreads) {
            const int k = e / DS, j = e % DS;
            a.part.q[base * DS + e] = (long long)acch[k * AS + j] * (1LL << fx.L) + (long long)accl[k * AS + j];
            a.part.o[base * DS + e] = accf[k * AS + j];
        }
        for (int k = tid; k < Ks; k += kThreads) a.part.cnt[base + k] = cnt[k];
        if (lb == 0 && tid == 0) a.part.F[chunk * a.M + m] = fx.F;
    }
    if (a.sse) {
        sse = warp_sum(sse);
        if ((tid & 31) == 0) s_sse[tid >> 5] = sse;
        __syncthreads();
        if (tid == 0) {
            double v = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) v += s_sse[w];
            atomicAdd(a.sse, v);
        }
    }
    if (a.rechecks) {
        unsigned r = warp_sum(rechecks);
        if ((tid & 31) == 0 && r) atomicAdd(a.rechecks, (unsigned long long)r);
    }
}

// One thread per (chunk, subspace, codeword, dimension): the blocks' int64 sums added
// exactly, the FP32 sums added with TwoSum (block order), the total scaled to a float-float
// value, divided by the member count in float-float, and added to the codeword.
__global__ void pq_finalize_kernel(const Partials part, int gx, int M, int Ks, int ds, float *C,
                                   unsigned long long *empties, int n_chunks, const int *__restrict__ chunk_blk,
                                   long long *__restrict__ counts)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_chunks * M * Ks * ds) return;
    const int j = (int)(idx % ds);
    const int64_t cw = idx / ds;
    const int c = (int)(cw / ((int64_t)M * Ks)), m = (int)((cw / Ks) % M), k = (int)(cw % Ks);
    const int b0 = chunk_blk ? chunk_blk[c] : 0, b1 = chunk_blk ? chunk_blk[c + 1] : gx;
    const long long n = finalize_element(part, M, Ks, ds, C, c, m, k, j, b0, b1);
    if (counts && j == 0) counts[cw] = n;
    if (n == 0 && empties && j == 0) atomicAdd(empties, 1ull);
}

// One thread per (row, subspace): reconstruction and/or squared error.
__global__ void decode_rmse_kernel(const uint8_t *__restrict__ codes, const float *__restrict__ C,
                                   const float *__restrict__ X, int64_t N, int D, int M, int Ks, int ds,
                                   float *__restrict__ Xhat, double *sse)
{
    __shared__ double s_sse[8];
    double acc = 0.0;
    const int64_t total = N * M;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = i / M;
        const int m = (int)(i - n * M);
        const int code = codes[i];
        if (code >= Ks) continue;  // not a codeword index: contributes nothing
        const float *c = C + ((size_t)m * Ks + code) * ds;
        const int64_t off = n * D + (int64_t)m * ds;
        float e = 0.0f;
        for (int j = 0; j < ds; ++j) {
            const float v = c[j];
            if (Xhat) Xhat[off + j] = v;
            if (X) {
                const float d = X[off + j] - v;
                e = fmaf(d, d, e);
            }
        }
        acc += (double)e;
    }
    if (sse) {
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) s_sse[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_sse[w];
            atomicAdd(sse, v);
        }
    }
}

template <int DS>
int launch_ds(PqPass &p, cudaStream_t s)
{
    const bool fit = p.part.active();
    const size_t smem = SmemLayout<DS>::bytes(p.Ks, fit);
    PQ_TRY_CUDA(cudaFuncSetAttribute(pq_pass_f32_kernel<DS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const bool vec = (p.D % 4 == 0) && ((reinterpret_cast<uintptr_t>(p.X) & 15) == 0);
    dim3 grid(p.gx, p.M);
    ProfScope ps("pq_pass_f32", s);
    pq_pass_f32_kernel<DS><<<grid, kThreads, smem, s>>>(p, vec);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

}  // namespace

int pq_pass_blocks_per_subspace(const PqPass &p)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    // about four resident blocks per SM over all subspaces, never more than the rows need
    const int64_t want = std::max<int64_t>(1, (4LL * sms + p.M - 1) / p.M);
    const int64_t need = (p.N + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min(want, need));
}

int launch_pq_pass_f32(PqPass &p, cudaStream_t s)
{
    if (p.gx <= 0) p.gx = pq_pass_blocks_per_subspace(p);
    switch (p.ds) {
    case 1: return launch_ds<1>(p, s);
    case 2: return launch_ds<2>(p, s);
    case 4: return launch_ds<4>(p, s);
    case 8: return launch_ds<8>(p, s);
    case 16: return launch_ds<16>(p, s);
    case 32: return launch_ds<32>(p, s);
    default: return fail(PQ_ENOTSUP, "subspace width Ds=%d not supported (1, 2, 4, 8, 16 or 32)", p.ds);
    }
}

int launch_pq_finalize(const Partials &part, int gx, int M, int Ks, int ds, float *C, unsigned long long *empties,
                       cudaStream_t s, int n_chunks, const int *chunk_blk, long long *counts)
{
    const int64_t n = (int64_t)n_chunks * M * Ks * ds;
    ProfScope ps("pq_finalize", s);
    pq_finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, gx, M, Ks, ds, C, empties, n_chunks,
                                                                  chunk_blk, counts);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

int launch_decode_rmse(const uint8_t *codes, const float *C, const float *X, int64_t N, int D, int M, int Ks,
                       float *Xhat, double *sse, cudaStream_t s)
{
    const int64_t total = N * M;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
    ProfScope ps("decode_rmse", s);
    decode_rmse_kernel<<<blocks, 256, 0, s>>>(codes, C, X, N, D, M, Ks, D / M, Xhat, sse);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

}  // namespace pqgb
