// common.cuh -- device helpers shared by the libpqgb kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "pqgb.h"

namespace pqgb {

// ---------------------------------------------------------------------------
// Host-side bookkeeping (defined in api.cu).
// ---------------------------------------------------------------------------
void count_launch(int n = 1);
int fail(int status, const char *fmt, ...);
void clear_error();  // empties this thread's last-error message (done on entry by every call)
int cuda_check(cudaError_t e, const char *what);
#define PQ_TRY_CUDA(expr)                                        \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) return ::pqgb::cuda_check(_e, #expr); \
    } while (0)
#define PQ_TRY(expr)                 \
    do {                             \
        int _s = (expr);             \
        if (_s != PQ_OK) return _s;  \
    } while (0)

// Optional per-kernel timing: while profiling is enabled (pq_profile_enable)
// a scope records a CUDA event pair around the launches it encloses on its
// stream; pq_profile_collect sums the elapsed times per kernel name.
struct ProfScope {
    int idx = -1;
    cudaStream_t s = nullptr;
    ProfScope(const char *name, cudaStream_t st);
    ~ProfScope();
};

// Device word where kernels record asynchronous failures (PQ_ETIMEOUT, ...).
int *device_error_word(int device);

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter-based generator:
// output i of the generator seeded with s is the finaliser applied to
// s + (i+1)*gamma.  Stream t of seed s is seeded with output t of seed s.
// ---------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStreamSubsample = 0xFFFFFFFFull;
constexpr uint64_t kStreamChunk = 0xFFFFFFFEull;

__host__ __device__ __forceinline__ uint64_t splitmix_out(uint64_t s, uint64_t i)
{
    uint64_t z = s + (i + 1) * kGamma;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t rng_draw(uint64_t seed, uint64_t stream, uint64_t i)
{
    return splitmix_out(splitmix_out(seed, stream), i);
}

// floor(r53 * n / 2^53): uniform index in [0, n) from a 53-bit draw.
__host__ __device__ __forceinline__ int64_t scale_index(uint64_t r53, uint64_t n)
{
#ifdef __CUDA_ARCH__
    uint64_t hi = __umul64hi(r53, n);
    uint64_t lo = r53 * n;
#else
    unsigned __int128 p = (unsigned __int128)r53 * n;
    uint64_t hi = (uint64_t)(p >> 64), lo = (uint64_t)p;
#endif
    return (int64_t)((hi << 11) | (lo >> 53));
}

// ---------------------------------------------------------------------------
// Exactly rounded building blocks (no contraction into fused multiply-add).
// ---------------------------------------------------------------------------

// FP64 squared distance, direct differences, dimension order.  This is the
// reference decision rule: every uncertain nearest-centroid choice is taken
// with it.
__device__ __forceinline__ double d2_fp64(const float *x, const float *c, int ds)
{
    double acc = 0.0;
    for (int j = 0; j < ds; ++j) {
        double t = __dsub_rn((double)x[j], (double)c[j]);
        acc = __dadd_rn(acc, __dmul_rn(t, t));
    }
    return acc;
}

// FP64 squared distance as a sum of subspace terms: each run of `ds` consecutive dimensions
// summed in dimension order from zero, the terms then added in subspace order -- the way a PQ
// distance table (one FP64 entry per subspace) adds up.  ds <= 0 means one run over all D.
__device__ __forceinline__ double d2_fp64_sub(const float *x, const float *c, int D, int ds)
{
    if (ds <= 0 || ds >= D) return d2_fp64(x, c, D);
    double acc = 0.0;
    for (int m0 = 0; m0 < D; m0 += ds) acc = __dadd_rn(acc, d2_fp64(x + m0, c + m0, ds));
    return acc;
}

// Error-free addition: s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// Fast TwoSum (Dekker): s + e == a + b exactly when |a| >= |b| or a == 0.
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fadd_rn(b, __fsub_rn(a, s));
}

// TwoProduct: p + e == a * b exactly (the FMA returns the rounding error of the product).
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Float-float ("double-float") sum of (ah + al) and (bh + bl), normalised.
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float &sh, float &sl)
{
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    fast_two_sum(s, e, sh, sl);
}

// Float-float quotient (ah + al) / (bh + bl): one correction step of the FP32 quotient.
__device__ __forceinline__ void ff_div(float ah, float al, float bh, float bl, float &qh, float &ql)
{
    const float q1 = __fdiv_rn(ah, bh);
    float p, pe;
    two_prod(q1, bh, p, pe);
    float r = __fsub_rn(__fsub_rn(ah, p), pe);
    r = __fadd_rn(r, al);
    r = __fsub_rn(r, __fmul_rn(q1, bl));
    fast_two_sum(q1, __fdiv_rn(r, bh), qh, ql);
}

// Exact float-float value of a 64-bit integer: v == hi + lo with |lo| <= ulp(hi)/2 (the
// remainder v - hi is below 2^40 in magnitude, so its conversion loses at most 2^-24 of it).
__device__ __forceinline__ void ll_to_ff(long long v, float &hi, float &lo)
{
    hi = __ll2float_rn(v);
    lo = __ll2float_rn(v - __float2ll_rn(hi));
}

// ---------------------------------------------------------------------------
// Centroid update in exact fixed point (both forms of the Lloyd pass).
//
// Each member adds its residual r = x - c_code.  An element becomes the integer
// q = rint(r * 2^F) and is added into a block's shared sums as two int32 parts,
// q >> L and q & (2^L - 1); with at most 2^b rows per block (b = bit length of
// the row bound), L = 31 - b keeps the low sum below 2^31 and |q| < 2^qb,
// qb = min(30, 61 - 2b), keeps the high sum below 2^31 and q an int32.  F puts the
// residual scale r0 at that limit: elements beyond r0 go to an FP32 sum
// instead.  The integer sums do not depend on the order of the additions; each
// block writes hi * 2^L + lo as one int64 per (subspace, codeword, dimension),
// and the finalise kernel adds the blocks in int64 (exact), converts the total to
// a float-float value, adds the FP32 sums with TwoSum and moves the codeword by
// the float-float mean residual.  An element's quantisation error is at most
// 2^-(F+1), i.e. 2^-(qb+1) of r0 (rows per block of 2^16: 2^-30 of r0).
// ---------------------------------------------------------------------------
struct FixFmt {
    int L, F;
    float scale, lim;
};
__host__ __device__ __forceinline__ FixFmt fix_format(int64_t rows, float r0)
{
    int b = 0;
    while (b < 62 && ((int64_t)1 << b) <= rows) ++b;  // bit length of the row bound
    FixFmt f;
    f.L = 31 - b;
    const int qb = (61 - 2 * b) < 30 ? (61 - 2 * b) : 30;  // |q| < 2^qb, and q fits an int32
    int e = 0;
    (void)frexpf(r0 > 0.0f ? r0 : 1.0f, &e);  // r0 < 2^e
    f.F = qb - e;
    f.F = f.F < -100 ? -100 : (f.F > 100 ? 100 : f.F);
    f.scale = ldexpf(1.0f, f.F);
    f.lim = ldexpf(1.0f, qb);
    return f;
}

// gamma_n = n u / (1 - n u), u = 2^-24: the classical bound on the relative
// error of an n-term FP32 sum of products.
__host__ __device__ __forceinline__ float gamma_f32(int n)
{
    const float u = 5.9604645e-8f;
    return (n * u) / (1.0f - n * u);
}

// ---------------------------------------------------------------------------
// Memory-model helpers for bounded device-wide waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Spin budget of every device-side wait: ~2^22 polls (each an L2 round trip or
// an mbarrier try-wait) is a few seconds at most on a healthy GPU.
constexpr unsigned kSpinLimit = 1u << 22;
// Budget the k-means++ seeding's inter-block waits use: kSpinLimit unless a test
// has lowered it (pq_test_set_spin_limit) to make those waits run out on purpose.
unsigned seeding_spin_limit();

// Barrier over the `nblk` blocks sharing `bar` ({arrive count, generation}).
// Blocks must be co-resident (cooperative launch).  Returns false, after
// recording PQ_ETIMEOUT in *err, if the wait ran out; every later barrier of
// the same kernel then returns false at once so the kernel can unwind.
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Barrier of the nblk co-resident blocks that share `bar` ([0] arrivals, [1] generation).
// The arrival is an acquire-release atomic and the wait an acquire load, so the block's
// writes (ordered before thread 0 by the first __syncthreads) are visible to every block
// after the barrier.  The wait is bounded: false (PQ_ETIMEOUT recorded) if it ran out
// or another block already failed.
__device__ __forceinline__ bool block_group_barrier(unsigned *bar, unsigned nblk, int *err,
                                                    unsigned limit = kSpinLimit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = (*(volatile int *)err == 0);
        if (ok) {
            const unsigned gen = ld_acquire_u32(bar + 1);
            const unsigned arrived = atom_add_acq_rel_u32(bar, 1u);
            if (arrived == nblk - 1) {
                atomicExch(bar, 0u);
                st_release_u32(bar + 1, gen + 1);
            } else {
                for (unsigned it = 0; ld_acquire_u32(bar + 1) == gen; ++it) {
                    if (it >= limit || ((it & 255) == 255 && *(volatile int *)err != 0)) {
                        atomicCAS(err, 0, PQ_ETIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace pqgb
