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

// Error-free addition: s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
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
