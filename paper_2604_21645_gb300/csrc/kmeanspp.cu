// kmeanspp.cu -- k-means++ (D^2 sampling) seeding of the per-subspace k-means
// of PQ fit (Sec. 2.1; the paper does not name the seeding, k-means++ is the
// reading taken here) and of the coarse quantizer.
//
// Sampling rule (identical, bit for bit, to the CPU reference because both
// sides use only exactly rounded FP32 operations and integer arithmetic):
//   round 0: pick floor(u * n) with u the first draw of stream m;
//   D2_i = FP32 squared distance of point i to its nearest seed so far
//          (products and sums rounded separately, dimension order);
//   after round 0 fix sh = 62 - ceil(log2 n) - E with max_i D2_i < 2^E;
//   round t >= 1: w_i = floor(D2_i * 2^sh) (integers), W = sum w_i, pick the
//          smallest i whose inclusive prefix sum exceeds floor(r * W / 2^53),
//          r the 53-bit draw t of stream m; W == 0 falls back to floor(u*n).
//
// One cooperative launch seeds all M subspaces: blocks (b, m) own a slice of
// the points of subspace m and keep its D2 values in shared memory; each
// round costs two barriers among the blocks of subspace m (bounded spins).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

constexpr int kThreads = 256;

struct KppArgs {
    const float *P;
    int64_t ld;
    int64_t n;
    int ds, M, Ks;
    uint64_t seed;
    float *C;                     // [M][Ks][ds]
    unsigned *bars;               // [M][2]
    unsigned long long *bsum;     // [M][bps]
    unsigned *dmax_bits;          // [M]
    long long *sel;               // [M]
    int *err;
    int bps;
    int64_t nb;                   // points per block
};

__device__ __forceinline__ float d2_f32_exact(const float *x, const float *c, int ds)
{
    float acc = 0.0f;
    for (int j = 0; j < ds; ++j) {
        float t = __fsub_rn(x[j], c[j]);
        acc = __fadd_rn(acc, __fmul_rn(t, t));
    }
    return acc;
}

__device__ __forceinline__ uint64_t weight(float d2, double scale, bool any)
{
    return any ? (uint64_t)__double2ull_rz(__dmul_rn((double)d2, scale)) : 0ull;
}

// Block-wide inclusive scan of one uint64 per thread; returns the inclusive value.
__device__ __forceinline__ uint64_t block_scan_u64(uint64_t v, uint64_t *sh_warp)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) sh_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint64_t w = (lane < kThreads / 32) ? sh_warp[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < kThreads / 32) sh_warp[lane] = w;
    }
    __syncthreads();
    uint64_t add = wid > 0 ? sh_warp[wid - 1] : 0ull;
    __syncthreads();
    return v + add;
}

__global__ void __launch_bounds__(kThreads) kmeanspp_kernel(KppArgs a)
{
    extern __shared__ float s_d2[];  // [nb]
    __shared__ float s_center[256];  // ds <= 256
    __shared__ uint64_t s_warp[kThreads / 32];
    __shared__ float s_fmax[kThreads / 32];
    __shared__ long long s_pick;

    const int m = blockIdx.y, b = blockIdx.x, tid = threadIdx.x;
    const int ds = a.ds;
    const int64_t i0 = (int64_t)b * a.nb;
    const int64_t i1 = min(a.n, i0 + a.nb);
    const int64_t cnt = i1 > i0 ? i1 - i0 : 0;
    const float *Pm = a.P + (int64_t)m * ds;
    unsigned *bar = a.bars + 2 * m;
    float *Cm = a.C + (size_t)m * a.Ks * ds;

    // ---- round 0 -----------------------------------------------------------
    long long pick = scale_index(rng_draw(a.seed, (uint64_t)m, 0) >> 11, (uint64_t)a.n);
    for (int j = tid; j < ds; j += kThreads) {
        float v = Pm[pick * a.ld + j];
        s_center[j] = v;
        if (b == 0) Cm[j] = v;
    }
    __syncthreads();
    float lmax = 0.0f;
    for (int64_t i = tid; i < cnt; i += kThreads) {
        float d = d2_f32_exact(Pm + (i0 + i) * a.ld, s_center, ds);
        s_d2[i] = d;
        lmax = fmaxf(lmax, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((tid & 31) == 0) s_fmax[tid >> 5] = lmax;
    __syncthreads();
    if (tid == 0) {
        float v = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) v = fmaxf(v, s_fmax[w]);
        atomicMax(a.dmax_bits + m, __float_as_uint(v));  // non-negative floats order as integers
    }
    if (!block_group_barrier(bar, a.bps, a.err)) return;
    const float dmax = __uint_as_float(ld_acquire_u32(a.dmax_bits + m));
    const bool any = dmax > 0.0f;
    int L = 0;
    while (((int64_t)1 << L) < a.n) ++L;
    int E = 0;
    if (any) E = ((__float_as_uint(dmax) >> 23) & 0xff) - 126;  // dmax in [2^(E-1), 2^E) (dmax normal)
    if (any && ((__float_as_uint(dmax) >> 23) & 0xff) == 0) {  // subnormal maximum
        unsigned mant = __float_as_uint(dmax) & 0x7fffff;
        E = -126 - (__clz(mant) - 9) ;
    }
    const int sh = 62 - L - E;
    const double scale = __longlong_as_double((long long)(sh + 1023) << 52);

    // Each thread owns a contiguous segment of the block's points for the scan.
    const int64_t seg = (cnt + kThreads - 1) / kThreads;
    const int64_t s0 = min(cnt, (int64_t)tid * seg), s1 = min(cnt, s0 + seg);

    for (int t = 1; t < a.Ks; ++t) {
        const uint64_t r = rng_draw(a.seed, (uint64_t)m, (uint64_t)t) >> 11;
        uint64_t part = 0;
        for (int64_t i = s0; i < s1; ++i) part += weight(s_d2[i], scale, any);
        const uint64_t incl = block_scan_u64(part, s_warp);
        if (tid == kThreads - 1) a.bsum[(size_t)m * a.bps + b] = incl;
        if (!block_group_barrier(bar, a.bps, a.err)) return;

        if (tid == 0) {
            uint64_t W = 0;
            for (int q = 0; q < a.bps; ++q) W += *(volatile unsigned long long *)(a.bsum + (size_t)m * a.bps + q);
            long long p = -1;
            int owner = -1;
            uint64_t thr_local = 0;
            if (W == 0) {
                p = scale_index(r, (uint64_t)a.n);
            } else {
                const uint64_t thr = (__umul64hi(r, W) << 11) | ((r * W) >> 53);
                uint64_t acc = 0;
                for (int q = 0; q < a.bps; ++q) {
                    uint64_t v = *(volatile unsigned long long *)(a.bsum + (size_t)m * a.bps + q);
                    if (acc + v > thr) { owner = q; thr_local = thr - acc; break; }
                    acc += v;
                }
            }
            s_pick = p;
            s_warp[0] = thr_local;
            s_fmax[0] = __int_as_float(owner);
        }
        __syncthreads();
        const int owner = __float_as_int(s_fmax[0]);
        const uint64_t thr_local = s_warp[0];
        __syncthreads();
        if (owner == b) {
            // inclusive prefix (exclusive of this thread's segment) then a sequential walk
            const uint64_t excl = incl - part;
            if (excl <= thr_local && thr_local < incl) {
                uint64_t acc = excl;
                for (int64_t i = s0; i < s1; ++i) {
                    acc += weight(s_d2[i], scale, any);
                    if (acc > thr_local) { a.sel[m] = i0 + i; break; }
                }
            }
        }
        if (!block_group_barrier(bar, a.bps, a.err)) return;
        pick = (s_pick >= 0) ? s_pick : *(volatile long long *)(a.sel + m);
        for (int j = tid; j < ds; j += kThreads) {
            float v = Pm[pick * a.ld + j];
            s_center[j] = v;
            if (b == 0) Cm[(size_t)t * ds + j] = v;
        }
        __syncthreads();
        for (int64_t i = tid; i < cnt; i += kThreads) {
            float d = d2_f32_exact(Pm + (i0 + i) * a.ld, s_center, ds);
            if (d < s_d2[i]) s_d2[i] = d;
        }
        // The update is strided over threads, the next round's sums walk contiguous segments.
        __syncthreads();
        // s_pick is rewritten by thread 0 only after the next barrier, which every thread passes first.
    }
}

__global__ void gather_subsample_kernel(const float *X, int64_t N, int D, int64_t n_s, uint64_t seed, float *P)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t l = warp; l < n_s; l += nw) {
        const int64_t row = scale_index(rng_draw(seed, kStreamSubsample, (uint64_t)l) >> 11, (uint64_t)N);
        const float *src = X + row * D;
        float *dst = P + l * D;
        for (int j = lane; j < D; j += 32) dst[j] = src[j];
    }
}

}  // namespace

int launch_gather_subsample(const float *X, int64_t N, int D, int64_t n_s, uint64_t seed, float *P, cudaStream_t s)
{
    int blocks = (int)std::min<int64_t>((n_s + 7) / 8, 152 * 16);
    ProfScope ps("gather_subsample", s);
    gather_subsample_kernel<<<blocks, 256, 0, s>>>(X, N, D, n_s, seed, P);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

int launch_kmeanspp(const float *P, int64_t ld, int64_t n, int ds, int M, int Ks, uint64_t seed, float *C,
                    Scratch &ws, int *err, cudaStream_t s)
{
    if (ds > 256) return fail(PQ_ENOTSUP, "k-means++ seeding supports subspace width <= 256 (got %d)", ds);
    int dev = 0, sms = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    PQ_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int smem_cap = 0;
    PQ_TRY_CUDA(cudaDeviceGetAttribute(&smem_cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    PQ_TRY_CUDA(cudaFuncGetAttributes(&fa, kmeanspp_kernel));
    smem_cap -= (int)fa.sharedSizeBytes;  // the opt-in limit covers static + dynamic shared memory

    // Blocks per subspace: enough that each block's D2 slice fits shared
    // memory, at most one point in 64 per block, and the whole grid co-resident.
    PQ_TRY_CUDA(cudaFuncSetAttribute(kmeanspp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_cap));
    const int64_t bps_min = std::max<int64_t>(1, ((int64_t)n * 4 + smem_cap - 1) / smem_cap);
    int64_t want = std::max<int64_t>(bps_min, std::min<int64_t>((n + 63) / 64, 4096));
    int64_t nb = 0;
    size_t smem = 0;
    bool ok = false;
    for (int iter = 0; iter < 16 && want >= bps_min; ++iter) {
        nb = (n + want - 1) / want;
        smem = (size_t)nb * sizeof(float);
        int per_sm = 0;
        PQ_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kmeanspp_kernel, kThreads, smem));
        const int64_t capacity = (int64_t)per_sm * sms;
        if (want * M <= capacity) { ok = true; break; }
        want = std::min<int64_t>(want - 1, capacity / M);
    }
    if (!ok)
        return fail(PQ_ENOTSUP, "k-means++ seeding: %lld points x %d subspaces do not fit one cooperative wave",
                    (long long)n, M);
    const int bps = (int)want;

    KppArgs a;
    a.P = P;
    a.ld = ld;
    a.n = n;
    a.ds = ds;
    a.M = M;
    a.Ks = Ks;
    a.seed = seed;
    a.C = C;
    a.bars = ws.get<unsigned>(2 * (size_t)M, true);
    a.bsum = ws.get<unsigned long long>((size_t)M * bps, true);
    a.dmax_bits = ws.get<unsigned>((size_t)M, true);
    a.sel = ws.get<long long>((size_t)M, true);
    if (ws.status) return ws.status;
    a.err = err;
    a.bps = bps;
    a.nb = nb;
    void *args[] = {&a};
    dim3 grid(bps, M);
    ProfScope ps("kmeanspp", s);
    PQ_TRY_CUDA(cudaLaunchCooperativeKernel((void *)kmeanspp_kernel, grid, dim3(kThreads), args, smem, s));
    count_launch();
    return PQ_OK;
}

}  // namespace pqgb
