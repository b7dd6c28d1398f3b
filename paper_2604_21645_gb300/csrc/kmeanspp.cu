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
// One cooperative launch seeds all M subspaces.  Block b of subspace m owns
// points [b*nb, (b+1)*nb).  Per round it folds the newest seed into its D2
// values, publishes the sum of its weights and meets the other blocks of
// subspace m at one bounded barrier; then every block finds, by itself, the
// block whose weights hold the threshold and walks that block's D2 values to
// the picked point.  D2 and the block sums are double-buffered in global
// memory (round t reads buffer t&1 and writes buffer (t+1)&1), so a block
// running ahead never overwrites what a slower block still reads.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kPer = 5;              // block sums per lane in the owner search
constexpr int kMaxBps = 32 * kPer;   // blocks per group
constexpr int64_t kDynSmemCap = 200 * 1024;  // dynamic shared memory of a block
constexpr int kTagStride = 32;       // one 128-byte line per block's tag and sum: every block polls every tag

struct KppArgs {
    const float *X;               // rows, stride ld floats
    int64_t ld;
    const int64_t *sub_rows;      // subsample row indices (chunks with sub_off >= 0)
    int ds, M, Ks;
    int n_chunks;
    int64_t nmax;                 // largest point count of a group
    float *C;                     // [n_chunks][M][Ks][ds]
    unsigned *bars;               // [groups][2]
    unsigned *tags;               // [2][groups][bps] 128-byte lines: word 0 the round of the published
                                  // block weight sum, words 2-3 that sum
    float *d2;                    // [2][groups][nmax]
    unsigned *dmax_bits;          // [groups]
    int *err;
    unsigned spin;                // poll budget of the inter-block waits
    int bps;
    int ncache;                   // points per block kept in shared memory
    int nb_pad;                   // floats of the per-block D2 copy (multiple of 4)
    float *gpts;                  // [groups][bps][ustride][ds] the other points, gathered contiguously
    int ustride;                  // points per block in gpts
    SeedChunk ch[kMaxSeedChunks];
};

// FP32 squared distance in dimension order (each difference, square and sum rounded
// separately) -- the order the CPU reference uses.  `c` is in shared memory.
__device__ __forceinline__ float d2_f32_exact(const float *x, const float *c, int ds)
{
    float acc = 0.0f;
    int j = 0;
    if ((ds & 3) == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        // loads are issued 32 floats ahead; the sum itself stays in dimension order
        for (; j + 32 <= ds; j += 32) {
            float4 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = __ldg(reinterpret_cast<const float4 *>(x + j) + q);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 cc = *reinterpret_cast<const float4 *>(c + j + 4 * q);
                const float e[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
                const float f[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float t = __fsub_rn(e[r], f[r]);
                    acc = __fadd_rn(acc, __fmul_rn(t, t));
                }
            }
        }
        for (; j < ds; j += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(x + j));
            const float4 cc = *reinterpret_cast<const float4 *>(c + j);
            const float e[4] = {v.x, v.y, v.z, v.w};
            const float f[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float t = __fsub_rn(e[r], f[r]);
                acc = __fadd_rn(acc, __fmul_rn(t, t));
            }
        }
        return acc;
    }
    for (; j < ds; ++j) {
        const float t = __fsub_rn(x[j], c[j]);
        acc = __fadd_rn(acc, __fmul_rn(t, t));
    }
    return acc;
}

// w = floor(d2 * 2^sh) for d2 >= 0, exactly, in integer arithmetic:
// d2 = m * 2^(e - 150) for a normal float, m * 2^-149 for a subnormal one.
__device__ __forceinline__ uint64_t weight(float d2, int sh, bool any)
{
    const unsigned u = __float_as_uint(d2);
    if (!any || u == 0u) return 0ull;
    const unsigned be = u >> 23;  // sign bit clear
    const uint64_t m = be ? ((u & 0x7fffffu) | 0x800000u) : (u & 0x7fffffu);
    const int sft = (be ? (int)be - 150 : -149) + sh;
    if (sft >= 0) return m << sft;  // below 2^62: d2 <= max D2 < 2^E and sh = 62 - L - E
    return sft > -64 ? (m >> (-sft)) : 0ull;
}

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide inclusive scan of one uint64 per thread.
__device__ __forceinline__ uint64_t block_scan_u64(uint64_t v, uint64_t *sh_warp)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_incl_scan(v);
    if (lane == 31) sh_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint64_t w = lane < kWarps ? sh_warp[lane] : 0ull;
        w = warp_incl_scan(w);
        if (lane < kWarps) sh_warp[lane] = w;
    }
    __syncthreads();
    const uint64_t add = wid > 0 ? sh_warp[wid - 1] : 0ull;
    __syncthreads();
    return v + add;
}

// Squared distance of the shared-memory copy of point i (float4 q of point i at
// pts4[q * ncache + i]) to the seed c, dimension order.
__device__ __forceinline__ float d2_f32_smem(const float4 *pts4, int ncache, int i, const float *c, int ds)
{
    float acc = 0.0f;
    for (int q = 0; q < ds / 4; ++q) {
        const float4 v = pts4[q * ncache + i];
        const float4 cc = *reinterpret_cast<const float4 *>(c + 4 * q);
        const float e[4] = {v.x, v.y, v.z, v.w};
        const float f[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float t = __fsub_rn(e[r], f[r]);
            acc = __fadd_rn(acc, __fmul_rn(t, t));
        }
    }
    return acc;
}

// The same distances for points whose float4 piece q is f(q) (for the gathered copy, pieces of one
// point are ustride float4s apart, so a warp's loads of one piece are contiguous).  Pieces are
// fetched eight at a time before the sums, which keep the dimension order.
template <typename F>
__device__ __forceinline__ float d2_f32_pieces(F f, const float *c, int ds)
{
    float acc = 0.0f;
    int q0 = 0;
    auto add4 = [&](const float4 v, int q) {
        const float4 cc = *reinterpret_cast<const float4 *>(c + 4 * q);
        const float e[4] = {v.x, v.y, v.z, v.w};
        const float g[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float t = __fsub_rn(e[r], g[r]);
            acc = __fadd_rn(acc, __fmul_rn(t, t));
        }
    };
    for (; q0 + 8 <= ds / 4; q0 += 8) {
        float4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = f(q0 + q);
#pragma unroll
        for (int q = 0; q < 8; ++q) add4(v[q], q0 + q);
    }
    for (; q0 < ds / 4; ++q0) add4(f(q0), q0);
    return acc;
}

template <typename F0, typename F1>
__device__ __forceinline__ void d2_f32_pieces2(F0 f0, F1 f1, const float *c, int ds, float &d0, float &d1)
{
    float a0 = 0.0f, a1 = 0.0f;
    auto add4 = [&](const float4 v0, const float4 v1, int q) {
        const float4 cc = *reinterpret_cast<const float4 *>(c + 4 * q);
        const float g[4] = {cc.x, cc.y, cc.z, cc.w};
        const float e0[4] = {v0.x, v0.y, v0.z, v0.w};
        const float e1[4] = {v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float t0 = __fsub_rn(e0[r], g[r]);
            const float t1 = __fsub_rn(e1[r], g[r]);
            a0 = __fadd_rn(a0, __fmul_rn(t0, t0));
            a1 = __fadd_rn(a1, __fmul_rn(t1, t1));
        }
    };
    int q0 = 0;
    for (; q0 + 8 <= ds / 4; q0 += 8) {
        float4 v0[8], v1[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v0[q] = f0(q0 + q);
            v1[q] = f1(q0 + q);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) add4(v0[q], v1[q], q0 + q);
    }
    for (; q0 < ds / 4; ++q0) add4(f0(q0), f1(q0), q0);
    d0 = a0;
    d1 = a1;
}

constexpr int kWalkRegs = 8;  // D2 values per thread kept in registers by the walk


__global__ void __launch_bounds__(kThreads, 1) kmeanspp_kernel(KppArgs a)
{
    __shared__ __align__(16) float s_center[256];  // ds <= 256
    __shared__ uint64_t s_warp[kWarps];
    __shared__ float s_fmax[kWarps];
    __shared__ long long s_pick;
    __shared__ int s_owner;
    __shared__ unsigned long long s_thr;
    __shared__ int s_fail;
    // dynamic: this block's D2 values [nb_pad], then the first ncache of its points [ds/4][ncache]
    extern __shared__ float4 s_dyn[];

    // group = (chunk, subspace); its points are the chunk's rows or its subsample
    const int grp = blockIdx.y, b = blockIdx.x, tid = threadIdx.x;
    const int chunk = grp / a.M, m = grp % a.M;
    const SeedChunk ck = a.ch[chunk];
    const int64_t n = ck.n;
    const uint64_t seed = ck.seed;
    const int ds = a.ds;
    const int64_t nb = (n + a.bps - 1) / a.bps;
    const int64_t i0 = (int64_t)b * nb;
    const int cnt = (int)max((int64_t)0, min(n, i0 + nb) - i0);
    const float *Pm = a.X + (int64_t)m * ds;
    const int64_t *sub = ck.sub_off >= 0 ? a.sub_rows + ck.sub_off : nullptr;
    auto point = [&](int64_t i) -> const float * { return Pm + (ck.r0 + (sub ? sub[i] : i)) * a.ld; };
    const bool vec_ok = (ds & 3) == 0 && (a.ld & 3) == 0 && (reinterpret_cast<uintptr_t>(Pm) & 15) == 0;
    const int ncache = vec_ok ? min(cnt, a.ncache) : 0;
    // a block alone in its group walks only its own shared-memory D2 copy: no global copy
    const bool solo = a.bps == 1;
    float *s_d2 = reinterpret_cast<float *>(s_dyn);
    // points past the shared-memory cache, gathered into a contiguous copy at round 0
    float *gp0 = (a.gpts && vec_ok) ? a.gpts + ((size_t)grp * a.bps + b) * a.ustride * ds : nullptr;
    // piece q (a float4) of point i past the cache: in the gathered copy, piece-major ([ds/4][ustride]),
    // so that consecutive threads read consecutive addresses.  The copy is written by this kernel
    // (round 0), so it is read through L2 (ld.global.cg), not the read-only cache path.
    float4 *gp4 = reinterpret_cast<float4 *>(gp0);
    // Which thread folds which point.  Several blocks per group: thread t takes points t, t + kThreads, ...;
    // the first ncache points are cached (slot i), the rest are in the gathered copy (slot i - ncache).
    // A block alone in its group (with a gathered copy): warp w takes the consecutive range [wlo, whi) and
    // lane l the consecutive piece [wlo + l*piece, wlo + (l+1)*piece) of it, so that the lane and warp sums
    // are sums of consecutive points and the walk goes straight to one piece.  The first cpl points of
    // every piece are cached, so that every lane has the same share of shared-memory and gathered points;
    // cache and gathered copy store point k of lane l's piece at slot 32k + l of the warp's part, so that a
    // warp's loads are consecutive.
    const bool wr = solo && gp0 != nullptr;
    const int wid = tid >> 5, lane = tid & 31;
    const int wlen = (int)(((int64_t)cnt + 32 * kWarps - 1) / (32 * kWarps)) * 32;
    const int piece = wlen / 32;
    const int wlo = wr ? min(cnt, wid * wlen) : 0;
    const int whi = wr ? min(cnt, wlo + wlen) : cnt;
    const int cpw = wr ? min(wlen, (a.ncache / kWarps) & ~31) : 0;
    const int cpl = cpw / 32;
    const int pfirst = wr ? min(whi, wlo + lane * piece) : tid;   // a thread's first point
    const int pstep = wr ? 1 : kThreads;                          // and the stride of its points
    const int pend = wr ? min(whi, pfirst + piece) : cnt;         // up to
    const int pcache = wr ? min(pend, pfirst + cpl) : ncache;     // its points below pcache are cached
    const int smul = wr ? 32 : 1;                                 // slot of point i: (i - pfirst) * smul + base
    const int cbase = wr ? wid * cpw + lane : pfirst;
    const int gbase = wr ? wid * (wlen - cpw) + lane - 32 * cpl : pfirst - ncache;
    // cache rows: the transposed slots of a range can pass its point count, so the warp-range layout uses
    // the allocation's row length (slots < kWarps * cpw <= a.ncache)
    const int cstride = wr ? a.ncache : ncache;
    auto cslot = [&](int i) { return (i - pfirst) * smul + cbase; };
    auto gslot = [&](int i) { return (i - pfirst) * smul + gbase; };
    auto upiece = [&](int i, int q) -> float4 {
        return gp0 ? __ldcg(gp4 + (size_t)q * a.ustride + gslot(i))
                   : __ldg(reinterpret_cast<const float4 *>(point(i0 + i)) + q);
    };
    const float4 *pts4 = s_dyn + a.nb_pad / 4;
    float4 *pts4w = s_dyn + a.nb_pad / 4;
    unsigned *bar = a.bars + 2 * grp;
    float *Cm = a.C + ((size_t)chunk * a.M + m) * a.Ks * ds;
    const int groups = a.n_chunks * a.M;
    const size_t plane = (size_t)groups * a.nmax;  // one D2 buffer
    float *d2m = a.d2 + (size_t)grp * a.nmax;      // + buffer * plane
    unsigned *tags = a.tags + (size_t)grp * a.bps * kTagStride;
    const size_t bplane = (size_t)groups * a.bps;

    // ---- round 0: first seed; D2 of every point; the cached points are copied --------
    long long pick = scale_index(rng_draw(seed, (uint64_t)m, 0) >> 11, (uint64_t)n);
    for (int j = tid; j < ds; j += kThreads) {
        const float v = point(pick)[j];
        s_center[j] = v;
        if (b == 0) Cm[j] = v;
    }
    __syncthreads();
    float lmax = 0.0f;
    for (int i = pfirst; i < pend; i += pstep) {
        float d;
        if (i < pcache) {
            const float *x = point(i0 + i);
            float acc = 0.0f;
            for (int q = 0; q < ds / 4; ++q) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(x) + q);
                pts4w[q * cstride + cslot(i)] = v;
                const float4 cc = *reinterpret_cast<const float4 *>(s_center + 4 * q);
                const float e[4] = {v.x, v.y, v.z, v.w};
                const float f[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float t = __fsub_rn(e[r], f[r]);
                    acc = __fadd_rn(acc, __fmul_rn(t, t));
                }
            }
            d = acc;
        } else if (gp0) {
            const float *x = point(i0 + i);
            float4 *dst = gp4 + gslot(i);
            float acc = 0.0f;
            for (int q = 0; q < ds / 4; ++q) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(x) + q);
                dst[(size_t)q * a.ustride] = v;
                const float4 cc = *reinterpret_cast<const float4 *>(s_center + 4 * q);
                const float e[4] = {v.x, v.y, v.z, v.w};
                const float f[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float t = __fsub_rn(e[r], f[r]);
                    acc = __fadd_rn(acc, __fmul_rn(t, t));
                }
            }
            d = acc;
        } else {
            d = d2_f32_exact(point(i0 + i), s_center, ds);
        }
        s_d2[i] = d;
        if (!solo) d2m[plane + i0 + i] = d;  // buffer 1 holds D2 for round 1
        lmax = fmaxf(lmax, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((tid & 31) == 0) s_fmax[tid >> 5] = lmax;
    __syncthreads();
    if (tid == 0) {
        float v = 0.0f;
        for (int w = 0; w < kWarps; ++w) v = fmaxf(v, s_fmax[w]);
        atomicMax(a.dmax_bits + grp, __float_as_uint(v));  // non-negative floats order as integers
    }
    if (!block_group_barrier(bar, a.bps, a.err, a.spin)) return;
    const float dmax = __uint_as_float(ld_acquire_u32(a.dmax_bits + grp));
    const bool any = dmax > 0.0f;
    int L = 0;
    while (((int64_t)1 << L) < n) ++L;
    int E = 0;
    if (any) {
        const unsigned bits = __float_as_uint(dmax);
        const int be = (bits >> 23) & 0xff;
        if (be != 0) E = be - 126;                       // dmax in [2^(E-1), 2^E)
        else E = -117 - __clz(bits & 0x7fffff);           // subnormal maximum
    }
    const int sh = 62 - L - E;

    for (int t = 1; t < a.Ks; ++t) {
        const int cur = t & 1;
        float *D2c = d2m + (size_t)cur * plane;
        // fold seed t-1 into this block's D2 (round 1 uses round 0's values) and sum the weights;
        // the block's own D2 values live in shared memory, the global copy serves the walk
        uint64_t part = 0;
        if (t == 1) {
            for (int i = pfirst; i < pend; i += pstep) part += weight(s_d2[i], sh, any);
        } else {
            int i = pfirst;
            for (; i < pcache; i += pstep) {
                const float d = fminf(d2_f32_smem(pts4, cstride, cslot(i), s_center, ds), s_d2[i]);
                s_d2[i] = d;
                if (!solo) D2c[i0 + i] = d;
                part += weight(d, sh, any);
            }
            if (vec_ok && ds == 8) {
                // eight uncached points per thread, all their loads in flight before the sums
                for (; i + 7 * pstep < pend; i += 8 * pstep) {
                    float4 u[8][2];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        u[q][0] = upiece(i + q * pstep, 0);
                        u[q][1] = upiece(i + q * pstep, 1);
                    }
                    const float4 c0 = *reinterpret_cast<const float4 *>(s_center);
                    const float4 c1 = *reinterpret_cast<const float4 *>(s_center + 4);
                    const float f[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float e[8] = {u[q][0].x, u[q][0].y, u[q][0].z, u[q][0].w,
                                            u[q][1].x, u[q][1].y, u[q][1].z, u[q][1].w};
                        float acc = 0.0f;
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            const float t = __fsub_rn(e[r], f[r]);
                            acc = __fadd_rn(acc, __fmul_rn(t, t));
                        }
                        const int ii = i + q * pstep;
                        const float d = fminf(acc, s_d2[ii]);
                        s_d2[ii] = d;
                        if (!solo) D2c[i0 + ii] = d;
                        part += weight(d, sh, any);
                    }
                }
            }
            if (vec_ok) {
                for (; i + pstep < pend; i += 2 * pstep) {
                    float d0, d1;
                    const int ia = i, ib = i + pstep;
                    d2_f32_pieces2([&](int q) { return upiece(ia, q); }, [&](int q) { return upiece(ib, q); }, s_center, ds,
                                   d0, d1);
                    d0 = fminf(d0, s_d2[i]);
                    d1 = fminf(d1, s_d2[i + pstep]);
                    s_d2[i] = d0;
                    s_d2[i + pstep] = d1;
                    if (!solo) {
                        D2c[i0 + i] = d0;
                        D2c[i0 + i + pstep] = d1;
                    }
                    part += weight(d0, sh, any) + weight(d1, sh, any);
                }
            }
            for (; i < pend; i += pstep) {
                const int ia = i;
                const float d = fminf(vec_ok ? d2_f32_pieces([&](int q) { return upiece(ia, q); }, s_center, ds)
                                             : d2_f32_exact(point(i0 + i), s_center, ds),
                                      s_d2[i]);
                s_d2[i] = d;
                if (!solo) D2c[i0 + i] = d;
                part += weight(d, sh, any);
            }
        }
        const uint64_t lane_part = part;  // the sum of this lane's piece (warp-range layout)
        part = warp_sum(part);
        if ((tid & 31) == 0) s_warp[tid >> 5] = part;
        __syncthreads();
        const uint64_t r = rng_draw(seed, (uint64_t)m, (uint64_t)t) >> 11;
        if (solo) {
            // a block alone in its group owns the whole threshold: no publication and no poll.  Warp 0 scans
            // the warp sums; in the warp-range layout the first warp whose inclusive sum passes the
            // threshold holds it
            if (tid < 32) {
                const uint64_t v = tid < kWarps ? s_warp[tid] : 0ull;
                const uint64_t incl = warp_incl_scan(v);
                const uint64_t W = __shfl_sync(0xffffffffu, incl, 31);
                if (W == 0) {
                    if (tid == 0) s_pick = scale_index(r, (uint64_t)n);
                } else {
                    const uint64_t thr = (__umul64hi(r, W) << 11) | ((r * W) >> 53);
                    const int ow = __ffs(__ballot_sync(0xffffffffu, tid < kWarps && incl > thr)) - 1;
                    if (tid == 0) {
                        s_pick = -1;
                        s_owner = wr ? ow : b;
                    }
                    if (tid == ow) s_thr = wr ? thr - (incl - v) : thr;
                }
                if (tid == 0) s_fail = 0;
            }
        } else {
            if (tid == 0) {
                uint64_t tot = 0;
                for (int w = 0; w < kWarps; ++w) tot += s_warp[w];
                unsigned *line = tags + ((size_t)cur * bplane + b) * kTagStride;
                *reinterpret_cast<unsigned long long *>(line + 2) = tot;
                // publishes the sum and (ordered before it by the __syncthreads above) the block's D2 copy
                st_release_u32(line, (unsigned)t);
            }

            // every block: wait for all round-t sums of its group, then find the owner block and
            // threshold.  Lane l polls and holds the sums of blocks [l*kPer, (l+1)*kPer).
            if (tid < 32) {
                const unsigned *tg = tags + (size_t)cur * bplane * kTagStride;
                bool ok = true;
                for (unsigned it = 0;; ++it) {
                    bool mine = true;
#pragma unroll
                    for (int q = 0; q < kPer; ++q) {
                        const int bi = tid * kPer + q;
                        if (bi < a.bps) mine &= ld_acquire_u32(tg + (size_t)bi * kTagStride) == (unsigned)t;
                    }
                    if (__all_sync(0xffffffffu, mine)) break;
                    // warp-uniform decision to give up (bounded wait)
                    const bool give_up = it >= a.spin || ((it & 255) == 255 && *(volatile int *)a.err != 0);
                    if (__any_sync(0xffffffffu, give_up)) {
                        if (tid == 0) atomicCAS(a.err, 0, PQ_ETIMEOUT);
                        ok = false;
                        break;
                    }
                }
                if (tid == 0) s_fail = !ok;
                // each block's sum sits in its tag's line, read after the acquire that saw the tag
                uint64_t v[kPer];
                uint64_t tot = 0;
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    const int bi = tid * kPer + q;
                    v[q] = bi < a.bps ? *reinterpret_cast<const volatile unsigned long long *>(tg + (size_t)bi * kTagStride + 2)
                                      : 0ull;
                    tot += v[q];
                }
                const uint64_t incl = warp_incl_scan(tot);
                const uint64_t W = __shfl_sync(0xffffffffu, incl, 31);
                long long p = -1;
                if (W == 0) {
                    p = scale_index(r, (uint64_t)n);
                } else {
                    const uint64_t thr = (__umul64hi(r, W) << 11) | ((r * W) >> 53);
                    const unsigned hit = __ballot_sync(0xffffffffu, incl > thr);
                    const int l = __ffs(hit) - 1;
                    if (tid == l) {
                        uint64_t acc = incl - tot;
                        int owner = -1;
                        uint64_t thr_local = 0;
#pragma unroll
                        for (int q = 0; q < kPer; ++q) {
                            if (owner < 0 && acc + v[q] > thr) {
                                owner = tid * kPer + q;
                                thr_local = thr - acc;
                            }
                            acc += v[q];
                        }
                        s_owner = owner;
                        s_thr = thr_local;
                    }
                }
                if (tid == 0) s_pick = p;
            }
        }
        __syncthreads();
        if (s_fail) return;
        if (wr && s_pick < 0) {
            // only the warp whose range holds the threshold walks: each lane sums a consecutive piece
            // of the range, one scan of the piece sums finds the lane, which walks its piece
            if (wid == s_owner) {
                const uint64_t thr_w = s_thr;
                const uint64_t incl = warp_incl_scan(lane_part);
                const uint64_t excl = incl - lane_part;
                const int hl = __ffs(__ballot_sync(0xffffffffu, excl <= thr_w && thr_w < incl)) - 1;
                // that lane's piece, 32 values at a time: one weight per lane, a scan, the first lane past
                // the threshold
                uint64_t acc = __shfl_sync(0xffffffffu, excl, hl);
                const int p0 = min(whi, wlo + hl * piece), p1 = min(whi, p0 + piece);
                for (int base = p0; base < p1; base += 32) {
                    const int j = base + lane;
                    const uint64_t inc = warp_incl_scan(j < p1 ? weight(s_d2[j], sh, any) : 0ull) + acc;
                    const unsigned past = __ballot_sync(0xffffffffu, j < p1 && inc > thr_w);
                    if (past) {
                        if (lane == __ffs(past) - 1) s_pick = i0 + j;
                        break;
                    }
                    acc = __shfl_sync(0xffffffffu, inc, 31);
                }
            }
            __syncthreads();
        } else if (s_pick < 0) {
            // walk the owner's D2 values in order to the threshold (the owner reads its own copy)
            const int owner = s_owner;
            const uint64_t thr_local = s_thr;
            const int64_t o0 = (int64_t)owner * nb;
            const int ocnt = (int)(min(n, o0 + nb) - o0);
            const int seg = (ocnt + kThreads - 1) / kThreads;
            const int s0 = min(ocnt, tid * seg), s1 = min(ocnt, s0 + seg);
            const float *src = owner == b ? s_d2 : nullptr;
            uint64_t w = 0;
            if (seg <= kWalkRegs) {
                float dv[kWalkRegs];
#pragma unroll
                for (int q = 0; q < kWalkRegs; ++q) {
                    const int i = s0 + q;
                    dv[q] = i < s1 ? (src ? src[i] : __ldcg(D2c + o0 + i)) : 0.0f;
                }
#pragma unroll
                for (int q = 0; q < kWalkRegs; ++q) w += s0 + q < s1 ? weight(dv[q], sh, any) : 0ull;
                const uint64_t incl = block_scan_u64(w, s_warp);
                const uint64_t excl = incl - w;
                if (excl <= thr_local && thr_local < incl) {
                    uint64_t acc = excl;
                    long long hit = -1;
#pragma unroll
                    for (int q = 0; q < kWalkRegs; ++q) {
                        if (hit < 0 && s0 + q < s1) {
                            acc += weight(dv[q], sh, any);
                            if (acc > thr_local) hit = o0 + s0 + q;
                        }
                    }
                    s_pick = hit;
                }
            } else {
                // eight values in flight at a time (the weights are integers: the order of the sum is free)
                auto d2at = [&](int i) { return src ? src[i] : __ldcg(D2c + o0 + i); };
                int i = s0;
                for (; i + 8 <= s1; i += 8) {
                    float dv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) dv[q] = d2at(i + q);
#pragma unroll
                    for (int q = 0; q < 8; ++q) w += weight(dv[q], sh, any);
                }
                for (; i < s1; ++i) w += weight(d2at(i), sh, any);
                const uint64_t incl = block_scan_u64(w, s_warp);
                const uint64_t excl = incl - w;
                if (excl <= thr_local && thr_local < incl) {
                    // the block of eight that crosses the threshold, then its values one at a time
                    uint64_t acc = excl;
                    int j = s0;
                    for (; j + 8 <= s1; j += 8) {
                        float dv[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) dv[q] = d2at(j + q);
                        uint64_t bs = 0;
#pragma unroll
                        for (int q = 0; q < 8; ++q) bs += weight(dv[q], sh, any);
                        if (acc + bs > thr_local) break;
                        acc += bs;
                    }
                    for (; j < s1; ++j) {
                        acc += weight(d2at(j), sh, any);
                        if (acc > thr_local) {
                            s_pick = o0 + j;
                            break;
                        }
                    }
                }
            }
            __syncthreads();
        }
        pick = s_pick;
        for (int j = tid; j < ds; j += kThreads) {
            const float v = point(pick)[j];
            s_center[j] = v;
            if (b == 0) Cm[(size_t)t * ds + j] = v;
        }
        __syncthreads();
    }
}

// Row indices of the with-replacement subsample of every chunk that needs one:
// index l of chunk c is floor(u * rows_c) with u draw l of the subsample stream of seed_c.
__global__ void subsample_rows_kernel(const KppArgs a, int64_t n_s, int64_t *sub_rows)
{
    const SeedChunk ck = a.ch[blockIdx.y];
    if (ck.sub_off < 0) return;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n_s; l += (int64_t)gridDim.x * blockDim.x)
        sub_rows[ck.sub_off + l] = scale_index(rng_draw(ck.seed, kStreamSubsample, (uint64_t)l) >> 11, (uint64_t)ck.rows);
}

// Row l of G = row floor(u_l * N) of X, u_l the draw l of the subsample stream: the rows the
// seeding of one chunk reads (the same draws as subsample_rows_kernel), one warp per row.
__global__ void gather_subsample_kernel(const float *__restrict__ X, int64_t N, int D, uint64_t seed, int64_t n_s,
                                        float *__restrict__ G)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; l < n_s; l += nw) {
        const int64_t row = scale_index(rng_draw(seed, kStreamSubsample, (uint64_t)l) >> 11, (uint64_t)N);
        const float *src = X + row * D;
        float *dst = G + l * D;
        if ((D & 3) == 0) {
            for (int j = lane; j < D / 4; j += 32)
                reinterpret_cast<float4 *>(dst)[j] = reinterpret_cast<const float4 *>(src)[j];
        } else {
            for (int j = lane; j < D; j += 32) dst[j] = src[j];
        }
    }
}

}  // namespace

int launch_gather_subsample(const float *X, int64_t N, int D, int Ks, uint64_t seed, float *G, cudaStream_t s)
{
    const int64_t n_s = 100LL * Ks;
    ProfScope ps("gather_subsample", s);
    gather_subsample_kernel<<<152 * 4, 256, 0, s>>>(X, N, D, seed, n_s, G);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

int launch_kmeanspp_chunks(const float *X, int64_t ld, const SeedChunk *chunks, int n_chunks, int ds, int M, int Ks,
                           float *C, Scratch &ws, int *err, cudaStream_t s, const char *tag)
{
    if (ds > 256) return fail(PQ_ENOTSUP, "k-means++ seeding supports subspace width <= 256 (got %d)", ds);
    if (n_chunks < 1 || n_chunks > kMaxSeedChunks) return fail(PQ_ENOTSUP, "at most %d chunks", kMaxSeedChunks);
    int dev = 0, sms = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    PQ_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t cap = 100LL * Ks;
    KppArgs a;
    a.X = X;
    a.ld = ld;
    a.ds = ds;
    a.M = M;
    a.Ks = Ks;
    a.n_chunks = n_chunks;
    a.nmax = 0;
    int64_t n_sub = 0;
    for (int c = 0; c < n_chunks; ++c) {
        a.ch[c] = chunks[c];
        if (chunks[c].rows > cap) {
            a.ch[c].n = cap;
            a.ch[c].sub_off = n_sub * cap;
            ++n_sub;
        } else {
            a.ch[c].n = chunks[c].rows;
            a.ch[c].sub_off = -1;
        }
        if (a.ch[c].n < Ks) return fail(PQ_EINVAL, "chunk %d has %lld rows, fewer than Ks=%d", c, (long long)a.ch[c].n, Ks);
        a.nmax = std::max(a.nmax, a.ch[c].n);
    }
    const int groups = n_chunks * M;
    // One chunk: about one block per SM over its subspaces, cooperative (blocks of a subspace
    // meet at barriers).  Several chunks: one block per (chunk, subspace), no inter-block waits.
    int bps = 1;
    bool coop = false;
    if (n_chunks == 1)
        bps = (int)std::max<int64_t>(
            1, std::min<int64_t>(std::min(sms / std::max(1, M), kMaxBps), (a.nmax + 255) / 256));
    // shared memory: the block's D2 copy, then as many of its points as fit
    const int64_t nb = (a.nmax + bps - 1) / bps;
    a.nb_pad = (int)((nb + 3) & ~int64_t(3));
    if ((int64_t)a.nb_pad * 4 > kDynSmemCap)
        return fail(PQ_ENOTSUP, "k-means++ seeding: %lld points per block exceed shared memory", (long long)nb);
    a.ncache = (ds % 4 == 0) ? (int)std::min<int64_t>(nb, (kDynSmemCap - (int64_t)a.nb_pad * 4) / (ds * 4)) : 0;
    a.ustride = (ds % 4 == 0) ? (int)(a.nb_pad - a.ncache) : 0;
    if (bps == 1 && a.ustride > 0) {
        // a block alone in its group caches the first cpw points of each warp's range (see the kernel):
        // the gathered copy then holds up to kWarps * (wlen - cpw) points
        const int64_t wlen = (nb + 32 * kWarps - 1) / (32 * kWarps) * 32;
        const int64_t cpw = std::min<int64_t>(wlen, (a.ncache / kWarps) & ~31);
        a.ustride = (int)std::max<int64_t>(a.ustride, kWarps * (wlen - cpw));
    }
    a.gpts = nullptr;
    const size_t dyn = (size_t)a.nb_pad * 4 + (size_t)a.ncache * ds * 4;
    PQ_TRY_CUDA(cudaFuncSetAttribute(kmeanspp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    if (n_chunks == 1) {
        int per_sm = 0;
        PQ_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kmeanspp_kernel, kThreads, dyn));
        if ((int64_t)bps * M > (int64_t)per_sm * sms)
            return fail(PQ_ENOTSUP, "k-means++ seeding: %d subspaces do not fit one cooperative wave", M);
        coop = true;
    }
    a.bps = bps;
    a.sub_rows = n_sub ? ws.get<int64_t>((size_t)n_sub * cap) : nullptr;
    a.C = C;
    a.bars = ws.get<unsigned>(2 * (size_t)groups, true);
    a.tags = ws.get<unsigned>(2 * (size_t)groups * bps * kTagStride, true);
    if (a.ustride > 0) a.gpts = ws.get<float>((size_t)groups * bps * a.ustride * ds);
    a.d2 = ws.get<float>(2 * (size_t)groups * a.nmax);
    a.dmax_bits = ws.get<unsigned>((size_t)groups, true);
    if (ws.status) return ws.status;
    a.err = err;
    a.spin = seeding_spin_limit();
    if (n_sub) {
        ProfScope ps("subsample_rows", s);
        subsample_rows_kernel<<<dim3((unsigned)((cap + 255) / 256), n_chunks), 256, 0, s>>>(a, cap,
                                                                                       const_cast<int64_t *>(a.sub_rows));
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
    }
    dim3 grid(bps, groups);
    ProfScope ps(tag, s);
    if (coop) {
        void *args[] = {&a};
        PQ_TRY_CUDA(cudaLaunchCooperativeKernel((void *)kmeanspp_kernel, grid, dim3(kThreads), args, dyn, s));
    } else {
        kmeanspp_kernel<<<grid, kThreads, dyn, s>>>(a);
        PQ_TRY_CUDA(cudaGetLastError());
    }
    count_launch();
    return PQ_OK;
}

int launch_kmeanspp(const float *X, int64_t N, int D, int M, int Ks, uint64_t seed, float *C, Scratch &ws, int *err,
                    cudaStream_t s, const char *tag)
{
    SeedChunk c;
    c.r0 = 0;
    c.rows = N;
    c.seed = seed;
    return launch_kmeanspp_chunks(X, D, &c, 1, D / M, M, Ks, C, ws, err, s, tag);
}

}  // namespace pqgb
