// coarse.cu -- coarse quantizer of the inverted index (Sec. 2.2; Rii is an
// IVFPQ-style index, Sec. 3.1): k-means on the raw D-dimensional rows,
// nearest-list assignment, and list-contiguous (CSR) bucketing of row ids and
// PQ codes.
//
// Assignment uses the same certified-argmin rule as the PQ pass: FP32 scores
// s_l = ||c_l||^2/2 - x.c_l from a tiled FFMA kernel, the two best kept per
// row; a row whose top-two gap does not clear the FP32 error bound is queued
// and re-decided by a warp in FP64 (direct differences over the candidates
// within the bound), so the list of every row is exact.
//
// The centroid update sums each list's rows in FP64 in ascending row order,
// one thread per dimension, which is exactly the reference computation.
#include <algorithm>
#include <cfloat>
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

constexpr int BM = 64, BN = 64, BK = 32;
constexpr int kTileRows = 512;   // rows per bucketing tile

__global__ void coarse_norms_kernel(const float *C, int nlist, int D, float *half_norm, float *maxes)
{
    float lmax = 0.0f;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlist; l += gridDim.x * blockDim.x) {
        float n = 0.0f;
        for (int j = 0; j < D; ++j) n = fmaf(C[(size_t)l * D + j], C[(size_t)l * D + j], n);
        half_norm[l] = 0.5f * n;
        lmax = fmaxf(lmax, 0.5f * n);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned *>(maxes), __float_as_uint(lmax));
}

__global__ void coarse_bound_finish(float *maxes, int D)
{
    const float nmax = maxes[0] * (1.0f + 4.0f * gamma_f32(D + 1));
    maxes[0] = nmax;
    maxes[1] = sqrtf(2.0f * nmax) * (1.0f + 1e-6f);
}

__device__ __forceinline__ float score_delta(float xn, float nmax, float cmax, int D)
{
    const float t = xn + cmax;
    return 2.2f * gamma_f32(D + 1) * (nmax + xn * cmax) + 1e-13f * t * t;
}

__device__ __forceinline__ void top2_merge(float &m1, int &i1, float &m2, float o1, int oi, float o2)
{
    const bool take = (o1 < m1) || (o1 == m1 && oi < i1);
    const float rest = take ? fminf(m1, o2) : fminf(m2, o1);
    if (take) { m1 = o1; i1 = oi; }
    m2 = rest;
}

// Tiled scores of rows against centroids.  TOP2: fused certified argmin per
// row (list id or -1 + queue entry).  !TOP2: write every score S[row][l].
template <bool TOP2>
__global__ void __launch_bounds__(256) coarse_scores_kernel(const float *__restrict__ X, int64_t N, int D,
                                                            const float *__restrict__ C, int nlist,
                                                            const float *__restrict__ half_norm,
                                                            const float *__restrict__ maxes,
                                                            int32_t *__restrict__ list_of_row,
                                                            int64_t *__restrict__ queue,
                                                            unsigned long long *__restrict__ queue_len,
                                                            float *__restrict__ S)
{
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Bs[BK][BN + 4];
    __shared__ float s_xn[BM];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t r0 = (int64_t)blockIdx.x * BM;

    if (TOP2) {
        // row norms: 4 threads per row
        const int r = tid >> 2, part = tid & 3;
        float acc = 0.0f;
        if (r0 + r < N)
            for (int j = part; j < D; j += 4) {
                const float v = X[(r0 + r) * D + j];
                acc = fmaf(v, v, acc);
            }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (part == 0) s_xn[r] = sqrtf(acc) * (1.0f + 1e-6f);
    }

    float m1[4], m2[4];
    int i1[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { m1[i] = FLT_MAX; m2[i] = FLT_MAX; i1[i] = 0; }

    for (int c0 = 0; c0 < nlist; c0 += BN) {
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
        for (int k0 = 0; k0 < D; k0 += BK) {
            __syncthreads();
            // 64 x 32 floats of each operand, 8 per thread, stored transposed
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int e = tid + t * 256;
                const int r = e / BK, kk = e % BK;
                const int64_t gr = r0 + r;
                const int gk = k0 + kk;
                As[kk][r] = (gr < N && gk < D) ? X[gr * D + gk] : 0.0f;
                const int gc = c0 + r;
                Bs[kk][r] = (gc < nlist && gk < D) ? C[(size_t)gc * D + gk] : 0.0f;
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < BK; ++kk) {
                const float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
                const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
                const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int l = c0 + tx * 4 + j;
            const float cn = l < nlist ? half_norm[l] : 0.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float s = l < nlist ? cn - acc[i][j] : FLT_MAX;
                if (TOP2) {
                    const bool lt = s < m1[i];
                    m2[i] = lt ? m1[i] : fminf(m2[i], s);
                    i1[i] = lt ? l : i1[i];
                    m1[i] = fminf(m1[i], s);
                } else {
                    const int64_t gr = r0 + ty * 4 + i;
                    if (gr < N && l < nlist) S[gr * nlist + l] = s;
                }
            }
        }
    }
    if (TOP2) {
        // merge across the 16 threads sharing the rows (one half-warp)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
                const float o1 = __shfl_xor_sync(0xffffffffu, m1[i], o);
                const int oi = __shfl_xor_sync(0xffffffffu, i1[i], o);
                const float o2 = __shfl_xor_sync(0xffffffffu, m2[i], o);
                top2_merge(m1[i], i1[i], m2[i], o1, oi, o2);
            }
        }
        if (tx == 0) {
            const float nmax = maxes[0], cmax = maxes[1];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t gr = r0 + ty * 4 + i;
                if (gr >= N) continue;
                const float delta = score_delta(s_xn[ty * 4 + i], nmax, cmax, D);
                if (m2[i] - m1[i] > 2.0f * delta) {
                    list_of_row[gr] = i1[i];
                } else {
                    list_of_row[gr] = -1;
                    const unsigned long long slot = atomicAdd(queue_len, 1ull);
                    queue[slot] = gr;
                }
            }
        }
    }
}

// One warp per queued row: FP64 direct differences over the candidate window.
__global__ void coarse_recheck_kernel(const float *__restrict__ X, int D, const float *__restrict__ C, int nlist,
                                      const float *__restrict__ half_norm, const float *__restrict__ maxes,
                                      const int64_t *__restrict__ queue, const unsigned long long *queue_len,
                                      int32_t *__restrict__ list_of_row, int sub)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long total = *queue_len;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < (int64_t)total; w += nw) {
        const int64_t row = queue[w];
        const float *x = X + row * D;
        float xx = 0.0f;
        for (int j = lane; j < D; j += 32) xx = fmaf(x[j], x[j], xx);
        xx = warp_sum(xx);
        const float xn = sqrtf(xx) * (1.0f + 1e-6f);
        float lmin = FLT_MAX;
        for (int l = lane; l < nlist; l += 32) {
            float acc = 0.0f;
            for (int j = 0; j < D; ++j) acc = fmaf(x[j], C[(size_t)l * D + j], acc);
            lmin = fminf(lmin, half_norm[l] - acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lmin = fminf(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
        const float win = 2.0f * score_delta(xn, maxes[0], maxes[1], D);
        double best = DBL_MAX;
        int bl = 0x7fffffff;
        for (int l = lane; l < nlist; l += 32) {
            float acc = 0.0f;
            for (int j = 0; j < D; ++j) acc = fmaf(x[j], C[(size_t)l * D + j], acc);
            if (half_norm[l] - acc <= lmin + win) {
                const double d = d2_fp64_sub(x, C + (size_t)l * D, D, sub);
                if (d < best) { best = d; bl = l; }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (ob < best || (ob == best && ol < bl)) { best = ob; bl = ol; }
        }
        if (lane == 0) list_of_row[row] = bl;
    }
}

// One warp per queued row whose candidates are confined to the 32-centroid chunks of
// its mask (as found by the tensor-core kernel): FP32 direct differences over those
// chunks, then FP64 among the FP32 near-ties.  A zero mask means every chunk.
// FP32 squared distance by direct differences: four partial sums over 16-byte loads when rows
// are 16-byte aligned (D % 4 == 0), one sum otherwise.  Either way its error is below gamma_D
// times the exact value, the bound the re-check's margin is built on.
__device__ __forceinline__ float d2_f32(const float *__restrict__ x, const float *__restrict__ c, int D)
{
    if ((D & 3) == 0) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x), *c4 = reinterpret_cast<const float4 *>(c);
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll 4
        for (int j = 0; j < D / 4; ++j) {
            const float4 u = x4[j], v = c4[j];
            const float t0 = u.x - v.x, t1 = u.y - v.y, t2 = u.z - v.z, t3 = u.w - v.w;
            a0 = fmaf(t0, t0, a0);
            a1 = fmaf(t1, t1, a1);
            a2 = fmaf(t2, t2, a2);
            a3 = fmaf(t3, t3, a3);
        }
        return (a0 + a1) + (a2 + a3);
    }
    float d = 0.0f;
    for (int j = 0; j < D; ++j) {
        const float t = x[j] - c[j];
        d = fmaf(t, t, d);
    }
    return d;
}

__global__ void coarse_recheck_masked_kernel(const float *__restrict__ X, int D, const float *__restrict__ C,
                                             int nlist, const int64_t *__restrict__ queue,
                                             const uint32_t *__restrict__ qmask,
                                             const unsigned long long *queue_len, int32_t *__restrict__ list_of_row,
                                             int sub)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long total = *queue_len;
    const int nchunks = (nlist + 31) / 32;
    // relative error of an FP32 direct-difference distance over D dimensions, with margin
    const float rel = 2.5f * (2.0f * 5.9604645e-8f + gamma_f32(D));
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < (int64_t)total; w += nw) {
        const int64_t row = queue[w];
        const uint32_t m = qmask[w];
        const float *x = X + row * D;
        float d1 = FLT_MAX, d2 = FLT_MAX;
        int i1 = 0x7fffffff;
        for (int c = 0; c < nchunks; ++c) {
            if (m != 0u && c < 32 && !((m >> c) & 1u)) continue;
            const int l = c * 32 + lane;
            if (l >= nlist) continue;
            const float d = d2_f32(x, C + (size_t)l * D, D);
            if (d < d1) { d2 = d1; d1 = d; i1 = l; }
            else if (d < d2) { d2 = d; }
        }
        // warp top-2
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float od1 = __shfl_xor_sync(0xffffffffu, d1, o);
            const float od2 = __shfl_xor_sync(0xffffffffu, d2, o);
            const int oi = __shfl_xor_sync(0xffffffffu, i1, o);
            const bool take = od1 < d1 || (od1 == d1 && oi < i1);
            const float rest = take ? fminf(d1, od2) : fminf(d2, od1);
            if (take) { d1 = od1; i1 = oi; }
            d2 = rest;
        }
        const float margin = rel * d2 + 1e-30f;
        int res = i1;
        if (!(d2 - d1 > margin)) {
            double best = DBL_MAX;
            int bl = 0x7fffffff;
            for (int c = 0; c < nchunks; ++c) {
                if (m != 0u && c < 32 && !((m >> c) & 1u)) continue;
                const int l = c * 32 + lane;
                if (l >= nlist) continue;
                const float *cl = C + (size_t)l * D;
                const float d = d2_f32(x, cl, D);
                if (d <= d1 + margin) {
                    const double e = d2_fp64_sub(x, cl, D, sub);
                    if (e < best || (e == best && l < bl)) { best = e; bl = l; }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
                if (ob < best || (ob == best && ol < bl)) { best = ob; bl = ol; }
            }
            res = bl;
        }
        if (lane == 0) list_of_row[row] = res;
    }
}

__global__ void bucket_hist_kernel(const int32_t *__restrict__ lst, int64_t N, int nlist, int *__restrict__ tile_cnt)
{
    extern __shared__ int s_hist[];
    for (int l = threadIdx.x; l < nlist; l += blockDim.x) s_hist[l] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kTileRows;
    const int64_t t1 = min(N, t0 + kTileRows);
    // an index outside [0, nlist) is only left behind by a kernel that reported a device-side
    // failure; both bucketing passes map it to list 0 so that no access leaves the histogram
    for (int64_t n = t0 + threadIdx.x; n < t1; n += blockDim.x) {
        const int l = lst[n];
        atomicAdd(s_hist + ((unsigned)l < (unsigned)nlist ? l : 0), 1);
    }
    __syncthreads();
    for (int l = threadIdx.x; l < nlist; l += blockDim.x) tile_cnt[(size_t)blockIdx.x * nlist + l] = s_hist[l];
}

// Per list: running count over tiles (in place) and the list total.  One warp per list takes
// 32 consecutive tiles at a time and scans them with shuffles.
__global__ void bucket_column_kernel(int *__restrict__ tile_cnt, int n_tiles, int nlist, int64_t *__restrict__ total)
{
    const int l = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (l >= nlist) return;  // whole warps only
    int64_t run = 0;
    for (int t0 = 0; t0 < n_tiles; t0 += 32) {
        const int t = t0 + lane;
        const int c = t < n_tiles ? tile_cnt[(size_t)t * nlist + l] : 0;
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (t < n_tiles) tile_cnt[(size_t)t * nlist + l] = (int)(run + inc - c);
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) total[l] = run;
}

// Exclusive scan of the list totals into offsets[0..nlist], one block.
__global__ void bucket_offsets_kernel(const int64_t *__restrict__ total, int nlist, int64_t *__restrict__ offsets)
{
    __shared__ int64_t s_carry;
    __shared__ int64_t s_warp[32];
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < nlist; base += blockDim.x) {
        const int l = base + threadIdx.x;
        int64_t v = l < nlist ? total[l] : 0;
        int64_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) s_warp[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int64_t w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            if (lane < nw) s_warp[lane] = w;
        }
        __syncthreads();
        const int64_t before = (wid > 0 ? s_warp[wid - 1] : 0) + s_carry;
        if (l < nlist) offsets[l] = before + inc - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = before + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) offsets[nlist] = s_carry;
}

// One warp per tile walks its rows in order; rows of one list keep ascending ids.
__global__ void bucket_scatter_kernel(const int32_t *__restrict__ lst, int64_t N, int nlist,
                                      const int *__restrict__ tile_base, const int64_t *__restrict__ offsets,
                                      const uint8_t *__restrict__ codes, int M, int64_t *__restrict__ ids,
                                      uint8_t *__restrict__ list_codes)
{
    extern __shared__ int s_run[];
    const int lane = threadIdx.x;
    for (int l = lane; l < nlist; l += 32) s_run[l] = 0;
    __syncwarp();
    const int64_t t0 = (int64_t)blockIdx.x * kTileRows;
    const int64_t t1 = min(N, t0 + kTileRows);
    const int *base = tile_base + (size_t)blockIdx.x * nlist;
    const bool vec16 = (M == 16) && codes && ((reinterpret_cast<uintptr_t>(codes) & 15) == 0) &&
                       ((reinterpret_cast<uintptr_t>(list_codes) & 15) == 0);
    for (int64_t c = t0; c < t1; c += 32) {
        const int64_t n = c + lane;
        const bool act = n < t1;
        const unsigned amask = __ballot_sync(0xffffffffu, act);
        int l = act ? lst[n] : -1;
        if (act && (unsigned)l >= (unsigned)nlist) l = 0;  // as in bucket_hist_kernel
        const unsigned peers = __match_any_sync(0xffffffffu, l);
        if (act) {
            const int rank = __popc(peers & ((1u << lane) - 1u));
            const int64_t pos = offsets[l] + base[l] + s_run[l] + rank;
            ids[pos] = n;
            if (codes) {
                if (vec16) {
                    *reinterpret_cast<uint4 *>(list_codes + pos * 16) =
                        *reinterpret_cast<const uint4 *>(codes + n * 16);
                } else {
                    for (int j = 0; j < M; ++j) list_codes[pos * M + j] = codes[n * M + j];
                }
            }
        }
        __syncwarp();
        if (act && lane == __ffs(peers & amask) - 1) s_run[l] += __popc(peers & amask);
        __syncwarp();
    }
}

// List means (the centroid update of Sec. 2.2), each equal to the sum of the list's rows in
// ascending row order in FP64, divided by the count and rounded to FP32.  The sequential FP64
// sum is obtained without FP64 additions whenever it is exact: a column whose elements are all
// multiples of 2^(e - 150) (e = the smallest biased exponent among them, subnormals counted as
// 1) and whose sum of magnitudes is below 2^(e - 150 + 53) has every partial sum representable
// in 53 bits, so each FP64 addition is exact and the sequential sum is the exact sum.  That sum
// is accumulated exactly as a 128-bit integer in units of 2^(g - 150), g = the smallest exponent
// of all of X, using integer instructions only.  A column that fails the test (or all columns,
// when X spans too many binades for 128 bits or holds Inf/NaN) is summed in FP64 in row order.

// Exponent range of the nonzero elements of X: r[0] = min, r[1] = max biased exponent
// (subnormals as 1, Inf/NaN as 255).
__global__ void x_exponent_range_kernel(const uint32_t *__restrict__ bits, int64_t n, unsigned *__restrict__ r)
{
    unsigned lo = 255u, hi = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = bits[i];
        if ((b & 0x7FFFFFFFu) == 0u) continue;
        const unsigned e = max((b >> 23) & 0xFFu, 1u);
        lo = min(lo, e);
        hi = max(hi, e);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(r, lo);
        atomicMax(r + 1, hi);
    }
}

constexpr int kMeanThreads = 1024;

// Row-order FP64 sum of column j over rows [b, e) of a list by one warp: 32 rows are loaded at a
// time (one per lane), then every lane adds them in row order, so all lanes hold the same sum.
__device__ double list_sum_fp64_warp(const float *__restrict__ X, int D, const int64_t *__restrict__ ids, int64_t b,
                                     int64_t e, int j, int lane)
{
    double s = 0.0;
    float v = (b + lane < e) ? X[ids[b + lane] * D + j] : 0.0f;
    for (int64_t p0 = b; p0 < e; p0 += 32) {
        const int64_t pn = p0 + 32 + lane;
        const float vn = pn < e ? X[ids[pn] * D + j] : 0.0f;  // next batch in flight
        const int cnt = (int)min((int64_t)32, e - p0);
        for (int k = 0; k < cnt; ++k) s = __dadd_rn(s, (double)__shfl_sync(0xffffffffu, v, k));
        v = vn;
    }
    return s;
}

// The exact list sums in two kernels, so that a long list is spread over many blocks: its rows are
// cut into pieces of kPieceRows.  list_partial_kernel: one block per piece, threads = row groups x
// columns; each thread adds its rows (a stride of the piece) exactly into a 128-bit integer and the
// row groups' partials are combined exactly.  list_mean_kernel: one block per list adds its pieces'
// partials exactly, so the sum is the same whatever the split.
constexpr int kPieceRows = 2048;

// Pieces of every list: list l has pieces [pbeg[l], pbeg[l+1]) (ceil(n_l / kPieceRows) of them), and
// piece_list[p] is the list of piece p.  One block: thread t takes the lists [t*per, (t+1)*per).
__global__ void __launch_bounds__(1024) list_pieces_kernel(const int64_t *__restrict__ offsets, int nlist,
                                                           int *__restrict__ pbeg, int *__restrict__ piece_list)
{
    __shared__ int s_sum[1024];
    const int t = threadIdx.x;
    const int per = (nlist + 1023) / 1024;
    const int l0 = min(nlist, t * per), l1 = min(nlist, l0 + per);
    int c = 0;
    for (int l = l0; l < l1; ++l) c += (int)((offsets[l + 1] - offsets[l] + kPieceRows - 1) / kPieceRows);
    s_sum[t] = c;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the thread counts
        const int v = t >= o ? s_sum[t - o] : 0;
        __syncthreads();
        s_sum[t] += v;
        __syncthreads();
    }
    int q = s_sum[t] - c;
    for (int l = l0; l < l1; ++l) {
        pbeg[l] = q;
        const int k = (int)((offsets[l + 1] - offsets[l] + kPieceRows - 1) / kPieceRows);
        for (int i = 0; i < k; ++i) piece_list[q + i] = l;
        q += k;
    }
    if (t == 1023) pbeg[nlist] = s_sum[1023];
}

// Exact-sum test of a list of n rows: the integer sums fit 128 bits.
__device__ __forceinline__ bool list_sum_fast(unsigned g, unsigned gmax, int64_t n)
{
    const int nbits = 64 - __clzll((unsigned long long)n);
    return gmax < 255u && (int)(gmax - g) + 24 + nbits + 1 <= 127;
}

__global__ void __launch_bounds__(kMeanThreads) list_partial_kernel(const float *__restrict__ X, int D,
                                                                    const int64_t *__restrict__ offsets,
                                                                    const int64_t *__restrict__ ids,
                                                                    const unsigned *__restrict__ xrange,
                                                                    const int *__restrict__ pbeg, int nlist,
                                                                    const int *__restrict__ piece_list,
                                                                    const ListMeanScratch part)
{
    __shared__ unsigned long long s_lo[kMeanThreads], s_hi[kMeanThreads];
    __shared__ unsigned s_neg[kMeanThreads], s_emin[kMeanThreads];
    __shared__ float s_abs[kMeanThreads];
    const int pc = blockIdx.x;
    if (pc >= pbeg[nlist]) return;
    const int l = piece_list[pc];
    const int64_t lb = offsets[l], le = offsets[l + 1];
    const int64_t b = lb + (int64_t)(pc - pbeg[l]) * kPieceRows, e = min(le, b + kPieceRows);
    unsigned g = xrange[0], gmax = xrange[1];
    if (g > gmax) g = gmax = 1u;  // X is all zeros
    // |sum| < n 2^(gmax - 126) = 2^(log2 n + gmax - g + 24) units, plus a sign bit
    if (!list_sum_fast(g, gmax, le - lb)) return;  // the list is summed in row order by list_mean_kernel
    const int Dp = (D + 31) & ~31, RG = blockDim.x / Dp;
    const int j = threadIdx.x % Dp, rg = threadIdx.x / Dp;
    {
        unsigned long long lo = 0ull, hi = 0ull;
        unsigned nneg = 0u, emin = 255u;
        float sabs = 0.0f;
        {
            // every lane takes part (the shuffles need the whole warp); lanes past the last column add zeros
            const uint32_t *xb = reinterpret_cast<const uint32_t *>(X);
            auto add = [&](uint32_t w) {
                const unsigned f = (w >> 23) & 0xFFu;
                const uint32_t m = (w & 0x7FFFFFu) | (f ? 0x800000u : 0u);
                const unsigned ee = max(f, 1u);
                emin = min(emin, m ? ee : 255u);
                sabs += fabsf(__uint_as_float(w));
                const unsigned sh = m ? ee - g : 0u;  // < 103: the fast test bounds gmax - g
                unsigned long long vlo, vhi;
                if (sh < 64u) {
                    vlo = (unsigned long long)m << sh;
                    vhi = sh > 40u ? (unsigned long long)m >> (64u - sh) : 0ull;
                } else {
                    vlo = 0ull;
                    vhi = (unsigned long long)m << (sh - 64u);
                }
                // a negative term adds its one's complement; the missing +1s are counted
                const unsigned long long neg = (w >> 31) ? ~0ull : 0ull;
                nneg += (unsigned)(w >> 31);
                asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(vlo ^ neg), "l"(vhi ^ neg));
            };
            // row group rg takes a consecutive run of the piece; its warps read 32 ids at a time (one per
            // lane, consecutive) and hand them round by shuffles, with eight row loads in flight
            const int64_t per = (e - b + RG - 1) / RG;
            const int64_t r0 = min(e, b + rg * per), r1 = min(e, r0 + per);
            const int lane = threadIdx.x & 31;
            for (int64_t p0 = r0; p0 < r1; p0 += 32) {
                const int cnt = (int)min((int64_t)32, r1 - p0);
                const int64_t myid = lane < cnt ? ids[p0 + lane] : 0;
                int t = 0;
                for (; t + 8 <= cnt; t += 8) {
                    uint32_t w[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int64_t row = __shfl_sync(0xffffffffu, myid, t + q);
                        w[q] = j < D ? xb[row * D + j] : 0u;
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) add(w[q]);
                }
                for (; t < cnt; ++t) {
                    const int64_t row = __shfl_sync(0xffffffffu, myid, t);
                    add(j < D ? xb[row * D + j] : 0u);
                }
            }
        }
        s_lo[threadIdx.x] = lo;
        s_hi[threadIdx.x] = hi;
        s_neg[threadIdx.x] = nneg;
        s_emin[threadIdx.x] = emin;
        s_abs[threadIdx.x] = sabs;
    }
    __syncthreads();
    if (rg == 0 && j < D) {
        unsigned long long lo = 0ull, hi = 0ull;
        unsigned nneg = 0u, emin = 255u;
        float sabs = 0.0f;
        for (int r = 0; r < RG; ++r) {
            const int t = r * Dp + j;
            asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(s_lo[t]), "l"(s_hi[t]));
            nneg += s_neg[t];
            emin = min(emin, s_emin[t]);
            sabs += s_abs[t];
        }
        const size_t o = (size_t)pc * D + j;
        part.lo[o] = lo;
        part.hi[o] = hi;
        part.neg[o] = nneg;
        part.emin[o] = emin;
        part.abs[o] = sabs;
    }
}

// The mean of every column of list l from its pieces' partials: exact when the row-order FP64 sum is
// provably the exact sum, else (flagged columns) that row-order sum by one warp per column.
__global__ void __launch_bounds__(kMeanThreads) list_mean_kernel(const float *__restrict__ X, int D,
                                                                 const int64_t *__restrict__ offsets,
                                                                 const int64_t *__restrict__ ids,
                                                                 const unsigned *__restrict__ xrange,
                                                                 const int *__restrict__ pbeg,
                                                                 const ListMeanScratch part, float *__restrict__ C)
{
    __shared__ int s_flag[256];
    __shared__ int s_nflag;
    const int l = blockIdx.x;
    const int64_t b = offsets[l], e = offsets[l + 1];
    if (e == b) return;  // empty list keeps its centroid
    const int64_t n = e - b;
    const int j = threadIdx.x;
    unsigned g = xrange[0], gmax = xrange[1];
    if (g > gmax) g = gmax = 1u;  // X is all zeros
    const bool fast = list_sum_fast(g, gmax, n);
    if (threadIdx.x == 0) s_nflag = 0;
    __syncthreads();
    if (j < D) {
        bool exact = false;
        double sum = 0.0;
        if (fast) {
            unsigned long long lo = 0ull, hi = 0ull, nneg = 0ull;
            unsigned emin = 255u;
            float sabs = 0.0f;
            for (int pc = pbeg[l]; pc < pbeg[l + 1]; ++pc) {
                const size_t o = (size_t)pc * D + j;
                asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(part.lo[o]), "l"(part.hi[o]));
                nneg += part.neg[o];
                emin = min(emin, part.emin[o]);
                sabs += part.abs[o];
            }
            asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(lo), "+l"(hi) : "l"(nneg));
            if (emin == 255u) {
                exact = true;  // every element is zero
            } else {
                // sum of magnitudes (FP32, relative error below n 2^-24) against 2^(emin - 97)
                const double bound = (double)sabs * (1.0 + 1.2e-7 * (double)n);
                if (bound < ldexp(1.0, (int)emin - 97)) {
                    const unsigned sh = emin - g;  // the sum is a multiple of 2^sh units
                    long long J;
                    if (sh >= 64u) {
                        J = (long long)hi >> (sh - 64u);
                    } else if (sh == 0u) {
                        J = (long long)lo;
                    } else {
                        J = (long long)((lo >> sh) | (hi << (64u - sh)));
                    }
                    sum = ldexp((double)J, (int)emin - 150);  // |J| < 2^53: exact
                    exact = true;
                }
            }
        }
        if (exact) {
            C[(size_t)l * D + j] = __double2float_rn(__ddiv_rn(sum, (double)n));
        } else {
            s_flag[atomicAdd(&s_nflag, 1)] = j;
        }
    }
    __syncthreads();
    // columns whose row-order FP64 sum is not provably exact: one warp each
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int f = warp; f < s_nflag; f += nwarps) {
        const int jj = s_flag[f];
        const double sum = list_sum_fp64_warp(X, D, ids, b, e, jj, lane);
        if (lane == 0) C[(size_t)l * D + jj] = __double2float_rn(__ddiv_rn(sum, (double)n));
    }
}

}  // namespace

int launch_coarse_norms(const float *C, int nlist, int D, CoarseBound &b, cudaStream_t s)
{
    PQ_TRY_CUDA(cudaMemsetAsync(b.maxes, 0, 2 * sizeof(float), s));
    const int blocks = std::max(1, std::min((nlist + 255) / 256, 152));
    ProfScope ps("coarse_norms", s);
    coarse_norms_kernel<<<blocks, 256, 0, s>>>(C, nlist, D, b.half_norm, b.maxes);
    coarse_bound_finish<<<1, 1, 0, s>>>(b.maxes, D);
    count_launch(2);
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

int coarse_assign(const float *X, int64_t N, int D, const float *C, int nlist, const CoarseBound &b,
                  int32_t *list_of_row, Scratch &ws, int prec, cudaStream_t s, int sub)
{
    int64_t *queue = ws.get<int64_t>((size_t)N);
    unsigned long long *qlen = ws.get<unsigned long long>(1, true);
    if (ws.status) return ws.status;
    if (prec == PQ_PREC_BF16 && coarse_tc_supported(D, nlist)) {
        uint32_t *qmask = ws.get<uint32_t>((size_t)N);
        if (ws.status) return ws.status;
        PQ_TRY(launch_coarse_tc(X, N, D, C, nlist, list_of_row, queue, qmask, qlen, ws, s));
        ProfScope ps("coarse_recheck", s);
        coarse_recheck_masked_kernel<<<152 * 4, 256, 0, s>>>(X, D, C, nlist, queue, qmask, qlen, list_of_row, sub);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
        return PQ_OK;
    } else {
        const int64_t blocks = (N + BM - 1) / BM;
        ProfScope ps("coarse_assign", s);
        coarse_scores_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(X, N, D, C, nlist, b.half_norm, b.maxes,
                                                                   list_of_row, queue, qlen, nullptr);
    }
    {
        ProfScope ps("coarse_recheck", s);
        coarse_recheck_kernel<<<152 * 4, 256, 0, s>>>(X, D, C, nlist, b.half_norm, b.maxes, queue, qlen,
                                                      list_of_row, sub);
    }
    count_launch(2);
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

int launch_coarse_all_scores(const float *Q, int64_t nq, int D, const float *C, int nlist, const CoarseBound &b,
                             float *S, cudaStream_t s)
{
    const int64_t blocks = (nq + BM - 1) / BM;
    ProfScope ps("probe_scores", s);
    coarse_scores_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(Q, nq, D, C, nlist, b.half_norm, b.maxes, nullptr,
                                                                nullptr, nullptr, S);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

int bucket_rows(const int32_t *list_of_row, int64_t N, int nlist, const uint8_t *codes, int M, int64_t *offsets,
                int64_t *ids, uint8_t *list_codes, Scratch &ws, cudaStream_t s)
{
    const int64_t n_tiles = (N + kTileRows - 1) / kTileRows;
    int *tile_cnt = ws.get<int>((size_t)n_tiles * nlist);
    int64_t *total = ws.get<int64_t>((size_t)nlist);
    if (ws.status) return ws.status;
    const size_t hsm = (size_t)nlist * sizeof(int);
    if (hsm > 200 * 1024) return fail(PQ_ENOTSUP, "nlist=%d too large for bucketing", nlist);
    PQ_TRY_CUDA(cudaFuncSetAttribute(bucket_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
    PQ_TRY_CUDA(cudaFuncSetAttribute(bucket_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
    ProfScope ps("bucket", s);
    bucket_hist_kernel<<<(unsigned)n_tiles, 256, hsm, s>>>(list_of_row, N, nlist, tile_cnt);
    bucket_column_kernel<<<(nlist + 7) / 8, 256, 0, s>>>(tile_cnt, (int)n_tiles, nlist, total);
    bucket_offsets_kernel<<<1, 1024, 0, s>>>(total, nlist, offsets);
    bucket_scatter_kernel<<<(unsigned)n_tiles, 32, hsm, s>>>(list_of_row, N, nlist, tile_cnt, offsets, codes, M, ids,
                                                              list_codes);
    count_launch(4);
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

int launch_x_exponent_range(const float *X, int64_t N, int D, unsigned *xrange, cudaStream_t s)
{
    PQ_TRY_CUDA(cudaMemsetAsync(xrange, 0xFF, sizeof(unsigned), s));
    PQ_TRY_CUDA(cudaMemsetAsync(xrange + 1, 0, sizeof(unsigned), s));
    ProfScope ps("x_exponent_range", s);
    x_exponent_range_kernel<<<152 * 4, 256, 0, s>>>(reinterpret_cast<const uint32_t *>(X), N * D, xrange);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

int list_mean_scratch(int64_t N, int D, int nlist, Scratch &ws, ListMeanScratch &lm)
{
    // at most N / kPieceRows + nlist pieces (every list rounds its piece count up once)
    lm.pmax = N / kPieceRows + nlist + 1;
    if (lm.pmax > INT_MAX / 2) return fail(PQ_ENOTSUP, "too many rows for list means");
    lm.pbeg = ws.get<int>((size_t)nlist + 1);
    lm.piece_list = ws.get<int>((size_t)lm.pmax);
    lm.lo = ws.get<unsigned long long>((size_t)lm.pmax * D);
    lm.hi = ws.get<unsigned long long>((size_t)lm.pmax * D);
    lm.neg = ws.get<unsigned>((size_t)lm.pmax * D);
    lm.emin = ws.get<unsigned>((size_t)lm.pmax * D);
    lm.abs = ws.get<float>((size_t)lm.pmax * D);
    return ws.status;
}

int launch_list_mean(const float *X, int D, const int64_t *offsets, const int64_t *ids, int nlist,
                     const unsigned *xrange, float *C, const ListMeanScratch &lm, cudaStream_t s)
{
    if (D > 256) return fail(PQ_ENOTSUP, "list means support D <= 256");
    if (lm.pmax <= 0) return fail(PQ_EINTERNAL, "list means without scratch");
    ProfScope ps("list_mean", s);
    const int Dp = (D + 31) / 32 * 32;
    list_pieces_kernel<<<1, 1024, 0, s>>>(offsets, nlist, lm.pbeg, lm.piece_list);
    list_partial_kernel<<<(unsigned)lm.pmax, Dp * (kMeanThreads / Dp), 0, s>>>(X, D, offsets, ids, xrange, lm.pbeg,
                                                                               nlist, lm.piece_list, lm);
    list_mean_kernel<<<nlist, kMeanThreads, 0, s>>>(X, D, offsets, ids, xrange, lm.pbeg, lm, C);
    count_launch(3);
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

}  // namespace pqgb
