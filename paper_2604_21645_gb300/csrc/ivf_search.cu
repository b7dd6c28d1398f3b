// ivf_search.cu -- k-nearest-neighbour query over the inverted lists with the
// PQ distance table (Sec. 2.2: inverted index over the codes, k nearest
// results; Sec. 3.1: Rii as an IVFPQ-style index).
//
// 1. Probe: FP32 scores of the query against every coarse centroid (tiled
//    kernel), then per query the nprobe lowest by exact FP64 distance (ties to
//    the lower list id): lists whose FP32 score is clearly inside the cut are
//    taken as they are, the few inside the FP32 error band around the cut are
//    re-ranked in FP64.
// 2. Scan: one block per query builds LUT[m][k] = ||q_m - c_{m,k}||^2 in
//    shared memory, streams the probed lists' codes with 128-bit loads, scores
//    each code as sum_m LUT[m][code_m] and keeps a threshold-filtered
//    candidate buffer that is compacted by a bitonic sort on (score, id).
#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "internal.h"

namespace pqgb {

int launch_coarse_all_scores(const float *Q, int64_t nq, int D, const float *C, int nlist, const CoarseBound &b,
                             float *S, cudaStream_t s);

namespace {

constexpr int kThreads = 256;
constexpr int kMaxProbe = 256;  // probed lists per query held in shared memory

struct Cand {
    float d;
    int id;
};

__device__ __forceinline__ bool cand_less(const Cand &a, const Cand &b)
{
    return a.d < b.d || (a.d == b.d && a.id < b.id);
}

// In-place ascending bitonic sort of n (power of two) entries by all threads.
__device__ void bitonic_sort(Cand *v, int n)
{
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                Cand a = v[lo], b = v[hi];
                if (cand_less(b, a) == up) { v[lo] = b; v[hi] = a; }
            }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) probe_select_kernel(const float *__restrict__ S, const float *__restrict__ Q,
                                                                int D, int nlist, int nlist_p2, int nprobe,
                                                                const float *__restrict__ coarse,
                                                                const float *__restrict__ maxes,
                                                                int32_t *__restrict__ probes, int sub)
{
    extern __shared__ Cand s_c[];  // [nlist_p2]
    __shared__ float s_xx[kThreads / 32];
    __shared__ int s_band_lo, s_band_hi;
    const int64_t q = blockIdx.x;
    const float *Sq = S + q * nlist;
    const float *qv = Q + q * D;
    float xx = 0.0f;
    for (int j = threadIdx.x; j < D; j += kThreads) xx = fmaf(qv[j], qv[j], xx);
    xx = warp_sum(xx);
    if ((threadIdx.x & 31) == 0) s_xx[threadIdx.x >> 5] = xx;
    for (int l = threadIdx.x; l < nlist_p2; l += kThreads) {
        s_c[l].d = l < nlist ? Sq[l] : FLT_MAX;
        s_c[l].id = l < nlist ? l : 0x7fffffff;
    }
    __syncthreads();
    bitonic_sort(s_c, nlist_p2);
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) t += s_xx[w];
        const float xn = sqrtf(t) * (1.0f + 1e-6f);
        const float cmax = maxes[1];
        const float u = xn + cmax;
        const float delta = 2.2f * gamma_f32(D + 1) * (maxes[0] + xn * cmax) + 1e-13f * u * u;
        const float vp = s_c[nprobe - 1].d;
        int lo = 0;
        while (lo < nlist && s_c[lo].d < vp - 2.0f * delta) ++lo;
        int hi = nprobe;
        while (hi < nlist && s_c[hi].d <= vp + 2.0f * delta) ++hi;
        s_band_lo = lo;
        s_band_hi = hi;
    }
    __syncthreads();
    const int lo = s_band_lo, hi = s_band_hi;
    int32_t *pq = probes + q * nprobe;
    for (int i = threadIdx.x; i < lo; i += kThreads) pq[i] = s_c[i].id;
    if (lo < nprobe) {
        // FP64 re-rank of the band [lo, hi): the scores are replaced by exact distances
        for (int i = lo + threadIdx.x; i < hi; i += kThreads) {
            const int l = s_c[i].id;
            s_c[i].d = __int_as_float(i);  // placeholder, overwritten below
            const double d = d2_fp64_sub(qv, coarse + (size_t)l * D, D, sub);
            reinterpret_cast<double *>(s_c + nlist_p2)[i - lo] = d;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double *dd = reinterpret_cast<double *>(s_c + nlist_p2);
            // selection of the nprobe - lo best (distance, list) pairs of the band
            for (int r = lo; r < nprobe; ++r) {
                int best = -1;
                for (int i = lo; i < hi; ++i) {
                    if (s_c[i].id < 0) continue;
                    if (best < 0 || dd[i - lo] < dd[best - lo] ||
                        (dd[i - lo] == dd[best - lo] && s_c[i].id < s_c[best].id))
                        best = i;
                }
                pq[r] = s_c[best].id;
                s_c[best].id = -1;
            }
        }
    }
}

template <int M>
__device__ __forceinline__ void load_codes(const uint8_t *p, uint8_t (&c)[M])
{
    if constexpr (M % 16 == 0) {
#pragma unroll
        for (int i = 0; i < M; i += 16) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p + i));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int b = 0; b < 16; ++b) c[i + b] = (uint8_t)(w[b >> 2] >> (8 * (b & 3)));
        }
    } else if constexpr (M % 8 == 0) {
#pragma unroll
        for (int i = 0; i < M; i += 8) {
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p + i));
            const uint32_t w[2] = {v.x, v.y};
#pragma unroll
            for (int b = 0; b < 8; ++b) c[i + b] = (uint8_t)(w[b >> 2] >> (8 * (b & 3)));
        }
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i) c[i] = __ldg(p + i);
    }
}

constexpr int kScanThreads = 256;
constexpr int kSelCap = 2048;      // candidate buffer entries per query
constexpr int kSamples = 512;      // codes scored first to set the candidate threshold ...
constexpr int kSamplesBig = 2048;  // ... and for a query with more than kBigScan probed codes
constexpr int kBigScan = 131072;
static_assert(kSamplesBig <= kSelCap, "the sample is sorted in the candidate buffer");

// In-place ascending bitonic sort of n (power of two) entries by every thread of the block.
__device__ void bitonic_sort_n(Cand *v, int n)
{
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                Cand x = v[lo], y = v[hi];
                if (cand_less(y, x) == up) { v[lo] = y; v[hi] = x; }
            }
        }
    }
    __syncthreads();
}

template <int M, int KS>
__device__ __forceinline__ float adc_score(const float *lut, const uint8_t *code)
{
    uint8_t c[M];
    load_codes<M>(code, c);
    float d = 0.0f;
#pragma unroll
    for (int m = 0; m < M; ++m) d += lut[m * KS + c[m]];
    return d;
}

// The same sum, left as soon as a partial sum exceeds tau.  Every LUT entry is a
// squared distance (>= 0) and a rounded FP32 sum of non-negative terms never
// decreases, so the full score of a code left early is above tau as well: the codes
// kept, and their scores (same terms in the same order), are those of adc_score.
template <int M, int KS>
__device__ __forceinline__ float adc_score_below(const float *lut, const uint8_t *code, float tau)
{
    uint8_t c[M];
    load_codes<M>(code, c);
    float d = 0.0f;
#pragma unroll
    for (int m = 0; m < M / 2; ++m) d += lut[m * KS + c[m]];
    if (d > tau) return d;
#pragma unroll
    for (int m = M / 2; m < (3 * M) / 4; ++m) d += lut[m * KS + c[m]];
    if (d > tau) return d;
#pragma unroll
    for (int m = (3 * M) / 4; m < M; ++m) d += lut[m * KS + c[m]];
    return d;
}

// Scan of one query (one block), in two phases.  (1) A threshold: the scores of
// S codes spread evenly over the probed lists are sorted (S = 512, or 2048 above
// kBigScan codes) and the one at about twice the expected rank of k is taken, but no
// higher than the rank expected to hold half the candidate buffer (with n probed
// codes, sample rank r stands for about (r + 1) n / (S + 1) codes).  (2) Every probed
// code is scored, left early once a partial sum passes the threshold, and the ones at
// or below the threshold (all ties included) go to the candidate buffer, which is
// sorted by (score, id) at the end.  If the threshold turns out too tight
// (fewer than k candidates) or too loose (buffer full), the scan is repeated with the
// threshold at +inf and the buffer compacted by sorting whenever it fills.
template <int M, int KS>
__global__ void __launch_bounds__(kScanThreads) adc_scan_kernel(const float *__restrict__ Q, int D, int Ks,
                                                                const float *__restrict__ codebooks,
                                                                const int32_t *__restrict__ probes, int nprobe,
                                                                const int64_t *__restrict__ offsets,
                                                                const int64_t *__restrict__ ids,
                                                                const uint8_t *__restrict__ list_codes, int k,
                                                                int64_t *__restrict__ out_ids, float *__restrict__ out_d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *lut = reinterpret_cast<float *>(smem_raw);                 // [M][KS]
    Cand *buf = reinterpret_cast<Cand *>(lut + M * KS);               // [kSelCap]
    __shared__ int64_t s_beg[kMaxProbe];
    __shared__ int s_pre[kMaxProbe + 1];
    __shared__ int s_count, s_n;
    const int64_t q = blockIdx.x;
    const float *qv = Q + q * D;
    const int ds = D / M;
    for (int e = threadIdx.x; e < M * KS; e += kScanThreads) {
        const int m = e / KS, kk = e % KS;
        float acc = 0.0f;
        if (kk < Ks) {
            const float *c = codebooks + ((size_t)m * Ks + kk) * ds;
            for (int j = 0; j < ds; ++j) {
                const float t = qv[m * ds + j] - c[j];
                acc = fmaf(t, t, acc);
            }
        }
        lut[e] = acc;
    }
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int p = 0; p < nprobe; ++p) {
            const int l = probes[q * nprobe + p];
            s_beg[p] = offsets[l];
            s_pre[p] = tot;
            const int64_t len = offsets[l + 1] - offsets[l];
            tot += (int)(len < 0x3fffffff - tot ? len : 0x3fffffff - tot);
        }
        s_pre[nprobe] = tot;
        s_n = tot;
        s_count = 0;
    }
    __syncthreads();
    const int n = s_n;
    auto code_at = [&](int pos, int &p) -> const uint8_t * {
        p = 0;
        while (s_pre[p + 1] <= pos) ++p;
        return list_codes + (size_t)(s_beg[p] + (pos - s_pre[p])) * M;
    };
    // ---- (1) threshold from a sorted sample --------------------------------
    float tau = FLT_MAX;
    const int S = n > kBigScan ? kSamplesBig : kSamples;
    if (n > S) {
        for (int j = threadIdx.x; j < S; j += kScanThreads) {
            int p;
            const int pos = (int)(((int64_t)j * n) / S);
            buf[j].d = adc_score<M, KS>(lut, code_at(pos, p));
            buf[j].id = j;
        }
        bitonic_sort_n(buf, S);
        const int64_t r_lo = ((int64_t)2 * k * S + n - 1) / n + 2;         // about twice the rank of k
        const int64_t r_hi = (int64_t)(kSelCap / 2) * (S + 1) / n - 1;     // about half the buffer
        const int64_t r = min(r_lo, r_hi);
        tau = r < S ? buf[max(r, (int64_t)0)].d : FLT_MAX;
        __syncthreads();
    }
    // ---- (2) filtered scan, repeated without a threshold if it missed -------
    for (int attempt = 0; attempt < 2; ++attempt) {
        const bool stream = attempt == 1;  // threshold +inf, compaction by sorting
        if (stream) tau = FLT_MAX;
        if (threadIdx.x == 0) s_count = 0;
        __syncthreads();
        bool overflow = false;
        for (int p = 0; p < nprobe; ++p) {
            const int len = s_pre[p + 1] - s_pre[p];
            const uint8_t *lc = list_codes + s_beg[p] * M;
            const int64_t ib = s_beg[p];
            for (int e0 = 0; e0 < len; e0 += kScanThreads) {
                const int e = e0 + threadIdx.x;
                if (e < len) {
                    const float d = adc_score_below<M, KS>(lut, lc + (size_t)e * M, tau);
                    if (d <= tau) {
                        const int slot = atomicAdd(&s_count, 1);
                        if (slot < kSelCap) {
                            buf[slot].d = d;
                            buf[slot].id = (int)ids[ib + e];
                        }
                    }
                }
                if (stream) {
                    // one block-uniform snapshot of the count: every thread takes the same branch,
                    // and no thread adds to the buffer before all of them have read it
                    __syncthreads();
                    const int cnt = s_count;
                    __syncthreads();
                    if (cnt > kSelCap - kScanThreads) {
                        for (int i = cnt + threadIdx.x; i < kSelCap; i += kScanThreads) {
                            buf[i].d = FLT_MAX;
                            buf[i].id = 0x7fffffff;
                        }
                        bitonic_sort_n(buf, kSelCap);
                        tau = cnt >= k ? buf[k - 1].d : FLT_MAX;
                        __syncthreads();
                        if (threadIdx.x == 0) s_count = min(cnt, k);
                        __syncthreads();
                    }
                }
            }
        }
        __syncthreads();
        const int cnt = s_count;
        overflow = cnt > kSelCap;
        if (!stream && (overflow || (cnt < k && cnt < n))) continue;  // threshold missed: scan again
        const int c = min(cnt, kSelCap);
        int p2 = 1;
        while (p2 < c) p2 <<= 1;
        for (int i = c + threadIdx.x; i < p2; i += kScanThreads) { buf[i].d = FLT_MAX; buf[i].id = 0x7fffffff; }
        bitonic_sort_n(buf, p2);
        const int kk = min(c, k);
        for (int r2 = threadIdx.x; r2 < k; r2 += kScanThreads) {
            out_ids[q * k + r2] = r2 < kk ? (int64_t)buf[r2].id : -1;
            out_d[q * k + r2] = r2 < kk ? buf[r2].d : __int_as_float(0x7f800000);
        }
        return;
    }
}

template <int M, int KS>
int launch_scan_ks(const SearchArgs &a, const int32_t *probes, cudaStream_t s)
{
    const size_t smem = (size_t)M * KS * sizeof(float) + kSelCap * sizeof(Cand);
    PQ_TRY_CUDA(cudaFuncSetAttribute(adc_scan_kernel<M, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps("adc_scan", s);
    adc_scan_kernel<M, KS><<<(unsigned)a.nq, kScanThreads, smem, s>>>(a.Q, a.D, a.Ks, a.codebooks, probes, a.nprobe,
                                                                     a.offsets, a.ids, a.list_codes, a.k, a.out_ids,
                                                                     a.out_d);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

// The LUT row length is a template parameter (codes index it with an immediate offset);
// a codebook with fewer codewords uses the next supported length, its extra entries unused.
template <int M>
int launch_scan(const SearchArgs &a, const int32_t *probes, cudaStream_t s)
{
    if (a.nprobe > kMaxProbe) return fail(PQ_ENOTSUP, "nprobe=%d exceeds %d", a.nprobe, kMaxProbe);
    if (a.Ks <= 64) return launch_scan_ks<M, 64>(a, probes, s);
    return launch_scan_ks<M, 256>(a, probes, s);
}

}  // namespace

int run_search(const SearchArgs &a, Scratch &ws, cudaStream_t s)
{
    if (a.k > 1024) return fail(PQ_EINVAL, "k=%d exceeds 1024", a.k);
    float *S = ws.get<float>((size_t)a.nq * a.nlist);
    int32_t *probes = ws.get<int32_t>((size_t)a.nq * a.nprobe);
    if (ws.status) return ws.status;
    PQ_TRY(launch_coarse_all_scores(a.Q, a.nq, a.D, a.coarse, a.nlist, *a.cb, S, s));
    int p2 = 1;
    while (p2 < a.nlist) p2 <<= 1;
    const size_t smem = (size_t)p2 * sizeof(Cand) + (size_t)p2 * sizeof(double);
    if (smem > 200 * 1024) return fail(PQ_ENOTSUP, "nlist=%d too large for probe selection", a.nlist);
    PQ_TRY_CUDA(cudaFuncSetAttribute(probe_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
    ProfScope ps("probe_select", s);
    probe_select_kernel<<<(unsigned)a.nq, kThreads, smem, s>>>(S, a.Q, a.D, a.nlist, p2, a.nprobe, a.coarse,
                                                              a.cb->maxes, probes, a.probe_sub);
    }
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    switch (a.M) {
    case 4: return launch_scan<4>(a, probes, s);
    case 8: return launch_scan<8>(a, probes, s);
    case 12: return launch_scan<12>(a, probes, s);
    case 16: return launch_scan<16>(a, probes, s);
    case 32: return launch_scan<32>(a, probes, s);
    default: return fail(PQ_ENOTSUP, "ivf_search supports M in {4, 8, 12, 16, 32} (got %d)", a.M);
    }
}

}  // namespace pqgb
