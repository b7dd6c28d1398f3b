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
constexpr int kCap = 2048;  // candidate buffer entries per query

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
                                                                int32_t *__restrict__ probes)
{
    extern __shared__ Cand s_c[];  // [nlist_p2]
    __shared__ float s_xx[kThreads / 32];
    __shared__ int s_nsure, s_band_lo, s_band_hi;
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
        s_nsure = lo;
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
            const double d = d2_fp64(qv, coarse + (size_t)l * D, D);
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

// Sort the buffer, keep the first k, return the new threshold.
__device__ float compact(Cand *buf, int *count, int k)
{
    const int n = *count;
    for (int i = n + threadIdx.x; i < kCap; i += blockDim.x) { buf[i].d = FLT_MAX; buf[i].id = 0x7fffffff; }
    bitonic_sort(buf, kCap);
    const int keep = min(n, k);
    float tau = (n >= k) ? buf[k - 1].d : FLT_MAX;
    __syncthreads();
    if (threadIdx.x == 0) *count = keep;
    __syncthreads();
    return tau;
}

template <int M>
__global__ void __launch_bounds__(kThreads) adc_scan_kernel(const float *__restrict__ Q, int D, int Ks,
                                                            const float *__restrict__ codebooks,
                                                            const int32_t *__restrict__ probes, int nprobe,
                                                            const int64_t *__restrict__ offsets,
                                                            const int64_t *__restrict__ ids,
                                                            const uint8_t *__restrict__ list_codes, int k,
                                                            int64_t *__restrict__ out_ids, float *__restrict__ out_d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *lut = reinterpret_cast<float *>(smem_raw);                 // [M][Ks]
    Cand *buf = reinterpret_cast<Cand *>(lut + (size_t)M * Ks);       // [kCap]
    __shared__ int s_count;
    const int64_t q = blockIdx.x;
    const float *qv = Q + q * D;
    const int ds = D / M;
    for (int e = threadIdx.x; e < M * Ks; e += kThreads) {
        const int m = e / Ks, kk = e % Ks;
        const float *c = codebooks + ((size_t)m * Ks + kk) * ds;
        float acc = 0.0f;
        for (int j = 0; j < ds; ++j) {
            const float t = qv[m * ds + j] - c[j];
            acc = fmaf(t, t, acc);
        }
        lut[e] = acc;
    }
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    float tau = FLT_MAX;
    for (int p = 0; p < nprobe; ++p) {
        const int l = probes[q * nprobe + p];
        const int64_t beg = offsets[l], end = offsets[l + 1];
        for (int64_t e0 = beg; e0 < end; e0 += kThreads) {
            const int64_t e = e0 + threadIdx.x;
            if (e < end) {
                uint8_t c[M];
                load_codes<M>(list_codes + e * M, c);
                float d = 0.0f;
#pragma unroll
                for (int m = 0; m < M; ++m) d += lut[m * Ks + c[m]];
                if (d <= tau) {
                    const int slot = atomicAdd(&s_count, 1);
                    buf[slot].d = d;
                    buf[slot].id = (int)ids[e];
                }
            }
            __syncthreads();
            if (s_count > kCap - kThreads) tau = compact(buf, &s_count, k);
        }
    }
    tau = compact(buf, &s_count, k);
    const int n = s_count;
    for (int r = threadIdx.x; r < k; r += kThreads) {
        out_ids[q * k + r] = r < n ? (int64_t)buf[r].id : -1;
        out_d[q * k + r] = r < n ? buf[r].d : __int_as_float(0x7f800000);
    }
}

template <int M>
int launch_scan(const SearchArgs &a, const int32_t *probes, cudaStream_t s)
{
    const size_t smem = (size_t)M * a.Ks * sizeof(float) + kCap * sizeof(Cand);
    PQ_TRY_CUDA(cudaFuncSetAttribute(adc_scan_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps("adc_scan", s);
    adc_scan_kernel<M><<<(unsigned)a.nq, kThreads, smem, s>>>(a.Q, a.D, a.Ks, a.codebooks, probes, a.nprobe,
                                                             a.offsets, a.ids, a.list_codes, a.k, a.out_ids, a.out_d);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
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
                                                              a.cb->maxes, probes);
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
