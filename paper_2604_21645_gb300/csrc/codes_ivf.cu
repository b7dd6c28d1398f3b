// codes_ivf.cu -- the code-space inverted index: Rii's reading of the paper's
// inverted index (Sec. 3.1: an IVFPQ-style index that Rii builds from the PQ
// codes themselves, Sec. 2.2: the codes are hashed into lists).
//
// The coarse centres are PQ codes.  They come from k-means over the codes with
// the symmetric distance SDC(a, b) = sum_m ||c_{m,a_m} - c_{m,b_m}||^2, which is
// the squared distance of the two reconstructions:
//   - start: nlist distinct rows drawn by Floyd's algorithm from the centre
//     stream of the seed (host side, the same SplitMix64 draws as the CPU
//     reference);
//   - assignment: every row's reconstruction to its nearest decoded centre, on
//     the exact coarse-assignment machinery (FP32 or BF16 scores with a proven
//     bound, FP64 re-check summed per subspace in subspace order -- the way the
//     SDC table adds up);
//   - update ("sparse voting"): for list l and subspace m, with h[j] the number
//     of members whose code in m is j, the new centre code is the k minimising
//     cost(k) = sum_j h[j] * ||c_{m,k} - c_{m,j}||^2; the costs of all (l, m, k)
//     are one FP32 GEMM per subspace (histogram x distance table) whose argmin is
//     accepted when the FP32 error bound separates it, and re-decided in FP64 in
//     the reference's order otherwise.  A list without members keeps its centre.
// Queries probe with their own ADC table: ADC(q, centre) = ||q - decoded centre||^2,
// so the probe step is the raw-space one on the decoded centres, its FP64 band
// re-rank summed per subspace.
#include <algorithm>
#include <cfloat>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

constexpr uint64_t kStreamCenters = 0xFFFFFFFDull;

// DT32[m][k][j] = ||c_{m,k} - c_{m,j}||^2 in FP32 (FMA), DT64 in FP64 by direct differences
__global__ void sdc_tables_kernel(const float *__restrict__ C, int M, int Ks, int ds, float *__restrict__ DT32,
                                  double *__restrict__ DT64)
{
    const int64_t total = (int64_t)M * Ks * Ks;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % Ks);
        const int64_t mk = e / Ks;
        const int k = (int)(mk % Ks), m = (int)(mk / Ks);
        const float *a = C + ((size_t)m * Ks + k) * ds;
        const float *b = C + ((size_t)m * Ks + j) * ds;
        float d = 0.0f;
        for (int t = 0; t < ds; ++t) {
            const float u = a[t] - b[t];
            d = fmaf(u, u, d);
        }
        DT32[e] = d;
        DT64[e] = d2_fp64(a, b, ds);
    }
}

__global__ void gather_codes_kernel(const uint8_t *__restrict__ codes, const int64_t *__restrict__ rows, int n, int M,
                                    uint8_t *__restrict__ out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n * M) out[e] = codes[rows[e / M] * M + e % M];
}

// h[l][m][j] += 1 for every row n in list l whose code in subspace m is j
__global__ void center_hist_kernel(const uint8_t *__restrict__ codes, const int32_t *__restrict__ lst, int64_t N,
                                   int M, int Ks, int *__restrict__ hist)
{
    const int64_t total = N * M;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = e / M;
        const int m = (int)(e - n * M);
        const int j = codes[e];
        if (j < Ks) atomicAdd(hist + ((size_t)lst[n] * M + m) * Ks + j, 1);  // a code beyond the codebook has no vote
    }
}

// Costs of one subspace for a tile of 64 lists and all (<= 256) candidate codes k:
// cost[l][k] = sum_j h[l][m][j] * DT32[m][k][j], FP32.  Warp w owns lists 8w..8w+7, lane t the
// codes 8t..8t+7; the warp's argmin over k with the second-best cost either settles the list's
// new code (the FP32 error bound separates them) or queues (l, m) for the FP64 re-check.
constexpr int kLT = 64, kJT = 16;
__global__ void __launch_bounds__(256) center_cost_kernel(const int *__restrict__ hist, const float *__restrict__ DT32,
                                                          int nlist, int M, int Ks, uint8_t *__restrict__ centers,
                                                          int *__restrict__ queue, unsigned *__restrict__ qlen)
{
    __shared__ float s_h[kJT][kLT + 1];
    __shared__ float s_dt[kJT][256 + 4];
    const int m = blockIdx.y, l0 = blockIdx.x * kLT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
    const float *DTm = DT32 + (size_t)m * Ks * Ks;
    for (int j0 = 0; j0 < Ks; j0 += kJT) {
        __syncthreads();
        for (int e = threadIdx.x; e < kJT * kLT; e += 256) {
            const int jj = e % kJT, ll = e / kJT;
            const int l = l0 + ll, j = j0 + jj;
            s_h[jj][ll] = (l < nlist && j < Ks) ? (float)hist[((size_t)l * M + m) * Ks + j] : 0.0f;
        }
        for (int e = threadIdx.x; e < kJT * 256; e += 256) {
            const int jj = e % kJT, k = e / kJT;
            const int j = j0 + jj;
            s_dt[jj][k] = (k < Ks && j < Ks) ? DTm[(size_t)k * Ks + j] : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < kJT; ++jj) {
            float hv[8], dv[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) hv[a] = s_h[jj][warp * 8 + a];
#pragma unroll
            for (int b = 0; b < 8; ++b) dv[b] = s_dt[jj][lane * 8 + b];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(hv[a], dv[b], acc[a][b]);
        }
    }
    // every term is >= 0: the FP32 sum of Ks products of exact counts and FP32 table entries is
    // within (Ks + 2 ds + 4) 2^-24 of its value; twice that, on both costs, separates the argmin
    const float rel = 2.0f * (float)(Ks + 40) * 5.9604645e-8f;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int l = l0 + warp * 8 + a;
        float d1 = FLT_MAX, d2 = FLT_MAX;
        int k1 = INT_MAX;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int k = lane * 8 + b;
            if (k >= Ks) continue;
            const float c = acc[a][b];
            if (c < d1) { d2 = d1; d1 = c; k1 = k; }
            else d2 = fminf(d2, c);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float e1 = __shfl_xor_sync(0xffffffffu, d1, o);
            const int j1 = __shfl_xor_sync(0xffffffffu, k1, o);
            const float e2 = __shfl_xor_sync(0xffffffffu, d2, o);
            if (e1 < d1 || (e1 == d1 && j1 < k1)) {
                d2 = fminf(d1, e2);
                d1 = e1;
                k1 = j1;
            } else {
                d2 = fminf(d2, e1);
            }
        }
        // members of the list (the histogram of any subspace sums to them)
        int n_l = 0;
        if (l < nlist) {
            const int *hm = hist + ((size_t)l * M + m) * Ks;
            for (int j = lane; j < Ks; j += 32) n_l += hm[j];
        }
        n_l = warp_sum(n_l);
        if (lane == 0 && l < nlist && n_l > 0) {  // an empty list keeps its centre
            if (d2 - d1 > rel * (d1 + d2) + 1e-30f) {
                centers[(size_t)l * M + m] = (uint8_t)k1;
            } else {
                const unsigned slot = atomicAdd(qlen, 1u);
                queue[slot] = l * M + m;
            }
        }
    }
}

// One block per queued (list, subspace): cost(k) = sum over j (ascending) of h[j] * DT64[m][k][j]
// in FP64, each product and sum rounded once -- the reference's arithmetic -- and the lowest k
// of the minimum cost.
__global__ void __launch_bounds__(256) center_recheck_kernel(const int *__restrict__ hist,
                                                             const double *__restrict__ DT64, int M, int Ks,
                                                             const int *__restrict__ queue,
                                                             const unsigned *__restrict__ qlen,
                                                             uint8_t *__restrict__ centers)
{
    __shared__ double s_best[8];
    __shared__ int s_bk[8];
    __shared__ int s_h[256];
    const unsigned total = *qlen;
    for (unsigned w = blockIdx.x; w < total; w += gridDim.x) {
        const int lm = queue[w];
        const int l = lm / M, m = lm % M;
        __syncthreads();
        for (int j = threadIdx.x; j < Ks; j += blockDim.x) s_h[j] = hist[((size_t)l * M + m) * Ks + j];
        __syncthreads();
        double best = DBL_MAX;
        int bk = INT_MAX;
        for (int k = threadIdx.x; k < Ks; k += blockDim.x) {
            const double *row = DT64 + ((size_t)m * Ks + k) * Ks;
            double c = 0.0;
            for (int j = 0; j < Ks; ++j) c = __dadd_rn(c, __dmul_rn((double)s_h[j], row[j]));
            if (c < best || (c == best && k < bk)) {
                best = c;
                bk = k;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double e = __shfl_xor_sync(0xffffffffu, best, o);
            const int j = __shfl_xor_sync(0xffffffffu, bk, o);
            if (e < best || (e == best && j < bk)) {
                best = e;
                bk = j;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            s_best[threadIdx.x >> 5] = best;
            s_bk[threadIdx.x >> 5] = bk;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
                if (s_best[i] < best || (s_best[i] == best && s_bk[i] < bk)) {
                    best = s_best[i];
                    bk = s_bk[i];
                }
            centers[(size_t)l * M + m] = (uint8_t)bk;
        }
    }
}

}  // namespace

// nlist distinct rows of [0, N): Floyd's sampling algorithm over the centre stream of `seed`
// (for j = N - nlist .. N - 1 draw t uniform in [0, j]; take t unless taken, else j).
void pick_distinct_rows(int64_t N, int nlist, uint64_t seed, std::vector<int64_t> &out)
{
    out.resize(nlist);
    for (int i = 0; i < nlist; ++i) {
        const int64_t j = N - nlist + i;
        const int64_t t = scale_index(rng_draw(seed, kStreamCenters, (uint64_t)i) >> 11, (uint64_t)(j + 1));
        bool taken = false;
        for (int q = 0; q < i && !taken; ++q) taken = out[q] == t;
        out[i] = taken ? j : t;
    }
}

int launch_decode_codes(const uint8_t *codes, const float *C, int64_t N, int D, int M, int Ks, float *Xhat,
                        cudaStream_t s)
{
    return launch_decode_rmse(codes, C, nullptr, N, D, M, Ks, Xhat, nullptr, s);
}

int run_ivf_build_codes(const uint8_t *codes, const float *C, int64_t N, int D, int M, int Ks, int nlist, int iters,
                        uint64_t seed, int prec, float *coarse, CoarseBound &b, uint8_t *centers,
                        int64_t *offsets, int64_t *ids, uint8_t *list_codes, Scratch &ws, cudaStream_t s)
{
    const int ds = D / M;
    float *Xhat = ws.get<float>((size_t)N * D);
    float *DT32 = ws.get<float>((size_t)M * Ks * Ks);
    double *DT64 = ws.get<double>((size_t)M * Ks * Ks);
    int *hist = ws.get<int>((size_t)nlist * M * Ks);
    int *queue = ws.get<int>((size_t)nlist * M);
    unsigned *qlen = ws.get<unsigned>(1);
    int64_t *pick_d = ws.get<int64_t>((size_t)nlist);
    int32_t *lst = ws.get<int32_t>((size_t)N);
    if (ws.status) return ws.status;
    {
        const int64_t total = (int64_t)M * Ks * Ks;
        ProfScope ps("sdc_tables", s);
        sdc_tables_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, s>>>(C, M, Ks, ds, DT32,
                                                                                              DT64);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
    }
    PQ_TRY(launch_decode_codes(codes, C, N, D, M, Ks, Xhat, s));
    std::vector<int64_t> pick;
    pick_distinct_rows(N, nlist, seed, pick);
    PQ_TRY_CUDA(cudaMemcpyAsync(pick_d, pick.data(), (size_t)nlist * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    {
        ProfScope ps("gather_codes", s);
        gather_codes_kernel<<<(nlist * M + 255) / 256, 256, 0, s>>>(codes, pick_d, nlist, M, centers);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
    }
    // the host copy of the draws must outlive the asynchronous copy above
    PQ_TRY_CUDA(cudaStreamSynchronize(s));
    for (int t = 0; t < iters; ++t) {
        PQ_TRY(launch_decode_codes(centers, C, nlist, D, M, Ks, coarse, s));
        PQ_TRY(launch_coarse_norms(coarse, nlist, D, b, s));
        PQ_TRY(coarse_assign(Xhat, N, D, coarse, nlist, b, lst, ws, prec, s, ds));
        PQ_TRY_CUDA(cudaMemsetAsync(hist, 0, (size_t)nlist * M * Ks * sizeof(int), s));
        PQ_TRY_CUDA(cudaMemsetAsync(qlen, 0, sizeof(unsigned), s));
        {
            ProfScope ps("center_hist", s);
            center_hist_kernel<<<152 * 8, 256, 0, s>>>(codes, lst, N, M, Ks, hist);
            count_launch();
            PQ_TRY_CUDA(cudaGetLastError());
        }
        {
            ProfScope ps("center_cost", s);
            center_cost_kernel<<<dim3((nlist + kLT - 1) / kLT, M), 256, 0, s>>>(hist, DT32, nlist, M, Ks, centers,
                                                                              queue, qlen);
            count_launch();
            PQ_TRY_CUDA(cudaGetLastError());
        }
        {
            ProfScope ps("center_recheck", s);
            center_recheck_kernel<<<152, 256, 0, s>>>(hist, DT64, M, Ks, queue, qlen, centers);
            count_launch();
            PQ_TRY_CUDA(cudaGetLastError());
        }
    }
    PQ_TRY(launch_decode_codes(centers, C, nlist, D, M, Ks, coarse, s));
    PQ_TRY(launch_coarse_norms(coarse, nlist, D, b, s));
    PQ_TRY(coarse_assign(Xhat, N, D, coarse, nlist, b, lst, ws, prec, s, ds));
    PQ_TRY(bucket_rows(lst, N, nlist, codes, M, offsets, ids, list_codes, ws, s));
    return ws.status;
}

}  // namespace pqgb
