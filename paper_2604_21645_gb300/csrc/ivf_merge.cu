// ivf_merge.cu -- growing an inverted index without rebuilding it (Sec. 3.1: Rii's
// add and merge of new codes, which the paper uses to build its index in parallel
// chunks).  Two CSR list sets over the same coarse quantizer become one: list l of
// the result is list l of the first set followed by list l of the second, whose ids
// are shifted past the first set's rows.  Ids stay ascending inside every list, so
// the result is the one a single build over the concatenated rows gives with the
// same coarse quantizer.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

// list of CSR position p: the l with off[l] <= p < off[l + 1] (binary search)
__device__ __forceinline__ int list_of_pos(const int64_t *__restrict__ off, int nlist, int64_t p)
{
    int lo = 0, hi = nlist;  // off[lo] <= p < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= p) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void merge_offsets_kernel(const int64_t *__restrict__ a_off, const int64_t *__restrict__ b_off, int nlist,
                                     int64_t *__restrict__ out_off)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l <= nlist) out_off[l] = a_off[l] + b_off[l];
}

// every entry of set `src` moves to its list's slot in the merged lists: entry p of list l lands
// at out_off[l] + (p - src_off[l]) + before[l], where before[l] is the length of list l in the
// set that precedes it there (0 for the first set, the first set's list length for the second)
__global__ void merge_scatter_kernel(const int64_t *__restrict__ src_off, const int64_t *__restrict__ src_ids,
                                     const uint8_t *__restrict__ src_codes, int64_t n, int nlist, int M,
                                     const int64_t *__restrict__ out_off, const int64_t *__restrict__ other_off,
                                     bool second, int64_t id_shift, int64_t *__restrict__ out_ids,
                                     uint8_t *__restrict__ out_codes)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int l = list_of_pos(src_off, nlist, p);
        const int64_t before = second ? other_off[l + 1] - other_off[l] : 0;
        const int64_t q = out_off[l] + before + (p - src_off[l]);
        out_ids[q] = src_ids[p] + id_shift;
        for (int m = 0; m < M; ++m) out_codes[q * M + m] = src_codes[p * M + m];
    }
}

}  // namespace

int launch_merge_lists(const int64_t *a_off, const int64_t *a_ids, const uint8_t *a_codes, int64_t a_n,
                       const int64_t *b_off, const int64_t *b_ids, const uint8_t *b_codes, int64_t b_n,
                       int64_t b_shift, int nlist, int M, int64_t *out_off, int64_t *out_ids, uint8_t *out_codes,
                       cudaStream_t s)
{
    ProfScope ps("merge_lists", s);
    merge_offsets_kernel<<<(nlist + 256) / 256, 256, 0, s>>>(a_off, b_off, nlist, out_off);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    if (a_n > 0) {
        merge_scatter_kernel<<<(unsigned)std::min<int64_t>((a_n + 255) / 256, 152 * 16), 256, 0, s>>>(
            a_off, a_ids, a_codes, a_n, nlist, M, out_off, b_off, false, 0, out_ids, out_codes);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
    }
    if (b_n > 0) {
        merge_scatter_kernel<<<(unsigned)std::min<int64_t>((b_n + 255) / 256, 152 * 16), 256, 0, s>>>(
            b_off, b_ids, b_codes, b_n, nlist, M, out_off, a_off, true, b_shift, out_ids, out_codes);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
    }
    return PQ_OK;
}

}  // namespace pqgb
