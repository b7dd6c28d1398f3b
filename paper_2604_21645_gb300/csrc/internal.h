// internal.h -- host-side launchers shared between the libpqgb translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

namespace pqgb {

// Stream-ordered scratch owned by one API call (freed, stream-ordered, when
// the call returns).
struct Scratch {
    cudaStream_t s = nullptr;
    std::vector<void *> ptrs;
    int status = 0;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch();
    template <typename T>
    T *get(size_t count, bool zero = false)
    {
        return static_cast<T *>(raw(count * sizeof(T), zero));
    }
    void *raw(size_t bytes, bool zero);
};

// ---- k-means++ seeding (kmeanspp.cu) --------------------------------------
// A chunk of rows [r0, r0 + rows) seeded with its own seed; chunks with more than
// 100*Ks rows are seeded on a with-replacement subsample of 100*Ks of them.
constexpr int kMaxSeedChunks = 512;
struct SeedChunk {
    int64_t r0 = 0, rows = 0;
    int64_t n = 0, sub_off = -1;  // filled in by the launcher
    uint64_t seed = 0;
};
// Ks codewords in each of the M subspaces (width ds) of every chunk; C is [n_chunks][M][Ks][ds].
int launch_kmeanspp_chunks(const float *X, int64_t ld, const SeedChunk *chunks, int n_chunks, int ds, int M, int Ks,
                           float *C, Scratch &ws, int *err, cudaStream_t s, const char *tag);
// The 100*Ks rows that the seeding of N > 100*Ks rows draws (its with-replacement subsample), in
// draw order, gathered into G [100*Ks][D]: seeding G as a whole gives the same codebooks.
int launch_gather_subsample(const float *X, int64_t N, int D, int Ks, uint64_t seed, float *G, cudaStream_t s);
// One chunk: all N rows of X (row stride D).
int launch_kmeanspp(const float *X, int64_t N, int D, int M, int Ks, uint64_t seed, float *C, Scratch &ws, int *err,
                    cudaStream_t s, const char *tag = "kmeanspp");

// ---- centroid update partials (both forms of the Lloyd pass) ------------------
// Per-block member sums of one Lloyd pass, in the exact fixed-point format of
// common.cuh (FixFmt): residual sums as int64 per (block, subspace, codeword,
// dimension), the FP32 sums of the rare residual elements beyond that format, member
// counts, and the format's exponent F per (chunk, subspace).
struct Partials {
    long long *q = nullptr;  // [gx][M][Ks][ds]
    float *o = nullptr;      // [gx][M][Ks][ds]
    int *cnt = nullptr;      // [gx][M][Ks]
    int *F = nullptr;        // [n_chunks][M]
    static size_t bytes(int gx, int M, int Ks, int ds, int n_chunks)
    {
        const size_t e = (size_t)gx * M * Ks * ds;
        return e * 8 + e * 4 + (size_t)gx * M * Ks * 4 + (size_t)n_chunks * M * 4 + 64;
    }
    // lays the four arrays out in `base` (256-byte aligned, Partials::bytes(...) long)
    void carve(void *base, int gx, int M, int Ks, int ds)
    {
        const size_t e = (size_t)gx * M * Ks * ds;
        unsigned char *b = static_cast<unsigned char *>(base);
        q = reinterpret_cast<long long *>(b);
        o = reinterpret_cast<float *>(b + e * 8);
        cnt = reinterpret_cast<int *>(b + e * 12);
        F = reinterpret_cast<int *>(b + e * 12 + (size_t)gx * M * Ks * 4);
    }
    __host__ __device__ bool active() const { return q != nullptr; }
};

#ifdef __CUDACC__
// The update of one codeword element (chunk c, subspace m, codeword k, dimension j) from the
// partial sums of blocks [b0, b1): the int64 sums added exactly, the FP32 sums added with TwoSum
// in block order, the total turned into a float-float value, divided by the member count in
// float-float and added to the codeword with one rounding.  An empty codeword keeps its value.
// Returns the member count.
__device__ __forceinline__ long long finalize_element(const Partials &part, int M, int Ks, int ds, float *C, int c,
                                                      int m, int k, int j, int b0, int b1)
{
    long long n = 0, q = 0;
    float oh = 0.0f, ol = 0.0f;
    for (int b = b0; b < b1; ++b) {
        const size_t e = ((size_t)b * M + m) * Ks + k;
        n += __ldcg(part.cnt + e);
        q += __ldcg(part.q + e * ds + j);
        float s, err;
        two_sum(oh, __ldcg(part.o + e * ds + j), s, err);
        oh = s;
        ol = __fadd_rn(ol, err);
    }
    if (n == 0) return 0;
    const int F = __ldcg(part.F + c * M + m);
    float sh, sl;
    ll_to_ff(q, sh, sl);
    sh = ldexpf(sh, -F);
    sl = ldexpf(sl, -F);
    ff_add(sh, sl, oh, ol, sh, sl);
    float nh, nl, mh, ml;
    ll_to_ff(n, nh, nl);
    ff_div(sh, sl, nh, nl, mh, ml);
    float *cp = C + (size_t)c * M * Ks * ds + ((size_t)m * Ks + k) * ds + j;
    float t, e;
    two_sum(__ldcg(cp), mh, t, e);
    *cp = __fadd_rn(t, __fadd_rn(e, ml));
    return n;
}
#endif

// ---- PQ Lloyd pass, FP32 SIMT form (lloyd_simt.cu) ------------------------
struct PqPass {
    const float *X = nullptr;
    int64_t N = 0;
    int D = 0, M = 0, Ks = 0, ds = 0;
    const float *C = nullptr;      // [M][Ks][ds]
    uint8_t *codes = nullptr;      // [N][M] or null
    Partials part;                 // per-block member sums, or inactive (no update)
    double *sse = nullptr;         // device scalar accumulator or null
    unsigned long long *rechecks = nullptr;
    int gx = 0;                    // blocks per subspace (set by the launcher)
    // Optional chunk table (batched form): grid block b belongs to chunk blk_chunk[b]; chunk c
    // owns rows [chunk_off[c], chunk_off[c+1]), grid blocks [chunk_blk[c], chunk_blk[c+1]) and
    // codebooks C + c*M*Ks*ds.  All null: one chunk, all rows, all blocks.
    const int *blk_chunk = nullptr;
    const int64_t *chunk_off = nullptr;
    const int *chunk_blk = nullptr;
    int n_chunks = 1;
};
int pq_pass_blocks_per_subspace(const PqPass &p);
int launch_pq_pass_f32(PqPass &p, cudaStream_t s);
// Adds the blocks' partials of every (chunk, subspace, codeword) and moves the codeword by
// its members' mean residual; a codeword without members keeps its value (counted in empties).
// counts (optional) [n_chunks][M][Ks] receives the member counts.
int launch_pq_finalize(const Partials &part, int gx, int M, int Ks, int ds, float *C, unsigned long long *empties,
                       cudaStream_t s, int n_chunks = 1, const int *chunk_blk = nullptr, long long *counts = nullptr);
int launch_decode_rmse(const uint8_t *codes, const float *C, const float *X, int64_t N, int D, int M, int Ks,
                       float *Xhat, double *sse, cudaStream_t s);

// ---- PQ Lloyd pass, BF16 tcgen05 form (lloyd_tc.cu) ------------------------
bool tc_pass_supported(int D, int M, int Ks);
int tc_pass_group();  // subspaces per CTA of the tensor-core pass
int pq_pass_tc_blocks(const PqPass &p);
// writes per-CTA residual sums (x - c_code) into p.part; finalise with launch_pq_finalize
int launch_pq_pass_tc(PqPass &p, cudaStream_t s);
// All `iters` Lloyd passes of the batched form (p: chunk table and partial sums set, p.gx its
// blocks) in one persistent cooperative launch: the (block, subspace group) units are shared out
// over the resident CTAs, and after each pass the last unit of a (chunk, group) to finish moves that
// chunk's codebooks (p.C, in place).  sync: persistent_sync_ints(p) zeroed ints (arrival counters,
// ready flags, the unit counter); counts: the member counts of the last update, or null.
int launch_pq_fit_persistent_tc(PqPass &p, int iters, int *sync, long long *counts, cudaStream_t s);
inline size_t persistent_sync_ints(int n_chunks, int M) { return (size_t)n_chunks * (M / 2) * 2 + 1; }

// ---- coarse quantizer and inverted lists (coarse.cu) ----------------------
struct CoarseBound {
    float *half_norm = nullptr;    // [nlist] 0.5*||c||^2
    float *maxes = nullptr;        // [2]: max half norm, max norm
};
int launch_coarse_norms(const float *C, int nlist, int D, CoarseBound &b, cudaStream_t s);
// Nearest coarse centroid of every row (exact: FP32 bound + FP64 re-check).  The FP64
// re-check sums the squared differences in one run over the D dimensions (sub = 0), or as
// per-subspace terms of width `sub` added in subspace order (the symmetric PQ distance of
// two decoded codes, d2_fp64_sub).
int coarse_assign(const float *X, int64_t N, int D, const float *C, int nlist, const CoarseBound &b,
                  int32_t *list_of_row, Scratch &ws, int prec, cudaStream_t s, int sub = 0);
// tensor-core scores (coarse_tc.cu): certified rows written, the rest queued for the FP64 re-check
bool coarse_tc_supported(int D, int nlist);
int launch_coarse_tc(const float *X, int64_t N, int D, const float *C, int nlist, int32_t *list_of_row,
                     int64_t *queue, uint32_t *qmask, unsigned long long *qlen, Scratch &ws, cudaStream_t s);
// Stable bucketing of rows by list: offsets[nlist+1], ids[N] ascending within a list,
// and, if codes != null, list_codes[N][M] in list order.
int bucket_rows(const int32_t *list_of_row, int64_t N, int nlist, const uint8_t *codes, int M, int64_t *offsets,
                int64_t *ids, uint8_t *list_codes, Scratch &ws, cudaStream_t s);
// Coarse centroid update: FP64 sums of each list's rows in ascending row order (computed as
// exact integer sums where those are provably equal).  xrange = [min, max] biased exponent of
// the nonzero elements of X, from launch_x_exponent_range (X is the same for every update).
int launch_x_exponent_range(const float *X, int64_t N, int D, unsigned *xrange, cudaStream_t s);
// The update cuts every list into pieces of up to 2,048 rows (one block each) and then adds each
// list's piece sums: its scratch, for N rows in nlist lists, is allocated once per build.
struct ListMeanScratch {
    int64_t pmax = 0;                       // pieces at most
    int *pbeg = nullptr;                    // [nlist + 1] first piece of every list
    int *piece_list = nullptr;              // [pmax] list of every piece
    unsigned long long *lo = nullptr, *hi = nullptr;  // [pmax][D] 128-bit integer column sums of a piece
    unsigned *neg = nullptr, *emin = nullptr;         // [pmax][D] negative terms, smallest exponent
    float *abs = nullptr;                   // [pmax][D] FP32 sum of magnitudes
};
int list_mean_scratch(int64_t N, int D, int nlist, Scratch &ws, ListMeanScratch &lm);
int launch_list_mean(const float *X, int D, const int64_t *offsets, const int64_t *ids, int nlist,
                     const unsigned *xrange, float *C, const ListMeanScratch &lm, cudaStream_t s);

// ---- code-space coarse quantizer (codes_ivf.cu) ----------------------------
// Centre codes [nlist][M] by k-means over the PQ codes (symmetric distance), the decoded
// centres in `coarse` [nlist][D] with their bounds in b, and the CSR lists of all rows.
int run_ivf_build_codes(const uint8_t *codes, const float *C, int64_t N, int D, int M, int Ks, int nlist, int iters,
                        uint64_t seed, int prec, float *coarse, CoarseBound &b, uint8_t *centers,
                        int64_t *offsets, int64_t *ids, uint8_t *list_codes, Scratch &ws, cudaStream_t s);
// Xhat [N][D] = the codewords the codes select
int launch_decode_codes(const uint8_t *codes, const float *C, int64_t N, int D, int M, int Ks, float *Xhat,
                        cudaStream_t s);

// ---- growing an index (ivf_merge.cu) ---------------------------------------
// Merged CSR lists: list l = list l of set a, then list l of set b with ids + b_shift.
int launch_merge_lists(const int64_t *a_off, const int64_t *a_ids, const uint8_t *a_codes, int64_t a_n,
                       const int64_t *b_off, const int64_t *b_ids, const uint8_t *b_codes, int64_t b_n,
                       int64_t b_shift, int nlist, int M, int64_t *out_off, int64_t *out_ids, uint8_t *out_codes,
                       cudaStream_t s);

// ---- optimized PQ (opq.cu) -------------------------------------------------
// Y [N][D] = X [N][D] R [D][D] (FP32, every output summed in k order)
int launch_rotate(const float *X, int64_t N, int D, const float *R, float *Y, cudaStream_t s);
// R_out [D][D] (device) = the orthogonal R minimising ||X R - Y||_F; synchronizes the stream
int run_procrustes(const float *X, const float *Y, int64_t N, int D, float *R_out, Scratch &ws, cudaStream_t s);

// ---- chunked divide and conquer (chunked.cu) -------------------------------
// weighted: each pooled codeword carries its member count in its chunk's last update, and the
// global model is the weighted fit of the pooled codewords
int run_pq_fit_chunked(const float *X, const int64_t *off, int n_chunks, int D, int M, int Ks, int iters,
                       uint64_t seed, int prec, float *global_cb, uint8_t *codes, double *rmse, cudaStream_t s,
                       bool weighted = false);

// ---- query path (ivf_search.cu) --------------------------------------------
struct SearchArgs {
    const float *Q = nullptr;
    int64_t nq = 0;
    int D = 0, M = 0, Ks = 0, nlist = 0, nprobe = 0, k = 0;
    const float *coarse = nullptr;
    const CoarseBound *cb = nullptr;
    int probe_sub = 0;             // FP64 probe re-rank: 0 = one run over D, else per-subspace terms
    const int64_t *offsets = nullptr;
    const int64_t *ids = nullptr;
    const uint8_t *list_codes = nullptr;
    const float *codebooks = nullptr;
    int64_t *out_ids = nullptr;
    float *out_d = nullptr;
};
int run_search(const SearchArgs &a, Scratch &ws, cudaStream_t s);

// ---- soft-assignment PQ loss and gradients (softpq.cu) --------------------
bool softpq_supported(int D, int M);
int run_softpq_forward(const float *X, int64_t N, int D, int M, int Ks, const float *C, float tau, float *loss,
                       cudaStream_t s);
int run_softpq_backward(const float *X, int64_t N, int D, int M, int Ks, const float *C, float tau,
                        const float *grad_loss, float *dC, float *dX, cudaStream_t s);

// ---- autotuner of the batched pass (chunked.cu) --------------------------
int run_pq_tune_chunked(const float *X, const int64_t *off, int n_chunks, int D, int M, int Ks, int prec,
                        int *best_per, float *best_ms, cudaStream_t s);
void clear_tuning();

}  // namespace pqgb
