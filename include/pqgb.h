/*
 * pqgb.h -- C ABI of libpqgb.so: product quantization (PQ) fit / encode /
 * decode-RMSE and an inverted-file index with asymmetric-distance (IVF-ADC)
 * k-nearest-neighbour search, on one sm_103a GPU.
 *
 * The operations follow the paper's statement of the method:
 *   - PQ fit (Sec. 2.1): the D dimensions are split into M contiguous
 *     subspaces of Ds = D/M dimensions; each subspace is clustered by k-means
 *     into Ks centroids, the codebooks.
 *   - PQ encode (Sec. 2.1): every row's sub-vector in subspace m is replaced
 *     by the index of its nearest centroid; a row becomes M codes.
 *   - Decode and RMSE (Sec. 2.1, Sec. 3): the reconstruction is the
 *     concatenation of the selected centroids; accuracy is the root mean
 *     squared reconstruction error.
 *   - Inverted index and query (Sec. 2.2, Sec. 3.1): ids are stored per
 *     list over the codes; a query returns its k nearest neighbours, scored
 *     with the PQ distance table.
 *   - Chunked divide and conquer (Sec. 3): per-chunk fits, codewords pooled
 *     into a centroid dataset, a global refit, then a global encode + RMSE.
 *
 * Conventions shared by every call:
 *   - Layouts are row-major and little-endian.  X is N x D float32; codebooks
 *     are M x Ks x Ds float32 (subspace-major); codes are N x M uint8.
 *   - Pointers are DEVICE pointers owned by the caller unless stated
 *     otherwise.  The library never frees caller memory.  Scratch space is
 *     taken with stream-ordered cudaMallocAsync on the caller's stream and
 *     returned before the call's work completes.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously; calls return after enqueue
 *     unless documented to synchronize.
 *   - Return value: PQ_OK or a negative status.  Argument errors are found
 *     before anything is enqueued.  Asynchronous device failures (including
 *     a device-side bounded wait that ran out, PQ_ETIMEOUT) are recorded and
 *     returned by pq_sync_status() or by the next synchronizing call.
 *     pq_last_error() gives a message for the last failure on this thread.
 *   - Distances are squared Euclidean.  Argmin ties go to the lowest index;
 *     query results are ordered by (distance, id).
 *   - Codes are exact: every nearest-centroid decision is either proven by an
 *     FP32 (or BF16) error bound or re-decided in FP64 by direct differences.
 */
#ifndef PQGB_H
#define PQGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PQ_OK = 0,
    PQ_EINVAL = -1,   /* bad argument (shape, null pointer, alignment)      */
    PQ_ENOMEM = -2,   /* device scratch or host allocation failed           */
    PQ_ECUDA = -3,    /* a CUDA runtime call failed                         */
    PQ_ETIMEOUT = -4, /* a device-side bounded wait ran out                 */
    PQ_ENOTSUP = -5,  /* valid but unsupported shape/precision combination  */
    PQ_EINTERNAL = -6 /* a device-side consistency check failed             */
};

/* Arithmetic of the distance contraction used to find nearest centroids. */
enum {
    PQ_PREC_FP32 = 0, /* FP32 FFMA on CUDA cores                               */
    PQ_PREC_BF16 = 1  /* BF16 tcgen05 tensor-core GEMM, FP32 accumulation,
                         exact FP32 re-rank of the candidates                  */
};

#define PQ_STATS_MAX_ITERS 64

/* Diagnostics of one pq_fit / pq_encode call (host struct, optional). */
typedef struct pq_stats {
    int32_t iters;            /* Lloyd iterations run                          */
    int32_t reserved;
    int64_t fp64_rechecks;    /* (row, subspace) decisions re-taken in FP64     */
    int64_t empty_clusters;   /* codewords left without members, all iterations */
    int64_t kernel_launches;  /* kernels this call launched                     */
    double sse[PQ_STATS_MAX_ITERS]; /* total squared error of each iteration's
                                       assignment (before its update)           */
} pq_stats;

/*
 * pq_fit -- PQ codebooks by per-subspace k-means (Sec. 2.1).
 *   X               [N][D] float32, 16-byte aligned, N >= Ks.
 *   D, M            D % M == 0, Ds = D/M <= 32.
 *   Ks              1 <= Ks <= 256.
 *   iters           Lloyd iterations, 0 <= iters <= PQ_STATS_MAX_ITERS.
 *   seed            k-means++ seed (SplitMix64 streams; when N > 100*Ks the
 *                   seeding runs on a with-replacement subsample of 100*Ks rows).
 *   prec            PQ_PREC_FP32 or PQ_PREC_BF16.
 *   init_codebooks  [M][Ks][Ds] or NULL (NULL = k-means++ seeding).
 *   codebooks       [M][Ks][Ds] output (may alias init_codebooks).
 *   stats           host pq_stats or NULL; non-NULL makes the call synchronize.
 * Each iteration assigns every (row, subspace) to its nearest codeword, then
 * replaces every codeword by the mean of its members; a codeword without
 * members keeps its value.  The member sums are exact integer sums of the
 * residuals x - c in a fixed-point format scaled to the codebook (each element's
 * quantisation error below 2^-(qb+1) of twice the largest codeword norm about
 * the codeword mean, qb = min(30, 61 - 2b), b = bit length of the rows one block
 * or CTA handles), plus
 * FP32 sums of the rare residuals beyond that format; blocks are combined in
 * int64 and the mean is taken in float-float (compensated FP32) arithmetic, so
 * no FP64 arithmetic is involved and the result does not depend on the order of
 * the additions.
 */
int pq_fit(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, int32_t iters, uint64_t seed,
           int32_t prec, const float *init_codebooks, float *codebooks, pq_stats *stats, void *stream);

/*
 * pq_init_kmeanspp -- only the k-means++ seeding step of pq_fit.
 *   Same arguments as pq_fit; writes codebooks [M][Ks][Ds].
 */
int pq_init_kmeanspp(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, uint64_t seed, float *codebooks,
                     void *stream);

/*
 * pq_fit_encode_host -- pq_fit followed by pq_encode of the same rows, for rows
 * that live in host memory (Sec. 2.1; the same results as the two device calls).
 *   X_host          [N][D] float32 in page-locked host memory (cudaHostAlloc or
 *                   cudaHostRegister), 16-byte aligned.  When N > 100*Ks the
 *                   seeding's subsample rows are gathered from it directly and
 *                   seeded while the whole matrix is copied to device scratch on
 *                   a second stream; the Lloyd passes wait only for that copy.
 *   codebooks_host  [M][Ks][Ds] float32 host output.
 *   codes_host      [N][M] uint8 host output, or NULL (codes not returned).
 *   iters, seed, prec as pq_fit (no init_codebooks, no stats).
 *   stream          every step is ordered on it: the outputs are complete when
 *                   the stream passes the call's work.  Page-locked outputs are
 *                   written asynchronously; the host buffers must stay valid
 *                   until then.
 * Returns PQ_EINVAL if X_host is not page-locked host memory of this device's
 * context, PQ_ENOMEM if the device scratch (about N*D*4 + N*M bytes) cannot be
 * allocated.
 */
int pq_fit_encode_host(const float *X_host, int64_t N, int32_t D, int32_t M, int32_t Ks, int32_t iters,
                       uint64_t seed, int32_t prec, float *codebooks_host, uint8_t *codes_host, void *stream);

/*
 * pq_encode -- PQ codes (Sec. 2.1).
 *   codes   [N][M] uint8 output.
 *   sse     NULL, or a device double that receives the total squared
 *           reconstruction error sum_{n,d} (x - xhat)^2 (overwritten).
 *   stats   host pq_stats or NULL (non-NULL synchronizes).
 */
int pq_encode(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, const float *codebooks, int32_t prec,
              uint8_t *codes, double *sse, pq_stats *stats, void *stream);

/*
 * pq_decode_rmse -- reconstruction and its RMSE (Sec. 2.1, Sec. 3).
 *   codes [N][M] uint8, codebooks [M][Ks][Ds].
 *   X     [N][D] or NULL; if non-NULL, *rmse (host) receives
 *         sqrt(sum (x - xhat)^2 / (N*D)) and the call synchronizes.
 *   Xhat  [N][D] output or NULL.
 * At least one of X (with rmse) and Xhat must be given.
 */
int pq_decode_rmse(const uint8_t *codes, const float *codebooks, const float *X, int64_t N, int32_t D, int32_t M,
                   int32_t Ks, float *Xhat, double *rmse, void *stream);

/*
 * pq_lloyd_noalloc -- the Lloyd iterations of pq_fit (FP32 form) from given
 * initial codebooks, without allocating any device memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate while
 * they run (a process whose GPU memory is reserved up front by its own
 * allocator, or a latency-bound loop where cudaMalloc could block or fail).
 *   X               [N][D] float32, 16-byte aligned, N >= Ks >= 1, Ks <= 256.
 *   init_codebooks  [M][Ks][Ds] (required: no k-means++ seeding here).
 *   codebooks       [M][Ks][Ds] output (may alias init_codebooks).
 * Results equal pq_fit(..., PQ_PREC_FP32, init_codebooks, ...) up to the FP64
 * summation order of the member sums.  Scratch is a fixed 8 MiB array inside
 * the library that every GPU loading it keeps until exit; shapes needing more
 * than that for one block per subspace, M*Ks*(8*D/M + 4) > 8 MiB, are rejected
 * with PQ_EINVAL, and subspace widths other than 1, 2, 4, 8, 16, 32 with
 * PQ_ENOTSUP, before anything is enqueued.  The first call on each device
 * looks up the array's device address and caches it (make that first call
 * before any stream capture; the cache assumes the device's primary context is
 * not reset while the library is loaded).  All calls share the array: calls
 * whose work overlaps on the GPU (other streams, other host threads) race and
 * must be serialized by the caller.
 */
int pq_lloyd_noalloc(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, int32_t iters,
                     const float *init_codebooks, float *codebooks, void *stream);

/*
 * pq_fit_chunked -- the paper's divide-and-conquer PQ (Sec. 3, "Methodology").
 *   X              [N][D] float32 rows, 16-byte aligned.
 *   chunk_offsets  HOST array [n_chunks + 1]: chunk c is rows
 *                  [chunk_offsets[c], chunk_offsets[c+1]); chunk_offsets[0] = 0,
 *                  every chunk has at least Ks rows, N = chunk_offsets[n_chunks],
 *                  1 <= n_chunks <= 512.
 *   codebooks      [M][Ks][Ds] output: the global model.
 *   codes          [N][M] output: every row encoded with the global model.
 *   rmse           host double or NULL; non-NULL makes the call synchronize and
 *                  receive sqrt(sum (x - xhat)^2 / (N*D)) of the global model.
 * Chunk c gets a PQ fit (k-means++ seeding from draw c of the chunk stream of
 * `seed`, then `iters` Lloyd iterations); the codewords of all chunks form the
 * centroid dataset (row c*Ks + k = concatenation over m of codeword k of
 * subspace m of chunk c), on which the global PQ is fitted with `seed`.  All
 * chunks are fitted together: one launch seeds every (chunk, subspace) pair, and
 * the Lloyd iterations of every (chunk, subspace group) run in one persistent
 * cooperative launch (BF16 form; its units of rows are shared out over the
 * resident CTAs, and after each pass the last unit of a (chunk, group) to finish
 * moves that chunk's codebooks and lets the group's next pass start; the FP32
 * form runs one launch per iteration).  The unit size is the one pq_tune_chunked
 * chose for this shape, else a default.  With rmse == NULL the call never
 * synchronizes and can be captured in a CUDA graph.
 */
int pq_fit_chunked(const float *X, const int64_t *chunk_offsets, int32_t n_chunks, int32_t D, int32_t M, int32_t Ks,
                   int32_t iters, uint64_t seed, int32_t prec, float *codebooks, uint8_t *codes, double *rmse,
                   void *stream);

/*
 * pq_fit_chunked_weighted -- pq_fit_chunked with a weighted centroid dataset
 * (a variant of Sec. 3's combine step).  Arguments and outputs as pq_fit_chunked.
 * Pooled codeword k of subspace m of chunk c carries the weight w = its member
 * count in the chunk's last Lloyd update (the number of the chunk's rows whose
 * mean it is; 1 when iters = 0), so a weighted mean of pooled codewords is a
 * mean of the rows behind them.  The global model is seeded by k-means++ on the
 * pooled codewords as they are, then `iters` rounds of exact nearest-codeword
 * assignment and weighted update c = sum w x / sum w (float-float sums in pooled
 * row order, one rounding; a codeword whose members weigh 0 keeps its value).
 */
int pq_fit_chunked_weighted(const float *X, const int64_t *chunk_offsets, int32_t n_chunks, int32_t D, int32_t M,
                            int32_t Ks, int32_t iters, uint64_t seed, int32_t prec, float *codebooks, uint8_t *codes,
                            double *rmse, void *stream);

/*
 * Optimized PQ (Sec. 2.1 names it; Sec. 3.1: NanoPQ's "PQ and Optimized PQ"): an
 * orthogonal rotation R of the rows learned jointly with the PQ codebooks of the rotated
 * rows, by alternating minimisation of ||X R - decode(encode(X R))||^2.
 * opq_fit -- R = I and codebooks = pq_fit(X, seed, pq_iters); then `outer` times: encode and
 *   decode X R, set R to the Procrustes solution of (X, reconstruction), refit the codebooks
 *   on X R from the previous ones (pq_iters Lloyd iterations).  Outputs R [D][D] (row-major;
 *   a row x maps to x R) and codebooks [M][Ks][Ds] of X R.  Synchronizes.  Scratch: about
 *   2*N*D*4 + N*M bytes.  Codes, indexes and queries then use rotated rows (opq_rotate).
 * opq_rotate -- Y [N][D] = X R in FP32 (every output summed in the same k order); Y must not
 *   alias X.
 * opq_procrustes -- R = U V^T for X^T Y = U S V^T, the orthogonal R minimising ||X R - Y||_F:
 *   X^T Y on the device (FP32 products over 1,024-row ranges, added in float-float), its SVD
 *   on the host in FP64 (one-sided Jacobi).  Synchronizes.
 * D <= 1024 for all three.
 */
int opq_fit(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, int32_t outer, int32_t pq_iters,
            uint64_t seed, int32_t prec, float *R, float *codebooks, void *stream);
int opq_rotate(const float *X, int64_t N, int32_t D, const float *R, float *Y, void *stream);
int opq_procrustes(const float *X, const float *Y, int64_t N, int32_t D, float *R, void *stream);

/*
 * softpq_forward / softpq_backward -- soft-assignment reconstruction loss for
 * codebook refinement, the differentiable relaxation of the hard assignment of
 * Sec. 2.1:
 *     p_k = softmax_k(-||x_m - c_{m,k}||^2 / tau),  xh_m = sum_k p_k c_{m,k},
 *     L   = (1/N) sum_n sum_m ||xh_m - x_m||^2.
 *   X          [N][D] float32 rows (device, 16-byte aligned), N >= 0.
 *   codebooks  [M][Ks][Ds] float32 (device), 1 <= Ks <= 256, Ds = D/M in {4, 8, 16}.
 *   tau        temperature, > 0.
 *   loss       device float [1] receiving L (0 for N = 0).
 *   grad_loss  device float [1] holding dOut/dL (the upstream gradient), or NULL for 1.
 *   dcodebooks [M][Ks][Ds] device output dOut/dC (overwritten).
 *   dX         [N][D] device output dOut/dX (overwritten, 16-byte aligned), or NULL.
 * FP32 arithmetic; the backward pass recomputes the soft assignments from X and
 * the codebooks (nothing is carried over from the forward call).  Neither call
 * synchronizes.  Errors: PQ_EINVAL for bad shapes, pointers or tau; PQ_ENOTSUP
 * for an unsupported Ds.
 */
int softpq_forward(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, const float *codebooks, float tau,
                   float *loss, void *stream);
int softpq_backward(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, const float *codebooks, float tau,
                    const float *grad_loss, float *dcodebooks, float *dX, void *stream);

/*
 * pq_tune_chunked -- autotuner of the batched Lloyd passes of pq_fit_chunked.
 *   Same X, chunk_offsets (HOST array), n_chunks, D, M, Ks and prec rules as
 *   pq_fit_chunked.  Seeds every chunk, then, for each candidate number of work
 *   units per subspace group (0.5x to 8x the default, shared out over the chunks
 *   in proportion to their rows, so that a unit is a run of ceil(tiles / units)
 *   128-row tiles of one chunk), times the batched passes: BF16, the persistent
 *   launch of three passes after a one-pass warm-up; FP32, the mean of three
 *   passes after a warm-up (CUDA events on `stream`).  The fastest is kept in a
 *   process-wide cache keyed by the shape (n_chunks, N, D, M, Ks, prec, SM
 *   count, chunk offsets); later pq_fit_chunked calls of that shape use it.
 *   Synchronizes `stream`.
 *   ctas     receives the chosen units per subspace group (nullable).
 *   pass_ms  receives its measured time per pass in milliseconds (nullable).
 * pq_tune_clear forgets every tuned shape.
 */
int pq_tune_chunked(const float *X, const int64_t *chunk_offsets, int32_t n_chunks, int32_t D, int32_t M, int32_t Ks,
                    int32_t prec, int32_t *ctas, float *pass_ms, void *stream);
int pq_tune_clear(void);

/* Opaque inverted-file index, allocated by ivf_build and owned by the library until ivf_free. */
typedef struct ivf_index ivf_index;

/*
 * ivf_build -- inverted lists over PQ codes (Sec. 2.2, Sec. 3.1).
 *   X      [N][D] float32 rows; codes [N][M] their PQ codes.
 *   nlist  coarse lists, 1 <= nlist <= N; the coarse quantizer is k-means on
 *          the raw rows (k-means++ seeding from `seed`, `iters` Lloyd steps).
 *   out    receives the new index (device-resident lists: ids ascending
 *          within a list).  The call synchronizes once to size the lists.
 */
int ivf_build(const float *X, const uint8_t *codes, int64_t N, int32_t D, int32_t M, int32_t nlist, int32_t iters,
              uint64_t seed, int32_t prec, ivf_index **out, void *stream);

/*
 * ivf_build_codes -- a code-space inverted index, Rii's reading of the index
 * (Sec. 3.1: an IVFPQ-style index that Rii builds from the PQ codes, Sec. 2.2:
 * the codes are hashed into lists).  The coarse centres are PQ codes:
 *   codes      [N][M] uint8 PQ codes of the rows (device); no raw rows needed.
 *   codebooks  [M][Ks][Ds] the codebooks of those codes (copied into the index).
 *   nlist      1 <= nlist <= min(N, 16384) lists; D = M*Ds <= 256.
 * Centres start as nlist distinct rows drawn by Floyd's algorithm from the
 * centre stream (0xFFFFFFFD) of `seed`, then `iters` rounds of k-means over the
 * codes: each row to its nearest centre by the symmetric distance
 * SDC(a, b) = sum_m ||c_{m,a_m} - c_{m,b_m}||^2 (ties to the lower list), and
 * each centre code, subspace by subspace, to the code k minimising the sum over
 * members of ||c_{m,k} - c_{m,a_m}||^2 (ties to the lower k; a list without
 * members keeps its centre).  Every decision is exact (FP32/BF16 bound, FP64
 * re-check in the reference's order).  ivf_search then probes the lists whose
 * centre codes have the lowest ADC distance to the query (sum over m of the
 * query's table entries), and scans them as for a raw-space index.  The call
 * synchronizes once.  Scratch: about N*D*4 bytes.
 */
int ivf_build_codes(const uint8_t *codes, const float *codebooks, int64_t N, int32_t D, int32_t M, int32_t Ks,
                    int32_t nlist, int32_t iters, uint64_t seed, int32_t prec, ivf_index **out, void *stream);

/*
 * Growing an index without rebuilding it (Sec. 3.1: Rii adds and merges new
 * codes; the paper builds its index in parallel chunks this way).  Lists keep
 * ids ascending, so the result equals the lists a single build over all rows
 * gives with the same coarse quantizer.
 * ivf_clone_empty -- a new index (caller frees it with ivf_free) with src's
 *   coarse quantizer (centroids or centre codes and codebooks) and no rows.
 * ivf_add -- appends n rows, ids N .. N+n-1, to the lists of their nearest
 *   coarse centre (exact decisions, as in the build).  X [n][D] (16-byte
 *   aligned) is required for a raw-space index and ignored (may be NULL) for a
 *   code-space one, which decides from the codes [n][M].  Synchronizes.
 * ivf_merge -- appends every row of src to dst (ids shifted by dst's row
 *   count); both must have the same kind, D, M, nlist and bit-identical coarse
 *   quantizers (PQ_EINVAL otherwise).  src is unchanged.  Synchronizes.
 */
int ivf_clone_empty(const ivf_index *src, ivf_index **out);
int ivf_add(ivf_index *index, const float *X, const uint8_t *codes, int64_t n, int32_t prec, void *stream);
int ivf_merge(ivf_index *dst, const ivf_index *src, void *stream);

/*
 * ivf_search -- k nearest neighbours by ADC over the probed lists (Sec. 2.2).
 *   codebooks [M][Ks][Ds] (the codebooks the stored codes were made with).
 *   Q         [nq][D] float32 queries.
 *   nprobe    1 <= nprobe <= nlist lists probed (nearest coarse centroids).
 *   k         1 <= k <= 1024 results per query.
 *   ids       [nq][k] int64 output, dists [nq][k] float32 output, ordered by
 *             (ADC distance, id); missing results are id -1, distance +inf.
 */
int ivf_search(const ivf_index *index, const float *codebooks, int32_t Ks, const float *Q, int64_t nq,
               int32_t nprobe, int32_t k, int64_t *ids, float *dists, void *stream);

/* Index accessors: copies of the device-resident parts (device destinations). */
int ivf_get_info(const ivf_index *index, int64_t *N, int32_t *D, int32_t *M, int32_t *nlist);
int ivf_copy_coarse(const ivf_index *index, float *coarse /* [nlist][D] */, void *stream);
int ivf_copy_lists(const ivf_index *index, int64_t *offsets /* [nlist+1] */, int64_t *ids /* [N] */,
                   uint8_t *list_codes /* [N][M] */, void *stream);
/* centre codes [nlist][M] of a code-space index (PQ_EINVAL for a raw-space one) */
int ivf_copy_centers(const ivf_index *index, uint8_t *centers, void *stream);
void ivf_free(ivf_index *index);

/* Synchronize `stream` and return (and clear) any recorded device failure. */
int pq_sync_status(void *stream);
/* Message of the last failure on the calling thread ("" if none). */
const char *pq_last_error(void);
/* Kernels launched by this library since load (a monotone counter). */
int64_t pq_launch_count(void);

/*
 * Failure injection for tests of the failure handling (no counterpart in the
 * paper).  Process-wide settings; they exercise error paths without faulting
 * or hanging the GPU.
 * pq_test_set_spin_limit -- poll budget of the waits on other blocks: the
 *   k-means++ seeding's (its group barrier and its per-round sum polls) and the
 *   persistent batched fit's (a unit's wait for the previous pass of its chunk
 *   and subspace group), normally 2^22 polls.  A small budget makes a wait run
 *   out: the block records PQ_ETIMEOUT in the device error word and returns (no
 *   bulk copies or MMAs of its own are in flight at these waits), the other
 *   blocks' waits give up on seeing the error word, and the call's later kernels
 *   finish or give up the same way; pq_sync_status then returns PQ_ETIMEOUT and
 *   clears the word.  0 restores the default.
 * pq_test_fail_alloc_after -- the (n+1)-th scratch allocation from now fails
 *   as if the device were out of memory: the call returns PQ_ENOMEM at that
 *   point, releasing the scratch it already took.  n < 0 turns this off.
 */
int pq_test_set_spin_limit(uint32_t polls);
int pq_test_fail_alloc_after(int32_t n);

/*
 * Per-kernel timing for measurement (no counterpart in the paper).
 * pq_profile_enable(1) clears old records and starts recording a CUDA event
 * pair around every kernel launch on the launch's own stream; (0) stops.
 * pq_profile_collect synchronizes the device and returns, for kernel `name`,
 * the number of recorded launches and their summed device time in ms.
 * pq_profile_names writes the comma-separated recorded names into buf
 * (PQ_EINVAL if it does not fit).
 */
int pq_profile_enable(int on);
int pq_profile_collect(const char *name, int64_t *count, double *total_ms);
int pq_profile_names(char *buf, int len);

#ifdef __cplusplus
}
#endif

#endif /* PQGB_H */
