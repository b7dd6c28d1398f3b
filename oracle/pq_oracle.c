/*
 * pq_oracle.c -- plain, slow FP64 CPU oracle for product quantization (PQ)
 * and the inverted-index (IVF-ADC) query path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load or call this library.  It shares no
 * code, header, table or helper with the CUDA path; both sides read the same
 * seeded inputs and nothing else.
 *
 * What is computed, and where it comes from:
 *   - PQ fit: split D dims into M contiguous subspaces, k-means with Ks
 *     centroids in each (the codebooks); encode: each row's sub-vector is
 *     replaced by the index of its nearest codeword, M codes per row; decode:
 *     concatenated codewords.  (Sec. 2.1, "Product Quantization")
 *   - Accuracy: root mean squared reconstruction error.  (Sec. 2.1, last
 *     paragraph; Sec. 3)
 *   - Inverted index: ids stored per list over the codes, k-nearest query.
 *     (Sec. 2.2; Rii as an IVFPQ-style index, Sec. 3.1)
 *   - Row-wise chunks, local fits, codewords pooled into a centroid dataset,
 *     global PQ refit, re-encode and RMSE.  (Sec. 3, "Methodology")
 * The paper prints no pseudo-code or equations; where it is silent the
 * readings used here are:
 *   - distances are squared Euclidean, computed as direct differences in
 *     FP64 in dimension order; argmin ties go to the lowest index;
 *   - k-means init is k-means++ (D^2 sampling) driven by SplitMix64, on a
 *     with-replacement subsample of 100*Ks rows when N > 100*Ks; the D^2
 *     sampling weights are FP32 squared distances quantised to integers (see
 *     orc_kmeanspp_slice) so that the draw is reproducible bit for bit;
 *   - Lloyd runs a fixed number of iterations, the new centroid is the FP64
 *     mean of its members rounded to float32, an empty cluster keeps its
 *     previous centroid;
 *   - RMSE is normalised per element: sqrt(sum (x - xhat)^2 / (N*D));
 *   - the coarse quantizer is k-means on the raw vectors; the PQ codes are
 *     not residuals, so one distance table per query serves every list;
 *   - query results are ordered by (ADC distance, id); missing results are
 *     id -1 and distance +inf;
 *   - chunk combine pools the codewords (not data rows), unweighted;
 *   - the soft-assignment refinement loss is the mean over rows of the
 *     squared reconstruction error with softmax(-d/tau) weights.
 *
 * Build: cc -O2 -std=c11 -fopenmp -ffp-contract=off -fPIC -shared.
 * -ffp-contract=off matters: the FP32 k-means++ weights must round exactly
 * as written (no fused multiply-add), on x86-64 and on aarch64 alike.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* Stream ids of the counter-based generator. */
#define ORC_STREAM_SUBSAMPLE 0xFFFFFFFFull
#define ORC_STREAM_CHUNK 0xFFFFFFFEull

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number     */
/* generators", OOPSLA 2014).  The state advances by the golden-ratio        */
/* constant and each output is the state passed through the finaliser.      */
/* ------------------------------------------------------------------------ */
static const uint64_t SM64_GAMMA = 0x9E3779B97F4A7C15ull;

static uint64_t sm64_finalise(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Output number i (0-based) of a SplitMix64 generator seeded with `seed`. */
uint64_t orc_sm64(uint64_t seed, uint64_t i)
{
    return sm64_finalise(seed + (i + 1) * SM64_GAMMA);
}

/* Draw number i of stream `stream`: the stream's generator is seeded with
 * output number `stream` of the generator seeded with `seed`. */
uint64_t orc_draw(uint64_t seed, uint64_t stream, uint64_t i)
{
    return orc_sm64(orc_sm64(seed, stream), i);
}

/* floor(r53 * n / 2^53) for a 53-bit r53: an index uniform in [0, n). */
int64_t orc_scale53(uint64_t r53, int64_t n)
{
    unsigned __int128 p = (unsigned __int128)r53 * (unsigned __int128)(uint64_t)n;
    return (int64_t)(p >> 53);
}

/* ------------------------------------------------------------------------ */
/* k-means++ seeding of one subspace.                                       */
/* ------------------------------------------------------------------------ */

/* FP32 squared distance, dimension order, each product and sum rounded. */
static float d2_f32(const float *x, const float *c, int ds)
{
    float acc = 0.0f;
    for (int j = 0; j < ds; ++j) {
        float t = x[j] - c[j];
        float sq = t * t;
        acc = acc + sq;
    }
    return acc;
}

static int ceil_log2_i64(int64_t n)
{
    int l = 0;
    while (((int64_t)1 << l) < n) ++l;
    return l;
}

/*
 * D^2 sampling of ks seeds from the n rows rows[0..n) of the column slice
 * [col0, col0+ds) of X (row stride ld floats).  Writes C[ks][ds].
 *
 * Round 0 picks floor(u*n).  Afterwards each point's weight is its FP32
 * squared distance to the nearest seed so far, quantised once per subspace
 * to an integer: w_i = floor(D2_i * 2^sh) with sh = 62 - ceil(log2 n) - E,
 * where 2^(E-1) <= max_i D2_i < 2^E after round 0.  D2 only shrinks, so the
 * weights stay below 2^(62-ceil(log2 n)) and their sum below 2^62.  With
 * W = sum w_i and r the 53-bit draw, the pick is the smallest i whose
 * inclusive prefix sum exceeds floor(r*W/2^53); points with zero weight are
 * never picked.  If every weight is zero the pick is uniform.
 */
void orc_kmeanspp_slice(const float *X, int64_t ld, int col0, int ds, const int64_t *rows, int64_t n,
                        int ks, uint64_t seed, uint64_t stream, float *C)
{
    float *d2 = (float *)malloc((size_t)n * sizeof(float));
    uint64_t *w = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    if (!d2 || !w) { free(d2); free(w); return; }

    int64_t pick = orc_scale53(orc_draw(seed, stream, 0) >> 11, n);
    memcpy(C, X + rows[pick] * ld + col0, (size_t)ds * sizeof(float));

    float dmax = 0.0f;
    for (int64_t i = 0; i < n; ++i) {
        d2[i] = d2_f32(X + rows[i] * ld + col0, C, ds);
        if (d2[i] > dmax) dmax = d2[i];
    }
    int L = ceil_log2_i64(n);
    int E = 0;
    if (dmax > 0.0f) frexp((double)dmax, &E);
    double scale = ldexp(1.0, 62 - L - E);

    for (int t = 1; t < ks; ++t) {
        uint64_t r = orc_draw(seed, stream, (uint64_t)t) >> 11;
        uint64_t W = 0;
        for (int64_t i = 0; i < n; ++i) {
            w[i] = (dmax > 0.0f) ? (uint64_t)((double)d2[i] * scale) : 0;
            W += w[i];
        }
        if (W == 0) {
            pick = orc_scale53(r, n);
        } else {
            uint64_t thr = (uint64_t)(((unsigned __int128)r * (unsigned __int128)W) >> 53);
            uint64_t acc = 0;
            pick = n - 1;
            for (int64_t i = 0; i < n; ++i) {
                acc += w[i];
                if (acc > thr) { pick = i; break; }
            }
        }
        float *ct = C + (size_t)t * ds;
        memcpy(ct, X + rows[pick] * ld + col0, (size_t)ds * sizeof(float));
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            float d = d2_f32(X + rows[i] * ld + col0, ct, ds);
            if (d < d2[i]) d2[i] = d;
        }
    }
    free(d2);
    free(w);
}

/* Rows used for seeding: all of them, or 100*ks drawn with replacement. */
static int64_t seeding_rows(int64_t N, int ks, uint64_t seed, int64_t **rows_out)
{
    int64_t cap = (int64_t)100 * ks;
    int64_t n = N > cap ? cap : N;
    int64_t *rows = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!rows) return -1;
    if (N > cap) {
        for (int64_t l = 0; l < n; ++l)
            rows[l] = orc_scale53(orc_draw(seed, ORC_STREAM_SUBSAMPLE, (uint64_t)l) >> 11, N);
    } else {
        for (int64_t l = 0; l < n; ++l) rows[l] = l;
    }
    *rows_out = rows;
    return n;
}

/* k-means++ codebooks for all M subspaces; C is [M][Ks][Ds]. */
int orc_kmeanspp(const float *X, int64_t N, int D, int M, int Ks, uint64_t seed, float *C)
{
    if (M <= 0 || D % M != 0 || Ks <= 0 || N < Ks) return ORC_EINVAL;
    int ds = D / M;
    int64_t *rows = NULL;
    int64_t n = seeding_rows(N, Ks, seed, &rows);
    if (n < 0) return ORC_ENOMEM;
    for (int m = 0; m < M; ++m)
        orc_kmeanspp_slice(X, D, m * ds, ds, rows, n, Ks, seed, (uint64_t)m, C + (size_t)m * Ks * ds);
    free(rows);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Lloyd k-means per subspace (Sec. 2.1).                                   */
/* ------------------------------------------------------------------------ */

/* FP64 squared Euclidean distance by direct differences, dimension order. */
static double d2_f64(const float *x, const float *c, int ds)
{
    double acc = 0.0;
    for (int j = 0; j < ds; ++j) {
        double t = (double)x[j] - (double)c[j];
        acc = acc + t * t;
    }
    return acc;
}

/*
 * Nearest codeword of every (row, subspace): codes[N][M] (int32), the
 * distance to it mind[N][M] and the gap to the second nearest gap[N][M]
 * (both nullable).  Ties go to the lowest index.
 */
void orc_assign(const float *X, int64_t N, int D, int M, int Ks, const float *C, int32_t *codes,
                double *mind, double *gap)
{
    int ds = D / M;
    #pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        for (int m = 0; m < M; ++m) {
            const float *x = X + n * D + (int64_t)m * ds;
            const float *Cm = C + (size_t)m * Ks * ds;
            double best = INFINITY, second = INFINITY;
            int32_t bk = 0;
            for (int k = 0; k < Ks; ++k) {
                double d = d2_f64(x, Cm + (size_t)k * ds, ds);
                if (d < best) { second = best; best = d; bk = k; }
                else if (d < second) { second = d; }
            }
            codes[n * M + m] = bk;
            if (mind) mind[n * M + m] = best;
            if (gap) gap[n * M + m] = second - best;
        }
    }
}

/*
 * Centroid update: every codeword becomes the mean of the rows assigned to
 * it (FP64 sums in row order, one rounding to float32); a codeword with no
 * members keeps its previous value.  counts[M][Ks] is optional.
 */
int orc_update(const float *X, int64_t N, int D, int M, int Ks, const int32_t *codes, float *C,
               int64_t *counts)
{
    int ds = D / M;
    double *sum = (double *)calloc((size_t)M * Ks * ds, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)M * Ks, sizeof(int64_t));
    if (!sum || !cnt) { free(sum); free(cnt); return ORC_ENOMEM; }
    for (int64_t n = 0; n < N; ++n) {
        for (int m = 0; m < M; ++m) {
            int32_t k = codes[n * M + m];
            double *s = sum + ((size_t)m * Ks + k) * ds;
            const float *x = X + n * D + (int64_t)m * ds;
            for (int j = 0; j < ds; ++j) s[j] += (double)x[j];
            cnt[(size_t)m * Ks + k] += 1;
        }
    }
    for (int m = 0; m < M; ++m) {
        for (int k = 0; k < Ks; ++k) {
            int64_t c = cnt[(size_t)m * Ks + k];
            if (counts) counts[(size_t)m * Ks + k] = c;
            if (c == 0) continue;
            for (int j = 0; j < ds; ++j)
                C[((size_t)m * Ks + k) * ds + j] = (float)(sum[((size_t)m * Ks + k) * ds + j] / (double)c);
        }
    }
    free(sum);
    free(cnt);
    return ORC_OK;
}

/*
 * PQ fit: codebooks C[M][Ks][Ds] from k-means++ (or a copy of `init` if it
 * is non-null), then `iters` Lloyd iterations of assign + update.  sse[t]
 * (nullable) is the total squared error of iteration t's assignment, taken
 * against the codebooks that iteration started from.
 */
int orc_pq_fit(const float *X, int64_t N, int D, int M, int Ks, int iters, uint64_t seed,
               const float *init, float *C, double *sse)
{
    if (M <= 0 || D % M != 0 || Ks <= 0 || N < Ks || iters < 0) return ORC_EINVAL;
    int ds = D / M;
    if (init) memcpy(C, init, (size_t)M * Ks * ds * sizeof(float));
    else {
        int rc = orc_kmeanspp(X, N, D, M, Ks, seed, C);
        if (rc) return rc;
    }
    int32_t *codes = (int32_t *)malloc((size_t)N * M * sizeof(int32_t));
    double *mind = (double *)malloc((size_t)N * M * sizeof(double));
    if (!codes || !mind) { free(codes); free(mind); return ORC_ENOMEM; }
    for (int t = 0; t < iters; ++t) {
        orc_assign(X, N, D, M, Ks, C, codes, mind, NULL);
        if (sse) {
            double s = 0.0;
            for (int64_t i = 0; i < N * M; ++i) s += mind[i];
            sse[t] = s;
        }
        int rc = orc_update(X, N, D, M, Ks, codes, C, NULL);
        if (rc) { free(codes); free(mind); return rc; }
    }
    free(codes);
    free(mind);
    return ORC_OK;
}

/* Encode: uint8 codes[N][M] against codebooks C (Ks <= 256). */
int orc_pq_encode(const float *X, int64_t N, int D, int M, int Ks, const float *C, uint8_t *codes)
{
    if (Ks > 256 || M <= 0 || D % M != 0) return ORC_EINVAL;
    int32_t *c32 = (int32_t *)malloc((size_t)N * M * sizeof(int32_t));
    if (!c32) return ORC_ENOMEM;
    orc_assign(X, N, D, M, Ks, C, c32, NULL, NULL);
    for (int64_t i = 0; i < N * M; ++i) codes[i] = (uint8_t)c32[i];
    free(c32);
    return ORC_OK;
}

/* Decode: Xhat[N][D] = concatenation of the M selected codewords. */
void orc_pq_decode(const uint8_t *codes, int64_t N, int D, int M, int Ks, const float *C, float *Xhat)
{
    int ds = D / M;
    for (int64_t n = 0; n < N; ++n)
        for (int m = 0; m < M; ++m)
            memcpy(Xhat + n * D + (int64_t)m * ds, C + ((size_t)m * Ks + codes[n * M + m]) * ds,
                   (size_t)ds * sizeof(float));
}

/* RMSE = sqrt( sum_{n,d} (x - xhat)^2 / (N*D) ), FP64, row order. */
double orc_pq_rmse(const float *X, const uint8_t *codes, int64_t N, int D, int M, int Ks, const float *C)
{
    int ds = D / M;
    double s = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        for (int m = 0; m < M; ++m) {
            const float *c = C + ((size_t)m * Ks + codes[n * M + m]) * ds;
            const float *x = X + n * D + (int64_t)m * ds;
            for (int j = 0; j < ds; ++j) {
                double t = (double)x[j] - (double)c[j];
                s += t * t;
            }
        }
    }
    return sqrt(s / ((double)N * (double)D));
}

/* ------------------------------------------------------------------------ */
/* Inverted index over the PQ codes (Sec. 2.2, Sec. 3.1).                    */
/* ------------------------------------------------------------------------ */

/*
 * Build: coarse centroids coarse[nlist][D] by k-means on the raw rows (same
 * seeding and Lloyd rules as PQ with M = 1, Ks = nlist); list of a row = its
 * nearest coarse centroid; CSR lists with ids ascending inside a list:
 * offsets[nlist+1], ids[N], list_codes[N][M] (codes in list order).
 */
int orc_ivf_build(const float *X, const uint8_t *codes, int64_t N, int D, int M, int nlist, int iters,
                  uint64_t seed, float *coarse, int64_t *offsets, int64_t *ids, uint8_t *list_codes,
                  int32_t *list_of_row)
{
    int rc = orc_pq_fit(X, N, D, 1, nlist, iters, seed, NULL, coarse, NULL);
    if (rc) return rc;
    int32_t *lst = list_of_row ? list_of_row : (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!lst) return ORC_ENOMEM;
    orc_assign(X, N, D, 1, nlist, coarse, lst, NULL, NULL);
    for (int l = 0; l <= nlist; ++l) offsets[l] = 0;
    for (int64_t n = 0; n < N; ++n) offsets[lst[n] + 1] += 1;
    for (int l = 0; l < nlist; ++l) offsets[l + 1] += offsets[l];
    int64_t *fill = (int64_t *)malloc((size_t)nlist * sizeof(int64_t));
    if (!fill) { if (!list_of_row) free(lst); return ORC_ENOMEM; }
    for (int l = 0; l < nlist; ++l) fill[l] = offsets[l];
    for (int64_t n = 0; n < N; ++n) {
        int64_t p = fill[lst[n]]++;
        ids[p] = n;
        memcpy(list_codes + p * M, codes + n * M, (size_t)M);
    }
    free(fill);
    if (!list_of_row) free(lst);
    return ORC_OK;
}

typedef struct { double d; int64_t id; } orc_cand;

static int cand_cmp(const void *a, const void *b)
{
    const orc_cand *x = (const orc_cand *)a, *y = (const orc_cand *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/*
 * Query: probe the nprobe lists with the nearest coarse centroids (ties to
 * the lower list id), build the per-query distance table
 * LUT[m][k] = ||q_m - c_{m,k}||^2 in FP64, score each stored code by the sum
 * over m of LUT[m][code_m], return the k best by (score, id).  probes
 * [nq][nprobe] is optional.
 */
int orc_ivf_search(const float *coarse, const int64_t *offsets, const int64_t *ids, const uint8_t *list_codes,
                   int nlist, int D, int M, int Ks, const float *C, const float *Q, int64_t nq, int nprobe,
                   int k, int64_t *out_ids, double *out_d, int32_t *probes)
{
    if (nprobe < 1 || nprobe > nlist || k < 1 || D % M != 0) return ORC_EINVAL;
    int ds = D / M;
    int rc = ORC_OK;
    #pragma omp parallel
    {
        orc_cand *cl = (orc_cand *)malloc((size_t)nlist * sizeof(orc_cand));
        double *lut = (double *)malloc((size_t)M * Ks * sizeof(double));
        size_t cap = 1024;
        orc_cand *cand = (orc_cand *)malloc(cap * sizeof(orc_cand));
        if (!cl || !lut || !cand) rc = ORC_ENOMEM;
        #pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < nq; ++q) {
            if (rc) continue;
            const float *qv = Q + q * D;
            for (int l = 0; l < nlist; ++l) {
                cl[l].d = d2_f64(qv, coarse + (size_t)l * D, D);
                cl[l].id = l;
            }
            qsort(cl, (size_t)nlist, sizeof(orc_cand), cand_cmp);
            for (int m = 0; m < M; ++m)
                for (int kk = 0; kk < Ks; ++kk)
                    lut[m * Ks + kk] = d2_f64(qv + m * ds, C + ((size_t)m * Ks + kk) * ds, ds);
            size_t nc = 0;
            for (int p = 0; p < nprobe; ++p) {
                int l = (int)cl[p].id;
                if (probes) probes[q * nprobe + p] = l;
                for (int64_t e = offsets[l]; e < offsets[l + 1]; ++e) {
                    const uint8_t *code = list_codes + e * M;
                    double s = 0.0;
                    for (int m = 0; m < M; ++m) s += lut[m * Ks + code[m]];
                    if (nc == cap) {
                        cap *= 2;
                        orc_cand *nb = (orc_cand *)realloc(cand, cap * sizeof(orc_cand));
                        if (!nb) { rc = ORC_ENOMEM; break; }
                        cand = nb;
                    }
                    cand[nc].d = s;
                    cand[nc].id = ids[e];
                    ++nc;
                }
            }
            qsort(cand, nc, sizeof(orc_cand), cand_cmp);
            for (int r = 0; r < k; ++r) {
                out_ids[q * k + r] = (size_t)r < nc ? cand[r].id : -1;
                out_d[q * k + r] = (size_t)r < nc ? cand[r].d : INFINITY;
            }
        }
        free(cl);
        free(lut);
        free(cand);
    }
    return rc;
}

/* Exhaustive FP64 k nearest neighbours of each query, ordered by (d, id). */
int orc_exact_knn(const float *X, int64_t N, int D, const float *Q, int64_t nq, int k, int64_t *out_ids,
                  double *out_d)
{
    int rc = ORC_OK;
    #pragma omp parallel
    {
        orc_cand *all = (orc_cand *)malloc((size_t)N * sizeof(orc_cand));
        if (!all) rc = ORC_ENOMEM;
        #pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < nq; ++q) {
            if (rc) continue;
            for (int64_t n = 0; n < N; ++n) {
                all[n].d = d2_f64(Q + q * D, X + n * D, D);
                all[n].id = n;
            }
            qsort(all, (size_t)N, sizeof(orc_cand), cand_cmp);
            for (int r = 0; r < k; ++r) {
                out_ids[q * k + r] = r < N ? all[r].id : -1;
                out_d[q * k + r] = r < N ? all[r].d : INFINITY;
            }
        }
        free(all);
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Chunked divide and conquer (Sec. 3, "Methodology").                       */
/* ------------------------------------------------------------------------ */

/*
 * Each chunk c (rows chunk_offsets[c]..chunk_offsets[c+1]) gets its own PQ
 * fit with seed_c = draw(seed, CHUNK stream, c).  The codewords of all
 * chunks form the centroid dataset: row c*Ks + k is the concatenation over
 * m of codeword k of subspace m of chunk c.  A global PQ is fitted on that
 * dataset (seed), every original row is encoded with it and the RMSE of the
 * reconstruction is returned.  local_C[n_chunks][M][Ks][Ds] is optional.
 */
int orc_pq_fit_chunked(const float *X, const int64_t *chunk_offsets, int n_chunks, int D, int M, int Ks,
                       int iters, uint64_t seed, float *global_C, uint8_t *codes, double *rmse,
                       float *local_C)
{
    if (n_chunks < 1 || M <= 0 || D % M != 0 || Ks <= 0 || Ks > 256) return ORC_EINVAL;
    int ds = D / M;
    size_t cb = (size_t)M * Ks * ds;
    float *Cc = (float *)malloc(cb * sizeof(float));
    float *pool = (float *)malloc((size_t)n_chunks * Ks * D * sizeof(float));
    if (!Cc || !pool) { free(Cc); free(pool); return ORC_ENOMEM; }
    for (int c = 0; c < n_chunks; ++c) {
        int64_t r0 = chunk_offsets[c], r1 = chunk_offsets[c + 1];
        uint64_t sc = orc_draw(seed, ORC_STREAM_CHUNK, (uint64_t)c);
        int rc = orc_pq_fit(X + r0 * D, r1 - r0, D, M, Ks, iters, sc, NULL, Cc, NULL);
        if (rc) { free(Cc); free(pool); return rc; }
        if (local_C) memcpy(local_C + (size_t)c * cb, Cc, cb * sizeof(float));
        for (int k = 0; k < Ks; ++k)
            for (int m = 0; m < M; ++m)
                memcpy(pool + ((size_t)c * Ks + k) * D + (size_t)m * ds, Cc + ((size_t)m * Ks + k) * ds,
                       (size_t)ds * sizeof(float));
    }
    int64_t npool = (int64_t)n_chunks * Ks;
    int rc = orc_pq_fit(pool, npool, D, M, Ks, iters, seed, NULL, global_C, NULL);
    if (!rc) {
        int64_t N = chunk_offsets[n_chunks];
        rc = orc_pq_encode(X, N, D, M, Ks, global_C, codes);
        if (!rc && rmse) *rmse = orc_pq_rmse(X, codes, N, D, M, Ks, global_C);
    }
    free(Cc);
    free(pool);
    return rc;
}

/*
 * PQ fit that also returns the member counts of its last update:
 * counts[M][Ks] = the number of rows whose nearest codeword (under the codebooks
 * the last iteration started from) is k -- the rows whose mean the final
 * codeword is.  With iters = 0 every count is 1.
 */
int orc_pq_fit_counts(const float *X, int64_t N, int D, int M, int Ks, int iters, uint64_t seed, float *C,
                      int64_t *counts)
{
    int rc = orc_kmeanspp(X, N, D, M, Ks, seed, C);
    if (rc) return rc;
    for (int64_t i = 0; i < (int64_t)M * Ks; ++i) counts[i] = 1;
    int32_t *codes = (int32_t *)malloc((size_t)N * M * sizeof(int32_t));
    if (!codes) return ORC_ENOMEM;
    for (int t = 0; t < iters && !rc; ++t) {
        orc_assign(X, N, D, M, Ks, C, codes, NULL, NULL);
        rc = orc_update(X, N, D, M, Ks, codes, C, counts);
    }
    free(codes);
    return rc;
}

/*
 * Weighted PQ fit of n points P[n][D] with per-(point, subspace) weights
 * W[n][M]: k-means++ seeding of the points as they are (unweighted), then
 * `iters` rounds of assignment (nearest codeword, as in orc_assign) and weighted
 * update: codeword k of subspace m becomes sum_p W[p][m] x_{p,m} / sum_p W[p][m]
 * over its members p (FP64 sums in point order, one rounding to float32); a
 * codeword whose members weigh 0 keeps its value.
 */
int orc_pq_fit_weighted(const float *P, const int64_t *W, int64_t n, int D, int M, int Ks, int iters, uint64_t seed,
                        float *C)
{
    if (M <= 0 || D % M != 0 || Ks <= 0 || n < Ks || iters < 0) return ORC_EINVAL;
    int ds = D / M;
    int rc = orc_kmeanspp(P, n, D, M, Ks, seed, C);
    if (rc) return rc;
    int32_t *codes = (int32_t *)malloc((size_t)n * M * sizeof(int32_t));
    double *sum = (double *)malloc((size_t)M * Ks * ds * sizeof(double));
    double *wt = (double *)malloc((size_t)M * Ks * sizeof(double));
    if (!codes || !sum || !wt) { free(codes); free(sum); free(wt); return ORC_ENOMEM; }
    for (int t = 0; t < iters; ++t) {
        orc_assign(P, n, D, M, Ks, C, codes, NULL, NULL);
        memset(sum, 0, (size_t)M * Ks * ds * sizeof(double));
        memset(wt, 0, (size_t)M * Ks * sizeof(double));
        for (int64_t p = 0; p < n; ++p) {
            for (int m = 0; m < M; ++m) {
                int32_t k = codes[p * M + m];
                double w = (double)W[p * M + m];
                const float *x = P + p * D + (int64_t)m * ds;
                double *s = sum + ((size_t)m * Ks + k) * ds;
                for (int j = 0; j < ds; ++j) s[j] += w * (double)x[j];
                wt[(size_t)m * Ks + k] += w;
            }
        }
        for (int m = 0; m < M; ++m)
            for (int k = 0; k < Ks; ++k) {
                double w = wt[(size_t)m * Ks + k];
                if (w == 0.0) continue;
                for (int j = 0; j < ds; ++j)
                    C[((size_t)m * Ks + k) * ds + j] = (float)(sum[((size_t)m * Ks + k) * ds + j] / w);
            }
    }
    free(codes);
    free(sum);
    free(wt);
    return ORC_OK;
}

/*
 * The divide-and-conquer fit with a weighted centroid dataset: as
 * orc_pq_fit_chunked, except that pooled codeword k of subspace m of chunk c
 * carries the weight W = its member count in the chunk's last Lloyd update (the
 * number of the chunk's rows it is the mean of), and the global model is the
 * weighted fit of the pooled codewords (orc_pq_fit_weighted).  weights
 * [n_chunks*Ks][M] (optional) receives W.
 */
int orc_pq_fit_chunked_weighted(const float *X, const int64_t *chunk_offsets, int n_chunks, int D, int M, int Ks,
                                int iters, uint64_t seed, float *global_C, uint8_t *codes, double *rmse,
                                float *local_C, int64_t *weights)
{
    if (n_chunks < 1 || M <= 0 || D % M != 0 || Ks <= 0 || Ks > 256) return ORC_EINVAL;
    int ds = D / M;
    size_t cb = (size_t)M * Ks * ds;
    int64_t npool = (int64_t)n_chunks * Ks;
    float *Cc = (float *)malloc(cb * sizeof(float));
    int64_t *cnt = (int64_t *)malloc((size_t)M * Ks * sizeof(int64_t));
    float *pool = (float *)malloc((size_t)npool * D * sizeof(float));
    int64_t *W = (int64_t *)malloc((size_t)npool * M * sizeof(int64_t));
    int rc = ORC_OK;
    if (!Cc || !cnt || !pool || !W) { rc = ORC_ENOMEM; goto done; }
    for (int c = 0; c < n_chunks; ++c) {
        int64_t r0 = chunk_offsets[c], r1 = chunk_offsets[c + 1];
        uint64_t sc = orc_draw(seed, ORC_STREAM_CHUNK, (uint64_t)c);
        rc = orc_pq_fit_counts(X + r0 * D, r1 - r0, D, M, Ks, iters, sc, Cc, cnt);
        if (rc) goto done;
        if (local_C) memcpy(local_C + (size_t)c * cb, Cc, cb * sizeof(float));
        for (int k = 0; k < Ks; ++k)
            for (int m = 0; m < M; ++m) {
                memcpy(pool + ((size_t)c * Ks + k) * D + (size_t)m * ds, Cc + ((size_t)m * Ks + k) * ds,
                       (size_t)ds * sizeof(float));
                W[((size_t)c * Ks + k) * M + m] = cnt[(size_t)m * Ks + k];
            }
    }
    if (weights) memcpy(weights, W, (size_t)npool * M * sizeof(int64_t));
    rc = orc_pq_fit_weighted(pool, W, npool, D, M, Ks, iters, seed, global_C);
    if (!rc) {
        int64_t N = chunk_offsets[n_chunks];
        rc = orc_pq_encode(X, N, D, M, Ks, global_C, codes);
        if (!rc && rmse) *rmse = orc_pq_rmse(X, codes, N, D, M, Ks, global_C);
    }
done:
    free(Cc);
    free(cnt);
    free(pool);
    free(W);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Soft-assignment codebook refinement (FP64 inputs).                        */
/* ------------------------------------------------------------------------ */

/*
 * For each row n and subspace m: d_k = ||x - c_k||^2, p = softmax_k(-d/tau)
 * (max-subtracted), xhat = sum_k p_k c_k, r = xhat - x.
 * L = (1/N) sum_n sum_m ||r||^2.  Returns L.
 */
double orc_softpq_forward(const double *X, int64_t N, int D, int M, int Ks, const double *C, double tau)
{
    int ds = D / M;
    double total = 0.0;
    double *d = (double *)malloc((size_t)Ks * sizeof(double));
    double *xh = (double *)malloc((size_t)ds * sizeof(double));
    for (int64_t n = 0; n < N; ++n) {
        for (int m = 0; m < M; ++m) {
            const double *x = X + n * D + (int64_t)m * ds;
            const double *Cm = C + (size_t)m * Ks * ds;
            double smax = -INFINITY;
            for (int k = 0; k < Ks; ++k) {
                double acc = 0.0;
                for (int j = 0; j < ds; ++j) { double t = x[j] - Cm[k * ds + j]; acc += t * t; }
                d[k] = -acc / tau;
                if (d[k] > smax) smax = d[k];
            }
            double z = 0.0;
            for (int k = 0; k < Ks; ++k) { d[k] = exp(d[k] - smax); z += d[k]; }
            for (int j = 0; j < ds; ++j) xh[j] = 0.0;
            for (int k = 0; k < Ks; ++k) {
                double p = d[k] / z;
                for (int j = 0; j < ds; ++j) xh[j] += p * Cm[k * ds + j];
            }
            for (int j = 0; j < ds; ++j) { double r = xh[j] - x[j]; total += r * r; }
        }
    }
    free(d);
    free(xh);
    return total / (double)N;
}

/*
 * Gradients of L above.  With G_k = (2/N) r . c_k and
 * g_k = p_k (G_k - sum_l p_l G_l) (the gradient with respect to the logit
 * s_k = -d_k/tau):
 *   dL/dc_k = (2/N) p_k r + (2/tau) g_k (x - c_k)
 *   dL/dx   = -(2/N) r - (2/tau) sum_k g_k (x - c_k)
 * dC[M][Ks][Ds] and dX[N][D] are overwritten.
 */
void orc_softpq_backward(const double *X, int64_t N, int D, int M, int Ks, const double *C, double tau,
                         double *dC, double *dX)
{
    int ds = D / M;
    double *p = (double *)malloc((size_t)Ks * sizeof(double));
    double *G = (double *)malloc((size_t)Ks * sizeof(double));
    double *r = (double *)malloc((size_t)ds * sizeof(double));
    memset(dC, 0, (size_t)M * Ks * ds * sizeof(double));
    double invN = 1.0 / (double)N;
    for (int64_t n = 0; n < N; ++n) {
        for (int m = 0; m < M; ++m) {
            const double *x = X + n * D + (int64_t)m * ds;
            const double *Cm = C + (size_t)m * Ks * ds;
            double *dCm = dC + (size_t)m * Ks * ds;
            double smax = -INFINITY;
            for (int k = 0; k < Ks; ++k) {
                double acc = 0.0;
                for (int j = 0; j < ds; ++j) { double t = x[j] - Cm[k * ds + j]; acc += t * t; }
                p[k] = -acc / tau;
                if (p[k] > smax) smax = p[k];
            }
            double z = 0.0;
            for (int k = 0; k < Ks; ++k) { p[k] = exp(p[k] - smax); z += p[k]; }
            for (int k = 0; k < Ks; ++k) p[k] /= z;
            for (int j = 0; j < ds; ++j) {
                double xh = 0.0;
                for (int k = 0; k < Ks; ++k) xh += p[k] * Cm[k * ds + j];
                r[j] = xh - x[j];
            }
            double pg = 0.0;
            for (int k = 0; k < Ks; ++k) {
                double acc = 0.0;
                for (int j = 0; j < ds; ++j) acc += r[j] * Cm[k * ds + j];
                G[k] = 2.0 * invN * acc;
                pg += p[k] * G[k];
            }
            double *dx = dX + n * D + (int64_t)m * ds;
            for (int j = 0; j < ds; ++j) dx[j] = -2.0 * invN * r[j];
            for (int k = 0; k < Ks; ++k) {
                double g = p[k] * (G[k] - pg);
                for (int j = 0; j < ds; ++j) {
                    double diff = x[j] - Cm[k * ds + j];
                    dCm[k * ds + j] += 2.0 * invN * p[k] * r[j] + (2.0 / tau) * g * diff;
                    dx[j] -= (2.0 / tau) * g * diff;
                }
            }
        }
    }
    free(p);
    free(G);
    free(r);
}

/* ------------------------------------------------------------------------ */
/* Code-space coarse quantizer: Rii's inverted index over the PQ codes       */
/* (Sec. 3.1: an IVFPQ-style index built from the codes themselves).         */
/* ------------------------------------------------------------------------ */

#define ORC_STREAM_CENTERS 0xFFFFFFFDull

/*
 * Symmetric distance table of the codebooks: DT[m][k][j] = ||c_{m,k} - c_{m,j}||^2
 * in FP64 by direct differences in dimension order.  The symmetric distance of
 * two codes a, b is SDC(a, b) = sum over m (in order) of DT[m][a_m][b_m]: the
 * squared distance of the two reconstructions, taken subspace by subspace.
 */
void orc_sdc_table(const float *C, int M, int Ks, int ds, double *DT)
{
    for (int m = 0; m < M; ++m)
        for (int k = 0; k < Ks; ++k)
            for (int j = 0; j < Ks; ++j)
                DT[((size_t)m * Ks + k) * Ks + j] =
                    d2_f64(C + ((size_t)m * Ks + k) * ds, C + ((size_t)m * Ks + j) * ds, ds);
}

static double sdc(const double *DT, int M, int Ks, const uint8_t *a, const uint8_t *b)
{
    double s = 0.0;
    for (int m = 0; m < M; ++m) s += DT[((size_t)m * Ks + a[m]) * Ks + b[m]];
    return s;
}

/*
 * nlist distinct row indices of [0, N) by Floyd's sampling algorithm (Bentley &
 * Floyd, "A sample of brilliance", CACM 1987): for j = N - nlist .. N - 1 draw t
 * uniform in [0, j]; take t unless it was taken already, else take j.  Draw i
 * is floor(u * (j + 1)) with u the 53-bit output i of the centre stream of
 * `seed`.  out[nlist] in the order taken.
 */
int orc_pick_distinct(int64_t N, int nlist, uint64_t seed, int64_t *out)
{
    if (nlist < 1 || nlist > N) return ORC_EINVAL;
    for (int i = 0; i < nlist; ++i) {
        int64_t j = N - nlist + i;
        int64_t t = orc_scale53(orc_draw(seed, ORC_STREAM_CENTERS, (uint64_t)i) >> 11, j + 1);
        int taken = 0;
        for (int q = 0; q < i; ++q) taken |= out[q] == t;
        out[i] = taken ? j : t;
    }
    return ORC_OK;
}

/* Nearest centre code of every row code by SDC (ties to the lower centre); its SDC in dist (nullable). */
void orc_assign_codes(const uint8_t *codes, int64_t N, int M, int Ks, const double *DT, const uint8_t *centers,
                      int nlist, int32_t *lst, double *dist)
{
    #pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double best = INFINITY;
        int32_t bl = 0;
        for (int l = 0; l < nlist; ++l) {
            double d = sdc(DT, M, Ks, codes + n * M, centers + (size_t)l * M);
            if (d < best) { best = d; bl = l; }
        }
        lst[n] = bl;
        if (dist) dist[n] = best;
    }
}

/*
 * Centre update (the "sparse voting" step of k-means over PQ codes): for every
 * list l and subspace m, with h[j] the number of members whose code in m is j,
 * the new centre code is argmin over k of cost(k) = sum over j (ascending) of
 * h[j] * DT[m][k][j] -- the code minimising the summed SDC term of that
 * subspace to the members -- ties to the lower k.  A list without members keeps
 * its centre.
 */
int orc_update_centers(const uint8_t *codes, int64_t N, int M, int Ks, const double *DT, const int32_t *lst,
                       int nlist, uint8_t *centers)
{
    int64_t *h = (int64_t *)calloc((size_t)nlist * M * Ks, sizeof(int64_t));
    int64_t *n_l = (int64_t *)calloc((size_t)nlist, sizeof(int64_t));
    if (!h || !n_l) { free(h); free(n_l); return ORC_ENOMEM; }
    for (int64_t n = 0; n < N; ++n) {
        n_l[lst[n]] += 1;
        for (int m = 0; m < M; ++m) h[((size_t)lst[n] * M + m) * Ks + codes[n * M + m]] += 1;
    }
    for (int l = 0; l < nlist; ++l) {
        if (n_l[l] == 0) continue;
        for (int m = 0; m < M; ++m) {
            const int64_t *hm = h + ((size_t)l * M + m) * Ks;
            double best = INFINITY;
            int bk = 0;
            for (int k = 0; k < Ks; ++k) {
                double cost = 0.0;
                for (int j = 0; j < Ks; ++j) cost += (double)hm[j] * DT[((size_t)m * Ks + k) * Ks + j];
                if (cost < best) { best = cost; bk = k; }
            }
            centers[(size_t)l * M + m] = (uint8_t)bk;
        }
    }
    free(h);
    free(n_l);
    return ORC_OK;
}

/*
 * Build: centre codes by k-means over the PQ codes (nlist rows picked by
 * orc_pick_distinct as the starting centres, `iters` rounds of
 * orc_assign_codes + orc_update_centers), then every row in the list of its
 * nearest centre, CSR lists with ids ascending.  obj[t] (nullable) is the total
 * SDC of round t's assignment to the centres it started from.
 */
int orc_ivf_build_codes(const uint8_t *codes, int64_t N, int M, int Ks, int ds, const float *C, int nlist,
                        int iters, uint64_t seed, uint8_t *centers, int64_t *offsets, int64_t *ids,
                        uint8_t *list_codes, int32_t *list_of_row, double *obj)
{
    if (nlist < 1 || nlist > N || Ks < 1 || Ks > 256 || iters < 0) return ORC_EINVAL;
    double *DT = (double *)malloc((size_t)M * Ks * Ks * sizeof(double));
    int64_t *pick = (int64_t *)malloc((size_t)nlist * sizeof(int64_t));
    int32_t *lst = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    double *dist = (double *)malloc((size_t)N * sizeof(double));
    int64_t *fill = (int64_t *)malloc((size_t)nlist * sizeof(int64_t));
    int rc = ORC_OK;
    if (!DT || !pick || !lst || !dist || !fill) { rc = ORC_ENOMEM; goto done; }
    orc_sdc_table(C, M, Ks, ds, DT);
    orc_pick_distinct(N, nlist, seed, pick);
    for (int l = 0; l < nlist; ++l) memcpy(centers + (size_t)l * M, codes + pick[l] * M, (size_t)M);
    for (int t = 0; t < iters; ++t) {
        orc_assign_codes(codes, N, M, Ks, DT, centers, nlist, lst, dist);
        if (obj) {
            double s = 0.0;
            for (int64_t n = 0; n < N; ++n) s += dist[n];
            obj[t] = s;
        }
        rc = orc_update_centers(codes, N, M, Ks, DT, lst, nlist, centers);
        if (rc) goto done;
    }
    orc_assign_codes(codes, N, M, Ks, DT, centers, nlist, lst, NULL);
    for (int l = 0; l <= nlist; ++l) offsets[l] = 0;
    for (int64_t n = 0; n < N; ++n) offsets[lst[n] + 1] += 1;
    for (int l = 0; l < nlist; ++l) offsets[l + 1] += offsets[l];
    for (int l = 0; l < nlist; ++l) fill[l] = offsets[l];
    for (int64_t n = 0; n < N; ++n) {
        int64_t p = fill[lst[n]]++;
        ids[p] = n;
        memcpy(list_codes + p * M, codes + n * M, (size_t)M);
    }
    if (list_of_row) memcpy(list_of_row, lst, (size_t)N * sizeof(int32_t));
done:
    free(DT);
    free(pick);
    free(lst);
    free(dist);
    free(fill);
    return rc;
}

/*
 * Query of the code-space index: the per-query table LUT[m][k] = ||q_m - c_{m,k}||^2
 * (FP64) scores both the centre codes (probe: the nprobe lowest sum over m of
 * LUT[m][centre_m], ties to the lower list) and the stored codes of the probed
 * lists; the k best by (score, id), missing results id -1 and +inf.
 */
int orc_ivf_search_codes(const uint8_t *centers, const int64_t *offsets, const int64_t *ids,
                         const uint8_t *list_codes, int nlist, int D, int M, int Ks, const float *C, const float *Q,
                         int64_t nq, int nprobe, int k, int64_t *out_ids, double *out_d, int32_t *probes)
{
    if (nprobe < 1 || nprobe > nlist || k < 1 || D % M != 0) return ORC_EINVAL;
    int ds = D / M;
    int rc = ORC_OK;
    #pragma omp parallel
    {
        orc_cand *cl = (orc_cand *)malloc((size_t)nlist * sizeof(orc_cand));
        double *lut = (double *)malloc((size_t)M * Ks * sizeof(double));
        size_t cap = 1024;
        orc_cand *cand = (orc_cand *)malloc(cap * sizeof(orc_cand));
        if (!cl || !lut || !cand) rc = ORC_ENOMEM;
        #pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < nq; ++q) {
            if (rc) continue;
            const float *qv = Q + q * D;
            for (int m = 0; m < M; ++m)
                for (int kk = 0; kk < Ks; ++kk)
                    lut[m * Ks + kk] = d2_f64(qv + m * ds, C + ((size_t)m * Ks + kk) * ds, ds);
            for (int l = 0; l < nlist; ++l) {
                double s = 0.0;
                for (int m = 0; m < M; ++m) s += lut[m * Ks + centers[(size_t)l * M + m]];
                cl[l].d = s;
                cl[l].id = l;
            }
            qsort(cl, (size_t)nlist, sizeof(orc_cand), cand_cmp);
            size_t nc = 0;
            for (int p = 0; p < nprobe; ++p) {
                int l = (int)cl[p].id;
                if (probes) probes[q * nprobe + p] = l;
                for (int64_t e = offsets[l]; e < offsets[l + 1]; ++e) {
                    const uint8_t *code = list_codes + e * M;
                    double s = 0.0;
                    for (int m = 0; m < M; ++m) s += lut[m * Ks + code[m]];
                    if (nc == cap) {
                        cap *= 2;
                        orc_cand *nb = (orc_cand *)realloc(cand, cap * sizeof(orc_cand));
                        if (!nb) { rc = ORC_ENOMEM; break; }
                        cand = nb;
                    }
                    cand[nc].d = s;
                    cand[nc].id = ids[e];
                    ++nc;
                }
            }
            qsort(cand, nc, sizeof(orc_cand), cand_cmp);
            for (int r = 0; r < k; ++r) {
                out_ids[q * k + r] = (size_t)r < nc ? cand[r].id : -1;
                out_d[q * k + r] = (size_t)r < nc ? cand[r].d : INFINITY;
            }
        }
        free(cl);
        free(lut);
        free(cand);
    }
    return rc;
}

/* Threads the OpenMP regions above will use. */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
