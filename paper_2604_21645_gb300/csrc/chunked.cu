// chunked.cu -- the paper's divide-and-conquer PQ (Sec. 3, "Methodology"):
// the rows are split into chunks, every chunk gets its own PQ fit, the
// codewords of all chunks are pooled into a centroid dataset (row c*Ks + k is
// the concatenation over subspaces of codeword k of chunk c), a global PQ is
// fitted on that dataset, and every original row is encoded with the global
// model and its reconstruction error measured.
//
// On one GPU the chunk fits are batched instead of run as separate tasks: one
// launch seeds every (chunk, subspace) pair, and every Lloyd iteration is one
// pass launch over all chunks (blocks are assigned to chunks in proportion to
// their rows) plus one finalise launch.  Chunk c is seeded with draw c of the
// chunk stream of the caller's seed, exactly as the CPU reference does.  The
// sequence is stream-ordered with no host synchronisation unless the RMSE is
// requested, so it can be captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

struct ChunkTableParams {
    int n;
    int64_t off[kMaxSeedChunks + 1];
    int blk[kMaxSeedChunks + 1];
};

__global__ void chunk_tables_kernel(const ChunkTableParams p, int gx, int64_t *off, int *blk, int *blk_chunk)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= p.n) {
        off[i] = p.off[i];
        blk[i] = p.blk[i];
    }
    if (i < gx) {
        int c = 0;
        while (c + 1 < p.n && p.blk[c + 1] <= i) ++c;
        blk_chunk[i] = c;
    }
}

// pool[(c*Ks + k)][m*ds + j] = C[c][m][k][j]
__global__ void pool_codewords_kernel(const float *__restrict__ C, int n_chunks, int M, int Ks, int ds,
                                      float *__restrict__ pool)
{
    const int64_t total = (int64_t)n_chunks * M * Ks * ds;
    const int D = M * ds;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % ds);
        const int64_t t = e / ds;
        const int k = (int)(t % Ks);
        const int64_t u = t / Ks;
        const int m = (int)(u % M);
        const int64_t c = u / M;
        pool[(c * Ks + k) * D + (int64_t)m * ds + j] = C[e];
    }
}

// W[(c*Ks + k)*M + m] = counts[(c*M + m)*Ks + k]: the weight of pooled row c*Ks + k in subspace m
__global__ void pool_weights_kernel(const long long *__restrict__ counts, int n_chunks, int M, int Ks,
                                    long long *__restrict__ W)
{
    const int64_t total = (int64_t)n_chunks * M * Ks;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % Ks);
        const int64_t cm = e / Ks;
        const int m = (int)(cm % M);
        const int64_t c = cm / M;
        W[(c * Ks + k) * M + m] = counts[e];
    }
}

__global__ void fill_ll_kernel(long long *p, int64_t n, long long v)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = v;
}

// Weighted update of the global model, one thread per (subspace, codeword, dimension): over the
// pooled rows p in order, the members of codeword k in subspace m add W[p][m] * x in float-float
// (each product exact by TwoProduct), their weights in int64; the codeword becomes the float-float
// quotient rounded once, or keeps its value when its members weigh nothing.
__global__ void weighted_update_kernel(const float *__restrict__ P, int64_t n, int D, int M, int Ks, int ds,
                                       const uint8_t *__restrict__ codes, const long long *__restrict__ W,
                                       float *__restrict__ C)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)M * Ks * ds) return;
    const int j = (int)(idx % ds);
    const int k = (int)((idx / ds) % Ks), m = (int)(idx / ((int64_t)ds * Ks));
    float sh = 0.0f, sl = 0.0f;
    long long wsum = 0;
    for (int64_t p = 0; p < n; ++p) {
        if (codes[p * M + m] != k) continue;
        const long long w = W[p * M + m];
        if (w == 0) continue;
        float wh, wl;
        ll_to_ff(w, wh, wl);
        const float x = P[p * D + (int64_t)m * ds + j];
        float ph, pe;
        two_prod(wh, x, ph, pe);
        pe = __fmaf_rn(wl, x, pe);
        ff_add(sh, sl, ph, pe, sh, sl);
        wsum += w;
    }
    if (wsum == 0) return;
    float nh, nl, qh, ql;
    ll_to_ff(wsum, nh, nl);
    ff_div(sh, sl, nh, nl, qh, ql);
    C[idx] = __fadd_rn(qh, ql);
}

// Grid blocks shared out over the chunks in proportion to their rows: `per` blocks
// for the whole data set, at least one and at most one row tile's worth per chunk.
int build_chunk_table(const int64_t *off, int n_chunks, int per, bool tc, ChunkTableParams &tp)
{
    const int64_t N = off[n_chunks];
    tp.n = n_chunks;
    tp.blk[0] = 0;
    for (int c = 0; c <= n_chunks; ++c) tp.off[c] = off[c];
    for (int c = 0; c < n_chunks; ++c) {
        const int64_t rows = off[c + 1] - off[c];
        int64_t g = std::max<int64_t>(1, (int64_t)std::llround((double)per * (double)rows / (double)N));
        g = std::min<int64_t>(g, tc ? (rows + 127) / 128 : (rows + 255) / 256);
        tp.blk[c + 1] = tp.blk[c] + (int)std::max<int64_t>(1, g);
    }
    return tp.blk[n_chunks];
}

int default_per(int sms, int64_t N, int M, bool tc)
{
    PqPass base;
    base.N = N;
    base.M = M;
    return tc ? std::max(1, sms / std::max(1, M / tc_pass_group())) : pq_pass_blocks_per_subspace(base);
}

// Tuned block counts of the batched pass, keyed by the shape of the problem.
using TuneKey = std::tuple<int, int64_t, int, int, int, int, int, uint64_t>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

TuneKey tune_key(const int64_t *off, int n_chunks, int D, int M, int Ks, int prec, int sms)
{
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the chunk offsets
    for (int c = 0; c <= n_chunks; ++c) {
        h ^= (uint64_t)off[c];
        h *= 1099511628211ull;
    }
    return TuneKey(n_chunks, off[n_chunks], D, M, Ks, prec, sms, h);
}

}  // namespace

int run_pq_fit_chunked(const float *X, const int64_t *off, int n_chunks, int D, int M, int Ks, int iters,
                       uint64_t seed, int prec, float *global_cb, uint8_t *codes, double *rmse, cudaStream_t s,
                       bool weighted)
{
    const int64_t N = off[n_chunks];
    const int ds = D / M;
    const bool tc = prec == PQ_PREC_BF16;
    int dev = 0, sms = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    PQ_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int *err = device_error_word(dev);
    if (!err) return fail(PQ_ENOMEM, "device error word");
    Scratch ws(s);
    const size_t cbsz = (size_t)M * Ks * ds;
    float *Cl = ws.get<float>((size_t)n_chunks * cbsz);
    if (ws.status) return ws.status;

    // (1) local seeding of every (chunk, subspace) in one launch
    std::vector<SeedChunk> ch(n_chunks);
    for (int c = 0; c < n_chunks; ++c) {
        ch[c].r0 = off[c];
        ch[c].rows = off[c + 1] - off[c];
        ch[c].seed = rng_draw(seed, kStreamChunk, (uint64_t)c);
    }
    PQ_TRY(launch_kmeanspp_chunks(X, D, ch.data(), n_chunks, ds, M, Ks, Cl, ws, err, s, "kmeanspp_chunks"));

    // (2) batched Lloyd iterations: blocks shared out in proportion to the rows, as many as
    // the autotuner chose for this shape (pq_tune_chunked) or the default
    int per = default_per(sms, N, M, tc);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(tune_key(off, n_chunks, D, M, Ks, prec, sms));
        if (it != g_tuned.end()) per = it->second;
    }
    ChunkTableParams tp;
    const int gx = build_chunk_table(off, n_chunks, per, tc, tp);
    int64_t *d_off = ws.get<int64_t>((size_t)n_chunks + 1);
    int *d_blk = ws.get<int>((size_t)n_chunks + 1);
    int *d_bc = ws.get<int>((size_t)gx);
    PqPass p;
    p.X = X;
    p.N = N;
    p.D = D;
    p.M = M;
    p.Ks = Ks;
    p.ds = ds;
    p.C = Cl;
    p.gx = gx;
    void *pb = ws.raw(Partials::bytes(gx, M, Ks, ds, n_chunks), false);
    if (ws.status) return ws.status;
    p.part.carve(pb, gx, M, Ks, ds);
    {
        const int n = std::max(n_chunks + 1, gx);
        ProfScope ps("chunk_tables", s);
        chunk_tables_kernel<<<(n + 127) / 128, 128, 0, s>>>(tp, gx, d_off, d_blk, d_bc);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
    }
    p.blk_chunk = d_bc;
    p.chunk_off = d_off;
    p.chunk_blk = d_blk;
    p.n_chunks = n_chunks;
    // member counts of each chunk's last update (the weights of the weighted combine)
    long long *counts = weighted ? ws.get<long long>((size_t)n_chunks * M * Ks) : nullptr;
    if (ws.status) return ws.status;
    if (weighted && iters == 0) {
        fill_ll_kernel<<<64, 256, 0, s>>>(counts, (int64_t)n_chunks * M * Ks, 1);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
    }
    if (tc) {
        // all the passes of every (chunk, subspace group) in one persistent launch
        int *sync = ws.get<int>(persistent_sync_ints(n_chunks, M), true);
        if (ws.status) return ws.status;
        PQ_TRY(launch_pq_fit_persistent_tc(p, iters, sync, counts, s));
    } else {
        for (int t = 0; t < iters; ++t) {
            PQ_TRY(launch_pq_pass_f32(p, s));
            PQ_TRY(launch_pq_finalize(p.part, gx, M, Ks, ds, Cl, nullptr, s, n_chunks, d_blk,
                                      t + 1 == iters ? counts : nullptr));
        }
    }

    // (3) centroid dataset of the pooled codewords, (4) global fit, (5) global encode + error
    const int64_t npool = (int64_t)n_chunks * Ks;
    float *pool = ws.get<float>((size_t)npool * D);
    double *sse = ws.get<double>(1, true);
    if (ws.status) return ws.status;
    {
        ProfScope ps("pool_codewords", s);
        const int64_t total = (int64_t)n_chunks * cbsz;
        pool_codewords_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, s>>>(Cl, n_chunks, M, Ks,
                                                                                                  ds, pool);
        count_launch();
        PQ_TRY_CUDA(cudaGetLastError());
    }
    if (!weighted) {
        PQ_TRY(pq_fit(pool, npool, D, M, Ks, iters, seed, prec, nullptr, global_cb, nullptr, s));
    } else {
        // weighted global fit: k-means++ seeding of the pooled rows, then rounds of exact assignment
        // (an encode pass) and the weighted update
        long long *W = ws.get<long long>((size_t)npool * M);
        uint8_t *pcodes = ws.get<uint8_t>((size_t)npool * M);
        if (ws.status) return ws.status;
        {
            ProfScope ps("pool_weights", s);
            pool_weights_kernel<<<64, 256, 0, s>>>(counts, n_chunks, M, Ks, W);
            count_launch();
            PQ_TRY_CUDA(cudaGetLastError());
        }
        PQ_TRY(pq_init_kmeanspp(pool, npool, D, M, Ks, seed, global_cb, s));
        PqPass gp;
        gp.X = pool;
        gp.N = npool;
        gp.D = D;
        gp.M = M;
        gp.Ks = Ks;
        gp.ds = ds;
        gp.C = global_cb;
        gp.codes = pcodes;
        const int64_t nth = (int64_t)M * Ks * ds;
        for (int t = 0; t < iters; ++t) {
            PqPass q = gp;
            PQ_TRY(tc ? launch_pq_pass_tc(q, s) : launch_pq_pass_f32(q, s));
            ProfScope ps("weighted_update", s);
            weighted_update_kernel<<<(unsigned)((nth + 127) / 128), 128, 0, s>>>(pool, npool, D, M, Ks, ds, pcodes, W,
                                                                              global_cb);
            count_launch();
            PQ_TRY_CUDA(cudaGetLastError());
        }
    }
    PQ_TRY(pq_encode(X, N, D, M, Ks, global_cb, prec, codes, sse, nullptr, s));
    if (rmse) {
        double h = 0.0;
        PQ_TRY_CUDA(cudaMemcpyAsync(&h, sse, sizeof(double), cudaMemcpyDeviceToHost, s));
        PQ_TRY_CUDA(cudaStreamSynchronize(s));
        *rmse = std::sqrt(h / ((double)N * (double)D));
    }
    return ws.status;
}

int run_pq_tune_chunked(const float *X, const int64_t *off, int n_chunks, int D, int M, int Ks, int prec,
                        int *best_per, float *best_ms, cudaStream_t s)
{
    const int64_t N = off[n_chunks];
    const int ds = D / M;
    const bool tc = prec == PQ_PREC_BF16;
    int dev = 0, sms = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    PQ_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int *err = device_error_word(dev);
    if (!err) return fail(PQ_ENOMEM, "device error word");
    Scratch ws(s);
    const size_t cbsz = (size_t)M * Ks * ds;
    float *Cl = ws.get<float>((size_t)n_chunks * cbsz);
    if (ws.status) return ws.status;
    // realistic codebooks: the local seeds of every chunk
    std::vector<SeedChunk> ch(n_chunks);
    for (int c = 0; c < n_chunks; ++c) {
        ch[c].r0 = off[c];
        ch[c].rows = off[c + 1] - off[c];
        ch[c].seed = rng_draw(0x7E57ull, kStreamChunk, (uint64_t)c);
    }
    PQ_TRY(launch_kmeanspp_chunks(X, D, ch.data(), n_chunks, ds, M, Ks, Cl, ws, err, s, "kmeanspp_chunks"));
    // candidate block counts around the default; the part buffers are sized for the largest
    const int base = default_per(sms, N, M, tc);
    const double scales[] = {0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 4.0, 6.0, 8.0};
    std::vector<int> cand;
    for (double f : scales) {
        const int v = std::max(1, (int)std::llround(base * f));
        if (std::find(cand.begin(), cand.end(), v) == cand.end()) cand.push_back(v);
    }
    ChunkTableParams tp;
    int gmax = 0;
    for (int v : cand) gmax = std::max(gmax, build_chunk_table(off, n_chunks, v, tc, tp));
    int64_t *d_off = ws.get<int64_t>((size_t)n_chunks + 1);
    int *d_blk = ws.get<int>((size_t)n_chunks + 1);
    int *d_bc = ws.get<int>((size_t)gmax);
    void *pb = ws.raw(Partials::bytes(gmax, M, Ks, ds, n_chunks), false);
    const size_t nsync = persistent_sync_ints(n_chunks, M);
    int *sync = tc ? ws.get<int>(nsync) : nullptr;
    if (ws.status) return ws.status;
    cudaEvent_t e0, e1;
    PQ_TRY_CUDA(cudaEventCreate(&e0));
    PQ_TRY_CUDA(cudaEventCreate(&e1));
    int best = base;
    float bms = 1e30f;
    int st = PQ_OK;
    for (int v : cand) {
        const int gx = build_chunk_table(off, n_chunks, v, tc, tp);
        chunk_tables_kernel<<<(std::max(n_chunks + 1, gx) + 127) / 128, 128, 0, s>>>(tp, gx, d_off, d_blk, d_bc);
        count_launch();
        PqPass p;
        p.X = X;
        p.N = N;
        p.D = D;
        p.M = M;
        p.Ks = Ks;
        p.ds = ds;
        p.C = Cl;
        p.gx = gx;
        p.part.carve(pb, gx, M, Ks, ds);
        p.blk_chunk = d_bc;
        p.chunk_off = d_off;
        p.chunk_blk = d_blk;
        p.n_chunks = n_chunks;
        if (tc) {
            // the persistent form: one launch of one pass to warm up, then one launch of three passes
            // (the codebooks of the tuning run are updated; they are scratch)
            for (int r = 0; r < 2 && st == PQ_OK; ++r) {
                if (r == 1) cudaEventRecord(e0, s);
                const cudaError_t ce = cudaMemsetAsync(sync, 0, nsync * sizeof(int), s);
                st = ce == cudaSuccess ? launch_pq_fit_persistent_tc(p, r == 0 ? 1 : 3, sync, nullptr, s)
                                       : cuda_check(ce, "pq_tune_chunked");
            }
        } else {
            // one pass to warm up, then the mean of three (the codebooks are not updated)
            for (int r = 0; r < 4 && st == PQ_OK; ++r) {
                if (r == 1) cudaEventRecord(e0, s);
                st = launch_pq_pass_f32(p, s);
            }
        }
        if (st != PQ_OK) break;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = cuda_check(cudaGetLastError(), "pq_tune_chunked");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.0f;
        if (ms < bms) {
            bms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PQ_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[tune_key(off, n_chunks, D, M, Ks, prec, sms)] = best;
    }
    if (best_per) *best_per = best;
    if (best_ms) *best_ms = bms;
    return ws.status;
}

void clear_tuning()
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
}

}  // namespace pqgb
