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

}  // namespace

int run_pq_fit_chunked(const float *X, const int64_t *off, int n_chunks, int D, int M, int Ks, int iters,
                       uint64_t seed, int prec, float *global_cb, uint8_t *codes, double *rmse, cudaStream_t s)
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

    // (2) batched Lloyd iterations: blocks shared out in proportion to the rows
    ChunkTableParams tp;
    tp.n = n_chunks;
    tp.blk[0] = 0;
    PqPass base;
    base.N = N;
    base.M = M;
    const int per = tc ? std::max(1, sms / std::max(1, M / tc_pass_group())) : pq_pass_blocks_per_subspace(base);
    for (int c = 0; c <= n_chunks; ++c) tp.off[c] = off[c];
    for (int c = 0; c < n_chunks; ++c) {
        const int64_t rows = off[c + 1] - off[c];
        int64_t g = std::max<int64_t>(1, (int64_t)std::llround((double)per * (double)rows / (double)N));
        g = std::min<int64_t>(g, tc ? (rows + 127) / 128 : (rows + 255) / 256);
        tp.blk[c + 1] = tp.blk[c] + (int)std::max<int64_t>(1, g);
    }
    const int gx = tp.blk[n_chunks];
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
    p.part = ws.get<double>((size_t)gx * M * Ks * ds);
    p.part_cnt = ws.get<int>((size_t)gx * M * Ks);
    if (ws.status) return ws.status;
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
    for (int t = 0; t < iters; ++t) {
        if (tc) {
            PQ_TRY(launch_pq_pass_tc(p, s));
            PQ_TRY(launch_pq_finalize_residual(p.part, p.part_cnt, gx, M, Ks, ds, Cl, nullptr, s, n_chunks, d_blk));
        } else {
            PQ_TRY(launch_pq_pass_f32(p, s));
            PQ_TRY(launch_pq_finalize(p.part, p.part_cnt, gx, M, Ks, ds, Cl, nullptr, s, n_chunks, d_blk));
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
    PQ_TRY(pq_fit(pool, npool, D, M, Ks, iters, seed, prec, nullptr, global_cb, nullptr, s));
    PQ_TRY(pq_encode(X, N, D, M, Ks, global_cb, prec, codes, sse, nullptr, s));
    if (rmse) {
        double h = 0.0;
        PQ_TRY_CUDA(cudaMemcpyAsync(&h, sse, sizeof(double), cudaMemcpyDeviceToHost, s));
        PQ_TRY_CUDA(cudaStreamSynchronize(s));
        *rmse = std::sqrt(h / ((double)N * (double)D));
    }
    return ws.status;
}

}  // namespace pqgb
