// api.cu -- the extern "C" entry points of libpqgb.so (declared in pqgb.h):
// argument validation, stream-ordered scratch, and the order of kernels that
// makes up PQ fit / encode / decode-RMSE (Sec. 2.1, Sec. 3) and the inverted
// index build / query (Sec. 2.2, Sec. 3.1).
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace pqgb {

static std::atomic<int64_t> g_launches{0};
static thread_local char g_msg[512] = "";
static std::mutex g_err_mu;
static int *g_err_word[64] = {};

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int fail(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return status;
}

void clear_error() { g_msg[0] = 0; }

// Failure-injection hooks for tests (pq_test_*): the seeding's poll budget, and an
// allocation that fails after a given number of successful ones (-1: never).
static std::atomic<unsigned> g_seed_spin{kSpinLimit};
static std::atomic<int> g_fail_alloc_after{-1};
unsigned seeding_spin_limit() { return g_seed_spin.load(std::memory_order_relaxed); }

int cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) return fail(PQ_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(PQ_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int *device_error_word(int device)
{
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_err_mu);
    if (!g_err_word[device]) {
        int *p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
        g_err_word[device] = p;
    }
    return g_err_word[device];
}

// One non-blocking copy stream per device (created on first use, never destroyed), for copies
// that run beside the caller's stream and are joined to it with events.
static cudaStream_t g_copy_stream[64];
static std::mutex g_copy_mu;
static cudaStream_t copy_stream(int device)
{
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_copy_mu);
    if (!g_copy_stream[device] && cudaStreamCreateWithFlags(&g_copy_stream[device], cudaStreamNonBlocking) != cudaSuccess)
        g_copy_stream[device] = nullptr;
    return g_copy_stream[device];
}

struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static std::atomic<bool> g_prof_on{false};
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_ev_pool;

static cudaEvent_t take_event()
{
    if (!g_ev_pool.empty()) {
        cudaEvent_t e = g_ev_pool.back();
        g_ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

ProfScope::ProfScope(const char *name, cudaStream_t st) : s(st)
{
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfRec r{name, take_event(), take_event()};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, s);
    idx = (int)g_prof.size();
    g_prof.push_back(r);
}

ProfScope::~ProfScope()
{
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_prof[idx].b, s);
}

void *Scratch::raw(size_t bytes, bool zero)
{
    if (status) return nullptr;
    void *p = nullptr;
    const size_t b = (bytes + 255) & ~size_t(255);
    for (int left = g_fail_alloc_after.load(); left >= 0;) {
        if (left == 0) {
            if (g_fail_alloc_after.compare_exchange_weak(left, -1)) {
                status = fail(PQ_ENOMEM, "cudaMallocAsync: injected allocation failure");
                return nullptr;
            }
        } else if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
            break;
        }
    }
    cudaError_t e = cudaMallocAsync(&p, b ? b : 256, s);
    if (e != cudaSuccess) { status = cuda_check(e, "cudaMallocAsync"); return nullptr; }
    ptrs.push_back(p);
    if (zero) {
        e = cudaMemsetAsync(p, 0, b ? b : 256, s);
        if (e != cudaSuccess) { status = cuda_check(e, "cudaMemsetAsync"); return nullptr; }
    }
    return p;
}

Scratch::~Scratch()
{
    for (void *p : ptrs) cudaFreeAsync(p, s);
}

}  // namespace pqgb

using namespace pqgb;

struct ivf_index {
    int device = 0;
    int64_t N = 0;
    int D = 0, M = 0, nlist = 0;
    int kind = 0;                  // 0: raw-space coarse centroids; 1: centre codes (code-space)
    int Ks = 0;                    // code-space: codewords per subspace of `cb`
    float *coarse = nullptr;       // [nlist][D] (code-space: the decoded centre codes)
    float *half_norm = nullptr;    // [nlist]
    float *maxes = nullptr;        // [2]
    uint8_t *centers = nullptr;    // code-space: [nlist][M] centre codes
    float *cb = nullptr;           // code-space: [M][Ks][D/M] the codebooks the codes were made with
    int64_t *offsets = nullptr;    // [nlist+1]
    int64_t *ids = nullptr;        // [N]
    uint8_t *codes = nullptr;      // [N][M]
};

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int check_pq_shape(int64_t N, int D, int M, int Ks, bool need_ks_le_n)
{
    if (N < 0) return fail(PQ_EINVAL, "N=%lld must be >= 0", (long long)N);
    if (D <= 0 || M <= 0 || D % M != 0) return fail(PQ_EINVAL, "D=%d must be a positive multiple of M=%d", D, M);
    if (Ks < 1 || Ks > 256) return fail(PQ_EINVAL, "Ks=%d must be in [1, 256]", Ks);
    if (need_ks_le_n && N < Ks) return fail(PQ_EINVAL, "N=%lld must be >= Ks=%d", (long long)N, Ks);
    const int ds = D / M;
    if (ds > 32) return fail(PQ_EINVAL, "subspace width D/M=%d must be <= 32", ds);
    return PQ_OK;
}

int check_prec(int prec)
{
    if (prec != PQ_PREC_FP32 && prec != PQ_PREC_BF16) return fail(PQ_EINVAL, "prec=%d unknown", prec);
    return PQ_OK;
}

int run_pass(PqPass &p, int prec, cudaStream_t s)
{
    if (prec == PQ_PREC_BF16) {
        if (!tc_pass_supported(p.D, p.M, p.Ks))
            return fail(PQ_ENOTSUP, "BF16 tensor-core pass needs D/M == 8 and M even");
        return launch_pq_pass_tc(p, s);
    }
    return launch_pq_pass_f32(p, s);
}

int status_from_device(int *err_word, cudaStream_t s, int *host_err)
{
    PQ_TRY_CUDA(cudaMemcpyAsync(host_err, err_word, sizeof(int), cudaMemcpyDeviceToHost, s));
    PQ_TRY_CUDA(cudaStreamSynchronize(s));
    return PQ_OK;
}

// Seeding rows: all rows, or 100*Ks drawn with replacement.
int seed_codebooks(const float *X, int64_t N, int D, int M, int Ks, uint64_t seed, float *C, Scratch &ws, int *err,
                   cudaStream_t s, const char *tag = "kmeanspp")
{
    return launch_kmeanspp(X, N, D, M, Ks, seed, C, ws, err, s, tag);
}

// Lloyd iterations over PQ codebooks C (in place).
int lloyd(const float *X, int64_t N, int D, int M, int Ks, int iters, int prec, float *C, double *sse_dev,
          unsigned long long *counters /* [2]: rechecks, empties */, Scratch &ws, cudaStream_t s)
{
    PqPass p;
    p.X = X;
    p.N = N;
    p.D = D;
    p.M = M;
    p.Ks = Ks;
    p.ds = D / M;
    p.C = C;
    const bool tc = prec == PQ_PREC_BF16;
    p.gx = tc ? pq_pass_tc_blocks(p) : pq_pass_blocks_per_subspace(p);
    void *pb = ws.raw(Partials::bytes(p.gx, M, Ks, p.ds, 1), false);
    if (ws.status) return ws.status;
    p.part.carve(pb, p.gx, M, Ks, p.ds);
    p.rechecks = counters;
    for (int t = 0; t < iters; ++t) {
        p.sse = sse_dev ? sse_dev + t : nullptr;
        PQ_TRY(run_pass(p, prec, s));
        PQ_TRY(launch_pq_finalize(p.part, p.gx, M, Ks, p.ds, C, counters + 1, s));
    }
    return PQ_OK;
}

}  // namespace

extern "C" {

int pq_init_kmeanspp(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, uint64_t seed, float *codebooks,
                     void *stream)
{
    g_msg[0] = 0;
    PQ_TRY(check_pq_shape(N, D, M, Ks, true));
    if (!X || !codebooks) return fail(PQ_EINVAL, "null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    int *err = device_error_word(dev);
    if (!err) return fail(PQ_ENOMEM, "device error word");
    Scratch ws(s);
    PQ_TRY(seed_codebooks(X, N, D, M, Ks, seed, codebooks, ws, err, s));
    return ws.status;
}

int pq_fit(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, int32_t iters, uint64_t seed, int32_t prec,
           const float *init_codebooks, float *codebooks, pq_stats *stats, void *stream)
{
    g_msg[0] = 0;
    PQ_TRY(check_pq_shape(N, D, M, Ks, true));
    PQ_TRY(check_prec(prec));
    if (!X || !codebooks) return fail(PQ_EINVAL, "null pointer");
    if (!aligned16(X)) return fail(PQ_EINVAL, "X must be 16-byte aligned");
    if (iters < 0 || iters > PQ_STATS_MAX_ITERS) return fail(PQ_EINVAL, "iters=%d must be in [0, %d]", iters,
                                                             PQ_STATS_MAX_ITERS);
    if (prec == PQ_PREC_BF16 && !tc_pass_supported(D, M, Ks))
        return fail(PQ_ENOTSUP, "BF16 tensor-core pass needs D/M == 8 and M even");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t l0 = g_launches.load();
    int dev = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    int *err = device_error_word(dev);
    if (!err) return fail(PQ_ENOMEM, "device error word");
    Scratch ws(s);
    const size_t cb_bytes = (size_t)M * Ks * (D / M) * sizeof(float);
    if (init_codebooks) {
        if (init_codebooks != codebooks)
            PQ_TRY_CUDA(cudaMemcpyAsync(codebooks, init_codebooks, cb_bytes, cudaMemcpyDeviceToDevice, s));
    } else {
        PQ_TRY(seed_codebooks(X, N, D, M, Ks, seed, codebooks, ws, err, s));
    }
    double *sse = stats ? ws.get<double>(PQ_STATS_MAX_ITERS, true) : nullptr;
    unsigned long long *counters = ws.get<unsigned long long>(2, true);
    if (ws.status) return ws.status;
    PQ_TRY(lloyd(X, N, D, M, Ks, iters, prec, codebooks, sse, counters, ws, s));
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        unsigned long long hc[2];
        PQ_TRY_CUDA(cudaMemcpyAsync(stats->sse, sse, sizeof(double) * iters, cudaMemcpyDeviceToHost, s));
        PQ_TRY_CUDA(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
        int herr = 0;
        PQ_TRY(status_from_device(err, s, &herr));
        stats->iters = iters;
        stats->fp64_rechecks = (int64_t)hc[0];
        stats->empty_clusters = (int64_t)hc[1];
        stats->kernel_launches = g_launches.load() - l0;
        if (herr) {
            cudaMemsetAsync(err, 0, sizeof(int), s);
            return fail(herr, "device-side failure %d during pq_fit", herr);
        }
    }
    return ws.status;
}

int pq_fit_encode_host(const float *X_host, int64_t N, int32_t D, int32_t M, int32_t Ks, int32_t iters,
                       uint64_t seed, int32_t prec, float *codebooks_host, uint8_t *codes_host, void *stream)
{
    g_msg[0] = 0;
    PQ_TRY(check_pq_shape(N, D, M, Ks, true));
    PQ_TRY(check_prec(prec));
    if (!X_host || !codebooks_host) return fail(PQ_EINVAL, "null pointer");
    if (!aligned16(X_host)) return fail(PQ_EINVAL, "X_host must be 16-byte aligned");
    if (iters < 0 || iters > PQ_STATS_MAX_ITERS) return fail(PQ_EINVAL, "iters=%d must be in [0, %d]", iters,
                                                             PQ_STATS_MAX_ITERS);
    if (prec == PQ_PREC_BF16 && !tc_pass_supported(D, M, Ks))
        return fail(PQ_ENOTSUP, "BF16 tensor-core pass needs D/M == 8 and M even");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, X_host) != cudaSuccess || at.type != cudaMemoryTypeHost || !at.devicePointer) {
        cudaGetLastError();
        return fail(PQ_EINVAL, "X_host must be page-locked host memory");
    }
    const float *X_map = static_cast<const float *>(at.devicePointer);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    int *err = device_error_word(dev);
    if (!err) return fail(PQ_ENOMEM, "device error word");
    cudaStream_t cs = copy_stream(dev);
    if (!cs) return fail(PQ_ECUDA, "copy stream");
    const int Ds = D / M;
    const size_t cb_bytes = (size_t)M * Ks * Ds * sizeof(float);
    Scratch ws(s);
    float *Xd = ws.get<float>((size_t)N * D);
    float *cb = ws.get<float>((size_t)M * Ks * Ds);
    uint8_t *codes = codes_host ? ws.get<uint8_t>((size_t)N * M) : nullptr;
    unsigned long long *counters = ws.get<unsigned long long>(2, true);
    if (ws.status) return ws.status;
    // When N > 100*Ks the seeding needs only its subsample rows: they are gathered from host
    // memory first (the copy would share the host link with the gather), then seeded while X
    // is copied on the second stream.
    const int64_t cap = 100LL * Ks;
    float *G = N > cap ? ws.get<float>((size_t)cap * D) : nullptr;
    if (ws.status) return ws.status;
    if (G) PQ_TRY(launch_gather_subsample(X_map, N, D, Ks, seed, G, s));
    cudaEvent_t ready = nullptr, copied = nullptr;
    PQ_TRY_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    if (cudaEventCreateWithFlags(&copied, cudaEventDisableTiming) != cudaSuccess) {
        cudaEventDestroy(ready);
        return fail(PQ_ECUDA, "event");
    }
    struct Events {
        cudaEvent_t a, b;
        ~Events()
        {
            cudaEventDestroy(a);  // released once pending work completes
            cudaEventDestroy(b);
        }
    } ev{ready, copied};
    PQ_TRY_CUDA(cudaEventRecord(ready, s));
    PQ_TRY_CUDA(cudaStreamWaitEvent(cs, ready, 0));
    PQ_TRY_CUDA(cudaMemcpyAsync(Xd, X_host, (size_t)N * D * sizeof(float), cudaMemcpyHostToDevice, cs));
    PQ_TRY_CUDA(cudaEventRecord(copied, cs));
    // every return from here on (errors included) leaves the caller's stream behind the copy,
    // so the scratch is never released while the copy writes it
    struct JoinCopy {
        cudaStream_t s;
        cudaEvent_t e;
        ~JoinCopy() { cudaStreamWaitEvent(s, e, 0); }
    } join{s, copied};
    if (G) {
        // seeding the gathered rows gives the codebooks that seeding all of X gives
        PQ_TRY(seed_codebooks(G, cap, D, M, Ks, seed, cb, ws, err, s));
        PQ_TRY_CUDA(cudaStreamWaitEvent(s, copied, 0));
    } else {
        PQ_TRY_CUDA(cudaStreamWaitEvent(s, copied, 0));
        PQ_TRY(seed_codebooks(Xd, N, D, M, Ks, seed, cb, ws, err, s));
    }
    PQ_TRY(lloyd(Xd, N, D, M, Ks, iters, prec, cb, nullptr, counters, ws, s));
    if (codes) {
        PqPass p;
        p.X = Xd;
        p.N = N;
        p.D = D;
        p.M = M;
        p.Ks = Ks;
        p.ds = Ds;
        p.C = cb;
        p.codes = codes;
        PQ_TRY(run_pass(p, prec, s));
        PQ_TRY_CUDA(cudaMemcpyAsync(codes_host, codes, (size_t)N * M, cudaMemcpyDeviceToHost, s));
    }
    PQ_TRY_CUDA(cudaMemcpyAsync(codebooks_host, cb, cb_bytes, cudaMemcpyDeviceToHost, s));
    return ws.status;
}

int pq_encode(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, const float *codebooks, int32_t prec,
              uint8_t *codes, double *sse, pq_stats *stats, void *stream)
{
    g_msg[0] = 0;
    PQ_TRY(check_pq_shape(N, D, M, Ks, false));
    PQ_TRY(check_prec(prec));
    if (!codebooks || (N > 0 && (!X || !codes))) return fail(PQ_EINVAL, "null pointer");
    if (N > 0 && !aligned16(X)) return fail(PQ_EINVAL, "X must be 16-byte aligned");
    if (prec == PQ_PREC_BF16 && !tc_pass_supported(D, M, Ks))
        return fail(PQ_ENOTSUP, "BF16 tensor-core pass needs D/M == 8 and M even");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t l0 = g_launches.load();
    if (sse) PQ_TRY_CUDA(cudaMemsetAsync(sse, 0, sizeof(double), s));
    if (N == 0) return PQ_OK;
    Scratch ws(s);
    unsigned long long *counters = stats ? ws.get<unsigned long long>(1, true) : nullptr;
    if (ws.status) return ws.status;
    PqPass p;
    p.X = X;
    p.N = N;
    p.D = D;
    p.M = M;
    p.Ks = Ks;
    p.ds = D / M;
    p.C = codebooks;
    p.codes = codes;
    p.sse = sse;
    p.rechecks = counters;
    PQ_TRY(run_pass(p, prec, s));
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        unsigned long long hc = 0;
        PQ_TRY_CUDA(cudaMemcpyAsync(&hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
        PQ_TRY_CUDA(cudaStreamSynchronize(s));
        stats->fp64_rechecks = (int64_t)hc;
        stats->kernel_launches = g_launches.load() - l0;
    }
    return ws.status;
}

int pq_decode_rmse(const uint8_t *codes, const float *codebooks, const float *X, int64_t N, int32_t D, int32_t M,
                   int32_t Ks, float *Xhat, double *rmse, void *stream)
{
    g_msg[0] = 0;
    PQ_TRY(check_pq_shape(N, D, M, Ks, false));
    if (!codebooks || (N > 0 && !codes)) return fail(PQ_EINVAL, "null pointer");
    if (N == 0 && rmse) {
        *rmse = 0.0;
        return PQ_OK;
    }
    if (!Xhat && !(X && rmse)) return fail(PQ_EINVAL, "nothing to compute: give Xhat and/or X with rmse");
    if (X && !rmse) return fail(PQ_EINVAL, "X given without rmse");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch ws(s);
    double *sse = X ? ws.get<double>(1, true) : nullptr;
    if (ws.status) return ws.status;
    if (N > 0) PQ_TRY(launch_decode_rmse(codes, codebooks, X, N, D, M, Ks, Xhat, sse, s));
    if (X) {
        double h = 0.0;
        PQ_TRY_CUDA(cudaMemcpyAsync(&h, sse, sizeof(double), cudaMemcpyDeviceToHost, s));
        PQ_TRY_CUDA(cudaStreamSynchronize(s));
        *rmse = N > 0 ? sqrt(h / ((double)N * (double)D)) : 0.0;
    }
    return ws.status;
}

static int chunked_entry(const float *X, const int64_t *chunk_offsets, int32_t n_chunks, int32_t D, int32_t M, int32_t Ks,
                   int32_t iters, uint64_t seed, int32_t prec, float *codebooks, uint8_t *codes, double *rmse,
                   void *stream, bool weighted)
{
    g_msg[0] = 0;
    if (!X || !chunk_offsets || !codebooks || !codes) return fail(PQ_EINVAL, "null pointer");
    if (n_chunks < 1 || n_chunks > kMaxSeedChunks) return fail(PQ_EINVAL, "n_chunks=%d must be in [1, %d]", n_chunks,
                                                               kMaxSeedChunks);
    if (chunk_offsets[0] != 0) return fail(PQ_EINVAL, "chunk_offsets[0] must be 0");
    for (int c = 0; c < n_chunks; ++c)
        if (chunk_offsets[c + 1] - chunk_offsets[c] < Ks)
            return fail(PQ_EINVAL, "chunk %d has %lld rows, fewer than Ks=%d", c,
                        (long long)(chunk_offsets[c + 1] - chunk_offsets[c]), Ks);
    const int64_t N = chunk_offsets[n_chunks];
    PQ_TRY(check_pq_shape(N, D, M, Ks, true));
    PQ_TRY(check_prec(prec));
    if (!aligned16(X)) return fail(PQ_EINVAL, "X must be 16-byte aligned");
    if (iters < 0 || iters > PQ_STATS_MAX_ITERS) return fail(PQ_EINVAL, "iters=%d must be in [0, %d]", iters,
                                                             PQ_STATS_MAX_ITERS);
    if (prec == PQ_PREC_BF16 && !tc_pass_supported(D, M, Ks))
        return fail(PQ_ENOTSUP, "BF16 tensor-core pass needs D/M == 8 and M even");
    if ((int64_t)n_chunks * Ks < Ks) return fail(PQ_EINVAL, "empty centroid dataset");
    return run_pq_fit_chunked(X, chunk_offsets, n_chunks, D, M, Ks, iters, seed, prec, codebooks, codes, rmse,
                              static_cast<cudaStream_t>(stream), weighted);
}

int pq_fit_chunked(const float *X, const int64_t *chunk_offsets, int32_t n_chunks, int32_t D, int32_t M, int32_t Ks,
                   int32_t iters, uint64_t seed, int32_t prec, float *codebooks, uint8_t *codes, double *rmse,
                   void *stream)
{
    return chunked_entry(X, chunk_offsets, n_chunks, D, M, Ks, iters, seed, prec, codebooks, codes, rmse, stream, false);
}

int pq_fit_chunked_weighted(const float *X, const int64_t *chunk_offsets, int32_t n_chunks, int32_t D, int32_t M,
                            int32_t Ks, int32_t iters, uint64_t seed, int32_t prec, float *codebooks, uint8_t *codes,
                            double *rmse, void *stream)
{
    return chunked_entry(X, chunk_offsets, n_chunks, D, M, Ks, iters, seed, prec, codebooks, codes, rmse, stream, true);
}

int pq_tune_chunked(const float *X, const int64_t *chunk_offsets, int32_t n_chunks, int32_t D, int32_t M, int32_t Ks,
                    int32_t prec, int32_t *ctas, float *pass_ms, void *stream)
{
    g_msg[0] = 0;
    if (!X || !chunk_offsets) return fail(PQ_EINVAL, "null pointer");
    if (n_chunks < 1 || n_chunks > kMaxSeedChunks) return fail(PQ_EINVAL, "n_chunks=%d must be in [1, %d]", n_chunks,
                                                               kMaxSeedChunks);
    if (chunk_offsets[0] != 0) return fail(PQ_EINVAL, "chunk_offsets[0] must be 0");
    for (int c = 0; c < n_chunks; ++c)
        if (chunk_offsets[c + 1] - chunk_offsets[c] < Ks)
            return fail(PQ_EINVAL, "chunk %d has %lld rows, fewer than Ks=%d", c,
                        (long long)(chunk_offsets[c + 1] - chunk_offsets[c]), Ks);
    PQ_TRY(check_pq_shape(chunk_offsets[n_chunks], D, M, Ks, true));
    PQ_TRY(check_prec(prec));
    if (!aligned16(X)) return fail(PQ_EINVAL, "X must be 16-byte aligned");
    if (prec == PQ_PREC_BF16 && !tc_pass_supported(D, M, Ks))
        return fail(PQ_ENOTSUP, "BF16 tensor-core pass needs D/M == 8 and M even");
    int best = 0;
    float ms = 0.0f;
    PQ_TRY(run_pq_tune_chunked(X, chunk_offsets, n_chunks, D, M, Ks, prec, &best, &ms, static_cast<cudaStream_t>(stream)));
    if (ctas) *ctas = best;
    if (pass_ms) *pass_ms = ms;
    return PQ_OK;
}

int pq_tune_clear(void)
{
    clear_tuning();
    return PQ_OK;
}

static int check_softpq(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, const float *codebooks, float tau)
{
    if (!codebooks || (N > 0 && !X)) return fail(PQ_EINVAL, "null pointer");
    if (N < 0) return fail(PQ_EINVAL, "N=%lld must be >= 0", (long long)N);
    if (D <= 0 || M <= 0 || D % M != 0) return fail(PQ_EINVAL, "D=%d must be a positive multiple of M=%d", D, M);
    if (Ks < 1 || Ks > 256) return fail(PQ_EINVAL, "Ks=%d must be in [1, 256]", Ks);
    if (!(tau > 0.0f) || !std::isfinite(tau)) return fail(PQ_EINVAL, "tau must be positive and finite");
    if (!softpq_supported(D, M)) return fail(PQ_ENOTSUP, "soft PQ supports D/M in {4, 8, 16}");
    if (N > 0 && !aligned16(X)) return fail(PQ_EINVAL, "X must be 16-byte aligned");
    return PQ_OK;
}

int softpq_forward(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, const float *codebooks, float tau,
                   float *loss, void *stream)
{
    g_msg[0] = 0;
    PQ_TRY(check_softpq(X, N, D, M, Ks, codebooks, tau));
    if (!loss) return fail(PQ_EINVAL, "null loss");
    return run_softpq_forward(X, N, D, M, Ks, codebooks, tau, loss, static_cast<cudaStream_t>(stream));
}

int softpq_backward(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, const float *codebooks, float tau,
                    const float *grad_loss, float *dcodebooks, float *dX, void *stream)
{
    g_msg[0] = 0;
    PQ_TRY(check_softpq(X, N, D, M, Ks, codebooks, tau));
    if (!dcodebooks) return fail(PQ_EINVAL, "null dcodebooks");
    if (dX && !aligned16(dX)) return fail(PQ_EINVAL, "dX must be 16-byte aligned");
    return run_softpq_backward(X, N, D, M, Ks, codebooks, tau, grad_loss, dcodebooks, dX,
                               static_cast<cudaStream_t>(stream));
}

int ivf_build(const float *X, const uint8_t *codes, int64_t N, int32_t D, int32_t M, int32_t nlist, int32_t iters,
              uint64_t seed, int32_t prec, ivf_index **out, void *stream)
{
    g_msg[0] = 0;
    if (!out) return fail(PQ_EINVAL, "null output handle");
    *out = nullptr;
    if (!X || !codes) return fail(PQ_EINVAL, "null pointer");
    if (N < 1 || N >= (1LL << 31)) return fail(PQ_EINVAL, "N=%lld must be in [1, 2^31)", (long long)N);
    if (D <= 0 || M <= 0 || D % M != 0) return fail(PQ_EINVAL, "D=%d must be a positive multiple of M=%d", D, M);
    if (nlist < 1 || nlist > N) return fail(PQ_EINVAL, "nlist=%d must be in [1, N]", nlist);
    if (nlist > 16384) return fail(PQ_ENOTSUP, "nlist=%d exceeds 16384", nlist);
    if (D > 256) return fail(PQ_ENOTSUP, "ivf_build supports D <= 256");
    if (iters < 0) return fail(PQ_EINVAL, "iters=%d must be >= 0", iters);
    PQ_TRY(check_prec(prec));
    if (!aligned16(X)) return fail(PQ_EINVAL, "X must be 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    int *err = device_error_word(dev);
    if (!err) return fail(PQ_ENOMEM, "device error word");

    ivf_index *idx = new ivf_index();
    idx->device = dev;
    idx->N = N;
    idx->D = D;
    idx->M = M;
    idx->nlist = nlist;
    auto cleanup = [&](int st) {
        ivf_free(idx);
        return st;
    };
    if (cudaMalloc(&idx->coarse, (size_t)nlist * D * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&idx->half_norm, (size_t)nlist * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&idx->maxes, 2 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&idx->offsets, (size_t)(nlist + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&idx->ids, (size_t)N * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&idx->codes, (size_t)N * M) != cudaSuccess)
        return cleanup(fail(PQ_ENOMEM, "index allocation"));
    int st = PQ_OK;
    {
        Scratch ws(s);
        int32_t *lst = ws.get<int32_t>((size_t)N);
        unsigned *xrange = ws.get<unsigned>(2);
        if (ws.status) return cleanup(ws.status);
        CoarseBound b{idx->half_norm, idx->maxes};
        ListMeanScratch lm;
        if (iters > 0) st = list_mean_scratch(N, D, nlist, ws, lm);
        if (st) return cleanup(st);
        if (iters > 0) st = launch_x_exponent_range(X, N, D, xrange, s);
        if (st) return cleanup(st);
        st = seed_codebooks(X, N, D, 1, nlist, seed, idx->coarse, ws, err, s, "kmeanspp_coarse");
        for (int t = 0; st == PQ_OK && t < iters; ++t) {
            st = launch_coarse_norms(idx->coarse, nlist, D, b, s);
            if (!st) st = coarse_assign(X, N, D, idx->coarse, nlist, b, lst, ws, prec, s);
            if (!st) st = bucket_rows(lst, N, nlist, nullptr, M, idx->offsets, idx->ids, nullptr, ws, s);
            if (!st) st = launch_list_mean(X, D, idx->offsets, idx->ids, nlist, xrange, idx->coarse, lm, s);
        }
        if (!st) st = launch_coarse_norms(idx->coarse, nlist, D, b, s);
        if (!st) st = coarse_assign(X, N, D, idx->coarse, nlist, b, lst, ws, prec, s);
        if (!st) st = bucket_rows(lst, N, nlist, codes, M, idx->offsets, idx->ids, idx->codes, ws, s);
        if (!st) st = ws.status;
    }
    if (st) return cleanup(st);
    int herr = 0;
    st = status_from_device(err, s, &herr);
    if (st) return cleanup(st);
    if (herr) {
        cudaMemsetAsync(err, 0, sizeof(int), s);
        return cleanup(fail(herr, "device-side failure %d during ivf_build", herr));
    }
    *out = idx;
    return PQ_OK;
}

int ivf_build_codes(const uint8_t *codes, const float *codebooks, int64_t N, int32_t D, int32_t M, int32_t Ks,
                    int32_t nlist, int32_t iters, uint64_t seed, int32_t prec, ivf_index **out, void *stream)
{
    g_msg[0] = 0;
    if (!out) return fail(PQ_EINVAL, "null output handle");
    *out = nullptr;
    if (!codes || !codebooks) return fail(PQ_EINVAL, "null pointer");
    if (N < 1 || N >= (1LL << 31)) return fail(PQ_EINVAL, "N=%lld must be in [1, 2^31)", (long long)N);
    PQ_TRY(check_pq_shape(N, D, M, Ks, false));
    if (nlist < 1 || nlist > N) return fail(PQ_EINVAL, "nlist=%d must be in [1, N]", nlist);
    if (nlist > 16384) return fail(PQ_ENOTSUP, "nlist=%d exceeds 16384", nlist);
    if (D > 256) return fail(PQ_ENOTSUP, "ivf_build_codes supports D <= 256");
    if (iters < 0) return fail(PQ_EINVAL, "iters=%d must be >= 0", iters);
    PQ_TRY(check_prec(prec));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    int *err = device_error_word(dev);
    if (!err) return fail(PQ_ENOMEM, "device error word");
    ivf_index *idx = new ivf_index();
    idx->device = dev;
    idx->N = N;
    idx->D = D;
    idx->M = M;
    idx->nlist = nlist;
    idx->kind = 1;
    idx->Ks = Ks;
    auto cleanup = [&](int st) {
        ivf_free(idx);
        return st;
    };
    const size_t cbn = (size_t)M * Ks * (D / M);
    if (cudaMalloc(&idx->coarse, (size_t)nlist * D * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&idx->half_norm, (size_t)nlist * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&idx->maxes, 2 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&idx->centers, (size_t)nlist * M) != cudaSuccess ||
        cudaMalloc(&idx->cb, cbn * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&idx->offsets, (size_t)(nlist + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&idx->ids, (size_t)N * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&idx->codes, (size_t)N * M) != cudaSuccess)
        return cleanup(fail(PQ_ENOMEM, "index allocation"));
    int st = PQ_OK;
    {
        Scratch ws(s);
        if (cudaMemcpyAsync(idx->cb, codebooks, cbn * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return cleanup(fail(PQ_ECUDA, "codebook copy"));
        CoarseBound b{idx->half_norm, idx->maxes};
        st = run_ivf_build_codes(codes, idx->cb, N, D, M, Ks, nlist, iters, seed, prec, idx->coarse, b, idx->centers,
                                 idx->offsets, idx->ids, idx->codes, ws, s);
        if (!st) st = ws.status;
    }
    if (st) return cleanup(st);
    int herr = 0;
    st = status_from_device(err, s, &herr);
    if (st) return cleanup(st);
    if (herr) {
        cudaMemsetAsync(err, 0, sizeof(int), s);
        return cleanup(fail(herr, "device-side failure %d during ivf_build_codes", herr));
    }
    *out = idx;
    return PQ_OK;
}

int ivf_search(const ivf_index *index, const float *codebooks, int32_t Ks, const float *Q, int64_t nq,
               int32_t nprobe, int32_t k, int64_t *ids, float *dists, void *stream)
{
    g_msg[0] = 0;
    if (!index || !codebooks || !Q || !ids || !dists) return fail(PQ_EINVAL, "null pointer");
    if (Ks < 1 || Ks > 256) return fail(PQ_EINVAL, "Ks=%d must be in [1, 256]", Ks);
    if (nq < 0) return fail(PQ_EINVAL, "nq must be >= 0");
    if (nprobe < 1 || nprobe > index->nlist)
        return fail(PQ_EINVAL, "nprobe=%d must be in [1, nlist=%d]", nprobe, index->nlist);
    if (k < 1 || k > 1024) return fail(PQ_EINVAL, "k=%d must be in [1, 1024]", k);
    if (nq == 0) return PQ_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch ws(s);
    CoarseBound b{index->half_norm, index->maxes};
    SearchArgs a;
    a.Q = Q;
    a.nq = nq;
    a.D = index->D;
    a.M = index->M;
    a.Ks = Ks;
    a.nlist = index->nlist;
    a.nprobe = nprobe;
    a.k = k;
    a.coarse = index->coarse;
    a.probe_sub = index->kind == 1 ? index->D / index->M : 0;
    a.cb = &b;
    a.offsets = index->offsets;
    a.ids = index->ids;
    a.list_codes = index->codes;
    a.codebooks = codebooks;
    a.out_ids = ids;
    a.out_d = dists;
    PQ_TRY(run_search(a, ws, s));
    return ws.status;
}

int ivf_get_info(const ivf_index *index, int64_t *N, int32_t *D, int32_t *M, int32_t *nlist)
{
    if (!index) return fail(PQ_EINVAL, "null index");
    if (N) *N = index->N;
    if (D) *D = index->D;
    if (M) *M = index->M;
    if (nlist) *nlist = index->nlist;
    return PQ_OK;
}

int ivf_copy_coarse(const ivf_index *index, float *coarse, void *stream)
{
    if (!index || !coarse) return fail(PQ_EINVAL, "null pointer");
    PQ_TRY_CUDA(cudaMemcpyAsync(coarse, index->coarse, (size_t)index->nlist * index->D * sizeof(float),
                                cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
    return PQ_OK;
}

}  // extern "C"

namespace {

// Replaces the lists of `dst` by the merge of its lists and the CSR set (b_off, b_ids, b_codes)
// of b_n rows, whose ids are shifted by dst->N.  Synchronizes the stream before freeing the old
// arrays.
int merge_into(ivf_index *dst, const int64_t *b_off, const int64_t *b_ids, const uint8_t *b_codes, int64_t b_n,
               cudaStream_t s)
{
    const int64_t total = dst->N + b_n;
    if (total >= (1LL << 31)) return fail(PQ_ENOTSUP, "an index holds fewer than 2^31 rows");
    int64_t *off = nullptr, *ids = nullptr;
    uint8_t *codes = nullptr;
    if (cudaMalloc(&off, (size_t)(dst->nlist + 1) * sizeof(int64_t)) != cudaSuccess ||
        (total > 0 && cudaMalloc(&ids, (size_t)total * sizeof(int64_t)) != cudaSuccess) ||
        (total > 0 && cudaMalloc(&codes, (size_t)total * dst->M) != cudaSuccess)) {
        cudaFree(off);
        cudaFree(ids);
        return fail(PQ_ENOMEM, "merged list allocation");
    }
    const int st = launch_merge_lists(dst->offsets, dst->ids, dst->codes, dst->N, b_off, b_ids, b_codes, b_n, dst->N,
                                      dst->nlist, dst->M, off, ids, codes, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (st != PQ_OK || e != cudaSuccess) {
        cudaFree(off);
        cudaFree(ids);
        cudaFree(codes);
        return st != PQ_OK ? st : cuda_check(e, "merge");
    }
    cudaFree(dst->offsets);
    cudaFree(dst->ids);
    cudaFree(dst->codes);
    dst->offsets = off;
    dst->ids = ids;
    dst->codes = codes;
    dst->N = total;
    return PQ_OK;
}

int copy_device(void **dst, const void *src, size_t bytes)
{
    if (!src) return PQ_OK;
    if (cudaMalloc(dst, bytes) != cudaSuccess) return fail(PQ_ENOMEM, "index allocation");
    PQ_TRY_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyDeviceToDevice));
    return PQ_OK;
}

}  // namespace

extern "C" {

int ivf_clone_empty(const ivf_index *src, ivf_index **out)
{
    g_msg[0] = 0;
    if (!src || !out) return fail(PQ_EINVAL, "null pointer");
    *out = nullptr;
    ivf_index *idx = new ivf_index();
    idx->device = src->device;
    idx->N = 0;
    idx->D = src->D;
    idx->M = src->M;
    idx->nlist = src->nlist;
    idx->kind = src->kind;
    idx->Ks = src->Ks;
    const size_t cbn = (size_t)src->M * src->Ks * (src->D / src->M);
    int st = copy_device((void **)&idx->coarse, src->coarse, (size_t)src->nlist * src->D * sizeof(float));
    if (!st) st = copy_device((void **)&idx->half_norm, src->half_norm, (size_t)src->nlist * sizeof(float));
    if (!st) st = copy_device((void **)&idx->maxes, src->maxes, 2 * sizeof(float));
    if (!st && src->kind == 1) st = copy_device((void **)&idx->centers, src->centers, (size_t)src->nlist * src->M);
    if (!st && src->kind == 1) st = copy_device((void **)&idx->cb, src->cb, cbn * sizeof(float));
    if (!st && cudaMalloc(&idx->offsets, (size_t)(src->nlist + 1) * sizeof(int64_t)) != cudaSuccess)
        st = fail(PQ_ENOMEM, "index allocation");
    if (!st && cudaMemset(idx->offsets, 0, (size_t)(src->nlist + 1) * sizeof(int64_t)) != cudaSuccess)
        st = fail(PQ_ECUDA, "cudaMemset");
    if (st) {
        ivf_free(idx);
        return st;
    }
    *out = idx;
    return PQ_OK;
}

int ivf_add(ivf_index *index, const float *X, const uint8_t *codes, int64_t n, int32_t prec, void *stream)
{
    g_msg[0] = 0;
    if (!index || !codes) return fail(PQ_EINVAL, "null pointer");
    if (n < 0) return fail(PQ_EINVAL, "n must be >= 0");
    PQ_TRY(check_prec(prec));
    if (index->kind == 0 && (!X || !aligned16(X))) return fail(PQ_EINVAL, "X (16-byte aligned) is required");
    if (n == 0) return PQ_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int D = index->D, M = index->M, nlist = index->nlist;
    Scratch ws(s);
    int32_t *lst = ws.get<int32_t>((size_t)n);
    int64_t *b_off = ws.get<int64_t>((size_t)nlist + 1);
    int64_t *b_ids = ws.get<int64_t>((size_t)n);
    uint8_t *b_codes = ws.get<uint8_t>((size_t)n * M);
    if (ws.status) return ws.status;
    CoarseBound b{index->half_norm, index->maxes};
    if (index->kind == 0) {
        PQ_TRY(coarse_assign(X, n, D, index->coarse, nlist, b, lst, ws, prec, s));
    } else {
        float *Xhat = ws.get<float>((size_t)n * D);
        if (ws.status) return ws.status;
        PQ_TRY(launch_decode_codes(codes, index->cb, n, D, M, index->Ks, Xhat, s));
        PQ_TRY(coarse_assign(Xhat, n, D, index->coarse, nlist, b, lst, ws, prec, s, D / M));
    }
    PQ_TRY(bucket_rows(lst, n, nlist, codes, M, b_off, b_ids, b_codes, ws, s));
    PQ_TRY(merge_into(index, b_off, b_ids, b_codes, n, s));
    return ws.status;
}

int ivf_merge(ivf_index *dst, const ivf_index *src, void *stream)
{
    g_msg[0] = 0;
    if (!dst || !src) return fail(PQ_EINVAL, "null pointer");
    if (dst == src) return fail(PQ_EINVAL, "an index cannot be merged into itself");
    if (dst->kind != src->kind || dst->D != src->D || dst->M != src->M || dst->nlist != src->nlist ||
        dst->Ks != src->Ks)
        return fail(PQ_EINVAL, "the indexes differ in kind, D, M, nlist or Ks");
    // the two must share their coarse quantizer bit for bit
    std::vector<float> ca((size_t)dst->nlist * dst->D), cb2((size_t)src->nlist * src->D);
    PQ_TRY_CUDA(cudaMemcpy(ca.data(), dst->coarse, ca.size() * sizeof(float), cudaMemcpyDeviceToHost));
    PQ_TRY_CUDA(cudaMemcpy(cb2.data(), src->coarse, cb2.size() * sizeof(float), cudaMemcpyDeviceToHost));
    if (memcmp(ca.data(), cb2.data(), ca.size() * sizeof(float)) != 0)
        return fail(PQ_EINVAL, "the indexes have different coarse quantizers");
    if (src->N == 0) return PQ_OK;
    return merge_into(dst, src->offsets, src->ids, src->codes, src->N, static_cast<cudaStream_t>(stream));
}

int opq_rotate(const float *X, int64_t N, int32_t D, const float *R, float *Y, void *stream)
{
    g_msg[0] = 0;
    if (!X || !R || !Y) return fail(PQ_EINVAL, "null pointer");
    if (N < 0 || D < 1 || D > 1024) return fail(PQ_EINVAL, "need N >= 0 and 1 <= D <= 1024");
    if (X == Y) return fail(PQ_EINVAL, "Y must not alias X");
    return launch_rotate(X, N, D, R, Y, static_cast<cudaStream_t>(stream));
}

int opq_procrustes(const float *X, const float *Y, int64_t N, int32_t D, float *R, void *stream)
{
    g_msg[0] = 0;
    if (!X || !Y || !R) return fail(PQ_EINVAL, "null pointer");
    if (N < 1 || D < 1 || D > 1024) return fail(PQ_EINVAL, "need N >= 1 and 1 <= D <= 1024");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch ws(s);
    PQ_TRY(run_procrustes(X, Y, N, D, R, ws, s));
    return ws.status;
}

int opq_fit(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, int32_t outer, int32_t pq_iters,
            uint64_t seed, int32_t prec, float *R, float *codebooks, void *stream)
{
    g_msg[0] = 0;
    PQ_TRY(check_pq_shape(N, D, M, Ks, true));
    PQ_TRY(check_prec(prec));
    if (!X || !R || !codebooks) return fail(PQ_EINVAL, "null pointer");
    if (!aligned16(X) || !aligned16(codebooks)) return fail(PQ_EINVAL, "X and codebooks must be 16-byte aligned");
    if (outer < 0 || pq_iters < 0 || pq_iters > PQ_STATS_MAX_ITERS) return fail(PQ_EINVAL, "bad iteration counts");
    if (D > 1024) return fail(PQ_ENOTSUP, "opq_fit supports D <= 1024");
    if (prec == PQ_PREC_BF16 && !tc_pass_supported(D, M, Ks))
        return fail(PQ_ENOTSUP, "BF16 tensor-core pass needs D/M == 8 and M even");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch ws(s);
    float *Y = ws.get<float>((size_t)N * D);
    float *Yh = ws.get<float>((size_t)N * D);
    uint8_t *codes = ws.get<uint8_t>((size_t)N * M);
    if (ws.status) return ws.status;
    // R = I, codebooks: the PQ fit of X itself
    std::vector<float> eye((size_t)D * D, 0.0f);
    for (int i = 0; i < D; ++i) eye[(size_t)i * D + i] = 1.0f;
    PQ_TRY_CUDA(cudaMemcpyAsync(R, eye.data(), eye.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    PQ_TRY_CUDA(cudaMemcpyAsync(Y, X, (size_t)N * D * sizeof(float), cudaMemcpyDeviceToDevice, s));
    PQ_TRY(pq_fit(Y, N, D, M, Ks, pq_iters, seed, prec, nullptr, codebooks, nullptr, stream));
    for (int t = 0; t < outer; ++t) {
        PQ_TRY(pq_encode(Y, N, D, M, Ks, codebooks, prec, codes, nullptr, nullptr, stream));
        PQ_TRY(launch_decode_codes(codes, codebooks, N, D, M, Ks, Yh, s));
        PQ_TRY(run_procrustes(X, Yh, N, D, R, ws, s));
        PQ_TRY(launch_rotate(X, N, D, R, Y, s));
        PQ_TRY(pq_fit(Y, N, D, M, Ks, pq_iters, 0, prec, codebooks, codebooks, nullptr, stream));
    }
    PQ_TRY_CUDA(cudaStreamSynchronize(s));  // the host identity matrix above is read asynchronously
    return ws.status;
}

int ivf_copy_centers(const ivf_index *index, uint8_t *centers, void *stream)
{
    if (!index || !centers) return fail(PQ_EINVAL, "null pointer");
    if (index->kind != 1) return fail(PQ_EINVAL, "the index has raw-space coarse centroids, not centre codes");
    PQ_TRY_CUDA(cudaMemcpyAsync(centers, index->centers, (size_t)index->nlist * index->M, cudaMemcpyDeviceToDevice,
                                static_cast<cudaStream_t>(stream)));
    return PQ_OK;
}

int ivf_copy_lists(const ivf_index *index, int64_t *offsets, int64_t *ids, uint8_t *list_codes, void *stream)
{
    if (!index) return fail(PQ_EINVAL, "null index");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (offsets)
        PQ_TRY_CUDA(cudaMemcpyAsync(offsets, index->offsets, (size_t)(index->nlist + 1) * sizeof(int64_t),
                                    cudaMemcpyDeviceToDevice, s));
    if (ids)
        PQ_TRY_CUDA(cudaMemcpyAsync(ids, index->ids, (size_t)index->N * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    if (list_codes)
        PQ_TRY_CUDA(cudaMemcpyAsync(list_codes, index->codes, (size_t)index->N * index->M, cudaMemcpyDeviceToDevice,
                                    s));
    return PQ_OK;
}

void ivf_free(ivf_index *index)
{
    if (!index) return;
    cudaFree(index->coarse);
    cudaFree(index->half_norm);
    cudaFree(index->maxes);
    cudaFree(index->centers);
    cudaFree(index->cb);
    cudaFree(index->offsets);
    cudaFree(index->ids);
    cudaFree(index->codes);
    delete index;
}

int pq_sync_status(void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(e, "cudaStreamSynchronize");
    int dev = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    int *err = device_error_word(dev);
    if (!err) return PQ_OK;
    int h = 0;
    PQ_TRY_CUDA(cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        cudaMemset(err, 0, sizeof(int));
        return fail(h, "device-side failure %d", h);
    }
    return PQ_OK;
}

const char *pq_last_error(void) { return g_msg; }

int64_t pq_launch_count(void) { return g_launches.load(); }

int pq_test_set_spin_limit(uint32_t polls)
{
    g_seed_spin.store(polls == 0 ? kSpinLimit : polls);
    return PQ_OK;
}

int pq_test_fail_alloc_after(int32_t n)
{
    g_fail_alloc_after.store(n < 0 ? -1 : n);
    return PQ_OK;
}

int pq_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_prof) {
        g_ev_pool.push_back(r.a);
        g_ev_pool.push_back(r.b);
    }
    g_prof.clear();
    g_prof_on.store(on != 0);
    return PQ_OK;
}

int pq_profile_collect(const char *name, int64_t *count, double *total_ms)
{
    if (!name || !count || !total_ms) return fail(PQ_EINVAL, "null pointer");
    PQ_TRY_CUDA(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int64_t c = 0;
    double t = 0.0;
    for (auto &r : g_prof) {
        if (strcmp(r.name, name) != 0) continue;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
        ++c;
        t += ms;
    }
    *count = c;
    *total_ms = t;
    return PQ_OK;
}

int pq_profile_names(char *buf, int len)
{
    if (!buf || len <= 0) return fail(PQ_EINVAL, "null buffer");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::string out;
    std::vector<std::string> seen;
    for (auto &r : g_prof) {
        bool dup = false;
        for (auto &n : seen) dup = dup || n == r.name;
        if (dup) continue;
        seen.emplace_back(r.name);
        if (!out.empty()) out += ",";
        out += r.name;
    }
    snprintf(buf, (size_t)len, "%s", out.c_str());
    return (int)out.size() < len ? PQ_OK : PQ_EINVAL;
}

}  // extern "C"
