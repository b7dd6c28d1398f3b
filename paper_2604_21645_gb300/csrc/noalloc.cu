// noalloc.cu -- pq_lloyd_noalloc: the Lloyd iterations of pq_fit (FP32 form)
// without any device allocation.
//
// Who needs this: callers that must not allocate device memory while they
// run.  Examples are a serving process whose GPU memory is reserved up front
// by its own allocator (and must not be fragmented or exhausted by a library
// that takes memory behind its back), or a latency-bound loop in which a
// cudaMalloc could block, synchronize the device or fail at the worst time.
// The regular entry points take stream-ordered scratch with cudaMallocAsync;
// this one keeps its scratch in a fixed array compiled into the library.
//
// The scratch is the per-block partial member sums and counts that the Lloyd
// pass writes and the finalise kernel reduces.  It lives in the file-scope
// array below (kNoAllocScratchBytes per GPU, held by every GPU that loads
// this code until the process exits).  Host code cannot pass the array's
// name to a kernel -- on the host that name is only a stand-in, not a device
// address -- so the first call on each device looks the address up with
// cudaGetSymbolAddress, with that device current, and caches it.  The cache
// assumes the device's primary context lives as long as the library: after a
// cudaDeviceReset the cached address is stale, and the library must not be
// called on that device again in this process.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_addr_mu;
void *g_addr[64] = {};

int scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= 64) return fail(PQ_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PQ_OK;
}

}  // namespace
}  // namespace pqgb

using namespace pqgb;

extern "C" int pq_lloyd_noalloc(const float *X, int64_t N, int32_t D, int32_t M, int32_t Ks, int32_t iters,
                                const float *init_codebooks, float *codebooks, void *stream)
{
    clear_error();
    if (!X || !init_codebooks || !codebooks) return fail(PQ_EINVAL, "null pointer");
    if (N < 1 || D <= 0 || M <= 0 || D % M != 0) return fail(PQ_EINVAL, "need N >= 1 and D a multiple of M");
    if (Ks < 1 || Ks > 256 || N < Ks) return fail(PQ_EINVAL, "need 1 <= Ks <= 256 and N >= Ks");
    if (iters < 0 || iters > PQ_STATS_MAX_ITERS) return fail(PQ_EINVAL, "iters=%d must be in [0, %d]", iters,
                                                             PQ_STATS_MAX_ITERS);
    if (reinterpret_cast<uintptr_t>(X) & 15) return fail(PQ_EINVAL, "X must be 16-byte aligned");
    const int ds = D / M;
    // the subspace widths the FP32 pass is compiled for; checked before anything is enqueued
    if (ds != 1 && ds != 2 && ds != 4 && ds != 8 && ds != 16 && ds != 32)
        return fail(PQ_ENOTSUP, "subspace width Ds=%d not supported (1, 2, 4, 8, 16 or 32)", ds);
    // One block needs, per subspace, Ks*ds int64 and Ks*ds FP32 sums and Ks int32 counts.
    const size_t need1 = Partials::bytes(1, M, Ks, ds, 1);
    if (need1 > kNoAllocScratchBytes)
        return fail(PQ_EINVAL,
                    "pq_lloyd_noalloc: M*Ks*(12*D/M + 4) + 4*M + 64 = %zu bytes exceeds its fixed scratch of %zu bytes",
                    need1, kNoAllocScratchBytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    void *base = nullptr;
    PQ_TRY(scratch_address(dev, &base));

    PqPass p;
    p.X = X;
    p.N = N;
    p.D = D;
    p.M = M;
    p.Ks = Ks;
    p.ds = ds;
    p.C = codebooks;
    p.gx = pq_pass_blocks_per_subspace(p);
    while (p.gx > 1 && Partials::bytes(p.gx, M, Ks, ds, 1) > kNoAllocScratchBytes) --p.gx;
    // Layout (Partials::carve): [gx][M][Ks][ds] int64 and FP32 sums, [gx][M][Ks] counts,
    // [M] exponents.  Every pass overwrites all of it before the finalise kernel reads it,
    // so nothing left by an earlier call needs clearing.
    p.part.carve(base, p.gx, M, Ks, ds);
    if (init_codebooks != codebooks)
        PQ_TRY_CUDA(cudaMemcpyAsync(codebooks, init_codebooks, (size_t)M * Ks * ds * sizeof(float),
                                    cudaMemcpyDeviceToDevice, s));
    for (int t = 0; t < iters; ++t) {
        PQ_TRY(launch_pq_pass_f32(p, s));
        PQ_TRY(launch_pq_finalize(p.part, p.gx, M, Ks, ds, codebooks, nullptr, s));
    }
    return PQ_OK;
}
