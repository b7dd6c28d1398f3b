// coarse_tc.cu -- nearest coarse centroid of every row on the tcgen05 tensor
// cores (the coarse quantizer of the inverted index, Sec. 2.2 / Sec. 3.1).
//
// Scores S_l = x'.c'_l - ||c'_l||^2/2 with x' = x - mu, c' = c - mu (mu = the mean
// of the centroids rounded to integers) are accumulated in TMEM over K = 3D + 16 bf16 lanes, the
// three-term split of the contraction
//     x'.c' ~ xh.ch + xl.ch + xh.cl        (x' = xh + xl, c' = ch + cl)
// plus the folded half norm (-nh - nl against a constant 1).  The error of S
// is below C1 ||x'|| max||c'|| + C2 max n' with C1 = 1.5 (3.1 u^2 + (3D+2) 2^-24),
// C2 = 1.5 (u^2 + (3D+2) 2^-24), u = 2^-8: bf16 split residuals plus a bound
// on the FP32 accumulation that is linear in the number of products.
//
// The epilogue keeps, per row over all centroid blocks, the chunk maxima and
// the best chunk of 32 scores, and accepts the argmax when no other score is
// within twice the bound; every other row goes to the FP64 re-check queue
// (coarse.cu), so the list of every row is exact.
//
// Pipeline, one CTA (384 threads) per SM, persistent over 128-row tiles: the
// centroid blocks of a tile alternate between two TMEM accumulators (256 centroids
// each), and each accumulator has a pipe of its own: a loading thread (warp 0 or
// 3) streams its blocks' pre-tiled B operand (8 KB tiles, bulk copies) through a
// 4-slot ring, and an issuing thread (warp 1 or 2) issues its M=128 N=256 K=16
// MMAs -- one issuing thread's own instruction chain cannot keep the tensor pipe
// busy.  Warps 4-7 build the A operand of the next tile (two stages) from rows
// read straight from global memory; warps 8-11 drain the accumulators and decide.
// When no row of a tile has a bf16 low part (integer rows within 256 of the
// integer centring), the MMAs of the xl.ch term are skipped: they would add exact
// zeros.  Every wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

constexpr int TM = 128;
constexpr int NBLK = 256;            // centroids per MMA / TMEM accumulator
constexpr int DMAX = 128;
constexpr int KDMAX = DMAX / 16;     // K steps of one term
// warp 0: B loads; warp 1: MMA issue; warps 2-3: spare; warps 4-7: A builder; warps 8-11: drain
constexpr int kThreads = 384;
constexpr int kBuild0 = 128, kDrain0 = 256;
constexpr int A_TILE = TM * 16 * 2;  // 4 KB
constexpr int A_STAGE = (2 * KDMAX + 1) * A_TILE;  // 68 KB: xh tiles, xl tiles, the constant tile
constexpr int NA = 2;                // A stages
constexpr int NXN = 4;               // row-norm slots (the builder runs at most 3 tiles ahead of the drain)
constexpr int B_TILE = NBLK * 16 * 2;  // 8 KB
constexpr int RING = 4;              // B slots per pipe (two pipes, one per TMEM buffer)
constexpr int OFF_A = 0;
constexpr int OFF_RING = OFF_A + NA * A_STAGE;
constexpr int OFF_MISC = OFF_RING + 2 * RING * B_TILE;        // mbarriers, TMEM slot, mu, low-part flags
constexpr int OFF_XN = OFF_MISC + 1024;                   // [NXN][TM] float: ||x'|| per row
constexpr int OFF_CMX = OFF_XN + NXN * TM * 4;            // [32 chunks][128 rows] chunk maxima
constexpr int SMEM_BYTES = OFF_CMX + 32 * TM * 4 + 1024;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory of one CTA");

// mbarrier slots
constexpr int MB_AREADY = 0 /*NA*/, MB_AFREE = 2 /*NA*/, MB_MMA = 4 /*2*/, MB_TFREE = 6 /*2*/,
              MB_RFULL = 8 /*2 x RING*/, MB_REMPTY = 8 + 2 * RING /*2 x RING*/, MB_XNREADY = 8 + 4 * RING /*NXN*/,
              MB_COUNT = 8 + 4 * RING + NXN;
constexpr int MISC_TSLOT = 8 * MB_COUNT, MISC_MU = 256, MISC_XLNZ = 768;  // xlnz: [NA][4] int
static_assert(MISC_TSLOT + 4 <= MISC_MU && MISC_MU + 4 * DMAX <= MISC_XLNZ && MISC_XLNZ + 4 * NA * 4 <= 1024,
              "misc area overlap");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t c)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(c) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int *err)
{
    for (unsigned it = 0;; ++it) {
        if (mbar_try(a, parity)) return true;
        if (it > kSpinLimit) {
            atomicCAS(err, 0, PQ_ETIMEOUT);
            return false;
        }
        if ((it & 255) == 255 && *(volatile int *)err != 0) return false;
    }
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(256 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
__host__ __device__ __forceinline__ uint32_t core_off(int r, int k)
{
    return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NBLK >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t da, uint64_t db, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(da), "l"(db), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
// 32 consecutive columns of this thread's TMEM lane (one row's scores) and, by the load's max
// reduction, their largest value m.  tcgen05.ld writes its registers asynchronously: the wait
// names them as in/out operands so that the compiler cannot move a use of the loaded values above it.
#define TC_LDMAX32(base, v, m)                                                                                      \
    asm volatile("tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"  \
                 "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %32, [%33];"             \
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),   \
                   "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]),         \
                   "=f"(v[15]), "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]),       \
                   "=f"(v[22]), "=f"(v[23]), "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]),       \
                   "=f"(v[29]), "=f"(v[30]), "=f"(v[31]), "=f"(m)                                                   \
                 : "r"(base))
#define TC_WAITMAX32(v, m)                                                                                        \
    asm volatile("tcgen05.wait::ld.sync.aligned;"                                                                 \
                 : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),  \
                   "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]),         \
                   "+f"(v[15]), "+f"(v[16]), "+f"(v[17]), "+f"(v[18]), "+f"(v[19]), "+f"(v[20]), "+f"(v[21]),       \
                   "+f"(v[22]), "+f"(v[23]), "+f"(v[24]), "+f"(v[25]), "+f"(v[26]), "+f"(v[27]), "+f"(v[28]),       \
                   "+f"(v[29]), "+f"(v[30]), "+f"(v[31]), "+f"(m)                                                   \
                 :                                                                                                \
                 : "memory")
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}
__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// ---- preparation: centring mean, bounds, tiled B operand -------------------
// Bp layout: [blk][tile][256 rows][16 bf16] core-matrix tiles; tile 2k = ch of K step k,
// 2k+1 = cl of K step k, 2*KD = the half-norm tile.
// mu = mean of the centroids rounded to an integer (the centring of the scores; any fixed value
// keeps the decisions exact, and an integer one keeps integer-valued rows of magnitude <= 256
// exact in bf16 after centring, so that their low parts vanish).  Block of 1024 threads: 8 groups
// of lists per dimension, added in a fixed order.
constexpr int kMuGroups = 8;
__global__ void __launch_bounds__(1024) coarse_mu_kernel(const float *C, int nlist, int D, float *mu)
{
    __shared__ float part[kMuGroups][DMAX];
    const int j = threadIdx.x % DMAX, g = threadIdx.x / DMAX;
    float s = 0.0f;
    if (j < D)
        for (int l = g; l < nlist; l += kMuGroups) s += C[(size_t)l * D + j];
    part[g][j] = s;
    __syncthreads();
    if (g == 0 && j < D) {
        float t = 0.0f;
        for (int q = 0; q < kMuGroups; ++q) t += part[q][j];
        mu[j] = rintf(t / (float)nlist);
    }
}

__global__ void coarse_prep_kernel(const float *C, int nlist, int nlist_pad, int D, const float *mu,
                                   unsigned char *Bp, unsigned *maxbits)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlist_pad) return;
    const int KD = D / 16, T = 2 * KD + 1;
    const int blk = l / NBLK, row = l % NBLK;
    unsigned char *base = Bp + (size_t)blk * T * B_TILE;
    float nc = 0.0f;
    for (int k = 0; k < KD; ++k) {
        float hi[16], lo[16];
        for (int q = 0; q < 16; ++q) {
            const float c = l < nlist ? C[(size_t)l * D + 16 * k + q] - mu[16 * k + q] : 0.0f;
            nc = fmaf(c, c, nc);
            hi[q] = bf16_round(c);
            lo[q] = c - hi[q];
        }
        unsigned char *th = base + (size_t)(2 * k) * B_TILE, *tl = base + (size_t)(2 * k + 1) * B_TILE;
        *reinterpret_cast<uint4 *>(th + core_off(row, 0)) =
            make_uint4(pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]), pack_bf16(hi[4], hi[5]), pack_bf16(hi[6], hi[7]));
        *reinterpret_cast<uint4 *>(th + core_off(row, 8)) = make_uint4(pack_bf16(hi[8], hi[9]), pack_bf16(hi[10], hi[11]),
                                                                       pack_bf16(hi[12], hi[13]), pack_bf16(hi[14], hi[15]));
        *reinterpret_cast<uint4 *>(tl + core_off(row, 0)) =
            make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]), pack_bf16(lo[4], lo[5]), pack_bf16(lo[6], lo[7]));
        *reinterpret_cast<uint4 *>(tl + core_off(row, 8)) = make_uint4(pack_bf16(lo[8], lo[9]), pack_bf16(lo[10], lo[11]),
                                                                       pack_bf16(lo[12], lo[13]), pack_bf16(lo[14], lo[15]));
    }
    const float n = 0.5f * nc;
    float nh, nl;
    if (l < nlist) {
        nh = bf16_round(n);
        nl = n - nh;
        atomicMax(maxbits + 0, __float_as_uint(n));
        atomicMax(maxbits + 1, __float_as_uint(sqrtf(nc)));
    } else {
        nh = 3.0e38f;
        nl = 0.0f;
    }
    unsigned char *tn = base + (size_t)(2 * KD) * B_TILE;
    *reinterpret_cast<uint4 *>(tn + core_off(row, 0)) = make_uint4(pack_bf16(-nh, -nl), 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(tn + core_off(row, 8)) = make_uint4(0u, 0u, 0u, 0u);
}

struct CoarseTcArgs {
    int64_t N;
    int D, nlist, nlist_pad, tiles;
    const float *X;
    const unsigned char *Bp;
    const float *mu;
    const unsigned *maxbits;
    int32_t *list_of_row;
    int64_t *queue;
    uint32_t *qmask;
    unsigned long long *qlen;
    int *err;
};

// NBT > 0: at most NBT centroid blocks (NBT * 8 chunks of 32 <= 32); the chunk maxima are kept
// and an uncertain row is queued with the mask of chunks that can hold its nearest centroid.
template <int NBT>
__global__ void __launch_bounds__(kThreads, 1) coarse_tc_kernel(const CoarseTcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    // aligned by an offset from the shared array itself, so that the compiler keeps every access
    // below in the shared address space
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem_raw);
    unsigned char *sm = smem_raw + (((sbase + 1023u) & ~1023u) - sbase);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = a.D, KD = D / 16, T = 2 * KD + 1, NB = a.nlist_pad / NBLK;
    uint64_t *mb = reinterpret_cast<uint64_t *>(sm + OFF_MISC);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + OFF_MISC + MISC_TSLOT);
    float *smu = reinterpret_cast<float *>(sm + OFF_MISC + MISC_MU);
    // per builder warp and A stage: does the tile's A operand have a nonzero low part?  When none
    // does, the MMAs of xl.ch (exact zeros) are skipped, which leaves every score unchanged
    volatile int *xlnz = reinterpret_cast<volatile int *>(sm + OFF_MISC + MISC_XLNZ);
    float *xn_s = reinterpret_cast<float *>(sm + OFF_XN);
    unsigned char *aop = sm + OFF_A;
    unsigned char *ring = sm + OFF_RING;

    for (int j = tid; j < D; j += kThreads) smu[j] = a.mu[j];
    if (tid == 0) {
        for (int i = 0; i < MB_COUNT; ++i) {
            uint32_t c = 1;
            if ((i >= MB_AREADY && i < MB_AREADY + NA) || i == MB_TFREE || i == MB_TFREE + 1 ||
                (i >= MB_XNREADY && i < MB_XNREADY + NXN))
                c = 4;
            if (i >= MB_AFREE && i < MB_AFREE + NA) c = 2;  // both MMA warps
            mbar_init(smem_u32(mb + i), c);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tslot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;
    const int n_my = (a.tiles > (int)blockIdx.x) ? (a.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == 0 || warp == 3) {
        // ---- B loads: pipe e (warp 0: e = 0, warp 3: e = 1) streams the tiles of the centroid
        // blocks whose sequence number v = i * NB + b has v % 2 == e, in MMA order, through its ring
        if (lane == 0) {
            const int e = warp == 0 ? 0 : 1;
            const uint32_t rfull0 = smem_u32(mb + MB_RFULL + e * RING), rempty0 = smem_u32(mb + MB_REMPTY + e * RING);
            unsigned char *rg = ring + e * RING * B_TILE;
            int z = 0;
            bool ok = true;
            for (int i = 0; i < n_my && ok; ++i)
                for (int b = 0; b < NB && ok; ++b) {
                    if (((i * NB + b) & 1) != e) continue;
                    for (int t = 0; t < T; ++t, ++z) {
                        const int slot = z % RING, use = z / RING;
                        if (use >= 1 && !mbar_wait(rempty0 + 8 * slot, (use - 1) & 1, a.err)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(rfull0 + 8 * slot, B_TILE);
                        bulk_load(smem_u32(rg + slot * B_TILE), a.Bp + ((size_t)b * T + t) * B_TILE, B_TILE,
                                  rfull0 + 8 * slot);
                    }
                }
            for (int q = (z > RING ? z - RING : 0); q < z; ++q) mbar_wait(rfull0 + 8 * (q % RING), (q / RING) & 1, a.err);
        }
    } else if (warp == 1 || warp == 2) {
        // ---- MMA issue, two warps: warp 1 + e issues the blocks of pipe e into TMEM buffer e.  A
        // single issuing thread's own instructions between two MMAs bound the tensor pipe, so two
        // issue in turn; descriptors are base values plus offsets, the ring position is a running
        // counter, and the wait for a B tile is a plain poll.
        if (lane == 0) {
            const int e = warp - 1;
            const uint64_t dA0 = smem_desc(smem_u32(aop)), dB0 = smem_desc(smem_u32(ring + e * RING * B_TILE));
            const uint32_t rfull0 = smem_u32(mb + MB_RFULL + e * RING), rempty0 = smem_u32(mb + MB_REMPTY + e * RING);
            int slot = 0;
            uint32_t ph = 0;
            bool ok = true;
            // the next B tile has landed (bounded poll)
            auto ring_wait = [&]() -> bool {
                for (unsigned it = 0; !mbar_try(rfull0 + 8 * slot, ph); ++it) {
                    if (it > kSpinLimit) {
                        atomicCAS(a.err, 0, PQ_ETIMEOUT);
                        return false;
                    }
                    if ((it & 255) == 255 && *(volatile int *)a.err != 0) return false;
                }
                return true;
            };
            auto ring_next = [&]() {
                mma_commit(rempty0 + 8 * slot);
                if (++slot == RING) {
                    slot = 0;
                    ph ^= 1u;
                }
            };
            for (int i = 0; i < n_my && ok; ++i) {
                const int as = i % NA;
                if (!mbar_wait(smem_u32(mb + MB_AREADY + as), (i / NA) & 1, a.err)) break;
                tc_after_sync();
                const bool xl = (xlnz[as * 4 + 0] | xlnz[as * 4 + 1] | xlnz[as * 4 + 2] | xlnz[as * 4 + 3]) != 0;
                const uint64_t dA = dA0 + (uint64_t)((as * A_STAGE) >> 4);
                for (int b = 0; b < NB && ok; ++b) {
                    const int v = i * NB + b, buf = v & 1, u = v >> 1;
                    if (buf != e) continue;
                    if (u >= 1 && !mbar_wait(smem_u32(mb + MB_TFREE + buf), (u - 1) & 1, a.err)) { ok = false; break; }
                    tc_after_sync();
                    const uint32_t d = tmem + (uint32_t)(buf * NBLK);
                    // B tiles in order ch_0, cl_0, ch_1, cl_1, ..., the half-norm tile
                    for (int k = 0; k < KD; ++k) {
                        if (!ring_wait()) { ok = false; break; }
                        const uint64_t dbh = dB0 + (uint64_t)((slot * B_TILE) >> 4);
                        mma_bf16(d, dA + (uint64_t)((k * A_TILE) >> 4), dbh, k == 0 ? 0u : 1u);  // xh.ch
                        if (xl) mma_bf16(d, dA + (uint64_t)(((KD + k) * A_TILE) >> 4), dbh, 1u);  // xl.ch
                        ring_next();
                        if (!ring_wait()) { ok = false; break; }
                        mma_bf16(d, dA + (uint64_t)((k * A_TILE) >> 4), dB0 + (uint64_t)((slot * B_TILE) >> 4), 1u);  // xh.cl
                        ring_next();
                    }
                    if (!ok || !ring_wait()) { ok = false; break; }
                    mma_bf16(d, dA + (uint64_t)((2 * KD * A_TILE) >> 4), dB0 + (uint64_t)((slot * B_TILE) >> 4), 1u);  // -n'
                    ring_next();
                    mma_commit(smem_u32(mb + MB_MMA + buf));
                }
                if (!ok) break;
                mma_commit(smem_u32(mb + MB_AFREE + as));
            }
        }
    } else if (warp >= kBuild0 / 32 && warp < kDrain0 / 32) {
        // ---- A builder: thread = row; the row read straight from global memory, centred, split into
        // bf16 high and low parts; rows past N read as zeros (their lists are never written)
        const int q = warp & 3, r = q * 32 + lane;
        for (int i = 0; i < n_my; ++i) {
            const int as = i % NA;
            if (i >= NA &&
                !__all_sync(0xffffffffu, mbar_wait(smem_u32(mb + MB_AFREE + as), ((i / NA) - 1) & 1, a.err)))
                break;
            const int64_t row = (int64_t)((int)blockIdx.x + i * (int)gridDim.x) * TM + r;
            const bool in = row < a.N;
            const float *xr = a.X + (in ? row : 0) * (int64_t)D;
            unsigned char *ab = aop + as * A_STAGE;
            float xx = 0.0f;
            bool nz = false;
            for (int k = 0; k < KD; ++k) {
                float hi[16], lo[16];
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const float4 v = in ? __ldg(reinterpret_cast<const float4 *>(xr + 16 * k + 4 * c4))
                                        : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const float xc = e[w] - smu[16 * k + 4 * c4 + w];
                        xx = fmaf(xc, xc, xx);
                        hi[4 * c4 + w] = bf16_round(xc);
                        lo[4 * c4 + w] = xc - hi[4 * c4 + w];
                        nz |= lo[4 * c4 + w] != 0.0f;
                    }
                }
                unsigned char *th = ab + k * A_TILE, *tlo = ab + (KD + k) * A_TILE;
                *reinterpret_cast<uint4 *>(th + core_off(r, 0)) = make_uint4(pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]),
                                                                             pack_bf16(hi[4], hi[5]), pack_bf16(hi[6], hi[7]));
                *reinterpret_cast<uint4 *>(th + core_off(r, 8)) = make_uint4(pack_bf16(hi[8], hi[9]), pack_bf16(hi[10], hi[11]),
                                                                             pack_bf16(hi[12], hi[13]), pack_bf16(hi[14], hi[15]));
                *reinterpret_cast<uint4 *>(tlo + core_off(r, 0)) = make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]),
                                                                              pack_bf16(lo[4], lo[5]), pack_bf16(lo[6], lo[7]));
                *reinterpret_cast<uint4 *>(tlo + core_off(r, 8)) = make_uint4(pack_bf16(lo[8], lo[9]), pack_bf16(lo[10], lo[11]),
                                                                              pack_bf16(lo[12], lo[13]), pack_bf16(lo[14], lo[15]));
            }
            {
                unsigned char *tn = ab + 2 * KD * A_TILE;
                *reinterpret_cast<uint4 *>(tn + core_off(r, 0)) = make_uint4(pack_bf16(1.0f, 1.0f), 0u, 0u, 0u);
                *reinterpret_cast<uint4 *>(tn + core_off(r, 8)) = make_uint4(0u, 0u, 0u, 0u);
            }
            xn_s[(i % NXN) * TM + r] = sqrtf(xx) * (1.0f + 1e-5f);
            fence_async_smem();
            const bool wnz = __any_sync(0xffffffffu, nz);
            if (lane == 0) {
                xlnz[as * 4 + q] = wnz ? 1 : 0;
                mbar_arrive(smem_u32(mb + MB_AREADY + as));
                mbar_arrive(smem_u32(mb + MB_XNREADY + i % NXN));
            }
        }
    } else if (warp >= kDrain0 / 32) {
        // ---- drain: thread = row = TMEM lane; the scores of every centroid block, the chunk maxima
        // from the loads' max reduction, the best chunk kept in registers
        const int q = warp & 3, r = q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        const float nmax = __uint_as_float(a.maxbits[0]) * (1.0f + 1e-5f);
        const float cmax = __uint_as_float(a.maxbits[1]) * (1.0f + 1e-5f);
        const float u2 = 1.52587890625e-05f;  // 2^-16
        const float acc_b = (float)(3 * D + 2) * 5.9604645e-8f;
        const float C1 = 1.5f * (3.1f * u2 + acc_b), C2 = 1.5f * (u2 + acc_b);
        float *cmx = reinterpret_cast<float *>(sm + OFF_CMX);
        for (int i = 0; i < n_my; ++i) {
            const int64_t row = (int64_t)((int)blockIdx.x + i * (int)gridDim.x) * TM + r;
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(mb + MB_XNREADY + i % NXN), (i / NXN) & 1, a.err))) break;
            const float xn = xn_s[(i % NXN) * TM + r];
            const float tt = xn + cmax;
            const float win = 2.0f * (C1 * xn * cmax + C2 * nmax + 1e-13f * tt * tt);
            float best = -FLT_MAX, cm2 = -FLT_MAX;
            int bestj = 0;
            float sv[32];
            bool ok = true;
            for (int b = 0; b < NB; ++b) {
                const int v = i * NB + b, buf = v & 1, u = v >> 1;
                if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(mb + MB_MMA + buf), u & 1, a.err))) { ok = false; break; }
                tc_after_sync();
                const uint32_t tb = tl + (uint32_t)(buf * NBLK);
#pragma unroll
                for (int cc = 0; cc < NBLK / 32; ++cc) {
                    float vv[32], cm;
                    TC_LDMAX32(tb + (uint32_t)(cc * 32), vv, cm);
                    TC_WAITMAX32(vv, cm);
                    const int j = b * (NBLK / 32) + cc;
                    if (NBT > 0) cmx[j * TM + r] = cm;
                    const bool better = cm > best;
                    cm2 = better ? best : fmaxf(cm2, cm);
                    best = better ? cm : best;
                    bestj = better ? j : bestj;
#pragma unroll
                    for (int q2 = 0; q2 < 32; ++q2) sv[q2] = (j == 0 || better) ? vv[q2] : sv[q2];
                }
                tc_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(mb + MB_TFREE + buf));
            }
            if (!ok) break;
            const float theta = best - win;
            int ib = 0, nin = 0;
#pragma unroll
            for (int q2 = 31; q2 >= 0; --q2) {
                ib = (sv[q2] == best) ? q2 : ib;
                nin += (sv[q2] >= theta) ? 1 : 0;
            }
            // the warp's uncertain rows take consecutive queue slots from one atomic
            const bool valid = row < a.N, cert = nin == 1 && cm2 < theta;
            const unsigned need = __ballot_sync(0xffffffffu, valid && !cert);
            unsigned long long base = 0;
            if (need) {
                const int leader = __ffs(need) - 1;
                if (lane == leader) base = atomicAdd(a.qlen, (unsigned long long)__popc(need));
                base = __shfl_sync(0xffffffffu, base, leader);
            }
            if (valid) {
                if (cert) {
                    const int l = bestj * 32 + ib;
                    // a padded centroid scores -3e38 and can never be certified; should one be,
                    // the scores were corrupt: report it instead of passing on an invalid list
                    if (l < a.nlist) {
                        a.list_of_row[row] = l;
                    } else {
                        a.list_of_row[row] = 0;
                        atomicCAS(a.err, 0, PQ_EINTERNAL);
                    }
                } else {
                    uint32_t mask = 0;
                    if (NBT > 0) {
#pragma unroll
                        for (int c = 0; c < NB * 8; ++c) mask |= (cmx[c * TM + r] >= theta ? 1u : 0u) << c;
                    }
                    a.list_of_row[row] = -1;
                    const unsigned long long slot = base + (unsigned)__popc(need & ((1u << lane) - 1u));
                    a.queue[slot] = row;
                    a.qmask[slot] = mask;  // 0: every centroid is a candidate
                }
            }
        }
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

}  // namespace

bool coarse_tc_supported(int D, int nlist) { return D % 32 == 0 && D >= 32 && D <= DMAX && nlist >= 1; }

// Scores on the tensor cores, certified rows written to list_of_row, the others queued
// (entries of queue, count in *qlen) for the FP64 re-check.
int launch_coarse_tc(const float *X, int64_t N, int D, const float *C, int nlist, int32_t *list_of_row,
                     int64_t *queue, uint32_t *qmask, unsigned long long *qlen, Scratch &ws, cudaStream_t s)
{
    if (!coarse_tc_supported(D, nlist)) return fail(PQ_ENOTSUP, "tensor-core coarse assignment needs D % 32 == 0, D <= 128");
    if (N >= (1LL << 31) - TM) return fail(PQ_ENOTSUP, "tensor-core coarse assignment supports N < 2^31");
    if (reinterpret_cast<uintptr_t>(X) & 15) return fail(PQ_EINVAL, "X must be 16-byte aligned");
    const int nlist_pad = (nlist + NBLK - 1) / NBLK * NBLK;
    const int KD = D / 16, T = 2 * KD + 1;
    float *mu = ws.get<float>((size_t)D);
    unsigned *maxbits = ws.get<unsigned>(2, true);
    unsigned char *Bp = ws.get<unsigned char>((size_t)(nlist_pad / NBLK) * T * B_TILE);
    if (ws.status) return ws.status;
    int dev = 0, sms = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    PQ_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int *err = device_error_word(dev);
    if (!err) return fail(PQ_ENOMEM, "device error word");
    {
        ProfScope ps("coarse_prep", s);
        coarse_mu_kernel<<<1, kMuGroups * DMAX, 0, s>>>(C, nlist, D, mu);
        coarse_prep_kernel<<<(nlist_pad + 127) / 128, 128, 0, s>>>(C, nlist, nlist_pad, D, mu, Bp, maxbits);
        count_launch(2);
        PQ_TRY_CUDA(cudaGetLastError());
    }
    CoarseTcArgs a;
    a.N = N;
    a.D = D;
    a.nlist = nlist;
    a.nlist_pad = nlist_pad;
    a.tiles = (int)((N + TM - 1) / TM);
    a.X = X;
    a.Bp = Bp;
    a.mu = mu;
    a.maxbits = maxbits;
    a.list_of_row = list_of_row;
    a.queue = queue;
    a.qmask = qmask;
    a.qlen = qlen;
    a.err = err;
    const int grid = std::max(1, std::min(a.tiles, sms));
    ProfScope ps("coarse_assign_tc", s);
    if (nlist_pad <= 4 * NBLK) {
        PQ_TRY_CUDA(cudaFuncSetAttribute(coarse_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        coarse_tc_kernel<4><<<grid, kThreads, SMEM_BYTES, s>>>(a);
    } else {
        PQ_TRY_CUDA(cudaFuncSetAttribute(coarse_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        coarse_tc_kernel<0><<<grid, kThreads, SMEM_BYTES, s>>>(a);
    }
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

}  // namespace pqgb
