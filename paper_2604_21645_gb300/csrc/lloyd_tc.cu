// lloyd_tc.cu -- PQ Lloyd pass on the tcgen05 tensor cores (Sec. 2.1: nearest
// codeword of every (row, subspace) and the mean update), BF16 operands with
// FP32 accumulation in tensor memory.
//
// Contraction.  Per subspace the scores S_k = x.c_k - ||c_k||^2/2 (argmax S_k
// == argmin ||x - c_k||^2) come from one M=128 x N=256 MMA over K=32 bf16
// lanes.  Both sides are first centred by the subspace's codeword mean mu
// (distances are translation invariant) and split into bf16 high and low
// parts, x' = xh + xl, c' = ch + cl, n' = ||c'||^2/2 = nh + nl:
//     A row  = [xh(8) xl(8) | xh(8) 1 1 0..]
//     B row  = [ch(8) ch(8) | cl(8) -nh -nl 0..]
//     S      = xh.ch + xl.ch + xh.cl - nh - nl
// The error of S is below C1 ||x'|| max||c'|| + C2 max n': the two-term bf16
// splits leave at most 3.1 u^2 ||x'|| ||c'|| (u = 2^-8) and u^2 n', the FP32
// accumulation of the 26 exact products is bounded by 32 * 2^-24 of their
// absolute sum (the largest error measured on this GPU is 2.6e-7 of it), and
// C1 = 7.5e-5, C2 = 2.7e-5 keep a 1.5x margin over the sum of those terms.
//
// Decision.  The epilogue reads each row's 256 scores from TMEM in chunks of
// 32, keeps the eight chunk maxima and the values of the best chunk, and
// accepts the argmax when no other score lies within twice the error bound of
// it.  For the other rows the complete candidate set -- every score within
// the bound, from the saved chunk and from any chunk whose maximum reaches the
// bound (re-read from TMEM) -- is re-ranked exactly: FP32 direct differences,
// then FP64 among the FP32 near-ties, the decision rule of the CPU reference.
// Codes are exact.
//
// Update.  Residuals x - c_code are added with shared-memory FP32 atomics into
// per-CTA sums; the finalise kernel adds the CTAs in a fixed order in FP64 and
// moves every codeword by the mean residual of its members.
//
// Pipeline (one CTA per SM, one group of 4 subspaces, persistent over row
// tiles of 128): warp 0 issues TMA loads of 128 x 32 float tiles (128B swizzle)
// into two stages; two lanes of warp 1 issue the MMAs; warps 2-9 form two
// warpgroups (thread = row = TMEM lane), warpgroup w handling subspaces 2w and
// 2w+1 of every tile with its own TMEM accumulator and a double-buffered A
// operand.  All hand-offs are mbarriers; every wait is bounded, and a
// timed-out wait records PQ_ETIMEOUT and lets the CTA unwind (its copies
// waited for, its tensor memory freed).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

constexpr int G = 4;        // subspaces per CTA
constexpr int TM = 128;     // rows per tile
constexpr int KSMAX = 256;  // codewords (MMA N)
constexpr int DS = 8;       // subspace width
constexpr int kCompute = 256;              // two warpgroups
constexpr int kThreads = 64 + kCompute;    // + producer warp + MMA warp

constexpr int XS_BYTES = TM * G * DS * 4;            // 16 KB per stage
constexpr int A_HALF = TM * 16 * 2;                  // 4 KB (K = 16 bf16)
constexpr int B_HALF = KSMAX * 16 * 2;               // 8 KB
constexpr int OFF_XS = 0;
constexpr int OFF_A = OFF_XS + 2 * XS_BYTES;                // [wg][buf][half]
constexpr int OFF_B = OFF_A + 2 * 2 * 2 * A_HALF;           // [g][half]
// Row strides of the FP32 codeword copy (12 floats: 16-byte aligned rows that fall on different
// bank groups for random codes) and of the update sums (9 floats: conflict-free scalar atomics).
constexpr int CB_STRIDE = 12;
constexpr int ACC_STRIDE = 9;
constexpr int OFF_CBF = OFF_B + G * 2 * B_HALF;
constexpr int OFF_CN = OFF_CBF + G * KSMAX * CB_STRIDE * 4;
constexpr int OFF_ACC = OFF_CN + G * KSMAX * 4;
constexpr int OFF_CNT = OFF_ACC + G * KSMAX * ACC_STRIDE * 4;
constexpr int OFF_MISC = OFF_CNT + G * KSMAX * 4;
constexpr int MISC_BYTES = 512;
constexpr int SMEM_BYTES = OFF_MISC + MISC_BYTES + 1024;  // + alignment slack

// mbarrier slots in the misc area
constexpr int MB_FULL = 0;      // [2] TMA -> compute
constexpr int MB_EMPTY = 2;     // [2] compute -> producer (8 warps)
constexpr int MB_AREADY = 4;    // [2] per warpgroup: compute -> MMA (4 warps)
constexpr int MB_MMA = 6;       // [2] per warpgroup: MMA -> compute (commit)
constexpr int MB_TFREE = 8;     // [2] per warpgroup: compute -> MMA (4 warps)
constexpr int MB_COUNT = 10;

constexpr float kC1 = 7.5e-5f;
constexpr float kC2 = 2.7e-5f;
constexpr int kMaxCand = 32;

struct TcArgs {
    int64_t N;
    int D, M, Ks;
    int tiles;
    const float *C;
    uint8_t *codes;
    double *part;
    int *part_cnt;
    double *sse;
    unsigned long long *rechecks;
    int *err;
    const int *blk_chunk;      // optional chunk table (batched form)
    const int64_t *chunk_off;
    const int *chunk_blk;
};

// ---- PTX wrappers ----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
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
// Bounded wait for the phase with the given parity; false (PQ_ETIMEOUT recorded) if it ran out.
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

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(map), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// no-swizzle K-major shared-memory matrix descriptor: core matrices of 8 rows x 16 B,
// LBO = distance between the two K core matrices, SBO = distance between 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(256 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// byte offset of element (row, k) in a K=16 operand tile
__device__ __forceinline__ uint32_t core_off(int r, int k) { return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// kind::f16, D = f32, A = B = bf16, both K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(KSMAX >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

#define TC_LD32(base, v)                                                                                            \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16," \
                 "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                             \
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),   \
                   "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]),         \
                   "=f"(v[15]), "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]),       \
                   "=f"(v[22]), "=f"(v[23]), "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]),       \
                   "=f"(v[29]), "=f"(v[30]), "=f"(v[31])                                                            \
                 : "r"(base))
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// float chunk (16 B) of row r in a 128B-swizzled TMA stage (row = 128 bytes)
__device__ __forceinline__ const float *xs_row_chunk(const float *stage, int r, int chunk)
{
    return stage + r * 32 + ((chunk ^ (r & 7)) << 2);
}

// Exact decision over all codewords (used only if a row has more than kMaxCand
// candidates): FP32 expansion scores with their error bound, then FP64 inside it.
__device__ __forceinline__ int exact_code(const float *x, const float *cb, const float *cn, int Ks, float nmax,
                                       float cmax)
{
    float xx = 0.0f;
#pragma unroll
    for (int j = 0; j < DS; ++j) xx = fmaf(x[j], x[j], xx);
    const float xn = sqrtf(xx) * (1.0f + 1e-6f);
    float m1 = FLT_MAX, m2 = FLT_MAX;
    int i1 = 0;
    for (int k = 0; k < Ks; ++k) {
        float s = cn[k];
#pragma unroll
        for (int j = 0; j < DS; ++j) s = fmaf(-x[j], cb[k * CB_STRIDE + j], s);
        const bool lt = s < m1;
        m2 = lt ? m1 : fminf(m2, s);
        i1 = lt ? k : i1;
        m1 = fminf(m1, s);
    }
    const float t = xn + cmax;
    const float win = 2.0f * (2.2f * gamma_f32(DS + 1) * (nmax + xn * cmax) + 1e-13f * t * t);
    if (m2 - m1 > win) return i1;
    double best = DBL_MAX;
    int bk = 0;
    for (int k = 0; k < Ks; ++k) {
        float s = cn[k];
#pragma unroll
        for (int j = 0; j < DS; ++j) s = fmaf(-x[j], cb[k * CB_STRIDE + j], s);
        if (s <= m1 + win) {
            const double d = d2_fp64(x, cb + k * CB_STRIDE, DS);
            if (d < best) { best = d; bk = k; }
        }
    }
    return bk;
}

// Exact decision among a complete candidate list: FP32 direct differences (relative error
// below 1e-6 for Ds = 8), then FP64 among the FP32 near-ties; ties to the lowest index.
__device__ __forceinline__ int rerank(const float *x, const float *cb, const int *cand, int nc)
{
    float d1 = FLT_MAX, d2 = FLT_MAX;
    int k1 = 0x7fffffff;
    for (int i = 0; i < nc; ++i) {
        const float *c = cb + cand[i] * CB_STRIDE;
        float d = 0.0f;
#pragma unroll
        for (int j = 0; j < DS; ++j) {
            const float t = x[j] - c[j];
            d = fmaf(t, t, d);
        }
        if (d < d1 || (d == d1 && cand[i] < k1)) { d2 = d1; d1 = d; k1 = cand[i]; }
        else if (d < d2) { d2 = d; }
    }
    const float margin = 4e-6f * d2 + 1e-30f;
    if (d2 - d1 > margin) return k1;
    double best = DBL_MAX;
    int bk = 0x7fffffff;
    for (int i = 0; i < nc; ++i) {
        const float *c = cb + cand[i] * CB_STRIDE;
        float d = 0.0f;
#pragma unroll
        for (int j = 0; j < DS; ++j) {
            const float t = x[j] - c[j];
            d = fmaf(t, t, d);
        }
        if (d <= d1 + margin) {
            const double e = d2_fp64(x, c, DS);
            if (e < best || (e == best && cand[i] < bk)) { best = e; bk = cand[i]; }
        }
    }
    return bk;
}

__global__ void __launch_bounds__(kThreads, 1) pq_pass_tc_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                  const TcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = blockIdx.y, m0 = grp * G;
    const int Ks = a.Ks;
    const bool fit = a.part != nullptr;
    // chunk of this CTA (batched form): its rows, its share of the CTAs, its codebooks
    int chunk = 0, lb = blockIdx.x, gxc = gridDim.x;
    int64_t r0 = 0, r1 = a.N;
    if (a.blk_chunk) {
        chunk = a.blk_chunk[blockIdx.x];
        lb = blockIdx.x - a.chunk_blk[chunk];
        gxc = a.chunk_blk[chunk + 1] - a.chunk_blk[chunk];
        r0 = a.chunk_off[chunk];
        r1 = a.chunk_off[chunk + 1];
    }
    const int tiles_c = (int)((r1 - r0 + TM - 1) / TM);
    const float *Cc = a.C + (size_t)chunk * a.M * Ks * DS;

    float *xs = reinterpret_cast<float *>(sm + OFF_XS);
    unsigned char *aop = sm + OFF_A;
    unsigned char *bop = sm + OFF_B;
    float *cbf = reinterpret_cast<float *>(sm + OFF_CBF);
    float *cn = reinterpret_cast<float *>(sm + OFF_CN);
    float *acc = reinterpret_cast<float *>(sm + OFF_ACC);
    int *cnt = reinterpret_cast<int *>(sm + OFF_CNT);
    uint64_t *mb = reinterpret_cast<uint64_t *>(sm + OFF_MISC);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + OFF_MISC + 8 * MB_COUNT);
    float *mu = reinterpret_cast<float *>(sm + OFF_MISC + 128);           // [G][8]
    unsigned *bnd = reinterpret_cast<unsigned *>(sm + OFF_MISC + 256);    // [G][4] float bits: n', c', n, c maxima

    // ---- set-up: codeword mean, B operands, FP32 copies, norms, bounds ------
    if (tid < G * DS) {
        const int g = tid / DS, j = tid % DS;
        const float *Cm = Cc + (size_t)(m0 + g) * Ks * DS;
        float s = 0.0f;
        for (int k = 0; k < Ks; ++k) s += Cm[k * DS + j];
        mu[tid] = s / (float)Ks;
    }
    if (tid < G * 4) bnd[tid] = 0u;
    __syncthreads();
    for (int e = tid; e < G * KSMAX; e += kThreads) {
        const int g = e / KSMAX, k = e % KSMAX;
        float c[DS], cc[DS];
        float nc = 0.0f, n = 0.0f, norm2c = 0.0f;
        if (k < Ks) {
            const float *src = Cc + ((size_t)(m0 + g) * Ks + k) * DS;
#pragma unroll
            for (int j = 0; j < DS; ++j) {
                c[j] = src[j];
                cc[j] = c[j] - mu[g * DS + j];
                nc = fmaf(cc[j], cc[j], nc);
                n = fmaf(c[j], c[j], n);
            }
            norm2c = nc;
            nc *= 0.5f;
            n *= 0.5f;
        } else {
#pragma unroll
            for (int j = 0; j < DS; ++j) { c[j] = 0.0f; cc[j] = 0.0f; }
        }
#pragma unroll
        for (int j = 0; j < DS; ++j) cbf[(g * KSMAX + k) * CB_STRIDE + j] = c[j];
        cn[g * KSMAX + k] = n;
        float ch[DS], cl[DS];
#pragma unroll
        for (int j = 0; j < DS; ++j) {
            ch[j] = __bfloat162float(__float2bfloat16_rn(cc[j]));
            cl[j] = cc[j] - ch[j];
        }
        float nh, nl;
        if (k < Ks) {
            nh = __bfloat162float(__float2bfloat16_rn(nc));
            nl = nc - nh;
        } else {
            nh = 3.0e38f;  // padding codeword: score -3e38, never the maximum
            nl = 0.0f;
        }
        unsigned char *b0 = bop + (g * 2 + 0) * B_HALF;
        unsigned char *b1 = bop + (g * 2 + 1) * B_HALF;
        const uint4 w = make_uint4(pack_bf16(ch[0], ch[1]), pack_bf16(ch[2], ch[3]), pack_bf16(ch[4], ch[5]),
                                   pack_bf16(ch[6], ch[7]));
        *reinterpret_cast<uint4 *>(b0 + core_off(k, 0)) = w;
        *reinterpret_cast<uint4 *>(b0 + core_off(k, 8)) = w;
        *reinterpret_cast<uint4 *>(b1 + core_off(k, 0)) =
            make_uint4(pack_bf16(cl[0], cl[1]), pack_bf16(cl[2], cl[3]), pack_bf16(cl[4], cl[5]), pack_bf16(cl[6], cl[7]));
        *reinterpret_cast<uint4 *>(b1 + core_off(k, 8)) = make_uint4(pack_bf16(-nh, -nl), 0u, 0u, 0u);
        if (k < Ks) {
            atomicMax(bnd + g * 4 + 0, __float_as_uint(nc));
            atomicMax(bnd + g * 4 + 1, __float_as_uint(sqrtf(norm2c)));
            atomicMax(bnd + g * 4 + 2, __float_as_uint(n));
            atomicMax(bnd + g * 4 + 3, __float_as_uint(sqrtf(2.0f * n)));
        }
        if (fit) {
#pragma unroll
            for (int j = 0; j < DS; ++j) acc[(g * KSMAX + k) * ACC_STRIDE + j] = 0.0f;
            cnt[g * KSMAX + k] = 0;
        }
    }
    if (tid == 0) {
        mbar_init(smem_u32(mb + MB_FULL + 0), 1);
        mbar_init(smem_u32(mb + MB_FULL + 1), 1);
        mbar_init(smem_u32(mb + MB_EMPTY + 0), kCompute / 32);
        mbar_init(smem_u32(mb + MB_EMPTY + 1), kCompute / 32);
        for (int w = 0; w < 2; ++w) {
            mbar_init(smem_u32(mb + MB_AREADY + w), 4);
            mbar_init(smem_u32(mb + MB_MMA + w), 1);
            mbar_init(smem_u32(mb + MB_TFREE + w), 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tslot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;

    const int n_my = (tiles_c > lb) ? (tiles_c - 1 - lb) / gxc + 1 : 0;
    const int wsteps = 2 * n_my;  // steps of each warpgroup

    if (warp == 0) {
        // ---- producer: TMA loads of the row tiles -----------------------------
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < n_my; ++i) {
                const int s = i & 1;
                if (i >= 2 && !mbar_wait(smem_u32(mb + MB_EMPTY + s), ((i >> 1) - 1) & 1, a.err)) break;
                mbar_expect_tx(smem_u32(mb + MB_FULL + s), XS_BYTES);
                tma_load_2d(smem_u32(reinterpret_cast<unsigned char *>(xs) + s * XS_BYTES), &tmap, m0 * DS,
                            (int)(r0 + (int64_t)(lb + i * gxc) * TM), smem_u32(mb + MB_FULL + s));
                ++issued;
            }
            // our own copies must have landed before the CTA can leave
            for (int i = (issued > 2 ? issued - 2 : 0); i < issued; ++i)
                mbar_wait(smem_u32(mb + MB_FULL + (i & 1)), (i >> 1) & 1, a.err);
        }
    } else if (warp == 1) {
        // ---- MMA issue: lane w serves warpgroup w ------------------------------
        if (lane < 2) {
            const int w = lane;
            for (int u = 0; u < wsteps; ++u) {
                if (!mbar_wait(smem_u32(mb + MB_AREADY + w), u & 1, a.err)) break;
                if (u >= 1 && !mbar_wait(smem_u32(mb + MB_TFREE + w), (u - 1) & 1, a.err)) break;
                tc_after_sync();
                const int g = 2 * w + (u & 1), buf = u & 1;
                const uint32_t d = tmem + (uint32_t)(w * KSMAX);
                const unsigned char *ab = aop + (w * 2 + buf) * 2 * A_HALF;
                mma_bf16(d, smem_desc(smem_u32(ab)), smem_desc(smem_u32(bop + (g * 2 + 0) * B_HALF)), 0u);
                mma_bf16(d, smem_desc(smem_u32(ab + A_HALF)), smem_desc(smem_u32(bop + (g * 2 + 1) * B_HALF)), 1u);
                mma_commit(smem_u32(mb + MB_MMA + w));
            }
        }
    } else {
        // ---- compute warpgroups: thread = row = TMEM lane --------------------
        const int w = (warp - 2) >> 2;
        const int q = warp & 3;
        const int r = q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(w * KSMAX);
        float nb_prime[2], cb_prime[2], nb_orig[2], cb_orig[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int g = 2 * w + h;
            nb_prime[h] = __uint_as_float(bnd[g * 4 + 0]) * (1.0f + 1e-5f);
            cb_prime[h] = __uint_as_float(bnd[g * 4 + 1]) * (1.0f + 1e-5f);
            nb_orig[h] = __uint_as_float(bnd[g * 4 + 2]) * (1.0f + 4.0f * gamma_f32(DS + 1));
            cb_orig[h] = __uint_as_float(bnd[g * 4 + 3]) * (1.0f + 1e-5f);
        }
        float sse_s = 0.0f, sse_c = 0.0f;  // Kahan pair
        unsigned rechecks = 0;
        uint32_t code_pair = 0;
        for (int u = 0; u < wsteps; ++u) {
            const int i = u >> 1, h = u & 1, g = 2 * w + h, s = i & 1, buf = u & 1;
            const int64_t row = r0 + (int64_t)(lb + i * gxc) * TM + r;
            const float *stage = xs + s * (XS_BYTES / 4);
            // (a) A operand of this step
            if (h == 0 && !__all_sync(0xffffffffu, mbar_wait(smem_u32(mb + MB_FULL + s), (i >> 1) & 1, a.err))) break;
            const float4 v0 = *reinterpret_cast<const float4 *>(xs_row_chunk(stage, r, 2 * g));
            const float4 v1 = *reinterpret_cast<const float4 *>(xs_row_chunk(stage, r, 2 * g + 1));
            const float x[DS] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            {
                float xh[DS], xl[DS];
#pragma unroll
                for (int d = 0; d < DS; ++d) {
                    const float xc = x[d] - mu[g * DS + d];
                    xh[d] = __bfloat162float(__float2bfloat16_rn(xc));
                    xl[d] = xc - xh[d];
                }
                unsigned char *a0 = aop + (w * 2 + buf) * 2 * A_HALF;
                unsigned char *a1 = a0 + A_HALF;
                const uint4 wh = make_uint4(pack_bf16(xh[0], xh[1]), pack_bf16(xh[2], xh[3]), pack_bf16(xh[4], xh[5]),
                                            pack_bf16(xh[6], xh[7]));
                *reinterpret_cast<uint4 *>(a0 + core_off(r, 0)) = wh;
                *reinterpret_cast<uint4 *>(a0 + core_off(r, 8)) = make_uint4(
                    pack_bf16(xl[0], xl[1]), pack_bf16(xl[2], xl[3]), pack_bf16(xl[4], xl[5]), pack_bf16(xl[6], xl[7]));
                *reinterpret_cast<uint4 *>(a1 + core_off(r, 0)) = wh;
                *reinterpret_cast<uint4 *>(a1 + core_off(r, 8)) = make_uint4(pack_bf16(1.0f, 1.0f), 0u, 0u, 0u);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(mb + MB_AREADY + w));
            // (b) scores of this step
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(mb + MB_MMA + w), u & 1, a.err))) break;
            tc_after_sync();
            float xx = 0.0f;
#pragma unroll
            for (int d = 0; d < DS; ++d) {
                const float xc = x[d] - mu[g * DS + d];
                xx = fmaf(xc, xc, xx);
            }
            const float xn = sqrtf(xx) * (1.0f + 1e-5f);
            const float tt = xn + cb_prime[h];
            const float win = 2.0f * (kC1 * xn * cb_prime[h] + kC2 * nb_prime[h] + 1e-13f * tt * tt);

            float best = -FLT_MAX, cm2 = -FLT_MAX;
            int bestj = 0;
            float cmx[KSMAX / 32];
            float sv[32];
#pragma unroll
            for (int q2 = 0; q2 < 32; ++q2) sv[q2] = -FLT_MAX;
#pragma unroll 1
            for (int cp = 0; cp < KSMAX / 64; ++cp) {
                float v2[2][32];
                TC_LD32(tl + (uint32_t)(cp * 64), v2[0]);
                TC_LD32(tl + (uint32_t)(cp * 64 + 32), v2[1]);
                tc_wait_ld();
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const float *v = v2[hh];
                    float m16[16];
#pragma unroll
                    for (int q2 = 0; q2 < 16; ++q2) m16[q2] = fmaxf(v[2 * q2], v[2 * q2 + 1]);
#pragma unroll
                    for (int q2 = 0; q2 < 8; ++q2) m16[q2] = fmaxf(m16[2 * q2], m16[2 * q2 + 1]);
#pragma unroll
                    for (int q2 = 0; q2 < 4; ++q2) m16[q2] = fmaxf(m16[2 * q2], m16[2 * q2 + 1]);
                    const float cm = fmaxf(fmaxf(m16[0], m16[1]), fmaxf(m16[2], m16[3]));
                    cmx[2 * cp + hh] = cm;
                    const bool better = cm > best;
                    cm2 = better ? best : fmaxf(cm2, cm);
                    best = better ? cm : best;
                    bestj = better ? 2 * cp + hh : bestj;
#pragma unroll
                    for (int q2 = 0; q2 < 32; ++q2) sv[q2] = better ? v[q2] : sv[q2];
                }
            }
            const float theta = best - win;
            int ib = 0, nin = 0;
#pragma unroll
            for (int q2 = 31; q2 >= 0; --q2) {
                ib = (sv[q2] == best) ? q2 : ib;
                nin += (sv[q2] >= theta) ? 1 : 0;
            }
            int code = bestj * 32 + ib;
            const bool valid = row < r1;
            const bool unsure = valid && !(nin == 1 && cm2 < theta);
            if (__any_sync(0xffffffffu, unsure)) {
                // complete candidate set: the saved chunk, plus every other chunk reaching theta
                int cand[kMaxCand];
                int nc = 0;
                bool over = false;
                if (unsure) {
#pragma unroll
                    for (int q2 = 0; q2 < 32; ++q2)
                        if (sv[q2] >= theta) cand[nc++] = bestj * 32 + q2;
                }
#pragma unroll 1
                for (int c = 0; c < KSMAX / 32; ++c) {
                    const bool need = unsure && c != bestj && cmx[c] >= theta;
                    if (!__any_sync(0xffffffffu, need)) continue;
                    float v[32];
                    TC_LD32(tl + (uint32_t)(c * 32), v);
                    tc_wait_ld();
                    if (need) {
#pragma unroll
                        for (int q2 = 0; q2 < 32; ++q2) {
                            if (v[q2] >= theta) {
                                if (nc < kMaxCand) cand[nc++] = c * 32 + q2;
                                else over = true;
                            }
                        }
                    }
                }
                if (unsure) {
                    const float *cbg = cbf + g * KSMAX * CB_STRIDE;
                    code = over ? exact_code(x, cbg, cn + g * KSMAX, Ks, nb_orig[h], cb_orig[h]) : rerank(x, cbg, cand, nc);
                    ++rechecks;
                }
            }
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(mb + MB_TFREE + w));
            if (valid) {
                const float *c = cbf + (g * KSMAX + code) * CB_STRIDE;
                float e = 0.0f;
                float res[DS];
                const float4 c0 = *reinterpret_cast<const float4 *>(c);
                const float4 c1 = *reinterpret_cast<const float4 *>(c + 4);
                const float cv[DS] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int d = 0; d < DS; ++d) {
                    res[d] = x[d] - cv[d];
                    e = fmaf(res[d], res[d], e);
                }
                const float y = e - sse_c;  // Kahan accumulation of the squared error
                const float t2 = sse_s + y;
                sse_c = (t2 - sse_s) - y;
                sse_s = t2;
                if (fit) {
                    float *ac = acc + (g * KSMAX + code) * ACC_STRIDE;
#pragma unroll
                    for (int d = 0; d < DS; ++d) atomicAdd(ac + d, res[d]);
                    atomicAdd(cnt + g * KSMAX + code, 1);
                }
                code_pair |= (uint32_t)code << (8 * h);
                if (h == 1 && a.codes)
                    *reinterpret_cast<uint16_t *>(a.codes + row * a.M + m0 + 2 * w) = (uint16_t)code_pair;
            }
            if (h == 1) {
                code_pair = 0;
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(mb + MB_EMPTY + s));
            }
        }
        // ---- results of this CTA -------------------------------------------
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (fit) {
            for (int e = tid - 64; e < G * KSMAX; e += kCompute) {
                const int g = e / KSMAX, k = e % KSMAX;
                if (k >= Ks) continue;
                const size_t base = ((size_t)blockIdx.x * a.M + m0 + g) * Ks + k;
#pragma unroll
                for (int d = 0; d < DS; ++d) a.part[base * DS + d] = (double)acc[(g * KSMAX + k) * ACC_STRIDE + d];
                a.part_cnt[base] = cnt[g * KSMAX + k];
            }
        }
        double tot = (double)sse_s - (double)sse_c;
        tot = warp_sum(tot);
        if (a.sse && lane == 0) atomicAdd(a.sse, tot);
        const unsigned rc = warp_sum(rechecks);
        if (a.rechecks && lane == 0 && rc) atomicAdd(a.rechecks, (unsigned long long)rc);
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

__global__ void pq_finalize_residual_kernel(const double *__restrict__ part, const int *__restrict__ part_cnt, int gx,
                                            int M, int Ks, int ds, float *C, unsigned long long *empties, int n_chunks,
                                            const int *__restrict__ chunk_blk)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_chunks * M * Ks) return;
    const int c = idx / (M * Ks), m = (idx / Ks) % M, k = idx % Ks;
    const int b0 = chunk_blk ? chunk_blk[c] : 0, b1 = chunk_blk ? chunk_blk[c + 1] : gx;
    C += (size_t)c * M * Ks * ds;
    long long n = 0;
    for (int b = b0; b < b1; ++b) n += part_cnt[((size_t)b * M + m) * Ks + k];
    if (n == 0) {
        if (empties) atomicAdd(empties, 1ull);
        return;
    }
    for (int j = 0; j < ds; ++j) {
        double s = 0.0;
        for (int b = b0; b < b1; ++b) s = __dadd_rn(s, part[(((size_t)b * M + m) * Ks + k) * ds + j]);
        float *c = C + ((size_t)m * Ks + k) * ds + j;
        *c = __double2float_rn(__dadd_rn((double)*c, __ddiv_rn(s, (double)n)));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

bool tc_pass_supported(int D, int M, int Ks) { return M > 0 && D == M * DS && M % G == 0 && Ks >= 1 && Ks <= KSMAX; }

int pq_pass_tc_blocks(const PqPass &p)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    const int groups = p.M / G;
    const int64_t tiles = (p.N + TM - 1) / TM;
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, std::max(1, sms / groups)));
}

int launch_pq_pass_tc(PqPass &p, cudaStream_t s)
{
    if (!tc_pass_supported(p.D, p.M, p.Ks)) return fail(PQ_ENOTSUP, "BF16 tensor-core pass needs D/M == 8, M % 4 == 0");
    if (p.N >= (1LL << 31) / TM * TM) return fail(PQ_ENOTSUP, "BF16 tensor-core pass supports N < 2^31");
    if (p.codes && (reinterpret_cast<uintptr_t>(p.codes) & 3))
        return fail(PQ_EINVAL, "codes must be 4-byte aligned for the tensor-core pass");
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc) return fail(PQ_ECUDA, "cuTensorMapEncodeTiled unavailable");
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)p.D, (cuuint64_t)p.N};
    const cuuint64_t gstride[1] = {(cuuint64_t)p.D * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)(G * DS), (cuuint32_t)TM};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(p.X), gdim, gstride, box,
                            estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return fail(PQ_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    int dev = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    int *err = device_error_word(dev);
    if (!err) return fail(PQ_ENOMEM, "device error word");
    if (p.gx <= 0) p.gx = pq_pass_tc_blocks(p);
    TcArgs a;
    a.N = p.N;
    a.D = p.D;
    a.M = p.M;
    a.Ks = p.Ks;
    a.tiles = (int)((p.N + TM - 1) / TM);
    a.C = p.C;
    a.codes = p.codes;
    a.part = p.part;
    a.part_cnt = p.part_cnt;
    a.sse = p.sse;
    a.rechecks = p.rechecks;
    a.err = err;
    a.blk_chunk = p.blk_chunk;
    a.chunk_off = p.chunk_off;
    a.chunk_blk = p.chunk_blk;
    PQ_TRY_CUDA(cudaFuncSetAttribute(pq_pass_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    dim3 grid(p.gx, p.M / G);
    ProfScope ps("pq_pass_tc", s);
    pq_pass_tc_kernel<<<grid, kThreads, SMEM_BYTES, s>>>(map, a);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

int launch_pq_finalize_residual(const double *part, const int *part_cnt, int gx, int M, int Ks, int ds, float *C,
                                unsigned long long *empties, cudaStream_t s, int n_chunks, const int *chunk_blk)
{
    const int n = n_chunks * M * Ks;
    ProfScope ps("pq_finalize", s);
    pq_finalize_residual_kernel<<<(n + 127) / 128, 128, 0, s>>>(part, part_cnt, gx, M, Ks, ds, C, empties, n_chunks,
                                                                chunk_blk);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

}  // namespace pqgb
