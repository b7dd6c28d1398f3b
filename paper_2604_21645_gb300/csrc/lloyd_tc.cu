// lloyd_tc.cu -- PQ Lloyd pass on the tcgen05 tensor cores (Sec. 2.1: nearest
// codeword of every (row, subspace) and the mean update), BF16 operands with
// FP32 accumulation in tensor memory.
//
// Contraction.  Per subspace the scores S_k = x.c_k - ||c_k||^2/2 (argmax S_k
// == argmin ||x - c_k||^2) come from M=128 x N=128 MMAs over K=32 bf16 lanes,
// one for each half of the 256 codewords.  Both sides are first centred by the
// subspace's codeword mean mu (distances are translation invariant) and split
// into bf16 high and low parts, x' = xh + xl, c' = ch + cl,
// n' = ||c'||^2/2 = nh + nl:
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
// 32 (each load also returns the chunk's maximum, tcgen05.ld.red), keeps the
// eight chunk maxima and, in registers, the values of the best chunk, and
// accepts the argmax when no other score lies within twice the error bound of
// it.  For the other rows (about 0.2% on clustered data) every codeword that
// may be the nearest -- the saved chunk's scores within the bound, and all
// codewords of any other chunk whose maximum reaches it -- is re-ranked exactly
// from the FP32 codebook copy in shared memory: FP32 direct differences, then
// FP64 among the FP32 near-ties, the decision rule of the CPU reference.
// Codes are exact.
//
// Update.  Residuals x - c_code are added with shared-memory int32 atomics, in
// the exact fixed-point format of common.cuh (FixFmt), into per-CTA sums that
// each CTA writes as int64; the finalise kernel adds the CTAs in int64 and moves
// every codeword by the float-float mean residual of its members.
//
// Pipeline (one CTA per SM, a group of 2 subspaces, persistent over row tiles
// of 128).  Warp 0 issues TMA loads of 128 x 16 float tiles (64B swizzle) into
// five stages.  Warp 3 (the operand warp) turns each tile into the bf16 A
// operands of both subspaces (four A stages).  Warps 1 and 2 issue the MMAs of
// subspace 0 and 1.  Warps 4-7 and 8-11 (the epilogue
// warpgroups; thread = row = TMEM lane) own subspace 0 and 1 and two 128-column
// TMEM buffers each, one per codeword half: the MMA of a half is issued as soon
// as the epilogue has read the same half of the previous tile, so the tensor
// core works while the epilogue runs.  Warpgroup 0 hands part of its registers
// to the epilogue warpgroups (setmaxnreg).  All hand-offs are mbarriers; every wait
// is bounded, and a timed-out wait records PQ_ETIMEOUT and lets the CTA unwind
// (its copies and MMAs waited for, its tensor memory freed).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

constexpr int G = 2;        // subspaces per CTA
constexpr int TM = 128;     // rows per tile
constexpr int KSMAX = 256;  // codewords
constexpr int NH = 128;     // codewords per MMA (one TMEM buffer)
constexpr int DS = 8;       // subspace width
constexpr int NXS = 5;      // X stages
constexpr int NAS = 4;      // A stages: the operand warp runs up to three tiles ahead of the MMAs
constexpr int kOpWarps = 1;                         // operand warps
constexpr int kOpRows = TM / (32 * kOpWarps);       // rows per operand thread
constexpr int kThreads = 96 + 32 * kOpWarps + 256;  // TMA warp, two MMA warps, operand warps, two epilogue warpgroups
constexpr int kOp0 = 96;                            // first operand thread
constexpr int kEpi0 = kOp0 + 32 * kOpWarps;         // first epilogue thread
// Registers: the block is launched with kRegLaunch per thread (12 warps fill the register file);
// warpgroup 0 (TMA, MMA and operand warps) then hands registers over to the two epilogue
// warpgroups (setmaxnreg), which hold a loaded 32-score chunk and the best chunk so far.
constexpr int kRegLaunch = 168;
constexpr int kRegLo = 112;
constexpr int kRegHi = 192;
static_assert(kEpi0 == 128, "warpgroup 0 must be exactly the TMA, MMA and operand warps");
static_assert(128 * kRegLo + 256 * kRegHi <= kThreads * kRegLaunch,
              "register hand-over exceeds the registers the block is launched with");
static_assert(kThreads * kRegLaunch <= 65536, "launch registers exceed the SM's register file");

constexpr int XS_BYTES = TM * G * DS * 4;  // 8 KB per stage (rows of 64 B)
constexpr int A_K16 = TM * 16 * 2;         // 4 KB: 128 rows x K=16 bf16
constexpr int A_SUB = 2 * A_K16;           // K = 32
constexpr int B_K16 = KSMAX * 16 * 2;      // 8 KB: 256 codewords x K=16
constexpr int B_SUB = 2 * B_K16;
constexpr int CB_STRIDE = 12;  // FP32 codeword rows: 16-byte aligned, spread over bank groups
constexpr int ACC_STRIDE = 9;  // update sums: conflict-free scalar atomics
constexpr int OFF_XS = 0;
constexpr int OFF_A = OFF_XS + NXS * XS_BYTES;  // [stage][g]
constexpr int OFF_B = OFF_A + NAS * G * A_SUB;  // [g]
constexpr int OFF_CBF = OFF_B + G * B_SUB;
constexpr int ACC_BYTES = G * KSMAX * ACC_STRIDE * 4;
constexpr int OFF_ACC = OFF_CBF + G * KSMAX * CB_STRIDE * 4;  // int32 [3][G][KSMAX][ACC_STRIDE]: high, low, float
constexpr int OFF_CNT = OFF_ACC + 3 * ACC_BYTES;
constexpr int OFF_MISC = OFF_CNT + G * KSMAX * 4;
constexpr int MISC_BYTES = 512;
constexpr int SMEM_BYTES = OFF_MISC + MISC_BYTES + 1024;  // + alignment slack
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory of the tensor-core pass exceeds one CTA's limit");

// mbarrier slots in the misc area
constexpr int MB_FULL = 0;                       // [NXS]  TMA -> operand + epilogue warps
constexpr int MB_EMPTY = MB_FULL + NXS;          // [NXS]  operand + epilogue warps -> TMA
constexpr int MB_AREADY = MB_EMPTY + NXS;        // [NAS][G] operand warp -> MMA warp g
constexpr int MB_AFREE = MB_AREADY + NAS * G;    // [NAS][G] MMA completion -> operand warp
constexpr int MB_MMAF = MB_AFREE + NAS * G;      // [G][2]  MMA completion of a half -> epilogue warpgroup g
constexpr int MB_TFREE = MB_MMAF + G * 2;        // [G][2]  epilogue warpgroup g (4 warps) -> MMA warp g
constexpr int MB_DRAIN = MB_TFREE + G * 2;       // [G]     final commit of MMA warp g
constexpr int MB_COUNT = MB_DRAIN + G;
constexpr int MISC_TSLOT = 8 * MB_COUNT;
constexpr int MISC_MU = 320;                     // [G][8] floats
constexpr int MISC_BND = 384;                    // [G][4] float bits
static_assert(MISC_TSLOT + 4 <= MISC_MU, "mbarriers overlap the misc data");

constexpr float kC1 = 7.5e-5f;
constexpr float kC2 = 2.7e-5f;

struct TcArgs {
    int64_t N;
    int D, M, Ks;
    int tiles;
    const float *C;
    uint8_t *codes;
    Partials part;
    double *sse;
    unsigned long long *rechecks;
    int *err;
    const int *blk_chunk;      // optional chunk table (batched form)
    const int64_t *chunk_off;
    const int *chunk_blk;
    // persistent form (the batched Lloyd iterations in one launch): `iters` passes over `units`
    // (x, group) units of the chunk table (x < gxu); the CTAs take the units of every pass in order
    // from the counter *next; after each pass over a (chunk, group) the last of its units to finish
    // moves its codebooks (Cw) and publishes the pass in ready[chunk * groups + group], counting
    // arrivals in arrive[]
    int iters, units, gxu;
    float *Cw;
    int *arrive, *ready, *next;
    unsigned spin;             // poll budget of a unit's wait for the previous pass
    long long *counts;         // member counts of the last update, or null
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

// kind::f16, D = f32, A = B = bf16, both K-major, N = 128, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NH >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

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

// 32 consecutive columns of this thread's TMEM lane (one row's scores) and, by the load's max
// reduction, their largest value m, so a chunk's maximum needs no instructions of its own.
// tcgen05.ld writes its registers asynchronously: the wait names them as in/out operands so that
// the compiler cannot move a use of the loaded values above it.
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

// 16-byte chunk c (0..3) of row r in a 64B-swizzled TMA stage (row = 64 bytes)
__device__ __forceinline__ const float4 *xs_chunk(const float *stage, int r, int c)
{
    return reinterpret_cast<const float4 *>(stage + r * 16 + ((c ^ ((r >> 1) & 3)) << 2));
}

// FP32 squared distance of one subspace row to a codeword, direct differences in dimension order.
__device__ __forceinline__ float d2_fp32(const float *x, const float *c)
{
    float d = 0.0f;
#pragma unroll
    for (int j = 0; j < DS; ++j) {
        const float t = x[j] - c[j];
        d = fmaf(t, t, d);
    }
    return d;
}

// Merge of two running (best, index, second-best) triples; ties of the best go to the lower index.
__device__ __forceinline__ void top2_merge(float &d1, int &k1, float &d2, float e1, int j1, float e2)
{
    if (e1 < d1 || (e1 == d1 && j1 < k1)) {
        d2 = fminf(d1, e2);
        d1 = e1;
        k1 = j1;
    } else {
        d2 = fminf(d2, e1);
    }
}

// Exact decision for the uncertain rows of a warp, warp-cooperatively.  The warp takes
// the uncertain lanes one at a time; each lane scores one candidate codeword of that row
// per pass -- the codewords of the saved chunk `bestj` whose scores reach the bound (bits
// of svmask), then all codewords of the chunks in cmask -- by FP32 direct differences
// (relative error below 1e-6 for Ds = 8), and a warp reduction gives the best and
// second-best distances (ties to the lower index).  Unless the FP32 gap settles it, the
// candidates within the FP32 margin are compared in FP64 (ties to the lower index) -- the
// decision rule of the CPU reference.  Every lane of the warp must call this.
__device__ __forceinline__ void decide_exact_warp(bool unsure, float4 v0, float4 v1, const float *cb,
                                                  unsigned svmask, int bestj, unsigned cmask, int Ks, int &code)
{
    const int lane = threadIdx.x & 31;
    for (unsigned todo = __ballot_sync(0xffffffffu, unsure); todo; todo &= todo - 1) {
        const int u = __ffs(todo) - 1;
        const float x[DS] = {__shfl_sync(0xffffffffu, v0.x, u), __shfl_sync(0xffffffffu, v0.y, u),
                             __shfl_sync(0xffffffffu, v0.z, u), __shfl_sync(0xffffffffu, v0.w, u),
                             __shfl_sync(0xffffffffu, v1.x, u), __shfl_sync(0xffffffffu, v1.y, u),
                             __shfl_sync(0xffffffffu, v1.z, u), __shfl_sync(0xffffffffu, v1.w, u)};
        const unsigned sm = __shfl_sync(0xffffffffu, svmask, u);
        const unsigned cm = __shfl_sync(0xffffffffu, cmask, u);
        const int bj = __shfl_sync(0xffffffffu, bestj, u);
        float d1 = FLT_MAX, d2 = FLT_MAX;
        int k1 = INT_MAX;
        if ((sm >> lane) & 1u) {
            const int k = bj * 32 + lane;
            top2_merge(d1, k1, d2, d2_fp32(x, cb + k * CB_STRIDE), k, FLT_MAX);
        }
        for (unsigned m = cm; m; m &= m - 1) {
            const int k = (__ffs(m) - 1) * 32 + lane;
            if (k < Ks) top2_merge(d1, k1, d2, d2_fp32(x, cb + k * CB_STRIDE), k, FLT_MAX);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float e1 = __shfl_xor_sync(0xffffffffu, d1, o);
            const int j1 = __shfl_xor_sync(0xffffffffu, k1, o);
            const float e2 = __shfl_xor_sync(0xffffffffu, d2, o);
            top2_merge(d1, k1, d2, e1, j1, e2);
        }
        int result = k1;
        const float margin = 4e-6f * d2 + 1e-30f;
        if (!(d2 - d1 > margin)) {
            const float lim = d1 + margin;
            double best = DBL_MAX;
            int bk = INT_MAX;
            auto fp64 = [&](int k) {
                const float *c = cb + k * CB_STRIDE;
                if (d2_fp32(x, c) <= lim) {
                    const double e = d2_fp64(x, c, DS);
                    if (e < best || (e == best && k < bk)) {
                        best = e;
                        bk = k;
                    }
                }
            };
            if ((sm >> lane) & 1u) fp64(bj * 32 + lane);
            for (unsigned m = cm; m; m &= m - 1) {
                const int k = (__ffs(m) - 1) * 32 + lane;
                if (k < Ks) fp64(k);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double e = __shfl_xor_sync(0xffffffffu, best, o);
                const int j = __shfl_xor_sync(0xffffffffu, bk, o);
                if (e < best || (e == best && j < bk)) {
                    best = e;
                    bk = j;
                }
            }
            result = bk;
        }
        if (lane == u) code = result;
    }
}

// PERSIST: the persistent form (see TcArgs): the CTA runs its units pass after pass, waiting before
// a unit for the previous pass of its (chunk, group) to be published; no register hand-over.
template <bool PERSIST>
__global__ void __maxnreg__(kRegLaunch) pq_pass_tc_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                  const TcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    // aligned by an offset from the shared array itself, so that the compiler keeps every access
    // below in the shared address space (shared loads, stores and atomics, not generic ones)
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem_raw);
    unsigned char *sm = smem_raw + (((sbase + 1023u) & ~1023u) - sbase);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Ks = a.Ks;
    const bool fit = a.part.active();

    float *xs = reinterpret_cast<float *>(sm + OFF_XS);
    unsigned char *aop = sm + OFF_A;
    unsigned char *bop = sm + OFF_B;
    float *cbf = reinterpret_cast<float *>(sm + OFF_CBF);
    int *acch = reinterpret_cast<int *>(sm + OFF_ACC);
    int *accl = acch + ACC_BYTES / 4;
    float *accf = reinterpret_cast<float *>(accl + ACC_BYTES / 4);
    int *cnt = reinterpret_cast<int *>(sm + OFF_CNT);
    uint64_t *mb = reinterpret_cast<uint64_t *>(sm + OFF_MISC);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + OFF_MISC + MISC_TSLOT);
    float *mu = reinterpret_cast<float *>(sm + OFF_MISC + MISC_MU);
    unsigned *bnd = reinterpret_cast<unsigned *>(sm + OFF_MISC + MISC_BND);  // [G][2] float bits: n', ||c'|| maxima
    auto bar = [&](int slot) { return smem_u32(mb + slot); };
    __shared__ int s_flag;

    // tensor memory, held for the whole launch
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tslot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;

    const int n_iter = PERSIST ? a.iters : 1;
    __shared__ int s_q;
    // the units, pass after pass: a CTA takes the next one in order (pass t's units all come before
    // pass t + 1's, so a unit only waits for units already taken, by CTAs that are all resident)
    for (int q_local = 0;; ++q_local) {
    int q;
    if constexpr (PERSIST) {
        if (tid == 0) s_q = atomicAdd(a.next, 1);
        __syncthreads();
        q = s_q;
        if (q >= a.iters * a.units) break;
    } else {
        if (q_local > 0) break;
        q = 0;
    }
    const int it = PERSIST ? q / a.units : 0;
    const int uu = PERSIST ? q % a.units : 0;
    const int ux = PERSIST ? uu % a.gxu : (int)blockIdx.x;
    const int grp = PERSIST ? uu / a.gxu : (int)blockIdx.y, m0 = grp * G;
    // chunk of this unit (batched form): its rows, its share of the units, its codebooks
    int chunk = 0, lb = ux, gxc = PERSIST ? a.gxu : (int)gridDim.x;
    int64_t r0 = 0, r1 = a.N;
    if (a.blk_chunk) {
        chunk = a.blk_chunk[ux];
        lb = ux - a.chunk_blk[chunk];
        gxc = a.chunk_blk[chunk + 1] - a.chunk_blk[chunk];
        r0 = a.chunk_off[chunk];
        r1 = a.chunk_off[chunk + 1];
    }
    const int tiles_c = (int)((r1 - r0 + TM - 1) / TM);
    const float *Cc = a.C + (size_t)chunk * a.M * Ks * DS;
    const int cg = chunk * (a.M / G) + grp;
    if (PERSIST && it > 0) {
        // the previous pass over this (chunk, group) has been published (bounded wait)
        if (tid == 0) {
            int ok = 1;
            for (unsigned spin = 0; *(volatile int *)(a.ready + cg) < it; ++spin) {
                if (spin > a.spin) {
                    atomicCAS(a.err, 0, PQ_ETIMEOUT);
                    ok = 0;
                    break;
                }
                if ((spin & 255) == 255 && *(volatile int *)a.err != 0) {
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
            __threadfence();
            s_flag = ok;
        }
        __syncthreads();
        if (!s_flag) break;
    }

    // ---- set-up: codeword mean, B operands, FP32 copies, bounds -------------
    if (tid < G * DS) {
        const int g = tid / DS, j = tid % DS;
        const float *Cm = Cc + (size_t)(m0 + g) * Ks * DS;
        float s = 0.0f;
        for (int k = 0; k < Ks; ++k) s += __ldcg(Cm + k * DS + j);
        mu[tid] = s / (float)Ks;
    }
    if (tid < G * 4) bnd[tid] = 0u;
    __syncthreads();
    for (int e = tid; e < G * KSMAX; e += kThreads) {
        const int g = e / KSMAX, k = e % KSMAX;
        float c[DS], cc[DS];
        float nc = 0.0f;
        if (k < Ks) {
            const float *src = Cc + ((size_t)(m0 + g) * Ks + k) * DS;
#pragma unroll
            for (int j = 0; j < DS; ++j) {
                c[j] = __ldcg(src + j);
                cc[j] = c[j] - mu[g * DS + j];
                nc = fmaf(cc[j], cc[j], nc);
            }
        } else {
#pragma unroll
            for (int j = 0; j < DS; ++j) { c[j] = 0.0f; cc[j] = 0.0f; }
        }
        const float norm2c = nc;
        nc *= 0.5f;
#pragma unroll
        for (int j = 0; j < DS; ++j) cbf[(g * KSMAX + k) * CB_STRIDE + j] = c[j];
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
        unsigned char *b0 = bop + g * B_SUB;
        unsigned char *b1 = b0 + B_K16;
        const uint4 w = make_uint4(pack_bf16(ch[0], ch[1]), pack_bf16(ch[2], ch[3]), pack_bf16(ch[4], ch[5]),
                                   pack_bf16(ch[6], ch[7]));
        *reinterpret_cast<uint4 *>(b0 + core_off(k, 0)) = w;
        *reinterpret_cast<uint4 *>(b0 + core_off(k, 8)) = w;
        *reinterpret_cast<uint4 *>(b1 + core_off(k, 0)) =
            make_uint4(pack_bf16(cl[0], cl[1]), pack_bf16(cl[2], cl[3]), pack_bf16(cl[4], cl[5]), pack_bf16(cl[6], cl[7]));
        *reinterpret_cast<uint4 *>(b1 + core_off(k, 8)) = make_uint4(pack_bf16(-nh, -nl), 0u, 0u, 0u);
        if (k < Ks) {
            atomicMax(bnd + g * 2 + 0, __float_as_uint(nc));
            atomicMax(bnd + g * 2 + 1, __float_as_uint(sqrtf(norm2c)));
        }
        if (fit) {
#pragma unroll
            for (int j = 0; j < DS; ++j) {
                acch[(g * KSMAX + k) * ACC_STRIDE + j] = 0;
                accl[(g * KSMAX + k) * ACC_STRIDE + j] = 0;
                accf[(g * KSMAX + k) * ACC_STRIDE + j] = 0.0f;
            }
            cnt[g * KSMAX + k] = 0;
        }
    }
    // constant K lanes 24..31 of every A stage: [1 1 0 0 0 0 0 0]
    for (int e = tid; e < NAS * G * TM; e += kThreads) {
        unsigned char *a1 = aop + (e / TM) * A_SUB + A_K16;
        *reinterpret_cast<uint4 *>(a1 + core_off(e % TM, 8)) = make_uint4(pack_bf16(1.0f, 1.0f), 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int s = 0; s < NXS; ++s) {
            mbar_init(bar(MB_FULL + s), 1);
            mbar_init(bar(MB_EMPTY + s), kOpWarps + 8);
        }
        for (int i = 0; i < NAS * G; ++i) {
            mbar_init(bar(MB_AREADY + i), kOpWarps);
            mbar_init(bar(MB_AFREE + i), 1);
        }
        for (int i = 0; i < G * 2; ++i) {
            mbar_init(bar(MB_MMAF + i), 1);
            mbar_init(bar(MB_TFREE + i), 4);
        }
        for (int g = 0; g < G; ++g) mbar_init(bar(MB_DRAIN + g), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();

    const int n_my = (tiles_c > lb) ? (tiles_c - 1 - lb) / gxc + 1 : 0;

    if (warp < kEpi0 / 32) {
        if constexpr (!PERSIST) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegLo));
    if (warp == 0) {
        // ---- producer: TMA loads of the row tiles -----------------------------
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < n_my; ++i) {
                const int s = i % NXS;
                if (i >= NXS && !mbar_wait(bar(MB_EMPTY + s), ((i / NXS) - 1) & 1, a.err)) break;
                mbar_expect_tx(bar(MB_FULL + s), XS_BYTES);
                tma_load_2d(smem_u32(reinterpret_cast<unsigned char *>(xs) + s * XS_BYTES), &tmap, m0 * DS,
                            (int)(r0 + (int64_t)(lb + i * gxc) * TM), bar(MB_FULL + s));
                ++issued;
            }
            // our own copies must have landed before the CTA can leave
            for (int i = (issued > NXS ? issued - NXS : 0); i < issued; ++i)
                mbar_wait(bar(MB_FULL + i % NXS), (i / NXS) & 1, a.err);
        }
    } else if (warp <= G) {
        // ---- MMA issue: warp 1 + g serves subspace g (one warp each, so that a wait of
        // one never holds up the other) --------------------------------------------
        if (lane == 0) {
            const int g = warp - 1;
            for (int i = 0; i < n_my; ++i) {
                const int as = i % NAS;
                if (!mbar_wait(bar(MB_AREADY + as * G + g), (i / NAS) & 1, a.err)) break;
                bool ok = true;
                for (int h = 0; h < 2 && ok; ++h) {
                    if (i >= 1 && !mbar_wait(bar(MB_TFREE + g * 2 + h), (i - 1) & 1, a.err)) {
                        ok = false;
                        break;
                    }
                    tc_after_sync();
                    const uint32_t d = tmem + (uint32_t)((g * 2 + h) * NH);
                    const unsigned char *ab = aop + (as * G + g) * A_SUB;
                    const unsigned char *bb = bop + g * B_SUB + h * (NH / 8) * 256;
                    mma_bf16(d, smem_desc(smem_u32(ab)), smem_desc(smem_u32(bb)), 0u);
                    mma_bf16(d, smem_desc(smem_u32(ab + A_K16)), smem_desc(smem_u32(bb + B_K16)), 1u);
                    mma_commit(bar(MB_MMAF + g * 2 + h));
                }
                if (!ok) break;
                mma_commit(bar(MB_AFREE + as * G + g));
            }
            // every MMA of this lane has completed before the tensor memory is freed
            mma_commit(bar(MB_DRAIN + g));
            mbar_wait(bar(MB_DRAIN + g), 0, a.err);
        }
    } else {
        // ---- operand warp: bf16 A operands of both subspaces, rows t + 32 rr
        const int t = tid - kOp0;
        for (int i = 0; i < n_my; ++i) {
            const int s = i % NXS, as = i % NAS;
            if (!__all_sync(0xffffffffu, mbar_wait(bar(MB_FULL + s), (i / NXS) & 1, a.err))) break;
            const float *stage = xs + s * (XS_BYTES / 4);
            float4 v[kOpRows][4];
#pragma unroll
            for (int rr = 0; rr < kOpRows; ++rr)
#pragma unroll
                for (int c = 0; c < 4; ++c) v[rr][c] = *xs_chunk(stage, t + 32 * kOpWarps * rr, c);
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(MB_EMPTY + s));
            bool ok = true;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (i >= NAS &&
                    !__all_sync(0xffffffffu, mbar_wait(bar(MB_AFREE + as * G + g), ((i / NAS) - 1) & 1, a.err))) {
                    ok = false;
                    break;
                }
                unsigned char *a0 = aop + (as * G + g) * A_SUB;
#pragma unroll
                for (int rr = 0; rr < kOpRows; ++rr) {
                    const int r = t + 32 * kOpWarps * rr;
                    const float x[DS] = {v[rr][2 * g].x, v[rr][2 * g].y, v[rr][2 * g].z, v[rr][2 * g].w,
                                         v[rr][2 * g + 1].x, v[rr][2 * g + 1].y, v[rr][2 * g + 1].z, v[rr][2 * g + 1].w};
                    // high parts packed straight from the centred pair, low parts from their exact
                    // bf16 values (bf16 -> float is a 16-bit shift)
                    float xl[DS];
                    uint32_t hw[DS / 2];
#pragma unroll
                    for (int d = 0; d < DS; d += 2) {
                        const float c0 = x[d] - mu[g * DS + d], c1 = x[d + 1] - mu[g * DS + d + 1];
                        hw[d / 2] = pack_bf16(c0, c1);
                        xl[d] = c0 - __uint_as_float(hw[d / 2] << 16);
                        xl[d + 1] = c1 - __uint_as_float(hw[d / 2] & 0xffff0000u);
                    }
                    const uint4 wh = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4 *>(a0 + core_off(r, 0)) = wh;
                    *reinterpret_cast<uint4 *>(a0 + core_off(r, 8)) =
                        make_uint4(pack_bf16(xl[0], xl[1]), pack_bf16(xl[2], xl[3]), pack_bf16(xl[4], xl[5]),
                                   pack_bf16(xl[6], xl[7]));
                    *reinterpret_cast<uint4 *>(a0 + A_K16 + core_off(r, 0)) = wh;
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(MB_AREADY + as * G + g));
            }
            if (!ok) break;
        }
    }
    } else {
        if constexpr (!PERSIST) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegHi));
        // ---- epilogue warpgroups: thread = row = TMEM lane, warpgroup g = subspace g
        const int g = (tid - kEpi0) >> 7;
        const int r = (warp & 3) * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(g * 2 * NH);
        const float nb_prime = __uint_as_float(bnd[g * 2 + 0]) * (1.0f + 1e-5f);
        const float cb_prime = __uint_as_float(bnd[g * 2 + 1]) * (1.0f + 1e-5f);
        const float *cbg = cbf + g * KSMAX * CB_STRIDE;
        float sse_s = 0.0f, sse_c = 0.0f;  // Kahan pair
        unsigned rechecks = 0;
        // one format for every CTA of the chunk: the row bound is the busiest CTA's rows
        const int64_t rows_bound = (int64_t)((tiles_c + gxc - 1) / gxc) * TM;
        const FixFmt fx = fix_format(rows_bound, 2.0f * __uint_as_float(bnd[g * 2 + 1]));
        for (int i = 0; i < n_my; ++i) {
            const int s = i % NXS;
            const int64_t row = r0 + (int64_t)(lb + i * gxc) * TM + r;
            if (!__all_sync(0xffffffffu, mbar_wait(bar(MB_FULL + s), (i / NXS) & 1, a.err))) break;
            const float *stage = xs + s * (XS_BYTES / 4);
            float xx = 0.0f;
            {
                const float4 v0 = *xs_chunk(stage, r, 2 * g);
                const float4 v1 = *xs_chunk(stage, r, 2 * g + 1);
                const float x[DS] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                for (int d = 0; d < DS; ++d) {
                    const float xc = x[d] - mu[g * DS + d];
                    xx = fmaf(xc, xc, xx);
                }
            }
            // sqrt as x * rsqrt(x): a few ulp, far inside the 1e-5 inflation
            const float xn = (xx > 0.0f ? xx * rsqrtf(xx) : 0.0f) * (1.0f + 1e-5f);
            const float tt = xn + cb_prime;
            const float win = 2.0f * (kC1 * xn * cb_prime + kC2 * nb_prime + 1e-13f * tt * tt);

            // scores, two halves of 128 codewords, each in its own TMEM buffer.  A load returns after
            // ~30 cycles, so chunks are loaded one at a time; the best chunk so far is copied in
            // registers (a shared-memory copy would put ~2k wavefronts per tile on the shared pipe).
            float best = -FLT_MAX, cm2 = -FLT_MAX;
            int bestj = 0;
            float cmx[KSMAX / 32];
            float sv[32];
            bool ok = __all_sync(0xffffffffu, mbar_wait(bar(MB_MMAF + g * 2 + 0), i & 1, a.err));
            if (!ok) break;
            tc_after_sync();
#pragma unroll
            for (int j = 0; j < KSMAX / 32; ++j) {
                if (j == NH / 32) {
                    // every load of the first buffer has completed: hand it back to the MMA warp
                    tc_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar(MB_TFREE + g * 2 + 0));
                    ok = __all_sync(0xffffffffu, mbar_wait(bar(MB_MMAF + g * 2 + 1), i & 1, a.err));
                    if (!ok) break;
                    tc_after_sync();
                }
                float v[32], cm;
                TC_LDMAX32(tl + (uint32_t)(j * 32), v, cm);
                TC_WAITMAX32(v, cm);
                cmx[j] = cm;
                const bool better = cm > best;
                cm2 = better ? best : fmaxf(cm2, cm);
                best = better ? cm : best;
                bestj = better ? j : bestj;
#pragma unroll
                for (int c = 0; c < 32; ++c) sv[c] = (j == 0 || better) ? v[c] : sv[c];
            }
            if (!ok) break;
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(MB_TFREE + g * 2 + 1));
            // the row again (not kept in registers across the chunks); the stage is not read again:
            // order the reads before the TMA that will refill it
            const float4 v0 = *xs_chunk(stage, r, 2 * g);
            const float4 v1 = *xs_chunk(stage, r, 2 * g + 1);
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(MB_EMPTY + s));
            const float x[DS] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            // certain when the best chunk holds exactly one score >= theta and no other chunk reaches it;
            // the sum below packs that count (low 6 bits) and the score's position (bits 6..)
            const float theta = best - win;
            // four independent partial sums (exact small integers, so the order does not matter)
            float tp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int q = 0; q < 32; ++q) tp[q & 3] = fmaf(sv[q] >= theta ? 1.0f : 0.0f, (float)(1 + 64 * q), tp[q & 3]);
            const int ti = (int)((tp[0] + tp[1]) + (tp[2] + tp[3]));
            int code = bestj * 32 + (ti >> 6);
            const bool valid = row < r1;
            const bool unsure = valid && !((ti & 63) == 1 && cm2 < theta);
            if (__any_sync(0xffffffffu, unsure)) {
                unsigned cmask = 0, svmask = 0;
#pragma unroll
                for (int c = 0; c < KSMAX / 32; ++c) cmask |= (c != bestj && cmx[c] >= theta) ? (1u << c) : 0u;
#pragma unroll
                for (int q = 0; q < 32; ++q) svmask |= (sv[q] >= theta) ? (1u << q) : 0u;
                decide_exact_warp(unsure, v0, v1, cbg, svmask, bestj, cmask, Ks, code);
                rechecks += unsure ? 1u : 0u;
            }
            if (valid) {
                const float *c = cbg + code * CB_STRIDE;
                float res[DS];
                const float4 c0 = *reinterpret_cast<const float4 *>(c);
                const float4 c1 = *reinterpret_cast<const float4 *>(c + 4);
                const float cv[DS] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int d = 0; d < DS; ++d) res[d] = x[d] - cv[d];
                if (a.sse) {
                    float e = 0.0f;
#pragma unroll
                    for (int d = 0; d < DS; ++d) e = fmaf(res[d], res[d], e);
                    const float y = e - sse_c;  // Kahan accumulation of the squared error
                    const float t2 = sse_s + y;
                    sse_c = (t2 - sse_s) - y;
                    sse_s = t2;
                }
                if (fit) {
                    const int o = (g * KSMAX + code) * ACC_STRIDE;
                    int q[DS];
                    bool big = false;
#pragma unroll
                    for (int d = 0; d < DS; ++d) {
                        const float t = __fmul_rn(res[d], fx.scale);
                        big |= !(fabsf(t) < fx.lim);
                        q[d] = __float2int_rn(t);
                    }
                    if (!big) {
#pragma unroll
                        for (int d = 0; d < DS; ++d) {
                            atomicAdd(acch + o + d, q[d] >> fx.L);
                            atomicAdd(accl + o + d, q[d] & ((1 << fx.L) - 1));
                        }
                    } else {
#pragma unroll
                        for (int d = 0; d < DS; ++d) atomicAdd(accf + o + d, res[d]);
                    }
                    atomicAdd(cnt + g * KSMAX + code, 1);
                }
                if (a.codes) a.codes[row * a.M + m0 + g] = (uint8_t)code;
            }
        }
        // ---- results of this CTA -------------------------------------------
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (fit) {
            const int64_t rows_bound = (int64_t)((tiles_c + gxc - 1) / gxc) * TM;
            for (int e = tid - kEpi0; e < G * KSMAX; e += 256) {
                const int gg = e / KSMAX, k = e % KSMAX;
                if (k >= Ks) continue;
                const size_t base = ((size_t)ux * a.M + m0 + gg) * Ks + k;
                const FixFmt f = fix_format(rows_bound, 2.0f * __uint_as_float(bnd[gg * 2 + 1]));
                const int o = (gg * KSMAX + k) * ACC_STRIDE;
#pragma unroll
                for (int d = 0; d < DS; ++d) {
                    a.part.q[base * DS + d] = (long long)acch[o + d] * (1LL << f.L) + (long long)accl[o + d];
                    a.part.o[base * DS + d] = accf[o + d];
                }
                a.part.cnt[base] = cnt[gg * KSMAX + k];
                if (lb == 0 && k == 0) a.part.F[chunk * a.M + m0 + gg] = f.F;
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
    if constexpr (PERSIST) {
        // the last unit of this (chunk, group) to finish the pass moves its codebooks and
        // publishes the pass
        if (tid == 0) {
            __threadfence();
            s_flag = atomicAdd(a.arrive + cg, 1) == (it + 1) * gxc - 1;
            __threadfence();
        }
        __syncthreads();
        if (s_flag) {
            const int b0 = a.chunk_blk[chunk], b1 = a.chunk_blk[chunk + 1];
            for (int e = tid; e < G * Ks * DS; e += kThreads) {
                const int gg = e / (Ks * DS), k = (e / DS) % Ks, j = e % DS;
                const long long n = finalize_element(a.part, a.M, Ks, DS, a.Cw, chunk, m0 + gg, k, j, b0, b1);
                if (a.counts && it + 1 == n_iter && j == 0) a.counts[((size_t)chunk * a.M + m0 + gg) * Ks + k] = n;
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) atomicExch(a.ready + cg, it + 1);
        }
        __syncthreads();
    }
    }  // units and passes
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
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

int tc_pass_group() { return G; }

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

namespace {

// the row tiles' tensor map and the kernel arguments of pass p
int prepare_tc(const PqPass &p, CUtensorMap &map, TcArgs &a)
{
    if (!tc_pass_supported(p.D, p.M, p.Ks)) return fail(PQ_ENOTSUP, "BF16 tensor-core pass needs D/M == 8 and M even");
    if (p.N >= (1LL << 31) / TM * TM) return fail(PQ_ENOTSUP, "BF16 tensor-core pass supports N < 2^31");
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc) return fail(PQ_ECUDA, "cuTensorMapEncodeTiled unavailable");
    const cuuint64_t gdim[2] = {(cuuint64_t)p.D, (cuuint64_t)p.N};
    const cuuint64_t gstride[1] = {(cuuint64_t)p.D * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)(G * DS), (cuuint32_t)TM};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(p.X), gdim, gstride, box,
                            estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return fail(PQ_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    int dev = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    int *err = device_error_word(dev);
    if (!err) return fail(PQ_ENOMEM, "device error word");
    a = TcArgs{};
    a.N = p.N;
    a.D = p.D;
    a.M = p.M;
    a.Ks = p.Ks;
    a.tiles = (int)((p.N + TM - 1) / TM);
    a.C = p.C;
    a.codes = p.codes;
    a.part = p.part;
    a.sse = p.sse;
    a.rechecks = p.rechecks;
    a.err = err;
    a.blk_chunk = p.blk_chunk;
    a.chunk_off = p.chunk_off;
    a.chunk_blk = p.chunk_blk;
    a.iters = 1;
    return PQ_OK;
}

}  // namespace

int launch_pq_pass_tc(PqPass &p, cudaStream_t s)
{
    CUtensorMap map;
    TcArgs a;
    PQ_TRY(prepare_tc(p, map, a));
    if (p.gx <= 0) p.gx = pq_pass_tc_blocks(p);
    PQ_TRY_CUDA(cudaFuncSetAttribute(pq_pass_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    // the register hand-over inside the kernel waits for registers the launch must have given it
    static int launch_regs = -1;
    if (launch_regs < 0) {
        cudaFuncAttributes fa;
        PQ_TRY_CUDA(cudaFuncGetAttributes(&fa, pq_pass_tc_kernel<false>));
        launch_regs = fa.numRegs;
    }
    if (launch_regs * kThreads < 128 * kRegLo + 256 * kRegHi)
        return fail(PQ_ECUDA, "tensor-core pass built with %d registers per thread, fewer than its register hand-over needs",
                    launch_regs);
    dim3 grid(p.gx, p.M / G);
    ProfScope ps("pq_pass_tc", s);
    pq_pass_tc_kernel<false><<<grid, kThreads, SMEM_BYTES, s>>>(map, a);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

int launch_pq_fit_persistent_tc(PqPass &p, int iters, int *sync, long long *counts, cudaStream_t s)
{
    if (!p.part.active() || !p.chunk_blk || p.gx <= 0)
        return fail(PQ_EINTERNAL, "persistent tensor-core fit needs a chunk table and partial sums");
    if (iters <= 0) return PQ_OK;
    CUtensorMap map;
    TcArgs a;
    PQ_TRY(prepare_tc(p, map, a));
    a.iters = iters;
    a.gxu = p.gx;
    a.units = p.gx * (p.M / G);
    a.Cw = const_cast<float *>(p.C);
    const int ncg = p.n_chunks * (p.M / G);
    a.arrive = sync;
    a.ready = sync + ncg;
    a.next = sync + 2 * ncg;
    a.counts = counts;
    a.spin = seeding_spin_limit();
    PQ_TRY_CUDA(cudaFuncSetAttribute(pq_pass_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    // every CTA must be resident at once (a unit may wait for units of other CTAs): a cooperative
    // launch of at most the co-resident CTAs
    int dev = 0, sms = 0, per_sm = 0;
    PQ_TRY_CUDA(cudaGetDevice(&dev));
    PQ_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PQ_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pq_pass_tc_kernel<true>, kThreads, SMEM_BYTES));
    if (per_sm < 1) return fail(PQ_ECUDA, "persistent tensor-core fit: no CTA fits an SM");
    const int grid = std::max(1, std::min(a.units, per_sm * sms));
    void *args[] = {&map, &a};
    ProfScope ps("pq_fit_persistent_tc", s);
    PQ_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)pq_pass_tc_kernel<true>, dim3(grid), dim3(kThreads), args,
                                            SMEM_BYTES, s));
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

}  // namespace pqgb
