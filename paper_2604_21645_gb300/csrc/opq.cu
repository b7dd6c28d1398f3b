// opq.cu -- optimized product quantization (Sec. 2.1 names Optimized PQ; Sec. 3.1 lists
// NanoPQ's "PQ and Optimized PQ"): an orthogonal rotation R of the rows learned jointly with
// the PQ codebooks of the rotated rows X R, by alternating minimisation of the distortion
// ||X R - decode(encode(X R))||^2 -- PQ refits with R fixed, and with the codes fixed the
// Procrustes solution R = U V^T of X^T Xhat = U S V^T.
//
// On the device: the rotation X R (a tiled FP32 GEMM, every output summed in the same
// k order) and the D x D cross-product X^T Xhat (the same GEMM, split over row ranges of
// 1,024 rows whose FP32 partial products are added in float-float).  On the host: the
// one-sided Jacobi SVD (Hestenes) of that D x D matrix in FP64 and R = U V^T.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pqgb {
namespace {

constexpr int TB = 64;   // output tile (rows and columns)
constexpr int TK = 16;   // k step
constexpr int kRowsPerPart = 1024;

// C[i][j] (+)= sum_k A(i, k) B(k, j) for a 64 x 64 tile; A(i, k) = A[i*lda + k] (or A[k*lda + i]
// when `at`), B(k, j) = B[k*ldb + j].  k runs over [k0, k1) in order, 16 at a time.  256 threads,
// 4 x 4 outputs each.
template <bool AT>
__device__ __forceinline__ void gemm_tile(const float *__restrict__ A, int64_t lda, const float *__restrict__ B,
                                          int64_t ldb, int64_t i0, int64_t j0, int64_t m_rows, int64_t n_cols,
                                          int64_t k0, int64_t k1, float (&acc)[4][4])
{
    __shared__ float sa[TK][TB + 4];
    __shared__ float sb[TK][TB + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int64_t kb = k0; kb < k1; kb += TK) {
        __syncthreads();
        for (int e = threadIdx.x; e < TK * TB; e += 256) {
            // A: consecutive threads take consecutive addresses (k inside a row, or i inside a k row)
            const int kk = AT ? e / TB : e % TK, ii = AT ? e % TB : e / TK;
            const int64_t k = kb + kk, i = i0 + ii;
            sa[kk][ii] = (k < k1 && i < m_rows) ? (AT ? A[k * lda + i] : A[i * lda + k]) : 0.0f;
            const int kb2 = e / TB, jj = e % TB;
            const int64_t k2 = kb + kb2, j = j0 + jj;
            sb[kb2][jj] = (k2 < k1 && j < n_cols) ? B[k2 * ldb + j] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = sa[kk][ty * 4 + u];
#pragma unroll
            for (int v = 0; v < 4; ++v) b[v] = sb[kk][tx * 4 + v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
    }
}

// Y[N][D] = X[N][D] R[D][D]
__global__ void __launch_bounds__(256) rotate_kernel(const float *__restrict__ X, int64_t N, int D,
                                                     const float *__restrict__ R, float *__restrict__ Y)
{
    const int64_t i0 = (int64_t)blockIdx.x * TB, j0 = (int64_t)blockIdx.y * TB;
    float acc[4][4] = {};
    gemm_tile<false>(X, D, R, D, i0, j0, N, D, 0, D, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
            if (i < N && j < D) Y[i * D + j] = acc[u][v];
        }
}

// partial[p][D][D] = sum over rows n of part p of X[n][i] Y[n][j]
__global__ void __launch_bounds__(256) xty_partial_kernel(const float *__restrict__ X, const float *__restrict__ Y,
                                                          int64_t N, int D, float *__restrict__ partial)
{
    const int64_t i0 = (int64_t)blockIdx.x * TB, j0 = (int64_t)blockIdx.y * TB;
    const int64_t r0 = (int64_t)blockIdx.z * kRowsPerPart, r1 = std::min<int64_t>(N, r0 + kRowsPerPart);
    float acc[4][4] = {};
    gemm_tile<true>(X, D, Y, D, i0, j0, D, D, r0, r1, acc);
    float *P = partial + (size_t)blockIdx.z * D * D;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
            if (i < D && j < D) P[i * D + j] = acc[u][v];
        }
}

// out[e] = float-float sum over the parts, in part order (hi, lo interleaved)
__global__ void ff_reduce_kernel(const float *__restrict__ partial, int parts, int n, float *__restrict__ out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float h = 0.0f, l = 0.0f;
    for (int p = 0; p < parts; ++p) ff_add(h, l, partial[(size_t)p * n + e], 0.0f, h, l);
    out[2 * e] = h;
    out[2 * e + 1] = l;
}

// One-sided Jacobi SVD (Hestenes) of the n x n matrix A (row-major, FP64) and the polar factor
// R = U V^T: the columns of A V are made pairwise orthogonal by plane rotations accumulated in V;
// U's columns are those of A V over their norms (completed by Gram-Schmidt where a norm vanishes).
void polar_factor(std::vector<double> &A, int n, std::vector<double> &R)
{
    std::vector<double> V((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int i = 0; i < n; ++i) {
                    const double ap = A[(size_t)i * n + p], aq = A[(size_t)i * n + q];
                    alpha += ap * ap;
                    beta += aq * aq;
                    gamma += ap * aq;
                }
                if (gamma == 0.0) continue;
                off = std::max(off, std::fabs(gamma) / std::sqrt(alpha * beta));
                const double zeta = (beta - alpha) / (2.0 * gamma);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < n; ++i) {
                    double &ap = A[(size_t)i * n + p], &aq = A[(size_t)i * n + q];
                    const double x = ap, y = aq;
                    ap = c * x - s * y;
                    aq = s * x + c * y;
                    double &vp = V[(size_t)i * n + p], &vq = V[(size_t)i * n + q];
                    const double u = vp, w = vq;
                    vp = c * u - s * w;
                    vq = s * u + c * w;
                }
            }
        if (off < 1e-14) break;
    }
    // U = A V normalised by columns; columns with a vanishing norm completed by Gram-Schmidt
    std::vector<double> U = A;
    double smax = 0.0;
    std::vector<double> sig(n);
    for (int j = 0; j < n; ++j) {
        double s2 = 0.0;
        for (int i = 0; i < n; ++i) s2 += U[(size_t)i * n + j] * U[(size_t)i * n + j];
        sig[j] = std::sqrt(s2);
        smax = std::max(smax, sig[j]);
    }
    for (int j = 0; j < n; ++j) {
        if (sig[j] > 1e-13 * smax && sig[j] > 0.0) {
            for (int i = 0; i < n; ++i) U[(size_t)i * n + j] /= sig[j];
            continue;
        }
        for (int e = 0; e < n; ++e) {  // a unit vector orthogonal to the other columns
            std::vector<double> v(n, 0.0);
            v[e] = 1.0;
            for (int c = 0; c < n; ++c) {
                if (c == j || (sig[c] <= 1e-13 * smax && c > j)) continue;
                double d = 0.0;
                for (int i = 0; i < n; ++i) d += v[i] * U[(size_t)i * n + c];
                for (int i = 0; i < n; ++i) v[i] -= d * U[(size_t)i * n + c];
            }
            double nv = 0.0;
            for (int i = 0; i < n; ++i) nv += v[i] * v[i];
            if (nv > 1e-6) {
                nv = std::sqrt(nv);
                for (int i = 0; i < n; ++i) U[(size_t)i * n + j] = v[i] / nv;
                sig[j] = smax;  // now a proper column for the later completions
                break;
            }
        }
    }
    R.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += U[(size_t)i * n + k] * V[(size_t)j * n + k];
            R[(size_t)i * n + j] = s;
        }
}

}  // namespace

int launch_rotate(const float *X, int64_t N, int D, const float *R, float *Y, cudaStream_t s)
{
    if (N == 0) return PQ_OK;
    dim3 grid((unsigned)((N + TB - 1) / TB), (unsigned)((D + TB - 1) / TB));
    ProfScope ps("opq_rotate", s);
    rotate_kernel<<<grid, 256, 0, s>>>(X, N, D, R, Y);
    count_launch();
    PQ_TRY_CUDA(cudaGetLastError());
    return PQ_OK;
}

// R_out (device, float32 [D][D]) = the orthogonal R minimising ||X R - Y||_F.  Synchronizes.
int run_procrustes(const float *X, const float *Y, int64_t N, int D, float *R_out, Scratch &ws, cudaStream_t s)
{
    const int parts = (int)std::max<int64_t>(1, (N + kRowsPerPart - 1) / kRowsPerPart);
    float *partial = ws.get<float>((size_t)parts * D * D);
    float *ff = ws.get<float>((size_t)2 * D * D);
    if (ws.status) return ws.status;
    {
        dim3 grid((unsigned)((D + TB - 1) / TB), (unsigned)((D + TB - 1) / TB), (unsigned)parts);
        ProfScope ps("opq_xty", s);
        xty_partial_kernel<<<grid, 256, 0, s>>>(X, Y, N, D, partial);
        ff_reduce_kernel<<<(D * D + 255) / 256, 256, 0, s>>>(partial, parts, D * D, ff);
        count_launch(2);
        PQ_TRY_CUDA(cudaGetLastError());
    }
    std::vector<float> h((size_t)2 * D * D);
    PQ_TRY_CUDA(cudaMemcpyAsync(h.data(), ff, h.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    PQ_TRY_CUDA(cudaStreamSynchronize(s));
    std::vector<double> A((size_t)D * D), R;
    for (size_t e = 0; e < A.size(); ++e) A[e] = (double)h[2 * e] + (double)h[2 * e + 1];
    polar_factor(A, D, R);
    std::vector<float> Rf(R.size());
    for (size_t e = 0; e < R.size(); ++e) Rf[e] = (float)R[e];
    PQ_TRY_CUDA(cudaMemcpyAsync(R_out, Rf.data(), Rf.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    PQ_TRY_CUDA(cudaStreamSynchronize(s));
    return PQ_OK;
}

}  // namespace pqgb
