// kpp_factor.cu -- memoised per-block factors (Sec. 4 "block memoization"; Sec. 5.2; Alg. 1 line 7;
// Alg. 3 line 8).
//
// For each block j of the fixed partition:
//   G_j  = A_{S_j} A_{S_j}^T + lam I    (K++; Eq. 1.3)   or   A_{S_j S_j} + lam I   (CD++; Eq. 5.1)
//   L_j  = chol(G_j)                     FP64, lower
//   G_j^{-1} = L_j^{-T} L_j^{-1}         FP64 (and an FP32 copy for the mixed-precision inner solve)
// The inverse is memoised so that each iteration applies (G_j)^{-1} as one dense s x s mat-vec,
// spread over the CTAs of the solve, instead of two substitutions of depth s.
//
// Kernels here are batched over blocks: one CTA (or a tile grid) per block.  The Gram of FP32/BF16
// storage is built on the tensor cores by kpp_gram_tc.cu; this file holds the FP64 CUDA-core Gram
// used for FP64 storage (and as the reference the tensor-core path is tested against).
#include <cmath>
#include <cstdio>

#include "kpp_internal.cuh"
#include "kpp_runtime.h"

namespace kpp {

// ---------------------------------------------------------------------------------------------
// Gram of one block with FP64 accumulation: G[a][c] = sum_k A[r0+a][k] A[r0+c][k] + lam [a==c].
// Grid: (nb, tiles_a, tiles_c) with 32x32 output tiles; only tiles with tc >= ta are computed and
// mirrored (G is symmetric).  256 threads, each 2x2 outputs.
// ---------------------------------------------------------------------------------------------
template <typename TA>
__global__ void __launch_bounds__(256) gram_f64_kernel(const TA *__restrict__ A, int64_t lda, int64_t rows,
                                                       int64_t cols, int s, double lam,
                                                       double *__restrict__ G /* nb x s x s */) {
    const int j = blockIdx.x, ta = blockIdx.y, tc = blockIdx.z;
    if (tc < ta) return;
    const int64_t r0 = (int64_t)j * s;
    const int len = (int)min64(s, rows - r0);
    const int a0 = ta * 32, c0 = tc * 32;
    if (a0 >= len || c0 >= len) return;
    __shared__ double sa[32][33];
    __shared__ double sc[32][33];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2x2 outputs each
    double acc[2][2] = {{0, 0}, {0, 0}};
    for (int64_t k0 = 0; k0 < cols; k0 += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            int rr = e >> 5, kk = e & 31;
            int64_t k = k0 + kk;
            sa[rr][kk] = (a0 + rr < len && k < cols) ? widen(A[(r0 + a0 + rr) * lda + k]) : 0.0;
            sc[rr][kk] = (c0 + rr < len && k < cols) ? widen(A[(r0 + c0 + rr) * lda + k]) : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            double x0 = sa[ty * 2 + 0][kk], x1 = sa[ty * 2 + 1][kk];
            double y0 = sc[tx * 2 + 0][kk], y1 = sc[tx * 2 + 1][kk];
            acc[0][0] = fma(x0, y0, acc[0][0]);
            acc[0][1] = fma(x0, y1, acc[0][1]);
            acc[1][0] = fma(x1, y0, acc[1][0]);
            acc[1][1] = fma(x1, y1, acc[1][1]);
        }
        __syncthreads();
    }
    double *Gj = G + (size_t)j * s * s;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            int a = a0 + ty * 2 + u, c = c0 + tx * 2 + v;
            if (a < len && c < len) {
                double g = acc[u][v] + (a == c ? lam : 0.0);
                Gj[(size_t)a * len + c] = g;
                Gj[(size_t)c * len + a] = g;
            }
        }
}

// CD++: principal block A_{S S} + lam I, widened to FP64.
template <typename TA>
__global__ void principal_block_kernel(const TA *__restrict__ A, int64_t lda, int64_t n, int s, double lam,
                                       double *__restrict__ G) {
    const int j = blockIdx.x;
    const int64_t r0 = (int64_t)j * s;
    const int len = (int)min64(s, n - r0);
    double *Gj = G + (size_t)j * s * s;
    for (int e = threadIdx.x; e < len * len; e += blockDim.x) {
        int a = e / len, c = e % len;
        Gj[e] = widen(A[(r0 + a) * lda + r0 + c]) + (a == c ? lam : 0.0);
    }
}

// ---------------------------------------------------------------------------------------------
// In-place lower Cholesky of each block's G (len x len, row-major, leading dimension len), then
// Linv = L^{-1} and Ginv = Linv^T Linv.  One CTA per block.  Works in global memory (the block sits
// in L2); right-looking, one column per step.  A non-positive or non-finite pivot records the block
// in *bad (atomicMin) and leaves that block's outputs as NaN.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(512) cholesky_inverse_kernel(int64_t rows, int s, double *__restrict__ G,
                                                               double *__restrict__ L, double *__restrict__ Linv,
                                                               double *__restrict__ Ginv, float *__restrict__ Ginv32,
                                                               int *__restrict__ bad) {
    const int j = blockIdx.x;
    const int len = (int)min64(s, rows - (int64_t)j * s);
    double *Gj = G + (size_t)j * s * s;
    double *Lj = L + (size_t)j * s * s;
    double *Ij = Linv + (size_t)j * s * s;
    double *Vj = Ginv + (size_t)j * s * s;
    __shared__ int s_fail;
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    for (int c = 0; c < len; ++c) {
        if (threadIdx.x == 0) {
            double d = Gj[(size_t)c * len + c];
            if (!(d > 0.0) || !isfinite(d)) {
                s_fail = 1;
            } else {
                Gj[(size_t)c * len + c] = sqrt(d);
            }
        }
        __syncthreads();
        if (s_fail) break;
        const double ljj = Gj[(size_t)c * len + c];
        for (int i = c + 1 + threadIdx.x; i < len; i += blockDim.x) Gj[(size_t)i * len + c] /= ljj;
        __syncthreads();
        // trailing update of the lower triangle: G[i][k] -= L[i][c] L[k][c], c < k <= i
        // (one warp per row i, lanes along k)
        {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
            for (int i = c + 1 + warp; i < len; i += nw) {
                const double lic = Gj[(size_t)i * len + c];
                for (int k = c + 1 + lane; k <= i; k += 32) Gj[(size_t)i * len + k] -= lic * Gj[(size_t)k * len + c];
            }
        }
        __syncthreads();
    }
    if (s_fail) {
        if (threadIdx.x == 0) atomicMin(bad, j);
        for (int e = threadIdx.x; e < len * len; e += blockDim.x) {
            Lj[e] = NAN;
            Vj[e] = NAN;
            if (Ginv32) Ginv32[(size_t)j * s * s + e] = NAN;
        }
        return;
    }
    // L with a zero upper triangle
    for (int e = threadIdx.x; e < len * len; e += blockDim.x) {
        int a = e / len, c = e % len;
        Lj[e] = (c <= a) ? Gj[e] : 0.0;
    }
    __syncthreads();
    // Linv column by column (one thread per column): forward substitution L X = I
    for (int c = threadIdx.x; c < len; c += blockDim.x) {
        for (int i = 0; i < c; ++i) Ij[(size_t)i * len + c] = 0.0;
        Ij[(size_t)c * len + c] = 1.0 / Lj[(size_t)c * len + c];
        for (int i = c + 1; i < len; ++i) {
            double v = 0.0;
            for (int k = c; k < i; ++k) v += Lj[(size_t)i * len + k] * Ij[(size_t)k * len + c];
            Ij[(size_t)i * len + c] = -v / Lj[(size_t)i * len + i];
        }
    }
    __syncthreads();
    // Ginv[a][b] = sum_{c >= max(a,b)} Linv[c][a] Linv[c][b]
    for (int e = threadIdx.x; e < len * len; e += blockDim.x) {
        int a = e / len, b = e % len;
        if (b < a) continue;
        double v = 0.0;
        for (int c = b; c < len; ++c) v += Ij[(size_t)c * len + a] * Ij[(size_t)c * len + b];
        Vj[(size_t)a * len + b] = v;
        Vj[(size_t)b * len + a] = v;
        if (Ginv32) {
            Ginv32[(size_t)j * s * s + (size_t)a * len + b] = (float)v;
            Ginv32[(size_t)j * s * s + (size_t)b * len + a] = (float)v;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// CD++ FP64: W_j = G_j^{-1} A_{S_j} for every block (rows j s .. j s + len of W).  With A symmetric,
// u = A_{:,S} y = A_S^T G^{-1} r = W_S^T r, so the solve applies the memoised inverse and the block
// rows in one pass.  Grid (nb, ceil(cols / 64)); each CTA computes a len x 64 tile, FP64.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) cd_w_kernel(const double *__restrict__ A, int64_t lda, int64_t n, int s,
                                                   const double *__restrict__ Ginv, double *__restrict__ W) {
    const int j = blockIdx.x;
    const int64_t r0 = (int64_t)j * s;
    const int len = (int)min64(s, n - r0);
    const int64_t col0 = (int64_t)blockIdx.y * 64;
    __shared__ double sg[64][65];
    __shared__ double sa[64][65];
    const double *Gj = Ginv + (size_t)j * s * s;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 4 x 4 outputs each
    for (int a0 = 0; a0 < len; a0 += 64) {
        double acc[4][4] = {};
        for (int d0 = 0; d0 < len; d0 += 64) {
            for (int e = threadIdx.x; e < 64 * 64; e += 256) {
                const int rr = e >> 6, cc = e & 63;
                sg[rr][cc] = (a0 + rr < len && d0 + cc < len) ? Gj[(size_t)(a0 + rr) * len + d0 + cc] : 0.0;
                sa[rr][cc] = (d0 + rr < len && col0 + cc < n) ? A[(r0 + d0 + rr) * lda + col0 + cc] : 0.0;
            }
            __syncthreads();
#pragma unroll 4
            for (int d = 0; d < 64; ++d) {
                double gv[4], av[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) gv[u] = sg[ty * 4 + u][d];
#pragma unroll
                for (int v = 0; v < 4; ++v) av[v] = sa[d][tx * 4 + v];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(gv[u], av[v], acc[u][v]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int a = a0 + ty * 4 + u;
                const int64_t c = col0 + tx * 4 + v;
                if (a < len && c < n) W[(r0 + a) * n + c] = acc[u][v];
            }
    }
}

// ---------------------------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------------------------
template <typename TA>
static void launch_gram(const void *A, int64_t lda, int64_t rows, int64_t cols, int s, double lam, double *G,
                        cudaStream_t st) {
    const int64_t nb = (rows + s - 1) / s;
    const int tiles = (s + 31) / 32;
    dim3 grid((unsigned)nb, tiles, tiles);
    gram_f64_kernel<TA><<<grid, 256, 0, st>>>((const TA *)A, lda, rows, cols, s, lam, G);
}

template <typename TA>
static void launch_principal(const void *A, int64_t lda, int64_t n, int s, double lam, double *G, cudaStream_t st) {
    const int64_t nb = (n + s - 1) / s;
    principal_block_kernel<TA><<<(unsigned)nb, 256, 0, st>>>((const TA *)A, lda, n, s, lam, G);
}

int block_gram(const kpp_matrix &A, int s, double lam, double *G, int engine, cudaStream_t st) {
    if (engine != 1 && A.dtype != KPP_F64 && gram_tc(A, s, lam, G, st, engine == 2)) return 2;
    if (engine == 2) return -1;
    if (A.dtype == KPP_F64) launch_gram<double>(A.data, A.ld, A.rows, A.cols, s, lam, G, st);
    else if (A.dtype == KPP_F32) launch_gram<float>(A.data, A.ld, A.rows, A.cols, s, lam, G, st);
    else launch_gram<__nv_bfloat16>(A.data, A.ld, A.rows, A.cols, s, lam, G, st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

kpp_status factor_blocks_impl(const kpp_matrix &A, int s, double lam, int mode, FactorSet &F, cudaStream_t st) {
    const int64_t rows = A.rows;
    const int64_t nb = (rows + s - 1) / s;
    const size_t blk = (size_t)s * s;
    F.nb = nb;
    F.s = s;
    F.rows = rows;
    F.lambda = lam;
    F.mode = mode;
    F.dtype = A.dtype;
    F.bad_block = -1;
    double *G = nullptr, *Linv = nullptr;
    int *bad = nullptr;
    kpp_status rc = KPP_OK;
#define KPP_TRY(call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) {                                             \
            rc = (e_ == cudaErrorMemoryAllocation) ? KPP_ERR_OOM : KPP_ERR_CUDA; \
            set_error("%s: %s", #call, cudaGetErrorString(e_));              \
            goto done;                                                       \
        }                                                                    \
    } while (0)
    KPP_TRY(cudaMalloc(&F.L, nb * blk * sizeof(double)));
    KPP_TRY(cudaMalloc(&F.Ginv, nb * blk * sizeof(double)));
    if (A.dtype != KPP_F64) KPP_TRY(cudaMalloc(&F.Ginv32, nb * blk * sizeof(float)));
    KPP_TRY(cudaMalloc(&G, nb * blk * sizeof(double)));
    KPP_TRY(cudaMalloc(&Linv, nb * blk * sizeof(double)));
    KPP_TRY(cudaMalloc(&bad, sizeof(int)));
    {
        int big = 0x7fffffff;
        KPP_TRY(cudaMemcpyAsync(bad, &big, sizeof(int), cudaMemcpyHostToDevice, st));
    }
    if (mode == 0) {
        if (block_gram(A, s, lam, G, 0, st) < 0) {
            rc = KPP_ERR_CUDA;
            set_error("block Gram launch failed");
            goto done;
        }
    } else {
        if (A.dtype == KPP_F64) launch_principal<double>(A.data, A.ld, rows, s, lam, G, st);
        else if (A.dtype == KPP_F32) launch_principal<float>(A.data, A.ld, rows, s, lam, G, st);
        else launch_principal<__nv_bfloat16>(A.data, A.ld, rows, s, lam, G, st);
    }
    KPP_TRY(cudaGetLastError());
    cholesky_inverse_kernel<<<(unsigned)nb, 512, 0, st>>>(rows, s, G, F.L, Linv, F.Ginv, F.Ginv32, bad);
    KPP_TRY(cudaGetLastError());
    {
        int hb = 0;
        KPP_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        KPP_TRY(cudaStreamSynchronize(st));
        if (hb != 0x7fffffff) {
            F.bad_block = hb;
            rc = KPP_ERR_NOT_SPD;
            set_error("block %d: Cholesky pivot not positive", hb);
        }
    }
    if (rc == KPP_OK && mode == 1 && A.dtype == KPP_F64) {
        KPP_TRY(cudaMalloc(&F.W, (size_t)rows * rows * sizeof(double)));
        dim3 grid((unsigned)nb, (unsigned)((rows + 63) / 64));
        cd_w_kernel<<<grid, 256, 0, st>>>((const double *)A.data, A.ld, rows, s, F.Ginv, F.W);
        KPP_TRY(cudaGetLastError());
    }
done:
#undef KPP_TRY
    if (G) cudaFree(G);
    if (Linv) cudaFree(Linv);
    if (bad) cudaFree(bad);
    return rc;
}

}  // namespace kpp
