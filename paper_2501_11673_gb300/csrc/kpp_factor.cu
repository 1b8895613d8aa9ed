// kpp_factor.cu -- memoised per-block factors (Sec. 4 "block memoization"; Sec. 5.2; Alg. 1;
// Alg. 3).
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
// In-place lower Cholesky of each block's G (len x len, row-major, leading dimension len), FP64.
// One CTA per block, working in global memory (the block sits in L2).  Right-looking, blocked by
// panels of PB columns: the panel is factored column by column, copied (transposed) to shared
// memory, and the trailing lower triangle takes one rank-PB update per panel, so every load of
// G[i][k] carries PB FMAs.  A non-positive or non-finite pivot records the block in *bad
// (atomicMin) and leaves its outputs NaN.
// ---------------------------------------------------------------------------------------------
constexpr int CHOL_PB = 8;
constexpr int CHOL_NT = 512;

__global__ void __launch_bounds__(CHOL_NT) cholesky_kernel(int64_t rows, int s, double *__restrict__ G,
                                                          double *__restrict__ L, int *__restrict__ bad, int j0,
                                                          const int *__restrict__ only) {
    const int j = j0 + (int)blockIdx.x;  // blocks j0 .. j0 + gridDim.x - 1
    if (only && !only[j]) return;        // refactoring only the blocks flagged by the FP32 pass
    const int len = (int)min64(s, rows - (int64_t)j * s);
    double *Gj = G + (size_t)j * s * s;
    double *Lj = L + (size_t)j * s * s;
    extern __shared__ double panelT[];  // CHOL_PB x s: panelT[c][i - jb]
    __shared__ int s_fail;
    __shared__ double s_rinv;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = CHOL_NT / 32;
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    for (int jb = 0; jb < len && !s_fail; jb += CHOL_PB) {
        const int pw = min(CHOL_PB, len - jb);
        // (a) factor the panel columns
        for (int c = jb; c < jb + pw; ++c) {
            if (threadIdx.x == 0) {
                const double d = Gj[(size_t)c * len + c];
                if (!(d > 0.0) || !isfinite(d)) {
                    s_fail = 1;
                } else {
                    const double l = sqrt(d);
                    Gj[(size_t)c * len + c] = l;
                    s_rinv = 1.0 / l;  // one division per column; the column is scaled by the reciprocal
                }
            }
            __syncthreads();
            if (s_fail) break;
            const double rinv = s_rinv;
            for (int i = c + 1 + threadIdx.x; i < len; i += CHOL_NT) Gj[(size_t)i * len + c] *= rinv;
            __syncthreads();
            // update the rest of the panel: G[i][c2] -= L[i][c] L[c2][c], c < c2 < jb + pw, i >= c2
            for (int c2 = c + 1; c2 < jb + pw; ++c2) {
                const double l2 = Gj[(size_t)c2 * len + c];
                for (int i = c2 + threadIdx.x; i < len; i += CHOL_NT) Gj[(size_t)i * len + c2] -= Gj[(size_t)i * len + c] * l2;
            }
            __syncthreads();
        }
        if (s_fail) break;
        const int t0 = jb + pw;  // first trailing row/column
        if (t0 >= len) break;
        // (b) panel rows below it, transposed into shared memory
        for (int e = threadIdx.x; e < pw * (len - jb); e += CHOL_NT) {
            const int c = e / (len - jb), i = e % (len - jb);
            panelT[c * s + i] = Gj[(size_t)(jb + i) * len + jb + c];
        }
        __syncthreads();
        // (c) trailing update of the lower triangle: warp per row i, lanes along k
        for (int i = t0 + warp; i < len; i += nw) {
            double li[CHOL_PB];
#pragma unroll
            for (int c = 0; c < CHOL_PB; ++c) li[c] = c < pw ? panelT[c * s + (i - jb)] : 0.0;
            double *row = Gj + (size_t)i * len;
            for (int k = t0 + lane; k <= i; k += 32) {
                double v = row[k];
#pragma unroll
                for (int c = 0; c < CHOL_PB; ++c) v = fma(-li[c], panelT[c * s + (k - jb)], v);
                row[k] = v;
            }
        }
        __syncthreads();
    }
    if (s_fail) {
        if (threadIdx.x == 0) atomicMin(bad, j);
        for (int e = threadIdx.x; e < len * len; e += CHOL_NT) Lj[e] = NAN;
        return;
    }
    for (int e = threadIdx.x; e < len * len; e += CHOL_NT) {
        const int a = e / len, c = e % len;
        Lj[e] = (c <= a) ? Gj[e] : 0.0;
    }
}

// The same factorisation with each block split over a cluster of two CTAs on two SMs, for the last
// round of blocks, which would otherwise leave most SMs idle.  Per panel: rank 0 factors the panel
// columns (as above); a cluster barrier makes them visible; both CTAs copy the panel rows into their
// own shared memory and update half of the trailing rows each (warp w of rank r takes rows
// t0 + 16 r + w, then every 32nd); a second cluster barrier precedes the next panel.  A failed pivot is
// seen by both CTAs after the first barrier (rank 1 reads rank 0's flag through distributed shared
// memory), so both leave the panel loop at the same point, and they leave the kernel through one more
// cluster barrier, so that rank 0's shared memory outlives rank 1's last read of it.  Hardware cluster
// barriers have no time limit; both CTAs always reach the same ones.
__device__ __forceinline__ void chol_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(CHOL_NT)
    cholesky_pair_kernel(int64_t rows, int s, double *__restrict__ G, double *__restrict__ L, int *__restrict__ bad,
                         int j0) {
    unsigned rank;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    const int j = j0 + (int)(blockIdx.x >> 1);
    const int len = (int)min64(s, rows - (int64_t)j * s);
    double *Gj = G + (size_t)j * s * s;
    double *Lj = L + (size_t)j * s * s;
    extern __shared__ double panelT[];  // CHOL_PB x s: panelT[c][i - jb]
    __shared__ int s_fail;
    __shared__ double s_rinv;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = CHOL_NT / 32;
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    uint32_t fail0;  // rank 0's s_fail in the cluster's shared window
    asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(fail0) : "r"((uint32_t)__cvta_generic_to_shared(&s_fail)));
    chol_cluster_sync();  // both CTAs are running before either reads the other's shared memory
    bool failed = false;
    for (int jb = 0; jb < len; jb += CHOL_PB) {
        const int pw = min(CHOL_PB, len - jb);
        if (rank == 0) {
            for (int c = jb; c < jb + pw; ++c) {
                if (threadIdx.x == 0) {
                    const double d = Gj[(size_t)c * len + c];
                    if (!(d > 0.0) || !isfinite(d)) {
                        s_fail = 1;
                    } else {
                        const double l = sqrt(d);
                        Gj[(size_t)c * len + c] = l;
                        s_rinv = 1.0 / l;
                    }
                }
                __syncthreads();
                if (s_fail) break;
                const double rinv = s_rinv;
                for (int i = c + 1 + threadIdx.x; i < len; i += CHOL_NT) Gj[(size_t)i * len + c] *= rinv;
                __syncthreads();
                for (int c2 = c + 1; c2 < jb + pw; ++c2) {
                    const double l2 = Gj[(size_t)c2 * len + c];
                    for (int i = c2 + threadIdx.x; i < len; i += CHOL_NT)
                        Gj[(size_t)i * len + c2] -= Gj[(size_t)i * len + c] * l2;
                }
                __syncthreads();
            }
        }
        __threadfence();
        chol_cluster_sync();
        {
            int f;
            asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(f) : "r"(fail0) : "memory");
            failed = f != 0;
        }
        if (failed) break;
        const int t0 = jb + pw;
        if (t0 >= len) break;
        for (int e = threadIdx.x; e < pw * (len - jb); e += CHOL_NT) {
            const int c = e / (len - jb), i = e % (len - jb);
            panelT[c * s + i] = Gj[(size_t)(jb + i) * len + jb + c];
        }
        __syncthreads();
        for (int i = t0 + (int)rank * nw + warp; i < len; i += 2 * nw) {
            double li[CHOL_PB];
#pragma unroll
            for (int c = 0; c < CHOL_PB; ++c) li[c] = c < pw ? panelT[c * s + (i - jb)] : 0.0;
            double *row = Gj + (size_t)i * len;
            for (int k = t0 + lane; k <= i; k += 32) {
                double v = row[k];
#pragma unroll
                for (int c = 0; c < CHOL_PB; ++c) v = fma(-li[c], panelT[c * s + (k - jb)], v);
                row[k] = v;
            }
        }
        __threadfence();
        chol_cluster_sync();
    }
    // both CTAs left the loop after the same barriers, with every update of G visible to both
    if (failed) {
        if (rank == 0 && threadIdx.x == 0) atomicMin(bad, j);
        for (int e = threadIdx.x + (int)rank * CHOL_NT; e < len * len; e += 2 * CHOL_NT) Lj[e] = NAN;
    } else {
        for (int e = threadIdx.x + (int)rank * CHOL_NT; e < len * len; e += 2 * CHOL_NT) {
            const int a = e / len, c = e % len;
            Lj[e] = (c <= a) ? Gj[e] : 0.0;
        }
    }
    chol_cluster_sync();
}

static cudaError_t launch_cholesky_pairs(int64_t rows, int s, double *G, double *L, int *bad, int j0, int count,
                                         cudaStream_t st) {
    const size_t smem = CHOL_PB * s * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(cholesky_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    cholesky_pair_kernel<<<(unsigned)(2 * count), CHOL_NT, smem, st>>>(rows, s, G, L, bad, j0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// FP32 Cholesky for the mixed-precision forms (FP32/BF16 storage), where G_j itself carries only FP32
// accuracy (tensor-core Gram, FP32 accumulation) and only the FP32 inverse feeds the inner solves.
// One CTA per block on an FP32 working copy of G_j's lower triangle (global memory, ld = ws), right-
// looking with 32-column panels:
//   (a) the panel's rows are copied, transposed, into shared memory (PT[c][i - jb]);
//   (b) one warp factors the 32 x 32 diagonal tile in registers (lane a holds row a);
//   (c) every row below it solves L21 L11^T = P21 by forward substitution (a thread per row);
//   (d) the panel's columns of L go out widened to FP64, with the zeros right of the diagonal tile;
//   (e) the trailing lower triangle takes the rank-32 update in 128 x 64 tiles, each thread an 8 x 4
//       register tile fed by 16-byte shared-memory loads.
// 256 threads and two CTAs per SM: the serial parts of one block's panel ((b), (c)) and the global
// read-modify-write of its tiles overlap with the other block's tile products.
// The pivots L_cc^2 are Schur-complement diagonals, so they lie in [lambda_min(G), lambda_max(G)] and
// their ratio is a lower bound on kappa(G).  The FP32 factor's backward error is at most (s + 1) 2^-24
// |L||L^T| componentwise; for a K++ Gram (n >= s columns, FP32 accumulation) that is no more than the
// Gram's own error, so the FP32 factor loses nothing as long as elimination stays clear of breakdown.
// A block whose FP32 pivot fails, or whose smallest pivot falls to the FP32 factor's rounding floor
// (ratio above kappa_max = 2^24 / (s + 1)), is flagged in need64[j] (and counted in *n64): the caller
// refactors it in FP64 from the untouched G.
// ---------------------------------------------------------------------------------------------
constexpr int C32_NT = 256;
constexpr int C32_TM = 128;  // trailing tile rows (16 row groups of 8)
constexpr int C32_TN = 64;   // trailing tile columns (16 column groups of 4)
static __host__ __device__ __forceinline__ int c32_ws(int s) { return (s + 3) & ~3; }
// PT row length: the trailing tiles read up to 158 entries past the block's last row, and 4 mod 32
// spreads the transposed accesses over banks while keeping 16-byte alignment.
static __host__ __device__ __forceinline__ int c32_ldp(int s) { return ((s + 160 + 31) / 32) * 32 + 4; }

__global__ void __launch_bounds__(C32_NT, 2)
    cholesky_f32_kernel(int64_t rows, int s, const double *__restrict__ G, float *__restrict__ Wk,
                        double *__restrict__ L, int *__restrict__ need64, int *__restrict__ n64, float kappa_max) {
    const int j = (int)blockIdx.x;
    const int len = (int)min64(s, rows - (int64_t)j * s);
    const int ws = c32_ws(s), ldp = c32_ldp(s);
    const double *Gj = G + (size_t)j * s * s;
    float *Wj = Wk + (size_t)j * ws * ws;
    double *Lj = L + (size_t)j * s * s;
    extern __shared__ __align__(16) float PT[];  // 32 x ldp
    __shared__ float sRd[32];
    __shared__ int s_fail;
    __shared__ float s_pmin, s_pmax;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = C32_NT / 32;
    if (tid == 0) {
        s_fail = 0;
        s_pmin = INFINITY;
        s_pmax = 0.f;
    }
    for (int e = tid; e < 32 * ldp; e += C32_NT) PT[e] = 0.f;
    for (int i = warp; i < len; i += nw)
        for (int k = lane; k <= i; k += 32) Wj[(size_t)i * ws + k] = (float)Gj[(size_t)i * len + k];
    __syncthreads();
    for (int jb = 0; jb < len; jb += 32) {
        const int pw = min(32, len - jb), T = len - jb;
        // (a)
        for (int e = tid; e < T * 32; e += C32_NT) {
            const int i = e >> 5, c = e & 31;
            PT[c * ldp + i] = (c < pw && c <= i) ? Wj[(size_t)(jb + i) * ws + jb + c] : 0.f;
        }
        __syncthreads();
        // (b)
        if (warp == 0) {
            float d[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) d[c] = (lane < pw) ? (c < pw ? PT[c * ldp + lane] : 0.f) : (lane == c ? 1.f : 0.f);
            bool bad = false;
            float pmin = INFINITY, pmax = 0.f;
#pragma unroll 32
            for (int c = 0; c < 32; ++c) {
                const float piv = __shfl_sync(0xffffffffu, d[c], c);
                if (c < pw) {
                    bad |= !(piv > 0.f) || !isfinite(piv);
                    pmin = fminf(pmin, piv);
                    pmax = fmaxf(pmax, piv);
                }
                const float l = sqrtf(piv), rl = 1.f / l;
                if (lane == c) {
                    d[c] = l;
                    sRd[c] = rl;
                } else if (lane > c) {
                    d[c] *= rl;
                }
#pragma unroll 31
                for (int c2 = c + 1; c2 < 32; ++c2) {
                    const float lc2 = __shfl_sync(0xffffffffu, d[c], c2);
                    if (lane >= c2) d[c2] = fmaf(-d[c], lc2, d[c2]);
                }
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) PT[c * ldp + lane] = (c <= lane) ? d[c] : 0.f;
            if (lane == 0) {
                if (bad) s_fail = 1;
                s_pmin = fminf(s_pmin, pmin);
                s_pmax = fmaxf(s_pmax, pmax);
            }
        }
        __syncthreads();
        if (s_fail) break;
        // (c) rows below the diagonal tile (pw == 32 whenever there are any)
        for (int i = 32 + tid; i < T; i += C32_NT) {
            float p[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) p[c] = PT[c * ldp + i];
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const float x = p[c] * sRd[c];
                p[c] = x;
#pragma unroll
                for (int c2 = c + 1; c2 < 32; ++c2) p[c2] = fmaf(-PT[c * ldp + c2], x, p[c2]);
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) PT[c * ldp + i] = p[c];
        }
        __syncthreads();
        // (d)
        for (int e = tid; e < T * 32; e += C32_NT) {
            const int i = e >> 5, c = e & 31;
            if (c < pw) Lj[(size_t)(jb + i) * len + jb + c] = (double)PT[c * ldp + i];
        }
        const int right = len - jb - pw;
        for (int e = tid; e < pw * right; e += C32_NT) {
            const int r = e / right, c = e % right;
            Lj[(size_t)(jb + r) * len + jb + pw + c] = 0.0;
        }
        // (e)
        const int t0 = jb + 32, Tt = len - t0;
        const int tr = tid >> 4, tc = tid & 15;
        for (int ti = 0; ti < Tt; ti += C32_TM) {
            for (int tk = 0; tk < ti + C32_TM && tk < Tt; tk += C32_TN) {
                float acc[8][4];
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
                const float *pa = PT + 32 + ti + tr * 8;
                const float *pb = PT + 32 + tk + tc * 4;
#pragma unroll 8
                for (int c = 0; c < 32; ++c) {
                    const float4 a0 = *reinterpret_cast<const float4 *>(pa + c * ldp);
                    const float4 a1 = *reinterpret_cast<const float4 *>(pa + c * ldp + 4);
                    const float4 b = *reinterpret_cast<const float4 *>(pb + c * ldp);
                    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int u = 0; u < 8; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
                }
                const int k0 = t0 + tk + tc * 4;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = t0 + ti + tr * 8 + u;
                    if (i < len && k0 <= i) {
                        float *w = Wj + (size_t)i * ws + k0;
                        if (k0 + 3 <= i) {
                            float4 x = *reinterpret_cast<float4 *>(w);
                            x.x -= acc[u][0];
                            x.y -= acc[u][1];
                            x.z -= acc[u][2];
                            x.w -= acc[u][3];
                            *reinterpret_cast<float4 *>(w) = x;
                        } else {
#pragma unroll
                            for (int v = 0; v < 4; ++v)
                                if (k0 + v <= i) w[v] -= acc[u][v];
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        const bool ill = s_fail || !(s_pmax <= kappa_max * s_pmin);
        need64[j] = ill ? 1 : 0;
        if (ill) atomicAdd(n64, 1);
    }
}

// G^{-1} = L^{-T} L^{-1} from the FP64 factor, in the arithmetic TI: FP64 for FP64 storage; FP32 for the
// FP32 inner solves of the mixed-precision form, where only the FP32 inverse is used.  (An approximate
// inverse changes the rate of the iteration, not its fixed point: the update vanishes exactly when the
// block residual does.)  One CTA per block, 64 x 64 tiles in shared memory:
//   1. Linv block row by block row: D = (L_II)^{-1} by substitution in shared memory, then
//      Linv_IJ = -D (sum_{K=J}^{I-1} L_IK Linv_KJ) for J < I (tile products);
//   2. Ginv_AB = sum_{C >= max(A,B)} Linv_CA^T Linv_CB for A <= B, mirrored.
// Every tile product has the form acc[r][c] += X^T[k][r] Y[k][c] with both operands stored k-major, so a
// thread's 4 x 4 register tile takes two 16-byte shared loads per 16 FMAs.  Left operands that are not
// already transposed (L_IK, D) are stored transposed: each thread reads four rows of one column
// (coalesced across the warp) and writes them as one 16-byte vector.  Blocks whose factor failed (NaN)
// give NaN.
constexpr int IT = 64;          // tile
constexpr int ITP = 68;         // leading dimension in shared memory (16-byte rows)
constexpr int INV_NT = 256;

template <typename TI>
struct Vec4 {
    TI v[4];
};
template <typename TI>
__device__ __forceinline__ Vec4<TI> lds4(const TI *p) {
    Vec4<TI> r;
    if constexpr (sizeof(TI) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        r.v[0] = q.x, r.v[1] = q.y, r.v[2] = q.z, r.v[3] = q.w;
    } else {
        const double2 q0 = *reinterpret_cast<const double2 *>(p), q1 = *reinterpret_cast<const double2 *>(p + 2);
        r.v[0] = q0.x, r.v[1] = q0.y, r.v[2] = q1.x, r.v[3] = q1.y;
    }
    return r;
}
template <typename TI>
__device__ __forceinline__ void sts4(TI *p, const Vec4<TI> &r) {
    if constexpr (sizeof(TI) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else {
        *reinterpret_cast<double2 *>(p) = make_double2(r.v[0], r.v[1]);
        *reinterpret_cast<double2 *>(p + 2) = make_double2(r.v[2], r.v[3]);
    }
}
// dst[c][r] = src[r0 + r][c0 + c] (transposed), zero outside len x len
template <typename TI, typename TS>
__device__ __forceinline__ void tile_load_T(TI *dst, const TS *src, int ld, int r0, int c0, int len) {
    for (int e = threadIdx.x; e < IT * (IT / 4); e += INV_NT) {
        const int c = e % IT, r4 = (e / IT) * 4, gc = c0 + c;
        Vec4<TI> q;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int gr = r0 + r4 + u;
            q.v[u] = (gr < len && gc < len) ? (TI)src[(size_t)gr * ld + gc] : (TI)0;
        }
        sts4(dst + c * ITP + r4, q);
    }
}
// dst[r][c] = src[r0 + r][c0 + c], zero outside len x len
template <typename TI>
__device__ __forceinline__ void tile_load(TI *dst, const TI *src, int ld, int r0, int c0, int len) {
    for (int e = threadIdx.x; e < IT * IT; e += INV_NT) {
        const int r = e / IT, c = e % IT;
        const int gr = r0 + r, gc = c0 + c;
        dst[r * ITP + c] = (gr < len && gc < len) ? src[(size_t)gr * ld + gc] : (TI)0;
    }
}
// acc[u][v] += sum_k XT[k][ty*4 + u] Y[k][tx*4 + v]
template <typename TI>
__device__ __forceinline__ void tile_mma(TI (&acc)[4][4], const TI *XT, const TI *Y) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll 8
    for (int k = 0; k < IT; ++k) {
        const Vec4<TI> a = lds4(XT + k * ITP + ty * 4);
        const Vec4<TI> b = lds4(Y + k * ITP + tx * 4);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a.v[u], b.v[v], acc[u][v]);
    }
}

template <typename TI>
__global__ void __launch_bounds__(INV_NT, 2) inverse_kernel(int64_t rows, int s, const double *__restrict__ L,
                                                            TI *__restrict__ Linv, TI *__restrict__ Ginv, int j0) {
    const int j = j0 + (int)blockIdx.x;  // blocks j0 .. j0 + gridDim.x - 1
    const int len = (int)min64(s, rows - (int64_t)j * s);
    const double *Lj = L + (size_t)j * s * s;
    TI *Xj = Linv + (size_t)j * s * s;
    TI *Vj = Ginv + (size_t)j * s * s;
    extern __shared__ __align__(16) unsigned char inv_smem[];
    TI *sA = (TI *)inv_smem;  // IT x ITP each: left operand (k-major)
    TI *sB = sA + IT * ITP;   // right operand (k-major)
    TI *sD = sB + IT * ITP;   // D^T: sD[k][r] = D[r][k]
    TI *sT = sD + IT * ITP;   // sum_K L_IK Linv_KJ, row-major (the right operand of D T)
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    if (isnan(Lj[0])) {
        for (int e = threadIdx.x; e < len * len; e += INV_NT) Vj[e] = (TI)NAN;
        return;
    }
    const int nt = (len + IT - 1) / IT;
    for (int I = 0; I < nt; ++I) {
        // D = inverse of the diagonal tile (lower triangular), by columns; thread c owns column c of D,
        // stored as row c of sD
        tile_load_T<TI, double>(sA, Lj, len, I * IT, I * IT, len);  // sA[k][i] = L_II[i][k]
        for (int e = threadIdx.x; e < IT * ITP; e += INV_NT) sD[e] = (TI)0;
        __syncthreads();
        const int tl = min(IT, len - I * IT);
        if (threadIdx.x < tl) {
            const int c = threadIdx.x;
            TI *dc = sD + c * ITP;
            dc[c] = (TI)1 / sA[c * ITP + c];
            for (int i = c + 1; i < tl; ++i) {
                TI v = (TI)0;
                for (int k = c; k < i; ++k) v = fma(sA[k * ITP + i], dc[k], v);
                dc[i] = -v / sA[i * ITP + i];
            }
        }
        __syncthreads();
        // Linv_II = D
        for (int e = threadIdx.x; e < IT * IT; e += INV_NT) {
            const int r = e / IT, c = e % IT;
            if (r < tl && c < tl) Xj[(size_t)(I * IT + r) * len + I * IT + c] = sD[c * ITP + r];
        }
        // Linv_IJ = -D sum_K L_IK Linv_KJ
        for (int J = 0; J < I; ++J) {
            TI acc[4][4] = {};
            for (int Kt = J; Kt < I; ++Kt) {
                __syncthreads();
                tile_load_T<TI, double>(sA, Lj, len, I * IT, Kt * IT, len);
                tile_load<TI>(sB, Xj, len, Kt * IT, J * IT, len);
                __syncthreads();
                tile_mma<TI>(acc, sA, sB);
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                Vec4<TI> q;
#pragma unroll
                for (int v = 0; v < 4; ++v) q.v[v] = acc[u][v];
                sts4(sT + (ty * 4 + u) * ITP + tx * 4, q);
            }
            __syncthreads();
            TI out[4][4] = {};
            tile_mma<TI>(out, sD, sT);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int r = I * IT + ty * 4 + u, c = J * IT + tx * 4 + v;
                    if (r < len && c < len) Xj[(size_t)r * len + c] = -out[u][v];
                }
        }
        // upper part of block row I is zero
        for (int e = threadIdx.x; e < tl * len; e += INV_NT) {
            const int r = I * IT + e / len, c = e % len;
            if (c >= (I + 1) * IT) Xj[(size_t)r * len + c] = (TI)0;
        }
        __syncthreads();
    }
    __threadfence_block();
    __syncthreads();
    // Ginv_AB = sum_{C >= B} Linv_CA^T Linv_CB  (A <= B), mirrored
    for (int A = 0; A < nt; ++A) {
        for (int B = A; B < nt; ++B) {
            TI acc[4][4] = {};
            for (int C = B; C < nt; ++C) {
                __syncthreads();
                tile_load<TI>(sA, Xj, len, C * IT, A * IT, len);
                tile_load<TI>(sB, Xj, len, C * IT, B * IT, len);
                __syncthreads();
                tile_mma<TI>(acc, sA, sB);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int r = A * IT + ty * 4 + u, c = B * IT + tx * 4 + v;
                    if (r < len && c < len) {
                        Vj[(size_t)r * len + c] = acc[u][v];
                        Vj[(size_t)c * len + r] = acc[u][v];
                    }
                }
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
    note_launch();
    gram_f64_kernel<TA><<<grid, 256, 0, st>>>((const TA *)A, lda, rows, cols, s, lam, G);
}

template <typename TA>
static void launch_principal(const void *A, int64_t lda, int64_t n, int s, double lam, double *G, cudaStream_t st) {
    const int64_t nb = (n + s - 1) / s;
    note_launch();
    principal_block_kernel<TA><<<(unsigned)nb, 256, 0, st>>>((const TA *)A, lda, n, s, lam, G);
}

int block_gram(const kpp_matrix &A, int s, double lam, double *G, int engine, cudaStream_t st) {
    // engine 2: one tensor-core product per tile (bf16, or plain tf32 for FP32 storage);
    // engine 3 / automatic for FP32: FP32 split into two tf32 halves, three products
    if (engine != 1 && A.dtype != KPP_F64 && gram_tc(A, s, lam, G, st, engine == 2)) return engine == 2 ? 2 : (A.dtype == KPP_F32 ? 3 : 2);
    if (engine == 2 || engine == 3) return -1;
    if (A.dtype == KPP_F64) launch_gram<double>(A.data, A.ld, A.rows, A.cols, s, lam, G, st);
    else if (A.dtype == KPP_F32) launch_gram<float>(A.data, A.ld, A.rows, A.cols, s, lam, G, st);
    else launch_gram<__nv_bfloat16>(A.data, A.ld, A.rows, A.cols, s, lam, G, st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

// FP64 Cholesky factors and inverses of nblk Grams given in G (block i: s x s, row-major, packed), for
// blocks formed elsewhere (the online memo's new subsets, the LSQR sketch preconditioners).  G is
// factored in place; Ginv receives G_i^{-1} (nblk x s x s); L_out and Linv_out, when given, keep the
// lower factors L_i and their inverses L_i^{-1} (lower, zero above the diagonal).  A block with a non-positive pivot sets *bad_block to its index (the smallest
// such) and the call returns KPP_ERR_NOT_SPD.
kpp_status factor_grams(double *G, int64_t nblk, int s, double *Ginv, int64_t *bad_block, cudaStream_t st,
                        double *L_out, double *Linv_out) {
    *bad_block = -1;
    if (nblk <= 0) return KPP_OK;
    const int64_t rows = nblk * s;
    const size_t blk = (size_t)s * s;
    double *L = nullptr, *Linv = nullptr;
    int *bad = nullptr;
    kpp_status rc = KPP_OK;
    const int big = 0x7fffffff;
    int hb = big;
    const size_t chol_smem = CHOL_PB * s * sizeof(double);
    const int sm64 = 4 * IT * ITP * (int)sizeof(double);
    L = L_out;
    Linv = Linv_out;
    if ((!L && dev_malloc_async((void **)&L, nblk * blk * sizeof(double), st) != cudaSuccess) ||
        (!Linv && dev_malloc_async((void **)&Linv, nblk * blk * sizeof(double), st) != cudaSuccess) ||
        dev_malloc_async((void **)&bad, sizeof(int), st) != cudaSuccess) {
        rc = KPP_ERR_OOM;
        set_error("factor_grams: out of device memory for %lld blocks", (long long)nblk);
    }
    if (rc == KPP_OK &&
        (cudaMemcpyAsync(bad, &big, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chol_smem) !=
             cudaSuccess ||
         cudaFuncSetAttribute(inverse_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm64) != cudaSuccess))
        rc = KPP_ERR_CUDA;
    if (rc == KPP_OK) {
        note_launch();
        cholesky_kernel<<<(unsigned)nblk, CHOL_NT, chol_smem, st>>>(rows, s, G, L, bad, 0, nullptr);
        note_launch();
        inverse_kernel<double><<<(unsigned)nblk, INV_NT, sm64, st>>>(rows, s, L, Linv, Ginv, 0);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = KPP_ERR_CUDA;
            set_error("factor_grams: launch failed");
        } else if (hb != big) {
            *bad_block = hb;
            rc = KPP_ERR_NOT_SPD;
        }
    }
    if (L && L != L_out) cudaFreeAsync(L, st);
    if (Linv && Linv != Linv_out) cudaFreeAsync(Linv, st);
    if (bad) cudaFreeAsync(bad, st);
    return rc;
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
    float *Wk = nullptr;
    int *bad = nullptr, *need64 = nullptr;
    kpp_status rc = KPP_OK;
    F.fp64_blocks = A.dtype == KPP_F64 ? nb : 0;
#define KPP_TRY(call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) {                                             \
            rc = (e_ == cudaErrorMemoryAllocation) ? KPP_ERR_OOM : KPP_ERR_CUDA; \
            set_error("%s: %s", #call, cudaGetErrorString(e_));              \
            goto done;                                                       \
        }                                                                    \
    } while (0)
    KPP_TRY(dev_malloc((void **)&F.L, nb * blk * sizeof(double)));
    // 64 bytes of slack: the iteration kernels copy G^{-1} rows in 16-byte multiples, which can run up
    // to 8 bytes past the last block when its rows have an odd length
    if (A.dtype == KPP_F64) KPP_TRY(dev_malloc((void **)&F.Ginv, nb * blk * sizeof(double) + 64));
    else KPP_TRY(dev_malloc((void **)&F.Ginv32, nb * blk * sizeof(float) + 64));
    KPP_TRY(dev_malloc((void **)&G, nb * blk * sizeof(double)));
    KPP_TRY(dev_malloc((void **)&Linv, nb * blk * sizeof(double)));
    KPP_TRY(dev_malloc((void **)&bad, sizeof(int)));
    {
        int big = 0x7fffffff;
        KPP_TRY(cudaMemcpyAsync(bad, &big, sizeof(int), cudaMemcpyHostToDevice, st));
    }
    for (cudaEvent_t &e : F.ev) KPP_TRY(cudaEventCreate(&e));
    KPP_TRY(cudaEventRecord(F.ev[0], st));
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
    KPP_TRY(cudaEventRecord(F.ev[1], st));
    if (A.dtype != KPP_F64) {
        // FP32/BF16 storage: the Cholesky runs in FP32, and only the blocks it flags as ill-conditioned
        // (or failed) are refactored in FP64 from the untouched G.
        const int ws = c32_ws(s);
        const size_t c32_smem = (size_t)32 * c32_ldp(s) * sizeof(float);
        const size_t chol_smem = CHOL_PB * s * sizeof(double);
        const float kappa_max = (float)(16777216.0 / (s + 1));  // smallest pivot above (s + 1) 2^-24 x largest
        KPP_TRY(dev_malloc((void **)&Wk, (size_t)nb * ws * ws * sizeof(float)));
        KPP_TRY(dev_malloc((void **)&need64, (size_t)(nb + 1) * sizeof(int)));
        KPP_TRY(cudaMemsetAsync(need64 + nb, 0, sizeof(int), st));
        KPP_TRY(cudaFuncSetAttribute(cholesky_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c32_smem));
        note_launch();
        cholesky_f32_kernel<<<(unsigned)nb, C32_NT, c32_smem, st>>>(rows, s, G, Wk, F.L, need64, need64 + nb, kappa_max);
        KPP_TRY(cudaGetLastError());
        KPP_TRY(cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chol_smem));
        note_launch();
        cholesky_kernel<<<(unsigned)nb, CHOL_NT, chol_smem, st>>>(rows, s, G, F.L, bad, 0, need64);
        KPP_TRY(cudaGetLastError());
    } else {
        // The Cholesky is one CTA per block on the FP64 pipe.  nb blocks over the SMs end in a last
        // round of nb mod SMs blocks, during which the other SMs would idle; when there are few enough,
        // that round runs as its own launch with each block split over a pair of CTAs (a cluster) on
        // two SMs.  (The inverses are left to follow: FP32 work beside the Cholesky slows its FP64 pipe
        // about as much as it would save.)
        const int nsm = sm_count();
        const int64_t tail = nb > nsm ? nb % nsm : 0;
        const bool pair = tail > 0 && 2 * tail <= nsm;
        const int64_t head = pair ? nb - tail : nb;
        const size_t chol_smem = CHOL_PB * s * sizeof(double);
        KPP_TRY(cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chol_smem));
        note_launch();
        cholesky_kernel<<<(unsigned)head, CHOL_NT, chol_smem, st>>>(rows, s, G, F.L, bad, 0, nullptr);
        KPP_TRY(cudaGetLastError());
        if (pair) KPP_TRY(launch_cholesky_pairs(rows, s, G, F.L, bad, (int)head, (int)tail, st));
    }
    KPP_TRY(cudaEventRecord(F.ev[2], st));
    if (A.dtype == KPP_F64) {
        const int sm64 = 4 * IT * ITP * (int)sizeof(double);
        KPP_TRY(cudaFuncSetAttribute(inverse_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm64));
        note_launch();
        inverse_kernel<double><<<(unsigned)nb, INV_NT, sm64, st>>>(rows, s, F.L, Linv, F.Ginv, 0);
    } else {
        const int sm32 = 4 * IT * ITP * (int)sizeof(float);
        KPP_TRY(cudaFuncSetAttribute(inverse_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm32));
        note_launch();
        inverse_kernel<float><<<(unsigned)nb, INV_NT, sm32, st>>>(rows, s, F.L, (float *)Linv, F.Ginv32, 0);
    }
    KPP_TRY(cudaGetLastError());
    KPP_TRY(cudaEventRecord(F.ev[3], st));
    {
        int hb = 0, h64 = 0;
        KPP_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (need64) KPP_TRY(cudaMemcpyAsync(&h64, need64 + nb, sizeof(int), cudaMemcpyDeviceToHost, st));
        KPP_TRY(cudaStreamSynchronize(st));
        if (need64) F.fp64_blocks = h64;
        if (hb != 0x7fffffff) {
            F.bad_block = hb;
            rc = KPP_ERR_NOT_SPD;
            set_error("block %d: Cholesky pivot not positive", hb);
        }
    }
    if (rc == KPP_OK && mode == 0 && A.dtype != KPP_F64 && kw_fits(A.dtype, rows, A.cols, s, 1, sm_count())) {
        // the large-block K++ kernel reads W_S = G^{-1} A_S instead of applying G^{-1} across the group
        KPP_TRY(dev_malloc((void **)&F.W32, (size_t)rows * A.cols * sizeof(float)));
        F.memo_cols = A.cols;
        rc = build_w32(A, s, F.Ginv32, F.W32, st);
        if (rc != KPP_OK) goto done;
    }
    if (rc == KPP_OK && mode == 1 && A.dtype != KPP_F64 && rows % s == 0 && s <= 64) {
        // CD++ inner FP32 iterations on one right-hand side read W_S = G^{-1} A_S (FP32), as FP64 reads W
        KPP_TRY(dev_malloc((void **)&F.W32, (size_t)rows * A.cols * sizeof(float)));
        F.memo_cols = A.cols;
        rc = build_w32(A, s, F.Ginv32, F.W32, st);
        if (rc != KPP_OK) goto done;
    }
    if (rc == KPP_OK && mode == 1 && A.dtype == KPP_F64) {
        KPP_TRY(dev_malloc((void **)&F.W, (size_t)rows * rows * sizeof(double)));
        dim3 grid((unsigned)nb, (unsigned)((rows + 63) / 64));
        note_launch();
        cd_w_kernel<<<grid, 256, 0, st>>>((const double *)A.data, A.ld, rows, s, F.Ginv, F.W);
        KPP_TRY(cudaGetLastError());
    }
    KPP_TRY(cudaEventRecord(F.ev[4], st));
done:
#undef KPP_TRY
    dev_free(G);
    dev_free(Linv);
    dev_free(Wk);
    dev_free(need64);
    dev_free(bad);
    return rc;
}

}  // namespace kpp
