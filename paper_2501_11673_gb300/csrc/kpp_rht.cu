// kpp_rht.cu -- randomized Hadamard preprocessing of a symmetric system for CD++ (Sec. 5.1: the
// preprocessing lines of Alg. 3 and its return D FHT(x); the FHT / SymFHT appendix).
//
//   Abar = Q A Q^T,  bbar = Q b,  x = Q^T xbar,   Q = H_n D,  D = diag(d) / sqrt(n),  d_i = +-1,
//
// with H_n the Sylvester-Hadamard matrix (H_2n = [[H_n, H_n], [H_n, -H_n]]; entry (i, j) is
// (-1)^popcount(i AND j)), so Q is orthogonal and CD++ on (Abar, bbar) solves the original system.
//
// The matrix takes two streaming passes:
//   1. rows:    R = (D A D) H   -- every row scaled by d_i d_j / n and transformed in shared memory;
//   2. columns: Abar = H R      -- CTAs gather four columns of R (32 contiguous bytes per row: whole
//      sectors), transform them in shared memory and write them out as four rows of Abar (Abar is
//      symmetric: its row c is H applied to column c of R).
// Each pass reads and writes the n x n matrix once, and adds log2 n FP64 butterflies per element.  On
// this GPU the FP64 additions, not HBM, bound the passes: 2 n^2 log2 n in all, at about 1.7 FP64 lanes
// per clock per SM.  The paper's SymFHT needs n^2 log2 n + 1.5 n^2 (it transforms one off-diagonal block
// for both at each level of its recursion); it is not used here, since the transform is a few percent
// of a CD++ solve.  Within a CTA the length-n transform runs as radix-16
// passes over 4 bits of the index each (the Sylvester factors commute), in registers, over a shared
// vector padded by one double per 16 so that strided and unit-stride groups are both conflict-free.
// Vectors and panels (b, x) use the column pass without the transpose.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/kpp.h"
#include "kpp_launch.h"
#include "kpp_runtime.h"

namespace kpp {

constexpr int RHT_NT = 256;
constexpr int RHT_MAXL = 14;  // n <= 16384: one padded FP64 vector is 136 KiB of shared memory

__device__ __forceinline__ int pidx(int e) { return e + (e >> 4); }
__host__ __device__ inline int padded(int n) { return n + (n >> 4); }

// H_R on v[0..R) (R = 2^RB, Sylvester order: bit b of the index pairs elements 2^b apart)
template <int RB>
__device__ __forceinline__ void hadamard_regs(double (&v)[1 << RB]) {
#pragma unroll
    for (int h = 1; h < (1 << RB); h <<= 1)
#pragma unroll
        for (int m = 0; m < (1 << RB); ++m)
            if (!(m & h)) {
                const double a = v[m], b = v[m | h];
                v[m] = a + b;
                v[m | h] = a - b;
            }
}

// One pass over index bits [p, p + RB) of the padded shared vector s: groups of R elements 2^p apart.
template <int RB>
__device__ void smem_pass(double *s, int n, int p) {
    constexpr int R = 1 << RB;
    const int ng = n >> RB;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const int base = (g & ((1 << p) - 1)) | ((g >> p) << (p + RB));
        double v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = s[pidx(base + (m << p))];
        hadamard_regs<RB>(v);
#pragma unroll
        for (int m = 0; m < R; ++m) s[pidx(base + (m << p))] = v[m];
    }
}

// s <- H_n s (n = 2^L) for a padded shared vector; starts and ends with a block barrier.
__device__ void fwht_smem(double *s, int n, int L) {
    int p = L;
    while (p >= 4) {
        p -= 4;
        __syncthreads();
        smem_pass<4>(s, n, p);
    }
    __syncthreads();
    switch (p) {  // the low bits left over
        case 3: smem_pass<3>(s, n, 0); break;
        case 2: smem_pass<2>(s, n, 0); break;
        case 1: smem_pass<1>(s, n, 0); break;
        default: break;
    }
    __syncthreads();
}

// R[i, :] = H applied to row i of D A D (scaled by d_i d_j / n: exact, d = +-1 and n a power of 2).
__global__ void __launch_bounds__(RHT_NT) rht_rows_kernel(int n, int L, const double *__restrict__ d,
                                                          const double *__restrict__ A, int64_t lda,
                                                          double *__restrict__ R) {
    extern __shared__ double sv[];
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const double di = d[i] / (double)n;
        __syncthreads();  // the previous row's output is read out
        for (int e = threadIdx.x; e < n; e += RHT_NT) sv[pidx(e)] = A[i * lda + e] * (di * d[e]);
        fwht_smem(sv, n, L);
        for (int e = threadIdx.x; e < n; e += RHT_NT) R[i * (int64_t)n + e] = sv[pidx(e)];
    }
}

// Columns c of an n x ncols row-major panel `in`, cpb at a time per CTA: H (diag(d_in) scale) in[:, c],
// then scaled by diag(d_out) scale; written as row c of `out` (transpose_out) or back as column c.
// Null d_in / d_out: no scaling on that side.  in == out is allowed: a CTA reads all of its columns
// before it writes any, and no two CTAs share a column.
__global__ void __launch_bounds__(RHT_NT) rht_cols_kernel(int n, int L, int ncols, int cpb,
                                                          const double *in, int64_t ldi, double *out, int64_t ldo,
                                                          int transpose_out, const double *__restrict__ d_in,
                                                          const double *__restrict__ d_out, double scale) {
    extern __shared__ double sv[];
    const int pn = padded(n);
    for (int c0 = blockIdx.x * cpb; c0 < ncols; c0 += gridDim.x * cpb) {
        const int nc = min(cpb, ncols - c0);
        __syncthreads();  // the previous columns are written out
        for (int e = threadIdx.x; e < n; e += RHT_NT) {
            const double sc = d_in ? d_in[e] * scale : 1.0;
            const double *src = in + (int64_t)e * ldi + c0;
            for (int c = 0; c < nc; ++c) sv[c * pn + pidx(e)] = src[c] * sc;
        }
        for (int c = 0; c < nc; ++c) fwht_smem(sv + c * pn, n, L);
        for (int c = 0; c < nc; ++c)
            for (int e = threadIdx.x; e < n; e += RHT_NT) {
                const double v = sv[c * pn + pidx(e)] * (d_out ? d_out[e] * scale : 1.0);
                if (transpose_out) out[(int64_t)(c0 + c) * ldo + e] = v;
                else out[(int64_t)e * ldo + c0 + c] = v;
            }
    }
}

static int exact_log2(int64_t n) {
    if (n < 1 || (n & (n - 1))) return -1;
    int L = 0;
    while ((int64_t(1) << L) < n) ++L;
    return L;
}

static cudaError_t launch_cols(int n, int L, int ncols, const double *in, int64_t ldi, double *out, int64_t ldo,
                               int transpose_out, const double *d_in, const double *d_out, double scale,
                               cudaStream_t st) {
    const size_t vec = (size_t)padded(n) * sizeof(double);
    const int cpb = (int)std::max<size_t>(1, std::min<size_t>(4, (200u << 10) / vec));
    const size_t smem = (size_t)cpb * vec;
    cudaError_t e = cudaFuncSetAttribute(rht_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int groups = (ncols + cpb - 1) / cpb;
    const int grid = std::min(groups, 4 * sm_count());
    note_launch();
    rht_cols_kernel<<<grid, RHT_NT, smem, st>>>(n, L, ncols, cpb, in, ldi, out, ldo, transpose_out, d_in, d_out,
                                                scale);
    return cudaGetLastError();
}

}  // namespace kpp

using namespace kpp;

extern "C" {

kpp_status kpp_rht_forward(int64_t n, const double *d, const kpp_matrix *A, double *Abar, const double *b,
                           double *bbar, int32_t k, void *stream) {
    clear_error();
    const int L = exact_log2(n);
    if (L < 0 || L > RHT_MAXL) {
        set_error("kpp_rht_forward: n = %lld must be a power of 2 no larger than %d", (long long)n, 1 << RHT_MAXL);
        return KPP_ERR_ARG;
    }
    if (!d || !Abar || !matrix_ok(A) || A->dtype != KPP_F64 || A->rows != n || A->cols != n || k < 0 ||
        (k > 0 && (!b || !bbar))) {
        set_error("kpp_rht_forward: invalid argument (A must be FP64 n x n; d, Abar, and b, bbar for k > 0)");
        return KPP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    kpp_status rc = KPP_OK;
    double *R = nullptr;
    const size_t vec = (size_t)padded((int)n) * sizeof(double);
    Scratch scr(st);
    CUDA_OR(scr.alloc((void **)&R, (size_t)n * n * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(cudaFuncSetAttribute(rht_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec),
            KPP_ERR_CUDA);
    note_launch();
    rht_rows_kernel<<<(unsigned)std::min<int64_t>(n, 8 * sm_count()), RHT_NT, vec, st>>>((int)n, L, d,
                                                                                        (const double *)A->data,
                                                                                        A->ld, R);
    CUDA_OR(cudaGetLastError(), KPP_ERR_CUDA);
    CUDA_OR(launch_cols((int)n, L, (int)n, R, n, Abar, n, 1, nullptr, nullptr, 1.0, st), KPP_ERR_CUDA);
    if (k > 0)
        CUDA_OR(launch_cols((int)n, L, k, b, k, bbar, k, 0, d, nullptr, 1.0 / std::sqrt((double)n), st),
                KPP_ERR_CUDA);
cleanup:
    return rc;
}

kpp_status kpp_rht_inverse(int64_t n, const double *d, const double *xbar, double *x, int32_t k, void *stream) {
    clear_error();
    const int L = exact_log2(n);
    if (L < 0 || L > RHT_MAXL || !d || k < 1 || !xbar || !x) {
        set_error("kpp_rht_inverse: invalid argument (n a power of 2 <= %d, k >= 1, non-null pointers)",
                  1 << RHT_MAXL);
        return KPP_ERR_ARG;
    }
    kpp_status rc = KPP_OK;
    CUDA_OR(launch_cols((int)n, L, k, xbar, k, x, k, 0, nullptr, d, 1.0 / std::sqrt((double)n), (cudaStream_t)stream),
            KPP_ERR_CUDA);
cleanup:
    return rc;
}

}  // extern "C"
