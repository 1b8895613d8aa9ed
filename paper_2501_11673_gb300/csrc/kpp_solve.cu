// kpp_solve.cu -- the general persistent solve kernel of Kaczmarz++ and CD++ (Alg. 1, Alg. 3, Alg. 5;
// Eq. 1.3 - 1.4, Eq. 5.1 - 5.3), the standalone FP64 residual and the small elementwise kernels of the
// refinement loop.  One launch runs every iteration of one or more systems, G CTAs per system; the body
// of a system's solve is solve_group (kpp_solve_group.cuh), which the serving loop's slots run as well.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "kpp_internal.cuh"
#include "kpp_runtime.h"
#include "kpp_solve.h"
#include "kpp_solve_device.cuh"
#include "kpp_solve_group.cuh"

namespace kpp {

template <typename TA, typename TC, int KP, bool CD>
__global__ void __launch_bounds__(NT, 1) solve_kernel(const SysArgs *__restrict__ systems, Common cm) {
    const SysArgs sa = systems[blockIdx.x / cm.G];
    GroupSync gs{sa.bar, sa.err, 0u, (unsigned)cm.G, cm.timeout_ns};
    solve_group<TA, TC, KP, CD>(sa, cm, (int)(blockIdx.x % cm.G), gs);
}

// ---------------------------------------------------------------------------------------------
// Standalone FP64 residual r = b - A x (rows x k) with per-CTA partial sums of |r|^2 (fixed grid and
// fixed order: deterministic).  Optionally stores r rounded to FP32 (the inner right-hand side of a
// refinement step).  Warp per row; each lane reads 16-byte vectors of the row (8 bf16 / 4 fp32 /
// 2 fp64 entries), several in flight; x comes from shared memory when it fits (k = 1, cols <= 24576),
// and when that x is exactly zero the row products are skipped (r = b; A is not read).
// Stored entries are widened exactly and every product and sum is FP64.
// ---------------------------------------------------------------------------------------------
template <typename TA> struct Vec16;
template <> struct Vec16<double> { static constexpr int n = 2; };
template <> struct Vec16<float> { static constexpr int n = 4; };
template <> struct Vec16<__nv_bfloat16> { static constexpr int n = 8; };

constexpr int RES_SMEM_COLS = 24576;

template <typename TA>
__global__ void __launch_bounds__(256) residual_kernel(const TA *__restrict__ A, int64_t lda, int64_t rows,
                                                       int64_t cols, int k, const double *__restrict__ b,
                                                       const double *__restrict__ x, float *__restrict__ r32,
                                                       double *__restrict__ part /* gridDim.x x k */,
                                                       const int *__restrict__ skip) {
    if (skip && *skip) return;  // the system is already done (batched plans)
    constexpr int V = Vec16<TA>::n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    extern __shared__ double xs[];
    __shared__ double s_acc[8][32];
    const bool vec_ok = ((lda * (int64_t)sizeof(TA)) % 16 == 0) && (((uintptr_t)A & 15) == 0);
    const bool x_in_smem = (k == 1) && x && cols <= RES_SMEM_COLS;
    if (x_in_smem) {
        int nz = 0;
        for (int64_t i = threadIdx.x; i < cols; i += blockDim.x) {
            const double v = x[i];
            xs[i] = v;
            nz |= v != 0.0;
        }
        // x = 0 (the first refinement step from x0 = 0): r = b, and A is not read
        if (!__syncthreads_or(nz)) x = nullptr;
    }
    double acc2[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc2[c] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < rows; i += (int64_t)gridDim.x * 8) {
        const TA *row = A + i * lda;
        if (k == 1) {
            double v = 0.0;
            if (x) {
                if (vec_ok) {
                    const int64_t nvec = cols / V;
                    const uint4 *rv = (const uint4 *)row;
                    int64_t q = lane;
#pragma unroll 1
                    for (; q + 96 < nvec; q += 128) {
                        uint4 w[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) w[u] = __ldg(rv + q + 32 * u);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const TA *e = (const TA *)&w[u];
                            const int64_t c0 = (q + 32 * u) * V;
#pragma unroll
                            for (int z = 0; z < V; ++z) v = fma(widen_fast(e[z]), x_in_smem ? xs[c0 + z] : x[c0 + z], v);
                        }
                    }
                    for (; q < nvec; q += 32) {
                        const uint4 w = __ldg(rv + q);
                        const TA *e = (const TA *)&w;
#pragma unroll
                        for (int z = 0; z < V; ++z) v = fma(widen_fast(e[z]), x_in_smem ? xs[q * V + z] : x[q * V + z], v);
                    }
                    for (int64_t col = nvec * V + lane; col < cols; col += 32) v = fma(widen(row[col]), x[col], v);
                } else {
                    for (int64_t col = lane; col < cols; col += 32) v = fma(widen(row[col]), x[col], v);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            const double r = b[i] - v;
            if (lane == 0 && r32) r32[i] = (float)r;
            acc2[0] += r * r;
            continue;
        }
        for (int c0 = 0; c0 < k; c0 += 8) {
            double v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = 0.0;
            if (x) {
                for (int64_t col = lane; col < cols; col += 32) {
                    const double a = widen(row[col]);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c0 + c < k) v[c] = fma(a, x[col * k + c0 + c], v[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
                if (c0 + c < k) {
                    const double r = b[i * k + c0 + c] - v[c];
                    if (lane == 0 && r32) r32[i * k + c0 + c] = (float)r;
#pragma unroll
                    for (int cc = 0; cc < 32; ++cc)
                        if (cc == c0 + c) acc2[cc] += r * r;
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 32; ++c)
        if (c < k && lane == 0) s_acc[warp][c] = acc2[c];
    __syncthreads();
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += s_acc[w][threadIdx.x];
        part[(size_t)blockIdx.x * k + threadIdx.x] = t;
    }
}

template <typename TA>
static void launch_res_t(const kpp_matrix &A, int k, const double *b, const double *x, float *r32, double *part,
                         int grid, cudaStream_t st, const int *skip) {
    const bool sm = (k == 1) && x && A.cols <= RES_SMEM_COLS;
    const size_t smem = sm ? (size_t)A.cols * sizeof(double) : 0;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(residual_kernel<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    residual_kernel<TA><<<grid, 256, smem, st>>>((const TA *)A.data, A.ld, A.rows, A.cols, k, b, x, r32, part, skip);
}

__global__ void axpy_f32_to_f64_kernel(int64_t n, const float *__restrict__ d, double *__restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}

__global__ void f64_to_f32_kernel(int64_t n, const double *__restrict__ a, float *__restrict__ o) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (float)a[i];
}

// ---------------------------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------------------------
size_t solve_smem_bytes(int s, int KP, int64_t CW, size_t tc_size) {
    return ((size_t)2 * s * KP + (size_t)NW * 32 * KP + (size_t)CW * KP) * tc_size;
}

template <typename TA, typename TC, int KP, bool CD>
static cudaError_t launch_solve_t(const SysArgs *d_sys, int nsys, const Common &cm, cudaStream_t st) {
    auto kern = solve_kernel<TA, TC, KP, CD>;
    const size_t smem = solve_smem_bytes(cm.s, KP, cm.CW, sizeof(TC));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if ((int64_t)per_sm * sm_count() < (int64_t)nsys * cm.G) return cudaErrorCooperativeLaunchTooLarge;
    Common c = cm;
    void *args[] = {(void *)&d_sys, (void *)&c};
    note_launch();
    return cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)(nsys * cm.G)), dim3(NT), args, smem, st);
}

template <typename TA, typename TC, bool CD>
static cudaError_t launch_kp(const SysArgs *d_sys, int nsys, const Common &cm, int KP, cudaStream_t st) {
    switch (KP) {
        case 1: return launch_solve_t<TA, TC, 1, CD>(d_sys, nsys, cm, st);
        case 8: return launch_solve_t<TA, TC, 8, CD>(d_sys, nsys, cm, st);
        case 32: return launch_solve_t<TA, TC, 32, CD>(d_sys, nsys, cm, st);
        default: return cudaErrorInvalidValue;
    }
}

int pick_kp(int k) { return k <= 1 ? 1 : (k <= 8 ? 8 : 32); }

cudaError_t launch_solve(int dtype, bool fp64_compute, bool cd, const SysArgs *d_sys, int nsys, const Common &cm,
                         int KP, cudaStream_t st) {
    if (dtype == KPP_F64) {
        return cd ? launch_kp<double, double, true>(d_sys, nsys, cm, KP, st)
                  : launch_kp<double, double, false>(d_sys, nsys, cm, KP, st);
    }
    (void)fp64_compute;
    if (dtype == KPP_F32) {
        return cd ? launch_kp<float, float, true>(d_sys, nsys, cm, KP, st)
                  : launch_kp<float, float, false>(d_sys, nsys, cm, KP, st);
    }
    return cd ? launch_kp<__nv_bfloat16, float, true>(d_sys, nsys, cm, KP, st)
              : launch_kp<__nv_bfloat16, float, false>(d_sys, nsys, cm, KP, st);
}

__global__ void sample_blocks_kernel(uint64_t seed, uint32_t sys, int64_t t0, int64_t count, int32_t nb,
                                     int32_t *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = draw_block(seed, t0 + i, sys, nb);
}

cudaError_t launch_sample_blocks(uint64_t seed, uint32_t sys, int64_t t0, int64_t count, int32_t nb, int32_t *out,
                                 cudaStream_t st) {
    if (count > 0) {
        note_launch();
        sample_blocks_kernel<<<2 * sm_count(), 256, 0, st>>>(seed, sys, t0, count, nb, out);
    }
    return cudaGetLastError();
}

int residual_grid() { return 4 * sm_count(); }

cudaError_t launch_residual(const kpp_matrix &A, int k, const double *b, const double *x, float *r32, double *part,
                            cudaStream_t st) {
    return launch_residual_grid(A, k, b, x, r32, part, residual_grid(), st);
}

cudaError_t launch_residual_grid(const kpp_matrix &A, int k, const double *b, const double *x, float *r32,
                                 double *part, int grid, cudaStream_t st, const int *skip) {
    switch (A.dtype) {
        case KPP_F64: launch_res_t<double>(A, k, b, x, r32, part, grid, st, skip); break;
        case KPP_F32: launch_res_t<float>(A, k, b, x, r32, part, grid, st, skip); break;
        default: launch_res_t<__nv_bfloat16>(A, k, b, x, r32, part, grid, st, skip);
    }
    return cudaGetLastError();
}

cudaError_t launch_axpy(int64_t n, const float *d, double *x, cudaStream_t st) {
    note_launch();
    axpy_f32_to_f64_kernel<<<2 * sm_count(), 256, 0, st>>>(n, d, x);
    return cudaGetLastError();
}

template <typename T>
__global__ void negate_copy_kernel(int64_t n, const T *__restrict__ a, T *__restrict__ o) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = -a[i];
}

cudaError_t launch_negate_copy(size_t n, const void *src, void *dst, bool f64, cudaStream_t st) {
    note_launch();
    if (f64) negate_copy_kernel<double><<<2 * sm_count(), 256, 0, st>>>((int64_t)n, (const double *)src, (double *)dst);
    else negate_copy_kernel<float><<<2 * sm_count(), 256, 0, st>>>((int64_t)n, (const float *)src, (float *)dst);
    return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(int64_t n, const double *a, float *o, cudaStream_t st) {
    note_launch();
    f64_to_f32_kernel<<<2 * sm_count(), 256, 0, st>>>(n, a, o);
    return cudaGetLastError();
}

}  // namespace kpp
