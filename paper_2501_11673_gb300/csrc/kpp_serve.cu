// kpp_serve.cu -- the device-resident request loop of the serving runtime (kpp_server_*).
//
// One persistent cooperative launch holds `nslots` slots of G CTAs.  CTA 0 of a slot claims the next
// published job (a compare-and-swap on a device counter, never past the count the host published in
// mapped host memory) and hands its number to the slot through the slot's group barrier.  The slot then
// runs the job's whole solve with its own CTAs:
//   * FP64 storage: one CD++ / K++ solve of A X = B (Alg. 3 / Alg. 5 with the memoised factors);
//   * BF16 / FP32 storage: the mixed-precision form -- an FP64 residual r = B - A X per column, an FP32
//     inner solve of A d = r from d = 0 (momentum restarted, rho and rhat carried, the Philox counter
//     continuing), X += d in FP64, until every column meets tol or max_outer steps were taken.  A column
//     that has met tol is frozen: later inner solves leave it at d = 0.
// and writes the job's completion record to mapped host memory (fields first, then the state word with
// release semantics at system scope).  A job's result depends on the job alone (its slot's G, fixed
// reduction orders), so a request gives the same bits alone and in any mix.
// Every wait is bounded: a slot that finds no job for idle_ns leaves, and the kernel ends when every
// slot has left; the host relaunches it when new jobs are published.  Group barriers keep their time
// limit; a slot whose barrier timed out records KPP_ERR_TIMEOUT in its job and leaves.
#include <cmath>

#include "kpp_internal.cuh"
#include "kpp_runtime.h"
#include "kpp_serve.h"
#include "kpp_solve.h"
#include "kpp_solve_device.cuh"
#include "kpp_solve_group.cuh"

namespace kpp {

namespace {

__device__ __forceinline__ long long ld_acquire_sys_s64(const int64_t *p) {
    long long v;
    asm volatile("ld.acquire.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_sys_s32(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys_s32(int32_t *p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_gpu_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// FP64 residual of the outer system over the slot: r = B - A X (rows x k), rows split over the G CTAs
// (warp per row, lanes over columns, FP64 products of the widened stored entries).  Writes r rounded
// to FP32 into rb (the inner right-hand side) and, for CD++, -r into Rx (the inner solve's maintained
// residual A d - r at d = 0).  Leaves |r|^2 per column in s_rn2 and, when bn2 is set, |B|^2 in s_bn2,
// both summed in a fixed order.  Returns false on a group error.
template <typename TA, bool CD, bool STORE>
__device__ bool serve_residual(const ServeJob &J, int g, GroupSync &gs, double *s_part, double *s_rn2, double *s_bn2,
                               bool bn2) {
    constexpr int KP = SERVE_KP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TA *A = (const TA *)J.sa.A;
    const int64_t lda = J.sa.lda, rows = J.cm.rows, cols = J.cm.cols;
    const int k = J.cm.k, G = J.cm.G;
    float *rb = (float *)J.sa.b;
    float *Rx = (float *)J.sa.Rx;
    double a2[KP], b2[KP];
#pragma unroll
    for (int c = 0; c < KP; ++c) a2[c] = b2[c] = 0.0;
    for (int64_t i = (int64_t)g + (int64_t)G * warp; i < rows; i += (int64_t)G * NW) {
        double v[KP];
#pragma unroll
        for (int c = 0; c < KP; ++c) v[c] = 0.0;
        const TA *row = A + i * lda;
        for (int64_t col = lane; col < cols; col += 32) {
            const double a = widen_fast(row[col]);
#pragma unroll
            for (int c = 0; c < KP; ++c)
                if (c < k) v[c] = fma(a, __ldcg(J.X + col * k + c), v[c]);
        }
#pragma unroll
        for (int c = 0; c < KP; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            if (c < k) {
                const double bv = J.B[i * k + c];
                const double r = bv - v[c];
                a2[c] += r * r;
                b2[c] += bv * bv;
                if (STORE && lane == 0) {
                    rb[i * k + c] = (float)r;
                    if (CD) Rx[i * k + c] = -(float)r;
                }
            }
        }
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            s_part[warp * 2 * KP + c] = a2[c];
            s_part[warp * 2 * KP + KP + c] = b2[c];
        }
    __syncthreads();
    double *rpart = J.sa.rpart;  // G x 2KP doubles
    if (threadIdx.x < 2 * KP) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += s_part[w * 2 * KP + threadIdx.x];
        rpart[(size_t)g * 2 * KP + threadIdx.x] = t;
    }
    if (!group_barrier(gs)) return false;
    if (threadIdx.x < 2 * KP) {
        double t = 0.0;
        for (int h = 0; h < G; ++h) t += __ldcg(rpart + (size_t)h * 2 * KP + threadIdx.x);
        if (threadIdx.x < KP) s_rn2[threadIdx.x] = t;
        else if (bn2) s_bn2[threadIdx.x - KP] = t;
    }
    __syncthreads();
    return group_barrier(gs);  // every CTA has read the partials before they are written again
}

template <typename TA, bool CD>
__device__ void serve_mixed(const ServeJob &J, ServeDone *D, int g, GroupSync &gs) {
    constexpr int KP = SERVE_KP;
    __shared__ double s_part[NW * 2 * KP];
    __shared__ double s_rn2[KP], s_bn2[KP];
    __shared__ int s_conv[KP], s_status;
    const int k = J.cm.k, G = J.cm.G;
    const int64_t cols = J.cm.cols;
    float *d = (float *)J.sa.x;
    float *m = (float *)J.sa.m;
    float *Rm = (float *)J.sa.Rm;
    SolveScalars *sc = J.sa.sc;
    int outer = 0, status = KPP_OK;
    bool ok = true;
    if (threadIdx.x < KP) s_conv[threadIdx.x] = 0;
    for (;;) {
        if (!serve_residual<TA, CD, true>(J, g, gs, s_part, s_rn2, s_bn2, outer == 0)) {
            ok = false;
            break;
        }
        if (threadIdx.x == 0) {
            int all = 1;
            for (int c = 0; c < k; ++c) {
                const double rel = s_bn2[c] > 0.0 ? sqrt(s_rn2[c] / s_bn2[c]) : sqrt(s_rn2[c]);
                if (rel <= J.tol) s_conv[c] = 1;
                all &= s_conv[c];
            }
            s_status = all ? 1 : 0;
        }
        __syncthreads();
        if (s_status || outer >= J.max_outer) break;
        // the inner solve from d = 0, m = 0 (and R_m = A m = 0); the converged columns stay inactive
        for (int64_t e = (int64_t)g * NT + threadIdx.x; e < cols * k; e += (int64_t)G * NT) {
            d[e] = 0.0f;
            m[e] = 0.0f;
            if (CD) Rm[e] = 0.0f;
        }
        if (g == 0 && threadIdx.x < k) {
            SolveScalars &s = sc[threadIdx.x];
            s.E0 = 0.0;
            s.E1 = 0.0;
            s.status = KPP_OK;
            s.active = s_conv[threadIdx.x] ? 0 : 1;
        }
        if (!group_barrier(gs)) {
            ok = false;
            break;
        }
        solve_group<TA, float, KP, CD, false>(J.sa, J.cm, g, gs);
        if (!group_barrier(gs)) {
            ok = false;
            break;
        }
        if (threadIdx.x == 0) {
            int bad = KPP_OK;
            for (int c = 0; c < k; ++c) {
                const int st = __ldcg(&sc[c].status);
                if (st != KPP_OK && st != KPP_ERR_NO_CONVERGENCE) bad = st;
            }
            s_status = bad;
        }
        __syncthreads();
        // X += d in FP64
        for (int64_t e = (int64_t)g * NT + threadIdx.x; e < cols * k; e += (int64_t)G * NT)
            J.X[e] += (double)__ldcg(d + e);
        outer += 1;
        const int bad = s_status;
        if (!group_barrier(gs)) {
            ok = false;
            break;
        }
        if (bad != KPP_OK) {
            status = bad;
            break;
        }
    }
    if (!ok) status = *(volatile int *)gs.err ? *(volatile int *)gs.err : KPP_ERR_TIMEOUT;
    if (g == 0 && threadIdx.x == 0) {
        int all = 1;
        for (int c = 0; c < KP; ++c) {
            const bool in = c < k;
            const double rel = in ? (s_bn2[c] > 0.0 ? sqrt(s_rn2[c] / s_bn2[c]) : sqrt(s_rn2[c])) : 0.0;
            D->rel_res[c] = rel;
            D->rho[c] = in ? __ldcg(&sc[c].rho) : 0.0;
            const int cs = !in ? KPP_OK : (status != KPP_OK ? status : (s_conv[c] ? KPP_OK : KPP_ERR_NO_CONVERGENCE));
            D->col_status[c] = cs;
            if (in && cs != KPP_OK) all = 0;
        }
        D->status = status != KPP_OK ? status : (all ? KPP_OK : KPP_ERR_NO_CONVERGENCE);
        D->outer = outer;
        D->iters = __ldcg(&sc[0].t);
        __threadfence_system();
        st_release_sys_s32(&D->state, 1);
    }
}

template <typename TA, bool CD>
__device__ void serve_fp64(const ServeJob &J, ServeDone *D, int g, GroupSync &gs) {
    constexpr int KP = SERVE_KP;
    __shared__ double s_part[NW * 2 * KP];
    __shared__ double s_rn2[KP], s_bn2[KP];
    solve_group<TA, double, KP, CD, false>(J.sa, J.cm, g, gs);
    bool ok = group_barrier(gs);
    // the reported residual: |B - A X| / |B| in FP64 over the slot
    if (ok) ok = serve_residual<TA, CD, false>(J, g, gs, s_part, s_rn2, s_bn2, true);
    if (g == 0 && threadIdx.x == 0) {
        const int k = J.cm.k;
        const SolveScalars *sc = J.sa.sc;
        int status = KPP_OK;
        for (int c = 0; c < KP; ++c) {
            const bool in = c < k;
            const int cs = !ok ? KPP_ERR_TIMEOUT : (in ? (__ldcg(&sc[c].active) ? KPP_ERR_NO_CONVERGENCE : __ldcg(&sc[c].status)) : KPP_OK);
            D->col_status[c] = cs;
            D->rel_res[c] = in ? (s_bn2[c] > 0.0 ? sqrt(s_rn2[c] / s_bn2[c]) : sqrt(s_rn2[c])) : 0.0;
            D->rho[c] = in ? __ldcg(&sc[c].rho) : 0.0;
            if (in && cs != KPP_OK && status == KPP_OK) status = cs;
        }
        D->status = status;
        D->outer = 0;
        D->iters = __ldcg(&sc[0].t);
        __threadfence_system();
        st_release_sys_s32(&D->state, 1);
    }
}

__global__ void __launch_bounds__(NT, 1) serve_kernel(ServeArgs a) {
    const int slot = blockIdx.x / a.G, g = blockIdx.x % a.G;
    ServeSlot *sl = a.slots + slot;
    GroupSync gs{&sl->bar, &sl->err, 0u, (unsigned)a.G, a.timeout_ns};
    __shared__ long long s_job;
    __shared__ __align__(16) unsigned char s_jobraw[sizeof(ServeJob)];
    for (;;) {
        if (g == 0 && threadIdx.x == 0) {
            long long job = -1;
            const uint64_t t0 = globaltimer_ns();
            for (;;) {
                const unsigned long long c = ld_relaxed_gpu_u64(a.claimed);
                const long long p = ld_acquire_sys_s64(&a.ctl->published);
                if ((long long)c < p) {
                    if (atomicCAS(a.claimed, c, c + 1ull) == c) {
                        job = (long long)c;
                        break;
                    }
                    continue;
                }
                if (ld_relaxed_sys_s32(&a.ctl->drain)) break;
                if (globaltimer_ns() - t0 > a.idle_ns) break;
                __nanosleep(2000);
            }
            *(volatile long long *)&sl->job = job;
        }
        if (!group_barrier(gs)) return;
        if (threadIdx.x == 0) s_job = *(volatile long long *)&sl->job;
        __syncthreads();
        const long long job = s_job;
        if (!group_barrier(gs)) return;  // every CTA has read the slot's job word
        if (job < 0) return;
        // the job's descriptor, read around the caches (the ring entry is reused by later jobs)
        {
            const unsigned long long *src = (const unsigned long long *)(a.jobs + job % a.R);
            unsigned long long *dst = (unsigned long long *)s_jobraw;
            for (int e = threadIdx.x; e < (int)(sizeof(ServeJob) / 8); e += NT) dst[e] = __ldcv(src + e);
        }
        __syncthreads();
        const ServeJob &J = *reinterpret_cast<const ServeJob *>(s_jobraw);
        ServeDone *D = a.done + job % a.R;
        if (J.dtype == KPP_F64) {
            if (J.mode == 1) serve_fp64<double, true>(J, D, g, gs);
            else serve_fp64<double, false>(J, D, g, gs);
        } else if (J.dtype == KPP_F32) {
            if (J.mode == 1) serve_mixed<float, true>(J, D, g, gs);
            else serve_mixed<float, false>(J, D, g, gs);
        } else {
            if (J.mode == 1) serve_mixed<__nv_bfloat16, true>(J, D, g, gs);
            else serve_mixed<__nv_bfloat16, false>(J, D, g, gs);
        }
        if (*(volatile int *)gs.err != 0) return;  // the slot's barriers are spent: leave
        __syncthreads();
    }
}

}  // namespace

size_t serve_smem_bytes(int s, int64_t CW) { return solve_smem_bytes(s, SERVE_KP, CW, sizeof(double)); }

int serve_max_ctas(size_t smem) {
    int per_sm = 0;
    if (cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_kernel, NT, smem) != cudaSuccess)
        return 0;
    return per_sm * sm_count();
}

cudaError_t launch_serve(const ServeArgs &a, int nslots, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ServeArgs arg = a;
    void *args[] = {&arg};
    note_launch();
    return cudaLaunchCooperativeKernel((const void *)serve_kernel, dim3((unsigned)(nslots * a.G)), dim3(NT), args,
                                       smem, st);
}

}  // namespace kpp
