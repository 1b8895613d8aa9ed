// kpp_solve_device.cuh -- device pieces shared by the persistent solve kernels (kpp_solve.cu,
// kpp_solve2.cu): per-column state, small reductions, and the FP64 true-residual phase that confirms
// the stopping rule (Alg. 3) and, for CD++, replaces the maintained residual.
#pragma once

#include "kpp_internal.cuh"
#include "kpp_solve.h"

namespace kpp {

constexpr int NT = 256;       // threads per CTA
constexpr int NW = NT / 32;   // warps per CTA

struct ColState {             // per right-hand-side column (shared memory copy in every CTA)
    double E0, E1, rhat, rho, bn2, res_true, res_est;
    long long ci;
    int active, status;
};

template <typename TC> __device__ __forceinline__ TC tfma(TC a, TC b, TC c);
template <> __device__ __forceinline__ double tfma<double>(double a, double b, double c) { return fma(a, b, c); }
template <> __device__ __forceinline__ float tfma<float>(float a, float b, float c) { return fmaf(a, b, c); }

template <typename TC, int KP>
__device__ __forceinline__ void warp_reduce(TC (&v)[KP]) {
#pragma unroll
    for (int c = 0; c < KP; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
}

// The true residual |A x - b|^2 per column, rows split over the G CTAs of the group (warp per row,
// FP64 accumulation).  Optionally writes the residual rows into Rx (CD++ residual replacement).
// Leaves the totals in st[c].res_true (as |.|/|b|) in every CTA.  Returns false on a group error.
template <typename TA, typename TC, int KP>
__device__ bool true_residual_phase(const SysArgs &sa, const Common &cm, int g, GroupSync &gs, ColState *st,
                                    double *s_part, TC *Rx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TA *A = (const TA *)sa.A;
    const TC *b = (const TC *)sa.b;
    const TC *x = (const TC *)sa.x;
    const int k = cm.k;
    double acc2[KP];
#pragma unroll
    for (int c = 0; c < KP; ++c) acc2[c] = 0.0;
    for (int64_t i = (int64_t)g + (int64_t)cm.G * warp; i < cm.rows; i += (int64_t)cm.G * NW) {
        double v[KP];
#pragma unroll
        for (int c = 0; c < KP; ++c) v[c] = 0.0;
        const TA *row = A + i * sa.lda;
        for (int64_t col = lane; col < cm.cols; col += 32) {
            double a = widen_fast(row[col]);
#pragma unroll
            for (int c = 0; c < KP; ++c)
                if (c < k) v[c] = fma(a, (double)__ldcg(x + col * k + c), v[c]);
        }
#pragma unroll
        for (int c = 0; c < KP; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            if (c < k) {
                double r = v[c] - (double)b[i * k + c];
                acc2[c] += r * r;
                if (Rx && lane == 0) Rx[i * k + c] = (TC)r;
            }
        }
    }
    // per-CTA partial (warps in order), then the group total in a fixed order
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < KP; ++c) s_part[warp * KP + c] = acc2[c];
    __syncthreads();
    double *rpart = sa.rpart;  // G x KP
    if (threadIdx.x < KP) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += s_part[w * KP + threadIdx.x];
        rpart[(size_t)g * KP + threadIdx.x] = t;
    }
    if (!group_barrier(gs)) return false;
    if (threadIdx.x < KP && threadIdx.x < k) {
        double t = 0.0;
        for (int h = 0; h < cm.G; ++h) t += __ldcg(rpart + (size_t)h * KP + threadIdx.x);
        const double bn2 = st[threadIdx.x].bn2;
        st[threadIdx.x].res_true = bn2 > 0.0 ? sqrt(t / bn2) : sqrt(t);
    }
    __syncthreads();
    // the partials are reused by the next call: make sure every CTA has read them
    return group_barrier(gs);
}

}  // namespace kpp

namespace kpp {

// The checkpoint of Alg. 3 (and of Alg. 5) for one right-hand-side column, after
// the optional true-residual check has filled cs.res_true: stop test, then the weighted ratio of
// Eq. 5.3 (a_i = (i+1)^{ln(i+1)}; the first checkpoint takes the ratio itself) and
// rho = 1 - rhat^(1/zeta), clamped to [0, 1 - 1e-12]; then E0 = E1 = 0.
__device__ __forceinline__ void checkpoint_column(ColState &cs, const Common &cm, int zeta) {
    cs.ci += 1;
    bool stop = false;
    if (cm.tol > 0.0 && cs.E1 <= cm.tol * cm.tol * cs.bn2) stop = cm.confirm ? (cs.res_true <= cm.tol) : true;
    if (!isfinite(cs.E1) || !isfinite(cs.E0)) {
        cs.status = KPP_ERR_NUMERIC;
        cs.active = 0;
    } else if (stop) {
        cs.status = KPP_OK;
        cs.active = 0;
    } else if (cm.adaptive) {
        const double q = cs.E0 > 0.0 ? cs.E1 / cs.E0 : 0.0;
        if (cs.ci == 1) {
            cs.rhat = q;
        } else {
            const double li = log((double)cs.ci), li1 = log((double)cs.ci + 1.0);
            const double wgt = exp(li * li - li1 * li1);
            cs.rhat = wgt * cs.rhat + (1.0 - wgt) * q;
        }
        double rho = 1.0 - pow(cs.rhat, 1.0 / (double)zeta);
        if (!(rho > 0.0)) rho = 0.0;
        if (rho > 1.0 - 1e-12) rho = 1.0 - 1e-12;
        cs.rho = rho;
    }
    cs.E0 = 0.0;
    cs.E1 = 0.0;
}

}  // namespace kpp
