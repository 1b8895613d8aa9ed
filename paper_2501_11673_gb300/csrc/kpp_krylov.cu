// kpp_krylov.cu -- the Krylov solvers the paper compares CD++ with (Sec. 6: conjugate gradients for
// PSD systems, GMRES), as FP64 persistent kernels: the reference points of the time-to-tolerance
// comparison on the GPU, next to the paper's flop model for them (CG 2n^2 + 11n per iteration; GMRES
// 2n^2 T + 4n T (T + 1) after T iterations).
//
// One cooperative launch runs a whole solve.  The G CTAs split the rows of A; a matrix-vector
// product reads the full direction vector (shared memory when it fits) and each warp forms whole
// row dot products in a fixed order.  Global reductions go through per-CTA partial sums and a bounded
// group barrier; every CTA sums the partials itself in CTA order, so all CTAs hold bitwise the same
// scalars and take the same decisions.
//
// CG (plain, x0 from x): r = b - A x, p = r; per iteration q = A p, alpha = r.r / p.q, x += alpha p,
// r -= alpha q, beta = r'.r' / r.r, p = r + beta p; stop when |r| <= tol |b| (the recurrence
// residual), three barriers per iteration.
//
// GMRES(m) (x0 from x): Arnoldi with classical Gram-Schmidt and one reorthogonalisation pass (CGS2),
// Givens rotations applied redundantly in every CTA, stop when the rotated residual |g_{j+1}| <=
// tol |b|, restart after m inner steps with x += V y.
#include <cmath>
#include <cstring>
#include <vector>

#include "kpp_internal.cuh"
#include "kpp_launch.h"
#include "kpp_runtime.h"
#include "kpp_solve.h"

namespace kpp {

constexpr int KR_NT = 256;
constexpr int KR_NW = KR_NT / 32;

struct KrylovArgs {
    const double *A;
    int64_t lda, n;
    const double *b;
    double *x;
    double *r, *p, *q;   // n each (GMRES: r is w, the new Arnoldi vector)
    double *V;           // GMRES: (m + 1) x n basis, vector l at V + l n
    double *H;           // GMRES: m x (m + 1) rotated Hessenberg columns (column j at H + j (m + 1))
    double *part;        // G x (m + 2) partial sums
    unsigned *bar;
    int *err;
    double tol;
    int64_t max_iters;
    int m;               // GMRES restart length
    uint64_t timeout_ns;
    double *out;         // [0] iterations, [1] residual estimate |r| / |b|, [2] status, [3] restarts
};

// v of my rows: out_i = sum_c A_ic v_c for rows [r0, r1).  A warp takes two rows at a time; its
// lanes read 16-byte pairs of columns, eight pairs of each row per round (lane l: pairs l + 32 u,
// u = 0 .. 7), so that 16 loads of 16 bytes are in flight per lane: the product streams A from HBM,
// and it needs that many bytes in flight per SM to approach the copy bandwidth.  Each row has four
// accumulators (pair u goes to accumulator u mod 4; the tail after the last full round to 0), summed (a0 + a1) + (a2 + a3) and then across the
// lanes by a fixed shuffle tree: a fixed order.  v comes from shared memory when staged there, else
// from global memory; odd n, an odd leading dimension or unaligned pointers take the plain loop.
__device__ __forceinline__ double2 kr_ld2(const double2 *p, int64_t i, bool v_shared) {
    return v_shared ? p[i] : __ldcg(p + i);
}

__device__ __forceinline__ void kr_matvec_rows(const KrylovArgs &a, int64_t r0, int64_t r1, const double *sv,
                                               const double *gv, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = a.n;
    const bool vec = ((n | a.lda) & 1) == 0 &&
                     ((reinterpret_cast<uintptr_t>(a.A) | reinterpret_cast<uintptr_t>(gv)) & 15) == 0;
    const bool vs = sv != nullptr;
    const double *v = vs ? sv : gv;
    for (int64_t i = r0 + 2 * warp; i < r1; i += 2 * KR_NW) {
        const bool two = i + 1 < r1;
        double ra[4] = {0.0, 0.0, 0.0, 0.0}, rb[4] = {0.0, 0.0, 0.0, 0.0};
        if (vec) {
            const double2 *xa = reinterpret_cast<const double2 *>(a.A + i * a.lda);
            const double2 *xb = reinterpret_cast<const double2 *>(a.A + (two ? i + 1 : i) * a.lda);
            const double2 *v2 = reinterpret_cast<const double2 *>(v);
            const int64_t n2 = n >> 1;
            int64_t q = lane;
            for (; q + 7 * 32 < n2; q += 8 * 32) {
                double2 la[8], lb[8], y[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    la[u] = xa[q + 32 * u];
                    lb[u] = xb[q + 32 * u];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) y[u] = kr_ld2(v2, q + 32 * u, vs);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    ra[u & 3] = fma(la[u].y, y[u].y, fma(la[u].x, y[u].x, ra[u & 3]));
                    rb[u & 3] = fma(lb[u].y, y[u].y, fma(lb[u].x, y[u].x, rb[u & 3]));
                }
            }
            for (; q < n2; q += 32) {  // the tail: accumulator 0
                const double2 la = xa[q], lb = xb[q], y = kr_ld2(v2, q, vs);
                ra[0] = fma(la.y, y.y, fma(la.x, y.x, ra[0]));
                rb[0] = fma(lb.y, y.y, fma(lb.x, y.x, rb[0]));
            }
        } else {
            const double *xa = a.A + i * a.lda, *xb = a.A + (two ? i + 1 : i) * a.lda;
            for (int64_t c = lane; c < n; c += 32) {
                const double y = vs ? v[c] : __ldcg(v + c);
                ra[0] = fma(xa[c], y, ra[0]);
                rb[0] = fma(xb[c], y, rb[0]);
            }
        }
        double da = (ra[0] + ra[1]) + (ra[2] + ra[3]);
        double db = (rb[0] + rb[1]) + (rb[2] + rb[3]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            da += __shfl_xor_sync(0xffffffffu, da, o);
            db += __shfl_xor_sync(0xffffffffu, db, o);
        }
        if (lane == 0) {
            out[i] = da;
            if (two) out[i + 1] = db;
        }
    }
}

// Block-wide sum of one double per thread (fixed tree), valid in every thread.
__device__ __forceinline__ double kr_block_sum(double v, double *red) {
    return block_sum<KR_NT>(v, red);
}

__global__ void __launch_bounds__(KR_NT, 1) cg_kernel(KrylovArgs a) {
    extern __shared__ __align__(16) double sv_dyn[];
    __shared__ double s_red[KR_NW];
    const int G = gridDim.x, g = blockIdx.x;
    const int64_t n = a.n;
    const int64_t R = (n + G - 1) / G;
    const int64_t r0 = (int64_t)g * R < n ? (int64_t)g * R : n;
    const int64_t r1 = r0 + R < n ? r0 + R : n;
    double *sv = a.m > 0 ? sv_dyn : nullptr;  // a.m > 0: the direction vector fits shared memory
    GroupSync gs{a.bar, a.err, 0u, (unsigned)G, a.timeout_ns};
    double *pq = a.part, *rr = a.part + G, *bb = a.part + 2 * G;
    int64_t it = 0;
    int status = KPP_ERR_NO_CONVERGENCE;
    double bn2 = 0.0, rho = 0.0;

    // r = b - A x, p = r, |b|^2 and |r|^2
    if (sv) {
        for (int64_t c = threadIdx.x; c < n; c += KR_NT) sv[c] = a.x[c];
        __syncthreads();
    }
    kr_matvec_rows(a, r0, r1, sv, a.x, a.q);
    __syncthreads();
    {
        double vb = 0.0, vr = 0.0;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += KR_NT) {
            const double ri = a.b[i] - a.q[i];
            a.r[i] = ri;
            a.p[i] = ri;
            vb = fma(a.b[i], a.b[i], vb);
            vr = fma(ri, ri, vr);
        }
        vb = kr_block_sum(vb, s_red);
        vr = kr_block_sum(vr, s_red);
        if (threadIdx.x == 0) {
            bb[g] = vb;
            rr[g] = vr;
        }
    }
    if (!group_barrier(gs)) goto done;
    for (int h = 0; h < G; ++h) {
        bn2 += __ldcg(bb + h);
        rho += __ldcg(rr + h);
    }
    while (true) {
        if (!isfinite(rho)) {
            status = KPP_ERR_NUMERIC;
            break;
        }
        if (sqrt(rho) <= a.tol * sqrt(bn2)) {
            status = KPP_OK;
            break;
        }
        if (it >= a.max_iters) break;
        // q = A p (p complete in every row: barrier at the end of the previous iteration)
        if (sv) {
            for (int64_t c = threadIdx.x; c < n; c += KR_NT) sv[c] = __ldcg(a.p + c);
            __syncthreads();
        }
        kr_matvec_rows(a, r0, r1, sv, a.p, a.q);
        __syncthreads();
        {
            double v = 0.0;
            for (int64_t i = r0 + threadIdx.x; i < r1; i += KR_NT) v = fma(a.p[i], a.q[i], v);
            v = kr_block_sum(v, s_red);
            if (threadIdx.x == 0) pq[g] = v;
        }
        if (!group_barrier(gs)) break;
        double pAp = 0.0;
        for (int h = 0; h < G; ++h) pAp += __ldcg(pq + h);
        const double alpha = rho / pAp;
        {
            double v = 0.0;
            for (int64_t i = r0 + threadIdx.x; i < r1; i += KR_NT) {
                a.x[i] = fma(alpha, a.p[i], a.x[i]);
                const double ri = fma(-alpha, a.q[i], a.r[i]);
                a.r[i] = ri;
                v = fma(ri, ri, v);
            }
            v = kr_block_sum(v, s_red);
            if (threadIdx.x == 0) rr[g] = v;
        }
        if (!group_barrier(gs)) break;
        double rho2 = 0.0;
        for (int h = 0; h < G; ++h) rho2 += __ldcg(rr + h);
        const double beta = rho2 / rho;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += KR_NT) a.p[i] = fma(beta, a.p[i], a.r[i]);
        rho = rho2;
        ++it;
        if (!group_barrier(gs)) break;
    }
done:
    if (g == 0 && threadIdx.x == 0) {
        a.out[0] = (double)it;
        a.out[1] = bn2 > 0.0 ? sqrt(rho / bn2) : sqrt(rho);
        a.out[2] = (double)status;
    }
}

constexpr int KR_MMAX = 512;  // GMRES restart length at most

// partial dot products of my rows: part[l] = sum_{i in [r0, r1)} V_l[i] w[i] for l = 0 .. j (warp per l)
__device__ __forceinline__ void kr_partial_dots(const double *V, int64_t n, const double *w, int64_t r0, int64_t r1,
                                                int j, double *part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = warp; l <= j; l += KR_NW) {
        const double *vl = V + (int64_t)l * n;
        double acc = 0.0;
        for (int64_t i = r0 + lane; i < r1; i += 32) acc = fma(__ldcg(vl + i), w[i], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) part[l] = acc;
    }
}

__global__ void __launch_bounds__(KR_NT, 1) gmres_kernel(KrylovArgs a, int stage_v) {
    extern __shared__ __align__(16) double sv_dyn[];
    __shared__ double s_red[KR_NW];
    __shared__ double cs[KR_MMAX], sn[KR_MMAX], gv[KR_MMAX + 1], hc[KR_MMAX + 1], yv[KR_MMAX];
    __shared__ int s_stop;
    const int G = gridDim.x, g = blockIdx.x;
    const int64_t n = a.n;
    const int m = a.m;
    const int PS = m + 2;  // partial sums per CTA
    const int64_t R = (n + G - 1) / G;
    const int64_t r0 = (int64_t)g * R < n ? (int64_t)g * R : n;
    const int64_t r1 = r0 + R < n ? r0 + R : n;
    double *sv = stage_v ? sv_dyn : nullptr;
    GroupSync gs{a.bar, a.err, 0u, (unsigned)G, a.timeout_ns};
    double *w = a.r;
    int64_t it = 0, restarts = 0;
    int status = KPP_ERR_NO_CONVERGENCE;
    double bn = 0.0, res = 0.0;
    bool fail = false;

    {
        double v = 0.0;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += KR_NT) v = fma(a.b[i], a.b[i], v);
        v = kr_block_sum(v, s_red);
        if (threadIdx.x == 0) a.part[(size_t)g * PS] = v;
        if (!group_barrier(gs)) goto done;
        double t = 0.0;
        for (int h = 0; h < G; ++h) t += __ldcg(a.part + (size_t)h * PS);
        bn = sqrt(t);
        if (!group_barrier(gs)) goto done;  // the partials are reused below
    }
    while (true) {
        // w = b - A x, beta = |w|
        if (sv) {
            for (int64_t c = threadIdx.x; c < n; c += KR_NT) sv[c] = __ldcg(a.x + c);
            __syncthreads();
        }
        kr_matvec_rows(a, r0, r1, sv, a.x, w);
        __syncthreads();
        {
            double v = 0.0;
            for (int64_t i = r0 + threadIdx.x; i < r1; i += KR_NT) {
                const double wi = a.b[i] - w[i];
                w[i] = wi;
                v = fma(wi, wi, v);
            }
            v = kr_block_sum(v, s_red);
            if (threadIdx.x == 0) a.part[(size_t)g * PS] = v;
        }
        if (!group_barrier(gs)) break;
        double beta2 = 0.0;
        for (int h = 0; h < G; ++h) beta2 += __ldcg(a.part + (size_t)h * PS);
        const double beta = sqrt(beta2);
        res = beta;
        if (!isfinite(beta)) {
            status = KPP_ERR_NUMERIC;
            break;
        }
        if (beta <= a.tol * bn) {
            status = KPP_OK;
            break;
        }
        if (it >= a.max_iters) break;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += KR_NT) a.V[i] = w[i] / beta;
        if (threadIdx.x == 0) {
            gv[0] = beta;
            s_stop = 0;
        }
        if (!group_barrier(gs)) break;  // V_0 complete (and the partials read)
        int k = 0;                      // inner steps done in this cycle
        for (int j = 0; j < m; ++j) {
            // w = A V_j
            const double *vj = a.V + (int64_t)j * n;
            if (sv) {
                for (int64_t c = threadIdx.x; c < n; c += KR_NT) sv[c] = __ldcg(vj + c);
                __syncthreads();
            }
            kr_matvec_rows(a, r0, r1, sv, vj, w);
            __syncthreads();
            // two classical Gram-Schmidt passes against V_0 .. V_j
            for (int pass = 0; pass < 2 && !fail; ++pass) {
                kr_partial_dots(a.V, n, w, r0, r1, j, a.part + (size_t)g * PS);
                if (!group_barrier(gs)) {
                    fail = true;
                    break;
                }
                for (int l = threadIdx.x; l <= j; l += KR_NT) {
                    double t = 0.0;
                    for (int h = 0; h < G; ++h) t += __ldcg(a.part + (size_t)h * PS + l);
                    hc[l] = pass == 0 ? t : hc[l] + t;
                    yv[l] = t;
                }
                __syncthreads();
                for (int64_t i = r0 + threadIdx.x; i < r1; i += KR_NT) {
                    double wi = w[i];
                    for (int l = 0; l <= j; ++l) wi = fma(-yv[l], __ldcg(a.V + (int64_t)l * n + i), wi);
                    w[i] = wi;
                }
                __syncthreads();
                if (!group_barrier(gs)) {  // every CTA has read the partials before they are rewritten
                    fail = true;
                    break;
                }
            }
            if (fail) break;
            {
                double v = 0.0;
                for (int64_t i = r0 + threadIdx.x; i < r1; i += KR_NT) v = fma(w[i], w[i], v);
                v = kr_block_sum(v, s_red);
                if (threadIdx.x == 0) a.part[(size_t)g * PS + m + 1] = v;
            }
            if (!group_barrier(gs)) {
                fail = true;
                break;
            }
            double hn2 = 0.0;
            for (int h = 0; h < G; ++h) hn2 += __ldcg(a.part + (size_t)h * PS + m + 1);
            const double hn = sqrt(hn2);
            if (hn > 0.0)
                for (int64_t i = r0 + threadIdx.x; i < r1; i += KR_NT) a.V[(int64_t)(j + 1) * n + i] = w[i] / hn;
            if (threadIdx.x == 0) {
                // rotate the new column by the earlier rotations, then zero its subdiagonal
                hc[j + 1] = hn;
                for (int l = 0; l < j; ++l) {
                    const double t = cs[l] * hc[l] + sn[l] * hc[l + 1];
                    hc[l + 1] = -sn[l] * hc[l] + cs[l] * hc[l + 1];
                    hc[l] = t;
                }
                const double d = hypot(hc[j], hc[j + 1]);
                const double c = d > 0.0 ? hc[j] / d : 1.0, sg = d > 0.0 ? hc[j + 1] / d : 0.0;
                cs[j] = c;
                sn[j] = sg;
                hc[j] = d;
                hc[j + 1] = 0.0;
                gv[j + 1] = -sg * gv[j];
                gv[j] = c * gv[j];
                s_stop = (!isfinite(gv[j + 1]) || fabs(gv[j + 1]) <= a.tol * bn || hn == 0.0 ||
                          it + 1 >= a.max_iters) ? 1 : 0;
            }
            __syncthreads();
            if (g == 0)
                for (int l = threadIdx.x; l <= j; l += KR_NT) a.H[(size_t)j * (m + 1) + l] = hc[l];
            ++it;
            k = j + 1;
            res = fabs(gv[j + 1]);
            if (!group_barrier(gs)) {  // V_{j+1} and column j of H complete
                fail = true;
                break;
            }
            if (s_stop) break;
        }
        if (fail) break;
        // y = R^{-1} g (R: the rotated columns in H, upper triangular), x += V y on my rows
        if (threadIdx.x == 0)
            for (int l = 0; l < k; ++l) yv[l] = gv[l];
        __syncthreads();
        for (int i = k - 1; i >= 0; --i) {
            if (threadIdx.x == 0) yv[i] = yv[i] / __ldcg(a.H + (size_t)i * (m + 1) + i);
            __syncthreads();
            for (int l = threadIdx.x; l < i; l += KR_NT) yv[l] -= __ldcg(a.H + (size_t)i * (m + 1) + l) * yv[i];
            __syncthreads();
        }
        for (int64_t i = r0 + threadIdx.x; i < r1; i += KR_NT) {
            double xi = a.x[i];
            for (int l = 0; l < k; ++l) xi = fma(yv[l], __ldcg(a.V + (int64_t)l * n + i), xi);
            a.x[i] = xi;
        }
        ++restarts;
        if (!group_barrier(gs)) break;  // x complete before the next residual
    }
done:
    if (g == 0 && threadIdx.x == 0) {
        a.out[0] = (double)it;
        a.out[1] = bn > 0.0 ? res / bn : res;
        a.out[2] = (double)status;
        a.out[3] = (double)restarts;
    }
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
static kpp_status krylov_solve(bool gmres, const kpp_matrix *A, const double *b, double *x, int m, double tol,
                               int64_t max_iters, kpp_report *rep, cudaStream_t st) {
    clear_error();
    if (!A || !A->data || !b || !x || A->dtype != KPP_F64 || A->rows != A->cols || A->rows < 1 || A->ld < A->cols ||
        max_iters < 0 || !(tol >= 0.0) || (gmres && (m < 1 || m > KR_MMAX))) {
        set_error("%s: needs an FP64 square matrix, non-null b and x, tol >= 0, max_iters >= 0%s",
                  gmres ? "kpp_gmres" : "kpp_cg", gmres ? ", 1 <= restart <= 512" : "");
        return KPP_ERR_ARG;
    }
    const int64_t n = A->rows;
    int G = (int)std::min<int64_t>((n + KR_NW - 1) / KR_NW, sm_count());
    if (G < 1) G = 1;
    const bool stage = n * 8 <= 160 * 1024;
    const size_t smem = stage ? (size_t)n * 8 : 0;
    kpp_status rc = KPP_OK;
    Scratch scr(st);
    KrylovArgs a;
    memset(&a, 0, sizeof(a));
    a.A = (const double *)A->data;
    a.lda = A->ld;
    a.n = n;
    a.b = b;
    a.x = x;
    a.tol = tol;
    a.max_iters = max_iters;
    a.m = gmres ? m : (stage ? 1 : 0);
    a.timeout_ns = 2000000000ull;
    double hout[4] = {0, 0, 0, 0};
    int herr = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    CUDA_OR(scr.alloc((void **)&a.r, n * 8), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.p, n * 8), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.q, n * 8), KPP_ERR_CUDA);
    if (gmres) {
        CUDA_OR(scr.alloc((void **)&a.V, (size_t)(m + 1) * n * 8), KPP_ERR_CUDA);
        CUDA_OR(scr.alloc((void **)&a.H, (size_t)m * (m + 1) * 8), KPP_ERR_CUDA);
        CUDA_OR(scr.alloc((void **)&a.part, (size_t)G * (m + 2) * 8), KPP_ERR_CUDA);
    } else {
        CUDA_OR(scr.alloc((void **)&a.part, (size_t)3 * G * 8), KPP_ERR_CUDA);
    }
    CUDA_OR(scr.alloc((void **)&a.bar, 64), KPP_ERR_CUDA);
    a.err = (int *)((char *)a.bar + 32);
    CUDA_OR(scr.alloc((void **)&a.out, 4 * 8), KPP_ERR_CUDA);
    CUDA_OR(cudaMemsetAsync(a.bar, 0, 64, st), KPP_ERR_CUDA);
    CUDA_OR(cudaMemsetAsync(a.out, 0, 32, st), KPP_ERR_CUDA);
    CUDA_OR(cudaEventCreate(&e0), KPP_ERR_CUDA);
    CUDA_OR(cudaEventCreate(&e1), KPP_ERR_CUDA);
    {
        const void *kern = gmres ? (const void *)gmres_kernel : (const void *)cg_kernel;
        CUDA_OR(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), KPP_ERR_CUDA);
        int per_sm = 0;
        CUDA_OR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, KR_NT, smem), KPP_ERR_CUDA);
        if (per_sm * sm_count() < G) {
            set_error("Krylov kernel: %d CTAs do not fit co-resident", G);
            rc = KPP_ERR_UNSUPPORTED;
            goto cleanup;
        }
        int sv_flag = stage ? 1 : 0;
        void *args_cg[] = {&a};
        void *args_gm[] = {&a, &sv_flag};
        CUDA_OR(cudaEventRecord(e0, st), KPP_ERR_CUDA);
        note_launch();
        CUDA_OR(cudaLaunchCooperativeKernel(kern, dim3((unsigned)G), dim3(KR_NT), gmres ? args_gm : args_cg, smem, st),
                KPP_ERR_CUDA);
        CUDA_OR(cudaEventRecord(e1, st), KPP_ERR_CUDA);
    }
    CUDA_OR(cudaMemcpyAsync(hout, a.out, sizeof(hout), cudaMemcpyDeviceToHost, st), KPP_ERR_CUDA);
    CUDA_OR(cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, st), KPP_ERR_CUDA);
    CUDA_OR(cudaStreamSynchronize(st), KPP_ERR_CUDA);
    cudaEventElapsedTime(&ms, e0, e1);
    {
        std::vector<double> r2, b2;
        kpp_status r3 = residual_norms(*A, 1, b, x, nullptr, r2, &b2, st);
        if (r3 != KPP_OK) {
            rc = r3;
            goto cleanup;
        }
        const double rel = b2[0] > 0 ? std::sqrt(r2[0] / b2[0]) : std::sqrt(r2[0]);
        kpp_status status = herr ? (kpp_status)herr : (kpp_status)(int)hout[2];
        if (status == KPP_OK && !std::isfinite(rel)) status = KPP_ERR_NUMERIC;
        if (rep) {
            memset(rep, 0, sizeof(*rep));
            rep->iters = (int64_t)hout[0];
            rep->outer = (int64_t)hout[3];
            rep->rel_res_true = rel;
            rep->rel_res_est = hout[1];
            rep->status = status;
            rep->bad_block = -1;
            rep->device_ms = ms;
            rep->kernel_ms = ms;
            rep->launches = 1;
        }
        rc = status;
        if (rc != KPP_OK) set_error("%s ended with %s", gmres ? "kpp_gmres" : "kpp_cg", kpp_status_string(rc));
    }
cleanup:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

}  // namespace kpp

using namespace kpp;

extern "C" {

kpp_status kpp_cg(const kpp_matrix *A, const double *b, double *x, double tol, int64_t max_iters, kpp_report *rep,
                  void *stream) {
    return krylov_solve(false, A, b, x, 0, tol, max_iters, rep, (cudaStream_t)stream);
}

kpp_status kpp_gmres(const kpp_matrix *A, const double *b, double *x, int32_t restart, double tol, int64_t max_iters,
                     kpp_report *rep, void *stream) {
    return krylov_solve(true, A, b, x, restart, tol, max_iters, rep, (cudaStream_t)stream);
}

}  // extern "C"
