// kpp_solve.cu -- the block-step iteration of Kaczmarz++ and CD++ as one persistent kernel.
//
// Paper: arXiv 2501.11673.  One launch runs every iteration of one or more systems:
//   K++  (Alg. 1; Alg. 5, exact projection through the memoised factor):
//        r = A_S x - b_S;  y = (A_S A_S^T + lam I)^{-1} r;  w = A_S^T y;
//        m <- beta (m - w);  x <- x - w + eta m;   beta = (1 - rho)/(1 + rho)          (Eq. 1.3, 1.4)
//   CD++ (Eq. 5.1; Alg. 3) with the residual kept up to date:
//        r = R_x[S];  y = (A_SS + lam I)^{-1} r;  u = A_{:,S} y  (= A_S^T y, A symmetric);
//        R_m <- beta (R_m - u);  R_x <- R_x - u + eta R_m;  m <- beta (m - I_S^T y);  x <- x - I_S^T y + eta m
//   then, every step, E0 / E1 += |r|^2 and every 2 zeta steps the checkpoint of Alg. 3:
//   stop test on E1 (confirmed by the true residual), weighted ratio (Eq. 5.3), rho = 1 - rhat^(1/zeta).
//
// Work split inside a system (G CTAs, one group barrier counter):
//   * column chunks: CTA g owns columns [c0, c1) of x, m (and R_x, R_m) and streams the block rows
//     A_S[:, c0:c1] -- warps take rows, lanes take columns (coalesced row segments);
//   * the s x s projection y = G^{-1} r is split by rows across all CTAs (warp per row);
//   * the K++ residual is reduced from per-CTA partial sums in a fixed order (deterministic).
// Every CTA recomputes the scalars (|r|^2, E0, E1, rho) from identical data in an identical order,
// so all CTAs agree on rho and on the stop decision without another exchange.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "kpp_internal.cuh"
#include "kpp_runtime.h"
#include "kpp_solve.h"
#include "kpp_solve_device.cuh"

namespace kpp {

template <typename TA, typename TC, int KP, bool CD>
__global__ void __launch_bounds__(NT, 1) solve_kernel(const SysArgs *__restrict__ systems, Common cm) {
    const SysArgs sa = systems[blockIdx.x / cm.G];
    const int g = blockIdx.x % cm.G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = cm.k, s = cm.s, nb = cm.nb;
    const int64_t rows = cm.rows, cols = cm.cols;
    const TA *__restrict__ A = (const TA *)sa.A;
    const int64_t lda = sa.lda;
    const TC *__restrict__ b = (const TC *)sa.b;
    TC *__restrict__ x = (TC *)sa.x;
    TC *__restrict__ mv = (TC *)sa.m;
    TC *__restrict__ Rx = (TC *)sa.Rx;
    TC *__restrict__ Rm = (TC *)sa.Rm;
    const TC *__restrict__ Ginv = (const TC *)sa.Ginv;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC *s_r = (TC *)smem_raw;                 // s x KP
    TC *s_y = s_r + (size_t)s * KP;           // s x KP
    TC *s_red = s_y + (size_t)s * KP;         // NW x 32 x KP
    TC *s_x = s_red + (size_t)NW * 32 * KP;   // CW x KP (K++ chunk of x)
    __shared__ ColState st[KP];
    __shared__ double s_part[NW * KP];
    __shared__ double s_rn2[KP];
    __shared__ int s_stop, s_need;

    GroupSync gs{sa.bar, sa.err, 0u, (unsigned)cm.G, cm.timeout_ns};
    // first and end step (read before the first group barrier: CTA 0 rewrites sc at the end)
    const int64_t t_begin = cm.t0_state ? sa.sc[0].t : sa.t0;
    int64_t t_end = cm.t0_state ? t_begin + cm.max_iters : cm.max_iters;
    if (cm.t0_state) {  // a system whose columns are all done does not iterate (t stays put)
        int any = 0;
        for (int c = 0; c < k; ++c) any |= sa.sc[c].active;
        if (!any) t_end = t_begin;
    }

    // my column chunk (aligned to 32-byte sectors of A)
    const int64_t c0 = min64((int64_t)g * cm.CW, cols);
    const int64_t c1 = min64(c0 + cm.CW, cols);

    // ---- set-up: column state, |b|^2, (CD++) R_x = A x0 - b ----
    if (threadIdx.x < KP) {
        const int c = threadIdx.x;
        ColState cs = {};
        if (c < k) {
            const SolveScalars &in = sa.sc[c];
            cs.E0 = in.E0; cs.E1 = in.E1; cs.rhat = in.rhat; cs.rho = in.rho; cs.ci = in.ci;
            cs.active = in.active; cs.status = in.status;
        }
        cs.res_true = NAN;
        cs.res_est = NAN;
        st[c] = cs;
    }
    {
        double acc[KP];
#pragma unroll
        for (int c = 0; c < KP; ++c) acc[c] = 0.0;
        for (int64_t i = (int64_t)g * NT + threadIdx.x; i < rows; i += (int64_t)cm.G * NT)
#pragma unroll
            for (int c = 0; c < KP; ++c)
                if (c < k) acc[c] += (double)b[i * k + c] * (double)b[i * k + c];
        __syncthreads();
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            double v = block_sum<NT>(acc[c], s_part);
            if (threadIdx.x == 0) sa.rpart[(size_t)g * KP + c] = v;
        }
        if (g == cm.test_hold_cta) goto finish;  // wait test: leave without arriving
        if (!group_barrier(gs)) goto finish;
        if (threadIdx.x < KP) {
            double t = 0.0;
            for (int h = 0; h < cm.G; ++h) t += __ldcg(sa.rpart + (size_t)h * KP + threadIdx.x);
            st[threadIdx.x].bn2 = t;
        }
        __syncthreads();
        if (!group_barrier(gs)) goto finish;
    }
    if (CD && cm.init_residual) {
        if (!true_residual_phase<TA, TC, KP>(sa, cm, g, gs, st, s_part, Rx)) goto finish;
    }

    {
        const int zeta = nb;
        int64_t t = t_begin;
        while (t < t_end) {
            // ---- sample the block (every CTA draws the same j) ----
            const int j = draw_block(cm.seed, t, sa.sys_id, nb);
            const int64_t S0 = (int64_t)j * s;
            const int len = (int)min64(s, rows - S0);
            const TC *__restrict__ Gj = Ginv + (size_t)j * s * s;

            // ---- block residual r (s_r) ----
            if (!CD) {
                // partial r over my column chunk: warps over rows, lanes over columns
                for (int e = threadIdx.x; e < (int)(c1 - c0) * KP; e += NT) {
                    const int cc = e / KP, c = e % KP;
                    s_x[e] = (c < k) ? __ldcg(x + (c0 + cc) * k + c) : (TC)0;
                }
                __syncthreads();
                TC *part = (TC *)sa.part;  // G x s x KP
                for (int a = warp; a < len; a += NW) {
                    TC acc[KP];
#pragma unroll
                    for (int c = 0; c < KP; ++c) acc[c] = (TC)0;
                    const TA *row = A + (S0 + a) * lda;
#pragma unroll 4
                    for (int64_t col = c0 + lane; col < c1; col += 32) {
                        const TC av = conv<TC>(row[col]);
                        const TC *xs = s_x + (col - c0) * KP;
#pragma unroll
                        for (int c = 0; c < KP; ++c) acc[c] = tfma<TC>(av, xs[c], acc[c]);
                    }
                    warp_reduce<TC, KP>(acc);
                    if (lane == 0)
#pragma unroll
                        for (int c = 0; c < KP; ++c) part[((size_t)g * s + a) * KP + c] = acc[c];
                }
                if (!group_barrier(gs)) break;
                if (cm.reduce_redundant) {
                    for (int e = threadIdx.x; e < len * KP; e += NT) {
                        const int a = e / KP, c = e % KP;
                        TC v = (TC)0;
                        if (c < k) {
                            for (int h = 0; h < cm.G; ++h) v += __ldcg(part + ((size_t)h * s + a) * KP + c);
                            v -= b[(S0 + a) * k + c];
                        }
                        s_r[e] = v;
                    }
                } else {
                    // one warp per entry: lanes sum strided partials, then a fixed shuffle tree
                    TC *rbuf = (TC *)sa.rbuf;
                    for (int e = g * NW + warp; e < len * KP; e += cm.G * NW) {
                        const int a = e / KP, c = e % KP;
                        TC v = (TC)0;
                        if (c < k)
                            for (int h = lane; h < cm.G; h += 32) v += __ldcg(part + ((size_t)h * s + a) * KP + c);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (lane == 0) rbuf[e] = (c < k) ? v - b[(S0 + a) * k + c] : (TC)0;
                    }
                    if (!group_barrier(gs)) break;
                    for (int e = threadIdx.x; e < len * KP; e += NT) s_r[e] = __ldcg(rbuf + e);
                }
            } else {
                for (int e = threadIdx.x; e < len * KP; e += NT) {
                    const int a = e / KP, c = e % KP;
                    s_r[e] = (c < k) ? __ldcg(Rx + (S0 + a) * k + c) : (TC)0;
                }
            }
            __syncthreads();
            // |r|^2 per column: warp c % NW, lanes over rows, fixed tree
            for (int c = warp; c < k; c += NW) {
                double v = 0.0;
                for (int a = lane; a < len; a += 32) {
                    const double r = (double)s_r[a * KP + c];
                    v += r * r;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) s_rn2[c] = v;
            }
            // ---- projection y = G_j^{-1} r: rows spread over all CTAs (warp per row) ----
            {
                TC *ybuf = (TC *)sa.ybuf;
                for (int a = g + cm.G * warp; a < len; a += cm.G * NW) {
                    TC acc[KP];
#pragma unroll
                    for (int c = 0; c < KP; ++c) acc[c] = (TC)0;
                    const TC *grow = Gj + (size_t)a * len;
                    for (int d = lane; d < len; d += 32) {
                        const TC gv = grow[d];
#pragma unroll
                        for (int c = 0; c < KP; ++c) acc[c] = tfma<TC>(gv, s_r[d * KP + c], acc[c]);
                    }
                    warp_reduce<TC, KP>(acc);
                    if (lane == 0)
#pragma unroll
                        for (int c = 0; c < KP; ++c) ybuf[(size_t)a * KP + c] = acc[c];
                }
                if (!group_barrier(gs)) break;
                for (int e = threadIdx.x; e < len * KP; e += NT) s_y[e] = __ldcg(ybuf + e);
            }
            __syncthreads();

            // ---- back-projection and update on my column chunk ----
            __shared__ TC s_beta[KP], s_keep[KP];  // read with a runtime rhs index below
            if (threadIdx.x < KP) {
                const double rho = st[threadIdx.x].rho;
                s_beta[threadIdx.x] = (TC)((1.0 - rho) / (1.0 + rho));
                s_keep[threadIdx.x] = (TC)((threadIdx.x < k && st[threadIdx.x].active) ? 1 : 0);
            }
            __syncthreads();
            const TC eta = (TC)cm.eta;
            for (int64_t cb = c0; cb < c1; cb += 32) {
                const int64_t col = cb + lane;
                const bool valid = col < c1;
                TC acc[KP];
#pragma unroll
                for (int c = 0; c < KP; ++c) acc[c] = (TC)0;
                if (valid) {
#pragma unroll 4
                    for (int a = warp; a < len; a += NW) {
                        const TC av = conv<TC>(A[(S0 + a) * lda + col]);
#pragma unroll
                        for (int c = 0; c < KP; ++c) acc[c] = tfma<TC>(av, s_y[a * KP + c], acc[c]);
                    }
                }
#pragma unroll
                for (int c = 0; c < KP; ++c) s_red[(warp * 32 + lane) * KP + c] = acc[c];
                __syncthreads();
                // combine the warps' partial sums; threads take (column, rhs) pairs
                for (int e = threadIdx.x; e < 32 * KP; e += NT) {
                    const int ln = e / KP, c = e % KP;
                    const int64_t cl = cb + ln;
                    if (cl < c1 && c < k && s_keep[c] != (TC)0) {
                        TC u = (TC)0;
#pragma unroll
                        for (int w = 0; w < NW; ++w) u += s_red[(w * 32 + ln) * KP + c];
                        const size_t idx = (size_t)cl * k + c;
                        if (!CD) {
                            const TC mm = s_beta[c] * (__ldcg(mv + idx) - u);
                            mv[idx] = mm;
                            x[idx] = __ldcg(x + idx) - u + eta * mm;
                        } else {
                            const TC rm = s_beta[c] * (__ldcg(Rm + idx) - u);
                            Rm[idx] = rm;
                            Rx[idx] = __ldcg(Rx + idx) - u + eta * rm;
                            const TC wv = (cl >= S0 && cl < S0 + len) ? s_y[(cl - S0) * KP + c] : (TC)0;
                            const TC mm = s_beta[c] * (__ldcg(mv + idx) - wv);
                            mv[idx] = mm;
                            x[idx] = __ldcg(x + idx) - wv + eta * mm;
                        }
                    }
                }
                __syncthreads();
            }
            if (CD) {
                if (!group_barrier(gs)) break;
            }

            // ---- residual estimate, checkpoint, adaptive rho (identical in every CTA) ----
            const int64_t ph = t % (2 * (int64_t)zeta);
            if (threadIdx.x == 0) {
                s_need = 0;
                s_stop = 0;
            }
            __syncthreads();
            if (threadIdx.x < k) {
                ColState &cs = st[threadIdx.x];
                if (cs.active) {
                    if (ph < zeta) cs.E0 += s_rn2[threadIdx.x];
                    else cs.E1 += s_rn2[threadIdx.x];
                    if (ph == 2 * zeta - 1) {
                        cs.res_est = cs.bn2 > 0.0 ? sqrt(cs.E1 / cs.bn2) : sqrt(cs.E1);
                        if (cm.tol > 0.0 && cs.E1 <= cm.tol * cm.tol * cs.bn2 && cm.confirm) atomicOr(&s_need, 1);
                    }
                }
            }
            __syncthreads();
            t += 1;
            if (ph == 2 * zeta - 1) {
                if (s_need) {
                    // x must be complete in every chunk before the true residual (K++ has no barrier yet)
                    if (!CD && !group_barrier(gs)) break;
                    if (!true_residual_phase<TA, TC, KP>(sa, cm, g, gs, st, s_part, CD ? Rx : (TC *)nullptr)) break;
                }
                if (threadIdx.x < k) {
                    ColState &cs = st[threadIdx.x];
                    if (cs.active) {
                        cs.ci += 1;
                        bool stop = false;
                        if (cm.tol > 0.0 && cs.E1 <= cm.tol * cm.tol * cs.bn2) stop = cm.confirm ? (cs.res_true <= cm.tol) : true;
                        if (!isfinite(cs.E1) || !isfinite(cs.E0)) {
                            cs.status = KPP_ERR_NUMERIC;
                            cs.active = 0;
                        } else if (stop) {
                            cs.status = KPP_OK;
                            cs.active = 0;
                        } else {
                            if (cm.adaptive) {
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
                        }
                        cs.E0 = 0.0;
                        cs.E1 = 0.0;
                    }
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    int any = 0;
                    for (int c = 0; c < k; ++c) any |= st[c].active;
                    s_stop = !any;
                }
                __syncthreads();
                if (s_stop) break;
            }
        }
        // ---- write back (CTA 0 of the group) ----
        if (g == 0 && threadIdx.x < k) {
            const ColState &cs = st[threadIdx.x];
            SolveScalars &out = sa.sc[threadIdx.x];
            out.E0 = cs.E0; out.E1 = cs.E1; out.rhat = cs.rhat; out.rho = cs.rho; out.ci = cs.ci;
            out.active = cs.active; out.status = cs.status; out.res_est = cs.res_est; out.bn2 = cs.bn2;
            out.t = t;
        }
    }
finish:
    return;
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
