// kpp_solve_group.cuh -- the body of the general persistent solve (Alg. 3 / Alg. 5 with memoised
// factors) as a device function over one group of G CTAs, so that the batched kernel (kpp_solve.cu) and
// the serving loop's slots (kpp_serve.cu) run the same code.
//
// Paper: arXiv 2501.11673.  One call runs every iteration of one system:
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
//     A_S[:, c0:c1] -- for the partial residual warps take rows and lanes take columns (coalesced row
//     segments); for the back-projection a warp takes 32-column groups and each lane its column;
//   * the s x s projection y = G^{-1} r is split by rows across all CTAs (warp per row);
//   * the K++ residual is reduced from per-CTA partial sums in a fixed order (deterministic).
// Every CTA recomputes the scalars (|r|^2, E0, E1, rho) from identical data in an identical order,
// so all CTAs agree on rho and on the stop decision without another exchange.
#pragma once

#include "kpp_internal.cuh"
#include "kpp_solve.h"
#include "kpp_solve_device.cuh"

namespace kpp {

// g: this CTA's rank in the group; gs: the group's barrier (its target carried by the caller).
// Returns when the system's iteration ends (every column stopped, the step cap, or a group error).
// CRMW: the back-projection's read-modify-write goes through shared memory so that it is coalesced (the
// batched kernel); without it each lane updates the k entries of its own column directly, which needs
// fewer registers (the serving loop, which holds six instantiations of this body in one kernel).
template <typename TA, typename TC, int KP, bool CD, bool CRMW = true>
__device__ void solve_group(const SysArgs &sa, const Common &cm, int g, GroupSync &gs) {
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
        if (g == cm.test_hold_cta) return;  // wait test: leave without arriving
        if (!group_barrier(gs)) return;
        if (threadIdx.x < KP) {
            double t = 0.0;
            for (int h = 0; h < cm.G; ++h) t += __ldcg(sa.rpart + (size_t)h * KP + threadIdx.x);
            st[threadIdx.x].bn2 = t;
        }
        __syncthreads();
        if (!group_barrier(gs)) return;
    }
    if (CD && cm.init_residual) {
        if (!true_residual_phase<TA, TC, KP>(sa, cm, g, gs, st, s_part, Rx)) return;
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
            // a warp takes whole 32-column groups of my chunk: each lane sums the len rows of A_S for its
            // column in row order (16 or 32 row loads in flight at a time); the sums then go through the
            // warp's slice of shared memory to the updates, so the phase needs no cross-warp reduction
            // and no block barrier
            for (int64_t cb = c0 + (int64_t)warp * 32; cb < c1; cb += (int64_t)NW * 32) {
                if (!CRMW && cb + lane >= c1) continue;
                const int64_t col = cb + lane < c1 ? cb + lane : c1 - 1;  // lanes past the chunk repeat
                TC acc[KP];                                                 // its last column (unused)
#pragma unroll
                for (int c = 0; c < KP; ++c) acc[c] = (TC)0;
                const TA *ap = A + S0 * lda + col;
                constexpr int RB = (KP * sizeof(TC) <= 32) ? 32 : 16;  // row loads in flight per lane
                int a = 0;
                for (; a + RB <= len; a += RB) {
                    TC av[RB];
#pragma unroll
                    for (int q = 0; q < RB; ++q) av[q] = conv<TC>(ap[(int64_t)(a + q) * lda]);
#pragma unroll
                    for (int q = 0; q < RB; ++q)
#pragma unroll
                        for (int c = 0; c < KP; ++c) acc[c] = tfma<TC>(av[q], s_y[(a + q) * KP + c], acc[c]);
                }
                for (; a < len; ++a) {
                    const TC av = conv<TC>(ap[(int64_t)a * lda]);
#pragma unroll
                    for (int c = 0; c < KP; ++c) acc[c] = tfma<TC>(av, s_y[a * KP + c], acc[c]);
                }
                if (CRMW) {
                    // the lanes then take consecutive (column, right-hand side) entries, so that every
                    // read-modify-write below is coalesced
                    TC *red = s_red + (size_t)warp * 32 * KP;
#pragma unroll
                    for (int c = 0; c < KP; ++c) red[lane * KP + c] = acc[c];
                    __syncwarp();
                    for (int e = lane; e < 32 * k; e += 32) {
                        const int ln = e / k, c = e % k;
                        const int64_t cl = cb + ln;
                        if (cl < c1 && s_keep[c] != (TC)0) {
                            const TC u = red[ln * KP + c];
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
                    __syncwarp();
                } else if (cb + lane < c1) {
#pragma unroll
                    for (int c = 0; c < KP; ++c) {
                        if (c < k && s_keep[c] != (TC)0) {
                            const TC u = acc[c];
                            const size_t idx = (size_t)col * k + c;
                            if (!CD) {
                                const TC mm = s_beta[c] * (__ldcg(mv + idx) - u);
                                mv[idx] = mm;
                                x[idx] = __ldcg(x + idx) - u + eta * mm;
                            } else {
                                const TC rm = s_beta[c] * (__ldcg(Rm + idx) - u);
                                Rm[idx] = rm;
                                Rx[idx] = __ldcg(Rx + idx) - u + eta * rm;
                                const TC wv = (col >= S0 && col < S0 + len) ? s_y[(col - S0) * KP + c] : (TC)0;
                                const TC mm = s_beta[c] * (__ldcg(mv + idx) - wv);
                                mv[idx] = mm;
                                x[idx] = __ldcg(x + idx) - wv + eta * mm;
                            }
                        }
                    }
                }
            }
            // the next step's block is known now (the draw depends only on t): bring its rows of A_S on
            // my columns, the G^{-1} rows of my projection rows and (CD++) its residual rows into L2
            if (t + 1 < t_end) {
                const int jn = draw_block(cm.seed, t + 1, sa.sys_id, nb);
                const int64_t Sn = (int64_t)jn * s;
                const int lenn = (int)min64(s, rows - Sn);
                for (int64_t cb = c0 + (int64_t)warp * 32; cb < c1; cb += (int64_t)NW * 32) {
                    const int64_t col = cb + lane;
                    if (col < c1)
                        for (int a = 0; a < lenn; ++a) prefetch_l2(A + (Sn + a) * lda + col);
                }
                const TC *Gn = Ginv + (size_t)jn * s * s;
                constexpr int LT = 128 / (int)sizeof(TC);  // entries per 128-byte line
                for (int a = g + cm.G * warp; a < lenn; a += cm.G * NW)
                    if (lane * LT < lenn) prefetch_l2(Gn + (size_t)a * lenn + lane * LT);
                if (CD && g == 0)
                    for (int e = threadIdx.x * LT; e < lenn * k; e += NT * LT) prefetch_l2(Rx + Sn * k + e);
            }
            __syncthreads();
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
}


}  // namespace kpp
