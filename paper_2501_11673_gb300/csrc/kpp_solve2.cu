// kpp_solve2.cu -- the persistent block-step kernel for small blocks (s <= 256, G^{-1} fits in shared
// memory): one grid barrier per iteration.
//
// Same method and same arithmetic definitions as kpp_solve.cu (K++: Eq. 1.3, 1.4, Alg. 1 / Alg. 5;
// CD++: Eq. 5.1, Alg. 3 with the maintained residual), reorganised for latency:
//   * each CTA keeps its column chunk of x, m (and R_x, R_m) in shared memory for the whole solve;
//   * the block sequence is known in advance (Philox), so the A tile of the next block
//     (A_S[:, chunk], one 2-D TMA box) and its memoised inverse G^{-1} (one bulk copy) are prefetched
//     into double-buffered shared memory one iteration ahead, tracked by mbarriers;
//   * every CTA applies y = G^{-1} r itself (G^{-1} is symmetric, read by columns: conflict-free),
//     so the projection needs no exchange between CTAs;
//   * K++ computes the next block's partial residual A_{S'}[:, chunk] x_{t+1} in the same iteration
//     (double-buffered partials), CD++ publishes its chunk of R_x into a double-buffered copy.
// The one exchange per iteration is a group barrier.  Every wait is bounded.
#include <cuda.h>

#include <cmath>
#include <cstdio>

#include "kpp_internal.cuh"
#include "kpp_runtime.h"
#include "kpp_solve.h"
#include "kpp_solve_device.cuh"

namespace kpp {

struct alignas(128) Sys2 {
    CUtensorMap tmapA;   // A (cols x rows), box {CW, s}
    SysArgs a;           // part: 2 x G x s x KP (K++); Rx: 2 x rows x k (CD++, published copies)
};

struct Smem2 {           // byte offsets into dynamic shared memory
    int tile[2], ginv[2], xc, mc, rxc, rmc, r, y, yp, red, grows, total;
};

// rows of G^{-1} one CTA applies in distributed-y mode: a = g + G * w, w = 0 .. dy_rows-1
__host__ __device__ inline int dy_rows(int s, int G) { return (s + G - 1) / G; }

__host__ __device__ inline int align128(int v) { return (v + 127) / 128 * 128; }

__host__ __device__ inline Smem2 smem2_layout(int s, int64_t CW, int KP, int ta_size, int tc_size, bool dist_y) {
    Smem2 L;
    int o = 0;
    const int tile = align128((int)(s * CW * ta_size));
    const int ginv = dist_y ? 0 : align128(s * s * tc_size);
    const int vec = align128((int)(CW * KP * tc_size));
    L.tile[0] = o; o += tile;
    L.tile[1] = o; o += tile;
    L.ginv[0] = o; o += ginv;
    L.ginv[1] = o; o += ginv;
    L.xc = o; o += vec;
    L.mc = o; o += vec;
    L.rxc = o; o += vec;
    L.rmc = o; o += vec;
    L.r = o; o += align128(s * KP * tc_size);
    L.y = o; o += align128(s * KP * tc_size);
    L.yp = o; o += align128(NT * KP * tc_size);
    L.red = o; o += align128(NW * 32 * KP * tc_size);
    L.grows = o;
    L.total = o;
    return L;
}

__host__ __device__ inline int smem2_total(int s, int64_t CW, int KP, int ta_size, int tc_size, bool dist_y, int G) {
    const Smem2 L = smem2_layout(s, CW, KP, ta_size, tc_size, dist_y);
    return L.total + (dist_y ? align128(dy_rows(s, G) * s * tc_size) : 0);
}

template <typename TA, typename TC, int KP, bool CD, bool DY>
__global__ void __launch_bounds__(NT, 1) solve2_kernel(const Sys2 *__restrict__ systems, Common cm) {
    const Sys2 &sys = systems[blockIdx.x / cm.G];
    const SysArgs sa = sys.a;
    const void *tmap = &sys.tmapA;
    const int g = blockIdx.x % cm.G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = cm.k, s = cm.s, nb = cm.nb;
    const int64_t rows = cm.rows, cols = cm.cols;
    const TC *__restrict__ b = (const TC *)sa.b;
    TC *__restrict__ x = (TC *)sa.x;
    const TC *__restrict__ Ginv = (const TC *)sa.Ginv;

    extern __shared__ __align__(128) unsigned char sm[];
    const Smem2 L = smem2_layout(s, cm.CW, KP, (int)sizeof(TA), (int)sizeof(TC), DY);
    // double buffers addressed by arithmetic (a runtime-indexed pointer array would live in local memory)
    unsigned char *const tile0 = sm + L.tile[0];
    const int tile_stride = L.tile[1] - L.tile[0];
    unsigned char *const ginv0 = sm + L.ginv[0];
    const int ginv_stride = L.ginv[1] - L.ginv[0];
#define TILE(bf) ((TA *)(tile0 + (bf) * tile_stride))
#define GINV(bf) ((TC *)(ginv0 + (bf) * ginv_stride))
    TC *xc = (TC *)(sm + L.xc);
    TC *mc = (TC *)(sm + L.mc);
    TC *rxc = (TC *)(sm + L.rxc);
    TC *rmc = (TC *)(sm + L.rmc);
    TC *s_r = (TC *)(sm + L.r);
    TC *s_y = (TC *)(sm + L.y);
    TC *s_yp = (TC *)(sm + L.yp);
    TC *s_red = (TC *)(sm + L.red);
    TC *s_grows = (TC *)(sm + L.grows);  // distributed y: my rows of G^{-1} for the current step
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ __align__(8) uint64_t mbar_g;
    __shared__ int s_gpending;
    __shared__ unsigned s_gphase;
    __shared__ ColState st[KP];
    __shared__ double s_part[NW * KP];
    __shared__ double s_rn2[KP];
    __shared__ int s_stop, s_need, s_fail;
    __shared__ int s_pending[2];
    __shared__ TC s_beta[KP], s_keep[KP];
    __shared__ unsigned s_phase[2];

    GroupSync gs{sa.bar, sa.err, 0u, (unsigned)cm.G, cm.timeout_ns};
    const int64_t c0 = min64((int64_t)g * cm.CW, cols);
    const int64_t c1 = min64(c0 + cm.CW, cols);
    const int cw = (int)(c1 - c0);
    const int CWs = (int)cm.CW;  // leading dimension of the shared tile
    const int zeta = nb;
    int64_t t = cm.t0_state ? sa.sc[0].t : sa.t0;
    int64_t t_end = cm.t0_state ? t + cm.max_iters : cm.max_iters;
    if (cm.t0_state) {  // a system whose columns are all done does not iterate (t stays put)
        int any = 0;
        for (int c = 0; c < cm.k; ++c) any |= sa.sc[c].active;
        if (!any) t_end = t;
    }
    int ph_c = (int)(t % (2 * (int64_t)zeta));  // t mod 2 zeta, advanced with t (no division per step)
    TC *const Rx0 = (TC *)sa.Rx;  // two published copies of R_x: Rx0 + parity * rows * k
#define RXP(par) (Rx0 + (size_t)(par) * rows * k)

    // ---- set-up ----
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
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init(&mbar_g, 1);
        fence_mbar_init();
        tensormap_acquire(tmap);
        s_pending[0] = s_pending[1] = 0;
        s_phase[0] = s_phase[1] = 0;
        s_gpending = 0;
        s_gphase = 0;
        s_fail = 0;
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
        if (!group_barrier(gs)) goto drain;
        if (threadIdx.x < KP) {
            double tt = 0.0;
            for (int h = 0; h < cm.G; ++h) tt += __ldcg(sa.rpart + (size_t)h * KP + threadIdx.x);
            st[threadIdx.x].bn2 = tt;
        }
        __syncthreads();
        if (!group_barrier(gs)) goto drain;
    }
    if (CD && cm.init_residual) {
        if (!true_residual_phase<TA, TC, KP>(sa, cm, g, gs, st, s_part, RXP(t & 1))) goto drain;
    }
    // chunk state into shared memory
    for (int e = threadIdx.x; e < cw * KP; e += NT) {
        const int cc = e / KP, c = e % KP;
        const size_t gi = (size_t)(c0 + cc) * k + c;
        xc[e] = (c < k) ? __ldcg(x + gi) : (TC)0;
        mc[e] = (TC)0;
        if (CD) {
            rxc[e] = (c < k) ? __ldcg(RXP(t & 1) + gi) : (TC)0;
            rmc[e] = (TC)0;
        }
    }

    {
        // prefetch the A tile and G^{-1} of step tt into buffer bf (thread 0 only)
        auto issue = [&](int64_t tt, int bf) {
            const int j = draw_block(cm.seed, tt, sa.sys_id, nb);
            const int len = (int)min64(s, rows - (int64_t)j * s);
            const unsigned gbytes = DY ? 0u : (unsigned)((len * len * (int)sizeof(TC) + 15) / 16 * 16);
            const int box = s < 256 ? s : 256;
            const int nbox = (s + box - 1) / box;
            const unsigned abytes = (unsigned)(nbox * box * CWs * (int)sizeof(TA));
            mbar_arrive_expect_tx(&mbar[bf], abytes + gbytes);
            for (int q = 0; q < nbox; ++q)
                tma_load_2d(TILE(bf) + (size_t)q * box * CWs, tmap, (int)c0, j * s + q * box, &mbar[bf]);
            if (gbytes) bulk_load(GINV(bf), Ginv + (size_t)j * s * s, gbytes, &mbar[bf]);
            s_pending[bf] = 1;
        };
        // distributed y: bulk-copy my rows a = g + G w of G^{-1}_{j(tt)} (each row len values, padded to 16 B)
        auto issue_rows = [&](int64_t tt) {
            const int j = draw_block(cm.seed, tt, sa.sys_id, nb);
            const int len = (int)min64(s, rows - (int64_t)j * s);
            const unsigned rb = (unsigned)((len * (int)sizeof(TC) + 15) / 16 * 16);
            const unsigned rbs = (unsigned)(s * sizeof(TC));  // row stride in the shared buffer
            int nr = 0;
            for (int a = g; a < len; a += cm.G) ++nr;
            mbar_arrive_expect_tx(&mbar_g, rb * (unsigned)nr);
            int w = 0;
            for (int a = g; a < len; a += cm.G, ++w)
                bulk_load((unsigned char *)s_grows + (size_t)w * rbs, Ginv + (size_t)j * s * s + (size_t)a * len, rb,
                          &mbar_g);
            s_gpending = 1;
        };
        // wait for buffer bf (all threads); false on timeout
        auto wait_buf = [&](int bf) -> bool {
            __syncthreads();
            if (threadIdx.x == 0) {
                if (!mbar_wait_bounded(&mbar[bf], s_phase[bf], cm.timeout_ns)) {
                    s_fail = 1;
                    group_fail(gs, KPP_ERR_TIMEOUT);
                } else {
                    s_phase[bf] ^= 1u;
                    s_pending[bf] = 0;
                }
            }
            __syncthreads();
            return s_fail == 0;
        };
        // K++: partial residual of step tt over my chunk into part[tt % 2][g]
        auto partial = [&](int64_t tt) {
            const int j = draw_block(cm.seed, tt, sa.sys_id, nb);
            const int len = (int)min64(s, rows - (int64_t)j * s);
            const TA *tl = TILE(tt & 1);
            TC *part = (TC *)sa.part + ((size_t)(tt & 1) * cm.G + g) * s * KP;
            for (int a = warp; a < len; a += NW) {
                TC acc[KP];
#pragma unroll
                for (int c = 0; c < KP; ++c) acc[c] = (TC)0;
                for (int cc = lane; cc < cw; cc += 32) {
                    const TC av = conv<TC>(tl[a * CWs + cc]);
#pragma unroll
                    for (int c = 0; c < KP; ++c) acc[c] = tfma<TC>(av, xc[cc * KP + c], acc[c]);
                }
                warp_reduce<TC, KP>(acc);
                if (lane == 0)
#pragma unroll
                    for (int c = 0; c < KP; ++c) part[(size_t)a * KP + c] = acc[c];
            }
        };

        if (threadIdx.x < KP) {
            const double rho = st[threadIdx.x].rho;
            s_beta[threadIdx.x] = (TC)((1.0 - rho) / (1.0 + rho));
            s_keep[threadIdx.x] = (TC)((threadIdx.x < k && st[threadIdx.x].active) ? 1 : 0);
        }
        __syncthreads();
        if (threadIdx.x == 0 && t < t_end) {
            issue(t, (int)(t & 1));
            if (t + 1 < t_end) issue(t + 1, (int)((t + 1) & 1));
            if (DY) issue_rows(t);
        }
        if (!CD && t < t_end) {
            if (!wait_buf((int)(t & 1))) goto drain;
            partial(t);
            if (!group_barrier(gs)) goto drain;
        }

        while (t < t_end) {
            const int bf = (int)(t & 1);
            const int j = draw_block(cm.seed, t, sa.sys_id, nb);
            const int64_t S0 = (int64_t)j * s;
            const int len = (int)min64(s, rows - S0);

            // ---- block residual r ----
            if (!CD) {
                const TC *part = (const TC *)sa.part + (size_t)bf * cm.G * s * KP;
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
                    // warp per entry across the group (lanes over partials, fixed tree), then exchange
                    TC *rbuf = (TC *)sa.rbuf;
                    for (int e = g * NW + warp; e < len * KP; e += cm.G * NW) {
                        const int a = e / KP, c = e % KP;
                        TC v = (TC)0;
                        if (c < k) {
#pragma unroll 8
                            for (int h = lane; h < cm.G; h += 32) v += __ldcg(part + ((size_t)h * s + a) * KP + c);
                        }
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
                    s_r[e] = (c < k) ? __ldcg(RXP(bf) + (S0 + a) * k + c) : (TC)0;
                }
                if (!wait_buf(bf)) break;
            }
            __syncthreads();
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

            // ---- y = G^{-1} r ----
            if (DY) {
                // rows of G^{-1} spread over the group (warp per row), then exchange
                __syncthreads();
                TC *ybuf = (TC *)sa.ybuf;
                if (threadIdx.x == 0) {
                    if (!mbar_wait_bounded(&mbar_g, s_gphase, cm.timeout_ns)) {
                        s_fail = 1;
                        group_fail(gs, KPP_ERR_TIMEOUT);
                    } else {
                        s_gphase ^= 1u;
                        s_gpending = 0;
                    }
                }
                __syncthreads();
                if (s_fail) break;
                int w = warp;
                for (int a = g + cm.G * warp; a < len; a += cm.G * NW, w += NW) {
                    TC acc[KP];
#pragma unroll
                    for (int c = 0; c < KP; ++c) acc[c] = (TC)0;
                    const TC *grow = s_grows + (size_t)w * s;
                    for (int d = lane; d < len; d += 32) {
                        const TC gval = grow[d];
#pragma unroll
                        for (int c = 0; c < KP; ++c) acc[c] = tfma<TC>(gval, s_r[d * KP + c], acc[c]);
                    }
                    warp_reduce<TC, KP>(acc);
                    if (lane == 0)
#pragma unroll
                        for (int c = 0; c < KP; ++c) ybuf[(size_t)a * KP + c] = acc[c];
                }
                __syncthreads();
                if (threadIdx.x == 0 && t + 1 < t_end) issue_rows(t + 1);
                if (!group_barrier(gs)) break;
                for (int e = threadIdx.x; e < len * KP; e += NT) s_y[e] = __ldcg(ybuf + e);
                __syncthreads();
            } else {
                const TC *gv = GINV(bf);
                const int RG = min(NT, (len + 31) / 32 * 32);
                const int Q = NT / RG;
                const int a = threadIdx.x % RG, q = threadIdx.x / RG;
                if (q < Q && a < len) {
                    const int d0 = q * len / Q, d1 = (q + 1) * len / Q;
                    TC acc[KP];
#pragma unroll
                    for (int c = 0; c < KP; ++c) acc[c] = (TC)0;
                    for (int d = d0; d < d1; ++d) {
                        const TC gval = gv[d * len + a];
#pragma unroll
                        for (int c = 0; c < KP; ++c) acc[c] = tfma<TC>(gval, s_r[d * KP + c], acc[c]);
                    }
#pragma unroll
                    for (int c = 0; c < KP; ++c) s_yp[(q * RG + a) * KP + c] = acc[c];
                }
                __syncthreads();
                for (int e = threadIdx.x; e < len * KP; e += NT) {
                    const int aa = e / KP, c = e % KP;
                    TC v = (TC)0;
                    for (int qq = 0; qq < Q; ++qq) v += s_yp[(qq * RG + aa) * KP + c];
                    s_y[e] = v;
                }
                __syncthreads();
            }

            // ---- back-projection and update of my chunk (shared memory) ----
            {
                const TC eta = (TC)cm.eta;
                const TA *tl = TILE(bf);
                for (int cg = 0; cg < cw; cg += 32) {
                    const int cc = cg + lane;
                    TC acc[KP];
#pragma unroll
                    for (int c = 0; c < KP; ++c) acc[c] = (TC)0;
                    if (cc < cw) {
                        for (int a = warp; a < len; a += NW) {
                            const TC av = conv<TC>(tl[a * CWs + cc]);
#pragma unroll
                            for (int c = 0; c < KP; ++c) acc[c] = tfma<TC>(av, s_y[a * KP + c], acc[c]);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < KP; ++c) s_red[(warp * 32 + lane) * KP + c] = acc[c];
                    __syncthreads();
                    for (int e = threadIdx.x; e < 32 * KP; e += NT) {
                        const int ln = e / KP, c = e % KP;
                        const int ccc = cg + ln;
                        if (ccc < cw && c < k && s_keep[c] != (TC)0) {
                            TC u = (TC)0;
#pragma unroll
                            for (int w = 0; w < NW; ++w) u += s_red[(w * 32 + ln) * KP + c];
                            const int li = ccc * KP + c;
                            if (!CD) {
                                const TC mm = s_beta[c] * (mc[li] - u);
                                mc[li] = mm;
                                xc[li] = xc[li] - u + eta * mm;
                            } else {
                                const int64_t col = c0 + ccc;
                                const TC rm = s_beta[c] * (rmc[li] - u);
                                rmc[li] = rm;
                                rxc[li] = rxc[li] - u + eta * rm;
                                const TC wv = (col >= S0 && col < S0 + len) ? s_y[(col - S0) * KP + c] : (TC)0;
                                const TC mm = s_beta[c] * (mc[li] - wv);
                                mc[li] = mm;
                                xc[li] = xc[li] - wv + eta * mm;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            // buffer bf is free: prefetch step t+2 into it
            if (threadIdx.x == 0 && t + 2 < t_end) issue(t + 2, bf);
            const int ph = ph_c;
            const bool ckpt = (ph == 2 * zeta - 1);
            if (CD) {
                // publish my chunk of R_x for the next step; x too at checkpoints
                TC *dst = RXP((t + 1) & 1);
                for (int e = threadIdx.x; e < cw * KP; e += NT) {
                    const int cc = e / KP, c = e % KP;
                    if (c < k) dst[(size_t)(c0 + cc) * k + c] = rxc[e];
                }
            }
            if (ckpt) {
                for (int e = threadIdx.x; e < cw * KP; e += NT) {
                    const int cc = e / KP, c = e % KP;
                    if (c < k) x[(size_t)(c0 + cc) * k + c] = xc[e];
                }
            }
            // ---- residual estimate and checkpoint (identical in every CTA) ----
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
                    if (ckpt) {
                        cs.res_est = cs.bn2 > 0.0 ? sqrt(cs.E1 / cs.bn2) : sqrt(cs.E1);
                        if (cm.tol > 0.0 && cs.E1 <= cm.tol * cm.tol * cs.bn2 && cm.confirm) atomicOr(&s_need, 1);
                    }
                }
            }
            __syncthreads();
            t += 1;
            if (++ph_c == 2 * zeta) ph_c = 0;
            if (!CD) {
                // next block's partial residual from the updated chunk
                if (t < t_end) {
                    if (!wait_buf((int)(t & 1))) break;
                    partial(t);
                }
            }
            if (!group_barrier(gs)) break;
            if (ckpt) {
                if (s_need) {
                    if (!true_residual_phase<TA, TC, KP>(sa, cm, g, gs, st, s_part, CD ? RXP(t & 1) : (TC *)nullptr))
                        break;
                    if (CD) {
                        // the replaced residual becomes my chunk's R_x
                        for (int e = threadIdx.x; e < cw * KP; e += NT) {
                            const int cc = e / KP, c = e % KP;
                            if (c < k) rxc[e] = __ldcg(RXP(t & 1) + (size_t)(c0 + cc) * k + c);
                        }
                    }
                }
                if (threadIdx.x < k && st[threadIdx.x].active) checkpoint_column(st[threadIdx.x], cm, zeta);
                if (threadIdx.x < KP) {
                    const double rho = st[threadIdx.x].rho;
                    s_beta[threadIdx.x] = (TC)((1.0 - rho) / (1.0 + rho));
                    s_keep[threadIdx.x] = (TC)((threadIdx.x < k && st[threadIdx.x].active) ? 1 : 0);
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
    }
drain:
    // write my chunk of x back, wait (bounded) for copies still in flight, report
    __syncthreads();
    for (int e = threadIdx.x; e < cw * KP; e += NT) {
        const int cc = e / KP, c = e % KP;
        if (c < k) x[(size_t)(c0 + cc) * k + c] = xc[e];
    }
    if (threadIdx.x == 0) {
        for (int bf = 0; bf < 2; ++bf)
            if (s_pending[bf]) {
                if (mbar_wait_bounded(&mbar[bf], s_phase[bf], cm.timeout_ns)) s_phase[bf] ^= 1u;
                else group_fail(gs, KPP_ERR_TIMEOUT);
                s_pending[bf] = 0;
            }
        if (DY && s_gpending) {
            if (mbar_wait_bounded(&mbar_g, s_gphase, cm.timeout_ns)) s_gphase ^= 1u;
            else group_fail(gs, KPP_ERR_TIMEOUT);
            s_gpending = 0;
        }
    }
    __syncthreads();
    if (g == 0 && threadIdx.x < k) {
        const ColState &cs = st[threadIdx.x];
        SolveScalars &out = sa.sc[threadIdx.x];
        out.E0 = cs.E0; out.E1 = cs.E1; out.rhat = cs.rhat; out.rho = cs.rho; out.ci = cs.ci;
        out.active = cs.active; out.status = cs.status; out.res_est = cs.res_est; out.bn2 = cs.bn2;
        out.t = t;
    }
#undef TILE
#undef GINV
#undef RXP
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

bool make_tmap_2d(void *out, const void *base, int dtype, uint64_t cols, uint64_t rows, uint64_t ld_elems,
                  uint32_t box_cols, uint32_t box_rows, bool swizzle128) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const size_t es = dtype == KPP_F64 ? 8 : (dtype == KPP_F32 ? 4 : 2);
    CUtensorMapDataType dt = dtype == KPP_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                             : dtype == KPP_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {ld_elems * es};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn((CUtensorMap *)out, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

size_t solve2_smem_bytes(int s, int64_t CW, int KP, int ta_size, int tc_size, bool dist_y, int G) {
    return (size_t)smem2_total(s, CW, KP, ta_size, tc_size, dist_y, G);
}

// G^{-1} double-buffered in shared memory when it fits; otherwise its rows are applied across the group.
static bool solve2_dist_y(int s, int64_t CW, int KP, int es, int tcs) {
    return solve2_smem_bytes(s, CW, KP, es, tcs, false, 1) > 200 * 1024;
}

bool solve2_eligible(const kpp_matrix &A, int s, int64_t CW, int KP, bool f64, bool cd, int G) {
    const int es = A.dtype == KPP_F64 ? 8 : (A.dtype == KPP_F32 ? 4 : 2);
    const int tcs = f64 ? 8 : 4;
    if (s < 2 || s > 1024 || (s & 1) || CW > 256 || CW < 1) return false;
    if (s > 256 && (s % 256)) return false;  // whole 256-row boxes
    if (((uintptr_t)A.data & 15) || ((A.ld * es) & 15) || ((CW * es) & 15)) return false;
    const bool dy = solve2_dist_y(s, CW, KP, es, tcs);
    if (dy && cd) return false;  // CD++ with large blocks stays on the general kernel
    if (solve2_smem_bytes(s, CW, KP, es, tcs, dy, G) > 200 * 1024) return false;
    // rows of G^{-1} are bulk-copied: every row offset must stay 16-byte aligned, so no ragged block
    if (dy && ((s * tcs) % 16 || A.rows % s)) return false;
    return encode_fn() != nullptr;
}

template <typename TA, typename TC, int KP, bool CD>
static cudaError_t launch2_t(const void *d_sys, int nsys, const Common &cm, cudaStream_t st) {
    const bool dy = solve2_dist_y(cm.s, cm.CW, KP, sizeof(TA), sizeof(TC));
    auto kern = dy ? solve2_kernel<TA, TC, KP, CD, true> : solve2_kernel<TA, TC, KP, CD, false>;
    const size_t smem = solve2_smem_bytes(cm.s, cm.CW, KP, sizeof(TA), sizeof(TC), dy, cm.G);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if ((int64_t)per_sm * sm_count() < (int64_t)nsys * cm.G) return cudaErrorCooperativeLaunchTooLarge;
    Common c = cm;
    const Sys2 *p = (const Sys2 *)d_sys;
    void *args[] = {(void *)&p, (void *)&c};
    note_launch();
    return cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)(nsys * cm.G)), dim3(NT), args, smem, st);
}

template <typename TA, typename TC, bool CD>
static cudaError_t launch2_kp(const void *d_sys, int nsys, const Common &cm, int KP, cudaStream_t st) {
    switch (KP) {
        case 1: return launch2_t<TA, TC, 1, CD>(d_sys, nsys, cm, st);
        case 8: return launch2_t<TA, TC, 8, CD>(d_sys, nsys, cm, st);
        case 32: return launch2_t<TA, TC, 32, CD>(d_sys, nsys, cm, st);
        default: return cudaErrorInvalidValue;
    }
}

size_t sys2_bytes() { return sizeof(Sys2); }

void sys2_fill(void *dst_host, const SysArgs &a, const void *tmap) {
    Sys2 *p = (Sys2 *)dst_host;
    memcpy(&p->tmapA, tmap, sizeof(CUtensorMap));
    p->a = a;
}

cudaError_t launch_solve2(int dtype, bool cd, const void *d_sys, int nsys, const Common &cm, int KP,
                          cudaStream_t st) {
    if (dtype == KPP_F64)
        return cd ? launch2_kp<double, double, true>(d_sys, nsys, cm, KP, st)
                  : launch2_kp<double, double, false>(d_sys, nsys, cm, KP, st);
    if (dtype == KPP_F32)
        return cd ? launch2_kp<float, float, true>(d_sys, nsys, cm, KP, st)
                  : launch2_kp<float, float, false>(d_sys, nsys, cm, KP, st);
    return cd ? launch2_kp<__nv_bfloat16, float, true>(d_sys, nsys, cm, KP, st)
              : launch2_kp<__nv_bfloat16, float, false>(d_sys, nsys, cm, KP, st);
}

}  // namespace kpp
