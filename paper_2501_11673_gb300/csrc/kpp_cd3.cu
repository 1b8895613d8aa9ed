// kpp_cd3.cu -- CD++ (Eq. 5.1; Alg. 3's loop, maintained residual) as a dataflow kernel.
//
// The only value one step of CD++ needs from other CTAs is r = R_x[S] of the next block, and only the
// CTAs owning the columns of that block produce it.  So instead of a group barrier per step:
//   * the owners of S_{t+1} write r_{t+1} into slot (t+1) mod R of a mailbox ring, each 64-bit word
//     carrying a 32-bit step tag and 32 bits of payload (an FP32 value, or half of an FP64 value);
//     word stores are single-copy atomic, so a word whose tag matches is valid on its own;
//   * every CTA polls slot t mod R until all tags of step t match, then runs the step on its chunk;
//   * a group barrier every P <= R/2 steps bounds how far CTAs drift apart, so a slot is never
//     rewritten while a slow CTA may still read it; checkpoints that need the true residual use
//     the cooperative FP64 residual phase (with barriers) as in the other kernels.
// FP64 (USE_W): the factor phase memoised W_j = G_j^{-1} A_{S_j}; a step streams the W tile of its chunk
// and computes u = W_S^T r directly (A_{:,S} G^{-1} r, A symmetric), with no s x s solve on the critical
// path.  Only the CTAs owning the columns of S apply G^{-1} to their rows, for the x and m update.
// FP32 inner solves (!USE_W): every CTA applies G^{-1} (cheap in FP32) and streams the A tile.
// Tiles and G^{-1} rows are prefetched one step ahead with TMA into double-buffered shared memory.
#include <cuda.h>

#include <cmath>
#include <cstdio>

#include "kpp_internal.cuh"
#include "kpp_runtime.h"
#include "kpp_solve.h"
#include "kpp_solve_device.cuh"

namespace kpp {

constexpr int CD3_RING = 64;     // mailbox slots
constexpr int CD3_PERIOD = 32;   // steps between group barriers (<= CD3_RING / 2)

struct alignas(128) Sys3 {
    CUtensorMap tmapT;           // tile source (W for USE_W, else A): cols x rows, box {CW, s}
    SysArgs a;                   // Rx: rows x k (single copy); part/rbuf/ybuf unused
    unsigned long long *mail;    // CD3_RING x s x KP x (words per value)
};

template <typename TC> struct MailWords;
template <> struct MailWords<double> { static constexpr int n = 2; };
template <> struct MailWords<float> { static constexpr int n = 1; };

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void mail_put(unsigned long long *w, double v, unsigned tag) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    st_relaxed_u64(w, ((unsigned long long)tag << 32) | (bits & 0xffffffffull));
    st_relaxed_u64(w + 1, ((unsigned long long)tag << 32) | (bits >> 32));
}
__device__ __forceinline__ void mail_put(unsigned long long *w, float v, unsigned tag) {
    st_relaxed_u64(w, ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v));
}
// returns true once the value of step `tag` is present
__device__ __forceinline__ bool mail_get(const unsigned long long *w, unsigned tag, double &v) {
    const unsigned long long lo = ld_relaxed_u64(w), hi = ld_relaxed_u64(w + 1);
    if ((unsigned)(lo >> 32) != tag || (unsigned)(hi >> 32) != tag) return false;
    v = __longlong_as_double((long long)(((hi & 0xffffffffull) << 32) | (lo & 0xffffffffull)));
    return true;
}
__device__ __forceinline__ bool mail_get(const unsigned long long *w, unsigned tag, float &v) {
    const unsigned long long x = ld_relaxed_u64(w);
    if ((unsigned)(x >> 32) != tag) return false;
    v = __uint_as_float((unsigned)x);
    return true;
}

struct Smem3 {
    int tile[2], ginv[2], xc, mc, rxc, rmc, r, y, yp, red, total;
};

__host__ __device__ inline Smem3 smem3_layout(int s, int64_t CW, int KP, int ta_size, int tc_size, bool use_w) {
    auto al = [](int v) { return (v + 127) / 128 * 128; };
    Smem3 L;
    int o = 0;
    const int tile = al((int)(s * CW * ta_size));
    // W path: only the G^{-1} rows of my chunk (at most CW rows); else the whole G^{-1}
    const int ginv = al((use_w ? (int)min64(CW + 2, s) : s) * s * tc_size);
    const int vec = al((int)(CW * KP * tc_size));
    L.tile[0] = o; o += tile;
    L.tile[1] = o; o += tile;
    L.ginv[0] = o; o += ginv;
    L.ginv[1] = o; o += ginv;
    L.xc = o; o += vec;
    L.mc = o; o += vec;
    L.rxc = o; o += vec;
    L.rmc = o; o += vec;
    L.r = o; o += al(s * KP * tc_size);
    L.y = o; o += al(s * KP * tc_size);
    L.yp = o; o += al(NT * KP * tc_size);
    L.red = o; o += al(NW * 32 * KP * tc_size);
    L.total = o;
    return L;
}

template <typename TA, typename TC, int KP, bool USE_W>
__global__ void __launch_bounds__(NT, 1) cd3_kernel(const Sys3 *__restrict__ systems, Common cm) {
    constexpr int MW = MailWords<TC>::n;
    const Sys3 &sys = systems[blockIdx.x / cm.G];
    const SysArgs sa = sys.a;
    const void *tmap = &sys.tmapT;
    unsigned long long *mail = sys.mail;
    const int g = blockIdx.x % cm.G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = cm.k, s = cm.s, nb = cm.nb;
    const int64_t n = cm.rows;
    const TC *__restrict__ b = (const TC *)sa.b;
    TC *__restrict__ x = (TC *)sa.x;
    TC *__restrict__ Rx = (TC *)sa.Rx;
    const TC *__restrict__ Ginv = (const TC *)sa.Ginv;

    extern __shared__ __align__(128) unsigned char sm[];
    const Smem3 L = smem3_layout(s, cm.CW, KP, (int)sizeof(TA), (int)sizeof(TC), USE_W);
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
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ ColState st[KP];
    __shared__ double s_part[NW * KP];
    __shared__ double s_rn2[KP];
    __shared__ int s_stop, s_need, s_fail;
    __shared__ int s_pending[2], s_glo[2];  // (shared: indexed by the runtime buffer number)
    __shared__ unsigned s_phase[2];
    __shared__ TC s_beta[KP], s_keep[KP];

    GroupSync gs{sa.bar, sa.err, 0u, (unsigned)cm.G, cm.timeout_ns};
    const int64_t c0 = min64((int64_t)g * cm.CW, n);
    const int64_t c1 = min64(c0 + cm.CW, n);
    const int cw = (int)(c1 - c0);
    const int CWs = (int)cm.CW;
    const int zeta = nb;
    int64_t t = cm.t0_state ? sa.sc[0].t : sa.t0;
    int64_t t_end = cm.t0_state ? t + cm.max_iters : cm.max_iters;
    if (cm.t0_state) {  // a system whose columns are all done does not iterate (t stays put)
        int any = 0;
        for (int c = 0; c < cm.k; ++c) any |= sa.sc[c].active;
        if (!any) t_end = t;
    }

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
        fence_mbar_init();
        tensormap_acquire(tmap);
        s_pending[0] = s_pending[1] = 0;
        s_phase[0] = s_phase[1] = 0;
        s_fail = 0;
    }
    {
        double acc[KP];
#pragma unroll
        for (int c = 0; c < KP; ++c) acc[c] = 0.0;
        for (int64_t i = (int64_t)g * NT + threadIdx.x; i < n; i += (int64_t)cm.G * NT)
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
    if (cm.init_residual) {
        if (!true_residual_phase<TA, TC, KP>(sa, cm, g, gs, st, s_part, Rx)) goto drain;
    }
    for (int e = threadIdx.x; e < cw * KP; e += NT) {
        const int cc = e / KP, c = e % KP;
        const size_t gi = (size_t)(c0 + cc) * k + c;
        xc[e] = (c < k) ? __ldcg(x + gi) : (TC)0;
        mc[e] = (TC)0;
        rxc[e] = (c < k) ? __ldcg(Rx + gi) : (TC)0;
        rmc[e] = (TC)0;
    }
    if (threadIdx.x < KP) {
        const double rho = st[threadIdx.x].rho;
        s_beta[threadIdx.x] = (TC)((1.0 - rho) / (1.0 + rho));
        s_keep[threadIdx.x] = (TC)((threadIdx.x < k && st[threadIdx.x].active) ? 1 : 0);
    }
    __syncthreads();

    {
        // prefetch of step tt into buffer bf: the tile of my chunk, and G^{-1} (all of it, or only
        // the rows of my chunk that fall in the block on the W path)
        auto issue = [&](int64_t tt, int bf) {
            const int j = draw_block(cm.seed, tt, sa.sys_id, nb);
            const int64_t S0 = (int64_t)j * s;
            const int len = (int)min64(s, n - S0);
            const unsigned abytes = (unsigned)(s * CWs * (int)sizeof(TA));
            int glo = 0, ghi = len;
            if (USE_W) {
                glo = (int)max64(0, c0 - S0);
                ghi = (int)min64(len, c1 - S0);
                if (ghi < glo) ghi = glo;
                if (len & 1) glo &= ~1;  // keep the copy's source 16-byte aligned (row offset even)
            }
            const unsigned gbytes = (unsigned)(((ghi - glo) * len * (int)sizeof(TC) + 15) / 16 * 16);
            mbar_arrive_expect_tx(&mbar[bf], abytes + gbytes);
            tma_load_2d(TILE(bf), tmap, (int)c0, (int)S0, &mbar[bf]);
            if (gbytes) bulk_load(GINV(bf), Ginv + (size_t)j * s * s + (size_t)glo * len, gbytes, &mbar[bf]);
            s_glo[bf] = glo;
            s_pending[bf] = 1;
        };
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
        // publish my part of r_tt = R_x[S_tt] (tag tt + 1) into slot tt mod R
        auto publish = [&](int64_t tt) {
            const int j = draw_block(cm.seed, tt, sa.sys_id, nb);
            const int64_t S0 = (int64_t)j * s;
            const int len = (int)min64(s, n - S0);
            const int64_t lo = max64(c0, S0), hi = min64(c1, S0 + len);
            unsigned long long *slot = mail + (size_t)(tt % CD3_RING) * s * KP * MW;
            const unsigned tag = (unsigned)(tt + 1);
            for (int e = threadIdx.x; e < (int)(hi - lo) * KP; e += NT) {
                const int ii = e / KP, c = e % KP;
                const int64_t col = lo + ii;
                mail_put(slot + ((size_t)(col - S0) * KP + c) * MW, rxc[(col - c0) * KP + c], tag);
            }
        };

        if (threadIdx.x == 0 && t < t_end) {
            issue(t, (int)(t & 1));
            if (t + 1 < t_end) issue(t + 1, (int)((t + 1) & 1));
        }
        if (t < t_end) publish(t);

        while (t < t_end) {
            const int bf = (int)(t & 1);
            const int j = draw_block(cm.seed, t, sa.sys_id, nb);
            const int64_t S0 = (int64_t)j * s;
            const int len = (int)min64(s, n - S0);

            // ---- gather r_t from the mailbox (bounded polling) ----
            {
                const unsigned long long *slot = mail + (size_t)(t % CD3_RING) * s * KP * MW;
                const unsigned tag = (unsigned)(t + 1);
                for (int e = threadIdx.x; e < len * KP; e += NT) {
                    const int c = e % KP;
                    TC v = (TC)0;
                    if (c < k) {
                        if (!mail_get(slot + (size_t)e * MW, tag, v)) {
                            const uint64_t t0 = globaltimer_ns();
                            unsigned polls = 0;
                            while (!mail_get(slot + (size_t)e * MW, tag, v)) {
                                if ((++polls & 63u) == 0u) {
                                    if (globaltimer_ns() - t0 > cm.timeout_ns) {
                                        s_fail = 1;
                                        group_fail(gs, KPP_ERR_TIMEOUT);
                                        break;
                                    }
                                    if (*(volatile int *)gs.err != 0) {  // another CTA failed
                                        s_fail = 1;
                                        break;
                                    }
                                }
                            }
                        }
                    }
                    s_r[e] = v;
                }
            }
            if (!wait_buf(bf)) break;
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

            // ---- y = G^{-1} r: all of it (FP32 path), or only my chunk's rows of the block (W path) ----
            const int64_t olo = max64(c0, S0), ohi = min64(c1, S0 + len);  // my columns inside S
            {
                const TC *gv = GINV(bf);
                if (!USE_W) {
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
                } else if (ohi > olo) {
                    // rows (olo - S0) .. (ohi - S0) of G^{-1}, stored from row s_glo[bf]: warp per row
                    const int glo = s_glo[bf];
                    for (int ri = (int)(olo - S0) + warp; ri < (int)(ohi - S0); ri += NW) {
                        TC acc[KP];
#pragma unroll
                        for (int c = 0; c < KP; ++c) acc[c] = (TC)0;
                        const TC *grow = gv + (size_t)(ri - glo) * len;
                        for (int d = lane; d < len; d += 32) {
                            const TC gval = grow[d];
#pragma unroll
                            for (int c = 0; c < KP; ++c) acc[c] = tfma<TC>(gval, s_r[d * KP + c], acc[c]);
                        }
                        warp_reduce<TC, KP>(acc);
                        if (lane == 0)
#pragma unroll
                            for (int c = 0; c < KP; ++c) s_y[ri * KP + c] = acc[c];
                    }
                }
                __syncthreads();
            }

            // ---- u on my chunk: W tile^T r (W path) or A tile^T y; update the chunk state ----
            {
                const TC eta = (TC)cm.eta;
                const TA *tl = TILE(bf);
                const TC *vin = USE_W ? s_r : s_y;
                for (int cg = 0; cg < cw; cg += 32) {
                    const int cc = cg + lane;
                    TC acc[KP];
#pragma unroll
                    for (int c = 0; c < KP; ++c) acc[c] = (TC)0;
                    if (cc < cw) {
                        for (int a = warp; a < len; a += NW) {
                            const TC av = conv<TC>(tl[a * CWs + cc]);
#pragma unroll
                            for (int c = 0; c < KP; ++c) acc[c] = tfma<TC>(av, vin[a * KP + c], acc[c]);
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
                    __syncthreads();
                }
            }
            if (threadIdx.x == 0 && t + 2 < t_end) issue(t + 2, bf);
            // hand r_{t+1} to the other CTAs as early as possible
            if (t + 1 < t_end) publish(t + 1);

            const int64_t ph = t % (2 * (int64_t)zeta);
            const bool ckpt = (ph == 2 * zeta - 1);
            if (ckpt) {
                for (int e = threadIdx.x; e < cw * KP; e += NT) {
                    const int cc = e / KP, c = e % KP;
                    if (c < k) x[(size_t)(c0 + cc) * k + c] = xc[e];
                }
            }
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
            if (ckpt) {
                if (s_need) {
                    if (!group_barrier(gs)) break;  // x complete in every chunk
                    // true residual; it also replaces R_x (the rows of my chunk are re-read below)
                    if (!true_residual_phase<TA, TC, KP>(sa, cm, g, gs, st, s_part, Rx)) break;
                    for (int e = threadIdx.x; e < cw * KP; e += NT) {
                        const int cc = e / KP, c = e % KP;
                        if (c < k) rxc[e] = __ldcg(Rx + (size_t)(c0 + cc) * k + c);
                    }
                    __syncthreads();
                    // republish r_t (already published from the old R_x) and let everyone see it
                    if (t < t_end) publish(t);
                    if (!group_barrier(gs)) break;
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
            // bound the drift between CTAs (mailbox slots are reused every CD3_RING steps)
            if ((t % CD3_PERIOD) == 0) {
                if (!group_barrier(gs)) break;
            }
        }
    }
drain:
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
}

// ---------------------------------------------------------------------------------------------
// cd4_kernel: the FP64 dataflow step for one right-hand side, scheduled for an FP64 pipe that
// issues a warp instruction every ~64 cycles per SMSP.
//
// Same dataflow and memo as cd3_kernel (owners of S_{t+1} hand r_{t+1} = R_x[S_{t+1}] over through
// the mailbox; u = W_S^T r with W = G^{-1} A_S memoised), but every FP64 instruction is placed so
// that the four SMSPs share the work and the owners' critical path carries nothing else:
//   * u = W_S^T r by warps 0-3 (one per SMSP, 16 rows each, two accumulation chains), then warp 0
//     alone (after a barrier of warps 0-3) updates R_m / R_x and writes r_{t+1} into the mailbox
//     straight from registers;
//   * warps 4-7 at the same time: y = G^{-1} r on the owners' rows of S_t (rows by lanes, the block
//     dimension split over the four warps; G^{-1} is symmetric, so its stored rows are the columns
//     needed), then warp 4 updates x and m (after a barrier of warps 4-7) and warp 5 prefetches;
//   * |r|^2 of each step is summed only by the CTAs that publish it (over their rows), and the
//     window sums E0 / E1 are reduced over the group at the checkpoints;
//   * block draws come from a table filled 64 steps ahead; tiles are triple-buffered and r double-
//     buffered so that one __syncthreads per step orders everything.
// Requirements (checked by the host): FP64 storage with W, k = 1, column chunk <= 32, 2 <= s <= 64.
// ---------------------------------------------------------------------------------------------
constexpr int CD4_RING = 128;    // mailbox slots (steps)
constexpr int CD4_PERIOD = 64;   // steps between drift-bounding group barriers (<= CD4_RING / 2)
constexpr int CD4_CW = 32;       // columns per CTA at most
constexpr int CD4_S = 64;        // block size at most
constexpr int CD4_JT = 128;      // block-draw table (steps)
constexpr int CD4_NB = 3;        // tile buffers (prefetch distance 2)

struct Smem4 {
    int tile[CD4_NB], ginv[CD4_NB], total;
};

__host__ __device__ inline Smem4 smem4_layout(int s, int64_t CW, int es) {
    auto al = [](int v) { return (v + 127) / 128 * 128; };
    Smem4 L;
    int o = 0;
    const int tile = al((int)(s * CW * es));
    const int ginv = al((int)min64(CW + 4, s) * s * es);  // my rows of G^-1 (start rounded down by <= 3)
    for (int i = 0; i < CD4_NB; ++i) {
        L.tile[i] = o;
        o += tile;
    }
    for (int i = 0; i < CD4_NB; ++i) {
        L.ginv[i] = o;
        o += ginv;
    }
    L.total = o;
    return L;
}

__device__ __forceinline__ void named_barrier(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

template <typename TA, typename TC>
__global__ void __launch_bounds__(NT, 1) cd4_kernel(const Sys3 *__restrict__ systems, Common cm) {
    constexpr int MW = MailWords<TC>::n;  // mailbox words per value
    const Sys3 &sys = systems[blockIdx.x / cm.G];
    const SysArgs sa = sys.a;
    const void *tmap = &sys.tmapT;
    unsigned long long *mail = sys.mail;
    const int g = blockIdx.x % cm.G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = cm.s, nb = cm.nb;
    const int64_t n = cm.rows;
    const TC *__restrict__ b = (const TC *)sa.b;
    TC *__restrict__ x = (TC *)sa.x;
    TC *__restrict__ Rx = (TC *)sa.Rx;
    const TC *__restrict__ Ginv = (const TC *)sa.Ginv;
    double *__restrict__ xpart = (double *)sa.part;  // G x 2: window-sum partials at checkpoints

    extern __shared__ __align__(128) unsigned char sm[];
    const Smem4 L = smem4_layout(s, cm.CW, (int)sizeof(TC));
    unsigned char *const tile0 = sm + L.tile[0];
    const int tile_stride = L.tile[1] - L.tile[0];
    unsigned char *const ginv0 = sm + L.ginv[0];
    const int ginv_stride = L.ginv[1] - L.ginv[0];
#define TILE4(bf) ((const TC *)(tile0 + (bf) * tile_stride))
#define GINV4(bf) ((const TC *)(ginv0 + (bf) * ginv_stride))
    __shared__ TC s_r[2][CD4_S];
    __shared__ TC s_red[4][CD4_CW], s_yred[4][CD4_CW];
    __shared__ TC xc[CD4_CW], mc[CD4_CW], rxc[CD4_CW], rmc[CD4_CW];
    __shared__ int s_jt[CD4_JT];
    __shared__ double s_epart[2][2];   // my partial window sums, by checkpoint-pair parity
    __shared__ double s_pend;          // |r|^2 over the rows I published last, not yet counted
    __shared__ __align__(8) uint64_t mbar[CD4_NB];
    __shared__ ColState st[1];
    __shared__ double s_part[NW];
    __shared__ int s_stop, s_need, s_fail, s_pending[CD4_NB], s_glo[CD4_NB];
    __shared__ unsigned s_phase[CD4_NB];
    __shared__ TC s_beta;

    GroupSync gs{sa.bar, sa.err, 0u, (unsigned)cm.G, cm.timeout_ns};
    const int64_t c0 = min64((int64_t)g * cm.CW, n);
    const int64_t c1 = min64(c0 + cm.CW, n);
    const int cw = (int)(c1 - c0);
    const int CWs = (int)cm.CW;
    const int zeta = nb;
    const int64_t t_begin = cm.t0_state ? sa.sc[0].t : sa.t0;
    int64_t t = t_begin;
    int64_t t_end = cm.t0_state ? t + cm.max_iters : cm.max_iters;
    if (cm.t0_state && !sa.sc[0].active) t_end = t;
    // running step counters (no 64-bit division in the loop)
    int ph = (int)(t % (2 * (int64_t)zeta));                 // t mod 2 zeta
    int pair = (int)((t / (2 * (int64_t)zeta)) & 1);        // parity of the checkpoint pair of t
    int since = 0;                                           // (t - t_begin) mod 64
    int per = (int)(t % CD4_PERIOD);                         // t mod CD4_PERIOD
    int buf = (int)(t % CD4_NB);                             // tile buffer of step t

    if (threadIdx.x == 0) {
        ColState cs = {};
        const SolveScalars &in = sa.sc[0];
        cs.E0 = in.E0; cs.E1 = in.E1; cs.rhat = in.rhat; cs.rho = in.rho; cs.ci = in.ci;
        cs.active = in.active; cs.status = in.status;
        cs.res_true = NAN;
        cs.res_est = NAN;
        st[0] = cs;
        for (int i = 0; i < CD4_NB; ++i) {
            mbar_init(&mbar[i], 1);
            s_pending[i] = 0;
            s_phase[i] = 0;
        }
        fence_mbar_init();
        tensormap_acquire(tmap);
        s_fail = 0;
        s_epart[0][0] = s_epart[0][1] = s_epart[1][0] = s_epart[1][1] = 0.0;
        s_pend = 0.0;
    }
    for (int e = threadIdx.x; e < CD4_JT; e += NT) {  // draws of steps t_begin .. t_begin + JT - 1
        const int64_t tt = t_begin + e;
        s_jt[tt % CD4_JT] = draw_block(cm.seed, tt, sa.sys_id, nb);
    }
    {
        // |b|^2 over the group (fixed order)
        double acc = 0.0;
        for (int64_t i = (int64_t)g * NT + threadIdx.x; i < n; i += (int64_t)cm.G * NT)
            acc += (double)b[i] * (double)b[i];
        __syncthreads();
        const double v = block_sum<NT>(acc, s_part);
        if (threadIdx.x == 0) sa.rpart[g] = v;
        if (!group_barrier(gs)) goto drain;
        if (threadIdx.x == 0) {
            double tt = 0.0;
            for (int h = 0; h < cm.G; ++h) tt += __ldcg(sa.rpart + h);
            st[0].bn2 = tt;
        }
        __syncthreads();
        if (!group_barrier(gs)) goto drain;
    }
    if (cm.init_residual) {
        if (!true_residual_phase<TA, TC, 1>(sa, cm, g, gs, st, s_part, Rx)) goto drain;
    }
    for (int e = threadIdx.x; e < cw; e += NT) {
        xc[e] = __ldcg(x + c0 + e);
        mc[e] = (TC)0;
        rxc[e] = __ldcg(Rx + c0 + e);
        rmc[e] = (TC)0;
    }
    if (threadIdx.x == 0) {
        const double rho = st[0].rho;
        s_beta = (TC)((1.0 - rho) / (1.0 + rho));
    }
    __syncthreads();

    {
        // prefetch of step tt into buffer bf: my chunk's W tile, and the G^{-1} rows of my chunk
        // that fall inside the block (symmetric: they are also the columns y needs)
        auto issue = [&](int64_t tt, int bf) {
            const int j = s_jt[tt % CD4_JT];
            const int64_t S0 = (int64_t)j * s;
            const int len = (int)min64(s, n - S0);
            const unsigned abytes = (unsigned)(s * CWs * sizeof(TC));
            int glo = (int)max64(0, c0 - S0);
            int ghi = (int)min64(len, c1 - S0);
            if (ghi < glo) ghi = glo;
            {
                // 16-byte aligned source: glo * len a multiple of ea = 16 / sizeof(TC) elements, so glo
                // is rounded down to a multiple of ea / gcd(len, ea) (at most 3 rows below my first)
                constexpr int ea = 16 / (int)sizeof(TC);
                int gc = ea;
                while (len % gc) gc >>= 1;
                const int step = ea / gc;
                glo = glo / step * step;
            }
            const unsigned gbytes = (unsigned)(((ghi - glo) * len * (int)sizeof(TC) + 15) / 16 * 16);
            mbar_arrive_expect_tx(&mbar[bf], abytes + gbytes);
            tma_load_2d((void *)TILE4(bf), tmap, (int)c0, (int)S0, &mbar[bf]);
            if (gbytes) bulk_load((void *)GINV4(bf), Ginv + (size_t)j * s * s + (size_t)glo * len, gbytes, &mbar[bf]);
            s_glo[bf] = glo;
            s_pending[bf] = 1;
        };
        // warp 0: publish my rows of r_tt (values in lanes) and note their |.|^2
        auto publish_lanes = [&](int64_t tt, TC v_lane) {
            const int j = s_jt[tt % CD4_JT];
            const int64_t S0 = (int64_t)j * s;
            const int len = (int)min64(s, n - S0);
            const int64_t col = c0 + lane;
            const bool mine = lane < cw && col >= S0 && col < S0 + len;
            unsigned long long *slot = mail + (size_t)(tt % CD4_RING) * s * MW;
            if (mine) mail_put(slot + (size_t)(col - S0) * MW, v_lane, (unsigned)(tt + 1));
            TC q = mine ? v_lane * v_lane : (TC)0;
            if (__any_sync(0xffffffffu, mine)) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
                if (lane == 0) s_pend = (double)q;
            } else if (lane == 0) {
                s_pend = 0.0;
            }
        };

        if (threadIdx.x == 0 && t < t_end) {
            issue(t, (int)(t % CD4_NB));
            if (t + 1 < t_end) issue(t + 1, (int)((t + 1) % CD4_NB));
        }
        if (warp == 0 && t < t_end) publish_lanes(t, lane < cw ? rxc[lane] : (TC)0);
        __syncthreads();

        while (t < t_end) {
            const int bf = buf;
            const int rb = (int)(t & 1);
            const int j = s_jt[t % CD4_JT];
            const int64_t S0 = (int64_t)j * s;
            const int len = (int)min64(s, n - S0);

            // ---- count |r_t|^2 of the rows I published (the writer of s_pend is thread 0 too);
            //      gather r_t; wait for the tiles ----
            if (threadIdx.x == 0) {
                s_epart[pair][ph < zeta ? 0 : 1] += s_pend;
                s_pend = 0.0;
            }
            if (threadIdx.x < len) {
                const unsigned long long *slot = mail + (size_t)(t % CD4_RING) * s * MW;
                const unsigned tag = (unsigned)(t + 1);
                TC v;
                if (!mail_get(slot + (size_t)threadIdx.x * MW, tag, v)) {
                    const uint64_t tq = globaltimer_ns();
                    unsigned polls = 0;
                    while (!mail_get(slot + (size_t)threadIdx.x * MW, tag, v)) {
                        if ((++polls & 63u) == 0u) {
                            if (globaltimer_ns() - tq > cm.timeout_ns) {
                                s_fail = 1;
                                group_fail(gs, KPP_ERR_TIMEOUT);
                                v = (TC)0;
                                break;
                            }
                            if (*(volatile int *)gs.err != 0) {
                                s_fail = 1;
                                v = (TC)0;
                                break;
                            }
                        }
                    }
                }
                s_r[rb][threadIdx.x] = v;
            } else if (threadIdx.x < CD4_S) {
                s_r[rb][threadIdx.x] = (TC)0;
            }
            if (threadIdx.x == 64) {
                if (!mbar_wait_bounded(&mbar[bf], s_phase[bf], cm.timeout_ns)) {
                    s_fail = 1;
                    group_fail(gs, KPP_ERR_TIMEOUT);
                } else {
                    s_phase[bf] ^= 1u;
                    s_pending[bf] = 0;
                }
            }
            __syncthreads();  // (A): r_t, the tiles of step t; every warp is done with step t - 1
            if (s_fail) break;

            const int64_t olo = max64(c0, S0), ohi = min64(c1, S0 + len);  // my columns inside S_t
            const TC *rv = s_r[rb];
            if (warp < 4) {
                // u partial: rows [16 warp, 16 warp + 16) of the W tile, lane = column, two chains
                const TC *tl = TILE4(bf);
                TC acc0 = (TC)0, acc1 = (TC)0;
                if (lane < cw) {
                    const int a0 = warp * 16, a1 = min(len, a0 + 16);
                    int a = a0;
                    for (; a + 1 < a1; a += 2) {
                        acc0 = tfma<TC>(tl[a * CWs + lane], rv[a], acc0);
                        acc1 = tfma<TC>(tl[(a + 1) * CWs + lane], rv[a + 1], acc1);
                    }
                    if (a < a1) acc0 = tfma<TC>(tl[a * CWs + lane], rv[a], acc0);
                }
                s_red[warp][lane] = acc0 + acc1;
                named_barrier(1, 128);
                if (warp == 0) {
                    // u, then R_m and R_x on my columns; hand r_{t+1} over at once
                    TC rx = (TC)0;
                    if (lane < cw) {
                        const TC u = (s_red[0][lane] + s_red[1][lane]) + (s_red[2][lane] + s_red[3][lane]);
                        const TC rm = s_beta * (rmc[lane] - u);
                        rmc[lane] = rm;
                        rx = rxc[lane] - u + (TC)cm.eta * rm;
                        rxc[lane] = rx;
                    }
                    if (t + 1 < t_end) publish_lanes(t + 1, rx);
                } else if (warp == 3 && since == 0 && t > t_begin) {
                    // refill the draw table 64 steps ahead (the slots of steps t - 64 .. t - 1)
                    for (int e = lane; e < 64; e += 32) {
                        const int64_t tt = t + 64 + e;
                        s_jt[tt % CD4_JT] = draw_block(cm.seed, tt, sa.sys_id, nb);
                    }
                }
            } else {
                if (warp == 5 && lane == 0 && t + 2 < t_end) {
                    // the buffer of step t + 2 was last read at step t - 1, before (A)
                    int b2 = bf + 2;
                    if (b2 >= CD4_NB) b2 -= CD4_NB;
                    issue(t + 2, b2);
                }
                const int q = warp - 4;
                if (ohi > olo) {
                    // y on my rows of S_t: lane = row (olo - S0 + lane), block index split over warps 4-7
                    const int rr = (int)(olo - S0) + lane;  // row of G^{-1} in the block
                    const int glo = s_glo[bf];
                    TC acc = (TC)0;
                    if (lane < (int)(ohi - olo)) {
                        const TC *grow = GINV4(bf) + (size_t)(rr - glo) * len;
                        const int d0 = q * len / 4, d1 = (q + 1) * len / 4;
                        const int span = d1 - d0;
                        // rotate the start so that lanes (stride len) hit different banks
                        for (int i = 0; i < span; ++i) {
                            int d = d0 + ((i + lane) % span);
                            acc = tfma<TC>(grow[d], rv[d], acc);
                        }
                    }
                    s_yred[q][lane] = acc;
                }
                named_barrier(2, 128);
                if (warp == 4) {
                    // x and m on my columns: w = y on the columns inside S_t
                    if (lane < cw) {
                        const int64_t col = c0 + lane;
                        TC wv = (TC)0;
                        if (col >= olo && col < ohi) {
                            const int l = (int)(col - olo);
                            wv = (s_yred[0][l] + s_yred[1][l]) + (s_yred[2][l] + s_yred[3][l]);
                        }
                        const TC mm = s_beta * (mc[lane] - wv);
                        mc[lane] = mm;
                        xc[lane] = xc[lane] - wv + (TC)cm.eta * mm;
                    }
                }
            }

            const bool ckpt = (ph == 2 * zeta - 1);
            t += 1;
            if (++ph == 2 * zeta) {
                ph = 0;
                pair ^= 1;
            }
            if (++since == 64) since = 0;
            if (++per == CD4_PERIOD) per = 0;
            if (++buf == CD4_NB) buf = 0;
            if (ckpt) {
                // window sums of the finished pair over the group, then the checkpoint of Alg. 3
                __syncthreads();
                if (threadIdx.x == 0) {
                    const int pr = pair ^ 1;  // the pair that just ended
                    xpart[(size_t)g * 2 + 0] = s_epart[pr][0];
                    xpart[(size_t)g * 2 + 1] = s_epart[pr][1];
                    s_epart[pr][0] = s_epart[pr][1] = 0.0;
                }
                for (int e = threadIdx.x; e < cw; e += NT) x[c0 + e] = xc[e];
                if (!group_barrier(gs)) break;
                if (threadIdx.x == 0) {
                    double e0 = 0.0, e1 = 0.0;
                    for (int h = 0; h < cm.G; ++h) {
                        e0 += __ldcg(xpart + (size_t)h * 2 + 0);
                        e1 += __ldcg(xpart + (size_t)h * 2 + 1);
                    }
                    ColState &cs = st[0];
                    cs.E0 += e0;
                    cs.E1 += e1;
                    cs.res_est = cs.bn2 > 0.0 ? sqrt(cs.E1 / cs.bn2) : sqrt(cs.E1);
                    s_need = (cm.tol > 0.0 && cs.E1 <= cm.tol * cm.tol * cs.bn2 && cm.confirm) ? 1 : 0;
                }
                __syncthreads();
                if (s_need) {
                    // true residual; it also replaces R_x (my rows are re-read below)
                    if (!true_residual_phase<TA, TC, 1>(sa, cm, g, gs, st, s_part, Rx)) break;
                    for (int e = threadIdx.x; e < cw; e += NT) rxc[e] = __ldcg(Rx + c0 + e);
                    __syncthreads();
                    // republish r_t from the new R_x (its |.|^2 replaces the pending one)
                    if (warp == 0 && t < t_end) publish_lanes(t, lane < cw ? rxc[lane] : (TC)0);
                    if (!group_barrier(gs)) break;
                }
                if (threadIdx.x == 0) {
                    if (st[0].active) checkpoint_column(st[0], cm, zeta);
                    const double rho = st[0].rho;
                    s_beta = (TC)((1.0 - rho) / (1.0 + rho));
                    s_stop = !st[0].active;
                }
                __syncthreads();
                if (s_stop) break;
            } else if (per == 0) {
                // bound the drift between CTAs (mailbox slots are reused every CD4_RING steps)
                if (!group_barrier(gs)) break;
            }
        }
    }
drain:
    __syncthreads();
    for (int e = threadIdx.x; e < cw; e += NT) x[c0 + e] = xc[e];
    if (threadIdx.x == 0) {
        for (int bf = 0; bf < CD4_NB; ++bf)
            if (s_pending[bf]) {
                if (mbar_wait_bounded(&mbar[bf], s_phase[bf], cm.timeout_ns)) s_phase[bf] ^= 1u;
                else group_fail(gs, KPP_ERR_TIMEOUT);
                s_pending[bf] = 0;
            }
    }
    __syncthreads();
    if (g == 0 && threadIdx.x == 0) {
        const ColState &cs = st[0];
        SolveScalars &out = sa.sc[0];
        out.E0 = cs.E0; out.E1 = cs.E1; out.rhat = cs.rhat; out.rho = cs.rho; out.ci = cs.ci;
        out.active = cs.active; out.status = cs.status; out.res_est = cs.res_est; out.bn2 = cs.bn2;
        out.t = t;
    }
#undef TILE4
#undef GINV4
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
size_t cd3_smem_bytes(int s, int64_t CW, int KP, int ta_size, int tc_size, bool use_w) {
    return (size_t)smem3_layout(s, CW, KP, ta_size, tc_size, use_w).total;
}

// sized for either kernel (the FP64 single-column kernel uses the longer ring)
size_t cd3_mail_bytes(int s, int KP, bool f64) {
    const int ring = CD3_RING > CD4_RING ? CD3_RING : CD4_RING;
    return (size_t)ring * s * KP * (f64 ? 2 : 1) * 8;
}

// s * es >= 16: the checkpoint partials (G x 2 doubles) live in the G x s partial buffer; the tile row of
// CW values of es bytes must be a multiple of 16 bytes (TMA)
bool cd4_fits(int s, int64_t CW, int es) {
    return s * es >= 16 && s <= CD4_S && CW >= 2 && CW <= CD4_CW && (CW * es) % 16 == 0;
}

template <typename TA, typename TC>
static cudaError_t launch4_t(const void *d_sys, int nsys, const Common &cm, cudaStream_t st) {
    auto kern = cd4_kernel<TA, TC>;
    const size_t smem = (size_t)smem4_layout(cm.s, cm.CW, (int)sizeof(TC)).total;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if ((int64_t)per_sm * sm_count() < (int64_t)nsys * cm.G) return cudaErrorCooperativeLaunchTooLarge;
    Common c = cm;
    const Sys3 *p = (const Sys3 *)d_sys;
    void *args[] = {(void *)&p, (void *)&c};
    note_launch();
    return cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)(nsys * cm.G)), dim3(NT), args, smem, st);
}

// The single-column dataflow kernel: FP64 on W, or FP32 on the FP32 memo W32 for FP32/BF16 storage.
cudaError_t launch_cd4(int dtype, const void *d_sys, int nsys, const Common &cm, cudaStream_t st) {
    if (dtype == KPP_F64) return launch4_t<double, double>(d_sys, nsys, cm, st);
    if (dtype == KPP_F32) return launch4_t<float, float>(d_sys, nsys, cm, st);
    return launch4_t<__nv_bfloat16, float>(d_sys, nsys, cm, st);
}

size_t sys3_bytes() { return sizeof(Sys3); }

void sys3_fill(void *dst_host, const SysArgs &a, const void *tmap, void *mail) {
    Sys3 *p = (Sys3 *)dst_host;
    memcpy(&p->tmapT, tmap, sizeof(CUtensorMap));
    p->a = a;
    p->mail = (unsigned long long *)mail;
}

template <typename TA, typename TC, int KP, bool USE_W>
static cudaError_t launch3_t(const void *d_sys, int nsys, const Common &cm, cudaStream_t st) {
    auto kern = cd3_kernel<TA, TC, KP, USE_W>;
    const size_t smem = cd3_smem_bytes(cm.s, cm.CW, KP, sizeof(TA), sizeof(TC), USE_W);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if ((int64_t)per_sm * sm_count() < (int64_t)nsys * cm.G) return cudaErrorCooperativeLaunchTooLarge;
    Common c = cm;
    const Sys3 *p = (const Sys3 *)d_sys;
    void *args[] = {(void *)&p, (void *)&c};
    note_launch();
    return cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)(nsys * cm.G)), dim3(NT), args, smem, st);
}

template <typename TA, typename TC, bool USE_W>
static cudaError_t launch3_kp(const void *d_sys, int nsys, const Common &cm, int KP, cudaStream_t st) {
    switch (KP) {
        case 1: return launch3_t<TA, TC, 1, USE_W>(d_sys, nsys, cm, st);
        case 8: return launch3_t<TA, TC, 8, USE_W>(d_sys, nsys, cm, st);
        case 32: return launch3_t<TA, TC, 32, USE_W>(d_sys, nsys, cm, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cd3(int dtype, const void *d_sys, int nsys, const Common &cm, int KP, cudaStream_t st) {
    if (dtype == KPP_F64) return launch3_kp<double, double, true>(d_sys, nsys, cm, KP, st);
    if (dtype == KPP_F32) return launch3_kp<float, float, false>(d_sys, nsys, cm, KP, st);
    return launch3_kp<__nv_bfloat16, float, false>(d_sys, nsys, cm, KP, st);
}

}  // namespace kpp
