// kpp_kw.cu -- K++ iterations in FP32 for large blocks (BF16 / FP32 storage, one right-hand side),
// with the memoised W_j = G_j^{-1} A_{S_j} and a single exchange per step.
//
// A K++ step (Eq. 1.3 - 1.4) needs r = A_S x - b_S summed over every column chunk, then on each chunk
// w = A_S^T G_j^{-1} r = W_S^T r, then m <- beta (m - w), x <- x - w + eta m.  With W memoised (the
// factor phase builds it next to G^{-1}), the only value a CTA needs from the others in a step is the
// s-vector r, so a step is:
//   1. exchange: the per-chunk partials of r are summed by a reduce-scatter inside each 4-CTA cluster
//      (each CTA pushes the rows of its partial into the owner's shared memory), a tagged mailbox
//      between the clusters (each CTA publishes s/4 cluster sums and reads the same slice from every
//      cluster), and an all-gather inside the cluster (each CTA pushes its slice of r to the others);
//   2. w = W_S^T r on my 32 columns, then m and x there;
//   3. the partial r of the next block on my columns (its A tile is already in shared memory).
// A tiles are prefetched two steps ahead and W tiles one step ahead by TMA; the copies, the block draws
// and the loads of b are issued while the mailbox is polled, off the step's critical path.  The window sums and checkpoints (Eq. 5.2 -
// 5.3, Alg. 3) are computed by every CTA from the same r in the same order, so every CTA takes the
// same decisions without a grid barrier.  Hardware cluster barriers cannot time out, so every exit
// from the step loop is taken by all CTAs of a cluster together (failures are OR-ed over the cluster
// at a fixed point of each step) and the CTAs of a cluster leave through one last cluster barrier.
#include <cuda.h>

#include <cmath>
#include <cstring>

#include "kpp_internal.cuh"
#include "kpp_runtime.h"
#include "kpp_solve.h"
#include "kpp_solve_device.cuh"

namespace kpp {

constexpr int KW_CW = 32;     // columns per CTA
constexpr int KW_CL = 4;      // CTAs per cluster (clusters of 8 do not all fit at one CTA per SM)
constexpr int KW_SMAX = 512;  // block size at most (BF16; FP32 storage: 256)
constexpr int KW_RING = 4;    // mailbox slots (steps); a cluster is never more than two steps ahead
constexpr int KW_MAXG = 152;  // CTAs per system at most
constexpr int KW_MAILMAX = (KW_MAXG / KW_CL) * (KW_SMAX / KW_CL);  // one step's words of my slice
constexpr int KW_PER_T = (KW_MAILMAX + NT - 1) / NT;                // of them per thread
static_assert(KW_PER_T <= 32, "one bit per word in the poll mask");

struct alignas(128) SysK {
    CUtensorMap tmA;             // A: cols x rows, box {32, min(s, 256)}
    CUtensorMap tmW;             // W (FP32): cols x rows, box {32, min(s, 256)}
    const float *b;              // rows (FP32 right-hand side)
    float *x;                    // cols (FP32)
    SolveScalars *sc;            // 1
    unsigned *bar;
    int *err;
    double *rpart;               // G doubles
    unsigned long long *mail;    // KW_RING x (G / 4) x s words
    uint32_t sys_id;
    int64_t t0;
};

__device__ __forceinline__ unsigned kw_cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned kw_cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void kw_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t kw_mapa(const void *p, unsigned rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ float kw_ld_cluster_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ int kw_ld_cluster_s32(uint32_t a) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void kw_st_cluster_f32(uint32_t a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void kw_st_cluster_s32(uint32_t a, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long kw_ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void kw_st_relaxed(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Dot product of one 16-byte piece of a tile row (8 BF16 or 4 FP32 values) with x values in registers.
template <typename TA> struct KwRow;
template <> struct KwRow<__nv_bfloat16> {
    static constexpr int PER = 8;  // values per 16-byte load
    __device__ __forceinline__ static float dot(const __nv_bfloat16 *p, const float (&xv)[8]) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p);
        float acc = __uint_as_float(q.x << 16) * xv[0];
        acc = fmaf(__uint_as_float(q.x & 0xffff0000u), xv[1], acc);
        acc = fmaf(__uint_as_float(q.y << 16), xv[2], acc);
        acc = fmaf(__uint_as_float(q.y & 0xffff0000u), xv[3], acc);
        acc = fmaf(__uint_as_float(q.z << 16), xv[4], acc);
        acc = fmaf(__uint_as_float(q.z & 0xffff0000u), xv[5], acc);
        acc = fmaf(__uint_as_float(q.w << 16), xv[6], acc);
        acc = fmaf(__uint_as_float(q.w & 0xffff0000u), xv[7], acc);
        return acc;
    }
};
template <> struct KwRow<float> {
    static constexpr int PER = 4;
    __device__ __forceinline__ static float dot(const float *p, const float (&xv)[8]) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        float acc = q.x * xv[0];
        acc = fmaf(q.y, xv[1], acc);
        acc = fmaf(q.z, xv[2], acc);
        acc = fmaf(q.w, xv[3], acc);
        return acc;
    }
};

struct SmemK {
    int w[2], a[2], total;
};
__host__ __device__ inline SmemK kw_layout(int s, int ta_size) {
    SmemK L;
    int o = 0;
    const int wt = s * KW_CW * 4, at = s * KW_CW * ta_size;
    L.w[0] = o; o += wt;
    L.w[1] = o; o += wt;
    L.a[0] = o; o += at;
    L.a[1] = o; o += at;
    L.total = o;
    return L;
}

template <typename TA>
__global__ void __launch_bounds__(NT, 1) kw_kernel(const SysK *__restrict__ systems, Common cm) {
    constexpr int PER = KwRow<TA>::PER;    // columns per 16-byte load
    constexpr int CG = KW_CW / PER;        // column groups of a row (4 for BF16, 8 for FP32)
    constexpr int RPW = 32 / CG;           // rows per warp pass of the partial-r loop
    const SysK &sys = systems[blockIdx.x / cm.G];
    const int g = blockIdx.x % cm.G;
    const unsigned q = kw_cluster_rank();  // rank in the cluster = my slice of r
    const int cl = g / KW_CL;              // cluster index within the system
    const int ncl = cm.G / KW_CL;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = cm.s, nb = cm.nb;
    const int SL = s / KW_CL;              // slice length
    const int box = s < 256 ? s : 256;
    const int64_t rows = cm.rows;
    const int64_t c0 = (int64_t)g * KW_CW;
    const float *__restrict__ b = sys.b;
    float *__restrict__ x = sys.x;

    extern __shared__ __align__(128) unsigned char sm[];
    const SmemK L = kw_layout(s, (int)sizeof(TA));
#define KW_W(i) ((const float *)(sm + L.w[i]))
#define KW_A(i) ((const TA *)(sm + L.a[i]))
    __shared__ float s_in[KW_CL][KW_SMAX / KW_CL];  // partials of my slice of r, by source rank (pushed)
    __shared__ __align__(16) float s_r[KW_SMAX];  // r of the step (read as float4)
    __shared__ float s_mail[KW_MAILMAX];     // my slice from every cluster (cluster-major)
    __shared__ float s_red[NW][KW_CW];
    __shared__ float s_rn[NW];
    __shared__ float xc[KW_CW], mc[KW_CW];
    __shared__ __align__(8) uint64_t mbW[2], mbA[2];
    __shared__ ColState st[1];
    __shared__ double s_part[NW];
    __shared__ int s_flag;              // my failure flag (read by the cluster)
    __shared__ int s_flags[KW_CL];      // every CTA's failure flag of the step (pushed)
    __shared__ int s_jq[4];             // block of steps t .. t + 3 (ring by t mod 4)
    __shared__ int s_fail, s_stop;
    __shared__ unsigned s_phW[2], s_phA[2];
    __shared__ int s_pendW[2], s_pendA[2];
    __shared__ float s_beta;

    GroupSync gs{sys.bar, sys.err, 0u, (unsigned)cm.G, cm.timeout_ns};
    // Every distributed-shared-memory address below assumes clusters of KW_CL CTAs.  A launch without
    // them (the host always sets the attribute) is refused here, uniformly over the grid, before any
    // shared-memory window of another CTA or any copy is touched.
    if (kw_cluster_size() != (unsigned)KW_CL) {
        if (threadIdx.x == 0) group_fail(gs, KPP_ERR_UNSUPPORTED);
        return;
    }
    const int zeta = nb;
    const int64_t t_begin = cm.t0_state ? sys.sc[0].t : sys.t0;
    int64_t t = t_begin;
    int64_t t_end = cm.t0_state ? t + cm.max_iters : cm.max_iters;
    if (cm.t0_state && !sys.sc[0].active) t_end = t;
    int ph = (int)(t % (2 * (int64_t)zeta));
    bool quit = false;

    if (threadIdx.x == 0) {
        ColState cs = {};
        const SolveScalars &in = sys.sc[0];
        cs.E0 = in.E0; cs.E1 = in.E1; cs.rhat = in.rhat; cs.rho = in.rho; cs.ci = in.ci;
        cs.active = in.active; cs.status = in.status;
        cs.res_true = NAN;
        cs.res_est = NAN;
        st[0] = cs;
        for (int i = 0; i < 2; ++i) {
            mbar_init(&mbW[i], 1);
            mbar_init(&mbA[i], 1);
            s_phW[i] = s_phA[i] = 0;
            s_pendW[i] = s_pendA[i] = 0;
        }
        fence_mbar_init();
        tensormap_acquire(&sys.tmA);
        tensormap_acquire(&sys.tmW);
        s_fail = 0;
        s_flag = 0;
        s_stop = 0;
        s_beta = (float)((1.0 - cs.rho) / (1.0 + cs.rho));
    }
    for (int c = threadIdx.x; c < KW_CW; c += NT) {
        xc[c] = x[c0 + c];
        mc[c] = 0.0f;
    }
    {
        // |b|^2 over the group (fixed order)
        double acc = 0.0;
        for (int64_t i = (int64_t)g * NT + threadIdx.x; i < rows; i += (int64_t)cm.G * NT)
            acc += (double)b[i] * (double)b[i];
        __syncthreads();
        const double v = block_sum<NT>(acc, s_part);
        if (threadIdx.x == 0) sys.rpart[g] = v;
        if (!group_barrier(gs)) s_fail = 1;
        if (threadIdx.x == 0 && !s_fail) {
            double tt = 0.0;
            for (int h = 0; h < cm.G; ++h) tt += __ldcg(sys.rpart + h);
            st[0].bn2 = tt;
        }
        __syncthreads();
        if (!group_barrier(gs)) s_fail = 1;
    }
    // A failure here must end the step loop for all CTAs of a cluster together: a CTA that skipped the
    // loop would meet its peers' first in-loop cluster barrier with its final one and leave while they
    // still read its shared memory.  So the flags are OR-ed over the cluster first.
    if (threadIdx.x == 0) s_flag = s_fail;
    kw_cluster_sync();
    if (threadIdx.x < KW_CL && kw_ld_cluster_s32(kw_mapa(&s_flag, threadIdx.x))) s_fail = 1;
    __syncthreads();
    if (s_fail) t_end = t;  // uniform over the cluster

    {
        // A buffer whose last copy was never seen complete (its wait timed out) is not given a new copy:
        // that would arm its barrier a second time while the first copy may still be landing.
        auto issueA = [&](int64_t tt, int i) {
            if (s_pendA[i]) {
                s_fail = 1;
                group_fail(gs, KPP_ERR_TIMEOUT);
                return;
            }
            const int S0 = s_jq[tt & 3] * s;
            mbar_arrive_expect_tx(&mbA[i], (unsigned)(s * KW_CW * sizeof(TA)));
            for (int r0 = 0; r0 < s; r0 += box)
                tma_load_2d((void *)(KW_A(i) + (size_t)r0 * KW_CW), &sys.tmA, (int)c0, S0 + r0, &mbA[i]);
            s_pendA[i] = 1;
        };
        auto issueW = [&](int64_t tt, int i) {
            if (s_pendW[i]) {
                s_fail = 1;
                group_fail(gs, KPP_ERR_TIMEOUT);
                return;
            }
            const int S0 = s_jq[tt & 3] * s;
            mbar_arrive_expect_tx(&mbW[i], (unsigned)(s * KW_CW * 4));
            for (int r0 = 0; r0 < s; r0 += box)
                tma_load_2d((void *)(KW_W(i) + (size_t)r0 * KW_CW), &sys.tmW, (int)c0, S0 + r0, &mbW[i]);
            s_pendW[i] = 1;
        };
        auto waitbuf = [&](uint64_t *mb, unsigned *phs, int *pend, int i) {
            if (threadIdx.x == 0) {
                if (mbar_wait_bounded(&mb[i], phs[i], cm.timeout_ns)) {
                    phs[i] ^= 1u;
                    pend[i] = 0;
                } else {
                    s_fail = 1;
                    group_fail(gs, KPP_ERR_TIMEOUT);
                }
            }
            __syncthreads();
        };
        // my partial of r for the block whose A tile is in buffer i: p[a] = sum_c A[a][c] x_c (c my columns),
        // pushed into the shared memory of row a's owner (rank a / SL), at my rank's place
        auto partial = [&](int i) {
            const TA *tl = KW_A(i);
            const int rs = lane / CG, cgi = lane % CG;
            float xv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) xv[e] = e < PER ? xc[cgi * PER + e] : 0.0f;
#pragma unroll 4
            for (int r0 = warp * RPW; r0 < s; r0 += NW * RPW) {
                const int a = r0 + rs;
                float acc = KwRow<TA>::dot(tl + (size_t)a * KW_CW + cgi * PER, xv);
#pragma unroll
                for (int o = 1; o < CG; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (cgi == 0) kw_st_cluster_f32(kw_mapa(&s_in[q][a % SL], (unsigned)(a / SL)), acc);
            }
        };

        // A of steps t, t + 1 and W of step t now; then, at step t, A of t + 2 and W of t + 1
        if (threadIdx.x == 0 && t < t_end) {
            for (int d = 0; d < 2; ++d) s_jq[(t + d) & 3] = draw_block(cm.seed, t + d, sys.sys_id, nb);
            issueA(t, (int)(t & 1));
            issueW(t, (int)(t & 1));
            if (t + 1 < t_end) issueA(t + 1, (int)((t + 1) & 1));
        }
        __syncthreads();
        if (t < t_end) {
            waitbuf(mbA, s_phA, s_pendA, (int)(t & 1));
            partial((int)(t & 1));
        }

        while (t < t_end) {
            const int bi = (int)(t & 1);
            const int S0 = s_jq[t & 3] * s;
            // my slice of b_S, loaded now and used after the mailbox
            const float bv = threadIdx.x < SL ? b[S0 + (int)q * SL + threadIdx.x] : 0.0f;

            // ---- 1. exchange: reduce-scatter in the cluster, mailbox between clusters, all-gather ----
            __syncthreads();
            kw_cluster_sync();  // partials of every CTA of the cluster have been pushed
            if (threadIdx.x < SL) {
                const int e = (int)q * SL + threadIdx.x;
                float v = 0.0f;
#pragma unroll
                for (int rr = 0; rr < KW_CL; ++rr) v += s_in[rr][threadIdx.x];
                unsigned long long *slot = sys.mail + ((size_t)(t % KW_RING) * ncl + cl) * s;
                kw_st_relaxed(slot + e, ((unsigned long long)(unsigned)(t + 1) << 32) | __float_as_uint(v));
            }
            // while the mailbox fills: the block of step t + 2 and the copies whose buffers are free (A of
            // step t went into my partial before this step; W of step t - 1 into its update)
            if (threadIdx.x == NT - 32) {
                if (t + 2 < t_end) {
                    s_jq[(t + 2) & 3] = draw_block(cm.seed, t + 2, sys.sys_id, nb);
                    issueA(t + 2, bi);
                }
                if (t + 1 < t_end) issueW(t + 1, bi ^ 1);
            }
            {
                // read my slice from every cluster: all threads issue their loads first, then re-poll the
                // words whose tag is not there yet (bounded)
                const unsigned tag = (unsigned)(t + 1);
                const unsigned long long *base = sys.mail + (size_t)(t % KW_RING) * ncl * s + (size_t)q * SL;
                const int total = ncl * SL;
                unsigned long long wv[KW_PER_T];
                unsigned missing = 0;  // bit i: word i not there yet
#pragma unroll
                for (int i = 0; i < KW_PER_T; ++i) {
                    const int l = threadIdx.x + i * NT;
                    if (l < total) {
                        wv[i] = kw_ld_relaxed(base + (size_t)(l / SL) * s + (l % SL));
                        missing |= 1u << i;
                    }
                }
                const uint64_t tq = globaltimer_ns();
                for (unsigned round = 0;; ++round) {
                    // take every word that has arrived; re-issue the loads of the others together
#pragma unroll
                    for (int i = 0; i < KW_PER_T; ++i) {
                        if (((missing >> i) & 1u) && (unsigned)(wv[i] >> 32) == tag) {
                            s_mail[threadIdx.x + i * NT] = __uint_as_float((unsigned)wv[i]);
                            missing &= ~(1u << i);
                        }
                    }
                    if (!missing) break;
                    if ((round & 15u) == 15u) {
                        if (globaltimer_ns() - tq > cm.timeout_ns) {
                            s_fail = 1;
                            group_fail(gs, KPP_ERR_TIMEOUT);
                            break;
                        }
                        if (*(volatile int *)gs.err != 0) {
                            s_fail = 1;
                            break;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < KW_PER_T; ++i) {
                        const int l = threadIdx.x + i * NT;
                        if ((missing >> i) & 1u) wv[i] = kw_ld_relaxed(base + (size_t)(l / SL) * s + (l % SL));
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x < SL) {
                const int eg = (int)q * SL + threadIdx.x;
                float v = 0.0f;
                for (int c = 0; c < ncl; ++c) v += s_mail[c * SL + threadIdx.x];  // cluster order
                v -= bv;
#pragma unroll
                for (int rr = 0; rr < KW_CL; ++rr) kw_st_cluster_f32(kw_mapa(&s_r[eg], (unsigned)rr), v);
            }
            if (threadIdx.x < KW_CL) kw_st_cluster_s32(kw_mapa(&s_flags[q], threadIdx.x), s_fail);
            kw_cluster_sync();  // slices of r and failure flags of every CTA of the cluster have been pushed
            if (threadIdx.x < KW_CL && s_flags[threadIdx.x]) s_fail = 1;  // benign race: every writer writes 1
            __syncthreads();
            if (s_fail) break;  // uniform over the cluster (every CTA saw every flag)

            // |r|^2 (FP32 in a fixed order, accumulated in FP64)
            {
                float v = 0.0f;
                for (int e = threadIdx.x; e < s; e += NT) v = fmaf(s_r[e], s_r[e], v);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) s_rn[warp] = v;
            }

            // ---- 2. w = W_S^T r on my columns, then m and x ----
            waitbuf(mbW, s_phW, s_pendW, bi);
            {
                const float *wt = KW_W(bi);
                float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
                const int rpw = s / NW;  // a multiple of 4
                const int ra = warp * rpw;
                for (int i0 = 0; i0 < rpw; i0 += 16) {
                    // 16 rows: r from shared memory as 4 float4 (broadcast), W column values
                    float rr[16];
                    const float4 *r4 = reinterpret_cast<const float4 *>(s_r + ra + i0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 v = r4[u];
                        rr[4 * u] = v.x; rr[4 * u + 1] = v.y; rr[4 * u + 2] = v.z; rr[4 * u + 3] = v.w;
                    }
                    const int n16 = rpw - i0 < 16 ? rpw - i0 : 16;
                    if (n16 == 16) {
#pragma unroll
                        for (int i = 0; i < 16; i += 4) {
                            a0 = fmaf(wt[(ra + i0 + i) * KW_CW + lane], rr[i], a0);
                            a1 = fmaf(wt[(ra + i0 + i + 1) * KW_CW + lane], rr[i + 1], a1);
                            a2 = fmaf(wt[(ra + i0 + i + 2) * KW_CW + lane], rr[i + 2], a2);
                            a3 = fmaf(wt[(ra + i0 + i + 3) * KW_CW + lane], rr[i + 3], a3);
                        }
                    } else {
                        for (int i = 0; i < n16; ++i) a0 = fmaf(wt[(ra + i0 + i) * KW_CW + lane], s_r[ra + i0 + i], a0);
                    }
                }
                s_red[warp][lane] = (a0 + a1) + (a2 + a3);
            }
            __syncthreads();
            if (threadIdx.x < KW_CW) {
                const int c = threadIdx.x;
                float w = 0.0f;
#pragma unroll
                for (int v = 0; v < NW; ++v) w += s_red[v][c];
                const float mm = s_beta * (mc[c] - w);
                mc[c] = mm;
                xc[c] = xc[c] - w + (float)cm.eta * mm;
            }
            if (threadIdx.x == 32) {
                float rn = 0.0f;
                for (int v = 0; v < NW; ++v) rn += s_rn[v];
                ColState &cs = st[0];
                if (ph < zeta) cs.E0 += (double)rn;
                else cs.E1 += (double)rn;
            }
            __syncthreads();

            // ---- 3. my partial of r_{t+1} ----
            if (t + 1 < t_end) {
                waitbuf(mbA, s_phA, s_pendA, bi ^ 1);
                partial(bi ^ 1);
            }

            // ---- checkpoint (identical in every CTA) ----
            const bool ckpt = (ph == 2 * zeta - 1);
            t += 1;
            if (++ph == 2 * zeta) ph = 0;
            if (ckpt) {
                __syncthreads();
                if (threadIdx.x == 0) {
                    ColState &cs = st[0];
                    cs.res_est = cs.bn2 > 0.0 ? sqrt(cs.E1 / cs.bn2) : sqrt(cs.E1);
                    if (cs.active) checkpoint_column(cs, cm, zeta);
                    s_beta = (float)((1.0 - cs.rho) / (1.0 + cs.rho));
                    s_stop = !cs.active;
                }
                __syncthreads();
                if (s_stop) break;
            }
        }
    }
    quit = true;
    (void)quit;
    // leave together: no CTA exits while a peer may still read its shared memory
    __syncthreads();
    kw_cluster_sync();
    for (int c = threadIdx.x; c < KW_CW; c += NT) x[c0 + c] = xc[c];
    // Drain: every copy issued to this CTA's shared memory lands before the CTA leaves.  A copy
    // from valid global memory always completes; the (longer) limit only keeps the wait bounded.
    if (threadIdx.x == 0) {
        const uint64_t drain_ns = 4 * cm.timeout_ns;
        for (int i = 0; i < 2; ++i) {
            if (s_pendA[i]) {
                if (mbar_wait_bounded(&mbA[i], s_phA[i], drain_ns)) s_phA[i] ^= 1u;
                else group_fail(gs, KPP_ERR_TIMEOUT);
            }
            if (s_pendW[i]) {
                if (mbar_wait_bounded(&mbW[i], s_phW[i], drain_ns)) s_phW[i] ^= 1u;
                else group_fail(gs, KPP_ERR_TIMEOUT);
            }
        }
    }
    __syncthreads();
    if (g == 0 && threadIdx.x == 0) {
        const ColState &cs = st[0];
        SolveScalars &out = sys.sc[0];
        out.E0 = cs.E0; out.E1 = cs.E1; out.rhat = cs.rhat; out.rho = cs.rho; out.ci = cs.ci;
        out.active = cs.active; out.status = cs.status; out.res_est = cs.res_est; out.bn2 = cs.bn2;
        out.t = t;
    }
#undef KW_W
#undef KW_A
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
bool kw_fits(int dtype, int64_t rows, int64_t cols, int s, int k, int sms) {
    if (dtype == KPP_F64 || k != 1) return false;
    const int smax = dtype == KPP_BF16 ? KW_SMAX : 256;
    if (s < 32 || s > smax || s % 32) return false;  // 8 warps x rows in fours
    if (s > 256 && s % 256) return false;  // whole 256-row TMA boxes
    if (rows % s) return false;
    if (cols % (KW_CW * KW_CL)) return false;
    const int64_t G = cols / KW_CW;
    if (G > sms || G > KW_MAXG) return false;
    return kw_layout(s, dtype == KPP_BF16 ? 2 : 4).total <= 200 * 1024;
}

int64_t kw_grid(int64_t cols) { return cols / KW_CW; }

size_t kw_mail_bytes(int s, int G) { return (size_t)KW_RING * (G / KW_CL) * s * 8; }

size_t sysk_bytes() { return sizeof(SysK); }

void sysk_fill(void *dst, const void *tmA, const void *tmW, const float *b, float *x, SolveScalars *sc, unsigned *bar,
               int *err, double *rpart, void *mail, uint32_t sys_id, int64_t t0) {
    SysK *p = (SysK *)dst;
    memcpy(&p->tmA, tmA, sizeof(CUtensorMap));
    memcpy(&p->tmW, tmW, sizeof(CUtensorMap));
    p->b = b;
    p->x = x;
    p->sc = sc;
    p->bar = bar;
    p->err = err;
    p->rpart = rpart;
    p->mail = (unsigned long long *)mail;
    p->sys_id = sys_id;
    p->t0 = t0;
}

template <typename TA>
static cudaError_t launch_kw_t(const void *d_sys, int nsys, const Common &cm, cudaStream_t st) {
    const size_t smem = (size_t)kw_layout(cm.s, (int)sizeof(TA)).total;
    cudaError_t e = cudaFuncSetAttribute(kw_kernel<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nsys * cm.G));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = KW_CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeCooperative;
    at[1].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, (const void *)kw_kernel<TA>, &cfg);
    if (e != cudaSuccess) return e;
    if ((int64_t)ncl * KW_CL < (int64_t)nsys * cm.G) return cudaErrorCooperativeLaunchTooLarge;
    const SysK *p = (const SysK *)d_sys;
    Common c = cm;
    note_launch();
    return cudaLaunchKernelEx(&cfg, kw_kernel<TA>, p, c);
}

template <typename TA> static int kw_max_clusters(int s) {
    const size_t smem = (size_t)kw_layout(s, (int)sizeof(TA)).total;
    if (cudaFuncSetAttribute(kw_kernel<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(KW_CL);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = KW_CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, (const void *)kw_kernel<TA>, &cfg) != cudaSuccess) return 0;
    return ncl;
}

// Whether nsys systems of `cols` columns fit co-resident as 4-CTA clusters (clusters live inside a GPC).
bool kw_can_launch(int dtype, int s, int64_t cols, int nsys) {
    const int need = (int)(nsys * kw_grid(cols) / KW_CL);
    const int have = dtype == KPP_BF16 ? kw_max_clusters<__nv_bfloat16>(s) : kw_max_clusters<float>(s);
    cudaGetLastError();
    return have >= need;
}

cudaError_t launch_kw(int dtype, const void *d_sys, int nsys, const Common &cm, cudaStream_t st) {
    return dtype == KPP_BF16 ? launch_kw_t<__nv_bfloat16>(d_sys, nsys, cm, st) : launch_kw_t<float>(d_sys, nsys, cm, st);
}

}  // namespace kpp
