// kpp_stream.cu -- batched K++ inner iteration for wide systems (FP32 / BF16 storage, FP32 arithmetic):
// many systems, each with a panel of k right-hand sides, in one persistent launch.
//
// The step is K++'s (Eq. 1.3, 1.4; Alg. 5 with exact memoised projections):
//   R = A_S X - B_S,  Y = G^{-1} R,  W = A_S^T Y,  M <- beta (M - W),  X <- X - W + eta M,
// every right-hand-side column with its own rho, residual estimate and stop test, all columns of a
// system sharing its block sequence.  For wide blocks (config of 256 rows x 65536 columns) a step is two
// streaming passes over A_S: the partial residual (P) and the back-projection (C).  The block does not
// fit on chip, so each CTA owns an even share of the column tiles of one system and streams them:
//   * one TMA tile stream per CTA through a 5-stage ring: A tile (s rows x 128 bytes, 128-byte swizzle:
//     thread-per-row 16-byte reads and lane-per-column reads are both conflict-free) plus bulk copies of
//     the X (and, in pass C, M) panel slices of the same columns;
//   * the stream never stops between passes or steps: the tiles of the next pass are already in flight
//     while the group exchanges its partial residuals (one group barrier per step);
//   * Y = G^{-1} R is applied redundantly in every CTA of the system (G^{-1} symmetric: read by
//     columns, coalesced), so the only exchange is the partial residual.
// The X / M updates are generic stores that a later bulk copy of the same system reads: a proxy fence
// orders them.  A chunk holds at least ST_MIN_TILES tiles, so a refill never reads a slice whose store
// is still the most recent one.  Every wait is bounded.
#include <cuda.h>

#include <cmath>
#include <cstdio>

#include "kpp_internal.cuh"
#include "kpp_runtime.h"
#include "kpp_solve.h"
#include "kpp_solve_device.cuh"

namespace kpp {

constexpr int ST_STAGES = 5;
constexpr int ST_MIN_TILES = 8;  // fewest tiles of a chunk (see wait())
static_assert(ST_MIN_TILES > ST_STAGES && 2 * ST_MIN_TILES >= ST_STAGES, "refill distance");
constexpr int ST_ROWB = 128;     // bytes of one tile row

struct alignas(128) Sys4 {
    CUtensorMap tmapA;      // A: cols x rows, box {128 B of columns, s rows}, 128-byte swizzle
    const float *b;         // rows x k (inner right-hand side)
    float *X;               // cols x k
    float *M;               // cols x k
    const float *Ginv;      // nb x s x s (block j: len x len, ld len)
    float *part;            // 2 x G x s x KP
    double *rpart;          // G x KP
    SolveScalars *sc;       // k
    unsigned *bar;
    int *err;
    uint32_t sys_id;
    int64_t t0;
};

template <typename TA>
__host__ __device__ constexpr int st_tk() { return ST_ROWB / (int)sizeof(TA); }

__host__ __device__ inline int st_stage_bytes(int s, int KP) {
    // A tile + X slice + M slice (TK <= 64 columns x KP floats each); every stage starts on a 1024-byte
    // boundary, which the 128-byte swizzle of the A tile requires
    const int a = (s * ST_ROWB + 1023) / 1024 * 1024;
    const int v = (64 * KP * 4 + 127) / 128 * 128;
    return (a + 2 * v + 1023) / 1024 * 1024;
}

template <typename TA, int KP>
__global__ void __launch_bounds__(256, 1) stream_kernel(const Sys4 *__restrict__ systems, Common cm) {
    constexpr int TK = st_tk<TA>();          // columns per tile
    constexpr int V = 16 / (int)sizeof(TA);  // values per 16-byte chunk
    const Sys4 &sys = systems[blockIdx.x / cm.G];
    const void *tmap = &sys.tmapA;
    const int g = blockIdx.x % cm.G;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = cm.k, s = cm.s, nb = cm.nb;
    const int64_t rows = cm.rows, cols = cm.cols;
    const float *__restrict__ b = sys.b;
    float *__restrict__ X = sys.X;
    float *__restrict__ M = sys.M;

    extern __shared__ __align__(1024) unsigned char st_raw[];
    // 1024-byte aligned by an offset from the shared array itself (an integer round trip would lose the
    // shared state space, and every tile read would become a generic load)
    unsigned char *sm = st_raw + ((1024u - (smem_u32(st_raw) & 1023u)) & 1023u);
    const int SB = st_stage_bytes(s, KP);
    const int AB = (s * ST_ROWB + 1023) / 1024 * 1024;
    const int VB = (64 * KP * 4 + 127) / 128 * 128;
    float *s_r = (float *)(sm + ST_STAGES * SB);     // s x KP
    float *s_y = s_r + 256 * KP;                     // s x KP
    float *s_red = s_y + 256 * KP;                   // 8 x 64 x KP  (row groups x columns x rhs)
    __shared__ __align__(8) uint64_t full[ST_STAGES];
    __shared__ ColState st[KP];
    __shared__ double s_part[8 * KP];
    __shared__ double s_rn2[KP];
    __shared__ float s_beta[KP], s_keep[KP];
    __shared__ int s_fail, s_stop;
    __shared__ int s_pend[ST_STAGES];
    __shared__ unsigned s_ppar[ST_STAGES];  // parity of the phase a pending stage completes

    GroupSync gs{sys.bar, sys.err, 0u, (unsigned)cm.G, cm.timeout_ns};
    // tiles [g T / G, (g + 1) T / G) of the T = cols / TK column tiles (cols is a multiple of TK); the
    // host keeps every chunk at ST_MIN_TILES tiles or more
    const int64_t T = cols / TK;
    const int64_t c0 = (int64_t)g * T / cm.G * TK;
    const int64_t c1 = (int64_t)(g + 1) * T / cm.G * TK;
    const int nt = (int)((c1 - c0) / TK);
    const int zeta = nb;
    const int64_t t0 = cm.t0_state ? sys.sc[0].t : sys.t0;
    int64_t t_end = cm.t0_state ? t0 + cm.max_iters : cm.max_iters;
    if (cm.t0_state) {  // a system whose columns are all done does not iterate (t stays put)
        int any = 0;
        for (int c = 0; c < cm.k; ++c) any |= sys.sc[c].active;
        if (!any) t_end = t0;
    }

    if (tid < KP) {
        ColState cs = {};
        if (tid < k) {
            const SolveScalars &in = sys.sc[tid];
            cs.E0 = in.E0; cs.E1 = in.E1; cs.rhat = in.rhat; cs.rho = in.rho; cs.ci = in.ci;
            cs.active = in.active; cs.status = in.status;
        }
        cs.res_true = NAN;
        cs.res_est = NAN;
        st[tid] = cs;
    }
    if (tid == 0) {
        for (int i = 0; i < ST_STAGES; ++i) {
            mbar_init(&full[i], 1);
            s_pend[i] = 0;
        }
        fence_mbar_init();
        tensormap_acquire(tmap);
        s_fail = 0;
    }
    // |b|^2 per column
    {
        double acc[KP];
#pragma unroll
        for (int c = 0; c < KP; ++c) acc[c] = 0.0;
        for (int64_t i = (int64_t)g * 256 + tid; i < rows; i += (int64_t)cm.G * 256)
#pragma unroll
            for (int c = 0; c < KP; ++c)
                if (c < k) acc[c] += (double)b[i * k + c] * (double)b[i * k + c];
        __syncthreads();
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            double v = block_sum<256>(acc[c], s_part);
            if (tid == 0) sys.rpart[(size_t)g * KP + c] = v;
        }
        if (!group_barrier(gs)) goto drain;
        if (tid < KP) {
            double tt = 0.0;
            for (int h = 0; h < cm.G; ++h) tt += __ldcg(sys.rpart + (size_t)h * KP + tid);
            st[tid].bn2 = tt;
            const double rho = st[tid].rho;
            s_beta[tid] = (float)((1.0 - rho) / (1.0 + rho));
            s_keep[tid] = (tid < k && st[tid].active) ? 1.f : 0.f;
        }
        __syncthreads();
    }

    {
        // Tile q of the stream: step t0 + q / (2 nt), pass (q / nt) % 2 (0: P, 1: C), column tile q % nt,
        // ring stage q % ST, mbarrier phase parity (q / ST) % 2.  Both ends walk the stream in order, so
        // they keep these as cursors instead of dividing (64-bit divisions on thread 0 would sit on
        // every tile's critical path).
        // Issue cursor (thread 0): the next tile to load, with its step's block draw.
        int64_t i_t = t0;
        int i_pass = 0, i_jt = 0, i_stg = 0, i_j = draw_block(cm.seed, t0, sys.sys_id, nb);
        unsigned i_par = 0;
        // load the tile at the cursor: A tile by TMA, the X slice (and in pass C the M slice) by bulk
        // copy, one mbarrier; then advance.  The X / M slices were last written by bulk stores of this
        // CTA, waited for before every refill.
        auto issue_next = [&]() {
            if (i_t >= t_end) return;
            const int stg = i_stg;
            const int64_t col = c0 + (int64_t)i_jt * TK;
            unsigned char *base = sm + stg * SB;
            const unsigned vbytes = (unsigned)(TK * k * 4);
            mbar_arrive_expect_tx(&full[stg], (unsigned)(s * ST_ROWB) + vbytes * (i_pass ? 2u : 1u));
            tma_load_2d(base, tmap, (int)col, i_j * s, &full[stg]);
            bulk_load(base + AB, X + col * k, vbytes, &full[stg]);
            if (i_pass) bulk_load(base + AB + VB, M + col * k, vbytes, &full[stg]);
            s_pend[stg] = 1;
            s_ppar[stg] = i_par;
            if (++i_stg == ST_STAGES) {
                i_stg = 0;
                i_par ^= 1u;
            }
            if (++i_jt == nt) {
                i_jt = 0;
                i_pass ^= 1;
                if (i_pass == 0 && ++i_t < t_end) i_j = draw_block(cm.seed, i_t, sys.sys_id, nb);
            }
        };
        // Consumer cursor (every thread): the stage and phase parity of the tile being consumed.
        int c_stg = 0;
        unsigned c_par = 0;
        auto next_stage = [&]() {
            if (++c_stg == ST_STAGES) {
                c_stg = 0;
                c_par ^= 1u;
            }
        };
        // wait for tile q; then refill the stage of tile q-2 (every thread is done with it) with tile
        // q-2+ST, after the bulk stores older than the most recent group have completed.  That covers the
        // stage's own pass-C store (tile q-2) and the last store of any X / M slice the refill reads
        // (tile q-2+ST-nt or older: chunks have nt >= ST_MIN_TILES > ST tiles, and the first ST tiles,
        // issued up front, all belong to the first step).  When tile q-1 opens a step (pass P, no
        // store), the stage's own store is the most recent group: wait for all of them.
        // opens_step: tile q-1 was the first tile of a step.  The refill is the issue cursor's tile,
        // which is q-2+ST: ST tiles are issued up front and one per wait from q = 2 on.
        auto wait = [&](int64_t q, bool opens_step) -> bool {
            if (tid == 0) {
                if (!mbar_wait_bounded(&full[c_stg], c_par, cm.timeout_ns)) {
                    s_fail = 1;
                    group_fail(gs, KPP_ERR_TIMEOUT);
                }
                s_pend[c_stg] = 0;
            }
            __syncthreads();
            if (tid == 0 && q >= 2) {
                if (opens_step) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
                else asm volatile("cp.async.bulk.wait_group 1;" ::: "memory");
                issue_next();
            }
            return !s_fail;
        };

        if (tid == 0)
            for (int i = 0; i < ST_STAGES; ++i) issue_next();  // all in the first step: 2 nt > ST
        int64_t q = 0;
        int64_t t = t0;
        while (t < t_end) {
            const int j = draw_block(cm.seed, t, sys.sys_id, nb);
            const int64_t S0 = (int64_t)j * s;
            const int len = (int)min64(s, rows - S0);
            // ---- pass P: partial R over my chunk.  Thread t: rows rp and rp + 128 (rp = t % 128), the
            // column half h = t / 128 of every tile; packed FP32 FMAs; the halves meet once per pass ----
            const int rp = tid & 127, hh = tid >> 7;
            const bool r0ok = rp < len, r1ok = rp + 128 < len;
            float2 p0[(KP + 1) / 2], p1[(KP + 1) / 2];
#pragma unroll
            for (int i = 0; i < (KP + 1) / 2; ++i) {
                p0[i] = make_float2(0.f, 0.f);
                p1[i] = make_float2(0.f, 0.f);
            }
            for (int jt = 0; jt < nt; ++jt, ++q, next_stage()) {
                if (!wait(q, jt == 1)) break;
                const unsigned char *base = sm + c_stg * SB;
                const float *xs = (const float *)(base + AB);
                if (k == KP && KP % 2 == 0) {
#pragma unroll
                    for (int cq = 0; cq < 4; ++cq) {
                        const int ch = hh * 4 + cq;
                        // rows at or beyond len are not part of this tile's block (or of the shared tile)
                        const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
                        const uint4 w0 = r0ok ? *(const uint4 *)(base + rp * ST_ROWB + ((ch ^ (rp & 7)) << 4)) : z4;
                        const uint4 w1 = r1ok ? *(const uint4 *)(base + (rp + 128) * ST_ROWB + ((ch ^ (rp & 7)) << 4)) : z4;
                        const TA *e0 = (const TA *)&w0;
                        const TA *e1 = (const TA *)&w1;
#pragma unroll
                        for (int z = 0; z < V; ++z) {
                            const float a0 = conv<float>(e0[z]);
                            const float a1 = conv<float>(e1[z]);
                            const float2 aa0 = make_float2(a0, a0), aa1 = make_float2(a1, a1);
                            const float2 *xr = (const float2 *)(xs + (ch * V + z) * KP);
#pragma unroll
                            for (int i = 0; i < KP / 2; ++i) {
                                const float2 xv = xr[i];
                                p0[i] = __ffma2_rn(aa0, xv, p0[i]);
                                p1[i] = __ffma2_rn(aa1, xv, p1[i]);
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int cq = 0; cq < 4; ++cq) {
                        const int ch = hh * 4 + cq;
                        // rows at or beyond len are not part of this tile's block (or of the shared tile)
                        const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
                        const uint4 w0 = r0ok ? *(const uint4 *)(base + rp * ST_ROWB + ((ch ^ (rp & 7)) << 4)) : z4;
                        const uint4 w1 = r1ok ? *(const uint4 *)(base + (rp + 128) * ST_ROWB + ((ch ^ (rp & 7)) << 4)) : z4;
                        const TA *e0 = (const TA *)&w0;
                        const TA *e1 = (const TA *)&w1;
#pragma unroll
                        for (int z = 0; z < V; ++z) {
                            const float a0 = conv<float>(e0[z]);
                            const float a1 = conv<float>(e1[z]);
                            const int cc = ch * V + z;
#pragma unroll
                            for (int c = 0; c < KP; ++c) {
                                const float xv = c < k ? xs[cc * k + c] : 0.f;
                                float *q0 = (float *)p0, *q1 = (float *)p1;
                                q0[c] = fmaf(a0, xv, q0[c]);
                                q1[c] = fmaf(a1, xv, q1[c]);
                            }
                        }
                    }
                }
            }
            if (s_fail) break;
            {
                // combine the two column halves (half 1 through shared memory), then publish
                float *hs = s_red;  // 256 rows x KP
                if (hh == 1) {
                    const float *q0 = (const float *)p0, *q1 = (const float *)p1;
#pragma unroll
                    for (int c = 0; c < KP; ++c) {
                        hs[rp * KP + c] = q0[c];
                        hs[(rp + 128) * KP + c] = q1[c];
                    }
                }
                __syncthreads();
                float *part = sys.part + ((size_t)(t & 1) * cm.G + g) * s * KP;
                if (hh == 0) {
                    const float *q0 = (const float *)p0, *q1 = (const float *)p1;
#pragma unroll
                    for (int c = 0; c < KP; ++c) {
                        if (r0ok) part[(size_t)rp * KP + c] = q0[c] + hs[rp * KP + c];
                        if (r1ok) part[(size_t)(rp + 128) * KP + c] = q1[c] + hs[(rp + 128) * KP + c];
                    }
                }
            }
            if (!group_barrier(gs)) break;
            // ---- R = sum of partials - B_S (every CTA, fixed order); |R|^2; Y = G^{-1} R ----
            {
                const float *part = sys.part + (size_t)(t & 1) * cm.G * s * KP;
                for (int e = tid; e < len * KP; e += 256) {
                    const int a = e / KP, c = e % KP;
                    float v = 0.f;
                    if (c < k) {
                        for (int h = 0; h < cm.G; ++h) v += __ldcg(part + ((size_t)h * s + a) * KP + c);
                        v -= b[(S0 + a) * k + c];
                    }
                    s_r[e] = v;
                }
                __syncthreads();
                for (int c = warp; c < k; c += 8) {
                    double v = 0.0;
                    for (int a = lane; a < len; a += 32) v += (double)s_r[a * KP + c] * (double)s_r[a * KP + c];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) s_rn2[c] = v;
                }
                const float *Gj = sys.Ginv + (size_t)j * s * s;
                if (tid < len) {
                    float yv[KP];
#pragma unroll
                    for (int c = 0; c < KP; ++c) yv[c] = 0.f;
#pragma unroll 16
                    for (int d = 0; d < len; ++d) {
                        const float gval = __ldg(Gj + (size_t)d * len + tid);  // G^{-1}[d][tid] = G^{-1}[tid][d]
#pragma unroll
                        for (int c = 0; c < KP; ++c) yv[c] = fmaf(gval, s_r[d * KP + c], yv[c]);
                    }
#pragma unroll
                    for (int c = 0; c < KP; ++c) s_y[tid * KP + c] = yv[c];
                }
                __syncthreads();
            }
            // ---- pass C: W = A_S^T Y on each tile, then M, X updates; thread = (column, row group) ----
            {
                constexpr int RGN = 256 / TK;  // row groups
                const int cc = tid % TK, rg = tid / TK;
                const float eta = (float)cm.eta;
                for (int jt = 0; jt < nt; ++jt, ++q, next_stage()) {
                    if (!wait(q, false)) break;
                    unsigned char *base = sm + c_stg * SB;
                    const float *xs = (const float *)(base + AB);
                    const float *ms = (const float *)(base + AB + VB);
                    float w[KP];
#pragma unroll
                    for (int c = 0; c < KP; ++c) w[c] = 0.f;
                    const int ch = cc / V, z = cc % V;
#pragma unroll 4
                    for (int a = rg; a < len; a += RGN) {
                        const TA *row = (const TA *)(base + a * ST_ROWB + ((ch ^ (a & 7)) << 4));
                        const float av = conv<float>(row[z]);
                        const float *yr = s_y + a * KP;
                        if (KP % 4 == 0) {
                            const float2 aa = make_float2(av, av);
#pragma unroll
                            for (int c4 = 0; c4 < KP; c4 += 4) {
                                const float4 yv = *(const float4 *)(yr + c4);
                                float2 w01 = make_float2(w[c4], w[c4 + 1]), w23 = make_float2(w[c4 + 2], w[c4 + 3]);
                                w01 = __ffma2_rn(aa, make_float2(yv.x, yv.y), w01);
                                w23 = __ffma2_rn(aa, make_float2(yv.z, yv.w), w23);
                                w[c4] = w01.x; w[c4 + 1] = w01.y; w[c4 + 2] = w23.x; w[c4 + 3] = w23.y;
                            }
                        } else {
#pragma unroll
                            for (int c = 0; c < KP; ++c) w[c] = fmaf(av, yr[c], w[c]);
                        }
                    }
                    if (KP % 4 == 0) {
#pragma unroll
                        for (int c4 = 0; c4 < KP; c4 += 4)
                            *(float4 *)(s_red + (rg * TK + cc) * KP + c4) = make_float4(w[c4], w[c4 + 1], w[c4 + 2], w[c4 + 3]);
                    } else {
#pragma unroll
                        for (int c = 0; c < KP; ++c) s_red[(rg * TK + cc) * KP + c] = w[c];
                    }
                    __syncthreads();
                    const int64_t col0 = c0 + (int64_t)jt * TK;
                    float *xw = (float *)xs, *mw = (float *)ms;
                    for (int e = tid; e < TK * KP; e += 256) {
                        const int ccc = e / KP, c = e % KP;
                        if (c < k && s_keep[c] != 0.f) {
                            float u = 0.f;
#pragma unroll
                            for (int r = 0; r < RGN; ++r) u += s_red[(r * TK + ccc) * KP + c];
                            const float mm = s_beta[c] * (mw[ccc * k + c] - u);
                            mw[ccc * k + c] = mm;
                            xw[ccc * k + c] = xw[ccc * k + c] - u + eta * mm;
                        }
                    }
                    // the updated slices go back with bulk stores (async proxy, like the loads)
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncthreads();
                    if (tid == 0) {
                        const unsigned vbytes = (unsigned)(TK * k * 4);
                        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(X + col0 * k),
                                     "r"(smem_u32(xw)), "r"(vbytes)
                                     : "memory");
                        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(M + col0 * k),
                                     "r"(smem_u32(mw)), "r"(vbytes)
                                     : "memory");
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    }
                }
                if (s_fail) break;
            }
            // ---- residual estimate, checkpoint, adaptive rho (identical in every CTA) ----
            const int64_t ph = t % (2 * (int64_t)zeta);
            if (tid < k) {
                ColState &cs = st[tid];
                if (cs.active) {
                    if (ph < zeta) cs.E0 += s_rn2[tid];
                    else cs.E1 += s_rn2[tid];
                    if (ph == 2 * zeta - 1) {
                        cs.res_est = cs.bn2 > 0.0 ? sqrt(cs.E1 / cs.bn2) : sqrt(cs.E1);
                        checkpoint_column(cs, cm, zeta);  // inner solves: no true-residual confirmation
                    }
                }
            }
            __syncthreads();
            t += 1;
            if (ph == 2 * zeta - 1) {
                if (tid < KP) {
                    const double rho = st[tid].rho;
                    s_beta[tid] = (float)((1.0 - rho) / (1.0 + rho));
                    s_keep[tid] = (tid < k && st[tid].active) ? 1.f : 0.f;
                }
                if (tid == 0) {
                    int any = 0;
                    for (int c = 0; c < k; ++c) any |= st[c].active;
                    s_stop = !any;
                }
                __syncthreads();
                if (s_stop) break;
            }
        }
        // write back (CTA 0 of the system)
        if (g == 0 && tid < k) {
            const ColState &cs = st[tid];
            SolveScalars &out = sys.sc[tid];
            out.E0 = cs.E0; out.E1 = cs.E1; out.rhat = cs.rhat; out.rho = cs.rho; out.ci = cs.ci;
            out.active = cs.active; out.status = cs.status; out.res_est = cs.res_est; out.bn2 = cs.bn2;
            out.t = t;
        }
    }
drain:
    __syncthreads();
    if (tid == 0) {
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // X / M stores complete
        // tiles still in flight: wait for each pending stage (bounded), oldest phase first
        for (int i = 0; i < ST_STAGES; ++i) {
            if (!s_pend[i]) continue;
            if (!mbar_wait_bounded(&full[i], s_ppar[i], cm.timeout_ns)) group_fail(gs, KPP_ERR_TIMEOUT);
            s_pend[i] = 0;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
size_t sys4_bytes() { return sizeof(Sys4); }

void sys4_fill(void *dst, const void *tmap, const float *b, float *X, float *M, const float *Ginv, float *part,
               double *rpart, SolveScalars *sc, unsigned *bar, int *err, uint32_t sys_id, int64_t t0) {
    Sys4 *p = (Sys4 *)dst;
    memcpy(&p->tmapA, tmap, sizeof(CUtensorMap));
    p->b = b; p->X = X; p->M = M; p->Ginv = Ginv; p->part = part; p->rpart = rpart; p->sc = sc;
    p->bar = bar; p->err = err; p->sys_id = sys_id; p->t0 = t0;
}

int stream_min_tiles() { return ST_MIN_TILES; }

int stream_tk(int dtype) { return dtype == KPP_BF16 ? st_tk<__nv_bfloat16>() : st_tk<float>(); }

size_t stream_smem_bytes(int s, int KP) {
    return 1024 + (size_t)ST_STAGES * st_stage_bytes(s, KP) + (size_t)(2 * 256 * KP + 8 * 64 * KP) * 4;
}

template <typename TA, int KP>
static cudaError_t launch_st(const void *d_sys, int nsys, const Common &cm, cudaStream_t st) {
    auto kern = stream_kernel<TA, KP>;
    const size_t smem = stream_smem_bytes(cm.s, KP);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    if ((int64_t)per_sm * sm_count() < (int64_t)nsys * cm.G) return cudaErrorCooperativeLaunchTooLarge;
    Common c = cm;
    const Sys4 *p = (const Sys4 *)d_sys;
    void *args[] = {(void *)&p, (void *)&c};
    note_launch();
    return cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)(nsys * cm.G)), dim3(256), args, smem, st);
}

int stream_per_sm(int dtype, int s, int KP) {
    const size_t smem = stream_smem_bytes(s, KP);
    int per_sm = 0;
    const void *f = dtype == KPP_BF16 ? (KP == 1 ? (const void *)stream_kernel<__nv_bfloat16, 1>
                                                 : (const void *)stream_kernel<__nv_bfloat16, 8>)
                                      : (KP == 1 ? (const void *)stream_kernel<float, 1> : (const void *)stream_kernel<float, 8>);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 256, smem) != cudaSuccess) return 0;
    return per_sm;
}

cudaError_t launch_stream(int dtype, const void *d_sys, int nsys, const Common &cm, int KP, cudaStream_t st) {
    if (dtype == KPP_BF16) return KP == 1 ? launch_st<__nv_bfloat16, 1>(d_sys, nsys, cm, st)
                                          : launch_st<__nv_bfloat16, 8>(d_sys, nsys, cm, st);
    return KP == 1 ? launch_st<float, 1>(d_sys, nsys, cm, st) : launch_st<float, 8>(d_sys, nsys, cm, st);
}

}  // namespace kpp
