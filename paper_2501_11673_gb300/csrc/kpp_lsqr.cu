// kpp_lsqr.cu -- K++ with the inexact block projection of Sec. 4.1 ("Computing the projection step";
// the supplement's Proj algorithm), FP64: kpp_factor_lsqr, kpp_proj_lsqr, kpp_solve_lsqr.
//
// The exact K++ step needs w = A_S^T (A_S A_S^T + lam I)^{-1} r, i.e. the argmin of |A_S w - r|^2 +
// lam |w|^2.  For large blocks the method instead runs a few LSQR iterations on the preconditioned
// system  M [w; v] = L^{-1} r,  M = L^{-1} [A_S, sqrt(lam) I],  with L L^T = Ahat Ahat^T + lam I and the
// sketch Ahat = A_S Pi^T of a subsampled randomized Hadamard transform:
//     Ahat = (A_S D H_{n'})[:, T] / sqrt(tau)      (n' = the power of 2 >= n, A_S padded with zeros;
//                                                   D = diag(d), d_i = +-1; T a tau-subset of [0, n'))
// The preconditioner of every block of the partition is memoised (a factor set of mode 2: L_j and
// L_j^{-1}).  The caller draws d and T.
//
// Factor phase (kpp_factor_lsqr): sketch_kernel forms Ahat for all rows (one CTA per row: the signed row
// in shared memory, the fast Walsh-Hadamard transform in place, the tau sampled entries), the library's
// FP64 block Grams give Ahat_j Ahat_j^T + lam I, and the library's Cholesky and inverse kernels give L_j
// and L_j^{-1}.
//
// Iteration (kpp_solve_lsqr, lsqr_kernel): a persistent cooperative kernel over column chunks of w and x
// (G CTAs, one group).  Each K++ step draws its block as the exact K++ does (Philox), forms r = A_S x -
// b_S, runs t_max LSQR iterations (Paige and Saunders' bidiagonalisation, ACM TOMS 8, 1982) from zero,
// and takes the first n entries of the LSQR solution as w in Alg. 1's momentum update; the window sums,
// checkpoints, stop rule and adaptive rho are Alg. 3's.  The s-vectors of the iteration (r, u, L^{-T} u,
// the v part of the unknowns) are replicated in every CTA's shared memory and computed in the same
// order everywhere; a product with A_S or A_S^T is split over the column chunks; a product with L^{-1}
// or L^{-T} is split by rows over the CTAs (entry i by CTA i mod G) and published.  Every exchange is a
// group barrier on a double-buffered array.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kpp_internal.cuh"
#include "kpp_launch.h"
#include "kpp_runtime.h"
#include "kpp_solve.h"

namespace kpp {

namespace {

constexpr int LT = 256;             // threads per CTA
constexpr int LW = LT / 32;
constexpr int LSQR_SMAX = 1024;     // block size at most (s-vectors in shared memory)
constexpr int64_t SKETCH_NMAX = 16384;  // padded row length at most (one row in shared memory)

// Ahat[row][q] = (A[row] * d, padded to np2, times H_np2)[T[q]] / sqrt(tau).  One CTA per row; the
// transform runs in shared memory, stage by stage from the widest butterfly down (Sylvester order).
__global__ void __launch_bounds__(256) sketch_kernel(const double *__restrict__ A, int64_t lda, int64_t rows,
                                                     int64_t n, int64_t np2, const double *__restrict__ d,
                                                     const int64_t *__restrict__ T, int64_t tau,
                                                     double *__restrict__ Ahat) {
    extern __shared__ double v[];  // np2
    const double sq = sqrt((double)tau);
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const double *ar = A + row * lda;
        for (int64_t k = threadIdx.x; k < np2; k += blockDim.x) v[k] = k < n ? ar[k] * d[k] : 0.0;
        __syncthreads();
        for (int64_t h = np2 >> 1; h >= 1; h >>= 1) {
            for (int64_t p = threadIdx.x; p < (np2 >> 1); p += blockDim.x) {
                const int64_t i = (p / h) * 2 * h + (p % h);  // i has bit h clear
                const double a = v[i], c = v[i + h];
                v[i] = a + c;
                v[i + h] = a - c;
            }
            __syncthreads();
        }
        for (int64_t q = threadIdx.x; q < tau; q += blockDim.x) Ahat[row * tau + q] = v[T[q]] / sq;
        __syncthreads();
    }
}

// B_j = A_j^T for nb blocks of s x s (one CTA per block at a time, 32 x 32 tiles through shared memory).
__global__ void transpose_blocks_kernel(const double *__restrict__ A, double *__restrict__ B, int64_t nb, int s) {
    __shared__ double tile[32][33];
    const int ntile = (s + 31) / 32;
    for (int64_t j = blockIdx.x; j < nb; j += gridDim.x) {
        const double *Aj = A + (size_t)j * s * s;
        double *Bj = B + (size_t)j * s * s;
        for (int tr = 0; tr < ntile; ++tr)
            for (int tc = 0; tc < ntile; ++tc) {
                for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
                    const int r = tr * 32 + e / 32, c = tc * 32 + e % 32;
                    tile[e / 32][e % 32] = (r < s && c < s) ? Aj[(size_t)r * s + c] : 0.0;
                }
                __syncthreads();
                for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
                    const int r = tc * 32 + e / 32, c = tr * 32 + e % 32;
                    if (r < s && c < s) Bj[(size_t)r * s + c] = tile[e % 32][e / 32];
                }
                __syncthreads();
            }
    }
}

struct LsqrScalars {  // the stopping rule's state (Alg. 3)
    double E0, E1, rhat, rho, bn2, res_est, res_true;
    long long ci, t;
    int active, status;
};

struct LsqrArgs {
    const double *A;        // m x n (leading dimension lda)
    int64_t lda;
    const double *b;        // m
    double *x, *mom;        // n
    const double *Linv;     // nb x s x s, L_j^{-1} (lower)
    const double *LinvT;    // nb x s x s, L_j^{-T} (upper)
    double *part;           // 2 x G x s: partials of a product with A_S over the column chunks
    double *pub;            // 2 x s: a published s-vector
    double *npart;          // 2 x G: partial squared norms
    double *vw, *wdw, *xw;  // n each: the w parts of the LSQR vectors v, w-bar and the solution
    double *rpart;          // G
    LsqrScalars *sc;
    unsigned *bar;
    int *err;
    int64_t m, n, nb, zeta, CW, count;
    int s, G, t_max, adaptive, confirm;
    uint64_t seed;
    uint32_t sys;
    double lam, eta, tol;
    uint64_t timeout_ns;
    // projection only (kpp_proj_lsqr): block proj_j, residual proj_r (s) -> proj_w (n); no K++ step
    int proj_only;
    int64_t proj_j;
    const double *proj_r;
    double *proj_w;
};

__global__ void __launch_bounds__(LT, 1) lsqr_kernel(const LsqrArgs a) {
    const int g = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = a.s, G = a.G;
    const int64_t n = a.n;
    const int64_t c0 = min64((int64_t)g * a.CW, n), c1 = min64(c0 + a.CW, n);
    const double sl = sqrt(a.lam);
    extern __shared__ double s_vecs[];  // 6 s-vectors (dynamic: up to 48 KiB at s = 1024)
    double *s_r = s_vecs, *s_u = s_vecs + s, *s_z = s_vecs + 2 * s;          // r, u, L^{-T} u (or M v)
    double *s_vv = s_vecs + 3 * s, *s_wv = s_vecs + 4 * s, *s_xv = s_vecs + 5 * s;  // v parts of v, w-bar, x
    __shared__ double s_red[LW][32];
    __shared__ double s_sum[LW];
    __shared__ LsqrScalars st;
    __shared__ int s_stop;
    double *__restrict__ x = a.x;
    double *__restrict__ mom = a.mom;
    double *__restrict__ vw = a.vw;
    double *__restrict__ wdw = a.wdw;
    double *__restrict__ xw = a.xw;
    GroupSync gs{a.bar, a.err, 0u, (unsigned)G, a.timeout_ns};
    unsigned pc = 0;  // exchanges so far: buffers alternate with its parity
    bool ok = true;

    // ---- exchanges (every CTA calls them in the same order; each ends in a group barrier) ----
    // y = A_S vsrc (+ add_scale * addv, + sub) of the block at As: partials over my columns, then row i
    // summed by CTA i mod G and published; out (shared, all s entries) in every CTA.
    auto product_AS = [&](const double *As, const double *vsrc, const double *addv, double add_scale,
                          const double *sub, double *out) -> bool {
        double *part = a.part + (size_t)(pc & 1) * G * s;
        // a thread per row: the row's entries on my columns share a few cache lines, and no shuffles
        for (int r = threadIdx.x; r < s; r += LT) {
            const double *row = As + (size_t)r * a.lda;
            double v0 = 0.0, v1 = 0.0;
            int64_t c = c0;
            for (; c + 1 < c1; c += 2) {
                v0 = fma(row[c], vsrc[c], v0);
                v1 = fma(row[c + 1], vsrc[c + 1], v1);
            }
            if (c < c1) v0 = fma(row[c], vsrc[c], v0);
            part[(size_t)g * s + r] = v0 + v1;
        }
        if (!group_barrier(gs)) return false;
        ++pc;
        double *pub = a.pub + (size_t)(pc & 1) * s;
        for (int r = g + G * warp; r < s; r += G * LW) {
            double v = 0.0;
            for (int h = lane; h < G; h += 32) v += __ldcg(part + (size_t)h * s + r);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) {
                if (addv) v += add_scale * addv[r];
                if (sub) v -= sub[r];
                pub[r] = v;
            }
        }
        if (!group_barrier(gs)) return false;
        ++pc;
        for (int r = threadIdx.x; r < s; r += LT) out[r] = __ldcg(pub + r);
        __syncthreads();
        return true;
    };
    // out = Lj^{-1} in (trans = false) or Lj^{-T} in (trans = true): entry i by CTA i mod G, published.
    // (Lj is L_j^{-1} for trans = false and L_j^{-T} for trans = true: a row either way)
    auto product_Linv = [&](const double *Lj, const double *in, double *out, bool trans) -> bool {
        double *pub = a.pub + (size_t)(pc & 1) * s;
        for (int i = g + G * warp; i < s; i += G * LW) {
            const double *row = Lj + (size_t)i * s;
            const int k0 = trans ? i : 0, k1 = trans ? s : i + 1;  // the nonzero part of the row
            double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
            int k = k0 + lane;
            for (; k + 96 < k1; k += 128) {
                v0 = fma(row[k], in[k], v0);
                v1 = fma(row[k + 32], in[k + 32], v1);
                v2 = fma(row[k + 64], in[k + 64], v2);
                v3 = fma(row[k + 96], in[k + 96], v3);
            }
            for (; k < k1; k += 32) v0 = fma(row[k], in[k], v0);
            double v = (v0 + v1) + (v2 + v3);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) pub[i] = v;
        }
        if (!group_barrier(gs)) return false;
        ++pc;
        for (int r = threadIdx.x; r < s; r += LT) out[r] = __ldcg(pub + r);
        __syncthreads();
        return true;
    };
    // |s-vector|^2, the same order in every CTA
    auto sq_s = [&](const double *v) -> double {
        double t = 0.0;
        for (int r = threadIdx.x; r < s; r += LT) t = fma(v[r], v[r], t);
        return block_sum<LT>(t, s_sum);
    };
    // |w part (column chunks)|^2 + |v part|^2 over the group, the same order in every CTA
    auto sq_nplus = [&](const double *w, const double *vpart, double &out) -> bool {
        double t = 0.0;
        for (int64_t c = c0 + threadIdx.x; c < c1; c += LT) t = fma(w[c], w[c], t);
        t = block_sum<LT>(t, s_sum);
        double *np = a.npart + (size_t)(pc & 1) * G;
        if (threadIdx.x == 0) np[g] = t;
        if (!group_barrier(gs)) return false;
        ++pc;
        // the G partials: warp 0, lanes strided then a fixed shuffle tree (the same order in every CTA)
        if (warp == 0) {
            double tot = 0.0;
            for (int h = lane; h < G; h += 32) tot += __ldcg(np + h);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
            if (lane == 0) s_red[0][0] = tot;
        }
        __syncthreads();
        const double tot = s_red[0][0];
        out = tot + sq_s(vpart);
        return true;
    };
    // dst = A_S^T z on my columns (warps over rows, lanes over columns, warp partials summed in order),
    // then dst = dst - sub_scale * sub (sub on my columns, may be null)
    auto product_AST = [&](const double *As, const double *z, double *dst, const double *sub, double sub_scale) {
        for (int64_t cb = c0; cb < c1; cb += 32) {
            const int64_t c = cb + lane;
            double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
            if (c < c1) {
                int r = warp;
                for (; r + 3 * LW < s; r += 4 * LW) {
                    v0 = fma(As[(size_t)r * a.lda + c], z[r], v0);
                    v1 = fma(As[(size_t)(r + LW) * a.lda + c], z[r + LW], v1);
                    v2 = fma(As[(size_t)(r + 2 * LW) * a.lda + c], z[r + 2 * LW], v2);
                    v3 = fma(As[(size_t)(r + 3 * LW) * a.lda + c], z[r + 3 * LW], v3);
                }
                for (; r < s; r += LW) v0 = fma(As[(size_t)r * a.lda + c], z[r], v0);
            }
            s_red[warp][lane] = (v0 + v1) + (v2 + v3);
            __syncthreads();
            if (warp == 0 && c < c1) {
                double t = 0.0;
#pragma unroll
                for (int w = 0; w < LW; ++w) t += s_red[w][lane];
                dst[c] = sub ? t - sub_scale * sub[c] : t;
            }
            __syncthreads();
        }
    };

    if (threadIdx.x == 0) {
        st = *a.sc;
        s_stop = 0;
    }
    __syncthreads();
    const int64_t steps = a.proj_only ? 1 : (st.active ? a.count : 0);
    int64_t t = st.t;
    for (int64_t q = 0; q < steps && ok; ++q) {
        const int64_t j = a.proj_only ? a.proj_j : (int64_t)draw_block(a.seed, t, a.sys, (int32_t)a.nb);
        const double *As = a.A + (size_t)j * s * a.lda;
        const double *Lj = a.Linv + (size_t)j * s * s;
        const double *LjT = a.LinvT + (size_t)j * s * s;
        // the next step's block: my columns of its rows and my rows of its L^{-1}, L^{-T} go to L2
        if (!a.proj_only && q + 1 < steps) {
            const int64_t jn = draw_block(a.seed, t + 1, a.sys, (int32_t)a.nb);
            const double *An = a.A + (size_t)jn * s * a.lda;
            for (int r = warp; r < s; r += LW)
                for (int64_t c = c0 + lane * 4; c < c1; c += 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(An + (size_t)r * a.lda + c));
            for (int i = g; i < s; i += G) {
                const double *l1 = a.Linv + ((size_t)jn * s + i) * s, *l2 = a.LinvT + ((size_t)jn * s + i) * s;
                for (int k = threadIdx.x * 4; k < s; k += LT * 4) {
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(l1 + k));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(l2 + k));
                }
            }
        }

        // ---- r = A_S x - b_S (or the given residual) ----
        double rn2 = 0.0;
        if (a.proj_only) {
            for (int r = threadIdx.x; r < s; r += LT) s_r[r] = a.proj_r[r];
            __syncthreads();
        } else {
            if (!(ok = product_AS(As, x, nullptr, 0.0, a.b + (size_t)j * s, s_r))) break;
            rn2 = sq_s(s_r);
        }

        // ---- LSQR on M [w; v] = L^{-1} r from zero, t_max iterations (as the oracle's Proj) ----
        for (int64_t c = c0 + threadIdx.x; c < c1; c += LT) xw[c] = 0.0;
        for (int r = threadIdx.x; r < s; r += LT) s_xv[r] = 0.0;
        if (!(ok = product_Linv(Lj, s_r, s_u, false))) break;  // u = L^{-1} r
        double beta = sqrt(sq_s(s_u));
        if (beta > 0.0) {
            for (int r = threadIdx.x; r < s; r += LT) s_u[r] /= beta;
            __syncthreads();
            // v = M^T u = [A_S^T z; sqrt(lam) z], z = L^{-T} u
            if (!(ok = product_Linv(LjT, s_u, s_z, true))) break;
            product_AST(As, s_z, vw, nullptr, 0.0);
            for (int r = threadIdx.x; r < s; r += LT) s_vv[r] = sl * s_z[r];
            __syncthreads();
            double alpha2 = 0.0;
            if (!(ok = sq_nplus(vw, s_vv, alpha2))) break;
            double alpha = sqrt(alpha2);
            if (alpha > 0.0) {
                for (int64_t c = c0 + threadIdx.x; c < c1; c += LT) {
                    vw[c] /= alpha;
                    wdw[c] = vw[c];
                }
                for (int r = threadIdx.x; r < s; r += LT) {
                    s_vv[r] /= alpha;
                    s_wv[r] = s_vv[r];
                }
                __syncthreads();
                double phibar = beta, rhobar = alpha;
                for (int it = 0; it < a.t_max; ++it) {
                    // u = M v - alpha u, M v = L^{-1} (A_S v_w + sqrt(lam) v_v)
                    if (!(ok = product_AS(As, vw, s_vv, sl, nullptr, s_z))) break;
                    if (!(ok = product_Linv(Lj, s_z, s_z, false))) break;
                    for (int r = threadIdx.x; r < s; r += LT) s_u[r] = s_z[r] - alpha * s_u[r];
                    __syncthreads();
                    beta = sqrt(sq_s(s_u));
                    if (beta > 0.0) {
                        for (int r = threadIdx.x; r < s; r += LT) s_u[r] /= beta;
                        __syncthreads();
                    }
                    // M^T u - beta v
                    if (!(ok = product_Linv(LjT, s_u, s_z, true))) break;
                    product_AST(As, s_z, vw, vw, beta);  // vw <- A_S^T z - beta vw (my columns)
                    for (int r = threadIdx.x; r < s; r += LT) s_vv[r] = sl * s_z[r] - beta * s_vv[r];
                    __syncthreads();
                    if (!(ok = sq_nplus(vw, s_vv, alpha2))) break;
                    alpha = sqrt(alpha2);
                    if (alpha > 0.0) {
                        for (int64_t c = c0 + threadIdx.x; c < c1; c += LT) vw[c] /= alpha;
                        for (int r = threadIdx.x; r < s; r += LT) s_vv[r] /= alpha;
                    }
                    const double rho = sqrt(rhobar * rhobar + beta * beta);
                    const double cs = rhobar / rho, sn = beta / rho;
                    const double theta = sn * alpha;
                    rhobar = -cs * alpha;
                    const double phi = cs * phibar;
                    phibar = sn * phibar;
                    for (int64_t c = c0 + threadIdx.x; c < c1; c += LT) {
                        xw[c] += (phi / rho) * wdw[c];
                        wdw[c] = vw[c] - (theta / rho) * wdw[c];
                    }
                    for (int r = threadIdx.x; r < s; r += LT) {
                        s_xv[r] += (phi / rho) * s_wv[r];
                        s_wv[r] = s_vv[r] - (theta / rho) * s_wv[r];
                    }
                    __syncthreads();
                    if (beta == 0.0 || alpha == 0.0) break;
                }
                if (!ok) break;
            }
        }

        if (a.proj_only) {
            for (int64_t c = c0 + threadIdx.x; c < c1; c += LT) a.proj_w[c] = xw[c];
            break;
        }
        // ---- the K++ update with w = the LSQR solution's first n entries (Alg. 1) ----
        const double bm = (1.0 - st.rho) / (1.0 + st.rho);
        for (int64_t c = c0 + threadIdx.x; c < c1; c += LT) {
            const double w = xw[c];
            const double mm = bm * (mom[c] - w);
            mom[c] = mm;
            x[c] = x[c] - w + a.eta * mm;
        }
        __syncthreads();
        const int64_t ph = t % (2 * a.zeta);
        if (threadIdx.x == 0) {
            if (ph < a.zeta) st.E0 += rn2;
            else st.E1 += rn2;
        }
        __syncthreads();
        t += 1;
        if (ph == 2 * a.zeta - 1) {
            // checkpoint (identical in every CTA); the stop is confirmed by the FP64 residual
            if (a.tol > 0.0 && st.E1 <= a.tol * a.tol * st.bn2 && a.confirm) {
                if (!(ok = group_barrier(gs))) break;
                double acc = 0.0;
                for (int64_t i = (int64_t)g + (int64_t)G * warp; i < a.m; i += (int64_t)G * LW) {
                    const double *row = a.A + (size_t)i * a.lda;
                    double v = 0.0;
                    for (int64_t c = lane; c < n; c += 32) v = fma(row[c], __ldcg(x + c), v);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    const double rr = v - a.b[i];
                    acc += rr * rr;
                }
                if (lane == 0) s_sum[warp] = acc;
                __syncthreads();
                if (threadIdx.x == 0) {
                    double tt = 0.0;
                    for (int w = 0; w < LW; ++w) tt += s_sum[w];
                    a.rpart[g] = tt;
                }
                if (!(ok = group_barrier(gs))) break;
                if (threadIdx.x == 0) {
                    double tt = 0.0;
                    for (int h = 0; h < G; ++h) tt += __ldcg(a.rpart + h);
                    st.res_true = st.bn2 > 0.0 ? sqrt(tt / st.bn2) : sqrt(tt);
                }
                if (!(ok = group_barrier(gs))) break;
            }
            if (threadIdx.x == 0) {
                st.ci += 1;
                st.res_est = st.bn2 > 0.0 ? sqrt(st.E1 / st.bn2) : sqrt(st.E1);
                if (!isfinite(st.E0) || !isfinite(st.E1)) {
                    st.status = KPP_ERR_NUMERIC;
                    st.active = 0;
                } else if (a.tol > 0.0 && st.E1 <= a.tol * a.tol * st.bn2 && (!a.confirm || st.res_true <= a.tol)) {
                    st.status = KPP_OK;
                    st.active = 0;
                } else {
                    if (a.adaptive) {
                        const double qq = st.E0 > 0.0 ? st.E1 / st.E0 : 0.0;
                        if (st.ci == 1) {
                            st.rhat = qq;
                        } else {
                            const double li = log((double)st.ci), li1 = log((double)st.ci + 1.0);
                            const double wgt = exp(li * li - li1 * li1);
                            st.rhat = wgt * st.rhat + (1.0 - wgt) * qq;
                        }
                        double rho = 1.0 - pow(st.rhat, 1.0 / (double)a.zeta);
                        if (!(rho > 0.0)) rho = 0.0;
                        if (rho > 1.0 - 1e-12) rho = 1.0 - 1e-12;
                        st.rho = rho;
                    }
                    st.E0 = 0.0;
                    st.E1 = 0.0;
                }
                s_stop = !st.active;
            }
            __syncthreads();
            if (s_stop) break;
        }
    }
    if (g == 0 && threadIdx.x == 0 && !a.proj_only) {
        st.t = t;
        *a.sc = st;
    }
}

}  // namespace

}  // namespace kpp

using namespace kpp;

extern "C" kpp_status kpp_factor_lsqr(const kpp_matrix *A, kpp_partition_t P, double lambda, int64_t tau,
                                      const int64_t *T, const double *d, kpp_factors_t *out, void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (out) *out = nullptr;
    if (!out || !P || !A || !A->data || A->dtype != KPP_F64 || A->rows != P->rows || A->cols < 1 ||
        A->ld < A->cols || P->s < 1 || P->s > LSQR_SMAX || A->rows % P->s || !(lambda >= 0.0) || !T || !d) {
        set_error("kpp_factor_lsqr: needs FP64 A with whole blocks of 1 <= s <= %d rows, lambda >= 0, T and d",
                  LSQR_SMAX);
        return KPP_ERR_ARG;
    }
    int64_t np2 = 1;
    while (np2 < A->cols) np2 *= 2;
    if (np2 > SKETCH_NMAX || tau < 1 || tau > np2) {
        set_error("kpp_factor_lsqr: the padded row length %lld exceeds %lld, or tau is not in [1, %lld]",
                  (long long)np2, (long long)SKETCH_NMAX, (long long)np2);
        return KPP_ERR_ARG;
    }
    for (int64_t q = 0; q < tau; ++q)
        if (T[q] < 0 || T[q] >= np2) {
            set_error("kpp_factor_lsqr: T[%lld] = %lld is outside [0, %lld)", (long long)q, (long long)T[q],
                      (long long)np2);
            return KPP_ERR_ARG;
        }
    const int s = P->s;
    const int64_t rows = A->rows, nb = rows / s;
    kpp_factors_t f = new kpp_factors_s;
    FactorSet &F = f->f;
    F.nb = nb;
    F.rows = rows;
    F.s = s;
    F.mode = 2;
    F.dtype = KPP_F64;
    F.lambda = lambda;
    F.bad_block = -1;
    F.memo_cols = A->cols;
    kpp_status rc = KPP_OK;
    int64_t *dT = nullptr;
    double *Ahat = nullptr, *G = nullptr, *Ginv = nullptr;
    const size_t blk = (size_t)s * s;
    const size_t smem = (size_t)np2 * sizeof(double);
    if (dev_malloc((void **)&F.L, nb * blk * sizeof(double)) != cudaSuccess ||
        dev_malloc((void **)&F.Linv, nb * blk * sizeof(double)) != cudaSuccess ||
        dev_malloc_async((void **)&dT, (size_t)tau * sizeof(int64_t), st) != cudaSuccess ||
        dev_malloc_async((void **)&Ahat, (size_t)rows * tau * sizeof(double), st) != cudaSuccess ||
        dev_malloc_async((void **)&G, nb * blk * sizeof(double), st) != cudaSuccess ||
        dev_malloc_async((void **)&Ginv, nb * blk * sizeof(double), st) != cudaSuccess) {
        rc = KPP_ERR_OOM;
        set_error("kpp_factor_lsqr: out of device memory");
    }
    if (rc == KPP_OK &&
        (cudaMemcpyAsync(dT, T, (size_t)tau * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaFuncSetAttribute(sketch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)) {
        rc = KPP_ERR_CUDA;
        set_error("kpp_factor_lsqr: set-up failed");
    }
    if (rc == KPP_OK) {
        note_launch();
        sketch_kernel<<<(unsigned)std::min<int64_t>(rows, 4 * (int64_t)sm_count()), 256, smem, st>>>(
            (const double *)A->data, A->ld, rows, A->cols, np2, d, dT, tau, Ahat);
        const kpp_matrix V{Ahat, KPP_F64, 0, rows, tau, tau};
        if (cudaGetLastError() != cudaSuccess || block_gram(V, s, lambda, G, 1, st) < 0) {
            rc = KPP_ERR_CUDA;
            set_error("kpp_factor_lsqr: sketch or Gram launch failed");
        }
    }
    if (rc == KPP_OK) {
        int64_t bad = -1;
        rc = factor_grams(G, nb, s, Ginv, &bad, st, F.L, F.Linv);  // synchronises st
        if (rc == KPP_ERR_NOT_SPD) {
            F.bad_block = bad;
            set_error("kpp_factor_lsqr: block %lld: sketched Gram not positive definite", (long long)bad);
        }
        if (rc == KPP_OK) {
            if (dev_malloc((void **)&F.LinvT, nb * blk * sizeof(double)) != cudaSuccess) {
                rc = KPP_ERR_OOM;
                set_error("kpp_factor_lsqr: out of device memory");
            } else {
                note_launch();
                transpose_blocks_kernel<<<(unsigned)std::min<int64_t>(nb, 4 * (int64_t)sm_count()), 256, 0, st>>>(
                    F.Linv, F.LinvT, nb, s);
                if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
                    rc = KPP_ERR_CUDA;
                    set_error("kpp_factor_lsqr: transpose failed");
                }
            }
        }
    }
    if (dT) cudaFreeAsync(dT, st);
    if (Ahat) cudaFreeAsync(Ahat, st);
    if (G) cudaFreeAsync(G, st);
    if (Ginv) cudaFreeAsync(Ginv, st);
    if (rc != KPP_OK && rc != KPP_ERR_NOT_SPD) {
        F.release();
        delete f;
        return rc;
    }
    *out = f;
    return rc;
}

namespace kpp {
namespace {

// Launch lsqr_kernel once (all scratch on the stream, freed at return); `sc` in/out on the host.
kpp_status lsqr_launch(const kpp_matrix &A, const double *b, double *x, const FactorSet &F, LsqrArgs a,
                       LsqrScalars &sc, float *ms, cudaStream_t st) {
    kpp_status rc = KPP_OK;
    Scratch scr(st);
    const int64_t n = A.cols;
    // every SM: a step's products with A_S and A_S^T are FP64 FMAs on the columns, and GB300's FP64 pipe
    // is narrow, so they are spread as widely as the columns allow (at least 8 per CTA)
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(sm_count(), (n + 7) / 8));
    const int s = F.s;
    a.A = (const double *)A.data;
    a.lda = A.ld;
    a.b = b;
    a.x = x;
    a.Linv = F.Linv;
    a.LinvT = F.LinvT;
    a.m = A.rows;
    a.n = n;
    a.nb = F.nb;
    a.zeta = F.nb;
    a.G = G;
    a.CW = (n + G - 1) / G;
    a.s = s;
    a.lam = F.lambda;
    a.timeout_ns = 2000000000ull;
    int herr = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int per_sm = 0;
    const size_t smem = (size_t)6 * s * sizeof(double);
    CUDA_OR(cudaFuncSetAttribute(lsqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), KPP_ERR_CUDA);
    CUDA_OR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lsqr_kernel, LT, smem), KPP_ERR_CUDA);
    if (per_sm * sm_count() < G) {
        set_error("lsqr: %d CTAs do not fit co-resident", G);
        return KPP_ERR_UNSUPPORTED;
    }
    CUDA_OR(scr.alloc((void **)&a.mom, (size_t)n * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.part, (size_t)2 * G * s * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.pub, (size_t)2 * s * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.npart, (size_t)2 * G * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.vw, (size_t)n * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.wdw, (size_t)n * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.xw, (size_t)n * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.rpart, (size_t)G * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.sc, sizeof(LsqrScalars)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.bar, sizeof(unsigned)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&a.err, sizeof(int)), KPP_ERR_CUDA);
    CUDA_OR(cudaMemsetAsync(a.mom, 0, (size_t)n * sizeof(double), st), KPP_ERR_CUDA);
    CUDA_OR(cudaMemsetAsync(a.bar, 0, sizeof(unsigned), st), KPP_ERR_CUDA);
    CUDA_OR(cudaMemsetAsync(a.err, 0, sizeof(int), st), KPP_ERR_CUDA);
    CUDA_OR(cudaMemcpyAsync(a.sc, &sc, sizeof(LsqrScalars), cudaMemcpyHostToDevice, st), KPP_ERR_CUDA);
    CUDA_OR(cudaEventCreate(&e0), KPP_ERR_CUDA);
    CUDA_OR(cudaEventCreate(&e1), KPP_ERR_CUDA);
    {
        void *args[] = {(void *)&a};
        CUDA_OR(cudaEventRecord(e0, st), KPP_ERR_CUDA);
        note_launch();
        CUDA_OR(cudaLaunchCooperativeKernel((const void *)lsqr_kernel, dim3((unsigned)G), dim3(LT), args, smem, st),
                KPP_ERR_CUDA);
        CUDA_OR(cudaEventRecord(e1, st), KPP_ERR_CUDA);
        CUDA_OR(cudaMemcpyAsync(&sc, a.sc, sizeof(LsqrScalars), cudaMemcpyDeviceToHost, st), KPP_ERR_CUDA);
        CUDA_OR(cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, st), KPP_ERR_CUDA);
        CUDA_OR(cudaStreamSynchronize(st), KPP_ERR_CUDA);
        if (ms) cudaEventElapsedTime(ms, e0, e1);
    }
    if (herr) {
        rc = (kpp_status)herr;
        set_error("lsqr: device error %s", kpp_status_string(rc));
    }
cleanup:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

bool lsqr_factors_ok(const kpp_matrix *A, kpp_partition_t P, kpp_factors_t F) {
    return A && A->data && P && F && A->dtype == KPP_F64 && A->ld >= A->cols && F->f.mode == 2 && F->f.Linv &&
           F->f.LinvT &&
           F->f.rows == A->rows && P->rows == A->rows && P->s == F->f.s && F->f.memo_cols == A->cols &&
           F->f.bad_block < 0;
}

}  // namespace
}  // namespace kpp

extern "C" kpp_status kpp_proj_lsqr(const kpp_matrix *A, kpp_partition_t P, kpp_factors_t F, int64_t j,
                                    const double *r, int32_t t_max, double *w, void *stream) {
    clear_error();
    if (!lsqr_factors_ok(A, P, F) || j < 0 || j >= F->f.nb || !r || !w || t_max < 1) {
        set_error("kpp_proj_lsqr: needs FP64 A, its partition, LSQR factors of it (kpp_factor_lsqr), a block "
                  "index, r, w and t_max >= 1");
        return KPP_ERR_ARG;
    }
    LsqrArgs a{};
    a.t_max = t_max;
    a.proj_only = 1;
    a.proj_j = j;
    a.proj_r = r;
    a.proj_w = w;
    LsqrScalars sc{};
    sc.active = 1;
    return lsqr_launch(*A, nullptr, nullptr, F->f, a, sc, nullptr, (cudaStream_t)stream);
}

extern "C" kpp_status kpp_solve_lsqr(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P,
                                     kpp_factors_t F, int32_t t_max, const kpp_params *pp, kpp_report *rep,
                                     void *stream) {
    clear_error();
    if (!lsqr_factors_ok(A, P, F) || !b || !x || !pp || t_max < 1 || pp->max_iters < 0 ||
        std::fabs(pp->lambda - F->f.lambda) > 1e-15 * std::max(1.0, std::fabs(pp->lambda))) {
        set_error("kpp_solve_lsqr: needs FP64 A, its partition, LSQR factors of it with p->lambda, b, x, p and "
                  "t_max >= 1");
        return KPP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const kpp_params p = *pp;
    LsqrScalars sc{};
    {
        std::vector<double> r2, b2;
        kpp_status rb = residual_norms(*A, 1, b, x, nullptr, r2, &b2, st);
        if (rb != KPP_OK) return rb;
        sc.bn2 = b2[0];
    }
    sc.rho = p.rho0;
    sc.active = 1;
    sc.status = KPP_ERR_NO_CONVERGENCE;
    sc.res_est = NAN;
    sc.res_true = NAN;
    LsqrArgs a{};
    a.t_max = t_max;
    a.count = p.max_iters;
    a.seed = p.seed;
    a.sys = p.sys_id;
    a.adaptive = p.adaptive_rho;
    a.confirm = 1;
    a.eta = default_eta(p, F->f.s, A->rows, A->cols);
    a.tol = p.tol;
    float ms = 0.f;
    kpp_status rc = lsqr_launch(*A, b, x, F->f, a, sc, &ms, st);
    if (rc != KPP_OK) return rc;
    std::vector<double> r2, b2;
    rc = residual_norms(*A, 1, b, x, nullptr, r2, &b2, st);
    if (rc != KPP_OK) return rc;
    const double rel = b2[0] > 0 ? std::sqrt(r2[0] / b2[0]) : std::sqrt(r2[0]);
    kpp_status status = (kpp_status)sc.status;
    if (status == KPP_OK && !std::isfinite(rel)) status = KPP_ERR_NUMERIC;
    if (rep) {
        memset(rep, 0, sizeof(*rep));
        rep->iters = sc.t;
        rep->rel_res_true = rel;
        rep->rel_res_est = sc.res_est;
        rep->rho_final = sc.rho;
        rep->status = status;
        rep->bad_block = -1;
        rep->device_ms = ms;
        rep->kernel_ms = ms;
        rep->launches = 1;
    }
    if (status != KPP_OK) set_error("kpp_solve_lsqr: solve ended with %s", kpp_status_string(status));
    return status;
}
