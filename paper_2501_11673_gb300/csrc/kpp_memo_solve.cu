// kpp_memo_solve.cu -- K++ and CD++ with the online block memoisation on the GPU (kpp_solve_memo;
// Sec. 4 "Block memoization", Sec. 5.2, the sampling steps of Alg. 3 and Alg. 5), FP64.
//
// Step t either samples a new uniformly random s-subset S of the rows (with probability p_t) and
// memoises the factor of its block, or reuses a memoised block picked uniformly; kpp_memo.cuh has the
// draws.  The block sequence depends only on (seed, t, system), never on the data, so the solve runs
// in windows of steps:
//   1. the host draws the window: each step's memo index and the subsets of the new blocks;
//   2. the new subsets' rows of A and b are gathered into a growing device store (memo block j = stored
//      rows j s .. j s + s - 1), their Grams formed (K++: A_S A_S^T + lam I; CD++: A_SS + lam I) and
//      factored in one batch by the library's FP64 Cholesky and inverse kernels; G_j^{-1} is kept;
//   3. memo_kernel runs the window's steps.
// The iterate, the momentum and the scalars of the stopping rule stay on the device between windows,
// so the windows do not change the trajectory.
//
// memo_kernel is a persistent cooperative kernel over column chunks of x (G CTAs, one group):
//   a. partial block residual over my columns, sum_c A_S[a][c] x_c, into a double-buffered array;
//      group barrier;
//   b. row i of r = A_S x - b_S is summed from the partials by CTA i mod G and published; group barrier;
//      every CTA reads r and forms |r|^2 (same order everywhere); y = G_j^{-1} r -- K++: row i by
//      CTA i mod G, published, one more group barrier; CD++: each CTA forms only the entries whose rows
//      are its columns.  (Every CTA reading all partials, or all of G_j^{-1}, made their L2 lines hot
//      spots that 128 SMs queued on.)  The next block's rows on my columns are prefetched to L2;
//   c. w on my columns -- K++: w = A_S^T y; CD++: w_{S[a]} = y_a and 0 elsewhere (the subset is sorted,
//      so a binary search finds my columns in it) -- then m <- beta (m - w), x <- x - w + eta m;
//   d. the window sums, and at a checkpoint the stop test (confirmed by the FP64 residual of the whole
//      system, which takes three more group barriers) and the adaptive rho (Eq. 5.2 - 5.3).
// Every CTA takes the same decisions from the same values.  Indices that come from the host tables are
// checked: a bad one is reported (KPP_ERR_ARG), never followed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kpp_internal.cuh"
#include "kpp_launch.h"
#include "kpp_memo.cuh"
#include "kpp_runtime.h"
#include "kpp_solve.h"

namespace kpp {

namespace {

constexpr int MT = 256;            // threads per CTA
constexpr int MW = MT / 32;
constexpr int MEMO_SMAX = 1024;    // block size at most (r and y in shared memory)

struct MemoScalars {  // the stopping rule's state (Alg. 3), one system
    double E0, E1, rhat, rho, bn2, res_est, res_true;
    long long ci, t;
    int active, status;
};

struct MemoArgs {
    const double *Ag;      // stored rows (nbm s x n)
    const double *bg;      // their entries of b (nbm s)
    const double *Ginv;    // nbm x s x s
    const int64_t *S;      // CD++: the rows of each block (nbm s), ascending per block
    const int32_t *blocks; // the window's memo indices (count)
    const double *A;       // the system (m x n, leading dimension lda): the confirming residual
    int64_t lda;
    const double *b;       // m
    double *x, *mom;       // n
    double *part;          // 2 x G x s
    double *rbuf, *ybuf;   // 2 x s each: r and (K++) y of the step, published by their owners
    double *rpart;         // G
    MemoScalars *sc;
    unsigned *bar;
    int *err;
    int64_t m, n, nbm, t_win, count, zeta;
    int64_t CW;            // columns per CTA
    int s, G, cd, adaptive, confirm;
    double eta, tol;
    uint64_t timeout_ns;
};

__global__ void __launch_bounds__(MT, 1) memo_kernel(const MemoArgs a) {
    const int g = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = a.s;
    const int64_t n = a.n;
    const int64_t c0 = min64((int64_t)g * a.CW, n), c1 = min64(c0 + a.CW, n);
    __shared__ double s_r[MEMO_SMAX], s_y[MEMO_SMAX];
    __shared__ int64_t s_S[MEMO_SMAX];  // CD++: the block's rows
    __shared__ double s_red[MW];
    __shared__ MemoScalars st;
    __shared__ int s_stop;
    GroupSync gs{a.bar, a.err, 0u, (unsigned)a.G, a.timeout_ns};
    double *__restrict__ x = a.x;
    double *__restrict__ mom = a.mom;
    const double *__restrict__ bg = a.bg;

    if (threadIdx.x == 0) {
        st = *a.sc;
        s_stop = 0;
    }
    __syncthreads();
    const int64_t t_end = st.active ? st.t + a.count : st.t;
    int64_t t = st.t;
    while (t < t_end) {
        // ---- the block of step t ----
        const int64_t ti = t - a.t_win;
        const int64_t j = (ti >= 0 && ti < a.count) ? (int64_t)a.blocks[ti] : -1;
        if (j < 0 || j >= a.nbm) {  // a host table error: reported, not followed
            if (threadIdx.x == 0) group_fail(gs, KPP_ERR_ARG);
            break;
        }
        const double *__restrict__ As = a.Ag + (size_t)j * s * n;
        const double *__restrict__ Gj = a.Ginv + (size_t)j * s * s;
        double *part = a.part + (size_t)(t & 1) * a.G * s;

        // a. my partial of r: a thread per row (the row's entries on my columns share a few cache lines)
        for (int r = threadIdx.x; r < s; r += MT) {
            const double *row = As + (size_t)r * n;
            double v0 = 0.0, v1 = 0.0;
            int64_t c = c0;
            for (; c + 1 < c1; c += 2) {
                v0 = fma(row[c], x[c], v0);
                v1 = fma(row[c + 1], x[c + 1], v1);
            }
            if (c < c1) v0 = fma(row[c], x[c], v0);
            part[(size_t)g * s + r] = v0 + v1;
        }
        if (!group_barrier(gs)) break;

        // b. r: row i of r is formed by CTA i mod G (a warp per row, lanes over the G partials, a fixed
        // shuffle tree) and published; no two CTAs read the same partials, so no L2 line is a hot spot
        double *rb = a.rbuf + (size_t)(t & 1) * s;
        double *yb = a.ybuf + (size_t)(t & 1) * s;
        for (int r = g + a.G * warp; r < s; r += a.G * MW) {
            double v = 0.0;
            for (int h = lane; h < a.G; h += 32) v += __ldcg(part + (size_t)h * s + r);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) rb[r] = v - bg[(size_t)j * s + r];
        }
        // the block of the next step: its rows on my columns go to L2 while this step finishes
        if (ti + 1 < a.count) {
            const int64_t jn = a.blocks[ti + 1];
            if (jn >= 0 && jn < a.nbm) {
                const double *An = a.Ag + (size_t)jn * s * n;
                for (int r = warp; r < s; r += MW)
                    for (int64_t c = c0 + lane * 4; c < c1; c += 128)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(An + (size_t)r * n + c));
            }
        }
        if (!group_barrier(gs)) break;
        for (int r = threadIdx.x; r < s; r += MT) {
            s_r[r] = __ldcg(rb + r);
            if (a.cd) s_S[r] = a.S[(size_t)j * s + r];
        }
        __syncthreads();
        // |r|^2 (every CTA, the same order)
        double rn2 = 0.0;
        if (warp == 0) {
            for (int r = lane; r < s; r += 32) rn2 = fma(s_r[r], s_r[r], rn2);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rn2 += __shfl_xor_sync(0xffffffffu, rn2, o);
        }
        // y = G_j^{-1} r: K++ needs all of y (row i formed by CTA i mod G and published, one more group
        // barrier); CD++ only the entries whose rows S[i] are my columns, formed here
        if (!a.cd) {
            for (int r = g + a.G * warp; r < s; r += a.G * MW) {
                double v = 0.0;
                for (int d = lane; d < s; d += 32) v = fma(Gj[(size_t)r * s + d], s_r[d], v);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) yb[r] = v;
            }
            if (!group_barrier(gs)) break;
            for (int r = threadIdx.x; r < s; r += MT) s_y[r] = __ldcg(yb + r);
        } else {
            for (int r = warp; r < s; r += MW) {
                if (s_S[r] < c0 || s_S[r] >= c1) continue;  // uniform over the warp
                double v = 0.0;
                for (int d = lane; d < s; d += 32) v = fma(Gj[(size_t)r * s + d], s_r[d], v);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) s_y[r] = v;
            }
        }
        if (threadIdx.x == 0 && st.active) {
            const int64_t ph = t % (2 * a.zeta);
            if (ph < a.zeta) st.E0 += rn2;
            else st.E1 += rn2;
        }
        __syncthreads();

        // c. w on my columns, then m and x
        const double beta = (1.0 - st.rho) / (1.0 + st.rho);
        if (st.active) {
            for (int64_t c = c0 + threadIdx.x; c < c1; c += MT) {
                double w = 0.0;
                if (!a.cd) {
                    for (int r = 0; r < s; ++r) w = fma(As[(size_t)r * n + c], s_y[r], w);
                } else {
                    int lo = 0, hi = s;  // first index with Sj[idx] >= c
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (s_S[mid] < c) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo < s && s_S[lo] == c) w = s_y[lo];
                }
                const double mm = beta * (mom[c] - w);
                mom[c] = mm;
                x[c] = x[c] - w + a.eta * mm;
            }
        }
        __syncthreads();  // the next partial reads my chunk of x through other threads

        // d. checkpoint (identical in every CTA)
        const int64_t ph = t % (2 * a.zeta);
        t += 1;
        if (ph == 2 * a.zeta - 1 && st.active) {
            const bool need = a.tol > 0.0 && st.E1 <= a.tol * a.tol * st.bn2 && a.confirm;
            if (need) {
                // the FP64 residual of the whole system: x must be complete in every chunk
                if (!group_barrier(gs)) break;
                double acc = 0.0;
                for (int64_t i = (int64_t)g + (int64_t)a.G * warp; i < a.m; i += (int64_t)a.G * MW) {
                    const double *row = a.A + (size_t)i * a.lda;
                    double v = 0.0;
                    for (int64_t c = lane; c < n; c += 32) v = fma(row[c], __ldcg(a.x + c), v);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    const double rr = v - a.b[i];
                    acc += rr * rr;  // every lane holds the row's value; lane 0's sum is used
                }
                if (lane == 0) s_red[warp] = acc;
                __syncthreads();
                if (threadIdx.x == 0) {
                    double tt = 0.0;
                    for (int w = 0; w < MW; ++w) tt += s_red[w];
                    a.rpart[g] = tt;
                }
                if (!group_barrier(gs)) break;
                if (threadIdx.x == 0) {
                    double tt = 0.0;
                    for (int h = 0; h < a.G; ++h) tt += __ldcg(a.rpart + h);
                    st.res_true = st.bn2 > 0.0 ? sqrt(tt / st.bn2) : sqrt(tt);
                }
                // every CTA has read the partials before a later checkpoint writes them again
                if (!group_barrier(gs)) break;
            }
            if (threadIdx.x == 0) {
                st.ci += 1;
                st.res_est = st.bn2 > 0.0 ? sqrt(st.E1 / st.bn2) : sqrt(st.E1);
                if (!isfinite(st.E0) || !isfinite(st.E1)) {
                    st.status = KPP_ERR_NUMERIC;
                    st.active = 0;
                } else if (a.tol > 0.0 && st.E1 <= a.tol * a.tol * st.bn2 &&
                           (!a.confirm || st.res_true <= a.tol)) {
                    st.status = KPP_OK;
                    st.active = 0;
                } else if (a.adaptive) {
                    const double q = st.E0 > 0.0 ? st.E1 / st.E0 : 0.0;
                    if (st.ci == 1) {
                        st.rhat = q;
                    } else {
                        const double li = log((double)st.ci), li1 = log((double)st.ci + 1.0);
                        const double wgt = exp(li * li - li1 * li1);
                        st.rhat = wgt * st.rhat + (1.0 - wgt) * q;
                    }
                    double rho = 1.0 - pow(st.rhat, 1.0 / (double)a.zeta);
                    if (!(rho > 0.0)) rho = 0.0;
                    if (rho > 1.0 - 1e-12) rho = 1.0 - 1e-12;
                    st.rho = rho;
                }
                st.E0 = 0.0;
                st.E1 = 0.0;
                s_stop = !st.active;
            }
            __syncthreads();
            if (s_stop) break;
        }
    }
    if (g == 0 && threadIdx.x == 0) {
        st.t = t;
        *a.sc = st;
    }
}

// Stored row r (of cnt) = A[idx[r]], with b; one CTA per row at a time.  A row index outside the
// matrix sets the error word and is skipped.
__global__ void memo_gather_kernel(const double *__restrict__ A, int64_t lda, const double *__restrict__ b,
                                   const int64_t *__restrict__ idx, int64_t cnt, int64_t n, int64_t m,
                                   double *__restrict__ Ag, double *__restrict__ bg, int *__restrict__ err) {
    for (int64_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const int64_t src = idx[r];
        if (src < 0 || src >= m) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            continue;
        }
        for (int64_t c = threadIdx.x; c < n; c += blockDim.x) Ag[r * n + c] = A[src * lda + c];
        if (threadIdx.x == 0) bg[r] = b[src];
    }
}

// CD++: G_i = A[S_i, S_i] + lam I for nblk new blocks (S_i = idx[i s .. i s + s - 1]); one CTA per block.
__global__ void memo_principal_kernel(const double *__restrict__ A, int64_t lda, const int64_t *__restrict__ idx,
                                      int64_t nblk, int s, int64_t m, double lam, double *__restrict__ G,
                                      int *__restrict__ err) {
    for (int64_t i = blockIdx.x; i < nblk; i += gridDim.x) {
        const int64_t *S = idx + i * s;
        double *Gi = G + (size_t)i * s * s;
        for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
            const int p = e / s, q = e % s;
            const int64_t r = S[p], c = S[q];
            if (r < 0 || r >= m || c < 0 || c >= m) {
                atomicExch(err, 1);
                Gi[e] = 0.0;
                continue;
            }
            Gi[e] = A[r * lda + c] + (p == q ? lam : 0.0);
        }
    }
}

// The memo's device store: grows by doubling, contents copied on the stream.
struct MemoStore {
    int64_t cap = 0, n = 0;
    int s = 0;
    double *Ag = nullptr, *bg = nullptr, *Ginv = nullptr;
    int64_t *S = nullptr;
    void release(cudaStream_t st) {
        if (Ag) cudaFreeAsync(Ag, st);
        if (bg) cudaFreeAsync(bg, st);
        if (Ginv) cudaFreeAsync(Ginv, st);
        if (S) cudaFreeAsync(S, st);
        Ag = bg = Ginv = nullptr;
        S = nullptr;
        cap = 0;
    }
    // room for `want` blocks, keeping the first `used`
    kpp_status reserve(int64_t want, int64_t used, cudaStream_t st) {
        if (want <= cap) return KPP_OK;
        int64_t nc = cap > 0 ? cap : 64;
        while (nc < want) nc *= 2;
        const size_t rs = (size_t)nc * s, blk = (size_t)s * s;
        double *nAg = nullptr, *nbg = nullptr, *nG = nullptr;
        int64_t *nS = nullptr;
        bool ok = dev_malloc_async((void **)&nAg, rs * n * sizeof(double), st) == cudaSuccess &&
                  dev_malloc_async((void **)&nbg, rs * sizeof(double), st) == cudaSuccess &&
                  dev_malloc_async((void **)&nG, (size_t)nc * blk * sizeof(double), st) == cudaSuccess &&
                  dev_malloc_async((void **)&nS, rs * sizeof(int64_t), st) == cudaSuccess;
        if (ok && used > 0) {
            const size_t ur = (size_t)used * s;
            ok = cudaMemcpyAsync(nAg, Ag, ur * n * sizeof(double), cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
                 cudaMemcpyAsync(nbg, bg, ur * sizeof(double), cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
                 cudaMemcpyAsync(nG, Ginv, (size_t)used * blk * sizeof(double), cudaMemcpyDeviceToDevice, st) ==
                     cudaSuccess &&
                 cudaMemcpyAsync(nS, S, ur * sizeof(int64_t), cudaMemcpyDeviceToDevice, st) == cudaSuccess;
        }
        if (!ok) {
            cudaGetLastError();
            for (void *p : {(void *)nAg, (void *)nbg, (void *)nG, (void *)nS})
                if (p) cudaFreeAsync(p, st);
            set_error("kpp_solve_memo: no device memory for %lld memoised blocks", (long long)nc);
            return KPP_ERR_OOM;
        }
        release(st);
        Ag = nAg;
        bg = nbg;
        Ginv = nG;
        S = nS;
        cap = nc;
        return KPP_OK;
    }
};

}  // namespace

static kpp_status memo_solve(const kpp_matrix *A, const double *b, double *x, int s, int cd, const kpp_params *pp,
                             kpp_report *rep, int64_t *nblocks_out, cudaStream_t st) {
    clear_error();
    if (!A || !A->data || !b || !x || !pp || A->dtype != KPP_F64 || A->rows < 1 || A->cols < 1 ||
        A->ld < A->cols || s < 1 || s > MEMO_SMAX || s > A->rows || (cd && A->rows != A->cols) ||
        !(pp->lambda >= 0.0) || pp->max_iters < 0) {
        set_error("kpp_solve_memo: needs FP64 A (square for CD++), 1 <= s <= min(rows, %d), lambda >= 0, "
                  "max_iters >= 0, non-null b, x, p", MEMO_SMAX);
        return KPP_ERR_ARG;
    }
    const kpp_params p = *pp;
    const int64_t m = A->rows, n = A->cols;
    const int64_t zeta = (m + s - 1) / s;
    const int64_t W = std::max<int64_t>(256, std::min<int64_t>(16 * zeta, 8192));  // steps per window
    const double eta = default_eta(p, s, m, n);
    const int G = auto_grid(n, 1);
    const int64_t CW = (n + G - 1) / G;
    kpp_status rc = KPP_OK;
    Scratch scr(st);
    MemoStore ms;
    ms.n = n;
    ms.s = s;
    double *mom = nullptr, *part = nullptr, *rpart = nullptr, *Gnew = nullptr, *rbuf = nullptr, *ybuf = nullptr;
    MemoScalars *d_sc = nullptr;
    unsigned *bar = nullptr;
    int *err = nullptr, *gerr = nullptr;
    int32_t *dblocks = nullptr;
    int64_t *d_new = nullptr;
    std::vector<int32_t> blocks_h((size_t)W);
    std::vector<int64_t> nb_after((size_t)W);  // blocks memoised once step i of the window has drawn
    std::vector<int64_t> subsets_h((size_t)W * s);
    int64_t t = 0, nb = 0, nb_used = 0, bad = -1, launches = 0;
    float kms_total = 0.f;
    MemoScalars sc{};
    {
        std::vector<double> r2, b2;
        rc = residual_norms(*A, 1, b, x, nullptr, r2, &b2, st);
        if (rc != KPP_OK) return rc;
        sc.bn2 = b2[0];
    }
    sc.rho = p.rho0;
    sc.active = 1;
    sc.status = KPP_ERR_NO_CONVERGENCE;
    sc.res_est = NAN;
    sc.res_true = NAN;
    CUDA_OR(scr.alloc((void **)&mom, (size_t)n * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&part, (size_t)2 * G * s * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&rpart, (size_t)G * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&rbuf, (size_t)2 * s * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&ybuf, (size_t)2 * s * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&d_sc, sizeof(MemoScalars)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&bar, sizeof(unsigned)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&err, sizeof(int)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&gerr, sizeof(int)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&dblocks, (size_t)W * sizeof(int32_t)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&d_new, (size_t)W * s * sizeof(int64_t)), KPP_ERR_CUDA);
    CUDA_OR(cudaMemsetAsync(mom, 0, (size_t)n * sizeof(double), st), KPP_ERR_CUDA);
    CUDA_OR(cudaMemsetAsync(gerr, 0, sizeof(int), st), KPP_ERR_CUDA);
    CUDA_OR(cudaMemcpyAsync(d_sc, &sc, sizeof(MemoScalars), cudaMemcpyHostToDevice, st), KPP_ERR_CUDA);
    while (t < p.max_iters) {
        const int64_t count = std::min<int64_t>(W, p.max_iters - t);
        // 1. the window's draws (data-independent)
        int64_t nb2 = nb;
        for (int64_t i = 0; i < count; ++i) {
            int64_t j = memo_pick(p.seed, t + i, p.sys_id, cd, m, n, s, nb2);
            if (j < 0) {
                memo_subset(p.seed, t + i, p.sys_id, m, s, subsets_h.data() + (size_t)(nb2 - nb) * s);
                j = nb2++;
            }
            blocks_h[(size_t)i] = (int32_t)j;
            nb_after[(size_t)i] = nb2;
        }
        if (nb2 > 0x7fffffffLL) {
            rc = KPP_ERR_UNSUPPORTED;
            set_error("kpp_solve_memo: more than 2^31 memoised blocks");
            goto cleanup;
        }
        // 2. gather and factor the new blocks
        if (nb2 > nb) {
            const int64_t newc = nb2 - nb;
            rc = ms.reserve(nb2, nb, st);
            if (rc != KPP_OK) goto cleanup;
            CUDA_OR(cudaMemcpyAsync(d_new, subsets_h.data(), (size_t)newc * s * sizeof(int64_t), cudaMemcpyHostToDevice,
                                    st),
                    KPP_ERR_CUDA);
            CUDA_OR(cudaMemcpyAsync(ms.S + (size_t)nb * s, d_new, (size_t)newc * s * sizeof(int64_t),
                                    cudaMemcpyDeviceToDevice, st),
                    KPP_ERR_CUDA);
            double *Ag_new = ms.Ag + (size_t)nb * s * n;
            note_launch();
            memo_gather_kernel<<<(unsigned)std::min<int64_t>(newc * s, 65535), 256, 0, st>>>(
                (const double *)A->data, A->ld, b, d_new, newc * s, n, m, Ag_new, ms.bg + (size_t)nb * s, gerr);
            CUDA_OR(cudaGetLastError(), KPP_ERR_CUDA);
            CUDA_OR(dev_malloc_async((void **)&Gnew, (size_t)newc * s * s * sizeof(double), st), KPP_ERR_OOM);
            if (cd) {
                note_launch();
                memo_principal_kernel<<<(unsigned)std::min<int64_t>(newc, 65535), 256, 0, st>>>(
                    (const double *)A->data, A->ld, d_new, newc, s, m, p.lambda, Gnew, gerr);
                CUDA_OR(cudaGetLastError(), KPP_ERR_CUDA);
            } else {
                // the stored rows of the new blocks are whole blocks of a row-major matrix: the library's Grams
                const kpp_matrix V{Ag_new, KPP_F64, 0, newc * s, n, n};
                if (block_gram(V, s, p.lambda, Gnew, 1, st) < 0) {
                    rc = KPP_ERR_CUDA;
                    set_error("kpp_solve_memo: block Gram launch failed");
                    goto cleanup;
                }
            }
            int64_t bad_new = -1;
            rc = factor_grams(Gnew, newc, s, ms.Ginv + (size_t)nb * s * s, &bad_new, st);  // synchronises st
            cudaFreeAsync(Gnew, st);
            Gnew = nullptr;
            {
                int herr = 0;
                if (cudaMemcpyAsync(&herr, gerr, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess) {
                    rc = KPP_ERR_CUDA;
                    goto cleanup;
                }
                if (herr) {
                    rc = KPP_ERR_ARG;
                    set_error("kpp_solve_memo: a drawn row index is outside the matrix");
                    goto cleanup;
                }
            }
            if (rc != KPP_OK) {
                if (rc == KPP_ERR_NOT_SPD) {
                    bad = nb + bad_new;
                    set_error("kpp_solve_memo: memoised block %lld: Cholesky pivot not positive", (long long)bad);
                }
                goto cleanup;
            }
            nb = nb2;
        }
        CUDA_OR(cudaMemcpyAsync(dblocks, blocks_h.data(), (size_t)count * sizeof(int32_t), cudaMemcpyHostToDevice, st),
                KPP_ERR_CUDA);
        // 3. the window's steps
        {
            MemoArgs a{};
            a.Ag = ms.Ag;
            a.bg = ms.bg;
            a.Ginv = ms.Ginv;
            a.S = cd ? ms.S : nullptr;
            a.blocks = dblocks;
            a.A = (const double *)A->data;
            a.lda = A->ld;
            a.b = b;
            a.x = x;
            a.mom = mom;
            a.part = part;
            a.rpart = rpart;
            a.rbuf = rbuf;
            a.ybuf = ybuf;
            a.sc = d_sc;
            a.bar = bar;
            a.err = err;
            a.m = m;
            a.n = n;
            a.nbm = nb;
            a.t_win = t;
            a.count = count;
            a.zeta = zeta;
            a.CW = CW;
            a.s = s;
            a.G = G;
            a.cd = cd;
            a.adaptive = p.adaptive_rho;
            a.confirm = 1;
            a.eta = eta;
            a.tol = p.tol;
            a.timeout_ns = 2000000000ull;
            int per_sm = 0;
            CUDA_OR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, memo_kernel, MT, 0), KPP_ERR_CUDA);
            if (per_sm * sm_count() < G) {
                rc = KPP_ERR_UNSUPPORTED;
                set_error("kpp_solve_memo: %d CTAs do not fit co-resident", G);
                goto cleanup;
            }
            CUDA_OR(cudaMemsetAsync(bar, 0, sizeof(unsigned), st), KPP_ERR_CUDA);
            CUDA_OR(cudaMemsetAsync(err, 0, sizeof(int), st), KPP_ERR_CUDA);
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            CUDA_OR(cudaEventCreate(&e0), KPP_ERR_CUDA);
            if (cudaEventCreate(&e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                rc = KPP_ERR_CUDA;
                goto cleanup;
            }
            void *args[] = {(void *)&a};
            cudaEventRecord(e0, st);
            note_launch();
            cudaError_t le =
                cudaLaunchCooperativeKernel((const void *)memo_kernel, dim3((unsigned)G), dim3(MT), args, 0, st);
            cudaEventRecord(e1, st);
            int herr = 0;
            if (le == cudaSuccess &&
                (cudaMemcpyAsync(&sc, d_sc, sizeof(MemoScalars), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                 cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                 cudaStreamSynchronize(st) != cudaSuccess))
                le = cudaErrorUnknown;
            float ms_w = 0.f;
            if (le == cudaSuccess) cudaEventElapsedTime(&ms_w, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (le != cudaSuccess) {
                rc = KPP_ERR_CUDA;
                set_error("kpp_solve_memo: kernel launch failed: %s", cudaGetErrorString(le));
                goto cleanup;
            }
            if (herr) {
                rc = (kpp_status)herr;
                set_error("kpp_solve_memo: device error %s", kpp_status_string(rc));
                goto cleanup;
            }
            kms_total += ms_w;
            ++launches;
        }
        // the window may end early (a stop): the blocks drawn for steps that did not run are not counted
        if (sc.t > t) nb_used = nb_after[(size_t)(std::min<int64_t>(sc.t - t, count) - 1)];
        t = sc.t;
        if (!sc.active) break;
    }
    {
        std::vector<double> r2, b2;
        kpp_status r3 = residual_norms(*A, 1, b, x, nullptr, r2, &b2, st);
        if (r3 != KPP_OK) {
            rc = r3;
            goto cleanup;
        }
        const double rel = b2[0] > 0 ? std::sqrt(r2[0] / b2[0]) : std::sqrt(r2[0]);
        kpp_status status = (kpp_status)sc.status;
        if (status == KPP_OK && !std::isfinite(rel)) status = KPP_ERR_NUMERIC;
        if (rep) {
            memset(rep, 0, sizeof(*rep));
            rep->iters = t;
            rep->rel_res_true = rel;
            rep->rel_res_est = sc.res_est;
            rep->rho_final = sc.rho;
            rep->status = status;
            rep->bad_block = -1;
            rep->device_ms = kms_total;
            rep->kernel_ms = kms_total;
            rep->launches = launches;
        }
        if (nblocks_out) *nblocks_out = nb_used;
        rc = status;
        if (rc != KPP_OK) set_error("kpp_solve_memo: solve ended with %s", kpp_status_string(rc));
    }
cleanup:
    if (Gnew) cudaFreeAsync(Gnew, st);
    if (rc == KPP_ERR_NOT_SPD && rep) {
        memset(rep, 0, sizeof(*rep));
        rep->status = rc;
        rep->bad_block = bad;
    }
    ms.release(st);
    return rc;
}

}  // namespace kpp

using namespace kpp;

extern "C" kpp_status kpp_solve_memo(const kpp_matrix *A, const double *b, double *x, int32_t s, int32_t mode,
                                     const kpp_params *p, kpp_report *rep, int64_t *nblocks_out, void *stream) {
    if (mode != 0 && mode != 1) {
        clear_error();
        set_error("kpp_solve_memo: mode must be 0 (K++) or 1 (CD++)");
        return KPP_ERR_ARG;
    }
    return memo_solve(A, b, x, s, mode, p, rep, nblocks_out, (cudaStream_t)stream);
}
