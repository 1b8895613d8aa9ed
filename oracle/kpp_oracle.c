/*
 * kpp_oracle.c -- plain, slow, FP64 CPU oracle for Kaczmarz++ and CD++.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this file; only
 * the tests, the smoke check and the benchmark's CPU-baseline leg do.  It shares no code with the
 * CUDA path (its own Philox, its own Cholesky, its own loops).
 *
 * Every loop is the textbook definition, summed left to right in FP64, with no blocking, fusion or
 * reordering.  Build with -ffp-contract=off so that x86 and Arm hosts give identical bits.
 *
 * What it computes (paper: Derezinski, Needell, Rebrova, Yang, "Randomized Kaczmarz Methods with
 * Beyond-Krylov Convergence", arXiv 2501.11673):
 *   - regularised block projection           w = A_S^T (A_S A_S^T + lam I)^{-1} (A_S x - b_S)   (Eq. 1.3)
 *   - Nesterov-style momentum                 m <- (1-rho)/(1+rho) (m - w),  x <- x - w + eta m     (Eq. 1.4, Alg. 1)
 *   - CD++ coordinate step                    w = I_S^T (A_SS + lam I)^{-1} (A_S x - b_S)           (Eq. 5.1, Thm 5.1)
 *   - residual estimate, adaptive rho, stop   E0/E1 windows of zeta steps, weighted ratio           (Eq. 5.2, Eq. 5.3, Alg. 3 / Alg. 5)
 *   - memoised per-block Cholesky factors     one factor per block of a fixed partition             (Sec. 4, Sec. 5.2)
 *   - plain conjugate gradients and restarted GMRES (context only; Sec. 6 compares against both)
 *   - Philox4x32-10 block sampling (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 *     1, 2, 3", SC'11): a counter-based generator, implemented here from its published definition.
 *
 * Readings where the paper is silent (shared with the GPU library by specification, not by code):
 *   - blocks are the contiguous partition  S_j = [j s, min((j+1) s, rows)),  nb = ceil(rows / s);
 *   - block draw at step t of system `sys`: out = Philox4x32-10(ctr = {t_lo, t_hi, sys, 0},
 *     key = {seed_lo, seed_hi});  j = (out[0] * nb) >> 32   (uniform with replacement, Alg. 1);
 *   - zeta = nb;  (t mod 2 zeta) < zeta adds |r|^2 to E0, otherwise to E1;
 *   - at t = 2 zeta - 1 (mod 2 zeta), checkpoint i (1, 2, ...): if E1 <= eps^2 |b|^2 the true
 *     residual |A x - b| / |b| is computed and the solve stops if it is <= eps; otherwise the ratio
 *     q = E1 / E0 enters  rhat = q (i = 1),  rhat = (a_{i-1}/a_i) rhat + (1 - a_{i-1}/a_i) q (i >= 2)
 *     with a_i = (i+1)^{ln(i+1)};  rho = 1 - rhat^{1/zeta} clamped to [0, 1 - 1e-12];  E0 = E1 = 0;
 *   - eta defaults to s / (2 min(rows, cols)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NO_CONVERGENCE 1
#define ORC_NOT_SPD 2
#define ORC_BAD_ARG 3

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11).  Round: (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2,                       */
/* c' = {hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0};  the key is bumped by the Weyl constants     */
/* between rounds.                                                                             */
/* ------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

int32_t orc_sample_block(uint64_t seed, int64_t t, uint32_t sys, int32_t nb) {
    uint32_t ctr[4] = {(uint32_t)(uint64_t)t, (uint32_t)((uint64_t)t >> 32), sys, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return (int32_t)(((uint64_t)out[0] * (uint64_t)(uint32_t)nb) >> 32);
}

/* ------------------------------------------------------------------------------------------ */
/* Dense linear algebra, row-major.                                                            */
/* ------------------------------------------------------------------------------------------ */

/* In place lower Cholesky of the s x s SPD matrix G (row-major, leading dimension s).
 * Returns 0, or (j+1) if the j-th pivot is not positive / not finite.  The strict upper triangle
 * is set to zero. */
int orc_cholesky(int s, double *G) {
    for (int j = 0; j < s; ++j) {
        double d = G[(size_t)j * s + j];
        for (int k = 0; k < j; ++k) d -= G[(size_t)j * s + k] * G[(size_t)j * s + k];
        if (!(d > 0.0) || !isfinite(d)) return j + 1;
        double ljj = sqrt(d);
        G[(size_t)j * s + j] = ljj;
        for (int i = j + 1; i < s; ++i) {
            double v = G[(size_t)i * s + j];
            for (int k = 0; k < j; ++k) v -= G[(size_t)i * s + k] * G[(size_t)j * s + k];
            G[(size_t)i * s + j] = v / ljj;
        }
        for (int k = j + 1; k < s; ++k) G[(size_t)j * s + k] = 0.0;
    }
    return 0;
}

/* Solve (L L^T) y = r in place: forward substitution L z = r, then back substitution L^T y = z. */
void orc_chol_solve(int s, const double *L, double *y) {
    for (int i = 0; i < s; ++i) {
        double v = y[i];
        for (int k = 0; k < i; ++k) v -= L[(size_t)i * s + k] * y[k];
        y[i] = v / L[(size_t)i * s + i];
    }
    for (int i = s - 1; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < s; ++k) v -= L[(size_t)k * s + i] * y[k];
        y[i] = v / L[(size_t)i * s + i];
    }
}

static double dot(int64_t n, const double *a, const double *b) {
    double acc = 0.0;
    for (int64_t k = 0; k < n; ++k) acc += a[k] * b[k];
    return acc;
}

/* |A x - b| / |b| in FP64. */
double orc_rel_residual(int64_t m, int64_t n, const double *A, const double *b, const double *x) {
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double r = dot(n, A + (size_t)i * n, x) - b[i];
        num += r * r;
        den += b[i] * b[i];
    }
    return den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
}

static int64_t nblocks(int64_t rows, int s) { return (rows + s - 1) / s; }
static int block_len(int64_t rows, int s, int64_t j) {
    int64_t lo = j * s, hi = lo + s < rows ? lo + s : rows;
    return (int)(hi - lo);
}

/* ------------------------------------------------------------------------------------------ */
/* Memoised factors (Sec. 4 / Sec. 5.2): one s x s lower factor per block, stored at L + j*s*s  */
/* (the last block may be shorter; its factor uses leading dimension equal to its length).      */
/* ------------------------------------------------------------------------------------------ */

/* K++: L_j = chol(A_{S_j} A_{S_j}^T + lam I).  Returns 0 or (block+1) of the first failure. */
int orc_kpp_factor(int64_t m, int64_t n, const double *A, int s, double lam, double *L) {
    int64_t nb = nblocks(m, s);
    for (int64_t j = 0; j < nb; ++j) {
        int len = block_len(m, s, j);
        double *G = L + (size_t)j * s * s;
        const double *As = A + (size_t)j * s * n;
        for (int a = 0; a < len; ++a)
            for (int c = 0; c < len; ++c)
                G[(size_t)a * len + c] = dot(n, As + (size_t)a * n, As + (size_t)c * n) + (a == c ? lam : 0.0);
        if (orc_cholesky(len, G) != 0) return (int)(j + 1);
    }
    return 0;
}

/* CD++: L_j = chol(A_{S_j,S_j} + lam I) for symmetric n x n A. */
int orc_cdpp_factor(int64_t n, const double *A, int s, double lam, double *L) {
    int64_t nb = nblocks(n, s);
    for (int64_t j = 0; j < nb; ++j) {
        int len = block_len(n, s, j);
        double *G = L + (size_t)j * s * s;
        int64_t r0 = j * s;
        for (int a = 0; a < len; ++a)
            for (int c = 0; c < len; ++c)
                G[(size_t)a * len + c] = A[(size_t)(r0 + a) * n + (r0 + c)] + (a == c ? lam : 0.0);
        if (orc_cholesky(len, G) != 0) return (int)(j + 1);
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* The iteration.                                                                              */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int32_t s;                 /* block size */
    int32_t cd;                /* 0: K++ step (Eq. 1.3), 1: CD++ step (Eq. 5.1) */
    double lam;                /* Tikhonov regulariser */
    double tol;                /* eps; 0 disables stopping */
    int64_t max_iters;         /* iteration cap (total, counting from state.t) */
    uint64_t seed;             /* Philox key */
    uint32_t sys;              /* Philox stream id (system / request) */
    int32_t adaptive;          /* 1: adaptive rho (Eq. 5.3); 0: rho fixed at state.rho */
    double eta;                /* momentum step (0: plain block Kaczmarz) */
    int32_t confirm;           /* 1: stop only once the true residual is <= tol */
} orc_params;

typedef struct {
    int64_t t;                 /* next iteration index */
    int64_t ci;                /* checkpoints completed */
    double E0, E1;             /* running window sums of |r_t|^2 */
    double rhat, rho;          /* weighted ratio estimate and current rho */
} orc_state;

typedef struct {
    int64_t iters;             /* iterations performed in this call */
    double rel_res_true;       /* |A x - b| / |b| at return (always computed) */
    double rel_res_est;        /* sqrt(E1)/|b| at the last checkpoint (NaN if none) */
    int32_t status;            /* ORC_* */
    int32_t pad;
} orc_report;

/* One block step on (x, mom), given the drawn block j and its factor.  Returns |r|^2. */
static double step(int64_t rows, int64_t n, const double *A, const double *b, int s, int cd,
                   const double *L, int64_t j, double beta, double eta, double *x, double *mom,
                   double *r, double *w) {
    int len = block_len(rows, s, j);
    int64_t r0 = j * s;
    const double *Lj = L + (size_t)j * s * s;
    /* r = A_S x - b_S */
    double rn2 = 0.0;
    for (int a = 0; a < len; ++a) {
        r[a] = dot(n, A + (size_t)(r0 + a) * n, x) - b[r0 + a];
        rn2 += r[a] * r[a];
    }
    /* y = (G + lam I)^{-1} r through the memoised factor (r is overwritten by y) */
    orc_chol_solve(len, Lj, r);
    /* w = A_S^T y (K++) or I_S^T y (CD++) */
    for (int64_t k = 0; k < n; ++k) w[k] = 0.0;
    if (cd) {
        for (int a = 0; a < len; ++a) w[r0 + a] = r[a];
    } else {
        for (int a = 0; a < len; ++a) {
            const double *row = A + (size_t)(r0 + a) * n;
            for (int64_t k = 0; k < n; ++k) w[k] += row[k] * r[a];
        }
    }
    /* momentum, then the update (Alg. 1: m_{t+1} first, x_{t+1} uses m_{t+1}) */
    for (int64_t k = 0; k < n; ++k) {
        mom[k] = beta * (mom[k] - w[k]);
        x[k] = x[k] - w[k] + eta * mom[k];
    }
    return rn2;
}

/* Run iterations from `st` until the stop rule fires or st->t reaches p->max_iters.
 * rows x n matrix A (CD++: rows == n, A symmetric), factors from orc_*_factor.
 * trace (optional, capacity trace_cap rows of 5 doubles): per checkpoint {t, E0, E1, rho, true_res or NaN}. */
int orc_run(int64_t rows, int64_t n, const double *A, const double *b, const double *L,
            const orc_params *p, orc_state *st, double *x, double *mom, orc_report *rep,
            double *trace, int64_t trace_cap) {
    if (p->s <= 0 || rows <= 0 || n <= 0 || (p->cd && rows != n)) return ORC_BAD_ARG;
    int s = p->s;
    int64_t nb = nblocks(rows, s);
    int64_t zeta = nb;
    double bn2 = dot(rows, b, b);
    double *r = (double *)malloc(sizeof(double) * (size_t)s);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t it0 = st->t;
    int status = ORC_NO_CONVERGENCE;
    rep->rel_res_est = NAN;
    int64_t ntrace = 0;
    while (st->t < p->max_iters) {
        int64_t t = st->t;
        int64_t j = orc_sample_block(p->seed, t, p->sys, (int32_t)nb);
        double beta = (1.0 - st->rho) / (1.0 + st->rho);
        double rn2 = step(rows, n, A, b, s, p->cd, L, j, beta, p->eta, x, mom, r, w);
        st->t = t + 1;
        if ((t % (2 * zeta)) < zeta) st->E0 += rn2; else st->E1 += rn2;
        if ((t % (2 * zeta)) == 2 * zeta - 1) {
            st->ci += 1;
            double tres = NAN;
            rep->rel_res_est = bn2 > 0.0 ? sqrt(st->E1 / bn2) : sqrt(st->E1);
            int stop = 0;
            if (p->tol > 0.0 && st->E1 <= p->tol * p->tol * bn2) {
                if (p->confirm) {
                    tres = orc_rel_residual(rows, n, A, b, x);
                    stop = tres <= p->tol;
                } else {
                    stop = 1;
                }
            }
            if (trace && ntrace < trace_cap) {
                double *tr = trace + 5 * ntrace;
                tr[0] = (double)t; tr[1] = st->E0; tr[2] = st->E1; tr[3] = st->rho; tr[4] = tres;
                ntrace++;
            }
            if (stop) { status = ORC_OK; break; }
            if (p->adaptive) {
                double q = st->E0 > 0.0 ? st->E1 / st->E0 : 0.0;
                if (st->ci == 1) {
                    st->rhat = q;
                } else {
                    double li = log((double)st->ci), li1 = log((double)st->ci + 1.0);
                    double wgt = exp(li * li - li1 * li1); /* a_{i-1} / a_i,  a_i = (i+1)^{ln(i+1)} */
                    st->rhat = wgt * st->rhat + (1.0 - wgt) * q;
                }
                double rho = 1.0 - pow(st->rhat, 1.0 / (double)zeta);
                if (!(rho > 0.0)) rho = 0.0;
                if (rho > 1.0 - 1e-12) rho = 1.0 - 1e-12;
                st->rho = rho;
            }
            st->E0 = 0.0;
            st->E1 = 0.0;
        }
    }
    rep->iters = st->t - it0;
    rep->rel_res_true = orc_rel_residual(rows, n, A, b, x);
    rep->status = status;
    free(r);
    free(w);
    return status;
}

/* Plain CG on SPD A (context only): x in/out, returns iterations; stops at |r|/|b| <= tol. */
int64_t orc_cg(int64_t n, const double *A, const double *b, double *x, double tol, int64_t max_iters,
               double *rel_res_out) {
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *pv = (double *)malloc(sizeof(double) * (size_t)n);
    double *Ap = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - dot(n, A + (size_t)i * n, x);
    memcpy(pv, r, sizeof(double) * (size_t)n);
    double bn = sqrt(dot(n, b, b));
    double rr = dot(n, r, r);
    int64_t it = 0;
    while (it < max_iters && sqrt(rr) > tol * bn) {
        for (int64_t i = 0; i < n; ++i) Ap[i] = dot(n, A + (size_t)i * n, pv);
        double alpha = rr / dot(n, pv, Ap);
        for (int64_t i = 0; i < n; ++i) {
            x[i] += alpha * pv[i];
            r[i] -= alpha * Ap[i];
        }
        double rr2 = dot(n, r, r);
        double bta = rr2 / rr;
        for (int64_t i = 0; i < n; ++i) pv[i] = r[i] + bta * pv[i];
        rr = rr2;
        ++it;
    }
    *rel_res_out = orc_rel_residual(n, n, A, b, x);
    free(r);
    free(pv);
    free(Ap);
    return it;
}

/* Restarted GMRES(restart) (Saad and Schultz), the other Krylov method Sec. 6 compares with:
 * the textbook algorithm written out.  A cycle starts from r0 = b - A x, v_1 = r0 / beta, g = beta e_1;
 * step j forms w = A v_j, orthogonalises it against v_1 .. v_j one vector at a time (modified
 * Gram-Schmidt), h_{j+1,j} = |w|, v_{j+1} = w / h_{j+1,j}; the earlier Givens rotations are applied to
 * column j of H and a new one zeroes h_{j+1,j}, updating g; the cycle ends when |g_{j+1}| <= tol |b|,
 * after `restart` steps or at max_iters steps in all, with x += V y, R y = g.  Returns the steps taken;
 * *cycles_out the cycles, *rel_res_out the true |A x - b| / |b|. */
int64_t orc_gmres(int64_t n, const double *A, const double *b, double *x, int64_t restart, double tol,
                  int64_t max_iters, double *rel_res_out, int64_t *cycles_out) {
    const int64_t m = restart;
    double *V = (double *)malloc(sizeof(double) * (size_t)(m + 1) * (size_t)n);
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double)); /* H[i * m + j] = h_{i,j} */
    double *cs = (double *)malloc(sizeof(double) * (size_t)m);
    double *sn = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    const double bn = sqrt(dot(n, b, b));
    int64_t it = 0, cycles = 0;
    for (;;) {
        for (int64_t i = 0; i < n; ++i) w[i] = b[i] - dot(n, A + (size_t)i * n, x);
        const double beta = sqrt(dot(n, w, w));
        if (!(beta > tol * bn) || it >= max_iters) break;
        for (int64_t i = 0; i < n; ++i) V[i] = w[i] / beta;
        for (int64_t i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int64_t k = 0;
        for (int64_t j = 0; j < m; ++j) {
            const double *vj = V + (size_t)j * (size_t)n;
            for (int64_t i = 0; i < n; ++i) w[i] = dot(n, A + (size_t)i * n, vj);
            for (int64_t l = 0; l <= j; ++l) {
                const double *vl = V + (size_t)l * (size_t)n;
                const double h = dot(n, vl, w);
                H[l * m + j] = h;
                for (int64_t i = 0; i < n; ++i) w[i] -= h * vl[i];
            }
            const double hn = sqrt(dot(n, w, w));
            H[(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (int64_t i = 0; i < n; ++i) V[(size_t)(j + 1) * (size_t)n + i] = w[i] / hn;
            for (int64_t l = 0; l < j; ++l) {
                const double t = cs[l] * H[l * m + j] + sn[l] * H[(l + 1) * m + j];
                H[(l + 1) * m + j] = -sn[l] * H[l * m + j] + cs[l] * H[(l + 1) * m + j];
                H[l * m + j] = t;
            }
            const double d = sqrt(H[j * m + j] * H[j * m + j] + hn * hn);
            cs[j] = d > 0.0 ? H[j * m + j] / d : 1.0;
            sn[j] = d > 0.0 ? hn / d : 0.0;
            H[j * m + j] = d;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            k = j + 1;
            if (fabs(g[j + 1]) <= tol * bn || hn == 0.0 || it >= max_iters) break;
        }
        for (int64_t i = k - 1; i >= 0; --i) {
            double t = g[i];
            for (int64_t l = i + 1; l < k; ++l) t -= H[i * m + l] * y[l];
            y[i] = t / H[i * m + i];
        }
        for (int64_t l = 0; l < k; ++l)
            for (int64_t i = 0; i < n; ++i) x[i] += y[l] * V[(size_t)l * (size_t)n + i];
        ++cycles;
    }
    *rel_res_out = orc_rel_residual(n, n, A, b, x);
    *cycles_out = cycles;
    free(V);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(y);
    free(w);
    return it;
}

/* ------------------------------------------------------------------------------------------------
 * Randomized Hadamard preprocessing of CD++ (Sec. 5.1, the preprocessing of Alg. 3 and the return
 * D FHT(x); App. on FHT / SymFHT).
 *
 * H_n (n a power of 2) is the Sylvester-Hadamard matrix: H_1 = [1], H_2n = [[H_n, H_n], [H_n, -H_n]].
 * Unrolling the recursion bit by bit gives its entries: (H_n)_{ij} = (-1)^{popcount(i AND j)}.
 * Q = H_n D with D = diag(d) / sqrt(n), d_i = +-1, so Q Q^T = H D^2 H = H H / n = I.  The system
 * A x = b becomes Abar xbar = bbar with Abar = Q A Q^T, bbar = Q b, and x = Q^T xbar = D H xbar.
 *
 * orc_rht_forward / orc_rht_inverse / orc_rht_entry are the definition written out: explicit entries
 * of H and plain left-to-right sums (O(n^3) for the matrix).  orc_symfht is the paper's recursive
 * SymFHT (H A H of a symmetric A, two half-size recursive calls plus one general transform of the
 * off-diagonal block), kept to pin its result and its operation count (Thm. on SymFHT:
 * at most n^2 (2.5 + log2 n) additions / subtractions).
 * ------------------------------------------------------------------------------------------------ */
static double had(int64_t i, int64_t j) { return (__builtin_popcountll((unsigned long long)(i & j)) & 1) ? -1.0 : 1.0; }

/* Abar = Q A Q^T (n x n), and bbar = Q b for a panel b of k columns (n x k row-major; k may be 0). */
void orc_rht_forward(int64_t n, const double *d, const double *A, int64_t k, const double *b, double *Abar,
                     double *bbar) {
    double *M = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *T = (double *)malloc(sizeof(double) * (size_t)(n * n));
    for (int64_t p = 0; p < n; ++p)
        for (int64_t q = 0; q < n; ++q) M[p * n + q] = d[p] * A[p * n + q] * d[q] / (double)n;  /* D A D */
    for (int64_t p = 0; p < n; ++p)                                                              /* T = M H */
        for (int64_t j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int64_t q = 0; q < n; ++q) acc += M[p * n + q] * had(q, j);
            T[p * n + j] = acc;
        }
    for (int64_t i = 0; i < n; ++i)                                                              /* H T */
        for (int64_t j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int64_t p = 0; p < n; ++p) acc += had(i, p) * T[p * n + j];
            Abar[i * n + j] = acc;
        }
    const double rs = 1.0 / sqrt((double)n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t c = 0; c < k; ++c) {
            double acc = 0.0;
            for (int64_t p = 0; p < n; ++p) acc += had(i, p) * (d[p] * rs * b[p * k + c]);
            bbar[i * k + c] = acc;
        }
    free(M);
    free(T);
}

/* x = Q^T xbar = D H xbar for a panel of k columns. */
void orc_rht_inverse(int64_t n, const double *d, int64_t k, const double *xbar, double *x) {
    const double rs = 1.0 / sqrt((double)n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t c = 0; c < k; ++c) {
            double acc = 0.0;
            for (int64_t p = 0; p < n; ++p) acc += had(i, p) * xbar[p * k + c];
            x[i * k + c] = d[i] * rs * acc;
        }
}

/* One entry (Q A Q^T)_{ij} = sum_p H_ip d_p / sqrt(n) sum_q A_pq d_q / sqrt(n) H_qj, O(n^2). */
double orc_rht_entry(int64_t n, const double *d, const double *A, int64_t i, int64_t j) {
    double acc = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        double row = 0.0;
        for (int64_t q = 0; q < n; ++q) row += A[p * n + q] * d[q] * had(q, j);
        acc += had(i, p) * d[p] * row;
    }
    return acc / (double)n;
}

/* FHT of a length-n vector with stride `st`, in place, by the recursion H_n v = [H(v1 + v2); H(v1 - v2)]
 * (v1, v2 the halves); n log2 n additions / subtractions, added to *ops. */
static void fht_vec(int64_t n, double *v, int64_t st, double *tmp, int64_t *ops) {
    if (n == 1) return;
    const int64_t h = n / 2;
    for (int64_t i = 0; i < h; ++i) {
        const double a = v[i * st], c = v[(i + h) * st];
        tmp[i] = a + c;
        tmp[i + h] = a - c;
    }
    *ops += n;
    for (int64_t i = 0; i < n; ++i) v[i * st] = tmp[i];
    fht_vec(h, v, st, tmp, ops);
    fht_vec(h, v + h * st, st, tmp, ops);
}

/* H_n v for k columns of an n x k row-major panel, in place; returns the operation count. */
int64_t orc_fht(int64_t n, int64_t k, double *V) {
    int64_t ops = 0;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t c = 0; c < k; ++c) fht_vec(n, V + c, k, tmp, &ops);
    free(tmp);
    return ops;
}

/* SymFHT of the symmetric n x n block at A (leading dimension ld), in place: the block becomes H A H.
 * With A = [[A11, A12], [A12^T, A22]] and B11 = H A11 H, B22 = H A22 H (recursive), B12 = H A12 H:
 *   C11 = B11 + B12^T, C12 = B11 - B12, C21 = B12 + B22, C22 = B12^T - B22,
 *   H A H = [[C11 + C21, C12 + C22], [(C12 + C22)^T, C12 - C22]]. */
static void symfht_rec(int64_t n, double *A, int64_t ld, double *tmp, int64_t *ops) {
    if (n == 1) return;
    const int64_t h = n / 2;
    double *A11 = A, *A12 = A + h, *A21 = A + h * ld, *A22 = A + h * ld + h;
    symfht_rec(h, A11, ld, tmp, ops);
    symfht_rec(h, A22, ld, tmp, ops);
    for (int64_t i = 0; i < h; ++i) fht_vec(h, A12 + i * ld, 1, tmp, ops);  /* rows:    A12 H   */
    for (int64_t j = 0; j < h; ++j) fht_vec(h, A12 + j, ld, tmp, ops);      /* columns: H A12 H */
    double *C = (double *)malloc(sizeof(double) * (size_t)(4 * h * h));
    double *C11 = C, *C12 = C + h * h, *C21 = C + 2 * h * h, *C22 = C + 3 * h * h;
    for (int64_t i = 0; i < h; ++i)
        for (int64_t j = 0; j < h; ++j) {
            const double b11 = A11[i * ld + j], b22 = A22[i * ld + j];
            const double b12 = A12[i * ld + j], b12t = A12[j * ld + i];
            C11[i * h + j] = b11 + b12t;
            C12[i * h + j] = b11 - b12;
            C21[i * h + j] = b12 + b22;
            C22[i * h + j] = b12t - b22;
        }
    *ops += 4 * h * h;
    for (int64_t i = 0; i < h; ++i)
        for (int64_t j = 0; j < h; ++j) {
            A11[i * ld + j] = C11[i * h + j] + C21[i * h + j];
            A12[i * ld + j] = C12[i * h + j] + C22[i * h + j];
            A22[i * ld + j] = C12[i * h + j] - C22[i * h + j];
        }
    for (int64_t i = 0; i < h; ++i)
        for (int64_t j = 0; j < h; ++j) A21[i * ld + j] = A12[j * ld + i];
    *ops += 3 * h * h;
    free(C);
}

/* H A H of a symmetric n x n row-major A, in place; returns the additions / subtractions used. */
int64_t orc_symfht(int64_t n, double *A) {
    int64_t ops = 0;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    symfht_rec(n, A, n, tmp, &ops);
    free(tmp);
    return ops;
}

/* ------------------------------------------------------------------------------------------------
 * Online block memoisation with random subsets (Sec. 4, "Block memoization"; Sec. 5.2, the
 * simplified scheme of CD++ in Alg. 3's sampling step; the sampling step of Alg. 5 for K++).
 *
 * The collection B of memoised blocks starts empty.  At step t a Bernoulli draw with probability
 *   CD++: p_t = min(1, (n / s) ln(n) / t)          K++: p_t = min(1, (m / s) ln(m) / t, (n / s) ln(m) / t)
 * (p_0 = 1) decides between a new uniformly random s-subset S of the rows (its factor is computed and
 * S joins B) and a uniform pick from B (its factor is reused).  The factor is chol(A_S A_S^T + lam I)
 * for K++ and chol(A_SS + lam I) for CD++; the step itself is the one of orc_run on the rows of S.
 *
 * Readings (the paper is silent): log is the natural log; the draws come from Philox4x32-10 with the
 * key {seed_lo, seed_hi}: counter {t_lo, t_hi, sys, 0} gives the Bernoulli word (out[1], new iff
 * out[1] < p_t 2^32) and the pick (out[2]: j = out[2] |B| >> 32); counter {t_lo, t_hi, sys, 1 + i/4}
 * gives word out[i mod 4] for the i-th draw of Floyd's sampling of S (R. W. Floyd's algorithm for a
 * uniform s-subset of [0, N): for j = N - s .. N - 1 take r uniform in [0, j] (r = word (j + 1) >> 32),
 * and add j if r is already taken, else r); S is then sorted ascending.  zeta = ceil(rows / s) as for
 * the fixed partition.  The memo lives for one call of orc_run_memo.
 * ------------------------------------------------------------------------------------------------ */
double orc_memo_prob(int cd, int64_t rows, int64_t n, int s, int64_t t) {
    if (t <= 0) return 1.0;
    double p;
    if (cd) {
        p = (double)n / (double)s * log((double)n) / (double)t;
    } else {
        const double lm = log((double)rows);
        const double a = (double)rows / (double)s * lm / (double)t, c = (double)n / (double)s * lm / (double)t;
        p = a < c ? a : c;
    }
    return p < 1.0 ? p : 1.0;
}

static void memo_words(uint64_t seed, int64_t t, uint32_t sys, uint32_t lane, uint32_t out[4]) {
    uint32_t ctr[4] = {(uint32_t)(uint64_t)t, (uint32_t)((uint64_t)t >> 32), sys, lane};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform s-subset of [0, N) drawn at step t (Floyd), sorted ascending into S[0..s). */
void orc_memo_subset(uint64_t seed, int64_t t, uint32_t sys, int64_t N, int s, int64_t *S) {
    uint32_t wv[4];
    int cnt = 0;
    for (int i = 0; i < s; ++i) {
        if (i % 4 == 0) memo_words(seed, t, sys, 1u + (uint32_t)(i / 4), wv);
        const int64_t j = N - s + i;
        const int64_t r = (int64_t)(((uint64_t)wv[i % 4] * (uint64_t)(j + 1)) >> 32);
        int taken = 0;
        for (int q = 0; q < cnt; ++q) taken |= (S[q] == r);
        S[cnt++] = taken ? j : r;
    }
    for (int a = 1; a < s; ++a) { /* insertion sort */
        const int64_t v = S[a];
        int q = a - 1;
        while (q >= 0 && S[q] > v) {
            S[q + 1] = S[q];
            --q;
        }
        S[q + 1] = v;
    }
}

/* The draw of step t with nb blocks memoised so far: -1 = sample a new subset, else the memo index. */
int64_t orc_memo_draw(uint64_t seed, int64_t t, uint32_t sys, int cd, int64_t rows, int64_t n, int s, int64_t nb) {
    if (nb <= 0) return -1;
    uint32_t o[4];
    memo_words(seed, t, sys, 0u, o);
    const double p = orc_memo_prob(cd, rows, n, s, t);
    if ((double)o[1] < p * 4294967296.0) return -1;
    return (int64_t)(((uint64_t)o[2] * (uint64_t)nb) >> 32);
}

/* Factor of the subset S (lower Cholesky, s x s): K++ A_S A_S^T + lam I, CD++ A_SS + lam I. */
static int subset_factor(int64_t n, const double *A, const int64_t *S, int s, int cd, double lam, double *L) {
    for (int a = 0; a < s; ++a)
        for (int c = 0; c < s; ++c) {
            double g = cd ? A[(size_t)S[a] * n + S[c]] : dot(n, A + (size_t)S[a] * n, A + (size_t)S[c] * n);
            L[(size_t)a * s + c] = g + (a == c ? lam : 0.0);
        }
    return orc_cholesky(s, L);
}

/* One step on the rows S with their factor L (as step() for a contiguous block).  Returns |r|^2. */
static double step_rows(int64_t n, const double *A, const double *b, const int64_t *S, int s, int cd,
                        const double *L, double beta, double eta, double *x, double *mom, double *r, double *w) {
    double rn2 = 0.0;
    for (int a = 0; a < s; ++a) {
        r[a] = dot(n, A + (size_t)S[a] * n, x) - b[S[a]];
        rn2 += r[a] * r[a];
    }
    orc_chol_solve(s, L, r);
    for (int64_t k = 0; k < n; ++k) w[k] = 0.0;
    if (cd) {
        for (int a = 0; a < s; ++a) w[S[a]] = r[a];
    } else {
        for (int a = 0; a < s; ++a) {
            const double *row = A + (size_t)S[a] * n;
            for (int64_t k = 0; k < n; ++k) w[k] += row[k] * r[a];
        }
    }
    for (int64_t k = 0; k < n; ++k) {
        mom[k] = beta * (mom[k] - w[k]);
        x[k] = x[k] - w[k] + eta * mom[k];
    }
    return rn2;
}

/* One step on a given subset (factor computed here): for the pins.  Returns ORC_OK or ORC_NOT_SPD. */
int orc_step_subset(int64_t rows, int64_t n, const double *A, const double *b, const int64_t *S, int s, int cd,
                    double lam, double beta, double eta, double *x, double *mom, double *rn2_out) {
    (void)rows;
    double *L = (double *)malloc(sizeof(double) * (size_t)s * s);
    double *r = (double *)malloc(sizeof(double) * (size_t)s);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    int rc = subset_factor(n, A, S, s, cd, lam, L) ? ORC_NOT_SPD : ORC_OK;
    if (rc == ORC_OK) *rn2_out = step_rows(n, A, b, S, s, cd, L, beta, eta, x, mom, r, w);
    free(L);
    free(r);
    free(w);
    return rc;
}

/* The solve with online memoisation: as orc_run, with the block of step t from the memo scheme.
 * *nblocks_out receives |B| at return; blocks_out (optional, capacity cap) the memo index of each
 * step (-1 never appears: a new block is recorded with its new index). */
int orc_run_memo(int64_t rows, int64_t n, const double *A, const double *b, const orc_params *p, orc_state *st,
                 double *x, double *mom, orc_report *rep, int64_t *nblocks_out, int64_t *blocks_out, int64_t cap) {
    if (p->s <= 0 || p->s > rows || rows <= 0 || n <= 0 || (p->cd && rows != n)) return ORC_BAD_ARG;
    const int s = p->s;
    const int64_t zeta = nblocks(rows, s);
    const double bn2 = dot(rows, b, b);
    int64_t nb = 0, mcap = 64;
    int64_t *Sset = (int64_t *)malloc(sizeof(int64_t) * (size_t)(mcap * s));
    double *Lset = (double *)malloc(sizeof(double) * (size_t)(mcap * s * s));
    double *r = (double *)malloc(sizeof(double) * (size_t)s);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    const int64_t it0 = st->t;
    int status = ORC_NO_CONVERGENCE;
    rep->rel_res_est = NAN;
    while (st->t < p->max_iters) {
        const int64_t t = st->t;
        int64_t j = orc_memo_draw(p->seed, t, p->sys, p->cd, rows, n, s, nb);
        if (j < 0) {
            if (nb == mcap) {
                mcap *= 2;
                Sset = (int64_t *)realloc(Sset, sizeof(int64_t) * (size_t)(mcap * s));
                Lset = (double *)realloc(Lset, sizeof(double) * (size_t)(mcap * s * s));
            }
            j = nb;
            orc_memo_subset(p->seed, t, p->sys, rows, s, Sset + (size_t)j * s);
            if (subset_factor(n, A, Sset + (size_t)j * s, s, p->cd, p->lam, Lset + (size_t)j * s * s)) {
                status = ORC_NOT_SPD;
                break;
            }
            ++nb;
        }
        if (blocks_out && t - it0 < cap) blocks_out[t - it0] = j;
        const double beta = (1.0 - st->rho) / (1.0 + st->rho);
        const double rn2 = step_rows(n, A, b, Sset + (size_t)j * s, s, p->cd, Lset + (size_t)j * s * s, beta,
                                     p->eta, x, mom, r, w);
        st->t = t + 1;
        if ((t % (2 * zeta)) < zeta) st->E0 += rn2; else st->E1 += rn2;
        if ((t % (2 * zeta)) == 2 * zeta - 1) {
            st->ci += 1;
            rep->rel_res_est = bn2 > 0.0 ? sqrt(st->E1 / bn2) : sqrt(st->E1);
            if (p->tol > 0.0 && st->E1 <= p->tol * p->tol * bn2 &&
                (!p->confirm || orc_rel_residual(rows, n, A, b, x) <= p->tol)) {
                status = ORC_OK;
                break;
            }
            if (p->adaptive) { /* Eq. 5.2 - 5.3, as in orc_run */
                const double q = st->E0 > 0.0 ? st->E1 / st->E0 : 0.0;
                if (st->ci == 1) {
                    st->rhat = q;
                } else {
                    const double li = log((double)st->ci), li1 = log((double)st->ci + 1.0);
                    const double wgt = exp(li * li - li1 * li1);
                    st->rhat = wgt * st->rhat + (1.0 - wgt) * q;
                }
                double rho = 1.0 - pow(st->rhat, 1.0 / (double)zeta);
                if (!(rho > 0.0)) rho = 0.0;
                if (rho > 1.0 - 1e-12) rho = 1.0 - 1e-12;
                st->rho = rho;
            }
            st->E0 = 0.0;
            st->E1 = 0.0;
        }
    }
    rep->iters = st->t - it0;
    rep->rel_res_true = orc_rel_residual(rows, n, A, b, x);
    rep->status = status;
    *nblocks_out = nb;
    free(Sset);
    free(Lset);
    free(r);
    free(w);
    return status;
}

/* ------------------------------------------------------------------------------------------------
 * Inexact projection by sketch-preconditioned LSQR (Sec. 4.1, "Computing the projection step", and
 * the Proj algorithm of the supplement): w = argmin |A_S w - r|^2 + lam |w|^2 is the first n entries
 * of the minimum-length solution of
 *     M [w; v] = L^{-1} r,   M = L^{-1} [A_S, sqrt(lam) I],   L L^T = Ahat Ahat^T + lam I,
 * with the sketch Ahat = A_S Pi^T of the subsampled randomized Hadamard transform
 *     Pi = sqrt(n'/tau) I_T H_{n'} D / sqrt(n')   (n' = the power of 2 >= n, A_S padded with zero
 * columns; D = diag(d), d_i = +-1; T a tau-subset of [0, n')),  i.e. Ahat = (A_S D H)[:, T] / sqrt(tau).
 * The signs d and the subset T are inputs.  L is lower triangular (the paper's R = L^T).  LSQR is Paige
 * and Saunders' bidiagonalisation method (ACM TOMS 8, 1982) from x = 0, t_max iterations.
 * ------------------------------------------------------------------------------------------------ */
static void lsolve_lower(int s, const double *L, double *y) { /* y <- L^{-1} y */
    for (int i = 0; i < s; ++i) {
        double v = y[i];
        for (int k = 0; k < i; ++k) v -= L[(size_t)i * s + k] * y[k];
        y[i] = v / L[(size_t)i * s + i];
    }
}
static void lsolve_upper_t(int s, const double *L, double *y) { /* y <- L^{-T} y */
    for (int i = s - 1; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < s; ++k) v -= L[(size_t)k * s + i] * y[k];
        y[i] = v / L[(size_t)i * s + i];
    }
}

/* The preconditioner L (s x s lower) from the SRHT sketch; returns 0 or ORC_NOT_SPD. */
int orc_proj_precond(int64_t n, const double *AS, int s, double lam, int64_t tau, const int64_t *T,
                     const double *d, double *L) {
    int64_t np2 = 1;
    while (np2 < n) np2 *= 2;
    double *row = (double *)malloc(sizeof(double) * (size_t)np2);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)np2);
    double *Ah = (double *)malloc(sizeof(double) * (size_t)(s * tau));
    int64_t ops = 0;
    for (int a = 0; a < s; ++a) {
        for (int64_t k = 0; k < np2; ++k) row[k] = k < n ? AS[(size_t)a * n + k] * d[k] : 0.0;
        fht_vec(np2, row, 1, tmp, &ops);
        for (int64_t q = 0; q < tau; ++q) Ah[(size_t)a * tau + q] = row[T[q]] / sqrt((double)tau);
    }
    for (int a = 0; a < s; ++a)
        for (int c = 0; c < s; ++c)
            L[(size_t)a * s + c] = dot(tau, Ah + (size_t)a * tau, Ah + (size_t)c * tau) + (a == c ? lam : 0.0);
    const int rc = orc_cholesky(s, L) ? ORC_NOT_SPD : ORC_OK;
    free(row);
    free(tmp);
    free(Ah);
    return rc;
}

/* w (n) from t_max LSQR iterations on the preconditioned system; returns the iterations taken. */
int orc_proj_lsqr(int64_t n, const double *AS, int s, const double *r, double lam, const double *L, int t_max,
                  double *w) {
    const int64_t N = n + s; /* unknowns [w; v] */
    const double sl = sqrt(lam);
    double *u = (double *)malloc(sizeof(double) * (size_t)s);
    double *z = (double *)malloc(sizeof(double) * (size_t)s);
    double *v = (double *)malloc(sizeof(double) * (size_t)N);
    double *wd = (double *)malloc(sizeof(double) * (size_t)N);
    double *x = (double *)calloc((size_t)N, sizeof(double));
    /* u = M v_in  (s):  L^{-1} (A_S v[0:n] + sqrt(lam) v[n:]) */
#define ORC_MV(out, in)                                                                   \
    do {                                                                                  \
        for (int a_ = 0; a_ < s; ++a_)                                                    \
            (out)[a_] = dot(n, AS + (size_t)a_ * n, (in)) + sl * (in)[n + a_];           \
        lsolve_lower(s, L, (out));                                                        \
    } while (0)
    /* v_out = M^T u_in (N):  z = L^{-T} u;  [A_S^T z; sqrt(lam) z] */
#define ORC_MTV(out, in)                                                                  \
    do {                                                                                  \
        for (int a_ = 0; a_ < s; ++a_) z[a_] = (in)[a_];                                  \
        lsolve_upper_t(s, L, z);                                                          \
        for (int64_t k_ = 0; k_ < n; ++k_) {                                              \
            double acc_ = 0.0;                                                            \
            for (int a_ = 0; a_ < s; ++a_) acc_ += AS[(size_t)a_ * n + k_] * z[a_];       \
            (out)[k_] = acc_;                                                             \
        }                                                                                 \
        for (int a_ = 0; a_ < s; ++a_) (out)[n + a_] = sl * z[a_];                        \
    } while (0)
    for (int a = 0; a < s; ++a) u[a] = r[a];
    lsolve_lower(s, L, u); /* c = L^{-1} r */
    double beta = sqrt(dot(s, u, u));
    int it = 0;
    if (beta > 0.0) {
        for (int a = 0; a < s; ++a) u[a] /= beta;
        ORC_MTV(v, u);
        double alpha = sqrt(dot(N, v, v));
        if (alpha > 0.0) {
            for (int64_t k = 0; k < N; ++k) v[k] /= alpha;
            for (int64_t k = 0; k < N; ++k) wd[k] = v[k];
            double phibar = beta, rhobar = alpha;
            double *Mv = (double *)malloc(sizeof(double) * (size_t)s);
            double *Mtu = (double *)malloc(sizeof(double) * (size_t)N);
            for (it = 0; it < t_max; ++it) {
                ORC_MV(Mv, v);
                for (int a = 0; a < s; ++a) u[a] = Mv[a] - alpha * u[a];
                beta = sqrt(dot(s, u, u));
                if (beta > 0.0)
                    for (int a = 0; a < s; ++a) u[a] /= beta;
                ORC_MTV(Mtu, u);
                for (int64_t k = 0; k < N; ++k) Mtu[k] -= beta * v[k];
                alpha = sqrt(dot(N, Mtu, Mtu));
                if (alpha > 0.0)
                    for (int64_t k = 0; k < N; ++k) v[k] = Mtu[k] / alpha;
                const double rho = sqrt(rhobar * rhobar + beta * beta);
                const double c = rhobar / rho, sn = beta / rho;
                const double theta = sn * alpha;
                rhobar = -c * alpha;
                const double phi = c * phibar;
                phibar = sn * phibar;
                for (int64_t k = 0; k < N; ++k) {
                    x[k] += (phi / rho) * wd[k];
                    wd[k] = v[k] - (theta / rho) * wd[k];
                }
                if (beta == 0.0 || alpha == 0.0) {
                    ++it;
                    break;
                }
            }
            free(Mv);
            free(Mtu);
        }
    }
#undef ORC_MV
#undef ORC_MTV
    for (int64_t k = 0; k < n; ++k) w[k] = x[k];
    free(u);
    free(z);
    free(v);
    free(wd);
    free(x);
    return it;
}

/* K++ with the inexact projection of Sec. 4.1: as orc_run (the block draw, the momentum update of
 * Alg. 1, the window sums, checkpoints, stop rule and adaptive rho of Alg. 3), with the block step's
 * w = A_S^T (A_S A_S^T + lam I)^{-1} r replaced by t_max iterations of sketch-preconditioned LSQR on
 * min |A_S w - r|^2 + lam |w|^2 (orc_proj_lsqr).  Lsk: the preconditioners from orc_proj_precond, block
 * j at Lsk + j s s (len x len, leading dimension len).  K++ only. */
int orc_run_lsqr(int64_t rows, int64_t n, const double *A, const double *b, const double *Lsk, int t_max,
                 const orc_params *p, orc_state *st, double *x, double *mom, orc_report *rep) {
    if (p->s <= 0 || rows <= 0 || n <= 0 || p->cd || t_max < 1) return ORC_BAD_ARG;
    const int s = p->s;
    const int64_t nb = nblocks(rows, s), zeta = nb;
    const double bn2 = dot(rows, b, b);
    double *r = (double *)malloc(sizeof(double) * (size_t)s);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    const int64_t it0 = st->t;
    int status = ORC_NO_CONVERGENCE;
    rep->rel_res_est = NAN;
    while (st->t < p->max_iters) {
        const int64_t t = st->t;
        const int64_t j = orc_sample_block(p->seed, t, p->sys, (int32_t)nb);
        const int len = block_len(rows, s, j);
        const double *AS = A + (size_t)j * s * n;
        double rn2 = 0.0;
        for (int a = 0; a < len; ++a) {
            r[a] = dot(n, AS + (size_t)a * n, x) - b[j * s + a];
            rn2 += r[a] * r[a];
        }
        orc_proj_lsqr(n, AS, len, r, p->lam, Lsk + (size_t)j * s * s, t_max, w);
        const double beta = (1.0 - st->rho) / (1.0 + st->rho);
        for (int64_t k = 0; k < n; ++k) {
            mom[k] = beta * (mom[k] - w[k]);
            x[k] = x[k] - w[k] + p->eta * mom[k];
        }
        st->t = t + 1;
        if ((t % (2 * zeta)) < zeta) st->E0 += rn2; else st->E1 += rn2;
        if ((t % (2 * zeta)) == 2 * zeta - 1) {
            st->ci += 1;
            rep->rel_res_est = bn2 > 0.0 ? sqrt(st->E1 / bn2) : sqrt(st->E1);
            if (p->tol > 0.0 && st->E1 <= p->tol * p->tol * bn2 &&
                (!p->confirm || orc_rel_residual(rows, n, A, b, x) <= p->tol)) {
                status = ORC_OK;
                break;
            }
            if (p->adaptive) {
                const double q = st->E0 > 0.0 ? st->E1 / st->E0 : 0.0;
                if (st->ci == 1) {
                    st->rhat = q;
                } else {
                    const double li = log((double)st->ci), li1 = log((double)st->ci + 1.0);
                    const double wgt = exp(li * li - li1 * li1);
                    st->rhat = wgt * st->rhat + (1.0 - wgt) * q;
                }
                double rho = 1.0 - pow(st->rhat, 1.0 / (double)zeta);
                if (!(rho > 0.0)) rho = 0.0;
                if (rho > 1.0 - 1e-12) rho = 1.0 - 1e-12;
                st->rho = rho;
            }
            st->E0 = 0.0;
            st->E1 = 0.0;
        }
    }
    rep->iters = st->t - it0;
    rep->rel_res_true = orc_rel_residual(rows, n, A, b, x);
    rep->status = status;
    free(r);
    free(w);
    return status;
}
