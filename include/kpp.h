/*
 * kpp.h -- C ABI of the GB300 (sm_103a) Kaczmarz++ / CD++ block-step library (libkpp.so).
 *
 * Method: Derezinski, Needell, Rebrova, Yang, "Randomized Kaczmarz Methods with Beyond-Krylov
 * Convergence" (arXiv 2501.11673).  Each solver iteration is one block step:
 *   1. draw a block S of a fixed contiguous row partition (Alg. 1, "draw a random S from B");
 *   2. block residual r = A_S x - b_S (Alg. 5) -- for CD++ the residual is kept up to date;
 *   3. regularised projection y = (A_S A_S^T + lam I)^{-1} r (Eq. 1.3), or (A_SS + lam I)^{-1} r for
 *      CD++ (Eq. 5.1), applied through a per-block factor memoised once (Sec. 4, Sec. 5.2);
 *   4. w = A_S^T y (CD++: w = I_S^T y), m <- (1-rho)/(1+rho) (m - w), x <- x - w + eta m (Eq. 1.4);
 *   5. residual estimate, adaptive rho and the stopping rule every 2 zeta steps (Eq. 5.2, Eq. 5.3,
 *      the checkpoints of Alg. 3 and Alg. 5), confirmed by the true FP64 residual |Ax - b|/|b|.
 *
 * Conventions shared by every entry point:
 *   - Matrices are row-major with a leading dimension `ld` (elements).  A `kpp_matrix` names memory
 *     the caller owns; the library never frees it.  Unless an entry point says otherwise, matrix and
 *     vector pointers are DEVICE pointers on the current CUDA device.
 *   - b and x are FP64 whatever the storage type of A.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Work is
 *     stream-ordered.  Calls that fill a host `kpp_report` synchronise that stream before returning.
 *   - Every call returns a kpp_status.  KPP_OK is 0.  On failure, kpp_last_error() returns a
 *     thread-local message.  No entry point aborts the process or traps the GPU.  Device-side waits
 *     are bounded; when the bound is hit the call returns KPP_ERR_TIMEOUT.
 *   - Block partition: block j holds rows [j s, min((j+1) s, rows)), and nb = ceil(rows / s).
 *   - Block draw at step t of system `sys_id`: out = Philox4x32-10(counter = {t_lo, t_hi, sys_id, 0},
 *     key = {seed_lo, seed_hi}) (Salmon et al., SC'11).  j = (out[0] * nb) >> 32.
 */
#ifndef KPP_H
#define KPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Storage type of the matrix entries. */
typedef enum { KPP_F64 = 0, KPP_F32 = 1, KPP_BF16 = 2 } kpp_dtype;

typedef enum {
    KPP_OK = 0,
    KPP_ERR_ARG = 1,            /* invalid argument: null pointer, bad size, dtype or partition mismatch */
    KPP_ERR_CUDA = 2,           /* a CUDA runtime call failed (message in kpp_last_error) */
    KPP_ERR_OOM = 3,            /* device allocation failed */
    KPP_ERR_NOT_SPD = 4,        /* a block matrix had a non-positive Cholesky pivot (report.bad_block) */
    KPP_ERR_NUMERIC = 5,        /* NaN or Inf appeared in the iterate or in a scalar */
    KPP_ERR_NO_CONVERGENCE = 6, /* max_iters (or max_outer) reached; x holds the last iterate */
    KPP_ERR_TIMEOUT = 7,        /* a bounded device-side wait expired; x holds the last iterate */
    KPP_ERR_BUDGET = 8,         /* a serving request does not fit the memory budget */
    KPP_ERR_UNSUPPORTED = 9     /* a combination the library does not implement */
} kpp_status;

/* A dense row-major matrix in caller-owned memory. */
typedef struct {
    const void *data;  /* first entry */
    int32_t dtype;     /* kpp_dtype */
    int32_t reserved;
    int64_t rows;
    int64_t cols;
    int64_t ld;        /* leading dimension in elements, >= cols */
} kpp_matrix;

/* Library-owned handles. */
typedef struct kpp_partition_s *kpp_partition_t;
typedef struct kpp_factors_s *kpp_factors_t;
typedef struct kpp_state_s *kpp_state_t;

/* Solver parameters.  Fill with kpp_params_default() and override fields as needed. */
typedef struct {
    double lambda;         /* Tikhonov regulariser (Eq. 1.3); must equal the factors' lambda */
    double tol;            /* eps: stop when |Ax-b|/|b| <= eps (Alg. 3's stop test) */
    int64_t max_iters;     /* cap on block iterations (per inner solve when refining) */
    uint64_t seed;         /* Philox key */
    uint32_t sys_id;       /* Philox stream id (system / request index) */
    int32_t adaptive_rho;  /* 1: adaptive rho (Eq. 5.3); 0: rho fixed at rho0 */
    double rho0;           /* initial rho (the paper starts from 0) or the fixed rho */
    double eta;            /* momentum step; NaN selects s / (2 min(rows, cols)) (Sec. 5.4) */
    int32_t grid;          /* CTAs per system; 0 selects automatically; KPP_GRID_TUNE (-1) autotunes */
    int32_t refine;        /* mixed precision: outer FP64 iterative refinement (F32/BF16 storage) */
    int32_t max_outer;     /* cap on refinement steps */
    int32_t reserved0;
    double inner_tol;      /* relative tolerance of each inner (FP32) solve */
    int64_t reserved1[4];
} kpp_params;

/* What a solve did. */
typedef struct {
    int64_t iters;         /* block iterations performed (all inner solves together) */
    int64_t outer;         /* refinement steps (0 without refinement) */
    double rel_res_true;   /* |A x - b| / |b| in FP64 at return */
    double rel_res_est;    /* sqrt(E1) / |b| at the last checkpoint (NaN if none) */
    double rho_final;      /* rho at return */
    int32_t status;        /* kpp_status of the solve */
    int32_t bad_block;     /* first block whose factorisation failed, else -1 */
    double device_ms;      /* device time of the solve (CUDA events on `stream`) */
    double kernel_ms;      /* of which inside the persistent iteration kernel's launches */
    int64_t launches;      /* launches of the persistent iteration kernel */
    int64_t reserved[2];
} kpp_report;

/* Defaults: lambda 0, tol 1e-8, max_iters 10^6, seed 0, adaptive rho from 0, eta NaN (s/(2 min)),
 * grid 0 (auto), refine 0, max_outer 20, inner_tol 1e-3. */
kpp_params kpp_params_default(void);

/* Human-readable name of a status code (static storage). */
const char *kpp_status_string(kpp_status st);

/* Message of the last failing call on this thread (empty string if none). */
const char *kpp_last_error(void);

/* Fixed contiguous partition of `rows` rows into blocks of `s` rows: the block collection B of
 * Alg. 1, held fixed so that every block's factor is memoised up front (Sec. 4).  The last
 * block holds rows mod s rows when s does not divide rows.  Errors: KPP_ERR_ARG if rows < 1, s < 1
 * or s > 1024.  Host-only; no device memory is used.  Free with kpp_partition_destroy. */
kpp_status kpp_partition(int64_t rows, int32_t s, kpp_partition_t *out);
void kpp_partition_destroy(kpp_partition_t p);
/* Number of blocks nb = ceil(rows / s) of a partition (0 for a null handle). */
int64_t kpp_partition_blocks(kpp_partition_t p);

/* Memoised per-block factors (Sec. 4; Sec. 5.2; Alg. 1; Alg. 3).
 *   mode 0 (K++):  G_j = A_{S_j} A_{S_j}^T + lambda I  (the block Gram; for F32/BF16 storage it is
 *                  built on the tensor cores with FP32 accumulation, then widened to FP64);
 *   mode 1 (CD++): G_j = A_{S_j S_j} + lambda I  (the principal block; A must be square and symmetric).
 * For every block the library stores the lower Cholesky factor L_j (G_j = L_j L_j^T; held in FP64,
 * computed in FP32 for F32/BF16 storage unless the block is ill-conditioned, see
 * kpp_factors_fp64_blocks) and the inverse G_j^{-1} = L_j^{-T} L_j^{-1} formed from it.  The inverse turns each per-step projection
 * into a parallel s x s matrix-vector product instead of two depth-s substitutions.  With F32/BF16
 * storage it also keeps an FP32 copy of G_j^{-1} for the inner solves.
 * A: device matrix, rows x cols (K++), or n x n symmetric (CD++).  Its rows must equal the
 * partition's rows.  The factors are device memory owned by the handle.  They stay valid while A is
 * unchanged.  Errors: KPP_ERR_ARG, KPP_ERR_OOM, KPP_ERR_CUDA, and KPP_ERR_NOT_SPD when a pivot is
 * <= 0 or not finite.  On NOT_SPD, *out is still created and kpp_factors_bad_block names the block.
 * Synchronises `stream`. */
kpp_status kpp_factor_blocks(const kpp_matrix *A, kpp_partition_t P, double lambda, int32_t mode,
                             kpp_factors_t *out, void *stream);
void kpp_factors_destroy(kpp_factors_t f);
/* First block whose factorisation failed, or -1. */
int64_t kpp_factors_bad_block(kpp_factors_t f);
/* Number of blocks whose Cholesky factor was computed in FP64.  FP64 storage: every block.  FP32/BF16
 * storage: the Cholesky runs in FP32 (the Gram carries FP32 accuracy and the inner solves use an FP32
 * inverse), and a block is refactored in FP64 only when the FP32 pass finds it too ill-conditioned
 * for FP32 elimination: a non-positive or non-finite FP32 pivot, or a ratio of largest to smallest
 * pivot L_cc^2 (a lower bound on kappa(G_j)) above 2^24 / (s + 1), where the smallest pivot reaches the
 * FP32 factor's rounding floor.  Below that the FP32 factor's backward error, (s + 1) 2^-24
 * componentwise, is no larger than the FP32-accumulated Gram's own.  -1 for a null handle. */
int64_t kpp_factors_fp64_blocks(kpp_factors_t f);
/* Copy rows row0 .. row0+nrows-1 of the FP32 memo W (block j's rows: W_j = G_j^{-1} A_{S_j}, Sec. 4's
 * projection folded into one operator; rows x cols, row-major) to host memory out_host (nrows * cols
 * floats).  The memo exists for BF16 / FP32 storage where the large-block K++ kernel or the
 * single-column CD++ kernel takes the shape.  For tests and inspection.  Errors: KPP_ERR_ARG when f
 * holds no FP32 memo or the rows are out of range; KPP_ERR_CUDA. */
kpp_status kpp_factors_get_memo(kpp_factors_t f, int64_t row0, int64_t nrows, float *out_host);
/* Device time of the factor phase that made f, in milliseconds, from events recorded on its stream:
 * ms_out[0] the block Grams G_j = A_Sj A_Sj^T + lambda I (K++) or principal blocks (CD++),
 * ms_out[1] the Cholesky of every block, ms_out[2] the inverses G_j^{-1}, ms_out[3] the memo
 * W_j = G_j^{-1} A_Sj where one is built (about 0 otherwise).  NaN for a stage that did not run
 * (a factor phase that failed early).  For measurement (Sec. 4's factor phase, the s^3/3 per block
 * the paper counts).  ms_out: host, 4 doubles.  Waits for the phase's last event.
 * Errors: KPP_ERR_ARG for a null argument. */
kpp_status kpp_factors_stage_ms(kpp_factors_t f, double *ms_out);
/* Copy the FP64 factor L_j (len x len, row-major, lower; len = length of block j) to host memory
 * `out` (len*len doubles).  For tests and inspection.  Errors: KPP_ERR_ARG for a bad j. */
kpp_status kpp_factors_get_block(kpp_factors_t f, int64_t j, double *out_host);

/* Kaczmarz++ solve of A x = b: Alg. 5 with exact memoised projections (the K++(Cholesky) variant of
 * App. F), a fixed partition, no randomised Hadamard preprocessing.
 * A: device rows x cols, any dtype.  b: device FP64 [rows].  x: device FP64 [cols], holding x0 on
 * entry and the last iterate on return.  F: from kpp_factor_blocks(mode 0) on the same A and P.
 * With F32/BF16 storage and p->refine = 1, each outer step computes r = b - A x in FP64, solves
 * A d = r with FP32 K++ to p->inner_tol, and updates x += d in FP64.  Without refinement the
 * iteration runs in the storage precision of A (FP64 or FP32 arithmetic).
 * rep (host, may be NULL): filled on return.  Errors: KPP_ERR_ARG on shape, dtype or lambda
 * mismatch; KPP_ERR_NO_CONVERGENCE; KPP_ERR_NUMERIC; KPP_ERR_TIMEOUT; KPP_ERR_CUDA.
 * Synchronises `stream`. */
kpp_status kpp_solve(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P,
                     kpp_factors_t F, const kpp_params *p, kpp_report *rep, void *stream);

/* CD++ solve of A x = b for symmetric positive (semi)definite A (Eq. 5.1; Alg. 3 without the
 * randomised Hadamard transform).  The residual R_x = A x - b and R_m = A m are kept up to date
 * (R_m <- beta (R_m - u), R_x <- R_x - u + eta R_m with u = A_{:,S} y), so a step reads the block
 * rows of A once and gathers r = R_x[S].  At each checkpoint that passes the estimate, the residual is
 * recomputed from A and replaces R_x.  Arguments and errors are as for kpp_solve; F must come from
 * kpp_factor_blocks(mode 1); A is n x n. */
kpp_status cdpp_solve(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P,
                      kpp_factors_t F, const kpp_params *p, kpp_report *rep, void *stream);

/* ---- Krylov reference solvers (the comparison systems of Sec. 6) --------------------------------
 * FP64 solves of A x = b on the GPU for the time-to-tolerance comparison with CD++ / K++ on the same
 * system, one persistent cooperative launch each.  The paper counts their cost in flops: CG
 * 2n^2 + 11n per iteration, GMRES 2n^2 T + 4n T (T + 1) after T iterations.
 * kpp_cg: plain conjugate gradients for symmetric positive definite A (n x n FP64, row-major,
 *   ld >= n), x0 from x: r = b - A x, p = r; per iteration q = A p, alpha = r.r / p.q, x += alpha p,
 *   r -= alpha q, beta = r'.r' / r.r, p = r + beta p; stops when |r| <= tol |b| for the recurrence
 *   residual r, or after max_iters iterations.
 * kpp_gmres: restarted GMRES(restart) for any nonsingular square A (same layout), x0 from x; Arnoldi
 *   with classical Gram-Schmidt and one reorthogonalisation pass, Givens rotations; an inner step stops
 *   when the rotated residual |g_{j+1}| <= tol |b|, a cycle ends after `restart` steps with x += V y and
 *   the true residual starts the next one; max_iters counts Arnoldi steps (1 <= restart <= 512).
 * b, x: device FP64 vectors of n entries (x in: x0, out: the last iterate).  rep (host): iters
 *   (iterations / Arnoldi steps), outer (GMRES cycles), rel_res_true (|Ax - b| / |b| in FP64, computed
 *   after the solve), rel_res_est (the recurrence's estimate), kernel_ms.  Errors: KPP_ERR_ARG;
 *   KPP_ERR_NO_CONVERGENCE (x holds the last iterate); KPP_ERR_NUMERIC; KPP_ERR_TIMEOUT (a bounded
 *   device wait ran out); KPP_ERR_CUDA; KPP_ERR_OOM for the scratch (GMRES: (restart + 1) n doubles).
 *   Synchronises `stream`. */
kpp_status kpp_cg(const kpp_matrix *A, const double *b, double *x, double tol, int64_t max_iters, kpp_report *rep,
                  void *stream);
kpp_status kpp_gmres(const kpp_matrix *A, const double *b, double *x, int32_t restart, double tol, int64_t max_iters,
                     kpp_report *rep, void *stream);

/* ---- Checkpoint and resume ----------------------------------------------------------------------
 * The state of the iteration after step t (Alg. 5 for K++, Alg. 3 for CD++): the momentum m of
 * Eq. 1.4 (cols x k); for CD++ also the maintained residual R_x = A x - b and R_m = A m of Eq. 5.1
 * (rows x k); and per right-hand-side column the window sums E0 / E1, the weighted ratio rhat and
 * rho of Eq. 5.2 - 5.3, the checkpoint count, the next step index t, the active flag and the status.
 * The iterate x stays the caller's (device, cols x k).
 *
 * kpp_state_create: a fresh state (t = 0, m = 0) for a system of rows x cols (CD++: cd = 1 and
 *   rows = cols) with k right-hand sides (1..32); device memory owned by the handle.  Errors: ARG,
 *   OOM, CUDA.
 * kpp_solve_resume / cdpp_solve_resume: run p->max_iters more steps from the state, or fewer if every
 *   column meets the stop rule, then leave the state at the last step.  The first call on a fresh state
 *   starts from x (x0) with m = 0 (CD++: R_x = A x0 - b, R_m = 0) and takes rho0 from p.  Arguments and
 *   errors as for kpp_solve / cdpp_solve, with A FP64 (other storage: KPP_ERR_UNSUPPORTED) and b, x
 *   panels of the state's k columns; the state's shape must match (else KPP_ERR_ARG).  p->refine is
 *   ignored.  The solve runs on the general persistent kernel, which keeps m, R_x and R_m in the
 *   state's device memory, so a solve split into calls at any step follows the uninterrupted one
 *   bitwise when p (seed, sys_id, grid, lambda, tol, eta) is the same in every call.  rep->iters is the
 *   state's step index t after the call.  Synchronises `stream`.
 * kpp_state_bytes: size of the flat checkpoint of the state and x.
 * kpp_state_save: copy the state and x (device, cols x k FP64) into host_buf (at least
 *   kpp_state_bytes bytes).  kpp_state_load: restore a saved checkpoint into a state of the same
 *   shape, rows, cols, k and method, and its x into x.  The checkpoint is a header, the per-column
 *   scalars as this library lays them out, then x, m and for CD++ R_x and R_m, all FP64; it is meant
 *   for this library on machines of the same byte order.  Errors: ARG (null, short buffer, another
 *   shape or not a checkpoint), CUDA.  Both synchronise `stream`.
 * kpp_state_step: the state's next step index t (-1 for a null handle).
 * There is no counterpart in the paper for the save / load format itself. */
kpp_status kpp_state_create(int64_t rows, int64_t cols, int32_t k, int32_t cd, kpp_state_t *out);
void kpp_state_destroy(kpp_state_t st);
int64_t kpp_state_step(kpp_state_t st);
size_t kpp_state_bytes(kpp_state_t st);
kpp_status kpp_state_save(kpp_state_t st, const double *x, void *host_buf, size_t bytes, void *stream);
kpp_status kpp_state_load(kpp_state_t st, double *x, const void *host_buf, size_t bytes, void *stream);
kpp_status kpp_solve_resume(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P, kpp_factors_t F,
                            const kpp_params *p, kpp_state_t st, kpp_report *rep, void *stream);
kpp_status cdpp_solve_resume(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P, kpp_factors_t F,
                             const kpp_params *p, kpp_state_t st, kpp_report *rep, void *stream);

/* End-to-end host variants: A (rows x cols, dtype per A->dtype, row-major), b and x are HOST
 * pointers.  The call copies A and b to the device, factors, solves and copies x back.  Device
 * buffers are allocated and freed inside the call.  mode 0 = K++, 1 = CD++. */
kpp_status kpp_solve_host(const kpp_matrix *A_host, const double *b_host, double *x_host, int32_t s,
                          int32_t mode, const kpp_params *p, kpp_report *rep, void *stream);

/* |A x - b|_2 / |b|_2 with FP64 accumulation (stored entries widened exactly) -- the stopping
 * rule's confirmation (Alg. 3).  A, b, x: device.  Result to *out_host.  Synchronises. */
kpp_status kpp_rel_residual(const kpp_matrix *A, const double *b, const double *x, double *out_host,
                            void *stream);

/* Batched K++ over `nsys` independent systems that share shape, dtype and block size, each with a
 * panel of k right-hand sides: system i has matrix A[i] (device,
 * rows x cols), right-hand sides B[i] (device FP64, rows x k, row-major) and iterates X[i] (device
 * FP64, cols x k, row-major, x0 on entry).  Factors F[i] come from kpp_factor_blocks(mode 0).
 * Every RHS column runs its own rho, residual estimate and stopping rule, and the k columns of a
 * system share the block sequence of Philox stream sys_id = p->sys_id + i.  All systems advance in
 * one persistent launch (p->grid CTAs per system).  reps (host, may be NULL): nsys * k reports in
 * system-major order.  Errors are as for kpp_solve.  The worst status is returned. */
kpp_status kpp_solve_batched(int32_t nsys, const kpp_matrix *A, const double *const *B, double *const *X,
                             int32_t k, kpp_partition_t P, const kpp_factors_t *F, const kpp_params *p,
                             kpp_report *reps, void *stream);

/* The block indices the solver draws at steps t0 .. t0+count-1 of Philox stream `sys_id` (see the
 * draw rule above), computed on the device by the same code the solve kernel uses.  out: device
 * int32[count].  Errors: KPP_ERR_ARG for count < 0, nb < 1 or a null pointer.  Stream-ordered. */
kpp_status kpp_sample_blocks(uint64_t seed, uint32_t sys_id, int64_t t0, int64_t count, int32_t nb, int32_t *out,
                             void *stream);

/* CD++ FP64 solve that allocates no device memory.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc, such as a process whose GPU memory is owned by
 * another allocator (a serving runtime or framework pool that reserved the device) or a request
 * path that must not block on the allocator or fail half way with an out-of-memory error.
 * It runs the general CD++ kernel with the launch shape cdpp_solve picks, i.e. what cdpp_solve runs
 * after kpp_set_kernel_variant(1); the default variant's dataflow kernels reach the same iterates in
 * another summation order.  Same arguments and results as cdpp_solve.  The scratch
 * (momentum, maintained residuals, projection buffer, scalars, barrier words, partial sums) lives
 * in one fixed device array of about 400 KiB inside the library.  Every GPU that loads the library
 * holds that array until the process exits.
 * Limits: A FP64, n <= 16384, s <= 256, one right-hand side.  Larger sizes return KPP_ERR_ARG with
 * a message; nothing is allocated.  The caller passes A, b, x and factors made by
 * kpp_factor_blocks(mode 1).  No timing is taken (report.device_ms is NaN).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All calls share the one array
 * and it keeps the last call's contents (each call clears what must start at zero), so calls whose
 * work overlaps on the GPU -- on different streams, or from different threads -- race and must not
 * be issued.  Synchronises `stream`. */
kpp_status cdpp_solve_noalloc(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P, kpp_factors_t F,
                              const kpp_params *p, kpp_report *rep, void *stream);

/* The block Grams of the K++ factor phase (Sec. 4; Eq. 1.3): G_j = A_{S_j} A_{S_j}^T + lambda I for
 * every block of the contiguous partition into blocks of s rows.  A: device matrix (any dtype).
 * G_out: device FP64 buffer of nb * s * s doubles; block j is written at G_out + j*s*s as a len x len
 * row-major matrix (leading dimension len, len = rows of block j).  Only its lower triangle (with the
 * diagonal) is written; the caller owns G_out.
 * engine: 0 automatic (tensor cores for BF16 and FP32 storage -- FP32 as engine 3 -- CUDA cores for
 * FP64), 1 CUDA cores with FP64 accumulation, 2 tcgen05 tensor cores with FP32 accumulation and one
 * product per element pair (kind::f16 for BF16, exact products; kind::tf32 for FP32, i.e. products of
 * 11-bit mantissas), 3 FP32 storage only: each value split as hi + lo with hi its TF32 rounding, and
 * hi*hi + hi*lo + lo*hi on kind::tf32 (products good to about 2^-22).  *engine_used (may be NULL)
 * receives 1, 2 or 3.
 * Errors: KPP_ERR_ARG; KPP_ERR_UNSUPPORTED when engine 2 cannot take the matrix (FP64 storage, rows
 * not 16-byte aligned); KPP_ERR_CUDA.  Synchronises `stream`. */
kpp_status kpp_block_gram(const kpp_matrix *A, int32_t s, double lambda, int32_t engine, double *G_out,
                          int32_t *engine_used, void *stream);

/* Randomized Hadamard preprocessing of a symmetric system for CD++ (Sec. 5.1: Alg. 3's transform of
 * A and b before the loop and its return D FHT(x); the FHT / SymFHT appendix):
 *   Abar = Q A Q^T,  bbar = Q b,   Q = H_n D,  D = diag(d) / sqrt(n),
 * H_n the Sylvester-Hadamard matrix (H_1 = [1], H_2n = [[H_n, H_n], [H_n, -H_n]]).  Q is orthogonal, so
 * Abar is symmetric (PSD if A is) with A's spectrum, and x = Q^T xbar solves A x = b when xbar solves
 * Abar xbar = bbar; |Abar xbar - bbar| = |A x - b|.
 * n: a power of 2, 1 <= n <= 16384.  d: device, n FP64 signs +1 / -1 (the caller draws them).
 * A: device FP64 n x n, row-major (A->ld >= n), symmetric.  Abar: device, n x n, leading dimension n;
 * it may be A->data itself when A->ld = n.  b, bbar: device n x k panels (row-major, leading dimension
 * k; k = 0 transforms the matrix only and b, bbar may be NULL); bbar may equal b.
 * Two streaming passes over the matrix plus an n x n FP64 scratch allocated and freed on `stream`.
 * Errors: KPP_ERR_ARG (size, dtype, null pointer), KPP_ERR_OOM, KPP_ERR_CUDA.  Stream-ordered. */
kpp_status kpp_rht_forward(int64_t n, const double *d, const kpp_matrix *A, double *Abar, const double *b,
                           double *bbar, int32_t k, void *stream);

/* x = Q^T xbar = diag(d) H_n xbar / sqrt(n) for an n x k device panel (row-major, leading dimension k;
 * k >= 1); x may equal xbar.  Errors: KPP_ERR_ARG, KPP_ERR_CUDA.  Stream-ordered. */
kpp_status kpp_rht_inverse(int64_t n, const double *d, const double *xbar, double *x, int32_t k, void *stream);

/* The block sequence of the online block memoisation (Sec. 4, "Block memoization"; Sec. 5.2; the
 * sampling steps of Alg. 3 and Alg. 5) for steps t0 .. t0 + count - 1 of Philox stream sys_id, with nb0
 * blocks memoised before t0.  Step t samples a new uniformly random s-subset of the rows with
 * probability p_0 = 1, p_t = min(1, (n/s) ln(n) / t) (mode 1, CD++) or min(1, (m/s) ln(m) / t,
 * (n/s) ln(m) / t) (mode 0, K++), and otherwise reuses a memoised block picked uniformly.  The draws:
 * Philox4x32-10, key {seed_lo, seed_hi}; counter {t_lo, t_hi, sys_id, 0}: out[1] < p_t 2^32 means new,
 * out[2] |B| >> 32 is the pick; counter {t_lo, t_hi, sys_id, 1 + i/4}: word i mod 4 of Floyd's sampling
 * of the subset, which is returned sorted.  The sequence does not depend on the data, so a window can
 * be drawn before its steps run.
 * blocks (host, count entries): the memo index each step uses; a new block takes the next index
 * (nb0, nb0 + 1, ...).  subsets (host, subsets_cap x s): the new blocks' row indices, in order.
 * *nb_out: the number of memoised blocks after the window.  rows, cols: the shape of A (CD++: square).
 * Host only: no device memory and no stream.  Errors: KPP_ERR_ARG for an invalid argument, or when
 * the window draws more than subsets_cap new blocks (subsets_cap >= count always suffices; *nb_out
 * then holds the count reached). */
/* K++ (mode 0) or CD++ (mode 1) with the online block memoisation (Sec. 4 "Block memoization", Sec.
 * 5.2; the sampling steps of Alg. 3 and Alg. 5) instead of a fixed partition: step t samples a new
 * uniformly random s-subset S of the rows with probability p_t (as kpp_memo_sequence draws it) and
 * memoises the factor of its block (K++: chol(A_S A_S^T + lambda I), CD++: chol(A_SS + lambda I)), or
 * reuses a memoised block picked uniformly.  The step on S is Eq. 1.3 - 1.4 (K++) or Eq. 5.1 (CD++,
 * with the block residual r = A_S x - b_S computed directly); zeta = ceil(rows / s) sets the windows of
 * the residual estimate, the adaptive rho and the stop rule (Eq. 5.2 - 5.3), and a stop is confirmed
 * by the FP64 residual of the whole system.
 * A: device FP64, rows x cols, row-major (ld >= cols); CD++: square and symmetric.  b (rows) and x
 * (cols; in: x0, out: the result): device FP64, one right-hand side.  s: 1 <= s <= min(rows, 1024).
 * p: lambda, tol, max_iters, seed, sys_id, eta, rho0, adaptive_rho as for kpp_solve (grid and refine
 * are ignored).  rep (host, may be NULL): iters, rel_res_true (FP64, after the solve), rel_res_est,
 * rho_final, status, kernel_ms, launches.  *nblocks_out (may be NULL): the number of blocks memoised
 * by the steps that ran (a window's draws beyond a stop are not counted).
 * The solve runs in windows of max(256, min(16 zeta, 8192)) steps: the host draws the window's block
 * sequence, the rows of the new subsets are gathered into a device store (about blocks x s x (cols + s)
 * doubles) and factored in one batch, and a persistent kernel runs the window's steps from a table.
 * Errors: KPP_ERR_ARG; KPP_ERR_NOT_SPD (rep->bad_block: the memo index); KPP_ERR_NO_CONVERGENCE (x
 * holds the last iterate); KPP_ERR_OOM; KPP_ERR_CUDA; KPP_ERR_TIMEOUT.  Synchronises `stream`. */
kpp_status kpp_solve_memo(const kpp_matrix *A, const double *b, double *x, int32_t s, int32_t mode, const kpp_params *p,
                          kpp_report *rep, int64_t *nblocks_out, void *stream);

kpp_status kpp_memo_sequence(uint64_t seed, uint32_t sys_id, int32_t mode, int64_t rows, int64_t cols, int32_t s,
                             int64_t t0, int64_t count, int64_t nb0, int64_t *blocks, int64_t *subsets,
                             int64_t subsets_cap, int64_t *nb_out);

/* The inexact block projection of Sec. 4.1 ("Computing the projection step"; the supplement's Proj
 * algorithm): K++ on large blocks without an exact factor of A_S A_S^T.  The projection's
 * w = argmin |A_S w - r|^2 + lambda |w|^2 is taken from t_max iterations of LSQR (Paige and Saunders)
 * on M [w; v] = L^{-1} r, M = L^{-1} [A_S, sqrt(lambda) I], preconditioned by L L^T = Ahat Ahat^T +
 * lambda I with the subsampled randomized Hadamard sketch Ahat = (A_S D H_{n'})[:, T] / sqrt(tau):
 * n' = the smallest power of 2 >= cols (A_S padded with zero columns), H_{n'} the Sylvester Hadamard
 * matrix, D = diag(d).  FP64 only.
 *
 * kpp_factor_lsqr: the preconditioner of every block of P (whole blocks: rows a multiple of s,
 * 1 <= s <= 1024), memoised as a factor set (kpp_factors_get_block returns L_j).  A: device FP64,
 * rows x cols with n' <= 16384.  tau: 1 .. n' (the paper takes 2 s).  T (host, tau entries): the
 * sampled columns, in [0, n').  d (device, n' entries): the signs (entries beyond cols are unused).
 * *out: the factor set, or NULL on error; it is not accepted by kpp_solve or cdpp_solve.  Errors:
 * KPP_ERR_ARG; KPP_ERR_NOT_SPD (kpp_factors_bad_block; the handle is returned); KPP_ERR_OOM;
 * KPP_ERR_CUDA.  Synchronises `stream`. */
kpp_status kpp_factor_lsqr(const kpp_matrix *A, kpp_partition_t P, double lambda, int64_t tau, const int64_t *T,
                           const double *d, kpp_factors_t *out, void *stream);

/* One inexact projection: w (device, cols) from t_max LSQR iterations for block j and the residual r
 * (device, s entries), from zero.  F from kpp_factor_lsqr on A and P.  Errors: KPP_ERR_ARG; KPP_ERR_CUDA;
 * KPP_ERR_TIMEOUT.  Synchronises `stream`. */
kpp_status kpp_proj_lsqr(const kpp_matrix *A, kpp_partition_t P, kpp_factors_t F, int64_t j, const double *r,
                         int32_t t_max, double *w, void *stream);

/* K++ with the inexact projection: Alg. 1's step with w from t_max LSQR iterations (above) in place of
 * the exact projection.  The block draw, the momentum, the windows of the residual estimate, the
 * adaptive rho and the stop rule (Eq. 5.2 - 5.3, confirmed by the FP64 residual) are those of
 * kpp_solve.  A (device FP64), b (rows) and x (cols; in: x0, out: the result) on the device; F from
 * kpp_factor_lsqr with p->lambda.  p: lambda, tol, max_iters, seed, sys_id, eta, rho0, adaptive_rho.
 * rep (may be NULL) as for kpp_solve.  Errors: KPP_ERR_ARG; KPP_ERR_NO_CONVERGENCE (x holds the last
 * iterate); KPP_ERR_NUMERIC; KPP_ERR_TIMEOUT; KPP_ERR_CUDA.  Synchronises `stream`. */
kpp_status kpp_solve_lsqr(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P, kpp_factors_t F,
                          int32_t t_max, const kpp_params *p, kpp_report *rep, void *stream);

/* Select the solve kernel for later calls in this process.  All variants compute the same iteration.
 *   3 (default): CD++ uses the dataflow kernel (no per-step barrier: the owners of the next block
 *     hand r over through a tagged mailbox; FP64 streams the memoised W_j = G_j^{-1} A_{S_j}); K++ uses
 *     the small-block kernel; each only where the shape allows it, else as below;
 *   2: the small-block kernel (one barrier per step, TMA-prefetched tiles and memoised inverses) where
 *     the shape allows it (s even and <= 256, row stride a multiple of 16 bytes, per-CTA chunk <= 256
 *     columns, shared memory fits), else the general kernel;
 *   1: the general kernel always.
 * Not thread-safe with concurrent solves.  Errors: KPP_ERR_ARG for another value. */
kpp_status kpp_set_kernel_variant(int32_t variant);

/* Test hook for the bounded device waits (failure handling; no counterpart in the paper).  Every
 * spin-wait of the persistent kernels (group barriers, mailbox polls, TMA completion waits) gives up
 * after a time limit, marks the group's error word KPP_ERR_TIMEOUT, releases the other waiters and
 * returns; the solve then returns KPP_ERR_TIMEOUT with x holding the last written iterate, and the
 * CUDA context stays usable.
 *   wait_ns:  the limit for every later launch; 0 restores the default (2 s).
 *   hold_cta: -1 (default) off; c >= 0 makes CTA c of every system leave the general kernel before
 *             its first group barrier without arriving, so that the other CTAs' wait runs out.  A solve
 *             made while it is set must run the general kernel (kpp_set_kernel_variant(1)) on a grid of
 *             more than c CTAs per system, else it returns KPP_ERR_UNSUPPORTED without launching.
 * Process-wide, not thread-safe with concurrent solves.  Errors: KPP_ERR_ARG for hold_cta < -1. */
kpp_status kpp_set_wait_test(uint64_t wait_ns, int32_t hold_cta);

/* ------------------------------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over registered matrices, resident on the device.
 * Requests arrive at any time and are admitted FIFO as soon as device memory under the budget allows: a
 * request's panels and scratch next to the memoised block factors (Sec. 4, Sec. 5.2) of the matrices in
 * use, which stay resident for later requests on the same matrix (idle factors are evicted when the
 * budget needs the room).  An admitted request becomes jobs of at most 8 right-hand-side columns.  One
 * persistent kernel holds `max_concurrent` slots of `grid_per_solve` CTAs; each slot claims the next
 * job from a queue in mapped host memory and runs its whole solve (the FP64 refinement loop of the
 * mixed-precision form around FP32 inner solves, or one FP64 solve) with its own CTAs, then claims the
 * next.  Jobs are queued shortest expected work first (iterations seen on the matrix x n x columns),
 * at most two per slot ahead of the running ones, so work that arrives while other solves run is taken
 * up as slots free up and overlaps with them.  The host launches no kernel per request; a library
 * thread publishes jobs, collects completions, and relaunches the loop after it has gone idle.  Factor
 * phases drain the loop first (they run on the whole GPU).  Solves are deterministic: a request's
 * result does not depend on the other requests in flight.
 * ------------------------------------------------------------------------------------------------ */
typedef struct kpp_server_s *kpp_server_t;

typedef struct {
    int64_t completed;      /* requests finished (any status) */
    int64_t failed;         /* requests finished with a status other than KPP_OK */
    double p50_ms, p99_ms, max_ms;  /* submission -> completion latency percentiles */
    double solves_per_s;    /* completed / (last completion - first submission) */
    double span_s;
    size_t peak_bytes;      /* largest device memory charged to the budget */
    size_t budget_bytes;
    int64_t loop_launches;  /* launches of the device-resident request loop so far */
    int64_t loop_slots;     /* slots of its last launch */
    int64_t reserved[2];
} kpp_serving_stats;

/* Create a server with a device-memory budget (bytes), `max_concurrent` slots of the request loop (jobs
 * in flight, 1..64; fewer when the GPU cannot hold that many at once) and `grid_per_solve` CTAs per slot
 * (0: 8; at most 64).  Uses the current CUDA device.  Errors: KPP_ERR_ARG; KPP_ERR_CUDA when the mapped
 * queue cannot be allocated. */
kpp_status kpp_server_create(size_t hbm_budget_bytes, int32_t max_concurrent, int32_t grid_per_solve,
                             kpp_server_t *out);
/* Register a device matrix (caller-owned, must outlive the server) for mode 0 (K++) or 1 (CD++; square
 * symmetric), block size s and regulariser lambda.  Factors are built on first use (with those of the
 * other registered matrices that fit half the budget).  *matrix_id receives its index.  Errors:
 * KPP_ERR_ARG, also when the block size and column chunk do not fit the loop's shared memory, or when
 * the server already holds 4096 matrices. */
kpp_status kpp_server_add_matrix(kpp_server_t sv, const kpp_matrix *A, int32_t s, double lambda, int32_t mode,
                                 int32_t *matrix_id);
/* Submit a request: B_host is rows x k (row-major FP64, copied before return), 1 <= k <= 32; p gives
 * tol, seed, sys_id, refine, ... (p->lambda is taken from the matrix).  Returns immediately with
 * *request_id.  KPP_ERR_BUDGET if the request alone cannot fit the budget (it is then complete with
 * that status). */
kpp_status kpp_server_submit(kpp_server_t sv, int32_t matrix_id, const double *B_host, int32_t k, const kpp_params *p,
                             int64_t *request_id);
/* Non-blocking: *done = 1 once the request finished; then X_host (cols x k FP64, may be NULL) and reps
 * (k reports, may be NULL) are filled and the request's status is returned. */
kpp_status kpp_server_poll(kpp_server_t sv, int64_t request_id, double *X_host, kpp_report *reps, int32_t *done);
/* Block until no request is queued or running, at most timeout_s seconds (KPP_ERR_TIMEOUT). */
kpp_status kpp_server_wait_all(kpp_server_t sv, double timeout_s);
kpp_status kpp_server_stats(kpp_server_t sv, kpp_serving_stats *out);
/* Start a new statistics window: latencies, completed / failed counts, the first-submission time and
 * the peak are reset (requests already submitted stay pollable).  Errors: KPP_ERR_ARG (null server). */
kpp_status kpp_server_reset_stats(kpp_server_t sv);
/* Stop the server: requests already submitted finish first, then the request loop is drained, its
 * thread joined, and the factors, the mapped queue and the device buffers freed. */
void kpp_server_destroy(kpp_server_t sv);

/* Batched CD++ (Eq. 5.1, Alg. 3): as kpp_solve_batched, for square symmetric systems whose factors
 * come from kpp_factor_blocks(mode 1); the k columns of a system share its block sequence and each has
 * its own rho, residual estimate and stop test. */
kpp_status cdpp_solve_batched(int32_t nsys, const kpp_matrix *A, const double *const *B, double *const *X, int32_t k,
                              kpp_partition_t P, const kpp_factors_t *F, const kpp_params *p, kpp_report *reps,
                              void *stream);

/* ---- Prepared batched solves (CUDA-graph capturable) ------------------------------------------
 *
 * A plan is the batched solve of kpp_solve_batched (mode 0, K++, Alg. 3 / Sec. 4) or
 * cdpp_solve_batched (mode 1, CD++, Alg. 5 / Sec. 5) with its systems, buffers and launch shape fixed
 * once.  The paper describes one solve at a time; batching the systems of one shape into one
 * persistent launch, and making that launch replayable, is this library's addition.
 *
 * kpp_plan_create checks the arguments as kpp_solve_batched does, chooses the kernel and the CTAs
 * per system (p->grid > 0: that many; 0: the built-in heuristic; KPP_GRID_TUNE (-1): the launch
 * autotuner below), allocates every scratch buffer, builds the TMA descriptors, and synchronises
 * `stream`.  A, B, X and F are bound to the plan: their device buffers must outlive it and keep their
 * addresses; their contents may change between launches.  The plan owns its scratch (freed by
 * kpp_plan_destroy).  Errors: those of kpp_solve_batched, KPP_ERR_OOM, KPP_ERR_UNSUPPORTED (the
 * systems x CTAs do not fit co-resident).
 *
 * kpp_plan_launch enqueues one complete solve of every system on `stream`: kernels and memsets only
 * (no allocation, no host synchronisation, no host copy), so it may be called while `stream` is being
 * captured into a CUDA graph, and the graph replayed.  On entry X holds the initial guesses (zero for
 * the default start); on completion it holds the solutions.  With F32 / BF16 storage and
 * p->refine = 1 the FP64 refinement loop runs on the device: each of p->max_outer steps computes
 * r = b - A x, stops the systems whose columns all satisfy |r| <= tol |b|, solves A d = r in FP32 for
 * the rest and adds d to x; steps after every system has stopped do no work.  A system whose inner
 * solve reports a device error stops there (its x keeps the last completed update).  Returns
 * KPP_ERR_ARG (null plan) or KPP_ERR_CUDA / KPP_ERR_UNSUPPORTED when a launch cannot be enqueued.
 *
 * kpp_plan_report synchronises `stream`, then writes nsys * k reports (system-major) with the true
 * FP64 relative residual of X, iterations, refinement steps, rho and the per-column status, and
 * returns the first non-OK column status (KPP_OK when every column met the tolerance).  device_ms
 * is 0: time plan launches with events on the caller's stream.
 *
 * kpp_plan_info returns the kernel (1 general, 2 small-block, 3 dataflow CD++, 4 streaming), the CTAs
 * per system and the kernel generation limit the plan uses (any pointer may be NULL). */
#define KPP_GRID_TUNE (-1)
typedef struct kpp_plan_s *kpp_plan_t;
kpp_status kpp_plan_create(int32_t nsys, const kpp_matrix *A, const double *const *B, double *const *X, int32_t k,
                           kpp_partition_t P, const kpp_factors_t *F, const kpp_params *p, int32_t mode, void *stream,
                           kpp_plan_t *out);
kpp_status kpp_plan_launch(kpp_plan_t plan, void *stream);
kpp_status kpp_plan_report(kpp_plan_t plan, kpp_report *reps, void *stream);
kpp_status kpp_plan_info(kpp_plan_t plan, int32_t *kernel, int32_t *grid, int32_t *variant);
/* Waits for the device to go idle, then frees the plan's scratch.  NULL is ignored. */
void kpp_plan_destroy(kpp_plan_t plan);

/* ---- Block-size autotuner ------------------------------------------------------------------------
 * Picks the block size s of the contiguous partition (the s of Alg. 1 / Alg. 5, which the paper fixes
 * by hand) for nsys systems A_i (same shape and storage) with right-hand-side panels B_i (device FP64,
 * rows x k), among the ncand candidates cand[] (1 <= cand <= min(1024, rows)).  For each candidate:
 * the factor phase of every system (its device time), then two segments of T = 6 zeta steps (24 ..
 * 1024) of the solve kernel with no stop test (the launch shape the heuristic picks; FP32 iterations
 * for FP32 / BF16 storage, FP64 otherwise): the first from x = 0 as a burn-in, the second continuing
 * from its x, each followed by every column's FP64 residual.  The contraction per step q is the
 * geometric mean over the columns of |r_2T| / |r_T|, to the power 1 / T, and the estimate of the time
 * to a relative residual p->tol is  factor ms + ms per step * (2T + log(tol / rel_2T) / log(q)).
 * out_s (host): the candidate with the smallest estimate.  est_ms (host, ncand doubles, may be NULL):
 * every estimate (INFINITY for a candidate that did not run or did not contract).  p: lambda, tol
 * (0 < tol < 1), seed, sys_id, eta, rho0 and adaptive_rho as for the solve.  cd = 1 tunes CD++ (square
 * A).  Errors: KPP_ERR_ARG; KPP_ERR_NO_CONVERGENCE when no candidate contracts; KPP_ERR_CUDA, OOM.
 * Synchronises `stream`; allocates the candidates' factors one at a time. */
kpp_status kpp_tune_block_size(int32_t nsys, const kpp_matrix *A, const double *const *B, int32_t k,
                               const int32_t *cand, int32_t ncand, const kpp_params *p, int32_t cd, int32_t *out_s,
                               double *est_ms, void *stream);

/* ---- Launch autotuner ------------------------------------------------------------------------------
 *
 * p->grid = KPP_GRID_TUNE in kpp_plan_create, kpp_solve, cdpp_solve or the batched solves times short
 * runs (about two sweeps over the blocks, no stop test, from x = 0 on the caller's right-hand sides)
 * of the persistent kernel for the kernel generations allowed by kpp_set_kernel_variant and a few CTA
 * counts around the heuristic's, and keeps the fastest time per step.  The choice is cached per
 * (device, shape, dtype, s, k, mode, nsys, generation limit) for the life of the process.  The launch
 * shape changes the order of floating-point sums, so a tuned solve matches an untuned one to rounding
 * only; with the choice cached, repeated solves are bitwise identical.  The cache can be written to a
 * text file (one "key variant grid" line per shape) and read back, e.g. at start-up.
 * save/load errors: KPP_ERR_ARG (null path, unreadable or malformed file; nothing is loaded then). */
int64_t kpp_tune_cache_size(void);
void kpp_tune_cache_clear(void);
kpp_status kpp_tune_cache_save(const char *path);
kpp_status kpp_tune_cache_load(const char *path);

/* Number of kernel launches this library has issued in the process so far (every launch site counts
 * once; a captured graph's replays are not counted).  Host only, never fails. */
uint64_t kpp_launch_count(void);

/* Number of device allocation requests this library has made in the process so far: factor sets,
 * solve scratch, plans, the server's panels and the host-buffer solve.  A request served from the
 * library's caches (kpp_device_cache_bytes) counts as well.  Allocations that cuBLAS makes on its own
 * are not counted.  Host only, never fails. */
uint64_t kpp_device_alloc_count(void);

/* Device memory the library holds for reuse on the current device, in bytes (runtime memory
 * management; no counterpart in the paper).  Released long-lived buffers (factor sets, states, device
 * copies of host inputs) stay on a free list, up to a quarter of the device's memory, and are handed
 * out again for a request of the same size: repeated solves of one shape map their memory once.
 * Stream-ordered scratch comes from a pool that keeps freed memory across synchronisations.  Never
 * fails (0 without a device). */
size_t kpp_device_cache_bytes(void);

/* Return the memory of both caches on the current device to the driver.  Synchronises the device
 * first.  Errors: KPP_ERR_CUDA if the synchronisation or the pool trim fails. */
kpp_status kpp_device_cache_trim(void);

/* Library build information: "sm_103a; <compiler>; <date>". */
const char *kpp_build_info(void);

#ifdef __cplusplus
}
#endif

#endif /* KPP_H */
