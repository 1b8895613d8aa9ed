// kpp_solve.h -- launch descriptors of the persistent solve kernel (host and device view).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kpp.h"

namespace kpp {

// Per right-hand-side column state, kept in device memory between launches (resume, refinement).
struct SolveScalars {
    double E0, E1, rhat, rho, bn2, res_est;
    long long ci;   // checkpoints completed
    long long t;    // next iteration index (written back by the kernel)
    int active;     // 1 while the column iterates
    int status;     // kpp_status of the column
};

// One system of a launch.
struct SysArgs {
    const void *A;       // rows x cols, storage type
    int64_t lda;
    const void *b;       // rows x k, compute type (TC)
    void *x;             // cols x k, TC
    void *m;             // cols x k, TC
    void *Rx, *Rm;       // CD++: n x k, TC (maintained residual and A m)
    const void *Ginv;    // nb x s x s, TC
    void *part;          // G x s x KP, TC (K++ partial residuals)
    void *rbuf;          // s x KP, TC
    void *ybuf;          // s x KP, TC
    double *rpart;       // G x KP
    SolveScalars *sc;    // k
    unsigned *bar;       // group barrier counter
    int *err;            // group error word
    uint32_t sys_id;
    int64_t t0;
};

// Shared by every system of a launch.
struct Common {
    int64_t rows, cols;
    int s, nb, k;
    int64_t CW;          // columns per CTA (multiple of the 32-byte sector)
    int G;               // CTAs per system
    double eta, tol;
    int adaptive, confirm;
    int reduce_redundant;  // K++: every CTA reduces the partial residuals itself (small G * s * k)
    int init_residual;     // CD++: compute R_x = A x0 - b at start
    int64_t max_iters;
    uint64_t seed;
    uint64_t timeout_ns;
    int t0_state;          // 1: start at sc[0].t (written by the previous launch) and run max_iters more steps
    int test_hold_cta;     // wait test (general kernel only): this CTA of each group never arrives at the
                           // first group barrier, so the others' bounded wait runs out; -1: off
};

size_t solve_smem_bytes(int s, int KP, int64_t CW, size_t tc_size);
int pick_kp(int k);
cudaError_t launch_solve(int dtype, bool fp64_compute, bool cd, const SysArgs *d_sys, int nsys, const Common &cm,
                         int KP, cudaStream_t st);
int residual_grid();
cudaError_t launch_sample_blocks(uint64_t seed, uint32_t sys, int64_t t0, int64_t count, int32_t nb, int32_t *out,
                                 cudaStream_t st);
cudaError_t launch_residual(const kpp_matrix &A, int k, const double *b, const double *x, float *r32, double *part,
                            cudaStream_t st);
// skip (device, may be null): the kernel returns at once when *skip != 0
cudaError_t launch_residual_grid(const kpp_matrix &A, int k, const double *b, const double *x, float *r32,
                                 double *part, int grid, cudaStream_t st, const int *skip = nullptr);
cudaError_t launch_axpy(int64_t n, const float *d, double *x, cudaStream_t st);
cudaError_t launch_f64_to_f32(int64_t n, const double *a, float *o, cudaStream_t st);
cudaError_t launch_negate_copy(size_t n, const void *src, void *dst, bool f64, cudaStream_t st);

// Small-block kernel (kpp_solve2.cu).
bool solve2_eligible(const kpp_matrix &A, int s, int64_t CW, int KP, bool f64, bool cd, int G);
// The large-block K++ kernel with the W memo (kpp_kw.cu): FP32 iterations, one right-hand side.
int64_t kw_grid(int64_t cols);
size_t kw_mail_bytes(int s, int G);
size_t sysk_bytes();
void sysk_fill(void *dst, const void *tmA, const void *tmW, const float *b, float *x, SolveScalars *sc, unsigned *bar,
               int *err, double *rpart, void *mail, uint32_t sys_id, int64_t t0);
cudaError_t launch_kw(int dtype, const void *d_sys, int nsys, const Common &cm, cudaStream_t st);
bool kw_can_launch(int dtype, int s, int64_t cols, int nsys);
// The single-column dataflow CD++ kernel (kpp_cd3.cu): FP64 over the memo W, FP32 over W32.
bool cd4_fits(int s, int64_t CW, int es);
cudaError_t launch_cd4(int dtype, const void *d_sys, int nsys, const Common &cm, cudaStream_t st);
bool make_tmap_2d(void *out, const void *base, int dtype, uint64_t cols, uint64_t rows, uint64_t ld_elems,
                  uint32_t box_cols, uint32_t box_rows, bool swizzle128 = false);
size_t sys2_bytes();
void sys2_fill(void *dst_host, const SysArgs &a, const void *tmap);
cudaError_t launch_solve2(int dtype, bool cd, const void *d_sys, int nsys, const Common &cm, int KP, cudaStream_t st);

// Dataflow CD++ kernel (kpp_cd3.cu).
size_t cd3_smem_bytes(int s, int64_t CW, int KP, int ta_size, int tc_size, bool use_w);
size_t cd3_mail_bytes(int s, int KP, bool f64);
size_t sys3_bytes();
void sys3_fill(void *dst_host, const SysArgs &a, const void *tmap, void *mail);
cudaError_t launch_cd3(int dtype, const void *d_sys, int nsys, const Common &cm, int KP, cudaStream_t st);

// Streaming batched K++ kernel for wide FP32 / BF16 systems (kpp_stream.cu).
size_t sys4_bytes();
void sys4_fill(void *dst, const void *tmap, const float *b, float *X, float *M, const float *Ginv, float *part,
               double *rpart, SolveScalars *sc, unsigned *bar, int *err, uint32_t sys_id, int64_t t0);
int stream_tk(int dtype);
size_t stream_smem_bytes(int s, int KP);
int stream_per_sm(int dtype, int s, int KP);
int stream_min_tiles();  // fewest column tiles of one CTA's chunk
cudaError_t launch_stream(int dtype, const void *d_sys, int nsys, const Common &cm, int KP, cudaStream_t st);

}  // namespace kpp
