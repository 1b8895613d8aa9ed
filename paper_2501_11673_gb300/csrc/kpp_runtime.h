// kpp_runtime.h -- host-side internals of libkpp shared between translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kpp.h"

namespace kpp {

// Thread-local last-error message (kpp_last_error).
void set_error(const char *fmt, ...);
void clear_error();

// Memoised factors of one matrix (Sec. 4 / Sec. 5.2), device memory owned by this struct.
struct FactorSet {
    int64_t nb = 0, rows = 0;
    int s = 0;
    int mode = 0;        // 0: K++ block Gram, 1: CD++ principal block, 2: LSQR sketch preconditioner
    int dtype = 0;       // storage dtype of the matrix the factors came from
    double lambda = 0.0;
    int64_t bad_block = -1;
    int64_t fp64_blocks = 0;  // blocks whose Cholesky ran in FP64 (all of them for FP64 storage)
    double *L = nullptr;      // nb x s x s, FP64 lower Cholesky factors (block j: len x len, ld len)
    double *Ginv = nullptr;   // nb x s x s, FP64 (G_j)^{-1}
    float *Ginv32 = nullptr;  // nb x s x s, FP32 copy (FP32/BF16 storage only)
    double *W = nullptr;      // CD++ FP64 only: rows x cols, block j rows = G_j^{-1} A_{S_j} (row-major, ld cols)
    float *W32 = nullptr;     // K++ with FP32/BF16 storage, large-block kernel only: G_j^{-1} A_{S_j} in FP32
    int64_t memo_cols = 0;    // columns of W / W32 (the matrix's columns)
    double *Linv = nullptr;   // mode 2 (sketch preconditioners of the LSQR projection): nb x s x s L_j^{-1}
    double *LinvT = nullptr;  // mode 2: L_j^{-T} (so that both products read rows)
    // Device time of the factor phase's stages (kpp_factors_stage_ms): events recorded on the stream
    // before the Grams / principal blocks, then after the Cholesky, the inverses and the W memo.
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    void release();
};

kpp_status factor_blocks_impl(const kpp_matrix &A, int s, double lam, int mode, FactorSet &F, cudaStream_t st);
// FP64 Cholesky and inverse of nblk packed s x s Grams (G factored in place, G^{-1} into Ginv); the
// smallest block with a non-positive pivot goes to *bad_block and the call returns KPP_ERR_NOT_SPD.
kpp_status factor_grams(double *G, int64_t nblk, int s, double *Ginv, int64_t *bad_block, cudaStream_t st,
                        double *L_out = nullptr, double *Linv_out = nullptr);  // optional: keep L and L^{-1}

// Tensor-core block Gram for FP32/BF16 storage (kpp_gram_tc.cu).  Writes G (nb x s x s, FP64,
// block j packed with leading dimension len) and returns true, or returns false when the shape is
// not supported by the tensor-core kernel (the caller then uses the CUDA-core kernel).
// FP32 storage goes through the tensor cores only when allow_tf32 is set (plain TF32 products).
bool gram_tc(const kpp_matrix &A, int s, double lam, double *G, cudaStream_t st, bool allow_tf32 = false);

// Block Grams only (lower triangles, FP64, packed per block with leading dimension len):
// engine 0 = automatic, 1 = CUDA cores with FP64 accumulation, 2 = tensor cores (BF16, or TF32 for
// FP32 storage).  Returns the engine used, or -1.
int block_gram(const kpp_matrix &A, int s, double lam, double *G, int engine, cudaStream_t st);

// The solve behind kpp_solve / cdpp_solve / kpp_solve_batched (nsys systems, k right-hand sides each).
kpp_status solve_systems_internal(int nsys, const kpp_matrix *A, const double *const *B, double *const *X, int k,
                                  kpp_partition_t P, const kpp_factors_t *F, const kpp_params *p, kpp_report *reps,
                                  cudaStream_t st, bool cd);

// The FP32 memo W_j = G_j^{-1} A_{S_j} for every block (whole blocks; kpp_wmemo.cu).
kpp_status build_w32(const kpp_matrix &A, int s, const float *Ginv32, float *W32, cudaStream_t st);

// The tcgen05 W memo for BF16 storage (kpp_wmemo_tc.cu) in parts, so that the memo of a range of
// blocks can be built as soon as their inverses exist: begin (shape checks, the transposed copy A^T,
// the tensor maps), blocks (W_j for j in [j0, j1); any number of calls, on the stream given), end (reads
// the error word, synchronising that stream, and releases the scratch).  begin returns
// KPP_ERR_UNSUPPORTED for a shape the kernel does not take; after any error the caller builds W32
// with build_w32 instead.
struct WmemoTC {
    void *AT = nullptr, *Gs = nullptr;  // A^T (cols x rows BF16); G^{-1} in three BF16 pieces
    int *d_err = nullptr;
    alignas(64) unsigned char tmG[128] = {}, tmB[128] = {};  // CUtensorMap of the pieces and of A^T
    int64_t rows = 0, cols = 0, ntl = 0;
    int s = 0, mt = 0;
    bool ready = false;
};
kpp_status wmemo_tc_begin(WmemoTC &w, const kpp_matrix &A, int s, cudaStream_t st);
kpp_status wmemo_tc_blocks(WmemoTC &w, const float *Ginv32, float *W32, int64_t j0, int64_t j1, cudaStream_t st);
kpp_status wmemo_tc_end(WmemoTC &w, cudaStream_t st);
// Whether the large-block K++ kernel (kpp_kw.cu) takes this shape.
bool kw_fits(int dtype, int64_t rows, int64_t cols, int s, int k, int sms);

// Number of SMs of the current device (cached).
int sm_count();

// Kernel launches issued by the library (every launch site calls note_launch; kpp_launch_count).
void note_launch();

// Device allocations made by the library (kpp_memory.cu): every device allocation of libkpp goes
// through these, which count the requests (kpp_device_alloc_count).  dev_malloc / dev_free serve
// long-lived buffers from a cache of released ones of the same size (dev_free synchronises the device,
// as cudaFree does); dev_malloc_async serves stream-ordered scratch from the library's pool, released
// with cudaFreeAsync.
cudaError_t dev_malloc(void **p, size_t bytes);
void dev_free(void *p);
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st);
unsigned long long dev_alloc_requests();
// A high-priority non-blocking stream of the current device, lent out until released (nullptr if none
// can be created).  The caller orders it against its own streams with events.
cudaStream_t priority_stream_acquire();
void priority_stream_release(cudaStream_t h);

}  // namespace kpp
