// kpp_launch.h -- host-side pieces shared by the one-shot entry points (kpp_api.cu) and the
// prepared, graph-capturable plans and the launch autotuner (kpp_plan.cu): handle layouts,
// scratch ownership, and the three stages of a persistent-kernel launch (prepare, enqueue, collect).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/kpp.h"
#include "kpp_runtime.h"
#include "kpp_solve.h"

struct kpp_partition_s {
    int64_t rows;
    int32_t s;
    int64_t nb;
};

struct kpp_factors_s {
    kpp::FactorSet f;
};

namespace kpp {

inline size_t dtype_size(int dt) { return dt == KPP_F64 ? 8 : (dt == KPP_F32 ? 4 : 2); }

inline bool matrix_ok(const kpp_matrix *A) {
    return A && A->data && A->rows > 0 && A->cols > 0 && A->ld >= A->cols &&
           (A->dtype == KPP_F64 || A->dtype == KPP_F32 || A->dtype == KPP_BF16);
}

// Needs `kpp_status rc` and a `cleanup:` label in the calling function.
#define CUDA_OR(call, code)                                                    \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            kpp::set_error("%s: %s", #call, cudaGetErrorString(e_));           \
            rc = (e_ == cudaErrorMemoryAllocation) ? KPP_ERR_OOM : (code);     \
            goto cleanup;                                                      \
        }                                                                      \
    } while (0)

// Device buffers released together: stream-ordered for one-shot calls, plain for plans (which
// outlive the stream they were created on).
struct Scratch {
    cudaStream_t st;
    bool ordered;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t s, bool stream_ordered = true) : st(s), ordered(stream_ordered) {}
    cudaError_t alloc(void **p, size_t bytes) {
        cudaError_t e = ordered ? dev_malloc_async(p, bytes ? bytes : 16, st) : dev_malloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    void release() {
        for (void *p : ptrs) {
            if (ordered) cudaFreeAsync(p, st);
            else cudaFree(p);
        }
        ptrs.clear();
    }
    ~Scratch() { release(); }
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
};

// One system's buffers for a launch of the persistent kernel.
struct SysInput {
    const kpp_matrix *A;
    const void *b;        // TC, rows x k
    void *x;              // TC, cols x k
    const FactorSet *F;
    uint32_t sys_id;
    SolveScalars *sc_host; // k entries, in/out (one-shot launches)
    SolveScalars *sc_dev = nullptr;  // k entries on the device, owned by the caller (plans); no copies
    // Solver state kept by the caller between launches (resumable solves, kpp_state_t): momentum
    // (cols x k) and, for CD++, R_x and R_m (rows x k).  The launch reads and writes them in place and
    // neither zeroes nor re-initialises them; only the general kernel takes them.
    void *m_ext = nullptr, *Rx_ext = nullptr, *Rm_ext = nullptr;
};

// A persistent-kernel launch over nsys systems that share shape, dtype, s and k, prepared once:
// the kernel choice, the chunking, every scratch buffer and the device descriptors.
// enqueue_persistent() then issues only memsets, small kernels and the cooperative launch (no
// allocation, no host synchronisation, no pageable copy), so it can run inside graph capture.
struct PersistentLaunch {
    int kind = 0;  // 1 general, 2 small-block, 3 dataflow CD++, 4 streaming, 6 large-block K++ with W,
                   // 7 single-column dataflow CD++ over a memo
    int dtype = 0, KP = 1, nsys = 0, k = 1;
    bool cd = false, f64 = false, init_residual = true;
    bool keep_state = false;  // the systems' m / R_x / R_m are the caller's state (SysInput::m_ext)
    int64_t t0 = 0;
    Common cm{};
    std::vector<SysArgs> args;
    std::vector<void *> mails;
    size_t mail_bytes = 0, vec_n = 0, vec_r = 0, tcs = 4;
    SysArgs *d_args = nullptr;
    void *d_sys2 = nullptr;
    unsigned *bars = nullptr;
    int *errs = nullptr;
};

extern int g_variant;  // kernel generation limit (kpp_set_kernel_variant)

int auto_grid(int64_t cols, int nsys);
void init_scalars(std::vector<SolveScalars> &sc, int k, double rho0);
double default_eta(const kpp_params &p, int s, int64_t rows, int64_t cols);

// Argument checks shared by every solve entry point (sets the error message).
kpp_status validate_systems(int nsys, const kpp_matrix *A, const double *const *B, double *const *X, int k,
                            kpp_partition_t P, const kpp_factors_t *F, const kpp_params *p, bool cd);

// |A x - b|^2 (and |b|^2) per column, summed on the host in a fixed order; synchronises.
kpp_status residual_norms(const kpp_matrix &A, int k, const double *b, const double *x, float *r32,
                          std::vector<double> &res2, std::vector<double> *bn2, cudaStream_t st);

kpp_status prepare_persistent(PersistentLaunch &L, std::vector<SysInput> &sys, int dtype, bool cd, int k, int s,
                              double eta, double tol, int adaptive, int confirm, int64_t max_iters, uint64_t seed,
                              int grid, bool init_residual, int64_t t0, bool t0_state, int variant, Scratch &scr,
                              cudaStream_t st);
// ev0 / ev1 (optional): recorded on `st` right before and after the kernel launch.
kpp_status enqueue_persistent(const PersistentLaunch &L, cudaStream_t st, cudaEvent_t ev0 = nullptr,
                              cudaEvent_t ev1 = nullptr);

// prepare + enqueue + copy the scalars back (synchronises).  variant < 0: the global limit.
kpp_status run_persistent(std::vector<SysInput> &sys, int dtype, bool cd, int k, int s, double eta, double tol,
                          int adaptive, int confirm, int64_t max_iters, uint64_t seed, int grid, bool init_residual,
                          int64_t t0, cudaStream_t st, float *ms_out, int *err_out, int variant = -1,
                          int *kind_out = nullptr, int *G_out = nullptr);

// Launch autotuner (kpp_plan.cu): the (kernel generation, CTAs per system) pair with the lowest
// measured time per step for this shape, from the process-wide cache or by timing short runs.
struct TuneChoice {
    int variant = -1, grid = 0;
};
kpp_status tune_launch(int nsys, const kpp_matrix *A, const double *const *B, int k, kpp_partition_t P,
                       const kpp_factors_t *F, const kpp_params &p, bool cd, cudaStream_t st, TuneChoice &out);

}  // namespace kpp
