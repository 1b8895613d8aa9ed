// kpp_noalloc.cu -- cdpp_solve_noalloc: the CD++ FP64 solve without any device allocation.
//
// Some callers cannot call cudaMalloc: a process whose device memory is owned by another allocator
// (a serving runtime or framework pool that has already reserved the GPU and forbids allocations
// behind its back), or a request path that must never block on the allocator or fail half way with
// an out-of-memory error.  For them this entry point runs the general persistent CD++ kernel
// (kpp_solve.cu's solve_kernel: what cdpp_solve runs after kpp_set_kernel_variant(1); the default
// variant picks the dataflow kernels instead, which reach the same iterates in another summation
// order), with the same launch shape and all of its scratch (momentum, maintained residuals, projection buffer, per-solve
// scalars, barrier words, launch descriptor and residual partial sums) carved out of one file-scope
// device array of fixed size.  The caller still passes the matrix, right-hand side, iterate and the
// memoised factors.
#include <atomic>
#include <cmath>
#include <cstring>

#include "kpp_internal.cuh"
#include "kpp_launch.h"
#include "kpp_runtime.h"
#include "kpp_solve.h"

namespace kpp {

// Limits of the allocation-free path (also stated in include/kpp.h).
constexpr int64_t NOALLOC_MAX_N = 16384;
constexpr int NOALLOC_MAX_S = 256;
constexpr int NOALLOC_MAX_G = 160;
constexpr int NOALLOC_RES_GRID = 256;

// Bytes of each region (multiples of 256).
constexpr size_t rup(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t OFF_M = 0;
constexpr size_t OFF_RX = OFF_M + rup(NOALLOC_MAX_N * 8);
constexpr size_t OFF_RM = OFF_RX + rup(NOALLOC_MAX_N * 8);
constexpr size_t OFF_YBUF = OFF_RM + rup(NOALLOC_MAX_N * 8);
constexpr size_t OFF_RBUF = OFF_YBUF + rup(NOALLOC_MAX_S * 8);
constexpr size_t OFF_RPART = OFF_RBUF + rup(NOALLOC_MAX_S * 8);
constexpr size_t OFF_RESPART = OFF_RPART + rup(NOALLOC_MAX_G * 8);
constexpr size_t OFF_SC = OFF_RESPART + rup(NOALLOC_RES_GRID * 8);
constexpr size_t OFF_WORDS = OFF_SC + rup(sizeof(SolveScalars));
constexpr size_t OFF_ARGS = OFF_WORDS + 256;
constexpr size_t NOALLOC_BYTES = OFF_ARGS + rup(sizeof(SysArgs));

// The scratch of every call on this device (each GPU that loads the library holds its own copy
// until the process exits).  Host code must not use this name as an address: it is a host-side
// stand-in.  The device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of the scratch, looked up once per device with that device current.  The cache is
// atomic so that first calls from several host threads do not race on it (they store the same value).
static unsigned char *scratch_ptr(kpp_status *rc) {
    static std::atomic<unsigned char *> cached[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        set_error("cdpp_solve_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
        *rc = KPP_ERR_CUDA;
        return nullptr;
    }
    unsigned char *ptr = cached[dev].load(std::memory_order_acquire);
    if (!ptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cdpp_solve_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            *rc = KPP_ERR_CUDA;
            return nullptr;
        }
        ptr = (unsigned char *)p;
        cached[dev].store(ptr, std::memory_order_release);
    }
    return ptr;
}

}  // namespace kpp

using namespace kpp;

extern "C" kpp_status cdpp_solve_noalloc(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P,
                                         kpp_factors_t F, const kpp_params *pp, kpp_report *rep, void *stream) {
    clear_error();
    if (!A || !A->data || !b || !x || !P || !F || !pp || A->dtype != KPP_F64 || A->rows != A->cols ||
        A->rows != P->rows || A->ld < A->cols) {
        set_error("cdpp_solve_noalloc: needs an FP64 square matrix matching the partition, and non-null b, x, F");
        return KPP_ERR_ARG;
    }
    const int64_t n = A->rows;
    const int s = P->s;
    if (n > NOALLOC_MAX_N || s > NOALLOC_MAX_S) {
        set_error("cdpp_solve_noalloc: n=%lld s=%d exceed the fixed scratch (n <= %lld, s <= %d)", (long long)n, s,
                  (long long)NOALLOC_MAX_N, NOALLOC_MAX_S);
        return KPP_ERR_ARG;
    }
    const FactorSet &f = F->f;
    if (f.mode != 1 || f.s != s || f.rows != n || f.dtype != KPP_F64 || f.bad_block >= 0 ||
        std::fabs(f.lambda - pp->lambda) > 1e-15 * std::max(1.0, std::fabs(pp->lambda))) {
        set_error("cdpp_solve_noalloc: factors do not match (CD++ mode, s, FP64, lambda)");
        return KPP_ERR_ARG;
    }
    kpp_status rc = KPP_OK;
    unsigned char *base = scratch_ptr(&rc);
    if (!base) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const kpp_params p = *pp;

    // grid and column chunk exactly as cdpp_solve picks them for one system (auto_grid, the chunk
    // rounded to a 32-byte sector, then no CTA without columns)
    int G = p.grid > 0 ? p.grid : auto_grid(n, 1);
    if (G > NOALLOC_MAX_G) G = NOALLOC_MAX_G;
    int64_t CW = (n + G - 1) / G;
    CW = (CW + 3) / 4 * 4;
    G = (int)((n + CW - 1) / CW);
    Common cm{};
    cm.rows = n;
    cm.cols = n;
    cm.s = s;
    cm.nb = (int)((n + s - 1) / s);
    cm.k = 1;
    cm.CW = CW;
    cm.G = G;
    cm.eta = std::isnan(p.eta) ? (double)s / (2.0 * (double)n) : p.eta;
    cm.tol = p.tol;
    cm.adaptive = p.adaptive_rho;
    cm.confirm = 1;
    cm.reduce_redundant = 1;
    cm.init_residual = 1;
    cm.max_iters = p.max_iters;
    cm.seed = p.seed;
    cm.timeout_ns = 2000000000ull;
    cm.test_hold_cta = -1;
    if (solve_smem_bytes(s, 1, CW, 8) > 220 * 1024) {
        set_error("cdpp_solve_noalloc: shared memory limit exceeded");
        return KPP_ERR_UNSUPPORTED;
    }

    SysArgs a;
    memset(&a, 0, sizeof(a));
    a.A = A->data;
    a.lda = A->ld;
    a.b = b;
    a.x = x;
    a.m = base + OFF_M;
    a.Rx = base + OFF_RX;
    a.Rm = base + OFF_RM;
    a.Ginv = f.Ginv;
    a.part = nullptr;  // CD++ gathers r from R_x: no partial residuals
    a.rbuf = base + OFF_RBUF;
    a.ybuf = base + OFF_YBUF;
    a.rpart = (double *)(base + OFF_RPART);
    a.sc = (SolveScalars *)(base + OFF_SC);
    a.bar = (unsigned *)(base + OFF_WORDS);
    a.err = (int *)(base + OFF_WORDS + 64);
    a.sys_id = p.sys_id;
    a.t0 = 0;
    SolveScalars sc0;
    memset(&sc0, 0, sizeof(sc0));
    sc0.rho = p.rho0;
    sc0.active = 1;
    sc0.status = KPP_ERR_NO_CONVERGENCE;
    sc0.res_est = NAN;

    SolveScalars sc_out;
    int herr = 0;
    double hpart[NOALLOC_RES_GRID];
    double res2 = 0.0, bn2 = 0.0;
    SysArgs *d_args = (SysArgs *)(base + OFF_ARGS);
    double *respart = (double *)(base + OFF_RESPART);
    // everything that must start at zero: momentum, R_m, the barrier and error words
    cudaError_t e = cudaMemsetAsync(base + OFF_M, 0, (size_t)n * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + OFF_RM, 0, (size_t)n * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + OFF_WORDS, 0, 256, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.sc, &sc0, sizeof(sc0), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_args, &a, sizeof(a), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_solve(KPP_F64, true, true, d_args, 1, cm, 1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sc_out, a.sc, sizeof(sc_out), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    // final |Ax - b| / |b| from fixed-grid partial sums kept in the same scratch
    if (e == cudaSuccess) e = launch_residual_grid(*A, 1, b, x, nullptr, respart, NOALLOC_RES_GRID, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hpart, respart, sizeof(hpart), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        for (int i = 0; i < NOALLOC_RES_GRID; ++i) res2 += hpart[i];
        e = launch_residual_grid(*A, 1, b, nullptr, nullptr, respart, NOALLOC_RES_GRID, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hpart, respart, sizeof(hpart), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("cdpp_solve_noalloc: %s", cudaGetErrorString(e));
        return KPP_ERR_CUDA;
    }
    for (int i = 0; i < NOALLOC_RES_GRID; ++i) bn2 += hpart[i];
    const double relres = bn2 > 0 ? std::sqrt(res2 / bn2) : std::sqrt(res2);
    kpp_status status = herr ? (kpp_status)herr : (kpp_status)sc_out.status;
    if (status == KPP_OK && !std::isfinite(relres)) status = KPP_ERR_NUMERIC;
    if (rep) {
        memset(rep, 0, sizeof(*rep));
        rep->iters = sc_out.t;
        rep->rel_res_true = relres;
        rep->rel_res_est = sc_out.res_est;
        rep->rho_final = sc_out.rho;
        rep->status = status;
        rep->bad_block = -1;
        rep->device_ms = NAN;
    }
    if (status != KPP_OK) set_error("cdpp_solve_noalloc: %s", kpp_status_string(status));
    return status;
}
