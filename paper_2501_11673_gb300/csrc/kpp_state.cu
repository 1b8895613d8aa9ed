// kpp_state.cu -- checkpoint and resume of a K++ / CD++ solve (kpp_state_*, kpp_solve_resume,
// cdpp_solve_resume).
//
// The iteration's state at step t is more than the iterate x: the momentum m (Eq. 1.4's second
// recurrence), for CD++ the maintained residual R_x = A x - b and R_m = A m (Eq. 5.1's update of
// both), and per right-hand-side column the window sums E0 / E1, the weighted ratio rhat, rho, the
// checkpoint count and the next step index (Eq. 5.2 - 5.3, the checkpoints of Alg. 3 / Alg. 5).  A
// kpp_state_t keeps all of it in device memory between launches of the general persistent kernel,
// which reads and writes m, R_x and R_m in global memory in place; a solve split into several calls
// therefore follows the uninterrupted trajectory bitwise (same grid, same kernel).  save / load move
// the state and x through a flat host buffer, so a solve can stop, be written out, and continue in
// another process.
#include <cmath>
#include <cstring>
#include <vector>

#include "kpp_internal.cuh"
#include "kpp_launch.h"
#include "kpp_runtime.h"
#include "kpp_solve.h"

struct kpp_state_s {
    int64_t rows = 0, cols = 0;
    int k = 1;
    int cd = 0;
    bool fresh = true;       // no step taken yet: the scalars are set from the first call's parameters
    int64_t t = 0;           // host copy of the next step index
    double *m = nullptr;     // cols x k
    double *Rx = nullptr;    // rows x k (CD++)
    double *Rm = nullptr;    // rows x k (CD++)
    kpp::SolveScalars *sc = nullptr;  // k
};

namespace kpp {

static const char STATE_MAGIC[8] = {'K', 'P', 'P', 'S', 'T', 'A', 'T', '1'};

struct StateHeader {
    char magic[8];
    int64_t rows, cols, k, cd, fresh, t;
};

static size_t state_bytes(const kpp_state_s &s) {
    const size_t nv = (size_t)s.cols * s.k, nr = (size_t)s.rows * s.k;
    return sizeof(StateHeader) + (size_t)s.k * sizeof(SolveScalars) + 2 * nv * 8 + (s.cd ? 2 * nr * 8 : 0);
}

static void state_free(kpp_state_s *s) {
    dev_free(s->m);
    dev_free(s->Rx);
    dev_free(s->Rm);
    dev_free(s->sc);
    delete s;
}

static kpp_status solve_resume(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P, kpp_factors_t F,
                               const kpp_params *pp, kpp_state_t S, kpp_report *reps, cudaStream_t st, bool cd) {
    clear_error();
    if (!S || !pp) {
        set_error("resume: null state or parameters");
        return KPP_ERR_ARG;
    }
    const int k = S->k;
    {
        const double *B[1] = {b};
        double *X[1] = {x};
        const kpp_factors_t Fs[1] = {F};
        kpp_status v = validate_systems(1, A, B, X, k, P, Fs, pp, cd);
        if (v != KPP_OK) return v;
    }
    if (A->dtype != KPP_F64) {
        set_error("resume: resumable solves take FP64 storage");
        return KPP_ERR_UNSUPPORTED;
    }
    if (S->rows != A->rows || S->cols != A->cols || S->cd != (cd ? 1 : 0)) {
        set_error("resume: the state was made for another shape or method");
        return KPP_ERR_ARG;
    }
    const kpp_params p = *pp;
    const int s = P->s;
    const double eta = default_eta(p, s, A->rows, A->cols);
    kpp_status rc = KPP_OK;
    std::vector<SolveScalars> sch;
    init_scalars(sch, k, p.rho0);
    if (S->fresh) {
        CUDA_OR(cudaMemcpyAsync(S->sc, sch.data(), (size_t)k * sizeof(SolveScalars), cudaMemcpyHostToDevice, st),
                KPP_ERR_CUDA);
    }
    {
        std::vector<SysInput> in(1);
        in[0] = SysInput{A, b, x, &F->f, p.sys_id, sch.data()};
        in[0].sc_dev = S->sc;
        in[0].m_ext = S->m;
        in[0].Rx_ext = S->Rx;
        in[0].Rm_ext = S->Rm;
        Scratch scr(st);
        PersistentLaunch L;
        // a fresh CD++ state starts from R_x = A x0 - b (computed into the state by the kernel)
        const bool init_residual = cd && S->fresh;
        rc = prepare_persistent(L, in, KPP_F64, cd, k, s, eta, p.tol, p.adaptive_rho, 1, p.max_iters, p.seed,
                                p.grid > 0 ? p.grid : 0, init_residual, 0, /*t0_state=*/true, /*variant=*/1, scr, st);
        if (rc != KPP_OK) return rc;
        S->fresh = false;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        int herr = 0;
        float ms = 0.f;
        CUDA_OR(cudaEventCreate(&e0), KPP_ERR_CUDA);
        CUDA_OR(cudaEventCreate(&e1), KPP_ERR_CUDA);
        rc = enqueue_persistent(L, st, e0, e1);
        if (rc == KPP_OK) {
            if (cudaMemcpyAsync(sch.data(), S->sc, (size_t)k * sizeof(SolveScalars), cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaMemcpyAsync(&herr, L.errs, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                set_error("resume: %s", cudaGetErrorString(cudaGetLastError()));
                rc = KPP_ERR_CUDA;
            }
        }
        if (rc == KPP_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (rc != KPP_OK) return rc;
        S->t = sch[0].t;
        std::vector<double> r2, b2;
        kpp_status r3 = residual_norms(*A, k, b, x, nullptr, r2, &b2, st);
        if (r3 != KPP_OK) return r3;
        kpp_status worst = KPP_OK;
        for (int c = 0; c < k; ++c) {
            const double rel = b2[c] > 0 ? std::sqrt(r2[c] / b2[c]) : std::sqrt(r2[c]);
            kpp_status cs = herr ? (kpp_status)herr : (kpp_status)sch[c].status;
            if (!herr && !std::isfinite(rel)) cs = KPP_ERR_NUMERIC;
            if (worst == KPP_OK) worst = cs;
            if (reps) {
                kpp_report &r = reps[c];
                memset(&r, 0, sizeof(r));
                r.iters = S->t;
                r.rel_res_true = rel;
                r.rel_res_est = sch[c].res_est;
                r.rho_final = sch[c].rho;
                r.status = cs;
                r.bad_block = -1;
                r.device_ms = ms;
                r.kernel_ms = ms;
                r.launches = 1;
            }
        }
        if (worst != KPP_OK) set_error("resume: solve ended with %s", kpp_status_string(worst));
        return worst;
    }
cleanup:
    return rc;
}

}  // namespace kpp

using namespace kpp;

extern "C" {

kpp_status kpp_state_create(int64_t rows, int64_t cols, int32_t k, int32_t cd, kpp_state_t *out) {
    clear_error();
    if (!out || rows < 1 || cols < 1 || k < 1 || k > 32 || (cd && rows != cols)) {
        set_error("kpp_state_create: invalid shape (rows=%lld, cols=%lld, k=%d, cd=%d)", (long long)rows,
                  (long long)cols, k, cd);
        return KPP_ERR_ARG;
    }
    *out = nullptr;
    kpp_state_s *s = new kpp_state_s;
    s->rows = rows;
    s->cols = cols;
    s->k = k;
    s->cd = cd ? 1 : 0;
    const size_t nv = (size_t)cols * k * 8, nr = (size_t)rows * k * 8;
    cudaError_t e = dev_malloc((void **)&s->m, nv);
    if (e == cudaSuccess && cd) e = dev_malloc((void **)&s->Rx, nr);
    if (e == cudaSuccess && cd) e = dev_malloc((void **)&s->Rm, nr);
    if (e == cudaSuccess) e = dev_malloc((void **)&s->sc, (size_t)k * sizeof(SolveScalars));
    if (e == cudaSuccess) e = cudaMemset(s->m, 0, nv);
    if (e == cudaSuccess && cd) e = cudaMemset(s->Rx, 0, nr);
    if (e == cudaSuccess && cd) e = cudaMemset(s->Rm, 0, nr);
    if (e != cudaSuccess) {
        set_error("kpp_state_create: %s", cudaGetErrorString(e));
        state_free(s);
        return e == cudaErrorMemoryAllocation ? KPP_ERR_OOM : KPP_ERR_CUDA;
    }
    *out = s;
    return KPP_OK;
}

void kpp_state_destroy(kpp_state_t st) {
    if (st) state_free(st);
}

int64_t kpp_state_step(kpp_state_t st) { return st ? st->t : -1; }

size_t kpp_state_bytes(kpp_state_t st) { return st ? state_bytes(*st) : 0; }

kpp_status kpp_state_save(kpp_state_t st, const double *x, void *host_buf, size_t bytes, void *stream) {
    clear_error();
    if (!st || !x || !host_buf || bytes < state_bytes(*st)) {
        set_error("kpp_state_save: null argument or buffer smaller than kpp_state_bytes()");
        return KPP_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *p = (unsigned char *)host_buf;
    StateHeader h;
    memcpy(h.magic, STATE_MAGIC, 8);
    h.rows = st->rows;
    h.cols = st->cols;
    h.k = st->k;
    h.cd = st->cd;
    h.fresh = st->fresh ? 1 : 0;
    h.t = st->t;
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const size_t nv = (size_t)st->cols * st->k * 8, nr = (size_t)st->rows * st->k * 8;
    cudaError_t e = cudaMemcpyAsync(p, st->sc, (size_t)st->k * sizeof(SolveScalars), cudaMemcpyDeviceToHost, s);
    p += (size_t)st->k * sizeof(SolveScalars);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, x, nv, cudaMemcpyDeviceToHost, s);
    p += nv;
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, st->m, nv, cudaMemcpyDeviceToHost, s);
    p += nv;
    if (st->cd) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(p, st->Rx, nr, cudaMemcpyDeviceToHost, s);
        p += nr;
        if (e == cudaSuccess) e = cudaMemcpyAsync(p, st->Rm, nr, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("kpp_state_save: %s", cudaGetErrorString(e));
        return KPP_ERR_CUDA;
    }
    return KPP_OK;
}

kpp_status kpp_state_load(kpp_state_t st, double *x, const void *host_buf, size_t bytes, void *stream) {
    clear_error();
    if (!st || !x || !host_buf || bytes < sizeof(StateHeader)) {
        set_error("kpp_state_load: null argument or short buffer");
        return KPP_ERR_ARG;
    }
    StateHeader h;
    memcpy(&h, host_buf, sizeof(h));
    if (memcmp(h.magic, STATE_MAGIC, 8) != 0 || h.rows != st->rows || h.cols != st->cols || h.k != st->k ||
        h.cd != st->cd || bytes < state_bytes(*st) || h.t < 0) {
        set_error("kpp_state_load: not a saved state of this shape (rows, cols, k, method) or a short buffer");
        return KPP_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned char *p = (const unsigned char *)host_buf + sizeof(h);
    const size_t nv = (size_t)st->cols * st->k * 8, nr = (size_t)st->rows * st->k * 8;
    cudaError_t e = cudaMemcpyAsync(st->sc, p, (size_t)st->k * sizeof(SolveScalars), cudaMemcpyHostToDevice, s);
    p += (size_t)st->k * sizeof(SolveScalars);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x, p, nv, cudaMemcpyHostToDevice, s);
    p += nv;
    if (e == cudaSuccess) e = cudaMemcpyAsync(st->m, p, nv, cudaMemcpyHostToDevice, s);
    p += nv;
    if (st->cd) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(st->Rx, p, nr, cudaMemcpyHostToDevice, s);
        p += nr;
        if (e == cudaSuccess) e = cudaMemcpyAsync(st->Rm, p, nr, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("kpp_state_load: %s", cudaGetErrorString(e));
        return KPP_ERR_CUDA;
    }
    st->fresh = h.fresh != 0;
    st->t = h.t;
    return KPP_OK;
}

kpp_status kpp_solve_resume(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P, kpp_factors_t F,
                            const kpp_params *p, kpp_state_t st, kpp_report *rep, void *stream) {
    return solve_resume(A, b, x, P, F, p, st, rep, (cudaStream_t)stream, false);
}

kpp_status cdpp_solve_resume(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P, kpp_factors_t F,
                             const kpp_params *p, kpp_state_t st, kpp_report *rep, void *stream) {
    return solve_resume(A, b, x, P, F, p, st, rep, (cudaStream_t)stream, true);
}

}  // extern "C"
