// kpp_server.cu -- continuous-batching serving runtime for K++ / CD++ solves (host C++, native).
//
// Requests (a registered matrix, a host panel of k right-hand sides, solver parameters) arrive at any
// time.  Each is admitted as soon as the device-memory budget allows: its panels, scratch and, on the
// matrix's first use, the memoised block factors (Sec. 4 / Sec. 5.2) must fit under the budget.  The
// factors then stay resident for every later request on that matrix.  Admitted requests run
// concurrently on a pool of worker threads, each with its own CUDA stream, so solves that arrive while
// others are on the GPU overlap on the device; finished requests free their memory and the next waiting
// requests are admitted (FIFO).  Every solve is deterministic, so a request's result does not depend
// on what else is running.  Latency is measured from submission to completion on the host clock.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "kpp_internal.cuh"
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

namespace {

using clk = std::chrono::steady_clock;

struct Matrix {
    kpp_matrix A;           // device, caller-owned
    int32_t s;
    int32_t mode;           // 0 K++, 1 CD++
    double lambda;
    kpp_partition_t P = nullptr;
    kpp_factors_t F = nullptr;
    size_t factor_bytes = 0;
    int users = 0;          // requests in flight on this matrix
    std::mutex mu;          // serialises the first factorisation
};

struct Request {
    int64_t id;
    int32_t mat;
    int32_t k;
    kpp_params p;
    std::vector<double> B;  // rows x k (host copy)
    std::vector<double> X;  // cols x k (result)
    std::vector<kpp_report> reps;
    size_t bytes = 0;       // device bytes charged while admitted
    int grid = 0;           // CTAs of its persistent launch (charged against the SM count)
    clk::time_point t_submit, t_done;
    int32_t state = 0;      // 0 queued, 1 running, 2 done
    kpp_status status = KPP_OK;
};

size_t dsize(int dt) { return dt == KPP_F64 ? 8 : (dt == KPP_F32 ? 4 : 2); }

}  // namespace

struct kpp_server_s {
    size_t budget;
    int workers_n;
    int grid;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::unique_ptr<Matrix>> mats;
    std::map<int64_t, std::shared_ptr<Request>> reqs;
    std::deque<std::shared_ptr<Request>> queue;     // waiting for admission
    std::deque<std::shared_ptr<Request>> ready;     // admitted, waiting for a worker
    size_t used = 0, peak = 0;
    int ctas_used = 0;      // CTAs of the admitted requests' launches (at most the SM count)
    int64_t next_id = 0;
    int64_t n_done = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    int64_t running = 0;  // admitted and not yet finished
    clk::time_point t_first{}, t_last{};
    clk::time_point t_reset{};  // statistics cover requests finished after this point
    bool have_first = false;
    std::vector<double> latencies_ms;
};

namespace {

// Device bytes a request holds while it runs: B, X (FP64), the FP32 copies of the refinement, and the
// solver scratch (momentum, residual copies, partials) -- a conservative per-request estimate.
size_t request_bytes(const Matrix &m, int k) {
    const size_t rows = (size_t)m.A.rows, cols = (size_t)m.A.cols;
    const size_t vec = (rows + cols) * (size_t)k;
    return vec * 8 * 2 + vec * 4 * 6 + (size_t)m.s * 256 * 32 * 8 + (1u << 20);
}

// CTAs for one request's persistent launch: the fewest whose column chunk still fits the dataflow
// (CD++) or small-block (K++) kernel, so that requests stay narrow and many run side by side.  Falls
// back to the SM count (the general kernel then takes any chunk).
int serve_grid(const Matrix &m, int k) {
    const int sms = kpp::sm_count();
    const int KP = k <= 1 ? 1 : (k <= 8 ? 8 : 32);
    const bool f64 = m.A.dtype == KPP_F64;
    const int tas = (int)dsize(m.A.dtype), tcs = f64 ? 8 : 4;
    const int64_t sector = 32 / tas, cols = m.A.cols;
    for (int G = std::max<int64_t>(1, (cols + 255) / 256); G <= sms; ++G) {
        int64_t CW = (cols + G - 1) / G;
        CW = (CW + sector - 1) / sector * sector;
        const int Gu = (int)((cols + CW - 1) / CW);
        if (!kpp::solve2_eligible(m.A, m.s, CW, KP, f64, m.mode == 1, Gu)) continue;
        if (m.mode == 1 && kpp::cd3_smem_bytes(m.s, CW, KP, f64 ? 8 : tas, tcs, f64) > 200 * 1024) continue;
        return Gu;
    }
    return sms;
}

size_t factor_bytes(const Matrix &m) {
    const size_t nb = (size_t)((m.A.rows + m.s - 1) / m.s);
    size_t b = nb * (size_t)m.s * m.s * (8 + 8 + 4);  // L, G^{-1} (FP64 or FP32) and the build's workspace
    if (m.mode == 1 && m.A.dtype == KPP_F64) b += (size_t)m.A.rows * m.A.cols * 8;  // W
    // W32 = G^{-1} A_S in FP32 (CD++ one-column kernel; large-block K++ kernel)
    if (m.A.dtype != KPP_F64 &&
        ((m.mode == 1 && m.A.rows % m.s == 0 && m.s <= 64) ||
         (m.mode == 0 && kpp::kw_fits(m.A.dtype, m.A.rows, m.A.cols, m.s, 1, kpp::sm_count()))))
        b += (size_t)m.A.rows * m.A.cols * 4;
    return b;
}

void run_request(kpp_server_s *sv, const std::shared_ptr<Request> &r) {
    cudaSetDevice(sv->device);
    Matrix &m = *sv->mats[r->mat];
    cudaStream_t st = nullptr;
    kpp_status rc = KPP_OK;
    double *dB = nullptr, *dX = nullptr;
    const size_t rows = (size_t)m.A.rows, cols = (size_t)m.A.cols, k = (size_t)r->k;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = KPP_ERR_CUDA;
    {
        std::lock_guard<std::mutex> g(m.mu);
        if (rc == KPP_OK && !m.F) {
            kpp_status fr = kpp_factor_blocks(&m.A, m.P, m.lambda, m.mode, &m.F, st);
            if (fr != KPP_OK) rc = fr;
        }
    }
    if (rc == KPP_OK && (kpp::dev_malloc_async((void **)&dB, rows * k * 8, st) != cudaSuccess ||
                         kpp::dev_malloc_async((void **)&dX, cols * k * 8, st) != cudaSuccess))
        rc = KPP_ERR_OOM;
    if (rc == KPP_OK) {
        cudaMemcpyAsync(dB, r->B.data(), rows * k * 8, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(dX, 0, cols * k * 8, st);
        kpp_params p = r->p;
        p.lambda = m.lambda;
        if (p.grid == 0) p.grid = r->grid;
        const double *Bp[1] = {dB};
        double *Xp[1] = {dX};
        r->reps.assign(k, kpp_report{});
        // all k columns in one launch (they share the block sequence; each has its own rho and stop test)
        rc = kpp::solve_systems_internal(1, &m.A, Bp, Xp, (int)k, m.P, &m.F, &p, r->reps.data(), st, m.mode == 1);
        r->X.assign(cols * k, 0.0);
        cudaMemcpyAsync(r->X.data(), dX, cols * k * 8, cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess && rc == KPP_OK) rc = KPP_ERR_CUDA;
    }
    if (dB) cudaFreeAsync(dB, st);
    if (dX) cudaFreeAsync(dX, st);
    if (st) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    std::lock_guard<std::mutex> g(sv->mu);
    r->status = rc;
    r->t_done = clk::now();
    r->state = 2;
    sv->used -= r->bytes;
    sv->ctas_used -= r->grid;
    m.users -= 1;
    sv->running -= 1;
    sv->n_done += 1;
    sv->t_last = r->t_done;
    sv->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    sv->cv.notify_all();
}

// Admission (FIFO): move queued requests to `ready` while their memory fits the budget.
void admit_locked(kpp_server_s *sv) {
    while (!sv->queue.empty()) {
        auto r = sv->queue.front();
        Matrix &m = *sv->mats[r->mat];
        size_t need = r->bytes;
        if (!m.F && m.factor_bytes == 0) need += factor_bytes(m);
        // co-residency: the admitted launches together never ask for more CTAs than there are SMs
        if (sv->ctas_used > 0 && sv->ctas_used + r->grid > kpp::sm_count()) return;
        if (sv->used + need > sv->budget) {
            // evict idle factors (least recently registered first) to make room
            for (auto &mp : sv->mats) {
                if (sv->used + need <= sv->budget) break;
                if (mp.get() != &m && mp->F && mp->users == 0) {
                    kpp_factors_destroy(mp->F);
                    mp->F = nullptr;
                    sv->used -= mp->factor_bytes;
                    mp->factor_bytes = 0;
                }
            }
            if (sv->used + need > sv->budget) return;  // wait for running requests to finish
        }
        sv->queue.pop_front();
        if (!m.F && m.factor_bytes == 0) {
            m.factor_bytes = factor_bytes(m);
            sv->used += m.factor_bytes;
        }
        sv->used += r->bytes;
        sv->ctas_used += r->grid;
        sv->peak = std::max(sv->peak, sv->used);
        m.users += 1;
        sv->running += 1;
        r->state = 1;
        sv->ready.push_back(r);
    }
}

void worker_main(kpp_server_s *sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait(lk, [&] {
                admit_locked(sv);
                return sv->stop || !sv->ready.empty();
            });
            if (sv->ready.empty()) {
                if (sv->stop) return;
                continue;
            }
            r = sv->ready.front();
            sv->ready.pop_front();
        }
        run_request(sv, r);
    }
}

}  // namespace

using namespace kpp;

extern "C" {

kpp_status kpp_server_create(size_t hbm_budget_bytes, int32_t max_concurrent, int32_t grid_per_solve,
                             kpp_server_t *out) {
    clear_error();
    if (!out || hbm_budget_bytes == 0 || max_concurrent < 1 || max_concurrent > 64 || grid_per_solve < 0) {
        set_error("kpp_server_create: invalid argument");
        return KPP_ERR_ARG;
    }
    auto *sv = new kpp_server_s;
    sv->budget = hbm_budget_bytes;
    sv->workers_n = max_concurrent;
    sv->grid = grid_per_solve;
    cudaGetDevice(&sv->device);
    for (int i = 0; i < max_concurrent; ++i) sv->workers.emplace_back(worker_main, sv);
    *out = sv;
    return KPP_OK;
}

kpp_status kpp_server_add_matrix(kpp_server_t sv, const kpp_matrix *A, int32_t s, double lambda, int32_t mode,
                                 int32_t *matrix_id) {
    clear_error();
    if (!sv || !A || !A->data || !matrix_id || s < 1 || s > 1024 || (mode != 0 && mode != 1) || !(lambda >= 0) ||
        (mode == 1 && A->rows != A->cols)) {
        set_error("kpp_server_add_matrix: invalid argument");
        return KPP_ERR_ARG;
    }
    auto m = std::make_unique<Matrix>();
    m->A = *A;
    m->s = s;
    m->mode = mode;
    m->lambda = lambda;
    kpp_status rc = kpp_partition(A->rows, s, &m->P);
    if (rc != KPP_OK) return rc;
    std::lock_guard<std::mutex> g(sv->mu);
    *matrix_id = (int32_t)sv->mats.size();
    sv->mats.push_back(std::move(m));
    return KPP_OK;
}

kpp_status kpp_server_submit(kpp_server_t sv, int32_t matrix_id, const double *B_host, int32_t k, const kpp_params *p,
                             int64_t *request_id) {
    clear_error();
    if (!sv || !B_host || !p || !request_id || k < 1 || k > 32) {
        set_error("kpp_server_submit: invalid argument");
        return KPP_ERR_ARG;
    }
    std::lock_guard<std::mutex> g(sv->mu);
    if (matrix_id < 0 || matrix_id >= (int32_t)sv->mats.size()) {
        set_error("kpp_server_submit: unknown matrix %d", matrix_id);
        return KPP_ERR_ARG;
    }
    Matrix &m = *sv->mats[matrix_id];
    auto r = std::make_shared<Request>();
    r->id = sv->next_id++;
    r->mat = matrix_id;
    r->k = k;
    r->p = *p;
    r->B.assign(B_host, B_host + (size_t)m.A.rows * k);
    r->bytes = request_bytes(m, k);
    r->grid = sv->grid > 0 ? sv->grid : serve_grid(m, k);
    r->t_submit = clk::now();
    if (!sv->have_first) {
        sv->t_first = r->t_submit;
        sv->have_first = true;
    }
    if (r->bytes + factor_bytes(m) > sv->budget) {
        r->state = 2;
        r->status = KPP_ERR_BUDGET;
        r->t_done = r->t_submit;
        sv->reqs[r->id] = r;
        *request_id = r->id;
        set_error("request needs %zu bytes, over the budget of %zu", r->bytes + factor_bytes(m), sv->budget);
        return KPP_ERR_BUDGET;
    }
    sv->reqs[r->id] = r;
    sv->queue.push_back(r);
    *request_id = r->id;
    sv->cv.notify_all();
    return KPP_OK;
}

kpp_status kpp_server_poll(kpp_server_t sv, int64_t request_id, double *X_host, kpp_report *reps, int32_t *done) {
    clear_error();
    if (!sv || !done) {
        set_error("kpp_server_poll: invalid argument");
        return KPP_ERR_ARG;
    }
    std::lock_guard<std::mutex> g(sv->mu);
    auto it = sv->reqs.find(request_id);
    if (it == sv->reqs.end()) {
        set_error("kpp_server_poll: unknown request %lld", (long long)request_id);
        return KPP_ERR_ARG;
    }
    auto &r = it->second;
    *done = r->state == 2 ? 1 : 0;
    if (r->state != 2) return KPP_OK;
    if (X_host && !r->X.empty()) memcpy(X_host, r->X.data(), r->X.size() * sizeof(double));
    if (reps && !r->reps.empty()) memcpy(reps, r->reps.data(), r->reps.size() * sizeof(kpp_report));
    return r->status;
}

kpp_status kpp_server_wait_all(kpp_server_t sv, double timeout_s) {
    clear_error();
    if (!sv) return KPP_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    const bool ok = sv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                    [&] { return sv->queue.empty() && sv->ready.empty() && sv->running == 0; });
    if (!ok) {
        set_error("kpp_server_wait_all: requests still running after %.1f s", timeout_s);
        return KPP_ERR_TIMEOUT;
    }
    return KPP_OK;
}

kpp_status kpp_server_stats(kpp_server_t sv, kpp_serving_stats *out) {
    clear_error();
    if (!sv || !out) return KPP_ERR_ARG;
    std::lock_guard<std::mutex> g(sv->mu);
    memset(out, 0, sizeof(*out));
    out->completed = sv->n_done;
    out->peak_bytes = sv->peak;
    out->budget_bytes = sv->budget;
    std::vector<double> l = sv->latencies_ms;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            const double pos = q * (double)(l.size() - 1);
            const size_t i = (size_t)pos;
            const double f = pos - (double)i;
            return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = l.back();
        const double span = std::chrono::duration<double>(sv->t_last - sv->t_first).count();
        out->solves_per_s = span > 0 ? (double)l.size() / span : 0.0;
        out->span_s = span;
    }
    int64_t failed = 0;
    for (auto &kv : sv->reqs)
        if (kv.second->state == 2 && kv.second->status != KPP_OK && kv.second->t_done >= sv->t_reset) ++failed;
    out->failed = failed;
    return KPP_OK;
}

kpp_status kpp_server_reset_stats(kpp_server_t sv) {
    clear_error();
    if (!sv) return KPP_ERR_ARG;
    std::lock_guard<std::mutex> g(sv->mu);
    sv->latencies_ms.clear();
    sv->n_done = 0;
    sv->have_first = false;
    sv->peak = sv->used;
    sv->t_reset = clk::now();
    return KPP_OK;
}

void kpp_server_destroy(kpp_server_t sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    for (auto &t : sv->workers) t.join();
    for (auto &m : sv->mats) {
        if (m->F) kpp_factors_destroy(m->F);
        if (m->P) kpp_partition_destroy(m->P);
    }
    delete sv;
}

}  // extern "C"
