// kpp_server.cu -- continuous-batching serving runtime for K++ / CD++ solves (host C++, native), around
// the device-resident request loop of kpp_serve.cu.
//
// Requests (a registered matrix, a host panel of k right-hand sides, solver parameters) arrive at any
// time.  A request is admitted as soon as the device-memory budget allows: its panels and solve scratch
// must fit, next to the memoised block factors (Sec. 4 / Sec. 5.2) of the matrices in use, which stay
// resident for every later request on the same matrix.  An admitted request becomes jobs of at most
// SERVE_KP columns; jobs are published into a ring in mapped host memory, shortest expected work first
// (iterations seen on the matrix so far x n x columns), while at most two jobs per slot wait unclaimed.
// One persistent kernel of slots claims and runs them on the device, each job on one slot's CTAs, so
// jobs that arrive while others run are taken up as slots free up and overlap with them; completion
// records come back through mapped memory.  One dispatcher thread does all of this: admission, copies,
// publication, (re)launches of the loop, completions.  The host never launches a kernel per request.
// Factor phases need the GPU to themselves: the dispatcher drains the loop (slots leave once nothing is
// published for them), factors every matrix that the admitted requests need (and every other registered
// matrix that fits the budget), and relaunches.  A job's result depends on the job alone, so a request
// gives the same bits alone and in any mix.  Latency runs from submission to completion (host clock).
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
#include "kpp_launch.h"
#include "kpp_runtime.h"
#include "kpp_serve.h"
#include "kpp_solve.h"

namespace {

using clk = std::chrono::steady_clock;
using kpp::SERVE_KP;
using kpp::ServeCtl;
using kpp::ServeDone;
using kpp::ServeJob;
using kpp::ServeSlot;

struct Matrix {
    kpp_matrix A;           // device, caller-owned
    int32_t s;
    int32_t mode;           // 0 K++, 1 CD++
    double lambda;
    kpp_partition_t P = nullptr;
    kpp_factors_t F = nullptr;
    size_t factor_bytes = 0;
    int users = 0;          // admitted requests on this matrix
    double iters_sum = 0.0; // block iterations of its completed requests (expected work)
    int64_t iters_n = 0;
};

struct Chunk {
    int c0 = 0, kc = 0;
    void *mem = nullptr;    // device block holding the chunk's buffers
    double *B = nullptr, *X = nullptr;
    int64_t jid = -1;       // job number once published
    bool done = false;
    ServeDone rec{};
    ServeJob job{};
};

struct Request {
    int64_t id;
    int32_t mat;
    int32_t k;
    kpp_params p;
    std::vector<double> B;  // rows x k (host copy)
    std::vector<double> X;  // cols x k (result)
    std::vector<kpp_report> reps;
    std::vector<Chunk> chunks;
    size_t bytes = 0;       // device bytes charged while admitted
    double work = 0.0;      // expected work (ordering of publication)
    clk::time_point t_submit, t_done;
    int32_t state = 0;      // 0 queued, 1 admitted, 2 done
    int32_t published = 0;  // chunks published
    int32_t pending = 0;    // chunks not yet complete
    kpp_status status = KPP_OK;
};

constexpr size_t kMaxMatrices = 4096;  // registered matrices per server

size_t dsize(int dt) { return kpp::dtype_size(dt); }
size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Column chunk of a slot's CTAs for a matrix: 32-byte sectors of A per CTA.
int64_t serve_cw(const kpp_matrix &A, int G) {
    const int64_t sector = 32 / (int64_t)dsize(A.dtype);
    int64_t CW = (A.cols + G - 1) / G;
    return (CW + sector - 1) / sector * sector;
}

// Device bytes of one job of kc columns (one allocation, carved in 256-byte pieces).
size_t chunk_bytes(const Matrix &m, int kc, int G) {
    const size_t rows = (size_t)m.A.rows, cols = (size_t)m.A.cols, KP = SERVE_KP, s = (size_t)m.s;
    const size_t tcs = m.A.dtype == KPP_F64 ? 8 : 4;
    size_t b = up256(rows * kc * 8) + up256(cols * kc * 8);                 // B, X (FP64)
    if (m.A.dtype != KPP_F64) b += up256(rows * kc * tcs) + up256(cols * kc * tcs);  // inner b = r, x = d
    b += up256(cols * kc * tcs);                                            // m
    if (m.mode == 1) b += 2 * up256(rows * kc * tcs);                       // R_x, R_m
    b += up256((size_t)G * s * KP * tcs) + 2 * up256(s * KP * tcs);        // part, rbuf, ybuf
    b += up256((size_t)G * 2 * KP * 8) + up256((size_t)kc * sizeof(kpp::SolveScalars));
    return b;
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

}  // namespace

struct kpp_server_s {
    size_t budget = 0;
    int slots_max = 1;
    int G = 8;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::unique_ptr<Matrix>> mats;
    std::map<int64_t, std::shared_ptr<Request>> reqs;
    std::deque<std::shared_ptr<Request>> queue;   // waiting for admission (FIFO)
    std::vector<std::shared_ptr<Request>> active;  // admitted, not done
    size_t used = 0, peak = 0;
    int64_t next_id = 0, n_done = 0;
    bool stop = false;
    clk::time_point t_first{}, t_last{}, t_reset{};
    bool have_first = false;
    std::vector<double> latencies_ms;
    // the device-resident loop (owned by the dispatcher thread)
    std::thread disp;
    cudaStream_t st_k = nullptr, st_io = nullptr;
    cudaEvent_t ev_k = nullptr;
    bool k_live = false;
    size_t k_smem = 0;
    int k_slots = 0;
    int64_t k_launches = 0;
    int R = 8192;
    ServeJob *jobs_h = nullptr, *jobs_d = nullptr;
    ServeDone *done_h = nullptr, *done_d = nullptr;
    ServeCtl *ctl_h = nullptr, *ctl_d = nullptr;
    ServeSlot *slots_d = nullptr;
    unsigned long long *claimed_d = nullptr;
    int64_t published = 0;     // jobs published so far
    std::vector<std::pair<std::shared_ptr<Request>, int>> ring;  // job % R -> (request, chunk)
};

namespace {

void publish_count(kpp_server_s *sv) {
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *(volatile int64_t *)&sv->ctl_h->published = sv->published;
    std::atomic_thread_fence(std::memory_order_seq_cst);
}
void set_drain(kpp_server_s *sv, int v) {
    *(volatile int32_t *)&sv->ctl_h->drain = v;
    std::atomic_thread_fence(std::memory_order_seq_cst);
}

// Is the loop still running?  (When it has ended, jobs it claimed but never finished are failed.)
bool loop_live(kpp_server_s *sv) {
    if (!sv->k_live) return false;
    if (cudaEventQuery(sv->ev_k) == cudaErrorNotReady) return true;
    sv->k_live = false;
    return false;
}

size_t smem_need(kpp_server_s *sv, const Matrix &m) {
    return kpp::serve_smem_bytes(m.s, serve_cw(m.A, sv->G));
}

// Fill chunk i's job descriptor and buffers (device memory on st_io); false on allocation failure.
bool prepare_chunk(kpp_server_s *sv, Request &r, Matrix &m, Chunk &ch) {
    using namespace kpp;
    const int G = sv->G, KP = SERVE_KP, kc = ch.kc;
    const size_t rows = (size_t)m.A.rows, cols = (size_t)m.A.cols, s = (size_t)m.s;
    const bool f64 = m.A.dtype == KPP_F64;
    const size_t tcs = f64 ? 8 : 4;
    const size_t total = chunk_bytes(m, kc, G);
    if (dev_malloc_async(&ch.mem, total, sv->st_io) != cudaSuccess) {
        ch.mem = nullptr;
        return false;
    }
    char *p = (char *)ch.mem;
    auto take = [&](size_t b) {
        void *q = p;
        p += up256(b);
        return q;
    };
    ch.B = (double *)take(rows * kc * 8);
    ch.X = (double *)take(cols * kc * 8);
    void *rb = f64 ? (void *)ch.B : take(rows * kc * tcs);
    void *d = f64 ? (void *)ch.X : take(cols * kc * tcs);
    void *mm = take(cols * kc * tcs);
    void *Rx = m.mode == 1 ? take(rows * kc * tcs) : nullptr;
    void *Rm = m.mode == 1 ? take(rows * kc * tcs) : nullptr;
    void *part = take((size_t)G * s * KP * tcs);
    void *rbuf = take(s * KP * tcs);
    void *ybuf = take(s * KP * tcs);
    double *rpart = (double *)take((size_t)G * 2 * KP * 8);
    SolveScalars *sc = (SolveScalars *)take((size_t)kc * sizeof(SolveScalars));
    // the chunk's columns of B, contiguous (rows x kc)
    std::vector<double> Bc(rows * kc);
    for (size_t i = 0; i < rows; ++i)
        for (int c = 0; c < kc; ++c) Bc[i * kc + c] = r.B[i * r.k + ch.c0 + c];
    std::vector<SolveScalars> sch(kc);
    for (auto &x : sch) {
        memset(&x, 0, sizeof(x));
        x.rho = r.p.rho0;
        x.active = 1;
    }
    // zeros by copy, not memset: a memset may run as a kernel, which would wait for the loop to end
    std::vector<double> zeros((cols * kc * 8 + 7) / 8, 0.0);
    if (cudaMemcpyAsync(ch.B, Bc.data(), rows * kc * 8, cudaMemcpyHostToDevice, sv->st_io) != cudaSuccess ||
        cudaMemcpyAsync(ch.X, zeros.data(), cols * kc * 8, cudaMemcpyHostToDevice, sv->st_io) != cudaSuccess ||
        cudaMemcpyAsync(sc, sch.data(), kc * sizeof(SolveScalars), cudaMemcpyHostToDevice, sv->st_io) != cudaSuccess ||
        cudaMemcpyAsync(mm, zeros.data(), cols * kc * tcs, cudaMemcpyHostToDevice, sv->st_io) != cudaSuccess ||
        (Rm && cudaMemcpyAsync(Rm, zeros.data(), rows * kc * tcs, cudaMemcpyHostToDevice, sv->st_io) != cudaSuccess))
        return false;
    // the copies must land before the job is published (pageable B: the copy is staged by then anyway)
    if (cudaStreamSynchronize(sv->st_io) != cudaSuccess) return false;
    ServeJob &J = ch.job;
    memset(&J, 0, sizeof(J));
    SysArgs &a = J.sa;
    a.A = m.A.data;
    a.lda = m.A.ld;
    a.b = rb;
    a.x = d;
    a.m = mm;
    a.Rx = Rx;
    a.Rm = Rm;
    a.Ginv = f64 ? (const void *)m.F->f.Ginv : (const void *)m.F->f.Ginv32;
    a.part = part;
    a.rbuf = rbuf;
    a.ybuf = ybuf;
    a.rpart = rpart;
    a.sc = sc;
    a.sys_id = r.p.sys_id;
    a.t0 = 0;
    Common &cm = J.cm;
    cm.rows = m.A.rows;
    cm.cols = m.A.cols;
    cm.s = m.s;
    cm.nb = (int)((m.A.rows + m.s - 1) / m.s);
    cm.k = kc;
    cm.CW = serve_cw(m.A, G);
    cm.G = G;
    cm.eta = std::isnan(r.p.eta) ? (double)m.s / (2.0 * (double)std::min(m.A.rows, m.A.cols)) : r.p.eta;
    const bool refine = !f64 && r.p.refine;
    cm.tol = f64 ? r.p.tol : (refine ? r.p.inner_tol : r.p.tol);
    cm.adaptive = r.p.adaptive_rho;
    cm.confirm = f64 ? 1 : 0;  // inner solves stop on the window estimate; the FP64 outer residual decides
    cm.reduce_redundant = ((int64_t)G * m.s * KP <= 8192) ? 1 : 0;
    cm.init_residual = (f64 && m.mode == 1) ? 1 : 0;
    cm.max_iters = r.p.max_iters;
    cm.seed = r.p.seed;
    cm.timeout_ns = 2000000000ull;
    cm.t0_state = f64 ? 0 : 1;
    cm.test_hold_cta = -1;
    J.B = ch.B;
    J.X = ch.X;
    J.tol = r.p.tol;
    J.max_outer = refine ? std::max(1, r.p.max_outer) : 1;
    J.dtype = m.A.dtype;
    J.mode = m.mode;
    return true;
}

void release_chunks(kpp_server_s *sv, Request &r) {
    for (auto &ch : r.chunks)
        if (ch.mem) {
            cudaFreeAsync(ch.mem, sv->st_io);
            ch.mem = nullptr;
        }
}

// Called with sv->mu held: the request is complete.
void finish_locked(kpp_server_s *sv, const std::shared_ptr<Request> &r, kpp_status rc) {
    Matrix &m = *sv->mats[r->mat];
    r->status = rc;
    r->t_done = clk::now();
    r->state = 2;
    sv->used -= r->bytes;
    m.users -= 1;
    sv->n_done += 1;
    sv->t_last = r->t_done;
    sv->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    sv->active.erase(std::remove(sv->active.begin(), sv->active.end(), r), sv->active.end());
    sv->cv.notify_all();
}

// Collect a finished request: X back to the host, reports, memory released.
void complete_request(kpp_server_s *sv, const std::shared_ptr<Request> &r) {
    Matrix &m = *sv->mats[r->mat];
    const size_t cols = (size_t)m.A.cols;
    kpp_status rc = KPP_OK;
    r->X.assign(cols * r->k, 0.0);
    r->reps.assign(r->k, kpp_report{});
    std::vector<double> Xc;
    int64_t iters_max = 0;
    for (auto &ch : r->chunks) {
        Xc.resize(cols * ch.kc);
        if (cudaMemcpyAsync(Xc.data(), ch.X, cols * ch.kc * 8, cudaMemcpyDeviceToHost, sv->st_io) != cudaSuccess ||
            cudaStreamSynchronize(sv->st_io) != cudaSuccess) {
            rc = KPP_ERR_CUDA;
            break;
        }
        for (size_t i = 0; i < cols; ++i)
            for (int c = 0; c < ch.kc; ++c) r->X[i * r->k + ch.c0 + c] = Xc[i * ch.kc + c];
        for (int c = 0; c < ch.kc; ++c) {
            kpp_report &rep = r->reps[ch.c0 + c];
            rep.iters = ch.rec.iters;
            rep.outer = ch.rec.outer;
            rep.rel_res_true = ch.rec.rel_res[c];
            rep.rel_res_est = NAN;
            rep.rho_final = ch.rec.rho[c];
            rep.status = ch.rec.col_status[c];
            rep.bad_block = -1;
            rep.device_ms = NAN;
            rep.kernel_ms = NAN;
            rep.launches = 0;
        }
        if (ch.rec.status != KPP_OK && rc == KPP_OK) rc = (kpp_status)ch.rec.status;
        iters_max = std::max<int64_t>(iters_max, ch.rec.iters);
    }
    release_chunks(sv, *r);
    cudaStreamSynchronize(sv->st_io);
    std::lock_guard<std::mutex> g(sv->mu);
    m.iters_sum += (double)iters_max;
    m.iters_n += 1;
    finish_locked(sv, r, rc);
}

// Admission under the budget, FIFO; with sv->mu held.  Returns the requests admitted now.
void admit_locked(kpp_server_s *sv, std::vector<std::shared_ptr<Request>> &out) {
    while (!sv->queue.empty()) {
        auto r = sv->queue.front();
        Matrix &m = *sv->mats[r->mat];
        size_t need = r->bytes + (m.F ? 0 : factor_bytes(m));
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
        sv->peak = std::max(sv->peak, sv->used);
        m.users += 1;
        r->state = 1;
        const double it = m.iters_n ? m.iters_sum / (double)m.iters_n : 64.0 * (double)m.A.rows / m.s;
        r->work = it * (double)m.A.rows * (double)m.A.cols * (double)r->k;
        sv->active.push_back(r);
        out.push_back(r);
    }
}

// Factor phases: the loop must be drained first (it holds the SMs).  Returns false if the loop is
// still running (call again).
bool factor_pending(kpp_server_s *sv, std::vector<std::shared_ptr<Request>> &need) {
    if (need.empty()) return true;
    if (loop_live(sv)) {
        set_drain(sv, 1);
        return false;
    }
    for (auto &r : need) {
        Matrix &m = *sv->mats[r->mat];
        if (m.F) continue;
        kpp_status fr = kpp_factor_blocks(&m.A, m.P, m.lambda, m.mode, &m.F, sv->st_io);
        if (fr != KPP_OK) {
            if (m.F) {
                kpp_factors_destroy(m.F);
                m.F = nullptr;
            }
            std::lock_guard<std::mutex> g(sv->mu);
            sv->used -= m.factor_bytes;
            m.factor_bytes = 0;
            r->chunks.clear();
            finish_locked(sv, r, fr);
        }
    }
    // while the loop is down: every other registered matrix whose factors fit the budget too, so that
    // later requests on them do not drain the loop again
    {
        std::lock_guard<std::mutex> g(sv->mu);
        for (auto &mp : sv->mats) {
            if (mp->F || mp->factor_bytes) continue;
            const size_t fb = factor_bytes(*mp);
            if (sv->used + fb > sv->budget / 2) continue;
            if (kpp_factor_blocks(&mp->A, mp->P, mp->lambda, mp->mode, &mp->F, sv->st_io) == KPP_OK) {
                mp->factor_bytes = fb;
                sv->used += fb;
                sv->peak = std::max(sv->peak, sv->used);
            } else if (mp->F) {
                kpp_factors_destroy(mp->F);
                mp->F = nullptr;
            }
        }
    }
    need.erase(std::remove_if(need.begin(), need.end(), [](const std::shared_ptr<Request> &r) { return r->state == 2; }),
               need.end());
    set_drain(sv, 0);
    return true;
}

bool launch_loop(kpp_server_s *sv, size_t smem) {
    using namespace kpp;
    const int cap = serve_max_ctas(smem) / sv->G;
    const int nslots = std::min(sv->slots_max, cap);
    if (nslots < 1) return false;
    if (cudaMemsetAsync(sv->slots_d, 0, sizeof(ServeSlot) * 256, sv->st_k) != cudaSuccess) return false;
    set_drain(sv, 0);
    ServeArgs a{};
    a.jobs = sv->jobs_d;
    a.done = sv->done_d;
    a.ctl = sv->ctl_d;
    a.slots = sv->slots_d;
    a.claimed = sv->claimed_d;
    a.R = sv->R;
    a.G = sv->G;
    a.idle_ns = 50000000ull;      // 50 ms without a job: the slot leaves
    a.timeout_ns = 2000000000ull; // group barriers
    if (launch_serve(a, nslots, smem, sv->st_k) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaEventRecord(sv->ev_k, sv->st_k);
    sv->k_live = true;
    sv->k_smem = smem;
    sv->k_slots = nslots;
    sv->k_launches += 1;
    return true;
}

void dispatcher_main(kpp_server_s *sv) {
    cudaSetDevice(sv->device);
    std::vector<std::shared_ptr<Request>> fresh;   // admitted, buffers not prepared
    std::vector<std::shared_ptr<Request>> ready;   // prepared, chunks to publish
    int64_t lo = 0;                                // oldest job without a completion seen
    int64_t outstanding = 0;                       // published jobs without a completion seen
    for (;;) {
        bool progress = false;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (sv->stop && sv->queue.empty() && sv->active.empty()) break;
            if (fresh.empty() && ready.empty() && lo == sv->published && sv->queue.empty())
                sv->cv.wait_for(lk, std::chrono::milliseconds(20));
            admit_locked(sv, fresh);
        }
        // factors for the admitted requests (drains the loop when needed)
        std::vector<std::shared_ptr<Request>> need;
        for (auto &r : fresh)
            if (!sv->mats[r->mat]->F) need.push_back(r);
        bool factors_ok = factor_pending(sv, need);
        if (factors_ok) {
            for (auto &r : fresh) {
                if (r->state == 2) continue;
                Matrix &m = *sv->mats[r->mat];
                bool ok = m.F != nullptr;
                for (int c0 = 0; ok && c0 < r->k; c0 += SERVE_KP) {
                    Chunk ch;
                    ch.c0 = c0;
                    ch.kc = std::min(SERVE_KP, r->k - c0);
                    r->chunks.push_back(ch);
                }
                for (auto &ch : r->chunks)
                    if (ok) ok = prepare_chunk(sv, *r, m, ch);
                r->pending = (int)r->chunks.size();
                if (!ok) {
                    release_chunks(sv, *r);
                    cudaStreamSynchronize(sv->st_io);
                    std::lock_guard<std::mutex> g(sv->mu);
                    finish_locked(sv, r, m.F ? KPP_ERR_OOM : KPP_ERR_NOT_SPD);
                    continue;
                }
                ready.push_back(r);
                progress = true;
            }
            fresh.clear();
        }
        // publish, shortest expected work first, while at most two jobs per slot wait beside the running ones
        if (!ready.empty()) {
            std::stable_sort(ready.begin(), ready.end(),
                             [](const std::shared_ptr<Request> &a, const std::shared_ptr<Request> &b) { return a->work < b->work; });
            const int64_t window = 3 * (int64_t)std::max(1, sv->k_live ? sv->k_slots : sv->slots_max);
            size_t i = 0;
            bool full = false;
            while (i < ready.size() && !full) {
                auto &r = ready[i];
                Matrix &m = *sv->mats[r->mat];
                if (sv->k_live && smem_need(sv, m) > sv->k_smem) {
                    // the running loop cannot take it: let it drain; the relaunch sizes for it
                    set_drain(sv, 1);
                    ++i;
                    continue;
                }
                while (r->published < (int)r->chunks.size()) {
                    if (outstanding >= window || sv->published - lo >= sv->R) {
                        full = true;
                        break;
                    }
                    Chunk &ch = r->chunks[r->published];
                    ch.jid = sv->published;
                    ch.job.id = ch.jid;
                    const int e = (int)(ch.jid % sv->R);
                    memcpy(&sv->jobs_h[e], &ch.job, sizeof(ServeJob));
                    memset(&sv->done_h[e], 0, sizeof(ServeDone));
                    sv->ring[e] = {r, r->published};
                    sv->published += 1;
                    r->published += 1;
                    outstanding += 1;
                    progress = true;
                }
                publish_count(sv);
                if (r->published == (int)r->chunks.size()) ready.erase(ready.begin() + i);
                else ++i;
            }
        }
        // (re)launch the loop when published jobs wait and it is not running
        if (!loop_live(sv) && lo < sv->published) {
            unsigned long long claimed = 0;
            cudaMemcpy(&claimed, sv->claimed_d, sizeof(claimed), cudaMemcpyDeviceToHost);
            // a job claimed by a slot that left without its record (a group error) is failed
            for (int64_t j = lo; j < (int64_t)claimed; ++j) {
                ServeDone &d = sv->done_h[j % sv->R];
                if (*(volatile int32_t *)&d.state == 0) {
                    d.status = KPP_ERR_TIMEOUT;
                    for (int c = 0; c < SERVE_KP; ++c) d.col_status[c] = KPP_ERR_TIMEOUT;
                    *(volatile int32_t *)&d.state = 1;
                }
            }
            if ((int64_t)claimed < sv->published) {
                size_t smem = 0;
                for (int64_t j = (int64_t)claimed; j < sv->published; ++j) {
                    auto &rr = sv->ring[j % sv->R];
                    smem = std::max(smem, smem_need(sv, *sv->mats[rr.first->mat]));
                }
                for (auto &r : ready) smem = std::max(smem, smem_need(sv, *sv->mats[r->mat]));
                if (!launch_loop(sv, smem)) {
                    // cannot run the loop: fail every published job that no slot claimed
                    for (int64_t j = (int64_t)claimed; j < sv->published; ++j) {
                        ServeDone &d = sv->done_h[j % sv->R];
                        d.status = KPP_ERR_CUDA;
                        for (int c = 0; c < SERVE_KP; ++c) d.col_status[c] = KPP_ERR_CUDA;
                        *(volatile int32_t *)&d.state = 1;
                    }
                    unsigned long long pub = (unsigned long long)sv->published;
                    cudaMemcpy(sv->claimed_d, &pub, sizeof(pub), cudaMemcpyHostToDevice);
                }
                progress = true;
            }
        }
        // completions
        for (int64_t j = lo; j < sv->published; ++j) {
            ServeDone &d = sv->done_h[j % sv->R];
            auto &slot = sv->ring[j % sv->R];
            if (!slot.first) continue;
            if (*(volatile int32_t *)&d.state != 1) continue;
            std::atomic_thread_fence(std::memory_order_acquire);
            auto r = slot.first;
            Chunk &ch = r->chunks[slot.second];
            ch.rec = d;
            ch.done = true;
            slot.first.reset();
            outstanding -= 1;
            progress = true;
            if (--r->pending == 0) complete_request(sv, r);
        }
        while (lo < sv->published && !sv->ring[lo % sv->R].first) ++lo;
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    // shut the loop down
    set_drain(sv, 1);
    if (sv->k_live) cudaEventSynchronize(sv->ev_k);
    sv->k_live = false;
}

}  // namespace

using namespace kpp;

extern "C" {

kpp_status kpp_server_create(size_t hbm_budget_bytes, int32_t max_concurrent, int32_t grid_per_solve,
                             kpp_server_t *out) {
    clear_error();
    if (!out || hbm_budget_bytes == 0 || max_concurrent < 1 || max_concurrent > 64 || grid_per_solve < 0 ||
        grid_per_solve > 64) {
        set_error("kpp_server_create: invalid argument");
        return KPP_ERR_ARG;
    }
    auto *sv = new kpp_server_s;
    sv->budget = hbm_budget_bytes;
    sv->slots_max = max_concurrent;
    sv->G = grid_per_solve > 0 ? grid_per_solve : 8;
    cudaGetDevice(&sv->device);
    bool ok = cudaStreamCreateWithFlags(&sv->st_k, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&sv->st_io, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&sv->ev_k, cudaEventDisableTiming) == cudaSuccess &&
              cudaHostAlloc((void **)&sv->jobs_h, sizeof(ServeJob) * sv->R, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc((void **)&sv->done_h, sizeof(ServeDone) * sv->R, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc((void **)&sv->ctl_h, sizeof(ServeCtl), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&sv->jobs_d, sv->jobs_h, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&sv->done_d, sv->done_h, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&sv->ctl_d, sv->ctl_h, 0) == cudaSuccess &&
              kpp::dev_malloc((void **)&sv->slots_d, sizeof(ServeSlot) * 256) == cudaSuccess &&
              kpp::dev_malloc((void **)&sv->claimed_d, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMemset(sv->claimed_d, 0, sizeof(unsigned long long)) == cudaSuccess;
    if (!ok) {
        set_error("kpp_server_create: %s", cudaGetErrorString(cudaGetLastError()));
        if (sv->jobs_h) cudaFreeHost(sv->jobs_h);
        if (sv->done_h) cudaFreeHost(sv->done_h);
        if (sv->ctl_h) cudaFreeHost(sv->ctl_h);
        if (sv->slots_d) kpp::dev_free(sv->slots_d);
        if (sv->claimed_d) kpp::dev_free(sv->claimed_d);
        if (sv->ev_k) cudaEventDestroy(sv->ev_k);
        if (sv->st_k) cudaStreamDestroy(sv->st_k);
        if (sv->st_io) cudaStreamDestroy(sv->st_io);
        delete sv;
        return KPP_ERR_CUDA;
    }
    // the dispatcher thread reads registered entries without the lock: the table never reallocates
    sv->mats.reserve(kMaxMatrices);
    memset(sv->ctl_h, 0, sizeof(ServeCtl));
    memset(sv->done_h, 0, sizeof(ServeDone) * sv->R);
    sv->ring.assign(sv->R, {});
    sv->disp = std::thread(dispatcher_main, sv);
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
    // the loop's shared memory holds s x 8 x 2 doubles and a column chunk of x: refuse what cannot fit
    if (kpp::serve_smem_bytes(s, serve_cw(*A, sv->G)) > 200 * 1024) {
        set_error("kpp_server_add_matrix: block size %d with %lld columns over %d CTAs per slot does not fit the "
                  "serving loop's shared memory",
                  s, (long long)A->cols, sv->G);
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
    if (sv->mats.size() >= kMaxMatrices) {
        kpp_partition_destroy(m->P);
        set_error("kpp_server_add_matrix: at most %d matrices per server", (int)kMaxMatrices);
        return KPP_ERR_ARG;
    }
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
    const clk::time_point t_call = clk::now();  // latency counts any wait for the server's lock
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
    r->bytes = 0;
    for (int c0 = 0; c0 < k; c0 += SERVE_KP) r->bytes += chunk_bytes(m, std::min(SERVE_KP, k - c0), sv->G);
    r->t_submit = t_call;
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
                                    [&] { return sv->queue.empty() && sv->active.empty(); });
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
    out->loop_launches = sv->k_launches;
    out->loop_slots = sv->k_slots;
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
    if (sv->disp.joinable()) sv->disp.join();
    cudaStreamSynchronize(sv->st_io);
    cudaStreamSynchronize(sv->st_k);
    for (auto &m : sv->mats) {
        if (m->F) kpp_factors_destroy(m->F);
        if (m->P) kpp_partition_destroy(m->P);
    }
    cudaFreeHost(sv->jobs_h);
    cudaFreeHost(sv->done_h);
    cudaFreeHost(sv->ctl_h);
    kpp::dev_free(sv->slots_d);
    kpp::dev_free(sv->claimed_d);
    cudaEventDestroy(sv->ev_k);
    cudaStreamDestroy(sv->st_k);
    cudaStreamDestroy(sv->st_io);
    delete sv;
}

}  // extern "C"
