// kpp_plan.cu -- prepared batched solves that run without host involvement, and the launch
// autotuner.
//
// A plan binds the systems of a batched K++ / CD++ solve (Alg. 3 / Alg. 5 run on nsys systems with k
// right-hand sides each) to every buffer and kernel descriptor it needs, once.  kpp_plan_launch then
// enqueues the whole solve -- for FP32 / BF16 storage including the FP64 iterative refinement -- as
// kernels and memsets only, so that a CUDA graph can capture it and replay it.  The host loop of the
// one-shot entry points decides after each refinement step which systems continue; here that
// decision is taken on the device by plan_check_kernel, and the graph always holds max_outer steps,
// which fall through at no cost once every system has converged.
//
// The autotuner times short runs of the persistent kernel for a few (kernel generation, CTAs per
// system) pairs and keeps the fastest per shape in a process-wide cache, which can be saved to and
// loaded from a text file.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kpp_internal.cuh"
#include "kpp_launch.h"

namespace kpp {

// Per-system state of a plan's refinement loop (device).
struct PlanSys {
    long long iters;    // inner steps run so far
    long long outer;    // refinement steps run so far
    long long t_start;  // first step of the current inner solve
    int run;            // 1: the system takes the current inner solve
    int done;           // 1: every column has met the tolerance (or the system failed)
    int err;            // first device error of the system's inner solves
    int pad;
};

// Reset of a plan's state at the start of a launch: scalars of every column from the initial
// template, the refinement bookkeeping and the global step counter.
__global__ void plan_reset_kernel(int nsys, int k, SolveScalars *__restrict__ sc, const SolveScalars *__restrict__ sc0,
                                  PlanSys *__restrict__ ps, long long *__restrict__ t_global) {
    for (int e = threadIdx.x; e < nsys * k; e += blockDim.x) sc[e] = sc0[e % k];
    for (int i = threadIdx.x; i < nsys; i += blockDim.x) ps[i] = PlanSys{0, 0, 0, 0, 0, 0, 0};
    if (threadIdx.x == 0) *t_global = 0;
}

// The check after r = b - A x of a refinement step (the host loop of the one-shot path, taken on the
// device): per system still going, |r|^2 (and on the first step |b|^2) from the residual kernel's
// per-CTA partials summed in CTA order; per column the stop test |r| <= tol |b|; the columns that
// continue restart their inner solve at the shared step counter (E0 = E1 = 0, rho kept).
__global__ void plan_check_kernel(int nsys, int k, int RG, const double *__restrict__ res_part,
                                  const double *__restrict__ bn2_part, double *__restrict__ res2,
                                  double *__restrict__ bn2, int first, int last, double tol, PlanSys *__restrict__ ps,
                                  SolveScalars *__restrict__ sc, const long long *__restrict__ t_global) {
    for (int i = threadIdx.x; i < nsys; i += blockDim.x) {
        PlanSys &q = ps[i];
        q.run = 0;
        if (q.done) continue;
        int active = 0;
        for (int c = 0; c < k; ++c) {
            double r2 = 0.0;
            for (int g = 0; g < RG; ++g) r2 += res_part[((size_t)i * RG + g) * k + c];
            res2[(size_t)i * k + c] = r2;
            if (first) {
                double b2 = 0.0;
                for (int g = 0; g < RG; ++g) b2 += bn2_part[((size_t)i * RG + g) * k + c];
                bn2[(size_t)i * k + c] = b2;
            }
            const double b2 = bn2[(size_t)i * k + c];
            const double rel = b2 > 0 ? sqrt(r2 / b2) : sqrt(r2);
            const bool conv = rel <= tol;
            SolveScalars &s = sc[(size_t)i * k + c];
            s.active = conv ? 0 : 1;
            s.status = conv ? KPP_OK : KPP_ERR_NO_CONVERGENCE;
            s.E0 = 0.0;
            s.E1 = 0.0;
            active += !conv;
        }
        if (!active) {
            q.done = 1;
            continue;
        }
        if (last) continue;
        q.run = 1;
        q.outer += 1;
        q.t_start = *t_global;
        for (int c = 0; c < k; ++c) sc[(size_t)i * k + c].t = *t_global;
    }
}

// After an inner solve: step counts, the shared step counter moved past every system's last step
// (so that the next inner solves draw fresh blocks), and device errors (the system stops).
__global__ void plan_post_kernel(int nsys, int k, PlanSys *__restrict__ ps, const SolveScalars *__restrict__ sc,
                                 const int *__restrict__ errs, long long *__restrict__ t_global) {
    if (threadIdx.x != 0) return;
    long long tmax = *t_global;
    for (int i = 0; i < nsys; ++i) {
        PlanSys &q = ps[i];
        if (!q.run) continue;
        const long long t = sc[(size_t)i * k].t;
        q.iters += t - q.t_start;
        tmax = t > tmax ? t : tmax;
        if (errs[i]) {
            q.err = errs[i];
            q.done = 1;
            q.run = 0;
        }
    }
    *t_global = tmax;
}

// x += d (FP64 += FP32) for the systems that took the inner solve.
__global__ void plan_axpy_kernel(int nsys, int64_t n, const float *const *__restrict__ d, double *const *__restrict__ X,
                                 const PlanSys *__restrict__ ps) {
    const int i = blockIdx.y;
    if (i >= nsys || !ps[i].run) return;
    const float *di = d[i];
    double *xi = X[i];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        xi[e] += (double)di[e];
}

// ---------------------------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------------------------
static std::mutex g_tune_mu;
static std::map<std::string, TuneChoice> g_tune_cache;

static std::string tune_key(const kpp_matrix &A, int nsys, int k, int s, bool cd, int limit) {
    int dev = 0, maj = 0, mnr = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev);
    char buf[192];
    snprintf(buf, sizeof(buf), "sm%d%d-n%d:r%lld:c%lld:d%d:s%d:k%d:m%d:n%d:v%d", maj, mnr, sm_count(),
             (long long)A.rows, (long long)A.cols, A.dtype, s, k, cd ? 1 : 0, nsys, limit);
    return buf;
}

// Trial buffers of the autotuner: a zero start, the right-hand sides in the compute type.
struct TuneTrial {
    int nsys, k, dtype, s;
    bool cd;
    double eta;
    const kpp_matrix *A;
    const kpp_factors_t *F;
    const kpp_params *p;
    std::vector<void *> xb, bb;
    std::vector<std::vector<SolveScalars>> sc;
    std::vector<SysInput> in;
    std::vector<int> errs;
};

// One timed run of T steps (no stop test) with the given generation and grid; the best of two runs
// (the first launch of a kernel also loads its module).  ms_out = INFINITY when the shape cannot run.
static kpp_status tune_measure(TuneTrial &tr, int variant, int grid, int64_t T, cudaStream_t st, float &ms_out,
                               int &G_out) {
    kpp_status rc = KPP_OK;
    const size_t tcs = tr.dtype == KPP_F64 ? 8 : 4;
    ms_out = INFINITY;
    for (int rep = 0; rep < 2; ++rep) {
        for (int i = 0; i < tr.nsys; ++i) {
            init_scalars(tr.sc[i], tr.k, tr.p->rho0);
            CUDA_OR(cudaMemsetAsync(tr.xb[i], 0, (size_t)tr.A[0].cols * tr.k * tcs, st), KPP_ERR_CUDA);
            tr.in[i] = SysInput{&tr.A[i], tr.bb[i], tr.xb[i], &tr.F[i]->f, tr.p->sys_id + (uint32_t)i, tr.sc[i].data()};
        }
        float ms = 0.f;
        int kind = 0;
        kpp_status r = run_persistent(tr.in, tr.dtype, tr.cd, tr.k, tr.s, tr.eta, /*tol=*/0.0, tr.p->adaptive_rho, 0,
                                      T, tr.p->seed, grid, true, 0, st, &ms, tr.errs.data(), variant, &kind, &G_out);
        if (r == KPP_ERR_UNSUPPORTED || r == KPP_ERR_TIMEOUT || r == KPP_ERR_NUMERIC) {
            ms_out = INFINITY;
            clear_error();
            return KPP_OK;
        }
        if (r != KPP_OK) return r;
        ms_out = std::min(ms_out, ms);
    }
cleanup:
    return rc;
}

kpp_status tune_launch(int nsys, const kpp_matrix *A, const double *const *B, int k, kpp_partition_t P,
                       const kpp_factors_t *F, const kpp_params &p, bool cd, cudaStream_t st, TuneChoice &out) {
    const std::string key = tune_key(A[0], nsys, k, P->s, cd, g_variant);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            out = it->second;
            return KPP_OK;
        }
    }
    kpp_status rc = KPP_OK;
    const int dtype = A[0].dtype;
    const size_t tcs = dtype == KPP_F64 ? 8 : 4;
    const int64_t rows = A[0].rows, cols = A[0].cols;
    const int nb = (int)((rows + P->s - 1) / P->s);
    Scratch scr(st);
    TuneTrial tr{nsys, k, dtype, P->s, cd, default_eta(p, P->s, rows, cols), A, F, &p, {}, {}, {}, {}, {}};
    tr.xb.assign(nsys, nullptr);
    tr.bb.assign(nsys, nullptr);
    tr.sc.assign(nsys, {});
    tr.in.assign(nsys, SysInput{});
    tr.errs.assign(nsys, 0);
    std::vector<int> variants{g_variant};
    if (cd && g_variant >= 3) variants.push_back(2);
    double best = INFINITY;
    TuneChoice pick;
    float ms = 0.f;
    int G0 = 0;
    // trial length: about two sweeps over the blocks, shortened for slow shapes to ~50 ms a run
    int64_t T = std::max<int64_t>(32, std::min<int64_t>(2 * (int64_t)nb, 512));
    for (int i = 0; i < nsys; ++i) {
        CUDA_OR(scr.alloc(&tr.xb[i], (size_t)cols * k * tcs), KPP_ERR_CUDA);
        if (dtype == KPP_F64) {
            tr.bb[i] = (void *)B[i];
        } else {
            CUDA_OR(scr.alloc(&tr.bb[i], (size_t)rows * k * tcs), KPP_ERR_CUDA);
            CUDA_OR(launch_f64_to_f32((int64_t)rows * k, B[i], (float *)tr.bb[i], st), KPP_ERR_CUDA);
        }
    }
    {
        kpp_status r = tune_measure(tr, g_variant, 0, T, st, ms, G0);
        if (r != KPP_OK) {
            rc = r;
            goto cleanup;
        }
        if (std::isfinite(ms) && ms > 50.f) T = std::max<int64_t>(16, (int64_t)((double)T * 50.0 / ms));
    }
    for (int v : variants) {
        int Gh = 0;
        kpp_status r = tune_measure(tr, v, 0, T, st, ms, Gh);  // the heuristic's shape
        if (r != KPP_OK) {
            rc = r;
            goto cleanup;
        }
        std::vector<int> grids;
        if (std::isfinite(ms)) {
            if (ms / T < best) {
                best = ms / T;
                pick = TuneChoice{v, Gh};
            }
            const int cap = std::max(1, 2 * sm_count() / nsys);
            for (int g : {Gh / 4, Gh / 2, (3 * Gh) / 4, (3 * Gh) / 2, 2 * Gh, sm_count() / nsys, cap}) {
                g = std::max(1, std::min(g, cap));
                if (g != Gh && std::find(grids.begin(), grids.end(), g) == grids.end()) grids.push_back(g);
            }
        }
        for (int g : grids) {
            int Gu = 0;
            r = tune_measure(tr, v, g, T, st, ms, Gu);
            if (r != KPP_OK) {
                rc = r;
                goto cleanup;
            }
            if (std::isfinite(ms) && ms / T < best) {
                best = ms / T;
                pick = TuneChoice{v, Gu};
            }
        }
    }
    if (!std::isfinite(best)) {
        set_error("autotuner: no launch shape ran");
        rc = KPP_ERR_UNSUPPORTED;
        goto cleanup;
    }
    out = pick;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = pick;
    }
cleanup:
    return rc;
}

}  // namespace kpp

using namespace kpp;

// ---------------------------------------------------------------------------------------------
// Plans
// ---------------------------------------------------------------------------------------------
struct kpp_plan_s {
    int nsys = 0, k = 1, dtype = 0, s = 0;
    bool cd = false;
    int form = 0;  // 0: FP64 iterations on b, x; 1: one FP32 solve; 2: FP32 solves + FP64 refinement
    kpp_params p{};
    TuneChoice tune;
    std::vector<kpp_matrix> A;
    std::vector<const double *> B;
    std::vector<double *> X;
    Scratch mem{nullptr, false};
    PersistentLaunch L;
    SolveScalars *sc = nullptr;   // nsys x k
    SolveScalars *sc0 = nullptr;  // k (initial values)
    PlanSys *ps = nullptr;        // nsys
    long long *t_global = nullptr;
    std::vector<float *> b32, d32;
    const float **d_d32 = nullptr;
    double **d_X = nullptr;
    int RG = 0;  // residual grid
    double *res_part = nullptr, *bn2_part = nullptr, *res2 = nullptr, *bn2 = nullptr;
};

extern "C" {

kpp_status kpp_plan_create(int32_t nsys, const kpp_matrix *A, const double *const *B, double *const *X, int32_t k,
                           kpp_partition_t P, const kpp_factors_t *F, const kpp_params *pp, int32_t mode,
                           void *stream, kpp_plan_t *out) {
    clear_error();
    if (!out || (mode != 0 && mode != 1)) {
        set_error("invalid argument (out=%p, mode=%d)", (void *)out, mode);
        return KPP_ERR_ARG;
    }
    *out = nullptr;
    const bool cd = mode == 1;
    {
        kpp_status v = validate_systems(nsys, A, B, X, k, P, F, pp, cd);
        if (v != KPP_OK) return v;
    }
    cudaStream_t st = (cudaStream_t)stream;
    kpp_status rc = KPP_OK;
    kpp_plan_s *pl = new kpp_plan_s();
    const kpp_params p = *pp;
    pl->nsys = nsys;
    pl->k = k;
    pl->dtype = A[0].dtype;
    pl->s = P->s;
    pl->cd = cd;
    pl->p = p;
    pl->form = pl->dtype == KPP_F64 ? 0 : (p.refine ? 2 : 1);
    pl->A.assign(A, A + nsys);
    pl->B.assign(B, B + nsys);
    pl->X.assign(X, X + nsys);
    const int64_t rows = A[0].rows, cols = A[0].cols;
    const size_t nr = (size_t)rows * k, nc = (size_t)cols * k;
    const double eta = default_eta(p, pl->s, rows, cols);
    std::vector<SolveScalars> sc0;
    std::vector<SysInput> in(nsys);
    init_scalars(sc0, k, p.rho0);
    pl->tune.grid = p.grid;
    if (p.grid < 0) {
        rc = tune_launch(nsys, A, B, k, P, F, p, cd, st, pl->tune);
        if (rc != KPP_OK) goto cleanup;
    }
    CUDA_OR(pl->mem.alloc((void **)&pl->sc, (size_t)nsys * k * sizeof(SolveScalars)), KPP_ERR_CUDA);
    CUDA_OR(pl->mem.alloc((void **)&pl->sc0, (size_t)k * sizeof(SolveScalars)), KPP_ERR_CUDA);
    CUDA_OR(pl->mem.alloc((void **)&pl->ps, (size_t)nsys * sizeof(PlanSys)), KPP_ERR_CUDA);
    CUDA_OR(pl->mem.alloc((void **)&pl->t_global, sizeof(long long)), KPP_ERR_CUDA);
    CUDA_OR(cudaMemcpyAsync(pl->sc0, sc0.data(), (size_t)k * sizeof(SolveScalars), cudaMemcpyHostToDevice, st),
            KPP_ERR_CUDA);
    if (pl->form > 0) {
        pl->b32.assign(nsys, nullptr);
        pl->d32.assign(nsys, nullptr);
        for (int i = 0; i < nsys; ++i) {
            CUDA_OR(pl->mem.alloc((void **)&pl->b32[i], nr * sizeof(float)), KPP_ERR_CUDA);
            CUDA_OR(pl->mem.alloc((void **)&pl->d32[i], nc * sizeof(float)), KPP_ERR_CUDA);
        }
    }
    if (pl->form == 2) {
        pl->RG = residual_grid();
        const size_t np = (size_t)nsys * pl->RG * k;
        CUDA_OR(pl->mem.alloc((void **)&pl->res_part, np * sizeof(double)), KPP_ERR_CUDA);
        CUDA_OR(pl->mem.alloc((void **)&pl->bn2_part, np * sizeof(double)), KPP_ERR_CUDA);
        CUDA_OR(pl->mem.alloc((void **)&pl->res2, (size_t)nsys * k * sizeof(double)), KPP_ERR_CUDA);
        CUDA_OR(pl->mem.alloc((void **)&pl->bn2, (size_t)nsys * k * sizeof(double)), KPP_ERR_CUDA);
        CUDA_OR(pl->mem.alloc((void **)&pl->d_d32, nsys * sizeof(float *)), KPP_ERR_CUDA);
        CUDA_OR(pl->mem.alloc((void **)&pl->d_X, nsys * sizeof(double *)), KPP_ERR_CUDA);
        CUDA_OR(cudaMemcpyAsync(pl->d_d32, pl->d32.data(), nsys * sizeof(float *), cudaMemcpyHostToDevice, st),
                KPP_ERR_CUDA);
        CUDA_OR(cudaMemcpyAsync(pl->d_X, pl->X.data(), nsys * sizeof(double *), cudaMemcpyHostToDevice, st),
                KPP_ERR_CUDA);
    }
    for (int i = 0; i < nsys; ++i) {
        const void *bi = pl->form == 0 ? (const void *)B[i] : (const void *)pl->b32[i];
        void *xi = pl->form == 0 ? (void *)X[i] : (void *)pl->d32[i];
        in[i] = SysInput{&pl->A[i], bi, xi, &F[i]->f, p.sys_id + (uint32_t)i, nullptr, pl->sc + (size_t)i * k};
    }
    if (pl->form == 2) {
        rc = prepare_persistent(pl->L, in, pl->dtype, cd, k, pl->s, eta, p.inner_tol, p.adaptive_rho, 0, p.max_iters,
                                p.seed, pl->tune.grid, /*init_residual=*/false, 0, /*t0_state=*/true,
                                pl->tune.variant < 0 ? g_variant : pl->tune.variant, pl->mem, st);
    } else {
        rc = prepare_persistent(pl->L, in, pl->dtype, cd, k, pl->s, eta, p.tol, p.adaptive_rho, pl->form == 0 ? 1 : 0,
                                p.max_iters, p.seed, pl->tune.grid, true, 0, false,
                                pl->tune.variant < 0 ? g_variant : pl->tune.variant, pl->mem, st);
    }
    if (rc != KPP_OK) goto cleanup;
    CUDA_OR(cudaStreamSynchronize(st), KPP_ERR_CUDA);
    *out = pl;
    return KPP_OK;
cleanup:
    cudaStreamSynchronize(st);
    delete pl;
    return rc;
}

kpp_status kpp_plan_launch(kpp_plan_t pl, void *stream) {
    clear_error();
    if (!pl) {
        set_error("null plan");
        return KPP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    kpp_status rc = KPP_OK;
    const int nsys = pl->nsys, k = pl->k;
    const size_t nr = (size_t)pl->A[0].rows * k, nc = (size_t)pl->A[0].cols * k;
    note_launch();
    plan_reset_kernel<<<1, 256, 0, st>>>(nsys, k, pl->sc, pl->sc0, pl->ps, pl->t_global);
    CUDA_OR(cudaGetLastError(), KPP_ERR_CUDA);
    if (pl->form == 0) {
        rc = enqueue_persistent(pl->L, st);
        if (rc != KPP_OK) goto cleanup;
    } else if (pl->form == 1) {
        for (int i = 0; i < nsys; ++i) {
            CUDA_OR(launch_f64_to_f32((int64_t)nr, pl->B[i], pl->b32[i], st), KPP_ERR_CUDA);
            CUDA_OR(launch_f64_to_f32((int64_t)nc, pl->X[i], pl->d32[i], st), KPP_ERR_CUDA);
        }
        rc = enqueue_persistent(pl->L, st);
        if (rc != KPP_OK) goto cleanup;
        for (int i = 0; i < nsys; ++i) {
            CUDA_OR(cudaMemsetAsync(pl->X[i], 0, nc * sizeof(double), st), KPP_ERR_CUDA);
            CUDA_OR(launch_axpy((int64_t)nc, pl->d32[i], pl->X[i], st), KPP_ERR_CUDA);
        }
    } else {
        const int max_outer = std::max(0, pl->p.max_outer);
        for (int o = 0; o <= max_outer; ++o) {
            for (int i = 0; i < nsys; ++i) {
                double *part = pl->res_part + (size_t)i * pl->RG * k;
                CUDA_OR(launch_residual_grid(pl->A[i], k, pl->B[i], pl->X[i], pl->b32[i], part, pl->RG, st,
                                             &pl->ps[i].done),
                        KPP_ERR_CUDA);
                if (o == 0)
                    CUDA_OR(launch_residual_grid(pl->A[i], k, pl->B[i], nullptr, nullptr,
                                                 pl->bn2_part + (size_t)i * pl->RG * k, pl->RG, st),
                            KPP_ERR_CUDA);
            }
            note_launch();
            plan_check_kernel<<<1, 128, 0, st>>>(nsys, k, pl->RG, pl->res_part, pl->bn2_part, pl->res2, pl->bn2,
                                                 o == 0, o == max_outer, pl->p.tol, pl->ps, pl->sc, pl->t_global);
            CUDA_OR(cudaGetLastError(), KPP_ERR_CUDA);
            if (o == max_outer) break;
            for (int i = 0; i < nsys; ++i) CUDA_OR(cudaMemsetAsync(pl->d32[i], 0, nc * sizeof(float), st), KPP_ERR_CUDA);
            rc = enqueue_persistent(pl->L, st);
            if (rc != KPP_OK) goto cleanup;
            note_launch();
            plan_post_kernel<<<1, 32, 0, st>>>(nsys, k, pl->ps, pl->sc, pl->L.errs, pl->t_global);
            CUDA_OR(cudaGetLastError(), KPP_ERR_CUDA);
            {
                const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)(nc + 255) / 256,
                                                                           std::max(1, 2 * sm_count() / nsys)));
                note_launch();
                plan_axpy_kernel<<<dim3(gx, nsys), 256, 0, st>>>(nsys, (int64_t)nc, pl->d_d32, pl->d_X, pl->ps);
                CUDA_OR(cudaGetLastError(), KPP_ERR_CUDA);
            }
        }
    }
cleanup:
    return rc;
}

kpp_status kpp_plan_report(kpp_plan_t pl, kpp_report *reps, void *stream) {
    clear_error();
    if (!pl) {
        set_error("null plan");
        return KPP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    kpp_status rc = KPP_OK;
    const int nsys = pl->nsys, k = pl->k;
    std::vector<SolveScalars> sc((size_t)nsys * k);
    std::vector<PlanSys> ps(nsys);
    std::vector<int> errs(nsys, 0);
    kpp_status worst = KPP_OK;
    CUDA_OR(cudaMemcpyAsync(sc.data(), pl->sc, sc.size() * sizeof(SolveScalars), cudaMemcpyDeviceToHost, st),
            KPP_ERR_CUDA);
    CUDA_OR(cudaMemcpyAsync(ps.data(), pl->ps, nsys * sizeof(PlanSys), cudaMemcpyDeviceToHost, st), KPP_ERR_CUDA);
    CUDA_OR(cudaMemcpyAsync(errs.data(), pl->L.errs, nsys * sizeof(int), cudaMemcpyDeviceToHost, st), KPP_ERR_CUDA);
    CUDA_OR(cudaStreamSynchronize(st), KPP_ERR_CUDA);
    for (int i = 0; i < nsys; ++i) {
        std::vector<double> r2, b2;
        kpp_status r3 = residual_norms(pl->A[i], k, pl->B[i], pl->X[i], nullptr, r2, &b2, st);
        if (r3 != KPP_OK) return r3;
        const int err = pl->form == 2 ? ps[i].err : errs[i];
        for (int c = 0; c < k; ++c) {
            const SolveScalars &s = sc[(size_t)i * k + c];
            const double rel = b2[c] > 0 ? std::sqrt(r2[c] / b2[c]) : std::sqrt(r2[c]);
            kpp_status cs = (kpp_status)s.status;
            if (err) cs = (kpp_status)err;
            else if (!std::isfinite(rel)) cs = KPP_ERR_NUMERIC;
            else if (pl->form == 2) cs = rel <= pl->p.tol ? KPP_OK : KPP_ERR_NO_CONVERGENCE;
            if (worst == KPP_OK) worst = cs;
            if (reps) {
                kpp_report &r = reps[(size_t)i * k + c];
                memset(&r, 0, sizeof(r));
                r.iters = pl->form == 2 ? ps[i].iters : sc[(size_t)i * k].t;
                r.outer = pl->form == 2 ? ps[i].outer : 0;
                r.rel_res_true = rel;
                r.rel_res_est = s.res_est;
                r.rho_final = s.rho;
                r.status = cs;
                r.bad_block = -1;
                r.device_ms = 0.0;
            }
        }
    }
    if (worst != KPP_OK) set_error("solve ended with %s", kpp_status_string(worst));
    return worst;
cleanup:
    return rc;
}

kpp_status kpp_plan_info(kpp_plan_t pl, int32_t *kernel, int32_t *grid, int32_t *variant) {
    clear_error();
    if (!pl) {
        set_error("null plan");
        return KPP_ERR_ARG;
    }
    if (kernel) *kernel = pl->L.kind;
    if (grid) *grid = pl->L.cm.G;
    if (variant) *variant = pl->tune.variant < 0 ? g_variant : pl->tune.variant;
    return KPP_OK;
}

void kpp_plan_destroy(kpp_plan_t pl) {
    if (!pl) return;
    cudaDeviceSynchronize();  // no launch of the plan may still be running
    delete pl;
}

int64_t kpp_tune_cache_size(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (int64_t)g_tune_cache.size();
}

void kpp_tune_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.clear();
}

kpp_status kpp_tune_cache_save(const char *path) {
    clear_error();
    if (!path) {
        set_error("null path");
        return KPP_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    FILE *f = fopen(path, "w");
    if (!f) {
        set_error("cannot open %s for writing", path);
        return KPP_ERR_ARG;
    }
    fprintf(f, "# libkpp launch autotuner cache: key variant grid\n");
    for (const auto &kv : g_tune_cache) fprintf(f, "%s %d %d\n", kv.first.c_str(), kv.second.variant, kv.second.grid);
    fclose(f);
    return KPP_OK;
}

kpp_status kpp_tune_cache_load(const char *path) {
    clear_error();
    if (!path) {
        set_error("null path");
        return KPP_ERR_ARG;
    }
    FILE *f = fopen(path, "r");
    if (!f) {
        set_error("cannot open %s", path);
        return KPP_ERR_ARG;
    }
    std::map<std::string, TuneChoice> got;
    char line[512];
    kpp_status rc = KPP_OK;
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        char key[256];
        int v = 0, g = 0;
        if (sscanf(line, "%255s %d %d", key, &v, &g) != 3 || v < 1 || v > 3 || g < 1) {
            set_error("malformed line in %s: %s", path, line);
            rc = KPP_ERR_ARG;
            break;
        }
        got[key] = TuneChoice{v, g};
    }
    fclose(f);
    if (rc != KPP_OK) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto &kv : got) g_tune_cache[kv.first] = kv.second;
    return KPP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Block-size autotuner
// ---------------------------------------------------------------------------------------------
// For each candidate block size (contiguous partition): the factor phase of every system (event
// time), then two segments of T steps of the persistent kernel with no stop test (the launch shape
// the heuristic picks for that s), each followed by the residual of every column.  The contraction per
// step over the second segment, q = (prod_c |r_2T| / |r_T|)^(1 / (T * columns)), gives the steps
// still needed to a relative residual tol, and the estimate factor_ms + ms_per_step * steps.  FP32 /
// BF16 storage runs the inner FP32 iteration (the refinement's cost per step), FP64 storage the FP64
// one.
extern "C" kpp_status kpp_tune_block_size(int32_t nsys, const kpp_matrix *A, const double *const *B, int32_t k,
                                          const int32_t *cand, int32_t ncand, const kpp_params *pp, int32_t cd,
                                          int32_t *out_s, double *est_ms, void *stream) {
    clear_error();
    if (nsys < 1 || !A || !B || k < 1 || k > 32 || !cand || ncand < 1 || !pp || !out_s || !(pp->tol > 0.0) ||
        pp->tol >= 1.0) {
        set_error("kpp_tune_block_size: invalid argument (needs 0 < tol < 1, 1 <= k <= 32, candidates)");
        return KPP_ERR_ARG;
    }
    for (int i = 0; i < nsys; ++i)
        if (!matrix_ok(&A[i]) || !B[i] || A[i].rows != A[0].rows || A[i].cols != A[0].cols ||
            A[i].dtype != A[0].dtype || (cd && A[i].rows != A[i].cols)) {
            set_error("kpp_tune_block_size: system %d does not match system 0 (or CD++ needs square)", i);
            return KPP_ERR_ARG;
        }
    for (int c = 0; c < ncand; ++c)
        if (cand[c] < 1 || cand[c] > 1024 || cand[c] > A[0].rows) {
            set_error("kpp_tune_block_size: candidate %d out of range", cand[c]);
            return KPP_ERR_ARG;
        }
    cudaStream_t st = (cudaStream_t)stream;
    const kpp_params p = *pp;
    const int dtype = A[0].dtype;
    const size_t tcs = dtype == KPP_F64 ? 8 : 4;
    const int64_t rows = A[0].rows, cols = A[0].cols;
    kpp_status rc = KPP_OK;
    double best = INFINITY;
    int best_s = -1;
    Scratch scr(st);
    std::vector<void *> xb(nsys), bb(nsys);
    std::vector<double> b2(nsys * k, 0.0);
    for (int i = 0; i < nsys; ++i) {
        CUDA_OR(scr.alloc(&xb[i], (size_t)cols * k * tcs), KPP_ERR_CUDA);
        if (dtype == KPP_F64) {
            bb[i] = (void *)B[i];
        } else {
            CUDA_OR(scr.alloc(&bb[i], (size_t)rows * k * tcs), KPP_ERR_CUDA);
            CUDA_OR(launch_f64_to_f32((int64_t)rows * k, B[i], (float *)bb[i], st), KPP_ERR_CUDA);
        }
        std::vector<double> r2, bn2;
        kpp_status r3 = residual_norms(A[i], k, B[i], nullptr, nullptr, r2, &bn2, st);
        if (r3 != KPP_OK) return r3;
        for (int c = 0; c < k; ++c) b2[(size_t)i * k + c] = bn2[c];
    }
    for (int ci = 0; ci < ncand; ++ci) {
        const int s = cand[ci];
        if (est_ms) est_ms[ci] = INFINITY;
        kpp_partition_s P{rows, s, (rows + s - 1) / s};
        std::vector<kpp_factors_t> F(nsys, nullptr);
        double fac_ms = 0.0;
        bool ok = true;
        for (int i = 0; i < nsys && ok; ++i) {
            kpp_status fr = kpp_factor_blocks(&A[i], &P, p.lambda, cd ? 1 : 0, &F[i], stream);
            if (fr != KPP_OK) {
                ok = false;
                break;
            }
            double sm[4];
            kpp_factors_stage_ms(F[i], sm);
            for (double v : sm)
                if (std::isfinite(v)) fac_ms += v;
        }
        if (ok) {
            // two segments of T steps (six sweeps over the blocks, 24 .. 1024): the first from x = 0 as a
            // burn-in (a Kaczmarz iteration shrinks the error, not always the residual, at first), the
            // second continuing from its x (momentum restarted, the Philox counter continuing); the
            // contraction is measured over the second
            const int64_t nb = P.nb;
            const int64_t T = std::max<int64_t>(24, std::min<int64_t>(6 * nb, 1024));
            std::vector<std::vector<SolveScalars>> sc(nsys);
            std::vector<SysInput> in(nsys);
            std::vector<int> errs(nsys, 0);
            std::vector<std::vector<double>> rr(2, std::vector<double>((size_t)nsys * k, 0.0));
            double seg_ms = 0.0;
            for (int i = 0; i < nsys; ++i)
                if (cudaMemsetAsync(xb[i], 0, (size_t)cols * k * tcs, st) != cudaSuccess) ok = false;
            for (int seg = 0; seg < 2 && ok; ++seg) {
                for (int i = 0; i < nsys; ++i) {
                    init_scalars(sc[i], k, p.rho0);
                    in[i] = SysInput{&A[i], bb[i], xb[i], &F[i]->f, p.sys_id + (uint32_t)i, sc[i].data()};
                }
                float ms = 0.f;
                kpp_status r = run_persistent(in, dtype, cd, k, s, default_eta(p, s, rows, cols), 0.0, p.adaptive_rho,
                                              0, seg * T + T, p.seed, 0, true, seg * T, st, &ms, errs.data(), -1);
                if (r == KPP_ERR_UNSUPPORTED || r == KPP_ERR_NUMERIC) {
                    ok = false;
                    break;
                }
                if (r != KPP_OK && r != KPP_ERR_NO_CONVERGENCE) {
                    rc = r;
                    ok = false;
                    break;
                }
                if (seg == 1) seg_ms = ms;
                for (int i = 0; i < nsys && ok; ++i) {
                    std::vector<double> r2;
                    kpp_status r3;
                    if (dtype == KPP_F64) {
                        r3 = residual_norms(A[i], k, B[i], (const double *)xb[i], nullptr, r2, nullptr, st);
                    } else {
                        double *x64 = nullptr;
                        r3 = scr.alloc((void **)&x64, (size_t)cols * k * 8) == cudaSuccess ? KPP_OK : KPP_ERR_OOM;
                        if (r3 == KPP_OK && (cudaMemsetAsync(x64, 0, (size_t)cols * k * 8, st) != cudaSuccess ||
                                             launch_axpy((int64_t)cols * k, (const float *)xb[i], x64, st) != cudaSuccess))
                            r3 = KPP_ERR_CUDA;
                        if (r3 == KPP_OK) r3 = residual_norms(A[i], k, B[i], x64, nullptr, r2, nullptr, st);
                    }
                    if (r3 != KPP_OK) {
                        ok = false;
                        break;
                    }
                    for (int c = 0; c < k; ++c) rr[seg][(size_t)i * k + c] = r2[c];
                }
            }
            if (ok) {
                // log of the contraction per step over the second segment (geometric mean over columns),
                // and the steps still needed after it to reach tol
                double lq = 0.0, lrel = 0.0;
                int cnt = 0;
                for (size_t c = 0; c < rr[0].size(); ++c) {
                    const double b0 = b2[c];
                    if (b0 > 0.0 && rr[0][c] > 0.0 && rr[1][c] > 0.0) {
                        lq += 0.5 * std::log(rr[1][c] / rr[0][c]);
                        lrel += 0.5 * std::log(rr[1][c] / b0);
                        ++cnt;
                    }
                }
                if (cnt > 0) {
                    lq /= (double)cnt * (double)T;
                    lrel /= (double)cnt;
                    if (lq < 0.0 && std::isfinite(lq)) {
                        const double more = std::max(0.0, (std::log(p.tol) - lrel) / lq);
                        const double est = fac_ms + seg_ms / (double)T * (2.0 * (double)T + more);
                        if (est_ms) est_ms[ci] = est;
                        if (est < best) {
                            best = est;
                            best_s = s;
                        }
                    }
                }
            }
        }
        for (kpp_factors_t f : F)
            if (f) kpp_factors_destroy(f);
        clear_error();
        if (rc != KPP_OK) return rc;
    }
    if (best_s < 0) {
        set_error("kpp_tune_block_size: no candidate reduced the residual");
        return KPP_ERR_NO_CONVERGENCE;
    }
    *out_s = best_s;
    return KPP_OK;
cleanup:
    return rc;
}
