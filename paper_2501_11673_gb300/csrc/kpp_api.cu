// kpp_api.cu -- the extern "C" boundary of libkpp (declared in include/kpp.h).
//
// Host-side orchestration only: argument checks, device buffers of a solve, the launch of the
// persistent solve kernel, the FP64 iterative-refinement loop of the mixed-precision form, and the
// report.  Every arithmetic step of the method runs in the kernels of kpp_solve.cu / kpp_factor.cu /
// kpp_gram_tc.cu.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kpp_internal.cuh"
#include "kpp_runtime.h"
#include "kpp_solve.h"
#include "kpp_launch.h"

namespace kpp {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}
void clear_error() { g_last_error.clear(); }

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }


// SM count of the current device, cached per device (atomic: the server's threads may ask first together).
int sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (!v) {
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        v = v > 0 ? v : 1;
        cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

void FactorSet::release() {
    dev_free(L);
    dev_free(Ginv);
    dev_free(Ginv32);
    dev_free(W32);
    W32 = nullptr;
    dev_free(W);
    W = nullptr;
    dev_free(Linv);
    Linv = nullptr;
    dev_free(LinvT);
    LinvT = nullptr;
    L = nullptr;
    Ginv = nullptr;
    Ginv32 = nullptr;
    for (cudaEvent_t &e : ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
}

// |A x - b|^2 and |b|^2 per column (deterministic: fixed grid, host sums in a fixed order).
kpp_status residual_norms(const kpp_matrix &A, int k, const double *b, const double *x, float *r32,
                                 std::vector<double> &res2, std::vector<double> *bn2, cudaStream_t st) {
    kpp_status rc = KPP_OK;
    const int grid = residual_grid();
    std::vector<double> h((size_t)grid * k);
    Scratch scr(st);
    double *part = nullptr;
    CUDA_OR(scr.alloc((void **)&part, (size_t)grid * k * sizeof(double)), KPP_ERR_CUDA);
    res2.assign(k, 0.0);
    CUDA_OR(launch_residual(A, k, b, x, r32, part, st), KPP_ERR_CUDA);
    CUDA_OR(cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st), KPP_ERR_CUDA);
    CUDA_OR(cudaStreamSynchronize(st), KPP_ERR_CUDA);
    for (int gi = 0; gi < grid; ++gi)
        for (int c = 0; c < k; ++c) res2[c] += h[(size_t)gi * k + c];
    if (bn2) {
        bn2->assign(k, 0.0);
        CUDA_OR(launch_residual(A, k, b, nullptr, nullptr, part, st), KPP_ERR_CUDA);
        CUDA_OR(cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st), KPP_ERR_CUDA);
        CUDA_OR(cudaStreamSynchronize(st), KPP_ERR_CUDA);
        for (int gi = 0; gi < grid; ++gi)
            for (int c = 0; c < k; ++c) (*bn2)[c] += h[(size_t)gi * k + c];
    }
cleanup:
    return rc;
}

int auto_grid(int64_t cols, int nsys) {
    // enough CTAs to spread the block rows, at most one CTA per SM for the whole launch
    int per = (int)std::min<int64_t>((cols + 31) / 32, 1024);
    int cap = std::max(1, sm_count() / std::max(1, nsys));
    return std::max(1, std::min(per, cap));
}

int g_variant = 3;
// The wait test (kpp_set_wait_test): the device wait limit of the persistent kernels (0: 2 s) and
// the CTA that the general kernel holds back from its first group barrier (-1: none).
static uint64_t g_wait_ns = 0;
static int g_hold_cta = -1;

kpp_status prepare_persistent(PersistentLaunch &L, std::vector<SysInput> &sys, int dtype, bool cd, int k,
                                     int s, double eta, double tol, int adaptive, int confirm, int64_t max_iters,
                                     uint64_t seed, int grid, bool init_residual, int64_t t0, bool t0_state,
                                     int variant, Scratch &scr, cudaStream_t st) {
    const bool use_v2 = variant >= 2;
    kpp_status rc = KPP_OK;
    const int nsys = (int)sys.size();
    const kpp_matrix &A0 = *sys[0].A;
    const bool f64 = dtype == KPP_F64;
    const size_t tcs = f64 ? 8 : 4;
    const int KP = pick_kp(k);
    int G = grid > 0 ? grid : auto_grid(A0.cols, nsys);
    const int64_t sector = 32 / (int64_t)dtype_size(dtype);
    int64_t CW = (A0.cols + G - 1) / G;
    CW = (CW + sector - 1) / sector * sector;
    G = (int)((A0.cols + CW - 1) / CW);  // no CTA without columns
    const int nb = (int)((A0.rows + s - 1) / s);
    bool v2 = use_v2;
    for (int i = 0; v2 && i < nsys; ++i) v2 = solve2_eligible(*sys[i].A, s, CW, KP, f64, cd, G);
    // CD++ dataflow kernel: same eligibility as v2, plus the memoised W for FP64
    bool v3 = cd && v2 && variant >= 3;
    for (int i = 0; v3 && i < nsys; ++i) {
        if (f64 && !sys[i].F->W) v3 = false;
        const size_t tas = f64 ? 8 : dtype_size(dtype);
        if (cd3_smem_bytes(s, CW, KP, (int)tas, (int)tcs, f64) > 200 * 1024) v3 = false;
    }
    if (v3) v2 = false;
    // wide FP32 / BF16 K++ systems: the streaming kernel (column chunks too wide for the small-block one)
    bool v4 = !f64 && !cd && variant >= 2 && !v2 && KP <= 8 && s >= 2 && s <= 256;
    if (v4) {
        const int64_t TK = stream_tk(dtype);
        for (int i = 0; v4 && i < nsys; ++i) {
            const kpp_matrix &Ai = *sys[i].A;
            if (((uintptr_t)Ai.data & 15) || ((Ai.ld * (int64_t)dtype_size(dtype)) & 15)) v4 = false;
        }
        if (A0.cols % TK) v4 = false;
        const int per_sm = v4 ? stream_per_sm(dtype, s, KP) : 0;
        // the column tiles are split evenly over the CTAs of a system (chunks differ by at most one tile)
        // and every chunk keeps stream_min_tiles() tiles: the kernel's prefetch runs that far ahead of
        // the X / M stores it depends on
        const int64_t T4 = A0.cols / TK, Gmax = T4 / stream_min_tiles();
        int64_t G4 = per_sm > 0 ? std::max(1, per_sm * sm_count() / nsys) : 0;
        if (grid > 0) {
            G4 = grid;
            if (G4 > Gmax) v4 = false;
        } else {
            G4 = std::min(G4, Gmax);
        }
        if (G4 < 1 || G4 * nsys > (int64_t)per_sm * sm_count()) v4 = false;
        if (v4) {
            G = (int)G4;
            CW = (T4 + G4 - 1) / G4 * TK;  // the widest chunk
        }
    }
    // large blocks of FP32/BF16 K++ with the W memo: one exchange per step (kpp_kw.cu)
    bool v6 = !f64 && !cd && k == 1 && variant >= 3 && (grid <= 0 || grid == kw_grid(A0.cols)) &&
              kw_fits(dtype, A0.rows, A0.cols, s, k, sm_count()) && nsys * kw_grid(A0.cols) <= sm_count();
    for (int i = 0; v6 && i < nsys; ++i) {
        const kpp_matrix &Ai = *sys[i].A;
        if (!sys[i].F->W32 || ((uintptr_t)Ai.data & 15) || ((Ai.ld * (int64_t)dtype_size(dtype)) & 15)) v6 = false;
    }
    if (v6) v6 = kw_can_launch(dtype, s, A0.cols, nsys);
    if (v6) {
        v2 = v3 = v4 = false;
        G = (int)kw_grid(A0.cols);
        CW = 32;
    }
    Common &cm = L.cm;
    cm = Common{};
    cm.rows = A0.rows;
    cm.cols = A0.cols;
    cm.s = s;
    cm.nb = nb;
    cm.k = k;
    cm.CW = CW;
    cm.G = G;
    cm.eta = eta;
    cm.tol = tol;
    cm.adaptive = adaptive;
    cm.confirm = confirm;
    cm.reduce_redundant = ((int64_t)G * s * KP <= 8192) ? 1 : 0;
    cm.init_residual = init_residual ? 1 : 0;
    cm.max_iters = max_iters;
    cm.seed = seed;
    cm.timeout_ns = g_wait_ns ? g_wait_ns : 2000000000ull;
    cm.t0_state = t0_state ? 1 : 0;
    cm.test_hold_cta = g_hold_cta;
    L.kind = v6 ? 6 : v4 ? 4 : v3 ? 3 : v2 ? 2 : 1;
    if (g_hold_cta >= 0 && (L.kind != 1 || g_hold_cta >= G)) {
        set_error("the wait test runs on the general kernel only (kernel variant 1), with a CTA index < %d", G);
        return KPP_ERR_UNSUPPORTED;
    }
    L.dtype = dtype;
    L.KP = KP;
    L.nsys = nsys;
    L.k = k;
    L.cd = cd;
    L.f64 = f64;
    L.init_residual = init_residual;
    L.t0 = t0;
    L.tcs = tcs;
    L.vec_n = (size_t)A0.cols * k;
    L.vec_r = (size_t)A0.rows * k;
    L.args.assign(nsys, SysArgs{});
    L.mails.assign(nsys, nullptr);

    const size_t smem = solve_smem_bytes(s, KP, CW, tcs);
    if (L.kind == 1 && smem > 220 * 1024) {
        set_error("shared memory %zu B exceeds the per-CTA limit (s=%d, k=%d, chunk=%lld)", smem, s, k, (long long)CW);
        return KPP_ERR_UNSUPPORTED;
    }
    std::vector<unsigned char> h2;
    CUDA_OR(scr.alloc((void **)&L.bars, nsys * sizeof(unsigned)), KPP_ERR_CUDA);
    CUDA_OR(scr.alloc((void **)&L.errs, nsys * sizeof(int)), KPP_ERR_CUDA);
    for (int i = 0; i < nsys; ++i) {
        SysArgs &a = L.args[i];
        a.A = sys[i].A->data;
        a.lda = sys[i].A->ld;
        a.b = sys[i].b;
        a.x = sys[i].x;
        a.Ginv = f64 ? (const void *)sys[i].F->Ginv : (const void *)sys[i].F->Ginv32;
        if (sys[i].m_ext) {
            if (L.kind != 1 || (cd && (!sys[i].Rx_ext || !sys[i].Rm_ext))) {
                set_error("a solve with a kept state runs on the general kernel (kernel variant 1)");
                return KPP_ERR_UNSUPPORTED;
            }
            L.keep_state = true;
            a.m = sys[i].m_ext;
        } else {
            CUDA_OR(scr.alloc(&a.m, L.vec_n * tcs), KPP_ERR_CUDA);
        }
        if (cd && sys[i].m_ext) {
            a.Rx = sys[i].Rx_ext;
            a.Rm = sys[i].Rm_ext;
        } else if (cd) {
            // v2 keeps two published copies of R_x (steps of even / odd index); v1 and v3 one
            CUDA_OR(scr.alloc(&a.Rx, (L.kind == 2 ? 2 : 1) * L.vec_r * tcs), KPP_ERR_CUDA);
            CUDA_OR(scr.alloc(&a.Rm, L.vec_r * tcs), KPP_ERR_CUDA);
        } else {
            a.Rx = a.Rm = nullptr;
        }
        CUDA_OR(scr.alloc(&a.part, (L.kind == 2 || L.kind == 4 ? 2 : 1) * (size_t)G * s * KP * tcs), KPP_ERR_CUDA);
        CUDA_OR(scr.alloc(&a.rbuf, (size_t)s * KP * tcs), KPP_ERR_CUDA);
        CUDA_OR(scr.alloc(&a.ybuf, (size_t)s * KP * tcs), KPP_ERR_CUDA);
        CUDA_OR(scr.alloc((void **)&a.rpart, (size_t)G * KP * sizeof(double)), KPP_ERR_CUDA);
        if (sys[i].sc_dev) {
            a.sc = sys[i].sc_dev;
        } else {
            CUDA_OR(scr.alloc((void **)&a.sc, (size_t)k * sizeof(SolveScalars)), KPP_ERR_CUDA);
            CUDA_OR(cudaMemcpyAsync(a.sc, sys[i].sc_host, (size_t)k * sizeof(SolveScalars), cudaMemcpyHostToDevice, st),
                    KPP_ERR_CUDA);
        }
        a.bar = L.bars + i;
        a.err = L.errs + i;
        a.sys_id = sys[i].sys_id;
        a.t0 = t0;
    }
    if (L.kind == 6) {
        const size_t sb = sysk_bytes();
        L.mail_bytes = kw_mail_bytes(s, G);
        h2.assign(sb * nsys, 0);
        const uint32_t box = (uint32_t)std::min(s, 256);
        for (int i = 0; i < nsys; ++i) {
            alignas(128) unsigned char tma[128], tmw[128];
            const kpp_matrix &Ai = *sys[i].A;
            CUDA_OR(scr.alloc(&L.mails[i], L.mail_bytes), KPP_ERR_CUDA);
            if (!make_tmap_2d(tma, Ai.data, dtype, Ai.cols, Ai.rows, Ai.ld, 32, box) ||
                !make_tmap_2d(tmw, sys[i].F->W32, KPP_F32, Ai.cols, Ai.rows, Ai.cols, 32, box)) {
                set_error("cuTensorMapEncodeTiled failed for system %d", i);
                return KPP_ERR_CUDA;
            }
            const SysArgs &a = L.args[i];
            sysk_fill(h2.data() + sb * i, tma, tmw, (const float *)a.b, (float *)a.x, a.sc, a.bar, a.err, a.rpart,
                      L.mails[i], a.sys_id, a.t0);
        }
    } else if (L.kind == 4) {
        const size_t sb = sys4_bytes();
        h2.assign(sb * nsys, 0);
        for (int i = 0; i < nsys; ++i) {
            alignas(128) unsigned char tm[128];
            const kpp_matrix &Ai = *sys[i].A;
            if (!make_tmap_2d(tm, Ai.data, dtype, Ai.cols, Ai.rows, Ai.ld, (uint32_t)stream_tk(dtype), (uint32_t)s, true)) {
                set_error("cuTensorMapEncodeTiled failed for system %d", i);
                return KPP_ERR_CUDA;
            }
            const SysArgs &a = L.args[i];
            sys4_fill(h2.data() + sb * i, tm, (const float *)a.b, (float *)a.x, (float *)a.m, (const float *)a.Ginv,
                      (float *)a.part, a.rpart, a.sc, a.bar, a.err, a.sys_id, a.t0);
        }
    } else if (L.kind == 3) {
        const size_t sb = sys3_bytes();
        L.mail_bytes = cd3_mail_bytes(s, KP, f64);
        h2.assign(sb * nsys, 0);
        // one right-hand side with a memo (W in FP64, W32 for FP32/BF16 storage): the single-column kernel
        bool c4 = k == 1 && KP == 1 && cd4_fits(s, CW, (int)tcs);
        for (int i = 0; c4 && i < nsys; ++i) c4 = f64 ? sys[i].F->W != nullptr : sys[i].F->W32 != nullptr;
        for (int i = 0; i < nsys; ++i) {
            alignas(128) unsigned char tm[128];
            const void *src = f64 ? (const void *)sys[i].F->W : (c4 ? (const void *)sys[i].F->W32 : sys[i].A->data);
            const int tdt = f64 ? KPP_F64 : (c4 ? KPP_F32 : dtype);
            const int64_t ld = (f64 || c4) ? sys[i].A->cols : sys[i].A->ld;
            CUDA_OR(scr.alloc(&L.mails[i], L.mail_bytes), KPP_ERR_CUDA);
            if (!make_tmap_2d(tm, src, tdt, sys[i].A->cols, sys[i].A->rows, ld, (uint32_t)CW, (uint32_t)s)) {
                set_error("cuTensorMapEncodeTiled failed for system %d", i);
                return KPP_ERR_CUDA;
            }
            sys3_fill(h2.data() + sb * i, L.args[i], tm, L.mails[i]);
        }
        if (c4) L.kind = 7;
    } else if (L.kind == 2) {
        const size_t sb = sys2_bytes();
        h2.assign(sb * nsys, 0);
        for (int i = 0; i < nsys; ++i) {
            alignas(128) unsigned char tm[128];
            if (!make_tmap_2d(tm, sys[i].A->data, dtype, sys[i].A->cols, sys[i].A->rows, sys[i].A->ld, (uint32_t)CW,
                              (uint32_t)std::min(s, 256))) {
                set_error("cuTensorMapEncodeTiled failed for system %d", i);
                return KPP_ERR_CUDA;
            }
            sys2_fill(h2.data() + sb * i, L.args[i], tm);
        }
    }
    if (L.kind >= 2) {
        CUDA_OR(scr.alloc(&L.d_sys2, h2.size()), KPP_ERR_CUDA);
        if ((uintptr_t)L.d_sys2 & 127) {  // tensor maps must be 64-byte aligned in memory
            set_error("descriptor buffer not 128-byte aligned");
            return KPP_ERR_CUDA;
        }
        CUDA_OR(cudaMemcpyAsync(L.d_sys2, h2.data(), h2.size(), cudaMemcpyHostToDevice, st), KPP_ERR_CUDA);
        CUDA_OR(cudaStreamSynchronize(st), KPP_ERR_CUDA);  // h2 is pageable and local
    } else {
        CUDA_OR(scr.alloc((void **)&L.d_args, nsys * sizeof(SysArgs)), KPP_ERR_CUDA);
        CUDA_OR(cudaMemcpyAsync(L.d_args, L.args.data(), nsys * sizeof(SysArgs), cudaMemcpyHostToDevice, st),
                KPP_ERR_CUDA);
        CUDA_OR(cudaStreamSynchronize(st), KPP_ERR_CUDA);
    }
cleanup:
    return rc;
}

// Reset the per-launch state and launch the kernel (graph-capturable).
kpp_status enqueue_persistent(const PersistentLaunch &L, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1) {
    kpp_status rc = KPP_OK;
    CUDA_OR(cudaMemsetAsync(L.bars, 0, L.nsys * sizeof(unsigned), st), KPP_ERR_CUDA);
    CUDA_OR(cudaMemsetAsync(L.errs, 0, L.nsys * sizeof(int), st), KPP_ERR_CUDA);
    for (int i = 0; i < L.nsys; ++i) {
        const SysArgs &a = L.args[i];
        if (L.keep_state) continue;  // the caller's state carries m, R_x and R_m over from the last launch
        CUDA_OR(cudaMemsetAsync(a.m, 0, L.vec_n * L.tcs, st), KPP_ERR_CUDA);
        if (L.cd) {
            CUDA_OR(cudaMemsetAsync(a.Rm, 0, L.vec_r * L.tcs, st), KPP_ERR_CUDA);
            if (!L.init_residual) {  // x0 = 0: R_x = -b (in the copy the first step reads)
                if (L.kind == 2 && L.cm.t0_state) {
                    // the first step is only known on the device: fill both published copies
                    CUDA_OR(launch_negate_copy(L.vec_r, a.b, a.Rx, L.f64, st), KPP_ERR_CUDA);
                    CUDA_OR(launch_negate_copy(L.vec_r, a.b, (char *)a.Rx + L.vec_r * L.tcs, L.f64, st), KPP_ERR_CUDA);
                } else {
                    void *dst = (L.kind == 2 && (L.t0 & 1)) ? (void *)((char *)a.Rx + L.vec_r * L.tcs) : a.Rx;
                    CUDA_OR(launch_negate_copy(L.vec_r, a.b, dst, L.f64, st), KPP_ERR_CUDA);
                }
            }
        }
        if (L.kind == 3 || L.kind == 6 || L.kind == 7)
            CUDA_OR(cudaMemsetAsync(L.mails[i], 0, L.mail_bytes, st), KPP_ERR_CUDA);
    }
    if (ev0) CUDA_OR(cudaEventRecord(ev0, st), KPP_ERR_CUDA);
    {
        cudaError_t le = L.kind == 7   ? launch_cd4(L.dtype, L.d_sys2, L.nsys, L.cm, st)
                         : L.kind == 6 ? launch_kw(L.dtype, L.d_sys2, L.nsys, L.cm, st)
                         : L.kind == 4 ? launch_stream(L.dtype, L.d_sys2, L.nsys, L.cm, L.KP, st)
                         : L.kind == 3 ? launch_cd3(L.dtype, L.d_sys2, L.nsys, L.cm, L.KP, st)
                         : L.kind == 2 ? launch_solve2(L.dtype, L.cd, L.d_sys2, L.nsys, L.cm, L.KP, st)
                                       : launch_solve(L.dtype, L.f64, L.cd, L.d_args, L.nsys, L.cm, L.KP, st);
        if (le == cudaErrorCooperativeLaunchTooLarge) {
            set_error("%d systems x %d CTAs do not fit co-resident on this GPU", L.nsys, L.cm.G);
            return KPP_ERR_UNSUPPORTED;
        }
        CUDA_OR(le, KPP_ERR_CUDA);
    }
    if (ev1) CUDA_OR(cudaEventRecord(ev1, st), KPP_ERR_CUDA);
cleanup:
    return rc;
}

// Run the persistent kernel over nsys systems that share shape, dtype, s and k (one shot).
kpp_status run_persistent(std::vector<SysInput> &sys, int dtype, bool cd, int k, int s, double eta,
                                 double tol, int adaptive, int confirm, int64_t max_iters, uint64_t seed, int grid,
                                 bool init_residual, int64_t t0, cudaStream_t st, float *ms_out, int *err_out,
                                 int variant, int *kind_out, int *G_out) {
    kpp_status rc = KPP_OK;
    const int nsys = (int)sys.size();
    Scratch scr(st);
    PersistentLaunch L;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<int> herr(nsys, 0);
    rc = prepare_persistent(L, sys, dtype, cd, k, s, eta, tol, adaptive, confirm, max_iters, seed, grid,
                            init_residual, t0, false, variant < 0 ? g_variant : variant, scr, st);
    if (rc != KPP_OK) return rc;
    if (kind_out) *kind_out = L.kind;
    if (G_out) *G_out = L.cm.G;
    CUDA_OR(cudaEventCreate(&e0), KPP_ERR_CUDA);
    CUDA_OR(cudaEventCreate(&e1), KPP_ERR_CUDA);
    rc = enqueue_persistent(L, st, e0, e1);  // events around the kernel launch itself
    if (rc != KPP_OK) goto cleanup;
    for (int i = 0; i < nsys; ++i)
        CUDA_OR(cudaMemcpyAsync(sys[i].sc_host, L.args[i].sc, (size_t)k * sizeof(SolveScalars), cudaMemcpyDeviceToHost, st),
                KPP_ERR_CUDA);
    CUDA_OR(cudaMemcpyAsync(herr.data(), L.errs, nsys * sizeof(int), cudaMemcpyDeviceToHost, st), KPP_ERR_CUDA);
    CUDA_OR(cudaStreamSynchronize(st), KPP_ERR_CUDA);
    if (ms_out) cudaEventElapsedTime(ms_out, e0, e1);
    for (int i = 0; i < nsys; ++i) {
        err_out[i] = herr[i];
        if (herr[i]) {
            set_error("system %d: device error %d (%s)", i, herr[i], kpp_status_string((kpp_status)herr[i]));
            if (rc == KPP_OK) rc = (kpp_status)herr[i];
        }
    }
cleanup:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

void init_scalars(std::vector<SolveScalars> &sc, int k, double rho0) {
    sc.assign(k, SolveScalars{});
    for (int c = 0; c < k; ++c) {
        sc[c].rho = rho0;
        sc[c].active = 1;
        sc[c].status = KPP_ERR_NO_CONVERGENCE;
        sc[c].res_est = NAN;
    }
}

double default_eta(const kpp_params &p, int s, int64_t rows, int64_t cols) {
    if (!std::isnan(p.eta)) return p.eta;
    return (double)s / (2.0 * (double)std::min(rows, cols));
}

static kpp_status worse(kpp_status a, kpp_status b) { return a != KPP_OK ? a : b; }

kpp_status validate_systems(int nsys, const kpp_matrix *A, const double *const *B, double *const *X, int k,
                            kpp_partition_t P, const kpp_factors_t *F, const kpp_params *pp, bool cd) {
    if (nsys < 1 || !A || !B || !X || !P || !F || !pp || k < 1 || k > 32) {
        set_error("invalid argument (nsys=%d, k=%d)", nsys, k);
        return KPP_ERR_ARG;
    }
    const kpp_params p = *pp;
    const int s = P->s;
    for (int i = 0; i < nsys; ++i) {
        if (!matrix_ok(&A[i]) || !B[i] || !X[i] || !F[i]) {
            set_error("system %d: null or malformed argument", i);
            return KPP_ERR_ARG;
        }
        if (A[i].rows != P->rows || A[i].rows != A[0].rows || A[i].cols != A[0].cols || A[i].dtype != A[0].dtype) {
            set_error("system %d: shape/dtype differs from the partition or from system 0", i);
            return KPP_ERR_ARG;
        }
        const FactorSet &f = F[i]->f;
        if (f.rows != A[i].rows || f.s != s || f.mode != (cd ? 1 : 0) || f.dtype != A[i].dtype || f.bad_block >= 0 ||
            std::fabs(f.lambda - p.lambda) > 1e-15 * std::max(1.0, std::fabs(p.lambda))) {
            set_error("system %d: factors do not match (mode, s, dtype, lambda or a failed block)", i);
            return KPP_ERR_ARG;
        }
        if (cd && A[i].rows != A[i].cols) {
            set_error("CD++ needs a square matrix");
            return KPP_ERR_ARG;
        }
    }
    return KPP_OK;
}

// The solve of `nsys` systems with k right-hand sides each (FP64 b/x on the device).
kpp_status solve_systems(int nsys, const kpp_matrix *A, const double *const *B, double *const *X, int k,
                                kpp_partition_t P, const kpp_factors_t *F, const kpp_params *pp, kpp_report *reps,
                                cudaStream_t st, bool cd) {
    clear_error();
    {
        kpp_status v = validate_systems(nsys, A, B, X, k, P, F, pp, cd);
        if (v != KPP_OK) return v;
    }
    const kpp_params p = *pp;
    const int s = P->s;
    const int dtype = A[0].dtype;
    const int64_t rows = A[0].rows, cols = A[0].cols;
    const double eta = default_eta(p, s, rows, cols);
    kpp_status rc = KPP_OK;
    // launch shape: the caller's grid, the heuristic (0), or the autotuner (negative)
    TuneChoice tune;
    tune.grid = p.grid;
    if (p.grid < 0) {
        kpp_status tr = tune_launch(nsys, A, B, k, P, F, p, cd, st, tune);
        if (tr != KPP_OK) return tr;
    }
    std::vector<std::vector<SolveScalars>> sc(nsys);
    std::vector<int> errs(nsys, 0);
    std::vector<SysInput> in(nsys);
    std::vector<double> dev_ms(nsys, 0.0);
    std::vector<int64_t> iters(nsys, 0), outer(nsys, 0), nlaunch(nsys, 0);
    std::vector<double> kern_ms(nsys, 0.0);
    for (int i = 0; i < nsys; ++i) init_scalars(sc[i], k, p.rho0);
    float ms = 0.f;
    // refinement: the last outer check already holds |r|^2 and |b|^2 of the returned x
    std::vector<std::vector<double>> bn2(nsys), res2(nsys);
    bool have_final = false;

    if (dtype == KPP_F64) {
        // plain FP64 path: the kernel iterates directly on the caller's b and x
        for (int i = 0; i < nsys; ++i) in[i] = SysInput{&A[i], B[i], X[i], &F[i]->f, p.sys_id + (uint32_t)i, sc[i].data()};
        rc = run_persistent(in, dtype, cd, k, s, eta, p.tol, p.adaptive_rho, 1, p.max_iters, p.seed, tune.grid,
                            /*init_residual=*/true, 0, st, &ms, errs.data(), tune.variant);
        for (int i = 0; i < nsys; ++i) {
            dev_ms[i] = ms;
            kern_ms[i] = ms;
            nlaunch[i] = 1;
            iters[i] = sc[i][0].t;
        }
    } else {
        // FP32 / BF16 storage: FP32 iterations, FP64 outer refinement (or a single FP32 solve)
        Scratch scr(st);
        std::vector<float *> b32(nsys), d32(nsys);
        std::vector<int> done(nsys, 0);
        const size_t nr = (size_t)rows * k, nc = (size_t)cols * k;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        int64_t t_global = 0;
        CUDA_OR(cudaEventCreate(&e0), KPP_ERR_CUDA);
        CUDA_OR(cudaEventCreate(&e1), KPP_ERR_CUDA);
        CUDA_OR(cudaEventRecord(e0, st), KPP_ERR_CUDA);
        for (int i = 0; i < nsys; ++i) {
            CUDA_OR(scr.alloc((void **)&b32[i], nr * sizeof(float)), KPP_ERR_CUDA);
            CUDA_OR(scr.alloc((void **)&d32[i], nc * sizeof(float)), KPP_ERR_CUDA);
        }
        if (!p.refine) {
            for (int i = 0; i < nsys; ++i) {
                CUDA_OR(launch_f64_to_f32(nr, B[i], b32[i], st), KPP_ERR_CUDA);
                CUDA_OR(launch_f64_to_f32(nc, X[i], d32[i], st), KPP_ERR_CUDA);
                in[i] = SysInput{&A[i], b32[i], d32[i], &F[i]->f, p.sys_id + (uint32_t)i, sc[i].data()};
            }
            float kms = 0.f;
            rc = run_persistent(in, dtype, cd, k, s, eta, p.tol, p.adaptive_rho, 0, p.max_iters, p.seed, tune.grid,
                                true, 0, st, &kms, errs.data(), tune.variant);
            for (int i = 0; i < nsys; ++i) {
                kern_ms[i] = kms;
                nlaunch[i] = 1;
                // x = double(x32): overwrite through the axpy of (x32 - x) is not exact; copy via zero + axpy
                CUDA_OR(cudaMemsetAsync(X[i], 0, nc * sizeof(double), st), KPP_ERR_CUDA);
                CUDA_OR(launch_axpy(nc, d32[i], X[i], st), KPP_ERR_CUDA);
                iters[i] = sc[i][0].t;
            }
        } else {
            for (int outer_it = 0; outer_it <= p.max_outer; ++outer_it) {
                // r = b - A x in FP64 (rounded copy to FP32 as the inner right-hand side)
                bool any = false;
                for (int i = 0; i < nsys; ++i) {
                    if (done[i]) continue;
                    kpp_status r2 = residual_norms(A[i], k, B[i], X[i], b32[i], res2[i], outer_it == 0 ? &bn2[i] : nullptr, st);
                    if (r2 != KPP_OK) {
                        rc = r2;
                        goto cleanup;
                    }
                    int active = 0;
                    for (int c = 0; c < k; ++c) {
                        const double rel = bn2[i][c] > 0 ? std::sqrt(res2[i][c] / bn2[i][c]) : std::sqrt(res2[i][c]);
                        const bool conv = rel <= p.tol;
                        sc[i][c].active = conv ? 0 : 1;
                        sc[i][c].status = conv ? KPP_OK : KPP_ERR_NO_CONVERGENCE;
                        sc[i][c].E0 = sc[i][c].E1 = 0.0;
                        active += !conv;
                    }
                    if (!active) done[i] = 1;
                    else any = true;
                }
                if (!any || outer_it == p.max_outer) {
                    have_final = true;
                    break;
                }
                // inner FP32 solve of A d = r from d = 0 (momentum restarts, rho carries over)
                std::vector<SysInput> act;
                std::vector<int> idx;
                for (int i = 0; i < nsys; ++i) {
                    if (done[i]) continue;
                    CUDA_OR(cudaMemsetAsync(d32[i], 0, nc * sizeof(float), st), KPP_ERR_CUDA);
                    act.push_back(SysInput{&A[i], b32[i], d32[i], &F[i]->f, p.sys_id + (uint32_t)i, sc[i].data()});
                    idx.push_back(i);
                    outer[i] += 1;
                }
                std::vector<int> e2(act.size(), 0);
                float kms = 0.f;
                kpp_status ri = run_persistent(act, dtype, cd, k, s, eta, p.inner_tol, p.adaptive_rho, 0,
                                               t_global + p.max_iters, p.seed, tune.grid, false, t_global, st, &kms,
                                               e2.data(), tune.variant);
                int64_t tmax = t_global;
                for (size_t q = 0; q < act.size(); ++q) {
                    const int i = idx[q];
                    errs[i] = e2[q];
                    kern_ms[i] += kms;
                    nlaunch[i] += 1;
                    iters[i] += sc[i][0].t - t_global;
                    tmax = std::max<int64_t>(tmax, sc[i][0].t);
                    CUDA_OR(launch_axpy(nc, d32[i], X[i], st), KPP_ERR_CUDA);
                }
                // keep the Philox counter moving so that inner solves do not replay one block sequence
                t_global = tmax;
                if (ri != KPP_OK && ri != KPP_ERR_NO_CONVERGENCE) {
                    rc = ri;
                    goto cleanup;
                }
            }
        }
        CUDA_OR(cudaEventRecord(e1, st), KPP_ERR_CUDA);
        CUDA_OR(cudaEventSynchronize(e1), KPP_ERR_CUDA);
        cudaEventElapsedTime(&ms, e0, e1);
        for (int i = 0; i < nsys; ++i) dev_ms[i] = ms;
    cleanup:
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (rc != KPP_OK && rc != KPP_ERR_NO_CONVERGENCE) return rc;
    }
    if (rc != KPP_OK && rc != KPP_ERR_NO_CONVERGENCE && rc != KPP_ERR_TIMEOUT && rc != KPP_ERR_NUMERIC) return rc;

    // final report: true FP64 residual of every column
    kpp_status worst = rc;
    for (int i = 0; i < nsys; ++i) {
        std::vector<double> r2, b2;
        if (have_final) {
            r2 = res2[i];
            b2 = bn2[i];
        } else {
            kpp_status r3 = residual_norms(A[i], k, B[i], X[i], nullptr, r2, &b2, st);
            if (r3 != KPP_OK) return r3;
        }
        for (int c = 0; c < k; ++c) {
            const double rel = b2[c] > 0 ? std::sqrt(r2[c] / b2[c]) : std::sqrt(r2[c]);
            kpp_status cs = (kpp_status)sc[i][c].status;
            if (errs[i]) cs = (kpp_status)errs[i];
            else if (!std::isfinite(rel)) cs = KPP_ERR_NUMERIC;
            else if (dtype != KPP_F64 && p.refine) cs = rel <= p.tol ? KPP_OK : KPP_ERR_NO_CONVERGENCE;
            worst = worse(worst, cs);
            if (reps) {
                kpp_report &r = reps[(size_t)i * k + c];
                memset(&r, 0, sizeof(r));
                r.iters = iters[i];
                r.outer = outer[i];
                r.rel_res_true = rel;
                r.rel_res_est = sc[i][c].res_est;
                r.rho_final = sc[i][c].rho;
                r.status = cs;
                r.bad_block = -1;
                r.device_ms = dev_ms[i];
                r.kernel_ms = kern_ms[i];
                r.launches = nlaunch[i];
            }
        }
    }
    if (worst != KPP_OK && g_last_error.empty()) set_error("solve ended with %s", kpp_status_string(worst));
    return worst;
}

kpp_status solve_systems_internal(int nsys, const kpp_matrix *A, const double *const *B, double *const *X, int k,
                                  kpp_partition_t P, const kpp_factors_t *F, const kpp_params *p, kpp_report *reps,
                                  cudaStream_t st, bool cd) {
    return solve_systems(nsys, A, B, X, k, P, F, p, reps, st, cd);
}

}  // namespace kpp

using namespace kpp;

extern "C" {

kpp_params kpp_params_default(void) {
    kpp_params p;
    memset(&p, 0, sizeof(p));
    p.lambda = 0.0;
    p.tol = 1e-8;
    p.max_iters = 1000000;
    p.seed = 0;
    p.sys_id = 0;
    p.adaptive_rho = 1;
    p.rho0 = 0.0;
    p.eta = NAN;
    p.grid = 0;
    p.refine = 0;
    p.max_outer = 20;
    p.inner_tol = 1e-3;
    return p;
}

const char *kpp_status_string(kpp_status st) {
    switch (st) {
        case KPP_OK: return "KPP_OK";
        case KPP_ERR_ARG: return "KPP_ERR_ARG";
        case KPP_ERR_CUDA: return "KPP_ERR_CUDA";
        case KPP_ERR_OOM: return "KPP_ERR_OOM";
        case KPP_ERR_NOT_SPD: return "KPP_ERR_NOT_SPD";
        case KPP_ERR_NUMERIC: return "KPP_ERR_NUMERIC";
        case KPP_ERR_NO_CONVERGENCE: return "KPP_ERR_NO_CONVERGENCE";
        case KPP_ERR_TIMEOUT: return "KPP_ERR_TIMEOUT";
        case KPP_ERR_BUDGET: return "KPP_ERR_BUDGET";
        case KPP_ERR_UNSUPPORTED: return "KPP_ERR_UNSUPPORTED";
    }
    return "KPP_ERR_UNKNOWN";
}

const char *kpp_last_error(void) { return g_last_error.c_str(); }

#define KPP_STR2(x) #x
#define KPP_STR(x) KPP_STR2(x)
uint64_t kpp_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }
uint64_t kpp_device_alloc_count(void) { return dev_alloc_requests(); }

const char *kpp_build_info(void) {
    return "sm_103a; nvcc " KPP_STR(__CUDACC_VER_MAJOR__) "." KPP_STR(__CUDACC_VER_MINOR__) "; " __DATE__;
}

kpp_status kpp_partition(int64_t rows, int32_t s, kpp_partition_t *out) {
    clear_error();
    if (!out || rows < 1 || s < 1 || s > 1024) {
        set_error("kpp_partition: rows=%lld s=%d", (long long)rows, s);
        return KPP_ERR_ARG;
    }
    kpp_partition_t p = new kpp_partition_s;
    p->rows = rows;
    p->s = s;
    p->nb = (rows + s - 1) / s;
    *out = p;
    return KPP_OK;
}

void kpp_partition_destroy(kpp_partition_t p) { delete p; }

int64_t kpp_partition_blocks(kpp_partition_t p) { return p ? p->nb : 0; }

kpp_status kpp_factor_blocks(const kpp_matrix *A, kpp_partition_t P, double lambda, int32_t mode, kpp_factors_t *out,
                             void *stream) {
    clear_error();
    if (!out || !P || !matrix_ok(A) || (mode != 0 && mode != 1) || !(lambda >= 0.0) || A->rows != P->rows ||
        (mode == 1 && A->rows != A->cols)) {
        set_error("kpp_factor_blocks: invalid argument");
        return KPP_ERR_ARG;
    }
    kpp_factors_t f = new kpp_factors_s;
    kpp_status rc = factor_blocks_impl(*A, P->s, lambda, mode, f->f, (cudaStream_t)stream);
    if (rc != KPP_OK && rc != KPP_ERR_NOT_SPD) {
        f->f.release();
        delete f;
        *out = nullptr;
        return rc;
    }
    *out = f;
    return rc;
}

void kpp_factors_destroy(kpp_factors_t f) {
    if (!f) return;
    f->f.release();
    delete f;
}

int64_t kpp_factors_bad_block(kpp_factors_t f) { return f ? f->f.bad_block : -1; }
int64_t kpp_factors_fp64_blocks(kpp_factors_t f) { return f ? f->f.fp64_blocks : -1; }

kpp_status kpp_factors_get_memo(kpp_factors_t f, int64_t row0, int64_t nrows, float *out_host) {
    clear_error();
    if (!f || !out_host || !f->f.W32 || row0 < 0 || nrows < 0 || row0 + nrows > f->f.rows) {
        set_error("kpp_factors_get_memo: no FP32 memo in these factors, or rows out of range");
        return KPP_ERR_ARG;
    }
    const int64_t cols = f->f.memo_cols;
    cudaError_t e = cudaMemcpy(out_host, f->f.W32 + row0 * cols, (size_t)nrows * cols * sizeof(float),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_error("cudaMemcpy: %s", cudaGetErrorString(e));
        return KPP_ERR_CUDA;
    }
    return KPP_OK;
}

kpp_status kpp_factors_stage_ms(kpp_factors_t f, double *ms_out) {
    clear_error();
    if (!f || !ms_out) {
        set_error("kpp_factors_stage_ms: null argument");
        return KPP_ERR_ARG;
    }
    for (int i = 0; i < 4; ++i) {
        ms_out[i] = NAN;
        float ms = 0.f;
        const cudaEvent_t a = f->f.ev[i], b = f->f.ev[i + 1];
        if (a && b && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
            ms_out[i] = ms;
    }
    cudaGetLastError();
    return KPP_OK;
}

kpp_status kpp_factors_get_block(kpp_factors_t f, int64_t j, double *out_host) {
    clear_error();
    if (!f || !out_host || j < 0 || j >= f->f.nb) {
        set_error("kpp_factors_get_block: bad handle or block index");
        return KPP_ERR_ARG;
    }
    const int64_t len = std::min<int64_t>(f->f.s, f->f.rows - j * f->f.s);
    cudaError_t e = cudaMemcpy(out_host, f->f.L + (size_t)j * f->f.s * f->f.s, (size_t)len * len * sizeof(double),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_error("cudaMemcpy: %s", cudaGetErrorString(e));
        return KPP_ERR_CUDA;
    }
    return KPP_OK;
}

kpp_status kpp_solve(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P, kpp_factors_t F,
                     const kpp_params *p, kpp_report *rep, void *stream) {
    const double *B[1] = {b};
    double *X[1] = {x};
    return solve_systems(1, A, B, X, 1, P, &F, p, rep, (cudaStream_t)stream, false);
}

kpp_status cdpp_solve(const kpp_matrix *A, const double *b, double *x, kpp_partition_t P, kpp_factors_t F,
                      const kpp_params *p, kpp_report *rep, void *stream) {
    const double *B[1] = {b};
    double *X[1] = {x};
    return solve_systems(1, A, B, X, 1, P, &F, p, rep, (cudaStream_t)stream, true);
}

kpp_status kpp_solve_batched(int32_t nsys, const kpp_matrix *A, const double *const *B, double *const *X, int32_t k,
                             kpp_partition_t P, const kpp_factors_t *F, const kpp_params *p, kpp_report *reps,
                             void *stream) {
    return solve_systems(nsys, A, B, X, k, P, F, p, reps, (cudaStream_t)stream, false);
}

kpp_status kpp_sample_blocks(uint64_t seed, uint32_t sys_id, int64_t t0, int64_t count, int32_t nb, int32_t *out,
                             void *stream) {
    clear_error();
    if (count < 0 || nb < 1 || (count > 0 && !out)) {
        set_error("kpp_sample_blocks: invalid argument");
        return KPP_ERR_ARG;
    }
    cudaError_t e = launch_sample_blocks(seed, sys_id, t0, count, nb, out, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error("sample kernel: %s", cudaGetErrorString(e));
        return KPP_ERR_CUDA;
    }
    return KPP_OK;
}

kpp_status kpp_set_wait_test(uint64_t wait_ns, int32_t hold_cta) {
    clear_error();
    if (hold_cta < -1) {
        set_error("kpp_set_wait_test: hold_cta must be -1 or a CTA index");
        return KPP_ERR_ARG;
    }
    g_wait_ns = wait_ns;
    g_hold_cta = hold_cta;
    return KPP_OK;
}

kpp_status kpp_set_kernel_variant(int32_t variant) {
    clear_error();
    if (variant < 1 || variant > 3) {
        set_error("kpp_set_kernel_variant: variant must be 1, 2 or 3");
        return KPP_ERR_ARG;
    }
    g_variant = variant;
    return KPP_OK;
}

kpp_status kpp_block_gram(const kpp_matrix *A, int32_t s, double lambda, int32_t engine, double *G_out,
                          int32_t *engine_used, void *stream) {
    clear_error();
    if (!matrix_ok(A) || s < 1 || s > 1024 || !G_out || engine < 0 || engine > 3) {
        set_error("kpp_block_gram: invalid argument");
        return KPP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int used = block_gram(*A, s, lambda, G_out, engine, st);
    if (engine_used) *engine_used = used;
    if (used < 0) {
        if (engine == 2 || engine == 3) {
            set_error("kpp_block_gram: the tensor-core Gram does not support this matrix (dtype, alignment)");
            return KPP_ERR_UNSUPPORTED;
        }
        set_error("kpp_block_gram: launch failed");
        return KPP_ERR_CUDA;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("kpp_block_gram: %s", cudaGetErrorString(e));
        return KPP_ERR_CUDA;
    }
    return KPP_OK;
}

kpp_status cdpp_solve_batched(int32_t nsys, const kpp_matrix *A, const double *const *B, double *const *X, int32_t k,
                              kpp_partition_t P, const kpp_factors_t *F, const kpp_params *p, kpp_report *reps,
                              void *stream) {
    return solve_systems(nsys, A, B, X, k, P, F, p, reps, (cudaStream_t)stream, true);
}

kpp_status kpp_rel_residual(const kpp_matrix *A, const double *b, const double *x, double *out_host, void *stream) {
    clear_error();
    if (!matrix_ok(A) || !b || !x || !out_host) {
        set_error("kpp_rel_residual: invalid argument");
        return KPP_ERR_ARG;
    }
    std::vector<double> r2, b2;
    kpp_status rc = residual_norms(*A, 1, b, x, nullptr, r2, &b2, (cudaStream_t)stream);
    if (rc != KPP_OK) return rc;
    *out_host = b2[0] > 0 ? std::sqrt(r2[0] / b2[0]) : std::sqrt(r2[0]);
    return KPP_OK;
}

kpp_status kpp_solve_host(const kpp_matrix *A_host, const double *b_host, double *x_host, int32_t s, int32_t mode,
                          const kpp_params *p, kpp_report *rep, void *stream) {
    clear_error();
    if (!matrix_ok(A_host) || !b_host || !x_host || !p || (mode != 0 && mode != 1)) {
        set_error("kpp_solve_host: invalid argument");
        return KPP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    kpp_status rc = KPP_OK;
    const size_t es = dtype_size(A_host->dtype);
    const size_t abytes = (size_t)A_host->rows * A_host->cols * es;
    void *dA = nullptr;
    double *db = nullptr, *dx = nullptr;
    kpp_partition_t P = nullptr;
    kpp_factors_t F = nullptr;
    kpp_matrix Ad = *A_host;
    CUDA_OR(dev_malloc(&dA, abytes), KPP_ERR_CUDA);
    CUDA_OR(dev_malloc((void **)&db, A_host->rows * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(dev_malloc((void **)&dx, A_host->cols * sizeof(double)), KPP_ERR_CUDA);
    CUDA_OR(cudaMemcpy2DAsync(dA, A_host->cols * es, A_host->data, A_host->ld * es, A_host->cols * es, A_host->rows,
                              cudaMemcpyHostToDevice, st),
            KPP_ERR_CUDA);
    CUDA_OR(cudaMemcpyAsync(db, b_host, A_host->rows * sizeof(double), cudaMemcpyHostToDevice, st), KPP_ERR_CUDA);
    CUDA_OR(cudaMemcpyAsync(dx, x_host, A_host->cols * sizeof(double), cudaMemcpyHostToDevice, st), KPP_ERR_CUDA);
    Ad.data = dA;
    Ad.ld = A_host->cols;
    rc = kpp_partition(A_host->rows, s, &P);
    if (rc != KPP_OK) goto cleanup;
    rc = kpp_factor_blocks(&Ad, P, p->lambda, mode, &F, stream);
    if (rc != KPP_OK) goto cleanup;
    rc = mode == 0 ? kpp_solve(&Ad, db, dx, P, F, p, rep, stream) : cdpp_solve(&Ad, db, dx, P, F, p, rep, stream);
    {
        cudaError_t e = cudaMemcpyAsync(x_host, dx, A_host->cols * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess && rc == KPP_OK) {
            set_error("copy back: %s", cudaGetErrorString(e));
            rc = KPP_ERR_CUDA;
        }
    }
cleanup:
    if (F) kpp_factors_destroy(F);
    if (P) kpp_partition_destroy(P);
    dev_free(dA);
    dev_free(db);
    dev_free(dx);
    return rc;
}

}  // extern "C"
