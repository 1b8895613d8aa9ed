// kpp_serve.h -- the device-resident request loop behind kpp_server_* (host and device view).
//
// A persistent cooperative kernel runs slots of G CTAs.  Each slot claims the next published job from a
// ring in mapped host memory, runs its whole solve (the FP64 refinement loop of the mixed-precision form
// around FP32 CD++ / K++ inner solves, or one FP64 solve) with the slot's CTAs only, writes a completion
// record back to mapped host memory and claims the next job.  The host side publishes jobs and reads
// completions; it never launches per-request kernels.
#pragma once

#include <stdint.h>

#include "kpp_solve.h"

namespace kpp {

constexpr int SERVE_KP = 8;  // right-hand-side columns per job (a request of k > 8 is split)

struct ServeJob {
    SysArgs sa;            // the solve's buffers: b, x are the inner system (FP32) or B, X (FP64 storage)
    Common cm;             // its shape and parameters (cm.G = the slot's CTAs)
    const double *B;       // rows x k FP64 right-hand sides (device)
    double *X;             // cols x k FP64 solution (device), zero on entry
    double tol;            // outer tolerance on |A x - b| / |b| (FP64)
    int32_t max_outer;     // refinement steps at most (mixed storage)
    int32_t dtype;         // storage type of A
    int32_t mode;          // 0 K++, 1 CD++
    int32_t pad;
    int64_t id;            // job number (ring entry id % R)
};

struct ServeDone {         // written by the device into mapped host memory
    int32_t state;         // 0 pending, 1 done (written last, with release semantics)
    int32_t status;        // kpp_status of the job
    int32_t outer;         // refinement steps taken
    int32_t pad;
    int64_t iters;         // block iterations (all inner solves, the panel's step count)
    double rel_res[SERVE_KP];
    double rho[SERVE_KP];
    int32_t col_status[SERVE_KP];
};

struct ServeCtl {          // mapped host memory, written by the host
    int64_t published;     // jobs [0, published) are in the ring
    int32_t drain;         // 1: slots exit once no published job is left unclaimed
    int32_t pad;
};

struct ServeSlot {         // device memory, one per slot, zeroed before each launch
    unsigned bar;
    int err;
    long long job;
    long long pad;
};

struct ServeArgs {
    const ServeJob *jobs;  // ring of R entries (device pointer to mapped host memory)
    ServeDone *done;       // ring of R entries (likewise)
    const ServeCtl *ctl;
    ServeSlot *slots;
    unsigned long long *claimed;  // jobs claimed so far (device memory; carried across launches)
    int R;
    int G;
    uint64_t idle_ns;      // a slot that finds no job for this long exits (the host relaunches on demand)
    uint64_t timeout_ns;   // group barrier limit
};

// Dynamic shared memory the kernel needs for jobs up to block size s and column chunk CW.
size_t serve_smem_bytes(int s, int64_t CW);
// CTAs of the launch (slots x G) that fit at once for that shared memory; 0 if none.
int serve_max_ctas(size_t smem);
cudaError_t launch_serve(const ServeArgs &a, int nslots, size_t smem, cudaStream_t st);

}  // namespace kpp
