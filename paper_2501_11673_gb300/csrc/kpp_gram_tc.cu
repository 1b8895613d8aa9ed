// kpp_gram_tc.cu -- block Gram G_j = A_{S_j} A_{S_j}^T + lam I on the tcgen05 tensor cores (Sec. 4:
// the memoised factor of K++ is chol(A_S A_S^T + lam I); Alg. 1).
//
// FP32 / BF16 storage only (kind::tf32 / kind::f16, FP32 accumulation in tensor memory); the result is
// widened to FP64 for the FP64 Cholesky.  One CTA computes one 128 x 256 tile of one block's Gram:
//   * warp 0, one thread: TMA producer -- K-major tiles of the block rows (128-byte swizzle) into a
//     4-stage shared-memory ring, one mbarrier per stage for "full" and one for "empty";
//   * warp 1, one thread: MMA issuer -- tcgen05.mma (M=128, N=256, K=16 bf16 / K=8 tf32) into 256 TMEM
//     columns; tcgen05.commit frees a stage when its MMAs are done, and signals the epilogue at the end;
//   * warps 0-3: epilogue -- tcgen05.ld of their 32 TMEM lanes, + lam on the diagonal, FP64 stores of
//     the lower triangle (all the Cholesky reads).
// Only tiles that touch the lower triangle of G are launched.  No cluster, no multicast: each CTA loads
// its own tiles.  Every wait is bounded; a wait that runs out sets the error word and the CTA winds
// down (it still waits, bounded, for its MMAs before releasing tensor memory).
#include <cuda.h>

#include <cstdio>
#include <cstdlib>
#include <vector>

#include "kpp_internal.cuh"
#include "kpp_runtime.h"
#include "kpp_solve.h"
#include "kpp_tc.cuh"

namespace kpp {

constexpr int TC_STAGES = 4;
constexpr int TC_ROWB = 128;                               // bytes of K per tile row (one swizzle atom row)
constexpr int TC_ABYTES = TC_M * TC_ROWB;                  // 16 KiB
constexpr int TC_BBYTES = TC_N * TC_ROWB;                  // 32 KiB
constexpr int TC_STAGE_BYTES = TC_ABYTES + TC_BBYTES;      // 48 KiB
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024; // + alignment slack
constexpr uint64_t TC_TIMEOUT_NS = 2000000000ull;

struct GramTile {
    int j, ta, tc;
};

// round an FP32 value to the nearest TF32 (10 explicit mantissa bits), ties to even
__device__ __forceinline__ float tf32_round(float v) {
    uint32_t u = __float_as_uint(v);
    u += 0xFFFu + ((u >> 13) & 1u);
    return __uint_as_float(u & 0xFFFFE000u);
}

template <int MODE>  // 0: bf16 (kind::f16); 1: tf32; 2: FP32 split as hi + lo TF32 (3 products)
__global__ void __launch_bounds__(128, 1) gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, int64_t rows,
                                                         int64_t cols, int s, double lam, const GramTile *tiles,
                                                         double *__restrict__ G, int *err) {
    constexpr bool BF16 = MODE == 0;
    constexpr bool SPLIT = MODE == 2;
    constexpr int STAGES = SPLIT ? 2 : TC_STAGES;
    constexpr int SBYTES = SPLIT ? 2 * TC_STAGE_BYTES : TC_STAGE_BYTES;  // split: hi tiles, then lo tiles
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);  // keeps the state space
    __shared__ __align__(8) uint64_t full_bar[TC_STAGES], empty_bar[TC_STAGES], split_bar[TC_STAGES], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_err;

    const GramTile tile = tiles[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)tile.j * s;
    const int len = (int)min64(s, rows - r0);
    const int BK = TC_ROWB / (BF16 ? 2 : 4);                 // K elements per stage
    const int KSTEP = BF16 ? 16 : 8;                         // K of one MMA
    const int nk = (int)((cols + BK - 1) / BK);
    constexpr uint32_t idesc = umma_idesc(BF16 ? 1u : 2u);

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full_bar[i], 1);
            mbar_init(&empty_bar[i], 1);
            mbar_init(&split_bar[i], 1);
        }
        mbar_init(&done_bar, 1);
        fence_mbar_init();
        s_err = 0;
    }
    if (warp == 0) {  // whole warp: allocate 256 TMEM columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // producer
        int stage = 0;
        unsigned phase = 0;
        for (int kt = 0; kt < nk; ++kt) {
            if (kt >= STAGES) {
                if (!mbar_wait_bounded(&empty_bar[stage], phase ^ 1u, TC_TIMEOUT_NS)) {
                    s_err = 1;
                    break;
                }
            }
            unsigned char *a_s = sm + stage * SBYTES;
            unsigned char *b_s = a_s + TC_ABYTES;
            mbar_arrive_expect_tx(&full_bar[stage], TC_STAGE_BYTES);
            const int kx = kt * BK;
            tma_load_2d(a_s, &tmap, kx, (int)(r0 + tile.ta * TC_M), &full_bar[stage]);
            tma_load_2d(b_s, &tmap, kx, (int)(r0 + tile.tc * TC_N), &full_bar[stage]);
            tma_load_2d(b_s + TC_ABYTES, &tmap, kx, (int)(r0 + tile.tc * TC_N + TC_M), &full_bar[stage]);
            if (++stage == STAGES) {
                stage = 0;
                phase ^= 1u;
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        int stage = 0;
        unsigned phase = 0;
        for (int kt = 0; kt < nk; ++kt) {
            if (!mbar_wait_bounded(SPLIT ? &split_bar[stage] : &full_bar[stage], phase, TC_TIMEOUT_NS)) {
                s_err = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(sm + stage * SBYTES);
            const uint32_t b_addr = a_addr + TC_ABYTES;
            for (int kk = 0; kk < BK / KSTEP; ++kk) {
                const uint32_t koff = (uint32_t)(kk * KSTEP * (BF16 ? 2 : 4));  // bytes along the 128-byte row
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                umma<BF16>(tmem, umma_desc_sw128(a_addr + koff), umma_desc_sw128(b_addr + koff), idesc, acc);
                if (SPLIT) {
                    const uint32_t lo = TC_STAGE_BYTES;  // lo tiles follow the hi tiles
                    umma<false>(tmem, umma_desc_sw128(a_addr + koff), umma_desc_sw128(b_addr + lo + koff), idesc, 1u);
                    umma<false>(tmem, umma_desc_sw128(a_addr + lo + koff), umma_desc_sw128(b_addr + koff), idesc, 1u);
                }
            }
            umma_commit(&empty_bar[stage]);  // stage reusable once these MMAs have read it
            if (++stage == STAGES) {
                stage = 0;
                phase ^= 1u;
            }
        }
        umma_commit(&done_bar);  // all issued MMAs complete (also on the error path)
    } else if (SPLIT && warp >= 2) {
        // splitters (64 threads): x -> hi = tf32(x) in place, lo = x - hi at the same offset of the lo tiles
        int stage = 0;
        unsigned phase = 0;
        const int t64 = threadIdx.x - 64;
        for (int kt = 0; kt < nk; ++kt) {
            bool ok = true;
            if (t64 == 0) ok = mbar_wait_bounded(&full_bar[stage], phase, TC_TIMEOUT_NS);
            asm volatile("bar.sync 1, 64;" ::: "memory");
            if (t64 == 0 && !ok) s_err = 1;
            asm volatile("bar.sync 1, 64;" ::: "memory");
            if (s_err) break;
            float4 *hi = (float4 *)(sm + stage * SBYTES);
            float4 *lo = (float4 *)(sm + stage * SBYTES + TC_STAGE_BYTES);
            for (int e = t64; e < TC_STAGE_BYTES / 16; e += 64) {
                const float4 v = hi[e];
                float4 h, l;
                h.x = tf32_round(v.x); l.x = v.x - h.x;
                h.y = tf32_round(v.y); l.y = v.y - h.y;
                h.z = tf32_round(v.z); l.z = v.z - h.z;
                h.w = tf32_round(v.w); l.w = v.w - h.w;
                hi[e] = h;
                lo[e] = l;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core reads
            asm volatile("bar.sync 1, 64;" ::: "memory");
            if (t64 == 0) mbar_arrive_expect_tx(&split_bar[stage], 0);
            if (++stage == STAGES) {
                stage = 0;
                phase ^= 1u;
            }
        }
    }
    __syncwarp();
    // epilogue: every thread owns TMEM lane (32 * warp + lane) = tile row
    bool ok = true;
    if (lane == 0) ok = mbar_wait_bounded(&done_bar, 0, TC_TIMEOUT_NS);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    tc_fence_after();
    if (ok && !s_err) {
        const int a = tile.ta * TC_M + warp * 32 + lane;  // row of G within the block
        double *Gj = G + (size_t)tile.j * s * s;
        for (int c0 = 0; c0 < TC_N; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            const int cb = tile.tc * TC_N + c0;
            if (a < len) {
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int c = cb + q;
                    if (c <= a && c < len) Gj[(size_t)a * len + c] = (double)__uint_as_float(v[q]) + (c == a ? lam : 0.0);
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
    }
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn2)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static bool gram_tc_disabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("KPP_GRAM_TC");
        v = (e && e[0] == '0') ? 1 : 0;
    }
    return v == 1;
}

bool gram_tc(const kpp_matrix &A, int s, double lam, double *G, cudaStream_t st, bool allow_tf32) {
    if (gram_tc_disabled()) return false;
    if (A.dtype != KPP_BF16 && A.dtype != KPP_F32) return false;
    const int mode = A.dtype == KPP_BF16 ? 0 : (allow_tf32 ? 1 : 2);
    const size_t es = A.dtype == KPP_F32 ? 4 : 2;
    if (((uintptr_t)A.data & 15) || ((A.ld * es) & 15) || A.rows > 0x7fffffffLL || A.cols > 0x7fffffffLL) return false;
    void *fnp = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fnp, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return false;
    EncodeTiledFn2 enc = (EncodeTiledFn2)fnp;
    CUtensorMap tm;
    cuuint64_t dims[2] = {(cuuint64_t)A.cols, (cuuint64_t)A.rows};
    cuuint64_t strides[1] = {(cuuint64_t)(A.ld * es)};
    cuuint32_t box[2] = {(cuuint32_t)(TC_ROWB / es), (cuuint32_t)TC_M};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&tm, A.dtype == KPP_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
            const_cast<void *>(A.data), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    // tiles of the lower triangle: row tile ta (128 rows), column tile tc (256 columns), 256 tc <= 128 ta + 127
    const int64_t nb = (A.rows + s - 1) / s;
    const int mt = (s + TC_M - 1) / TC_M, ntl = (s + TC_N - 1) / TC_N;
    std::vector<GramTile> tl;
    for (int64_t j = 0; j < nb; ++j)
        for (int ta = 0; ta < mt; ++ta)
            for (int tc = 0; tc < ntl; ++tc)
                if (tc * TC_N <= ta * TC_M + TC_M - 1) tl.push_back(GramTile{(int)j, ta, tc});
    GramTile *d_tiles = nullptr;
    int *d_err = nullptr;
    int herr = 0;
    bool ok = dev_malloc_async((void **)&d_tiles, tl.size() * sizeof(GramTile), st) == cudaSuccess;
    ok = ok && dev_malloc_async((void **)&d_err, sizeof(int), st) == cudaSuccess;
    ok = ok && cudaMemsetAsync(d_err, 0, sizeof(int), st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(d_tiles, tl.data(), tl.size() * sizeof(GramTile), cudaMemcpyHostToDevice, st) ==
                   cudaSuccess;
    if (ok) {
        auto kern = mode == 0 ? gram_tc_kernel<0> : (mode == 1 ? gram_tc_kernel<1> : gram_tc_kernel<2>);
        const int smem = mode == 2 ? 2 * 2 * TC_STAGE_BYTES + 1024 : TC_SMEM;
        ok = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
        if (ok) {
            note_launch();
            kern<<<(unsigned)tl.size(), 128, smem, st>>>(tm, A.rows, A.cols, s, lam, d_tiles, G, d_err);
            ok = cudaGetLastError() == cudaSuccess;
        }
        ok = ok && cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
        ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    }
    if (d_tiles) cudaFreeAsync(d_tiles, st);
    if (d_err) cudaFreeAsync(d_err, st);
    if (!ok || herr) {
        set_error("tensor-core Gram failed (%s); using the CUDA-core Gram", herr ? "device wait expired" : "launch");
        return false;
    }
    return true;
}

}  // namespace kpp
