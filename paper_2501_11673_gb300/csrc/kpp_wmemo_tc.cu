// kpp_wmemo_tc.cu -- the memo W_j = G_j^{-1} A_{S_j} (FP32) on the tcgen05 tensor cores, for BF16
// storage (Sec. 4's memoised projection, folded into one operator per block so that a K++ step of
// the large-block kernel needs a single exchange: w = A_S^T G^{-1} r = W_S^T r).
//
// One GEMM per block: M = s (rows of W_j), N = n (columns of A), K = s.  Both operands are fed
// K-major with the 128-byte swizzle:
//   * A operand: G_j^{-1} in three BF16 pieces g = g_hi + g_mid + g_lo, each the BF16 rounding of
//     what the earlier pieces leave (the differences are exact in FP32), so the three carry the 24
//     significant bits of the FP32 inverse; stacked as [3][rows][s], block j's rows at j*s;
//   * B operand: A_{S_j}^T, i.e. rows c of a transposed copy A^T (n x rows), K = the block's rows.
// A BF16 entry of A is exact in the MMA, each product is exact in FP32, and the three MMAs (smallest
// piece first) accumulate in FP32 in tensor memory: W carries FP32 accuracy without widening A.
// One CTA computes one 128 x 256 tile of one W_j:
//   * warp 0, one thread: TMA producer into a 2-stage ring (three G^{-1} pieces + one A^T tile a stage);
//   * warp 1, one thread: MMA issuer (M = 128, N = 256, K = 16 per MMA, kind::f16);
//   * warps 0-3: epilogue, tcgen05.ld of their 32 lanes and FP32 stores of the tile's rows.
// Every wait is bounded; a wait that runs out sets the error word, and the CTA still waits (bounded)
// for its issued MMAs before it releases tensor memory.  The caller falls back to the library GEMM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <vector>

#include "kpp_internal.cuh"
#include "kpp_runtime.h"
#include "kpp_solve.h"
#include "kpp_tc.cuh"

namespace kpp {

constexpr int WM_STAGES = 2;
constexpr int WM_ROWB = 128;                               // bytes of K per tile row (64 BF16)
constexpr int WM_BK = WM_ROWB / 2;                         // K elements per stage
constexpr int WM_ABYTES = TC_M * WM_ROWB;                  // one G^{-1} piece: 16 KiB
constexpr int WM_BBYTES = TC_N * WM_ROWB;                  // the A^T tile: 32 KiB
constexpr int WM_STAGE_BYTES = 3 * WM_ABYTES + WM_BBYTES;  // 80 KiB
constexpr int WM_SMEM = WM_STAGES * WM_STAGE_BYTES + 1024; // + alignment slack
constexpr uint64_t WM_TIMEOUT_NS = 2000000000ull;


// G^{-1} (n values, FP32) -> pieces hi, mid, lo (BF16) at out, out + n, out + 2n, for entries [i0, i1).
__global__ void split3_bf16_kernel(int64_t n, int64_t i0, int64_t i1, const float *__restrict__ g,
                                   __nv_bfloat16 *__restrict__ out) {
    for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = g[i];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(m);
        out[i] = h;
        out[n + i] = m;
        out[2 * n + i] = __float2bfloat16_rn(r2);
    }
}

// A (rows x cols BF16, leading dimension lda) -> A^T (cols x rows BF16), 64 x 64 tiles in shared memory,
// 16-byte loads and stores (rows, cols and lda multiples of 8, the base 16-byte aligned: checked by the
// host).  Tile element (r, c) sits at word (r, c / 2) of a row padded to 33 words, so the column reads
// of the second phase fall in distinct banks.
__global__ void __launch_bounds__(256) transpose_bf16_kernel(int64_t rows, int64_t cols,
                                                             const __nv_bfloat16 *__restrict__ a, int64_t lda,
                                                             __nv_bfloat16 *__restrict__ at) {
    __shared__ uint32_t t[64][33];
    const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
    // phase 1: 64 rows x 8 chunks of 8 values; thread -> (row, chunk)
    for (int e = threadIdx.x; e < 64 * 8; e += 256) {
        const int rr = e >> 3, ch = e & 7;
        const int64_t r = r0 + rr, c = c0 + ch * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < rows && c < cols) v = *reinterpret_cast<const uint4 *>(a + r * lda + c);
        t[rr][ch * 4 + 0] = v.x;
        t[rr][ch * 4 + 1] = v.y;
        t[rr][ch * 4 + 2] = v.z;
        t[rr][ch * 4 + 3] = v.w;
    }
    __syncthreads();
    // phase 2: 64 columns x 8 chunks of 8 rows; thread -> (column, chunk)
    for (int e = threadIdx.x; e < 64 * 8; e += 256) {
        const int cc = e >> 3, ch = e & 7;
        const int64_t c = c0 + cc, r = r0 + ch * 8;
        uint32_t h[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint32_t wv = t[ch * 8 + q][cc >> 1];
            h[q] = (cc & 1) ? (wv >> 16) : (wv & 0xffffu);
        }
        if (c < cols && r < rows)
            *reinterpret_cast<uint4 *>(at + c * rows + r) =
                make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
    }
}

__global__ void __launch_bounds__(128, 1) wmemo_tc_kernel(const __grid_constant__ CUtensorMap tmG,
                                                          const __grid_constant__ CUtensorMap tmB, int64_t rows,
                                                          int64_t cols, int s, int mt, int ntl,
                                                          float *__restrict__ W, int *err, int j0) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full_bar[WM_STAGES], empty_bar[WM_STAGES], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_err;

    // tile (block j, row tile ta, column tile tc) of this CTA, column tiles fastest
    struct {
        int j, ta, tc;
    } tile;
    tile.tc = (int)(blockIdx.x % (unsigned)ntl);
    tile.ta = (int)((blockIdx.x / (unsigned)ntl) % (unsigned)mt);
    tile.j = j0 + (int)(blockIdx.x / ((unsigned)ntl * (unsigned)mt));  // blocks from j0 on
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)tile.j * s;
    const int nk = (s + WM_BK - 1) / WM_BK;
    constexpr uint32_t idesc = umma_idesc(1u);

    if (threadIdx.x == 0) {
        for (int i = 0; i < WM_STAGES; ++i) {
            mbar_init(&full_bar[i], 1);
            mbar_init(&empty_bar[i], 1);
        }
        mbar_init(&done_bar, 1);
        fence_mbar_init();
        s_err = 0;
    }
    if (warp == 0) {  // whole warp: 256 TMEM columns for the 128 x 256 FP32 accumulator
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
        const int ya = (int)(r0 + tile.ta * TC_M);
        const int yb = tile.tc * TC_N;
        for (int kt = 0; kt < nk; ++kt) {
            if (kt >= WM_STAGES) {
                if (!mbar_wait_bounded(&empty_bar[stage], phase ^ 1u, WM_TIMEOUT_NS)) {
                    s_err = 1;
                    break;
                }
            }
            unsigned char *a_s = sm + stage * WM_STAGE_BYTES;
            unsigned char *b_s = a_s + 3 * WM_ABYTES;
            mbar_arrive_expect_tx(&full_bar[stage], WM_STAGE_BYTES);
            for (int p = 0; p < 3; ++p)
                tma_load_2d(a_s + p * WM_ABYTES, &tmG, kt * WM_BK, (int)(p * rows) + ya, &full_bar[stage]);
            const int kx = (int)r0 + kt * WM_BK;
            tma_load_2d(b_s, &tmB, kx, yb, &full_bar[stage]);
            tma_load_2d(b_s + WM_ABYTES, &tmB, kx, yb + TC_M, &full_bar[stage]);
            if (++stage == WM_STAGES) {
                stage = 0;
                phase ^= 1u;
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: per 16-wide K slice, lo, mid, then hi into the same accumulator
        int stage = 0;
        unsigned phase = 0;
        for (int kt = 0; kt < nk; ++kt) {
            if (!mbar_wait_bounded(&full_bar[stage], phase, WM_TIMEOUT_NS)) {
                s_err = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(sm + stage * WM_STAGE_BYTES);
            const uint32_t b_addr = a_addr + 3 * WM_ABYTES;
            for (int kk = 0; kk < WM_BK / 16; ++kk) {
                const uint32_t koff = (uint32_t)(kk * 32);  // 16 BF16 along the 128-byte row
                for (int p = 2; p >= 0; --p) {
                    const uint32_t acc = (kt > 0 || kk > 0 || p != 2) ? 1u : 0u;
                    umma<true>(tmem, umma_desc_sw128(a_addr + p * WM_ABYTES + koff), umma_desc_sw128(b_addr + koff),
                               idesc, acc);
                }
            }
            umma_commit(&empty_bar[stage]);
            if (++stage == WM_STAGES) {
                stage = 0;
                phase ^= 1u;
            }
        }
        umma_commit(&done_bar);  // every issued MMA complete (also on the error path)
    }
    __syncwarp();
    // epilogue: thread (warp, lane) owns TMEM lane 32 warp + lane = row a of the tile
    bool ok = true;
    if (lane == 0) ok = mbar_wait_bounded(&done_bar, 0, WM_TIMEOUT_NS);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    tc_fence_after();
    if (ok && !s_err) {
        const int a = tile.ta * TC_M + warp * 32 + lane;
        float *wrow = W + (r0 + a) * cols;
        for (int c0 = 0; c0 < TC_N; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            const int64_t cb = (int64_t)tile.tc * TC_N + c0;
            if (a < s) {
                if (cb + 32 <= cols) {
                    float4 *d4 = reinterpret_cast<float4 *>(wrow + cb);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        d4[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                            __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
                } else {
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (cb + q < cols) wrow[cb + q] = __uint_as_float(v[q]);
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

// Host side, in three parts so that the factor phase can build the memo of a range of blocks as soon
// as their inverses exist (kpp_runtime.h, WmemoTC):
//   begin: shape checks, the transposed copy A^T and the tensor maps (on the stream given);
//   blocks: the BF16 pieces of G_j^{-1} and W_j for blocks [j0, j1);
//   end: the error word (synchronises), and the scratch is released.
// An error leaves nothing of W32 relied on: the caller then uses the library GEMM.
kpp_status wmemo_tc_begin(WmemoTC &w, const kpp_matrix &A, int s, cudaStream_t st) {
    w = WmemoTC{};
    const int64_t rows = A.rows, cols = A.cols;
    if (A.dtype != KPP_BF16 || rows % s || s % 8 || rows % 8 || cols % 4 || ((uintptr_t)A.data & 15) ||
        ((A.ld * 2) & 15) || 3 * rows > 0x7fffffffLL || cols > 0x7fffffffLL || cols % 8)
        return KPP_ERR_UNSUPPORTED;
    const int64_t nb = rows / s;
    const int mt = (s + TC_M - 1) / TC_M;
    const int64_t ntl = (cols + TC_N - 1) / TC_N;
    if (nb * mt * ntl > 0x7fffffffLL) return KPP_ERR_UNSUPPORTED;
    w.rows = rows;
    w.cols = cols;
    w.s = s;
    w.mt = mt;
    w.ntl = ntl;
    bool ok = dev_malloc_async((void **)&w.AT, (size_t)rows * cols * 2, st) == cudaSuccess;
    ok = ok && dev_malloc_async((void **)&w.Gs, (size_t)3 * rows * s * 2, st) == cudaSuccess;
    ok = ok && dev_malloc_async((void **)&w.d_err, sizeof(int), st) == cudaSuccess;
    if (!ok) {
        wmemo_tc_end(w, st);
        return KPP_ERR_OOM;
    }
    ok = cudaMemsetAsync(w.d_err, 0, sizeof(int), st) == cudaSuccess;
    note_launch();
    transpose_bf16_kernel<<<dim3((unsigned)((cols + 63) / 64), (unsigned)((rows + 63) / 64)), 256, 0, st>>>(
        rows, cols, (const __nv_bfloat16 *)A.data, A.ld, (__nv_bfloat16 *)w.AT);
    ok = ok && cudaGetLastError() == cudaSuccess;
    static_assert(sizeof(CUtensorMap) <= sizeof(w.tmG), "tensor map storage");
    ok = ok && make_tmap_2d(w.tmG, w.Gs, KPP_BF16, (uint64_t)s, (uint64_t)(3 * rows), (uint64_t)s, WM_BK, TC_M, true);
    ok = ok && make_tmap_2d(w.tmB, w.AT, KPP_BF16, (uint64_t)rows, (uint64_t)cols, (uint64_t)rows, WM_BK, TC_M, true);
    ok = ok && cudaFuncSetAttribute(wmemo_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WM_SMEM) == cudaSuccess;
    if (!ok) {
        wmemo_tc_end(w, st);
        return KPP_ERR_CUDA;
    }
    w.ready = true;
    return KPP_OK;
}

kpp_status wmemo_tc_blocks(WmemoTC &w, const float *Ginv32, float *W32, int64_t j0, int64_t j1, cudaStream_t st) {
    if (!w.ready || ((uintptr_t)W32 & 15)) return KPP_ERR_UNSUPPORTED;
    if (j1 <= j0) return KPP_OK;
    const int64_t n = w.rows * w.s;
    note_launch();
    split3_bf16_kernel<<<4 * sm_count(), 256, 0, st>>>(n, j0 * w.s * w.s, j1 * w.s * w.s, Ginv32, (__nv_bfloat16 *)w.Gs);
    note_launch();
    wmemo_tc_kernel<<<(unsigned)((j1 - j0) * w.mt * w.ntl), 128, WM_SMEM, st>>>(
        *reinterpret_cast<const CUtensorMap *>(w.tmG), *reinterpret_cast<const CUtensorMap *>(w.tmB), w.rows, w.cols,
        w.s, w.mt, (int)w.ntl, W32, w.d_err, (int)j0);
    return cudaGetLastError() == cudaSuccess ? KPP_OK : KPP_ERR_CUDA;
}

kpp_status wmemo_tc_end(WmemoTC &w, cudaStream_t st) {
    int herr = 0;
    kpp_status rc = KPP_OK;
    if (w.ready && (cudaMemcpyAsync(&herr, w.d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess || herr))
        rc = KPP_ERR_CUDA;
    if (w.AT) cudaFreeAsync(w.AT, st);
    if (w.Gs) cudaFreeAsync(w.Gs, st);
    if (w.d_err) cudaFreeAsync(w.d_err, st);
    if (rc != KPP_OK) {
        cudaGetLastError();
        set_error("tensor-core W memo failed (%s); using the library GEMM", herr ? "device wait expired" : "setup");
    }
    w = WmemoTC{};
    return rc;
}

kpp_status build_w32_tc(const kpp_matrix &A, int s, const float *Ginv32, float *W32, cudaStream_t st) {
    WmemoTC w;
    kpp_status rc = wmemo_tc_begin(w, A, s, st);
    if (rc != KPP_OK) return rc;
    rc = wmemo_tc_blocks(w, Ginv32, W32, 0, A.rows / s, st);
    const kpp_status re = wmemo_tc_end(w, st);
    return rc != KPP_OK ? rc : re;
}

}  // namespace kpp
