// kpp_internal.cuh -- device helpers shared by the kernels of libkpp (sm_103a).
//
// Nothing here is shared with the CPU oracle: the Philox generator below is written from its
// published definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11), independently of the oracle's copy.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kpp.h"

namespace kpp {

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 and the block draw (uniform over nb blocks, with replacement).
// ---------------------------------------------------------------------------------------------
struct u32x4 {
    uint32_t x, y, z, w;
};

__host__ __device__ inline u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        u32x4 n;
        n.x = (uint32_t)(p1 >> 32) ^ c.y ^ k0;
        n.y = (uint32_t)p1;
        n.z = (uint32_t)(p0 >> 32) ^ c.w ^ k1;
        n.w = (uint32_t)p0;
        c = n;
    }
    return c;
}

__host__ __device__ inline int32_t draw_block(uint64_t seed, int64_t t, uint32_t sys, int32_t nb) {
    u32x4 c{(uint32_t)(uint64_t)t, (uint32_t)((uint64_t)t >> 32), sys, 0u};
    u32x4 o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return (int32_t)(((uint64_t)o.x * (uint64_t)(uint32_t)nb) >> 32);
}

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------------------------------------
// Storage types.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return (double)v; }
__device__ __forceinline__ double widen(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// Exact FP32 -> FP64 widening with integer operations only, so that an FP64-bound loop spends its FP64
// pipe on FMAs.  On this GPU the conversion instruction occupies the FP64 pipe like an FMA, and even a
// predicated-off one for the rare case costs the same issue on that pipe, so no case uses it:
//   normal (exponent e in 1..254): exponent e + 896 (bias 127 -> 1023), mantissa shifted 23 -> 52 bits;
//   inf / NaN (e = 255): exponent 2047, mantissa shifted;
//   zero: the sign alone;
//   subnormal m 2^-149 (e = 0, m != 0): with p the position of m's leading one, the value is
//   2^(p - 149) (1 + (m - 2^p) / 2^p): exponent p + 874, fraction (m - 2^p) << (52 - p).
__device__ __forceinline__ double widen_int(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t sgn = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    const uint32_t eb = e == 255u ? 2047u : e + 896u;
    uint32_t hi = sgn | (eb << 20) | (m >> 3);
    uint32_t lo = m << 29;
    if (e == 0u) {
        const int p = 31 - __clz((int)(m | 1u));
        const uint64_t frac = (uint64_t)(m ^ (1u << p)) << (52 - p);
        hi = m ? (sgn | ((uint32_t)(p + 874) << 20) | (uint32_t)(frac >> 32)) : sgn;
        lo = m ? (uint32_t)frac : 0u;
    }
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen_fast(double v) { return v; }
__device__ __forceinline__ double widen_fast(float v) { return widen_int(v); }
__device__ __forceinline__ double widen_fast(__nv_bfloat16 v) { return widen_int(__bfloat162float(v)); }

template <typename T> __device__ __forceinline__ T load_as(const double v);
template <> __device__ __forceinline__ double load_as<double>(const double v) { return v; }
template <> __device__ __forceinline__ float load_as<float>(const double v) { return (float)v; }

template <typename TC> __device__ __forceinline__ TC conv(double v) { return (TC)v; }
template <typename TC> __device__ __forceinline__ TC conv(float v) { return (TC)v; }
template <typename TC> __device__ __forceinline__ TC conv(__nv_bfloat16 v) { return (TC)__bfloat162float(v); }

// ---------------------------------------------------------------------------------------------
// Bounded inter-CTA barrier for a group of G co-resident CTAs (cooperative launch).
//
// The counter only grows: barrier number q waits until it reaches q*G.  An error (a bounded wait
// that expired, or a numeric failure) adds ERR_BIAS to the counter, which releases every waiter at
// once; waiters recognise the bias and return false.  The wait polls with acquire loads and
// reads %globaltimer every 256 polls; after `timeout_ns` it raises KPP_ERR_TIMEOUT.
// ---------------------------------------------------------------------------------------------
constexpr unsigned ERR_BIAS = 0x40000000u;

// Bring the 128-byte line holding p into L2 (no register result, no fault on the hint itself).
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct GroupSync {
    unsigned *ctr;      // group counter (zeroed before launch)
    int *err;           // group error word (kpp_status; zeroed before launch)
    unsigned target;    // per-CTA copy of the next target
    unsigned G;         // CTAs in the group
    uint64_t timeout_ns;
};

// Raise an error for the whole group (any thread may call; idempotent on the error word).
__device__ __forceinline__ void group_fail(GroupSync &gs, int code) {
    if (atomicCAS(gs.err, 0, code) == 0) atomicAdd(gs.ctr, ERR_BIAS);
}

// Returns true when every CTA of the group arrived, false on a group error.  All threads of the
// CTA must call it (it contains __syncthreads()).
__device__ __forceinline__ bool group_barrier(GroupSync &gs) {
    __shared__ int s_ok;
    __syncthreads();
    gs.target += 1u;
    if (threadIdx.x == 0) {
        unsigned want = gs.target * gs.G;
        // release: the CTA's writes (ordered before this thread by __syncthreads) become visible
        // to any CTA whose acquire load sees this arrival
        red_release_add_u32(gs.ctr, 1u);
        unsigned v = ld_acquire_u32(gs.ctr);
        uint64_t t0 = 0;
        unsigned polls = 0;
        while ((int)(v - want) < 0) {
            if ((++polls & 255u) == 0u) {
                uint64_t now = globaltimer_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > gs.timeout_ns) {
                    group_fail(gs, KPP_ERR_TIMEOUT);
                }
            }
            v = ld_acquire_u32(gs.ctr);
        }
        s_ok = ((int)(v - want) < (int)(ERR_BIAS / 2u)) ? 1 : 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// Deterministic block-wide sum of one double per thread (fixed tree), result valid in all threads.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red /* NT/32 doubles */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    return s;
}

}  // namespace kpp

// ---------------------------------------------------------------------------------------------
// TMA and mbarrier helpers (inline PTX, sm_90+ forms available on sm_103a).
// ---------------------------------------------------------------------------------------------
namespace kpp {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on an mbarrier phase: returns false after `timeout_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > timeout_ns) return false;
    }
    return true;
}
// 2-D tiled TMA load of box {x .. x+box0, y .. y+box1} (out-of-range elements are zero-filled).
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// 1-D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tensormap_acquire(const void *tmap) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}

}  // namespace kpp
