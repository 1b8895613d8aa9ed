// kpp_memo.cuh -- the draws of the online block memoisation (Sec. 4, "Block memoization"; Sec. 5.2, the
// simplified scheme of CD++; the sampling steps of Alg. 3 and Alg. 5), host and device.
//
// Step t either samples a new uniformly random s-subset S of the rows (with probability p_t; it joins
// the memo with the next index) or reuses a memoised block picked uniformly.  p_0 = 1, and for t >= 1
//   CD++: p_t = min(1, (n / s) ln(n) / t),    K++: p_t = min(1, (m / s) ln(m) / t, (n / s) ln(m) / t).
// The draws are Philox4x32-10 words, key {seed_lo, seed_hi}: counter {t_lo, t_hi, sys, 0} gives the
// Bernoulli word (out.y: new iff out.y < p_t 2^32) and the pick (out.z: index (out.z |B|) >> 32);
// counter {t_lo, t_hi, sys, 1 + i / 4} gives word i mod 4 of the subset draw, which is Floyd's sampling
// (for j = N - s .. N - 1: r = (word (j + 1)) >> 32; take j if r is already in S, else r), then sorted.
// The block sequence depends only on (seed, t, sys), never on the data, so it can be drawn ahead of
// the iteration, one window of steps at a time.
#pragma once

#include <stdint.h>

#include <cmath>

#include "kpp_internal.cuh"

namespace kpp {

__host__ __device__ inline double memo_prob(int cd, int64_t rows, int64_t n, int s, int64_t t) {
    if (t <= 0) return 1.0;
    double p;
    if (cd) {
        p = (double)n / (double)s * log((double)n) / (double)t;
    } else {
        const double lm = log((double)rows);
        const double a = (double)rows / (double)s * lm / (double)t, c = (double)n / (double)s * lm / (double)t;
        p = a < c ? a : c;
    }
    return p < 1.0 ? p : 1.0;
}

// -1: step t samples a new subset; otherwise the memo index (in [0, nb)) it reuses.
__host__ __device__ inline int64_t memo_pick(uint64_t seed, int64_t t, uint32_t sys, int cd, int64_t rows, int64_t n,
                                             int s, int64_t nb) {
    if (nb <= 0) return -1;
    const u32x4 c{(uint32_t)(uint64_t)t, (uint32_t)((uint64_t)t >> 32), sys, 0u};
    const u32x4 o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    if ((double)o.y < memo_prob(cd, rows, n, s, t) * 4294967296.0) return -1;
    return (int64_t)(((uint64_t)o.z * (uint64_t)nb) >> 32);
}

// The s-subset of [0, N) drawn at step t, ascending, into S[0 .. s).
__host__ __device__ inline void memo_subset(uint64_t seed, int64_t t, uint32_t sys, int64_t N, int s, int64_t *S) {
    u32x4 o{0u, 0u, 0u, 0u};
    for (int i = 0; i < s; ++i) {
        if ((i & 3) == 0) {
            const u32x4 c{(uint32_t)(uint64_t)t, (uint32_t)((uint64_t)t >> 32), sys, 1u + (uint32_t)(i >> 2)};
            o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        }
        const uint32_t w = (i & 3) == 0 ? o.x : (i & 3) == 1 ? o.y : (i & 3) == 2 ? o.z : o.w;
        const int64_t j = N - s + i;
        const int64_t r = (int64_t)(((uint64_t)w * (uint64_t)(j + 1)) >> 32);
        bool taken = false;
        for (int q = 0; q < i; ++q) taken = taken || S[q] == r;
        S[i] = taken ? j : r;
    }
    for (int a = 1; a < s; ++a) {  // insertion sort: s is a block size
        const int64_t v = S[a];
        int q = a - 1;
        while (q >= 0 && S[q] > v) {
            S[q + 1] = S[q];
            --q;
        }
        S[q + 1] = v;
    }
}

}  // namespace kpp
