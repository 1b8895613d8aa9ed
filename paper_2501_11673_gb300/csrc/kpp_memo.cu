// kpp_memo.cu -- host side of the online block memoisation: the block sequence of a window of steps
// (kpp_memo_sequence).  See kpp_memo.cuh for the scheme and its draws.
#include "../../include/kpp.h"
#include "kpp_memo.cuh"
#include "kpp_runtime.h"

using namespace kpp;

extern "C" {

kpp_status kpp_memo_sequence(uint64_t seed, uint32_t sys_id, int32_t mode, int64_t rows, int64_t cols, int32_t s,
                             int64_t t0, int64_t count, int64_t nb0, int64_t *blocks, int64_t *subsets,
                             int64_t subsets_cap, int64_t *nb_out) {
    clear_error();
    if ((mode != 0 && mode != 1) || rows < 1 || cols < 1 || s < 1 || s > rows || t0 < 0 || count < 0 || nb0 < 0 ||
        subsets_cap < 0 || !nb_out || (count > 0 && !blocks) || (subsets_cap > 0 && !subsets) ||
        (mode == 1 && rows != cols)) {
        set_error("kpp_memo_sequence: invalid argument");
        return KPP_ERR_ARG;
    }
    int64_t nb = nb0, fresh = 0;
    for (int64_t i = 0; i < count; ++i) {
        const int64_t t = t0 + i;
        int64_t j = memo_pick(seed, t, sys_id, mode, rows, cols, s, nb);
        if (j < 0) {
            if (fresh == subsets_cap) {
                *nb_out = nb;
                set_error("kpp_memo_sequence: more than %lld new blocks in the window (subsets_cap)",
                          (long long)subsets_cap);
                return KPP_ERR_ARG;
            }
            memo_subset(seed, t, sys_id, rows, s, subsets + fresh * s);
            ++fresh;
            j = nb++;
        }
        blocks[i] = j;
    }
    *nb_out = nb;
    return KPP_OK;
}

}  // extern "C"
