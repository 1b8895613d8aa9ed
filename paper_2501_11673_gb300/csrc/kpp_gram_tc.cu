// kpp_gram_tc.cu -- block Gram A_S A_S^T on the tcgen05 tensor cores (FP32/BF16 storage).
#include "kpp_internal.cuh"
#include "kpp_runtime.h"

namespace kpp {

bool gram_tc(const kpp_matrix &A, int s, double lam, double *G, cudaStream_t st) {
    (void)A; (void)s; (void)lam; (void)G; (void)st;
    return false;
}

}  // namespace kpp
