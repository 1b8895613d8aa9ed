// kpp_wmemo.cu -- the memoised W_j = G_j^{-1} A_{S_j} (FP32) of the large-block K++ kernel.
//
// BF16 storage: the library's own tcgen05 kernel (kpp_wmemo_tc.cu).  FP32 storage, and any shape the
// tcgen05 kernel does not take: a plain batched GEMM per block of the partition (s x s times s x n)
// on cuBLAS, with the FP32 compute type that splits each operand into three BF16 parts on the tensor
// cores (FP32 accuracy); BF16 storage is then widened to FP32 a chunk of blocks at a time.
// KPP_WMEMO_TC=0 in the environment sends every shape to cuBLAS (for comparisons).
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <cstdlib>
#include <map>
#include <mutex>

#include "kpp_runtime.h"

namespace kpp {

static cublasHandle_t blas_handle() {
    // one handle per thread and device (handles are not shared between host threads)
    thread_local std::map<int, cublasHandle_t> handles;
    int dev = 0;
    cudaGetDevice(&dev);
    auto it = handles.find(dev);
    if (it != handles.end()) return it->second;
    cublasHandle_t h = nullptr;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return nullptr;
    handles[dev] = h;
    return h;
}

__global__ void widen_bf16_kernel(int64_t rows, int64_t cols, const __nv_bfloat16 *__restrict__ a, int64_t lda,
                                  float *__restrict__ o) {
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / cols, c = e - r * cols;
        o[e] = __bfloat162float(a[r * lda + c]);
    }
}

kpp_status build_w32_tc(const kpp_matrix &A, int s, const float *Ginv32, float *W32, cudaStream_t st);

kpp_status build_w32(const kpp_matrix &A, int s, const float *Ginv32, float *W32, cudaStream_t st) {
    const char *tc_env = getenv("KPP_WMEMO_TC");
    if (A.dtype == KPP_BF16 && !(tc_env && tc_env[0] == '0')) {
        if (build_w32_tc(A, s, Ginv32, W32, st) == KPP_OK) return KPP_OK;
        // not taken or failed: the library GEMM below rewrites every block
    }
    const int64_t rows = A.rows, cols = A.cols;
    const int64_t nb = rows / s;  // whole blocks only (checked by the caller)
    cublasHandle_t h = blas_handle();
    if (!h) {
        set_error("cublasCreate failed");
        return KPP_ERR_CUDA;
    }
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) {
        set_error("cublasSetStream failed");
        return KPP_ERR_CUDA;
    }
    const float one = 1.f, zero = 0.f;
    const int64_t bsz = (int64_t)s * cols;
    float *tmp = nullptr;
    int64_t chunk = nb;
    if (A.dtype == KPP_BF16) {
        chunk = (int64_t)((512ull << 20) / ((size_t)bsz * 4));
        if (chunk < 1) chunk = 1;
        if (chunk > nb) chunk = nb;
        if (dev_malloc_async((void **)&tmp, (size_t)chunk * bsz * 4, st) != cudaSuccess) {
            set_error("out of device memory for the W memo");
            return KPP_ERR_OOM;
        }
    }
    kpp_status rc = KPP_OK;
    for (int64_t j0 = 0; j0 < nb && rc == KPP_OK; j0 += chunk) {
        const int64_t cnt = nb - j0 < chunk ? nb - j0 : chunk;
        const float *a;
        int64_t lda;
        if (A.dtype == KPP_BF16) {
            note_launch();
            widen_bf16_kernel<<<4 * sm_count(), 256, 0, st>>>(cnt * s, cols,
                                                             (const __nv_bfloat16 *)A.data + j0 * s * A.ld, A.ld, tmp);
            if (cudaGetLastError() != cudaSuccess) {
                set_error("widening launch failed");
                rc = KPP_ERR_CUDA;
                break;
            }
            a = tmp;
            lda = cols;
        } else {
            a = (const float *)A.data + j0 * s * A.ld;
            lda = A.ld;
        }
        // row-major W_j (s x n) = G_j^{-1} (s x s) A_j (s x n), i.e. column-major W_j^T = A_j^T G_j^{-T}
        const cublasStatus_t bs = cublasGemmStridedBatchedEx(
            h, CUBLAS_OP_N, CUBLAS_OP_N, (int)cols, s, s, &one, a, CUDA_R_32F, (int)lda, (long long)s * lda,
            Ginv32 + j0 * (int64_t)s * s, CUDA_R_32F, s, (long long)s * s, &zero, W32 + j0 * bsz, CUDA_R_32F,
            (int)cols, (long long)bsz, (int)cnt, CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT);
        if (bs != CUBLAS_STATUS_SUCCESS) {
            set_error("cublasGemmStridedBatchedEx (W memo) failed: %d", (int)bs);
            rc = KPP_ERR_CUDA;
        }
    }
    if (tmp) cudaFreeAsync(tmp, st);
    return rc;
}

}  // namespace kpp
