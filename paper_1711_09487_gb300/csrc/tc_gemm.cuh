// Tensor-core (tcgen05, 3xTF32) complex-FP32 GEMM; host launcher.
#pragma once
#include "dense.cuh"

namespace rfdd {
bool tc_enabled();  // false when the environment variable RFDD_TC is "0"
// C = beta*C + alpha*A*B for every item (complex, row-major, no transposes)
void tc_gemm_complex(cudaStream_t st, const std::vector<GemmItem<cx<float>>> &items, double alpha, double beta);
// C = beta*C + alpha*A*B for real FP32 items (same kernel, 3xTF32)
void tc_gemm_real(cudaStream_t st, const std::vector<GemmItem<float>> &items, double alpha, double beta);
// returns and clears the device-side error flags of the tensor-core kernels (DS_* bits)
int tc_take_error();
// allocation-free variant: packed operands in a static device array (m, n <= 1024, k <= 128)
void tc_gemm_complex_noalloc(cudaStream_t st, const cx<float> *A, int64_t lda, const cx<float> *B, int64_t ldb,
                             cx<float> *C, int64_t ldc, int m, int n, int k, double alpha, double beta);
}  // namespace rfdd
