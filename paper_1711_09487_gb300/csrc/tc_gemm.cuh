// Tensor-core (tcgen05, 3xTF32) complex-FP32 GEMM; host launcher.
#pragma once
#include "dense.cuh"

#include <string>

namespace rfdd {
// Status word (device int) that the tensor-core launches issued by the calling host thread record
// a failed wait in (DS_WAIT_TIMEOUT), for the lifetime of the scope.  A launch outside any scope is
// refused with RFDD_ESTATE.
struct TcStatusScope {
  int *prev;
  explicit TcStatusScope(int *word);
  ~TcStatusScope();
  TcStatusScope(const TcStatusScope &) = delete;
  TcStatusScope &operator=(const TcStatusScope &) = delete;
};
// While alive, the tensor-core kernel launches of the calling host thread record ab[0] just before
// and ab[1] just after the kernel (not the operand packing): the probes time the MMA kernel alone.
struct TcKernelEvents {
  const cudaEvent_t *prev;
  explicit TcKernelEvents(const cudaEvent_t *ab);
  ~TcKernelEvents();
  TcKernelEvents(const TcKernelEvents &) = delete;
  TcKernelEvents &operator=(const TcKernelEvents &) = delete;
};
// While alive, the tensor-core launches of the calling host thread use one kernel: 1 the one-CTA
// kernel (128 x 256 tiles), 2 the two-CTA kernel (256 x 256 tiles on SM pairs), 0 the automatic
// choice.  For tests that check both kernels.
struct TcEngineScope {
  int prev;
  explicit TcEngineScope(int engine);
  ~TcEngineScope();
  TcEngineScope(const TcEngineScope &) = delete;
  TcEngineScope &operator=(const TcEngineScope &) = delete;
};
// C = beta*C + alpha*A*B for every item (complex, row-major, no transposes)
void tc_gemm_complex(cudaStream_t st, const std::vector<GemmItem<cx<float>>> &items, double alpha, double beta);
// C = beta*C + alpha*A*B for real FP32 items (same kernel, 3xTF32)
void tc_gemm_real(cudaStream_t st, const std::vector<GemmItem<float>> &items, double alpha, double beta);
// the same with one TF32 product per multiply (operands rounded to TF32): the throughput probe of
// the plain TF32 tensor path, not used by the solver
void tc_gemm_real_tf32(cudaStream_t st, const std::vector<GemmItem<float>> &items, double alpha, double beta);

// The tile-shape autotuner: mode 0 off (fixed rule), 1 on, 2 forget every class (re-tune);
// returns whether it was on.  tc_autotune_table: one line per class (tc_tune.h, Tuner::dump).
int tc_autotune(int mode);
std::string tc_autotune_table();
// A operand already split into TF32 hi/lo and laid out in the kernel's tiles (tc_pack_a_batched):
// tile (mt, kt) of the operand at hi/lo + (mt * mt_stride + kt) * tile size.  Lets a factor that
// is multiplied many times (triangular-solve updates, border products) be packed once.
struct TcPackedA {
  const float *hi = nullptr, *lo = nullptr;
  int64_t mt_stride = 0;
};
// items[i] uses pa[i] as its A operand when pa[i].hi is set (items[i].A is then not read)
void tc_gemm_complex_pa(cudaStream_t st, const std::vector<GemmItem<cx<float>>> &items,
                        const std::vector<TcPackedA> &pa, double alpha, double beta);
// packing of complex m x k matrices (row-major, leading dimension lda) into hi/lo tile arrays
// of tc_packed_a_floats(m, k) floats each (rows and K padded with zeros to whole tiles)
struct TcPackJob {
  const cx<float> *A;
  int64_t lda, m, k;
  float *hi, *lo;
};
int64_t tc_packed_a_ktiles(int64_t k);
int64_t tc_packed_a_floats(int64_t m, int64_t k);
void tc_pack_a_batched(cudaStream_t st, const std::vector<TcPackJob> &jobs);
// the sub-matrix of a packed m x k_full operand starting at row r0 (a multiple of 128) and complex
// column c0 (a multiple of 16)
TcPackedA tc_packed_view(const float *hi, const float *lo, int64_t k_full, int64_t r0, int64_t c0);
// TFLOP/s of kind::tf32 MMAs issued back to back from operand tiles resident in shared memory
// (one CTA per SM, no operand loads): the tensor pipe's own TF32 rate.  Time-outs go to *dev_status.
double tc_mma_probe_tflops(cudaStream_t st, int *dev_status);
// tile walk of a GEMM item with mtc x ntc output tiles and nkt K tiles: 1 down the columns, 0
// along the rows (see tc_gemm.cu)
int tc_tile_order(int mtc, int ntc, int nkt);
// allocation-free variant: packed operands in a static device array (m, n <= 1024, k <= 128);
// waits for `st` and returns the launch's DS_* status bits (0 = ok)
int tc_gemm_complex_noalloc(cudaStream_t st, const cx<float> *A, int64_t lda, const cx<float> *B, int64_t ldb,
                             cx<float> *C, int64_t ldc, int m, int n, int k, double alpha, double beta);
}  // namespace rfdd
