// Throughput probes of the arithmetic units the solver's kernels are bound by (measurement hooks,
// no counterpart in the paper): the tensor pipe's TF32 MMA rate (operands resident in shared
// memory), a plain TF32 GEMM through the solver's tensor-core kernel (one MMA per product,
// operands fed from memory), and fused multiply-adds on the CUDA cores in FP64 and FP32.  Each probe is timed with
// CUDA events on its own stream after a warm-up launch; the best of a few launches is returned.
#include <algorithm>
#include <vector>

#include "dense.cuh"
#include "probe.cuh"
#include "tc_gemm.cuh"

namespace rfdd {

constexpr int PROBE_CHAINS = 8;    // independent FMA chains per thread (hide the pipe latency)
constexpr int PROBE_ITERS = 4096;  // steps of each chain

// Every thread runs PROBE_CHAINS independent chains a <- a * x + y; the sum is stored so that the
// work is not removed.  2 * PROBE_CHAINS * PROBE_ITERS flops per thread.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T x, T y, T *out) {
  T a[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = (T)(threadIdx.x + c);
#pragma unroll 16
  for (int i = 0; i < PROBE_ITERS; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = fma(a[c], x, y);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += a[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

namespace {

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    RFDD_CUDA(cudaEventCreate(&a));
    RFDD_CUDA(cudaEventCreate(&b));
  }
  ~EventPair() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

template <typename T>
double fma_probe(cudaStream_t st) {
  int nsm = 0, dev = 0;
  RFDD_CUDA(cudaGetDevice(&dev));
  RFDD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * 8, threads = 256;
  T *out = nullptr;
  RFDD_CUDA(cudaMallocAsync((void **)&out, (size_t)blocks * threads * sizeof(T), st));
  EventPair ev;
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch is a warm-up
    RFDD_CUDA(cudaEventRecord(ev.a, st));
    fma_probe_kernel<T><<<blocks, threads, 0, st>>>((T)0.999999, (T)1e-7, out);
    RFDD_CHECK_LAUNCH();
    RFDD_CUDA(cudaEventRecord(ev.b, st));
    RFDD_CUDA(cudaEventSynchronize(ev.b));
    float ms = 0.f;
    RFDD_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
    const double fl = 2.0 * PROBE_CHAINS * PROBE_ITERS * (double)blocks * threads;
    if (rep > 0 && ms > 0.f) best = std::max(best, fl / (ms * 1e-3) / 1e12);
  }
  RFDD_CUDA(cudaFreeAsync(out, st));
  RFDD_CUDA(cudaStreamSynchronize(st));
  return best;
}

__global__ void fill_probe_kernel(float *x, size_t n, float v) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] = v * (float)((i * 2654435761u) & 1023) / 1024.f;
}

double tf32_probe(cudaStream_t st) {
  constexpr int N = 8192;
  const size_t e = (size_t)N * N;
  float *A = nullptr, *B = nullptr, *C = nullptr;
  RFDD_CUDA(cudaMallocAsync((void **)&A, e * sizeof(float), st));
  RFDD_CUDA(cudaMallocAsync((void **)&B, e * sizeof(float), st));
  RFDD_CUDA(cudaMallocAsync((void **)&C, e * sizeof(float), st));
  fill_probe_kernel<<<1024, 256, 0, st>>>(A, e, 1.f);
  RFDD_CHECK_LAUNCH();
  fill_probe_kernel<<<1024, 256, 0, st>>>(B, e, 0.5f);
  RFDD_CHECK_LAUNCH();
  int *status = nullptr;
  RFDD_CUDA(cudaMallocAsync((void **)&status, sizeof(int), st));
  RFDD_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  std::vector<GemmItem<float>> it = {{A, B, C, N, N, N, N, N, N}};
  double best = 0.0;
  {
    TcStatusScope tcs(status);
    EventPair ev;
    const cudaEvent_t ab[2] = {ev.a, ev.b};
    TcKernelEvents kev(ab);  // the events bracket the MMA kernel, not the operand packing
    for (int rep = 0; rep < 4; ++rep) {
      tc_gemm_real_tf32(st, it, 1.0, 0.0);
      RFDD_CUDA(cudaEventSynchronize(ev.b));
      float ms = 0.f;
      RFDD_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
      if (rep > 0 && ms > 0.f) best = std::max(best, 2.0 * N * (double)N * N / (ms * 1e-3) / 1e12);
    }
  }
  int stt = 0;
  RFDD_CUDA(cudaMemcpyAsync(&stt, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  RFDD_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(A, st);
  cudaFreeAsync(B, st);
  cudaFreeAsync(C, st);
  cudaFreeAsync(status, st);
  RFDD_CUDA(cudaStreamSynchronize(st));
  RFDD_REQUIRE(stt == 0, RFDD_ECUDA, "TF32 probe: tensor-core GEMM reported a time-out");
  return best;
}

double mma_probe(cudaStream_t st) {
  int *status = nullptr;
  RFDD_CUDA(cudaMallocAsync((void **)&status, sizeof(int), st));
  RFDD_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  double r = 0.0;
  try {
    r = tc_mma_probe_tflops(st, status);
  } catch (...) {
    cudaFreeAsync(status, st);
    throw;
  }
  int stt = 0;
  RFDD_CUDA(cudaMemcpyAsync(&stt, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  RFDD_CUDA(cudaFreeAsync(status, st));
  RFDD_CUDA(cudaStreamSynchronize(st));
  RFDD_REQUIRE(stt == 0, RFDD_ECUDA, "MMA probe: a wait timed out");
  return r;
}

}  // namespace

double peak_probe(int which) {
  cudaStream_t st = nullptr;
  RFDD_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  double r = 0.0;
  try {
    if (which == 0) r = mma_probe(st);
    else if (which == 1) r = fma_probe<double>(st);
    else if (which == 2) r = fma_probe<float>(st);
    else if (which == 3) r = tf32_probe(st);
    else throw Error(RFDD_EINVAL, "peak probe: which must be 0..3");
  } catch (...) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    throw;
  }
  RFDD_CUDA(cudaStreamSynchronize(st));
  RFDD_CUDA(cudaStreamDestroy(st));
  return r;
}

}  // namespace rfdd
