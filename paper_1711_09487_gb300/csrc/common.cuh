// Shared device/host helpers for the RF-DDES GB300 library: complex arithmetic, error
// handling, batched-launch descriptors.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <stdexcept>
#include <atomic>

#include "../../include/rfdd.h"

namespace rfdd {

// ------------------------------------------------------------------------------------
// Errors: every library failure is a C++ exception carrying an rfdd status code; the C-ABI
// layer converts it to the return value and records the message for rfdd_last_error().
// ------------------------------------------------------------------------------------
struct Error : public std::runtime_error {
  int code;
  Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define RFDD_CUDA(call)                                                                    \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::rfdd::Error(RFDD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_) + \
                                          " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"); \
  } while (0)

// Every kernel launch of the library goes through RFDD_CHECK_LAUNCH, which also counts it.
extern std::atomic<long long> g_kernel_launches;
// launches issued by the calling host thread (phases that run on two threads count their own)
extern thread_local long long g_thread_launches;
#define RFDD_CHECK_LAUNCH()                                           \
  do {                                                                \
    ::rfdd::g_kernel_launches.fetch_add(1, std::memory_order_relaxed); \
    ++::rfdd::g_thread_launches;                                      \
    RFDD_CUDA(cudaGetLastError());                                    \
  } while (0)

// Optional CUDA-event timing of the dense contraction kernels (the dominant work of the
// factorisations and triangular solves), enabled through rfdd_profile().
struct ProfileRec {
  cudaEvent_t a, b;
  double flops;   // algorithmic flops of the launch (complex multiply-add = 8 real flops)
  int kind;       // 0: SIMT GEMM, 1: tensor-core GEMM
  double bytes;   // compulsory DRAM bytes of the launch (operands read once, C read and/or written)
};
bool profiling_enabled();
void profile_push(cudaEvent_t a, cudaEvent_t b, double flops, int kind, double bytes = 0.0);
cudaEvent_t profile_event();

#define RFDD_REQUIRE(cond, code, msg)                 \
  do {                                                \
    if (!(cond)) throw ::rfdd::Error((code), (msg));  \
  } while (0)

// ------------------------------------------------------------------------------------
// Complex numbers (interleaved re, im), usable on host and device.
// ------------------------------------------------------------------------------------
template <typename R>
struct cx {
  R re, im;
  __host__ __device__ cx() : re(0), im(0) {}
  __host__ __device__ cx(R r) : re(r), im(0) {}
  __host__ __device__ cx(R r, R i) : re(r), im(i) {}
};

template <typename R> __host__ __device__ inline cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __host__ __device__ inline cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __host__ __device__ inline cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <typename R> __host__ __device__ inline cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __host__ __device__ inline cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }

// Scalar traits so that the dense kernels are written once for float, double, cx<float>,
// cx<double>.
template <typename T> struct ST;
template <> struct ST<float> {
  using real = float;
  static constexpr bool is_complex = false;
  __host__ __device__ static float zero() { return 0.f; }
  __host__ __device__ static float one() { return 1.f; }
  __host__ __device__ static float abs1(float a) { return fabsf(a); }
  __host__ __device__ static float fma(float a, float b, float c) { return fmaf(a, b, c); }   // c + a*b
  __host__ __device__ static float fms(float a, float b, float c) { return fmaf(-a, b, c); }  // c - a*b
  __host__ __device__ static float div(float a, float b) { return a / b; }
  __host__ __device__ static bool finite(float a) { return isfinite(a); }
  __host__ __device__ static float from_re(double a) { return (float)a; }
};
template <> struct ST<double> {
  using real = double;
  static constexpr bool is_complex = false;
  __host__ __device__ static double zero() { return 0.0; }
  __host__ __device__ static double one() { return 1.0; }
  __host__ __device__ static double abs1(double a) { return fabs(a); }
  __host__ __device__ static double fma(double a, double b, double c) { return ::fma(a, b, c); }
  __host__ __device__ static double fms(double a, double b, double c) { return ::fma(-a, b, c); }
  __host__ __device__ static double div(double a, double b) { return a / b; }
  __host__ __device__ static bool finite(double a) { return isfinite(a); }
  __host__ __device__ static double from_re(double a) { return a; }
};
template <typename R> struct STC {
  using T = cx<R>;
  using real = R;
  static constexpr bool is_complex = true;
  __host__ __device__ static T zero() { return T(0, 0); }
  __host__ __device__ static T one() { return T(1, 0); }
  // LAPACK's cabs1 convention for pivot search: |re| + |im|
  __host__ __device__ static R abs1(T a) { return (a.re < 0 ? -a.re : a.re) + (a.im < 0 ? -a.im : a.im); }
  __host__ __device__ static T fma(T a, T b, T c) {  // c + a*b
    T r;
    r.re = c.re + a.re * b.re - a.im * b.im;
    r.im = c.im + a.re * b.im + a.im * b.re;
    return r;
  }
  __host__ __device__ static T fms(T a, T b, T c) {  // c - a*b
    T r;
    r.re = c.re - a.re * b.re + a.im * b.im;
    r.im = c.im - a.re * b.im - a.im * b.re;
    return r;
  }
  __host__ __device__ static T div(T a, T b) {
    // Smith's algorithm for complex division (avoids overflow of |b|^2)
    R ar = b.re < 0 ? -b.re : b.re, ai = b.im < 0 ? -b.im : b.im;
    if (ar >= ai) {
      R r = b.im / b.re, den = b.re + b.im * r;
      return T((a.re + a.im * r) / den, (a.im - a.re * r) / den);
    } else {
      R r = b.re / b.im, den = b.re * r + b.im;
      return T((a.re * r + a.im) / den, (a.im * r - a.re) / den);
    }
  }
  __host__ __device__ static bool finite(T a) { return isfinite(a.re) && isfinite(a.im); }
  __host__ __device__ static T from_re(double a) { return T((R)a, (R)0); }
};
template <> struct ST<cx<float>> : STC<float> {};
template <> struct ST<cx<double>> : STC<double> {};

// ------------------------------------------------------------------------------------
// Device status flags (one int per solve): kernels record failures here instead of trapping.
// ------------------------------------------------------------------------------------
enum DevStatus : int {
  DS_OK = 0,
  DS_ZERO_PIVOT = 1,
  DS_NONFINITE = 2,
  DS_BAD_SIZE = 4,
  DS_WAIT_TIMEOUT = 8,
};

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Sizes that set the device memory of a solve (admission estimates).
struct SolveShape {
  int64_t n = 0, s = 0, nnz = 0;
  int p = 0;
  const int64_t *d = nullptr;  // interior sizes d_j
  const int64_t *D = nullptr;  // bordered sizes D_j = d_j + s_j
  int precision = RFDD_MIXED, keep_schur = 0, min_guard = 8, m_align = 128;
  double guard_frac = 0.3;
  int pack_factors = -1;  // rfdd_options.pack_factors
  size_t mem_budget = 0;
  // two-level interface factorisation: groups (0 = one dense S per node), level-2 size, and per
  // group the level-1 size n1 and the level-2 border n2
  int lv_groups = 0;
  int64_t lv_s2 = 0;
  const int64_t *lv_n1 = nullptr, *lv_n2 = nullptr;
};
// whether the mixed solve keeps tile copies of its factors (rfdd_options.pack_factors)
bool packed_factors(const SolveShape &g, int nc);
size_t factor_bytes_of(const SolveShape &g, int nc);
size_t solve_bytes_of(const SolveShape &g, int nc, int64_t nev_guess, bool with_setup);

}  // namespace rfdd
