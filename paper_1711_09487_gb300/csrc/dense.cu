// Batched dense kernels: SIMT GEMM, blocked LU with tournament (CALU-style) pivoting on
// bordered matrices, triangular solves.  The paper factors B_zeta and S_zeta with sparse
// direct solvers (PARDISO/MUMPS, Section 6); here every shifted block is dense and all
// (subdomain, node) pairs are factored in one batch per step.
#include "dense.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <climits>
#include <mutex>
#include <type_traits>

namespace rfdd {

// ======================================================================================
// GEMM (CUDA cores).  64x64 output tile per CTA, 16-deep K slices staged in shared memory,
// 4x4 outputs per thread.
// ======================================================================================
// Split-K: item i runs nsplit[i] K-chunks of depth kchunk (grid z = item * smax + chunk); with
// nsplit[i] > 1 each chunk writes its unscaled partial tile to ws[i] + chunk * m * n (ld n) and
// splitk_reduce_kernel sums the chunks in order, so the result does not depend on scheduling.
template <typename T>
struct GemmBatchP {
  GemmItem<T> it[MAXB];
  T *ws[MAXB];
  int nsplit[MAXB];
  int smax, kchunk;
  unsigned long long symmask;  // bit i: item i is a symmetric product (upper tiles computed, mirrored)
};

template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_simt_kernel(GemmBatchP<T> batch, typename ST<T>::real alpha,
                                                        typename ST<T>::real beta) {
  using S = ST<T>;
  const int item = blockIdx.z / batch.smax, chunk = blockIdx.z % batch.smax;
  if (chunk >= batch.nsplit[item]) return;
  const GemmItem<T> g = batch.it[item];
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  if (i0 >= g.m || j0 >= g.n) return;
  const bool sym = (batch.symmask >> item) & 1ull;
  if (sym && i0 > j0) return;  // lower tiles are mirrored from the upper ones
  T *const ws = batch.nsplit[item] > 1 ? batch.ws[item] + (int64_t)chunk * g.m * g.n : nullptr;
  const int kb = ws ? chunk * batch.kchunk : 0;
  const int ke = ws ? min(g.k, kb + batch.kchunk) : g.k;
  __shared__ T As[16][65];
  __shared__ T Bs[16][65];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = S::zero();
  for (int k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * 256;
      int ii, kk;
      if (!TA) { kk = e & 15; ii = e >> 4; } else { ii = e & 63; kk = e >> 6; }
      const int gi = i0 + ii, gk = k0 + kk;
      T v = S::zero();
      if (gi < g.m && gk < ke) v = TA ? g.A[(int64_t)gk * g.lda + gi] : g.A[(int64_t)gi * g.lda + gk];
      As[kk][ii] = v;
      int jj, kb;
      if (!TB) { jj = e & 63; kb = e >> 6; } else { kb = e & 15; jj = e >> 4; }
      const int gj = j0 + jj, gkb = k0 + kb;
      T u = S::zero();
      if (gj < g.n && gkb < ke) u = TB ? g.B[(int64_t)gj * g.ldb + gkb] : g.B[(int64_t)gkb * g.ldb + gj];
      Bs[kb][jj] = u;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = S::fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 16 * r;
    if (i >= g.m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx + 16 * c;
      if (j >= g.n) continue;
      if (ws) {
        ws[(int64_t)i * g.n + j] = acc[r][c];
        continue;
      }
      if (sym && i > j) continue;  // diagonal tile: the upper triangle is mirrored below
      T *p = g.C + (int64_t)i * g.ldc + j;
      T v = alpha * acc[r][c];
      if (beta != 0) v = v + beta * (*p);
      *p = v;
      if (sym && i != j) {
        T *q = g.C + (int64_t)j * g.ldc + i;
        T w = alpha * acc[r][c];
        if (beta != 0) w = w + beta * (*q);
        *q = w;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) splitk_reduce_kernel(GemmBatchP<T> batch, typename ST<T>::real alpha,
                                                            typename ST<T>::real beta) {
  const int item = blockIdx.y, ns = batch.nsplit[item];
  if (ns <= 1) return;
  const GemmItem<T> g = batch.it[item];
  const int64_t mn = (int64_t)g.m * g.n;
  const T *ws = batch.ws[item];
  const bool sym = (batch.symmask >> item) & 1ull;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < mn; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / g.n, j = e % g.n;
    // a symmetric product takes its lower triangle from the upper one (exactly symmetric result)
    const int64_t src = (sym && i > j) ? j * g.n + i : e;
    T v = ws[src];
    for (int c = 1; c < ns; ++c) v = v + ws[c * mn + src];
    T *p = g.C + i * g.ldc + j;
    v = alpha * v;
    if (beta != 0) v = v + beta * (*p);
    *p = v;
  }
}

// SM count of the current device (looked up once per device; several host threads may launch)
int sm_count() {
  static std::mutex mu;
  static std::vector<int> nsm;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  if ((int)nsm.size() <= dev) nsm.resize(dev + 1, 0);
  if (nsm[dev] <= 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 148;
    }
    nsm[dev] = v;
  }
  return nsm[dev];
}

// ======================================================================================
// FP64 GEMM in double-FP32 arithmetic.  GB300's FP64 pipes run at a small fraction of FP32, so
// the products on the eigenvector bases (Gram matrices, projections, basis updates) split each
// FP64 operand x into hi = fl32(x), lo = fl32(x - hi) (|x - hi - lo| <= 2^-48 |x|) and form
//   a b ~ ah bh + (ah bl + al bh)
// with ah bh split exactly by an FMA (TwoProduct) and the running sum kept as an unevaluated
// pair (s, c) updated by TwoSum (Knuth, TAOCP Vol. 2, 4.2.2).  Per multiply-add that is 12 FP32
// operations; the result has a relative error near 2^-46 of sum |a_k b_k| instead of 2^-53.
// Same tiling as gemm_simt_kernel (64x64 tile, 16-deep K slices, 4x4 outputs per thread), with
// split-K and symmetric-product support.
// ======================================================================================
__device__ __forceinline__ void split_df(double v, float &hi, float &lo) {
  hi = __double2float_rn(v);
  lo = __double2float_rn(v - (double)hi);
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_df64_kernel(GemmBatchP<double> batch, double alpha, double beta) {
  const int item = blockIdx.z / batch.smax, chunk = blockIdx.z % batch.smax;
  if (chunk >= batch.nsplit[item]) return;
  const GemmItem<double> g = batch.it[item];
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  if (i0 >= g.m || j0 >= g.n) return;
  const bool sym = (batch.symmask >> item) & 1ull;
  if (sym && i0 > j0) return;  // lower tiles are mirrored from the upper ones
  double *const ws = batch.nsplit[item] > 1 ? batch.ws[item] + (int64_t)chunk * g.m * g.n : nullptr;
  const int kb = ws ? chunk * batch.kchunk : 0;
  const int ke = ws ? min(g.k, kb + batch.kchunk) : g.k;
  __shared__ float Ah[16][65], Al[16][65], Bh[16][65], Bl[16][65];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) sh[r][c] = sl[r][c] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * 256;
      int ii, kk;
      if (!TA) { kk = e & 15; ii = e >> 4; } else { ii = e & 63; kk = e >> 6; }
      const int gi = i0 + ii, gk = k0 + kk;
      double v = 0.0;
      if (gi < g.m && gk < ke) v = TA ? g.A[(int64_t)gk * g.lda + gi] : g.A[(int64_t)gi * g.lda + gk];
      split_df(v, Ah[kk][ii], Al[kk][ii]);
      int jj, kq;
      if (!TB) { jj = e & 63; kq = e >> 6; } else { kq = e & 15; jj = e >> 4; }
      const int gj = j0 + jj, gkq = k0 + kq;
      double u = 0.0;
      if (gj < g.n && gkq < ke) u = TB ? g.B[(int64_t)gj * g.ldb + gkq] : g.B[(int64_t)gkq * g.ldb + gj];
      split_df(u, Bh[kq][jj], Bl[kq][jj]);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        ah[r] = Ah[kk][ty + 16 * r];
        al[r] = Al[kk][ty + 16 * r];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        bh[c] = Bh[kk][tx + 16 * c];
        bl[c] = Bl[kk][tx + 16 * c];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          // intrinsics keep the compiler from contracting the error-free transformations
          const float p = __fmul_rn(ah[r], bh[c]);
          const float e = __fmaf_rn(ah[r], bh[c], -p);
          const float t = __fmaf_rn(ah[r], bl[c], __fmaf_rn(al[r], bh[c], e));
          const float s1 = __fadd_rn(sh[r][c], p);
          const float bb = __fsub_rn(s1, sh[r][c]);
          const float err = __fadd_rn(__fsub_rn(sh[r][c], __fsub_rn(s1, bb)), __fsub_rn(p, bb));
          sh[r][c] = s1;
          sl[r][c] = __fadd_rn(sl[r][c], __fadd_rn(err, t));
        }
    }
    // renormalise (FastTwoSum, |sl| << |sh|): the correction term stays near 2^-24 |sh|, so its
    // own rounding errors stay near 2^-48 |sh| per slice
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float s1 = __fadd_rn(sh[r][c], sl[r][c]);
        sl[r][c] = __fsub_rn(sl[r][c], __fsub_rn(s1, sh[r][c]));
        sh[r][c] = s1;
      }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 16 * r;
    if (i >= g.m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx + 16 * c;
      if (j >= g.n) continue;
      const double acc = (double)sh[r][c] + (double)sl[r][c];
      if (ws) {
        ws[(int64_t)i * g.n + j] = acc;
        continue;
      }
      if (sym && i > j) continue;  // diagonal tile: the upper triangle is mirrored below
      double *p = g.C + (int64_t)i * g.ldc + j;
      *p = beta != 0.0 ? alpha * acc + beta * (*p) : alpha * acc;
      if (sym && i != j) {
        double *q = g.C + (int64_t)j * g.ldc + i;
        *q = beta != 0.0 ? alpha * acc + beta * (*q) : alpha * acc;
      }
    }
  }
}

// Shared launch logic of the CUDA-core GEMMs: batching, split-K choice, partial workspace.
template <typename T, typename Launch>
void gemm_launch_batches(cudaStream_t st, const std::vector<GemmItem<T>> &live, const std::vector<char> &symv,
                         double alpha, double beta, Launch &&launch) {
  using R = typename ST<T>::real;
  for (size_t s = 0; s < live.size(); s += MAXB) {
    GemmBatchP<T> b;
    memset(&b, 0, sizeof(b));
    int cnt = (int)std::min<size_t>(MAXB, live.size() - s), mm = 0, nn = 0;
    for (int i = 0; i < cnt; ++i) {
      b.it[i] = live[s + i];
      mm = std::max(mm, b.it[i].m);
      nn = std::max(nn, b.it[i].n);
      if (!symv.empty() && symv[s + i]) {
        RFDD_REQUIRE(b.it[i].m == b.it[i].n, RFDD_EINVAL, "gemm: symmetric product must be square");
        b.symmask |= 1ull << i;
      }
    }
    // Few output tiles over a deep K (Gram matrices, projections on a basis): split K so that
    // about four CTAs per SM have work; chunks no shallower than kmin.
    double work = 0.0;
    for (int i = 0; i < cnt; ++i) {
      const GemmItem<T> &g = b.it[i];
      double tiles = (double)ceil_div(g.m, 64) * ceil_div(g.n, 64);
      if ((b.symmask >> i) & 1ull) tiles = 0.5 * (tiles + ceil_div(g.m, 64));
      work += tiles * std::max(g.k, 1);
    }
    const int kmin = sizeof(R) == 8 ? 128 : 256;
    int kchunk = (int)std::min<double>(2e9, std::ceil(work / (4.0 * sm_count())));
    kchunk = std::max(kmin, (kchunk + 15) / 16 * 16);
    b.smax = 1;
    b.kchunk = kchunk;
    for (int i = 0; i < cnt; ++i) {
      const GemmItem<T> &g = b.it[i];
      b.nsplit[i] = g.k > kchunk ? std::min(64, ceil_div(g.k, kchunk)) : 1;
      // the chunk count cap can leave chunks deeper than kchunk: widen kchunk for all items
      if (b.nsplit[i] > 1) b.kchunk = std::max(b.kchunk, (ceil_div(g.k, b.nsplit[i]) + 15) / 16 * 16);
    }
    size_t wsz = 0;
    for (int i = 0; i < cnt; ++i) {
      const GemmItem<T> &g = b.it[i];
      if (b.nsplit[i] > 1) b.nsplit[i] = ceil_div(g.k, b.kchunk);
      b.smax = std::max(b.smax, b.nsplit[i]);
      if (b.nsplit[i] > 1) wsz += (size_t)b.nsplit[i] * g.m * g.n;
    }
    T *wsbase = nullptr;
    if (wsz) {
      RFDD_CUDA(cudaMallocAsync((void **)&wsbase, wsz * sizeof(T), st));
      size_t o = 0;
      for (int i = 0; i < cnt; ++i)
        if (b.nsplit[i] > 1) {
          b.ws[i] = wsbase + o;
          o += (size_t)b.nsplit[i] * b.it[i].m * b.it[i].n;
        }
    }
    dim3 grid(ceil_div(nn, 64), ceil_div(mm, 64), cnt * b.smax);
    RFDD_REQUIRE(grid.y <= 65535 && grid.z <= 65535, RFDD_EINVAL, "gemm: too many row tiles");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double flops = 0.0;
    if (profiling_enabled()) {
      for (int i = 0; i < cnt; ++i) flops += (ST<T>::is_complex ? 8.0 : 2.0) * b.it[i].m * (double)b.it[i].n * b.it[i].k;
      e0 = profile_event();
      e1 = profile_event();
      cudaEventRecord(e0, st);
    }
    launch(grid, b);
    RFDD_CHECK_LAUNCH();
    if (wsbase) {
      int64_t mnmax = 0;
      for (int i = 0; i < cnt; ++i) mnmax = std::max<int64_t>(mnmax, (int64_t)b.it[i].m * b.it[i].n);
      splitk_reduce_kernel<T><<<dim3((unsigned)std::min<int64_t>(1024, ceil_div(mnmax, 256)), cnt), 256, 0, st>>>(
          b, (R)alpha, (R)beta);
      RFDD_CHECK_LAUNCH();
      RFDD_CUDA(cudaFreeAsync(wsbase, st));
    }
    if (e0) {
      cudaEventRecord(e1, st);
      profile_push(e0, e1, flops, 0);
    }
  }
}

void gemm_f64x2_batched(cudaStream_t st, const std::vector<GemmItem<double>> &items, bool ta, bool tb, double alpha,
                        double beta, const std::vector<char> &sym) {
  std::vector<GemmItem<double>> live;
  std::vector<char> symv;
  for (size_t i = 0; i < items.size(); ++i)
    if (items[i].m > 0 && items[i].n > 0) {
      live.push_back(items[i]);
      symv.push_back(sym.empty() ? 0 : sym[i]);
    }
  gemm_launch_batches<double>(st, live, symv, alpha, beta, [&](dim3 grid, const GemmBatchP<double> &b) {
    if (!ta && !tb) gemm_df64_kernel<false, false><<<grid, 256, 0, st>>>(b, alpha, beta);
    else if (ta && !tb) gemm_df64_kernel<true, false><<<grid, 256, 0, st>>>(b, alpha, beta);
    else if (!ta && tb) gemm_df64_kernel<false, true><<<grid, 256, 0, st>>>(b, alpha, beta);
    else gemm_df64_kernel<true, true><<<grid, 256, 0, st>>>(b, alpha, beta);
  });
}

template <typename T>
void gemm_batched(cudaStream_t st, const std::vector<GemmItem<T>> &items, bool ta, bool tb,
                  double alpha, double beta) {
  if constexpr (std::is_same<T, cx<float>>::value) {
    // complex FP32 products go to the tensor cores (3xTF32 split, FP32 accumulation)
    if (!ta && !tb) {
      std::vector<GemmItem<T>> live;
      for (auto &g : items)
        if (g.m > 0 && g.n > 0 && g.k > 0) live.push_back(g);
      if (!live.empty()) tc_gemm_complex(st, live, alpha, beta);
      // k == 0 items still need C = beta*C
      std::vector<GemmItem<T>> k0;
      for (auto &g : items)
        if (g.m > 0 && g.n > 0 && g.k <= 0 && beta != 1.0) k0.push_back(g);
      if (!k0.empty()) gemm_simt_batched<T>(st, k0, false, false, alpha, beta);
      return;
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    if (!ta && !tb) {
      std::vector<GemmItem<T>> live, k0;
      for (auto &g : items) {
        if (g.m > 0 && g.n > 0 && g.k > 0) live.push_back(g);
        else if (g.m > 0 && g.n > 0 && beta != 1.0) k0.push_back(g);
      }
      if (!live.empty()) tc_gemm_real(st, live, alpha, beta);
      if (!k0.empty()) gemm_simt_batched<T>(st, k0, false, false, alpha, beta);
      return;
    }
  }
  gemm_simt_batched<T>(st, items, ta, tb, alpha, beta);
}

template <typename T>
void gemm_simt_batched(cudaStream_t st, const std::vector<GemmItem<T>> &items, bool ta, bool tb,
                       double alpha, double beta, const std::vector<char> &sym) {
  using R = typename ST<T>::real;
  std::vector<GemmItem<T>> live;
  std::vector<char> symv;
  for (size_t i = 0; i < items.size(); ++i)
    if (items[i].m > 0 && items[i].n > 0) {
      live.push_back(items[i]);
      symv.push_back(sym.empty() ? 0 : sym[i]);
    }
  bool anysym = false;
  for (char c : symv) anysym |= c != 0;
  RFDD_REQUIRE(!anysym || !ST<T>::is_complex, RFDD_EINVAL, "gemm: symmetric products are real only");
  gemm_launch_batches<T>(st, live, symv, alpha, beta, [&](dim3 grid, const GemmBatchP<T> &b) {
    if (!ta && !tb) gemm_simt_kernel<T, false, false><<<grid, 256, 0, st>>>(b, (R)alpha, (R)beta);
    else if (ta && !tb) gemm_simt_kernel<T, true, false><<<grid, 256, 0, st>>>(b, (R)alpha, (R)beta);
    else if (!ta && tb) gemm_simt_kernel<T, false, true><<<grid, 256, 0, st>>>(b, (R)alpha, (R)beta);
    else gemm_simt_kernel<T, true, true><<<grid, 256, 0, st>>>(b, (R)alpha, (R)beta);
  });
}

// ======================================================================================
// LU with tournament pivoting.
// One inner step factors the panel columns [k0, k0+w) of every matrix:
//  (1) tournament: each CTA runs partial pivoting (|re|+|im|, ties to the lower row index)
//      on a chunk of R candidate rows held in shared memory and keeps the w pivot rows it
//      chose; chosen sets are merged G at a time until one set of w rows remains;
//  (2) the w interchanges that bring the winners to rows k0.. are applied to whole rows;
//  (3) the winners' w x w block is factored without pivoting (it reproduces the final round
//      of the tournament) and L21 = A21 U11^{-1} is formed for all rows below, border
//      rows included;
//  (4) U12 = L11^{-1} A12 for the columns of the current outer strip;
//  (5) the strip's trailing columns get A22 -= L21 U12.
// After an outer strip of width nbo is done, its U12 over all trailing columns is solved and
// the whole trailing matrix is updated with one GEMM of depth nbo.
// ======================================================================================
template <typename T>
struct LuBatchP {
  LuItem<T> it[MAXB];
};

constexpr int TOURN_G = 8;   // candidate sets merged per CTA

template <typename T>
struct TournRows {           // rows per tournament CTA (R = G * NB): one per thread
  static constexpr int R = TOURN_G * LU_NB;
};

__device__ inline int strip_end(int K0, int nbo, int dp) { return min(K0 + nbo, dp); }

// number of candidate sets at a given tournament level for a matrix
__device__ inline int tourn_sets(int rows, int R, int level) {
  int n = (rows + R - 1) / R;
  for (int l = 0; l < level; ++l) n = (n + TOURN_G - 1) / TOURN_G;
  return n;
}

// Calls f(std::integral_constant<int, i>) for i = I .. N-1 in order.
template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F &f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// One tournament round of the panel's pivot search.  A CTA takes up to R = G * NB candidate rows of
// the panel's w columns (level 0: a slice of consecutive rows; above it: the winners of G sets of
// the level below), runs LU with partial pivoting on them and emits the pivot rows in the order
// chosen.  Thread i keeps candidate row i in registers for the whole elimination: each step is a
// block-wide argmax of |a_it| over the rows not yet chosen (ties go to the lower row index, so
// the winner does not depend on where a row sits), the winner publishes its row through shared
// memory, and every other row forms its multiplier and rank-1 update in its own registers.  The
// multipliers and updates are the same operations, in the same order, as LU on the gathered
// rows.  Only the row indices leave the CTA.
template <typename T>
__global__ void __launch_bounds__(256) lu_tourn_kernel(LuBatchP<T> lb, int K0, int nbo, int k0, int level,
                                                       const int *__restrict__ cin, int *__restrict__ cout,
                                                       int cand_stride) {
  using S = ST<T>;
  using Rl = typename S::real;
  constexpr int NB = LU_NB;
  constexpr int R = TournRows<T>::R;
  static_assert(R == 256, "one candidate row per thread of a 256-thread CTA");
  const LuItem<T> it = lb.it[blockIdx.y];
  const int wend = strip_end(K0, nbo, it.dp);
  const int w = min(NB, wend - k0);
  if (w <= 0) return;
  const int rows_total = it.dp - k0;
  const int set = blockIdx.x;
  if (set >= tourn_sets(rows_total, R, level)) return;
  __shared__ T prow[NB];
  __shared__ Rl red_v[R / 32];
  __shared__ int red_r[R / 32];
  const int tid = threadIdx.x;
  int my = -1;  // global index of this thread's candidate row; -1 when it has none (or it was chosen)
  if (level == 0) {
    const int r = k0 + set * R + tid;
    if (r < it.dp) my = r;
  } else {
    const int *c = cin + (int64_t)blockIdx.y * cand_stride + (int64_t)set * TOURN_G * NB;
    const int nsets_in = tourn_sets(rows_total, R, level - 1);
    const int nin = min(TOURN_G, nsets_in - set * TOURN_G) * NB;
    if (tid < nin) my = c[tid];  // empty slots hold -1
  }
  T row[NB];
  {
    const T *src = it.A + (int64_t)(my >= 0 ? my : 0) * it.ld + k0;
#pragma unroll
    for (int c = 0; c < NB; ++c) row[c] = (my >= 0 && c < w) ? src[c] : S::zero();
  }
  int *o = cout + (int64_t)blockIdx.y * cand_stride + (int64_t)set * NB;
  int steps = 0;
  bool live = true;  // false once the panel's w columns or the candidate rows are used up
  // step t of the elimination, t a compile-time constant so that row[] stays in registers
  auto step = [&](auto tc) {
    constexpr int t = decltype(tc)::value;
    if (!live || t >= w) { live = false; return; }
    Rl v = (Rl)-1;
    int r = INT_MAX;
    if (my >= 0) {
      v = S::abs1(row[t]);
      if (v != v) v = (Rl)INFINITY;  // a NaN row still counts as a candidate
      r = my;
    }
    for (int off = 16; off > 0; off >>= 1) {
      const Rl v2 = __shfl_xor_sync(0xffffffffu, v, off);
      const int r2 = __shfl_xor_sync(0xffffffffu, r, off);
      if (v2 > v || (v2 == v && r2 < r)) { v = v2; r = r2; }
    }
    if ((tid & 31) == 0) { red_v[tid >> 5] = v; red_r[tid >> 5] = r; }
    __syncthreads();
    v = red_v[0];
    r = red_r[0];
#pragma unroll
    for (int q = 1; q < R / 32; ++q)
      if (red_v[q] > v || (red_v[q] == v && red_r[q] < r)) { v = red_v[q]; r = red_r[q]; }
    if (v < (Rl)0) { live = false; return; }  // no row left: the same decision in every thread
    if (my == r) {
#pragma unroll
      for (int c = t; c < NB; ++c) prow[c] = row[c];
      o[t] = my;
      my = -1;
    }
    ++steps;
    __syncthreads();
    if (my >= 0) {
      const T pv = prow[t];
      if (S::abs1(pv) != (Rl)0) {
        const T l = S::div(row[t], pv);
#pragma unroll
        for (int c = t + 1; c < NB; ++c)
          if (c < w) row[c] = S::fms(l, prow[c], row[c]);
      }
    }
  };
  static_for<0, NB>(step);
  for (int t = steps + tid; t < NB; t += blockDim.x) o[t] = -1;
}

// The panel's interchanges, once per item: LAPACK-style pivots into it.piv, and their composition
// as a permutation of the touched rows, perm = [n, key[0..2NB), val[0..2NB)]: row position
// key[i] receives original row val[i].
template <typename T>
__global__ void __launch_bounds__(32) lu_perm_kernel(LuBatchP<T> lb, int K0, int nbo, int k0,
                                                     const int *__restrict__ cfinal, int cand_stride,
                                                     int *__restrict__ perm) {
  constexpr int NB = LU_NB;
  const LuItem<T> it = lb.it[blockIdx.x];
  const int wend = strip_end(K0, nbo, it.dp);
  const int w = min(NB, wend - k0);
  if (w <= 0) return;
  // one warp: the map (key -> val) lives in shared memory, entry i with lanes i and i - 32
  __shared__ int key[2 * NB], val[2 * NB];
  const int lane = threadIdx.x;
  const unsigned full = 0xffffffffu;
  const int *pr = cfinal + (int64_t)blockIdx.x * cand_stride;
  int nk = 0;
  // the entry whose field equals v (keys and values are each distinct), or -1
  auto find = [&](const int *f, int v) {
    int at = -1;
    for (int i0 = 0; i0 < nk; i0 += 32) {
      const int i = i0 + lane;
      const unsigned m = __ballot_sync(full, i < nk && f[i] == v);
      if (m) { at = i0 + __ffs(m) - 1; break; }
    }
    return at;
  };
  for (int t = 0; t < w; ++t) {
    const int target = pr[t];
    const int iq = find(val, target);
    const int q = iq >= 0 ? key[iq] : target;
    if (lane == 0) it.piv[k0 + t] = q;
    const int pa = k0 + t;
    const int ia = find(key, pa), ib = find(key, q);
    const int ra = ia >= 0 ? val[ia] : pa, rb = ib >= 0 ? val[ib] : q;
    __syncwarp();
    if (lane == 0) {
      if (ia >= 0) val[ia] = rb;
      if (ib >= 0 && ib != ia) val[ib] = ra;
      int n = nk;
      if (ia < 0) { key[n] = pa; val[n] = rb; ++n; }
      if (ib < 0 && q != pa) { key[n] = q; val[n] = ra; ++n; }
    }
    nk += (ia < 0 ? 1 : 0) + (ib < 0 && q != pa ? 1 : 0);
    __syncwarp();
  }
  int *pm = perm + (int64_t)blockIdx.x * (1 + 4 * NB);
  if (lane == 0) pm[0] = nk;
  for (int i = lane; i < nk; i += 32) {
    pm[1 + i] = key[i];
    pm[1 + 2 * NB + i] = val[i];
  }
}

// Interchanges on whole rows: each thread moves one column of the touched rows, all of its
// source values first (independent loads), then all of its destinations.
template <typename T>
__global__ void __launch_bounds__(256) lu_swap_kernel(LuBatchP<T> lb, int K0, int nbo, int k0,
                                                      const int *__restrict__ perm) {
  constexpr int NB = LU_NB;
  const LuItem<T> it = lb.it[blockIdx.y];
  const int wend = strip_end(K0, nbo, it.dp);
  const int w = min(NB, wend - k0);
  if (w <= 0) return;
  __shared__ int pkey[2 * NB], pval[2 * NB];
  __shared__ int pn;
  const int *pm = perm + (int64_t)blockIdx.y * (1 + 4 * NB);
  if (threadIdx.x == 0) pn = pm[0];
  for (int i = threadIdx.x; i < 2 * NB; i += blockDim.x) {
    pkey[i] = pm[1 + i];
    pval[i] = pm[1 + 2 * NB + i];
  }
  __syncthreads();
  const int n = pn;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= it.D || n == 0) return;
  constexpr int CH = sizeof(T) <= 8 ? 2 * NB : 16;  // values held in registers at once
  if (n <= CH) {
    T x[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i)
      if (i < n) x[i] = it.A[(int64_t)pval[i] * it.ld + c];
#pragma unroll
    for (int i = 0; i < CH; ++i)
      if (i < n) it.A[(int64_t)pkey[i] * it.ld + c] = x[i];
    return;
  }
  // more touched rows than registers (complex FP64): the interchanges one after another, in the
  // order of the LAPACK-style pivots that lu_perm_kernel stored
  for (int t = 0; t < w; ++t) {
    const int q = it.piv[k0 + t];
    if (q != k0 + t) {
      T *a = it.A + (int64_t)(k0 + t) * it.ld + c;
      T *b = it.A + (int64_t)q * it.ld + c;
      T x = *a;
      *a = *b;
      *b = x;
    }
  }
}

// LU without pivoting of the w x w diagonal block of the panel (its rows are the tournament's
// pivots, already in place), once per item: the combined L\U block into top (NB x NB, leading
// dimension w) and the reciprocals of U's diagonal after it (NB entries); zero or non-finite
// pivots are recorded in status.
template <typename T>
__global__ void __launch_bounds__(256) lu_diag_kernel(LuBatchP<T> lb, int K0, int nbo, int k0, T *top, int *status) {
  using S = ST<T>;
  using Rl = typename S::real;
  constexpr int NB = LU_NB;
  const LuItem<T> it = lb.it[blockIdx.y];
  const int wend = strip_end(K0, nbo, it.dp);
  const int w = min(NB, wend - k0);
  if (w <= 0) return;
  __shared__ T U[NB][NB + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int r = e / w, c = e % w;
    U[r][c] = it.A[(int64_t)(k0 + r) * it.ld + k0 + c];
  }
  __syncthreads();
  for (int t = 0; t < w; ++t) {
    const T pv = U[t][t];
    const bool nz = S::abs1(pv) != (Rl)0;
    if (nz)
      for (int r = t + 1 + tid; r < w; r += blockDim.x) U[r][t] = S::div(U[r][t], pv);
    __syncthreads();
    const int c = tid & 31;
    if (nz && c > t && c < w)
      for (int r = t + 1 + (tid >> 5); r < w; r += (int)(blockDim.x >> 5)) U[r][c] = S::fms(U[r][t], U[t][c], U[r][c]);
    __syncthreads();
  }
  T *tp = top + (int64_t)blockIdx.y * (NB * NB + NB);
  for (int e = tid; e < w * w; e += blockDim.x) tp[e] = U[e / w][e % w];
  if (tid < w) {
    const T d = U[tid][tid];
    tp[NB * NB + tid] = S::abs1(d) != (Rl)0 ? S::div(S::one(), d) : S::one();
    if (!S::finite(d)) atomicOr(status, DS_NONFINITE);
    else if (S::abs1(d) == (Rl)0) atomicOr(status, DS_ZERO_PIVOT);
  }
}

// L21 = A21 U11^{-1} for the rows below the panel's diagonal block, one thread per row, with the
// diagonal block's factors from lu_diag_kernel.  Each warp moves its 32 rows' panel columns
// through shared memory so that global loads and stores run along the rows (coalesced).
constexpr int FIN_THREADS = 128;
template <typename T>
__global__ void __launch_bounds__(FIN_THREADS) lu_finish_kernel(LuBatchP<T> lb, int K0, int nbo, int k0,
                                                                const T *top) {
  using S = ST<T>;
  constexpr int NB = LU_NB;
  const LuItem<T> it = lb.it[blockIdx.y];
  const int wend = strip_end(K0, nbo, it.dp);
  const int w = min(NB, wend - k0);
  if (w <= 0) return;
  __shared__ T U[NB][NB + 1];
  __shared__ T rdiag[NB];
  __shared__ T stage[FIN_THREADS / 32][32][NB + 1];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const T *tp = top + (int64_t)blockIdx.y * (NB * NB + NB);
  for (int e = tid; e < w * w; e += blockDim.x) U[e / w][e % w] = tp[e];
  if (tid < w) rdiag[tid] = tp[NB * NB + tid];
  const int rbase = k0 + w + blockIdx.x * blockDim.x + wid * 32;  // first row of this warp
  T(*st)[NB + 1] = stage[wid];
  for (int rr = 0; rr < 32; ++rr)
    if (rbase + rr < it.D && lane < w) st[rr][lane] = it.A[(int64_t)(rbase + rr) * it.ld + k0 + lane];
  __syncthreads();  // U, rdiag and every warp's rows
  const bool mine = rbase + lane < it.D;
  T x[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c)
    if (c < w && mine) x[c] = st[lane][c];
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c < w && mine) {
      T v = x[c];
#pragma unroll
      for (int t = 0; t < NB; ++t)
        if (t < c) v = S::fms(x[t], U[t][c], v);
      x[c] = v * rdiag[c];
    }
  }
#pragma unroll
  for (int c = 0; c < NB; ++c)
    if (c < w && mine) st[lane][c] = x[c];
  __syncwarp();
  for (int rr = 0; rr < 32; ++rr)
    if (rbase + rr < it.D && lane < w) it.A[(int64_t)(rbase + rr) * it.ld + k0 + lane] = st[rr][lane];
}

template <typename T>
__global__ void __launch_bounds__(256) lu_u12_kernel(LuBatchP<T> lb, int K0, int nbo, int k0,
                                                     const T *__restrict__ top) {
  using S = ST<T>;
  constexpr int NB = LU_NB;
  const LuItem<T> it = lb.it[blockIdx.y];
  const int wend = strip_end(K0, nbo, it.dp);
  const int w = min(NB, wend - k0);
  if (w <= 0) return;
  __shared__ T L[NB][NB + 1];
  const T *tp = top + (int64_t)blockIdx.y * (NB * NB + NB);
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) L[e / w][e % w] = tp[e];
  __syncthreads();
  if (blockIdx.x == 0)
    for (int e = threadIdx.x; e < w * w; e += blockDim.x)
      it.A[(int64_t)(k0 + e / w) * it.ld + k0 + e % w] = L[e / w][e % w];
  const int c = k0 + w + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= wend) return;
  T x[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t)
    if (t < w) x[t] = it.A[(int64_t)(k0 + t) * it.ld + c];
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    if (t < w) {
      T v = x[t];
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q < t) v = S::fms(L[t][q], x[q], v);
      x[t] = v;
    }
  }
#pragma unroll
  for (int t = 0; t < NB; ++t)
    if (t < w) it.A[(int64_t)(k0 + t) * it.ld + c] = x[t];
}

// ======================================================================================
// Triangular solves on 32-row diagonal blocks (thread per right-hand-side column).
// ======================================================================================
template <typename T>
struct TriItem {
  const T *L;   // top-left of the w x w diagonal block
  int ldl;
  T *X;         // first row of the w-row slab of right-hand sides
  int ldx;
  int w, ncols;
};
template <typename T>
struct TriBatchP {
  TriItem<T> it[MAXB];
};

template <typename T, bool UPPER>
__global__ void __launch_bounds__(256) trsm_diag_kernel(TriBatchP<T> tb) {
  using S = ST<T>;
  using Rl = typename S::real;
  constexpr int NB = LU_NB;
  const TriItem<T> it = tb.it[blockIdx.y];
  __shared__ T L[NB][NB + 1];
  __shared__ T rdiag[NB];
  const int w = it.w;
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) L[e / w][e % w] = it.L[(int64_t)(e / w) * it.ldl + e % w];
  if (UPPER && threadIdx.x < w) {
    const T d = it.L[(int64_t)threadIdx.x * it.ldl + threadIdx.x];
    rdiag[threadIdx.x] = S::abs1(d) != (Rl)0 ? S::div(S::one(), d) : S::one();
  }
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= it.ncols) return;
  T x[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t)
    if (t < w) x[t] = it.X[(int64_t)t * it.ldx + c];
  if (!UPPER) {
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      if (t < w) {
        T v = x[t];
#pragma unroll
        for (int q = 0; q < NB; ++q)
          if (q < t) v = S::fms(L[t][q], x[q], v);
        x[t] = v;
      }
    }
  } else {
#pragma unroll
    for (int t = NB - 1; t >= 0; --t) {
      if (t < w) {
        T v = x[t];
#pragma unroll
        for (int q = 0; q < NB; ++q)
          if (q > t && q < w) v = S::fms(L[t][q], x[q], v);
        x[t] = v * rdiag[t];
      }
    }
  }
#pragma unroll
  for (int t = 0; t < NB; ++t)
    if (t < w) it.X[(int64_t)t * it.ldx + c] = x[t];
}

template <typename T, bool UPPER>
static void launch_trsm_diag(cudaStream_t st, const std::vector<TriItem<T>> &items) {
  for (size_t s = 0; s < items.size(); s += MAXB) {
    TriBatchP<T> b;
    memset(&b, 0, sizeof(b));
    int cnt = (int)std::min<size_t>(MAXB, items.size() - s), nc = 1;
    for (int i = 0; i < cnt; ++i) { b.it[i] = items[s + i]; nc = std::max(nc, b.it[i].ncols); }
    trsm_diag_kernel<T, UPPER><<<dim3(ceil_div(nc, 256), cnt), 256, 0, st>>>(b);
    RFDD_CHECK_LAUNCH();
  }
}

// ======================================================================================
// Pivot application to right-hand sides (row interchanges in order, thread per column).
// ======================================================================================
template <typename T>
struct PivItem {
  const int *piv;
  int npiv;
  T *X;
  int ldx, ncols;
};
template <typename T>
struct PivBatchP {
  PivItem<T> it[MAXB];
};

template <typename T>
__global__ void __launch_bounds__(256) apply_piv_kernel(PivBatchP<T> pb) {
  const PivItem<T> it = pb.it[blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= it.ncols) return;
  for (int t = 0; t < it.npiv; ++t) {
    const int q = __ldg(it.piv + t);
    if (q != t) {
      T *a = it.X + (int64_t)t * it.ldx + c;
      T *b = it.X + (int64_t)q * it.ldx + c;
      T x = *a;
      *a = *b;
      *b = x;
    }
  }
}

// ======================================================================================
// Host drivers
// ======================================================================================
template <typename T>
static void launch_lu_common(cudaStream_t st, const std::vector<LuItem<T>> &items, int K0, int nbo,
                             int k0, LuWork &wk, int *perm, int *status) {
  constexpr int NB = LU_NB;
  constexpr int R = TournRows<T>::R;
  for (size_t s = 0; s < items.size(); s += MAXB) {
    LuBatchP<T> b;
    memset(&b, 0, sizeof(b));
    const int cnt = (int)std::min<size_t>(MAXB, items.size() - s);
    int rows_max = 0, dmax = 0, wmax = 0;
    for (int i = 0; i < cnt; ++i) {
      b.it[i] = items[s + i];
      rows_max = std::max(rows_max, b.it[i].dp - k0);
      dmax = std::max(dmax, b.it[i].D);
      wmax = std::max(wmax, std::min(NB, std::min(K0 + nbo, b.it[i].dp) - k0));
    }
    if (rows_max <= 0 || wmax <= 0) continue;
    const int stride = (int)(wk.cand_ints / (2 * MAXB));
    int *ca = wk.cand, *cb = wk.cand + (size_t)MAXB * stride;
    // (1) tournament
    int nsets = ceil_div(rows_max, R);
    lu_tourn_kernel<T><<<dim3(nsets, cnt), R, 0, st>>>(b, K0, nbo, k0, 0, nullptr, ca, stride);
    RFDD_CHECK_LAUNCH();
    int level = 0;
    while (nsets > 1) {
      ++level;
      nsets = ceil_div(nsets, TOURN_G);
      lu_tourn_kernel<T><<<dim3(nsets, cnt), R, 0, st>>>(b, K0, nbo, k0, level, ca, cb, stride);
      RFDD_CHECK_LAUNCH();
      std::swap(ca, cb);
    }
    // (2) interchanges on whole rows
    lu_perm_kernel<T><<<cnt, 32, 0, st>>>(b, K0, nbo, k0, ca, stride, perm);
    RFDD_CHECK_LAUNCH();
    lu_swap_kernel<T><<<dim3(ceil_div(dmax, 256), cnt), 256, 0, st>>>(b, K0, nbo, k0, perm);
    RFDD_CHECK_LAUNCH();
    // (3) U11/L11 once per item, then L21
    lu_diag_kernel<T><<<dim3(1, cnt), 256, 0, st>>>(b, K0, nbo, k0, (T *)wk.top, status);
    RFDD_CHECK_LAUNCH();
    lu_finish_kernel<T><<<dim3(std::max(1, ceil_div(dmax - k0 - 1, FIN_THREADS)), cnt), FIN_THREADS, 0, st>>>(
        b, K0, nbo, k0, (const T *)wk.top);
    RFDD_CHECK_LAUNCH();
    // (4) U12 inside the strip (also stores L11/U11 into the matrix)
    lu_u12_kernel<T><<<dim3(std::max(1, ceil_div(nbo, 256)), cnt), 256, 0, st>>>(b, K0, nbo, k0,
                                                                                (const T *)wk.top);
    RFDD_CHECK_LAUNCH();
  }
  // (5) strip-internal trailing update
  std::vector<GemmItem<T>> g;
  for (auto &it : items) {
    const int wend = std::min(K0 + nbo, it.dp);
    const int w = std::min(NB, wend - k0);
    if (w <= 0) continue;
    GemmItem<T> x;
    x.A = it.A + (int64_t)(k0 + w) * it.ld + k0;
    x.B = it.A + (int64_t)k0 * it.ld + k0 + w;
    x.C = it.A + (int64_t)(k0 + w) * it.ld + k0 + w;
    x.m = it.D - k0 - w;
    x.n = wend - k0 - w;
    x.k = w;
    x.lda = x.ldb = x.ldc = it.ld;
    g.push_back(x);
  }
  gemm_batched<T>(st, g, false, false, -1.0, 1.0);
}

template <typename T>
void lu_batched(cudaStream_t st, const std::vector<LuItem<T>> &items, int nbo, int *dev_status) {
  constexpr int NB = LU_NB;
  constexpr int R = TournRows<T>::R;
  RFDD_REQUIRE(nbo % NB == 0 && nbo > 0, RFDD_EINVAL, "lu: outer block must be a multiple of 32");
  if (items.empty()) return;
  int dpmax = 0;
  for (auto &it : items) {
    RFDD_REQUIRE(it.dp >= 0 && it.D >= it.dp && it.ld >= it.D, RFDD_EINVAL, "lu: bad sizes");
    dpmax = std::max(dpmax, it.dp);
  }
  if (dpmax == 0) return;
  LuWork wk;
  const int stride = (ceil_div(dpmax, R) + 1) * NB;
  wk.cand_ints = (size_t)2 * MAXB * stride;
  wk.top_bytes = (size_t)MAXB * (NB * NB + NB) * sizeof(T);
  RFDD_CUDA(cudaMallocAsync((void **)&wk.cand, wk.cand_ints * sizeof(int), st));
  RFDD_CUDA(cudaMallocAsync(&wk.top, wk.top_bytes, st));
  int *perm = nullptr;  // composed interchanges of each item's panel (lu_perm_kernel)
  RFDD_CUDA(cudaMallocAsync((void **)&perm, (size_t)MAXB * (1 + 4 * NB) * sizeof(int), st));
  try {
    for (int K0 = 0; K0 < dpmax; K0 += nbo) {
      std::vector<LuItem<T>> act;
      for (auto &it : items)
        if (it.dp > K0) act.push_back(it);
      for (int k0 = K0; k0 < K0 + nbo && k0 < dpmax; k0 += NB) {
        std::vector<LuItem<T>> in;
        for (auto &it : act)
          if (std::min(K0 + nbo, it.dp) > k0) in.push_back(it);
        if (!in.empty()) launch_lu_common<T>(st, in, K0, nbo, k0, wk, perm, dev_status);
      }
      // outer strip: U12 over all trailing columns, then the deep trailing update
      std::vector<SolveItem<T>> tri;
      std::vector<GemmItem<T>> g;
      for (auto &it : act) {
        const int wend = std::min(K0 + nbo, it.dp);
        const int wo = wend - K0;
        const int nc = it.D - wend;
        if (wo <= 0 || nc <= 0) continue;
        SolveItem<T> s;
        s.LU = it.A + (int64_t)K0 * it.ld + K0;
        s.piv = nullptr;
        s.n = wo;
        s.ld = it.ld;
        s.X = it.A + (int64_t)K0 * it.ld + wend;
        s.ldx = it.ld;
        s.ncols = nc;
        tri.push_back(s);
        GemmItem<T> x;
        x.A = it.A + (int64_t)wend * it.ld + K0;
        x.B = it.A + (int64_t)K0 * it.ld + wend;
        x.C = it.A + (int64_t)wend * it.ld + wend;
        x.m = it.D - wend;
        x.n = nc;
        x.k = wo;
        x.lda = x.ldb = x.ldc = it.ld;
        g.push_back(x);
      }
      // U12 = L11^{-1} A12 over all trailing columns: invert the strip's unit lower block (small
      // substitution on identity), then one deep product instead of nbo/32 shallow ones
      if (!tri.empty()) {
        T *inv = nullptr;
        RFDD_CUDA(cudaMallocAsync((void **)&inv, tri.size() * (size_t)nbo * nbo * sizeof(T), st));
        std::vector<T *> li(tri.size()), ui(tri.size(), nullptr);
        for (size_t i = 0; i < tri.size(); ++i) li[i] = inv + i * (size_t)nbo * nbo;
        lu_block_inverses<T>(st, tri, nbo, li, ui);
        for (size_t i = 0; i < tri.size(); ++i) {
          tri[i].Linv = li[i];
          tri[i].nbi = nbo;
        }
        trsm_lower_unit<T>(st, tri, nbo);
        RFDD_CUDA(cudaFreeAsync(inv, st));
      }
      gemm_batched<T>(st, g, false, false, -1.0, 1.0);
    }
  } catch (...) {
    cudaFreeAsync(wk.cand, st);
    cudaFreeAsync(wk.top, st);
    cudaFreeAsync(perm, st);
    throw;
  }
  RFDD_CUDA(cudaFreeAsync(wk.cand, st));
  RFDD_CUDA(cudaFreeAsync(wk.top, st));
  RFDD_CUDA(cudaFreeAsync(perm, st));
}

template <typename T>
void apply_pivots(cudaStream_t st, const std::vector<SolveItem<T>> &items) {
  for (size_t s = 0; s < items.size(); s += MAXB) {
    PivBatchP<T> b;
    memset(&b, 0, sizeof(b));
    int cnt = (int)std::min<size_t>(MAXB, items.size() - s), nc = 1;
    for (int i = 0; i < cnt; ++i) {
      const auto &it = items[s + i];
      b.it[i].piv = it.piv;
      b.it[i].npiv = it.n;
      b.it[i].X = it.X;
      b.it[i].ldx = it.ldx;
      b.it[i].ncols = it.ncols;
      nc = std::max(nc, it.ncols);
    }
    apply_piv_kernel<T><<<dim3(ceil_div(nc, 256), cnt), 256, 0, st>>>(b);
    RFDD_CHECK_LAUNCH();
  }
}

// ======================================================================================
// Triangular solves with inverted diagonal blocks: per nbo-block, X_b <- inv(T_bb) X_b as one
// product into a scratch slab copied back, then the deep update of the rows still to solve.
// ======================================================================================
template <typename T>
struct CopyItem {
  const T *src;
  T *dst;
  int lds, ldd, rows, cols;
};
template <typename T>
struct CopyBatchP {
  CopyItem<T> it[MAXB];
};
template <typename T>
__global__ void copy_rows_batched_kernel(CopyBatchP<T> b) {
  const CopyItem<T> c = b.it[blockIdx.y];
  const int64_t tot = (int64_t)c.rows * c.cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / c.cols, q = e % c.cols;
    c.dst[r * c.ldd + q] = c.src[r * c.lds + q];
  }
}
template <typename T>
static void copy_rows_batched(cudaStream_t st, const std::vector<CopyItem<T>> &items) {
  for (size_t s = 0; s < items.size(); s += MAXB) {
    CopyBatchP<T> b;
    memset(&b, 0, sizeof(b));
    const int cnt = (int)std::min<size_t>(MAXB, items.size() - s);
    int64_t mx = 1;
    for (int i = 0; i < cnt; ++i) {
      b.it[i] = items[s + i];
      mx = std::max<int64_t>(mx, (int64_t)b.it[i].rows * b.it[i].cols);
    }
    copy_rows_batched_kernel<T><<<dim3((unsigned)std::min<int64_t>(ceil_div(mx, 256), 1024), cnt), 256, 0, st>>>(b);
    RFDD_CHECK_LAUNCH();
  }
}

template <typename T>
__global__ void identity_blocks_kernel(T *base, int64_t nblk, int nbi) {
  const int64_t tot = nblk * nbi * nbi;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = e % ((int64_t)nbi * nbi);
    base[e] = (w / nbi == w % nbi) ? ST<T>::one() : ST<T>::zero();
  }
}

template <typename T>
void trsm_lower_unit(cudaStream_t st, const std::vector<SolveItem<T>> &items, int nbo);
template <typename T>
void trsm_upper(cudaStream_t st, const std::vector<SolveItem<T>> &items, int nbo);

template <typename T>
void lu_block_inverses(cudaStream_t st, const std::vector<SolveItem<T>> &items, int nbi, const std::vector<T *> &Linv,
                       const std::vector<T *> &Uinv) {
  for (int which = 0; which < 2; ++which) {
    const std::vector<T *> &inv = which == 0 ? Linv : Uinv;
    std::vector<SolveItem<T>> bl;
    for (size_t i = 0; i < items.size(); ++i) {
      if (!inv[i] || items[i].n <= 0) continue;
      const SolveItem<T> &it = items[i];
      const int64_t nblk = ceil_div(it.n, nbi);
      identity_blocks_kernel<T><<<(unsigned)std::min<int64_t>(ceil_div(nblk * nbi * nbi, 256), 4096), 256, 0, st>>>(
          inv[i], nblk, nbi);
      RFDD_CHECK_LAUNCH();
      for (int64_t b = 0; b < nblk; ++b) {
        const int k0 = (int)(b * nbi), w = std::min(nbi, it.n - k0);
        SolveItem<T> x;
        x.LU = it.LU + (int64_t)k0 * it.ld + k0;
        x.piv = nullptr;
        x.n = w;
        x.ld = it.ld;
        x.X = inv[i] + b * nbi * nbi;
        x.ldx = nbi;
        x.ncols = w;
        bl.push_back(x);
      }
    }
    if (bl.empty()) continue;
    if (which == 0) trsm_lower_unit<T>(st, bl, nbi);
    else trsm_upper<T>(st, bl, nbi);
  }
}

template <typename T>
static bool has_block_inverses(const std::vector<SolveItem<T>> &items, int nbo, bool upper) {
  if (items.empty()) return false;
  for (auto &it : items)
    if ((upper ? it.Uinv : it.Linv) == nullptr || it.nbi != nbo) return false;
  return true;
}

// upper = false: X <- L^{-1} X (blocks top to bottom); true: X <- U^{-1} X (bottom to top)
template <typename T>
static void trsm_block_inverse(cudaStream_t st, const std::vector<SolveItem<T>> &items, int nbo, bool upper) {
  // Each block step forms t_b = inv_b x_b into a full-height copy t of X and updates the other
  // rows from t_b; X takes t in one copy at the end (instead of one small copy per block step).
  int nmax = 0;
  size_t tmp_elems = 0;
  std::vector<size_t> toff(items.size());
  for (size_t i = 0; i < items.size(); ++i) {
    nmax = std::max(nmax, items[i].n);
    toff[i] = tmp_elems;
    tmp_elems += (size_t)std::max(items[i].n, 0) * std::max(items[i].ncols, 0);
  }
  if (nmax == 0 || tmp_elems == 0) return;
  T *tmp = nullptr;
  RFDD_CUDA(cudaMallocAsync((void **)&tmp, tmp_elems * sizeof(T), st));
  const int nblk = ceil_div(nmax, nbo);
  for (int step = 0; step < nblk; ++step) {
    const int b = upper ? nblk - 1 - step : step;
    const int K0 = b * nbo;
    std::vector<GemmItem<T>> g1, g2;
    std::vector<TcPackedA> p1, p2;
    for (size_t i = 0; i < items.size(); ++i) {
      const SolveItem<T> &it = items[i];
      if (K0 >= it.n || it.ncols <= 0) continue;
      const int w = std::min(nbo, it.n - K0);
      const T *inv = (upper ? it.Uinv : it.Linv) + (int64_t)b * nbo * nbo;
      T *xb = it.X + (int64_t)K0 * it.ldx, *t = tmp + toff[i] + (int64_t)K0 * it.ncols;
      g1.push_back({inv, xb, t, w, it.ncols, w, nbo, it.ldx, it.ncols});
      const float *ih = upper ? it.Uinvp_hi : it.Linvp_hi, *il = upper ? it.Uinvp_lo : it.Linvp_lo;
      const int64_t bf = tc_packed_a_floats(nbo, nbo);
      p1.push_back(ih ? TcPackedA{ih + b * bf, il + b * bf, tc_packed_a_ktiles(nbo)} : TcPackedA{});
      if (!upper && it.n - K0 - w > 0) {  // rows below: X[K0+w:] -= L[K0+w:, K0:K0+w] t_b
        g2.push_back({it.LU + (int64_t)(K0 + w) * it.ld + K0, t, it.X + (int64_t)(K0 + w) * it.ldx, it.n - K0 - w,
                      it.ncols, w, it.ld, it.ncols, it.ldx});
        p2.push_back(it.LUp_hi ? tc_packed_view(it.LUp_hi, it.LUp_lo, it.n, K0 + w, K0) : TcPackedA{});
      }
      if (upper && K0 > 0) {  // rows above: X[0:K0] -= U[0:K0, K0:K0+w] t_b
        g2.push_back({it.LU + K0, t, it.X, K0, it.ncols, w, it.ld, it.ncols, it.ldx});
        p2.push_back(it.LUp_hi ? tc_packed_view(it.LUp_hi, it.LUp_lo, it.n, 0, K0) : TcPackedA{});
      }
    }
    bool use_pa = false;
    if constexpr (std::is_same<T, cx<float>>::value) use_pa = true;
    if (use_pa) {
      if constexpr (std::is_same<T, cx<float>>::value) {
        tc_gemm_complex_pa(st, g1, p1, 1.0, 0.0);
        tc_gemm_complex_pa(st, g2, p2, -1.0, 1.0);
      }
    } else {
      gemm_batched<T>(st, g1, false, false, 1.0, 0.0);
      gemm_batched<T>(st, g2, false, false, -1.0, 1.0);
    }
  }
  std::vector<CopyItem<T>> cp;
  for (size_t i = 0; i < items.size(); ++i) {
    const SolveItem<T> &it = items[i];
    if (it.n > 0 && it.ncols > 0) cp.push_back({tmp + toff[i], it.X, it.ncols, it.ldx, it.n, it.ncols});
  }
  copy_rows_batched<T>(st, cp);
  RFDD_CUDA(cudaFreeAsync(tmp, st));
}

// X <- L^{-1} X, L unit lower (n x n): 32-row diagonal solves and GEMM updates, two levels
// (updates inside an nbo-row block, then one deep update of everything below it).
template <typename T>
void trsm_lower_unit(cudaStream_t st, const std::vector<SolveItem<T>> &items, int nbo) {
  if (has_block_inverses(items, nbo, false)) {
    trsm_block_inverse<T>(st, items, nbo, false);
    return;
  }
  constexpr int NB = LU_NB;
  int nmax = 0;
  for (auto &it : items) nmax = std::max(nmax, it.n);
  for (int K0 = 0; K0 < nmax; K0 += nbo) {
    for (int k0 = K0; k0 < K0 + nbo && k0 < nmax; k0 += NB) {
      std::vector<TriItem<T>> d;
      std::vector<GemmItem<T>> g;
      for (auto &it : items) {
        const int kend = std::min(K0 + nbo, it.n);
        if (k0 >= kend || it.ncols <= 0) continue;
        const int w = std::min(NB, kend - k0);
        TriItem<T> t{it.LU + (int64_t)k0 * it.ld + k0, it.ld, it.X + (int64_t)k0 * it.ldx, it.ldx, w, it.ncols};
        d.push_back(t);
        if (kend - k0 - w > 0) {
          GemmItem<T> x{it.LU + (int64_t)(k0 + w) * it.ld + k0, it.X + (int64_t)k0 * it.ldx,
                        it.X + (int64_t)(k0 + w) * it.ldx, kend - k0 - w, it.ncols, w, it.ld, it.ldx, it.ldx};
          g.push_back(x);
        }
      }
      launch_trsm_diag<T, false>(st, d);
      gemm_simt_batched<T>(st, g, false, false, -1.0, 1.0);  // small in-block updates
    }
    std::vector<GemmItem<T>> g;
    for (auto &it : items) {
      const int kend = std::min(K0 + nbo, it.n);
      if (K0 >= it.n || it.n - kend <= 0 || it.ncols <= 0) continue;
      GemmItem<T> x{it.LU + (int64_t)kend * it.ld + K0, it.X + (int64_t)K0 * it.ldx, it.X + (int64_t)kend * it.ldx,
                    it.n - kend, it.ncols, kend - K0, it.ld, it.ldx, it.ldx};
      g.push_back(x);
    }
    gemm_batched<T>(st, g, false, false, -1.0, 1.0);
  }
}

// X <- U^{-1} X, U upper (n x n) with its diagonal.
template <typename T>
void trsm_upper(cudaStream_t st, const std::vector<SolveItem<T>> &items, int nbo) {
  if (has_block_inverses(items, nbo, true)) {
    trsm_block_inverse<T>(st, items, nbo, true);
    return;
  }
  constexpr int NB = LU_NB;
  int nmax = 0;
  for (auto &it : items) nmax = std::max(nmax, it.n);
  if (nmax == 0) return;
  for (int K0 = ((nmax - 1) / nbo) * nbo; K0 >= 0; K0 -= nbo) {
    for (int k0 = K0 + nbo - NB; k0 >= K0; k0 -= NB) {
      std::vector<TriItem<T>> d;
      std::vector<GemmItem<T>> g;
      for (auto &it : items) {
        if (k0 >= it.n || it.ncols <= 0) continue;
        const int w = std::min(NB, it.n - k0);
        TriItem<T> t{it.LU + (int64_t)k0 * it.ld + k0, it.ld, it.X + (int64_t)k0 * it.ldx, it.ldx, w, it.ncols};
        d.push_back(t);
        if (k0 - K0 > 0) {
          GemmItem<T> x{it.LU + (int64_t)K0 * it.ld + k0, it.X + (int64_t)k0 * it.ldx, it.X + (int64_t)K0 * it.ldx,
                        k0 - K0, it.ncols, w, it.ld, it.ldx, it.ldx};
          g.push_back(x);
        }
      }
      launch_trsm_diag<T, true>(st, d);
      gemm_simt_batched<T>(st, g, false, false, -1.0, 1.0);  // small in-block updates
    }
    std::vector<GemmItem<T>> g;
    for (auto &it : items) {
      if (K0 >= it.n || K0 == 0 || it.ncols <= 0) continue;
      const int kend = std::min(K0 + nbo, it.n);
      GemmItem<T> x{it.LU + K0, it.X + (int64_t)K0 * it.ldx, it.X, K0, it.ncols, kend - K0, it.ld, it.ldx, it.ldx};
      g.push_back(x);
    }
    gemm_batched<T>(st, g, false, false, -1.0, 1.0);
  }
}

template <typename T>
void lu_solve_batched(cudaStream_t st, const std::vector<SolveItem<T>> &items, int nbo) {
  apply_pivots<T>(st, items);
  trsm_lower_unit<T>(st, items, nbo);
  trsm_upper<T>(st, items, nbo);
}

#define RFDD_INST_DENSE(T)                                                                          \
  template void gemm_batched<T>(cudaStream_t, const std::vector<GemmItem<T>> &, bool, bool, double, double); \
  template void gemm_simt_batched<T>(cudaStream_t, const std::vector<GemmItem<T>> &, bool, bool, double, double, \
                                     const std::vector<char> &);                                               \
  template void lu_batched<T>(cudaStream_t, const std::vector<LuItem<T>> &, int, int *);          \
  template void lu_solve_batched<T>(cudaStream_t, const std::vector<SolveItem<T>> &, int);        \
  template void apply_pivots<T>(cudaStream_t, const std::vector<SolveItem<T>> &);                 \
  template void trsm_lower_unit<T>(cudaStream_t, const std::vector<SolveItem<T>> &, int);         \
  template void trsm_upper<T>(cudaStream_t, const std::vector<SolveItem<T>> &, int);                \
  template void lu_block_inverses<T>(cudaStream_t, const std::vector<SolveItem<T>> &, int, const std::vector<T *> &, \
                                     const std::vector<T *> &);

RFDD_INST_DENSE(float)
RFDD_INST_DENSE(double)
RFDD_INST_DENSE(cx<float>)
RFDD_INST_DENSE(cx<double>)

}  // namespace rfdd
