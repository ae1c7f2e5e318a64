// Small dense FP64 kernels for block orthonormalisation and Rayleigh-Ritz bookkeeping.
#include "small.cuh"
#include "dense.cuh"

#include <algorithm>
#include <climits>

namespace rfdd {

constexpr int CH_MAXB = 64;
struct CholBatchP {
  CholItem it[CH_MAXB];
};

// Right-looking Cholesky G = R^T R on the upper triangle, one CTA per matrix (global memory).
// A pivot <= tol * (largest diagonal) marks its column dead: its row of R is zeroed and the
// column is skipped, so the kept columns get an orthonormal basis and dead ones a zero column.
__global__ void __launch_bounds__(512) chol_inv_kernel(CholBatchP bp, double tol) {
  const CholItem it = bp.it[blockIdx.x];
  const int b = it.b;
  double *G = it.G;
  __shared__ double dmax_s;
  __shared__ int dead_s;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < b; ++i) m = fmax(m, G[(int64_t)i * b + i]);
    dmax_s = m;
  }
  __syncthreads();
  const double thr = tol * dmax_s;
  for (int t = 0; t < b; ++t) {
    if (threadIdx.x == 0) {
      const double pv = G[(int64_t)t * b + t];
      dead_s = !(pv > thr) || !isfinite(pv);
      it.dead[t] = dead_s;
      if (!dead_s) G[(int64_t)t * b + t] = sqrt(pv);
    }
    __syncthreads();
    const double rtt = G[(int64_t)t * b + t];
    if (dead_s) {
      for (int c = t + threadIdx.x; c < b; c += blockDim.x) G[(int64_t)t * b + c] = 0.0;
    } else {
      for (int c = t + 1 + threadIdx.x; c < b; c += blockDim.x) G[(int64_t)t * b + c] /= rtt;
    }
    __syncthreads();
    if (!dead_s) {
      const int w = b - t - 1;
      for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
        const int i = t + 1 + e / w, c = t + 1 + e % w;
        if (c >= i) G[(int64_t)i * b + c] -= G[(int64_t)t * b + i] * G[(int64_t)t * b + c];
      }
    }
    __syncthreads();
  }
  // zero the strict lower triangle so that G holds exactly R
  for (int e = threadIdx.x; e < b * b; e += blockDim.x)
    if (e / b > e % b) G[e] = 0.0;
  __syncthreads();
  // R^{-1} by back substitution, thread per column
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    for (int i = b - 1; i >= 0; --i) {
      double v;
      if (it.dead[i]) {
        v = 0.0;
      } else {
        v = (i == c) ? 1.0 : 0.0;
        for (int k = i + 1; k <= c; ++k) v -= G[(int64_t)i * b + k] * it.Rinv[(int64_t)k * b + c];
        v /= G[(int64_t)i * b + i];
      }
      if (i > c) v = 0.0;
      it.Rinv[(int64_t)i * b + c] = v;
    }
  }
}

void chol_inv_batched(cudaStream_t st, const std::vector<CholItem> &items, double tol) {
  for (size_t s = 0; s < items.size(); s += CH_MAXB) {
    CholBatchP b;
    memset(&b, 0, sizeof(b));
    const int cnt = (int)std::min<size_t>(CH_MAXB, items.size() - s);
    for (int i = 0; i < cnt; ++i) b.it[i] = items[s + i];
    chol_inv_kernel<<<cnt, 512, 0, st>>>(b, tol);
    RFDD_CHECK_LAUNCH();
  }
}

static int gridn(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 152 * 32); }

__global__ void scale_sym_kernel(double *A, int64_t k, const double *__restrict__ d) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += (int64_t)gridDim.x * blockDim.x)
    A[e] *= d[e / k] * d[e % k];
}
void scale_sym(cudaStream_t st, double *A, int64_t k, const double *d) {
  if (k <= 0) return;
  scale_sym_kernel<<<gridn(k * k), 256, 0, st>>>(A, k, d);
  RFDD_CHECK_LAUNCH();
}

__global__ void scale_rows_cols_kernel(const double *__restrict__ U, int64_t r, int64_t k, const double *__restrict__ d,
                                       const double *__restrict__ f, double *out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < r * k; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = U[e] * d[e % k] * f[e / k];
}
void scale_rows_cols(cudaStream_t st, const double *U, int64_t r, int64_t k, const double *d, const double *f,
                     double *out) {
  if (r * k <= 0) return;
  scale_rows_cols_kernel<<<gridn(r * k), 256, 0, st>>>(U, r, k, d, f, out);
  RFDD_CHECK_LAUNCH();
}

__global__ void inv_sqrt_diag_kernel(const double *__restrict__ G, int64_t k, double *d) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < k; c += (int64_t)gridDim.x * blockDim.x) {
    const double g = G[c * k + c];
    d[c] = g > 0.0 ? 1.0 / sqrt(g) : 0.0;
  }
}
void inv_sqrt_diag(cudaStream_t st, const double *G, int64_t k, double *d) {
  if (k <= 0) return;
  inv_sqrt_diag_kernel<<<gridn(k), 256, 0, st>>>(G, k, d);
  RFDD_CHECK_LAUNCH();
}

__global__ void inv_sqrt_vec_kernel(const double *__restrict__ lam, int64_t r, double *f) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < r; q += (int64_t)gridDim.x * blockDim.x)
    f[q] = 1.0 / sqrt(lam[q]);
}
void inv_sqrt_vec(cudaStream_t st, const double *lam, int64_t r, double *f) {
  if (r <= 0) return;
  inv_sqrt_vec_kernel<<<gridn(r), 256, 0, st>>>(lam, r, f);
  RFDD_CHECK_LAUNCH();
}

__global__ void ritz_residuals_kernel(const double *__restrict__ AX, const double *__restrict__ MX,
                                      const double *__restrict__ theta, int64_t n, int64_t b, double *res) {
  const int64_t c = blockIdx.x;
  const double th = theta[c];
  double sr = 0.0, sm = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double mx = MX[i * b + c];
    const double r = AX[i * b + c] - th * mx;
    sr = fma(r, r, sr);
    sm = fma(mx, mx, sm);
  }
  __shared__ double r1[256], r2[256];
  r1[threadIdx.x] = sr;
  r2[threadIdx.x] = sm;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) { r1[threadIdx.x] += r1[threadIdx.x + o]; r2[threadIdx.x] += r2[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) res[c] = sqrt(r1[0]) / (fabs(th) * sqrt(r2[0]));
}
void ritz_residuals(cudaStream_t st, const double *AX, const double *MX, const double *theta, int64_t n, int64_t b,
                    double *res) {
  if (b <= 0) return;
  ritz_residuals_kernel<<<(unsigned)b, 256, 0, st>>>(AX, MX, theta, n, b, res);
  RFDD_CHECK_LAUNCH();
}

// out[c] = sum_i X[i][c] Y[i][c]  (n x b row-major blocks; fixed-order block reduction)
__global__ void col_dots_kernel(const double *__restrict__ X, const double *__restrict__ Y, int64_t n, int64_t b,
                                double *out) {
  const int64_t c = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(X[i * b + c], Y[i * b + c], s);
  __shared__ double r1[256];
  r1[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) r1[threadIdx.x] += r1[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = r1[0];
}
void col_dots(cudaStream_t st, const double *X, const double *Y, int64_t n, int64_t b, double *out) {
  if (b <= 0) return;
  col_dots_kernel<<<(unsigned)b, 256, 0, st>>>(X, Y, n, b, out);
  RFDD_CHECK_LAUNCH();
}

template <typename T>
__global__ void sub_inplace_kernel(const T *__restrict__ x, T *__restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = y[i] - x[i];
}
template <typename T>
void sub_inplace(cudaStream_t st, const T *x, T *y, int64_t n) {
  if (n <= 0) return;
  sub_inplace_kernel<T><<<gridn(n), 256, 0, st>>>(x, y, n);
  RFDD_CHECK_LAUNCH();
}
template void sub_inplace<cx<float>>(cudaStream_t, const cx<float> *, cx<float> *, int64_t);
template void sub_inplace<cx<double>>(cudaStream_t, const cx<double> *, cx<double> *, int64_t);
template void sub_inplace<double>(cudaStream_t, const double *, double *, int64_t);

}  // namespace rfdd

namespace rfdd {

// ---------------------------------------------------------------------------------------
// Pivoted Cholesky P^T G P = R^T R, right-looking, on the upper triangle only (the lower
// triangle is not read), one step per launch pair.
// Step t: choose the largest remaining diagonal entry (a contiguous copy dg of the diagonal is
// kept; its argmax compares the IEEE bit patterns as integers, which orders the non-negative
// values like the doubles and costs no FP64 instruction; smallest index on ties), stop
// (rank = t) when it is <= tol or not finite, interchange t and p symmetrically within the upper
// triangle (the factored rows' trailing parts included); then update the trailing upper triangle
// with the unscaled row g = G[t][t+1..]: G_ij -= (g_i g_j) / G_tt.  Rows of R are scaled by
// 1/sqrt(G_tt) once at the end (pchol_scale_kernel).  FP64 arithmetic is scarce on this GPU, so
// each step does one division and two FP64 operations per trailing upper entry.  On exit the
// leading rank x rank upper triangle holds R on the kept directions.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) pchol_pivot_kernel(double *G, int k, int *perm, int t, double tol, int *rank,
                                                           double *dg, double *dinv) {
  if (*rank >= 0) return;
  __shared__ long long bv[32];
  __shared__ int bi[32];
  __shared__ int piv_s;
  long long v = LLONG_MIN;
  int idx = k;
  for (int i = t + threadIdx.x; i < k; i += blockDim.x) {
    const long long g = __double_as_longlong(dg[i]);
    if (g > v) { v = g; idx = i; }  // i increases within a thread: the first maximum is kept
  }
  for (int o = 16; o > 0; o >>= 1) {
    const long long v2 = __shfl_down_sync(0xffffffffu, v, o);
    const int i2 = __shfl_down_sync(0xffffffffu, idx, o);
    if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
  }
  if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = v; bi[threadIdx.x >> 5] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long bvv = bv[0];
    int bii = bi[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bv[w] > bvv || (bv[w] == bvv && bi[w] < bii)) { bvv = bv[w]; bii = bi[w]; }
    const double d = bii < k ? dg[bii] : -1.0;
    piv_s = (d > tol && isfinite(d)) ? bii : -1;
    if (piv_s < 0) *rank = t;
    else *dinv = 1.0 / d;
  }
  __syncthreads();
  const int p = piv_s;
  if (p < 0 || p == t) return;
  // symmetric interchange of t < p in upper storage:
  //   r < t: G[r][t] <-> G[r][p];  t < r < p: G[t][r] <-> G[r][p];  r > p: G[t][r] <-> G[p][r];
  //   diagonal G[t][t] <-> G[p][p];  G[t][p] stays
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    double *a, *b;
    if (r < t) {
      a = G + (int64_t)r * k + t;
      b = G + (int64_t)r * k + p;
    } else if (r == t) {
      a = G + (int64_t)t * k + t;
      b = G + (int64_t)p * k + p;
    } else if (r < p) {
      a = G + (int64_t)t * k + r;
      b = G + (int64_t)r * k + p;
    } else if (r == p) {
      continue;
    } else {
      a = G + (int64_t)t * k + r;
      b = G + (int64_t)p * k + r;
    }
    const double x = *a;
    *a = *b;
    *b = x;
  }
  if (threadIdx.x == 0) {
    const int a = perm[t];
    perm[t] = perm[p];
    perm[p] = a;
    const double d = dg[t];
    dg[t] = dg[p];
    dg[p] = d;
  }
}

// trailing upper triangle: row t+1+i (grid-stride over rows), columns j >= i by the block's threads
__global__ void pchol_update_kernel(double *G, int k, int t, const int *rank, double *dg, const double *dinv_p) {
  if (*rank >= 0) return;
  const int len = k - t - 1;
  const double *g = G + (int64_t)t * k + t + 1;
  const double dinv = *dinv_p;
  for (int i = blockIdx.x; i < len; i += gridDim.x) {
    const double gi = g[i];
    double *row = G + (int64_t)(t + 1 + i) * k + t + 1;
    for (int j = i + threadIdx.x; j < len; j += blockDim.x) {
      const double nv = fma(-(gi * g[j]), dinv, row[j]);
      row[j] = nv;
      if (j == i) dg[t + 1 + i] = nv;
    }
  }
}

// R rows: G[t][c] /= sqrt(G_tt) for c > t, G[t][t] = sqrt(G_tt), t < rank (rows in parallel)
__global__ void pchol_scale_kernel(double *G, int k, const int *rank) {
  const int r = *rank < 0 ? k : *rank;
  for (int t = blockIdx.x; t < r; t += gridDim.x) {
    double *row = G + (int64_t)t * k;
    const double rt = sqrt(row[t]);
    const double inv = 1.0 / rt;
    __syncthreads();
    for (int c = t + 1 + threadIdx.x; c < k; c += blockDim.x) row[c] *= inv;
    __syncthreads();
    if (threadIdx.x == 0) row[t] = rt;
  }
}

__global__ void pchol_diag_kernel(const double *G, int k, double *dg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) dg[i] = G[(int64_t)i * k + i];
}

__global__ void iota_kernel(int *p, int k) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) p[i] = i;
}
__global__ void set_int_kernel(int *p, int v) { *p = v; }

int pivoted_cholesky(cudaStream_t st, double *G, int k, int *perm, double tol, int *rank_dev) {
  iota_kernel<<<ceil_div(k, 256), 256, 0, st>>>(perm, k);
  RFDD_CHECK_LAUNCH();
  set_int_kernel<<<1, 1, 0, st>>>(rank_dev, -1);
  RFDD_CHECK_LAUNCH();
  double *dg = nullptr;  // k diagonal entries, then 1 / (the current pivot)
  RFDD_CUDA(cudaMallocAsync((void **)&dg, (size_t)(k + 1) * sizeof(double), st));
  double *dinv = dg + k;
  pchol_diag_kernel<<<ceil_div(k, 256), 256, 0, st>>>(G, k, dg);
  RFDD_CHECK_LAUNCH();
  for (int t = 0; t < k; ++t) {
    pchol_pivot_kernel<<<1, 1024, 0, st>>>(G, k, perm, t, tol, rank_dev, dg, dinv);
    RFDD_CHECK_LAUNCH();
    const int len = k - t - 1;
    if (len > 0) {
      pchol_update_kernel<<<std::min(len, 8 * sm_count()), 256, 0, st>>>(G, k, t, rank_dev, dg, dinv);
      RFDD_CHECK_LAUNCH();
    }
  }
  pchol_scale_kernel<<<std::min(k, 1024), 256, 0, st>>>(G, k, rank_dev);
  RFDD_CHECK_LAUNCH();
  RFDD_CUDA(cudaFreeAsync(dg, st));
  int rank = -1;
  RFDD_CUDA(cudaMemcpyAsync(&rank, rank_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  RFDD_CUDA(cudaStreamSynchronize(st));
  return rank < 0 ? k : rank;
}

// out[i][j] = K[perm[i]][perm[j]] for i, j < r
__global__ void gather_sym_kernel(const double *__restrict__ K, int k, const int *__restrict__ perm, int r,
                                  double *out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)r * r; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e % r);
    out[e] = K[(int64_t)perm[i] * k + perm[j]];
  }
}
void gather_sym(cudaStream_t st, const double *K, int k, const int *perm, int r, double *out) {
  if (r <= 0) return;
  gather_sym_kernel<<<gridn((int64_t)r * r), 256, 0, st>>>(K, k, perm, r, out);
  RFDD_CHECK_LAUNCH();
}

// Lt[i][j] = R[j][i] / R[i][i] (j < i), 1 (j == i), 0 (j > i): unit lower, from upper R (ld ldr)
__global__ void unit_lower_from_upper_kernel(const double *__restrict__ R, int ldr, int r, double *Lt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)r * r; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e % r);
    Lt[e] = j < i ? R[(int64_t)j * ldr + i] / R[(int64_t)i * ldr + i] : (i == j ? 1.0 : 0.0);
  }
}
void unit_lower_from_upper(cudaStream_t st, const double *R, int ldr, int r, double *Lt) {
  if (r <= 0) return;
  unit_lower_from_upper_kernel<<<gridn((int64_t)r * r), 256, 0, st>>>(R, ldr, r, Lt);
  RFDD_CHECK_LAUNCH();
}

// out[i][j] = (trans ? in[j][i] : in[i][j]) / R[i][i]   (r x r)
__global__ void scale_rows_by_rdiag_kernel(const double *__restrict__ in, int r, int trans, const double *__restrict__ R,
                                           int ldr, double *out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)r * r; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e % r);
    const double v = trans ? in[(int64_t)j * r + i] : in[e];
    out[e] = v / R[(int64_t)i * ldr + i];
  }
}
void scale_rows_by_rdiag(cudaStream_t st, const double *in, int r, bool trans, const double *R, int ldr, double *out) {
  if (r <= 0) return;
  scale_rows_by_rdiag_kernel<<<gridn((int64_t)r * r), 256, 0, st>>>(in, r, trans ? 1 : 0, R, ldr, out);
  RFDD_CHECK_LAUNCH();
}

// out = (A + A^T)/2 (r x r), into a separate buffer
__global__ void symmetrize_kernel(const double *__restrict__ A, int r, double *out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)r * r; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e % r);
    out[e] = 0.5 * (A[e] + A[(int64_t)j * r + i]);
  }
}
void symmetrize(cudaStream_t st, const double *A, int r, double *out) {
  if (r <= 0) return;
  symmetrize_kernel<<<gridn((int64_t)r * r), 256, 0, st>>>(A, r, out);
  RFDD_CHECK_LAUNCH();
}

// out (b x a) = in^T (in: a x b row-major)
__global__ void transpose_kernel(const double *__restrict__ in, int a, int b, double *out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)a * b; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / b), j = (int)(e % b);
    out[(int64_t)j * a + i] = in[e];
  }
}
void transpose(cudaStream_t st, const double *in, int a, int b, double *out) {
  if ((int64_t)a * b <= 0) return;
  transpose_kernel<<<gridn((int64_t)a * b), 256, 0, st>>>(in, a, b, out);
  RFDD_CHECK_LAUNCH();
}

// Cfull[perm[i]][c] = d[perm[i]] * Cr[i][c] for i < r (other rows untouched; caller zeroes)
__global__ void scatter_rows_kernel(const double *__restrict__ Cr, int r, int ns, const int *__restrict__ perm,
                                    const double *__restrict__ d, double *Cfull) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)r * ns; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ns), c = (int)(e % ns);
    const int row = perm[i];
    Cfull[(int64_t)row * ns + c] = d[row] * Cr[e];
  }
}
void scatter_rows_perm(cudaStream_t st, const double *Cr, int r, int ns, const int *perm, const double *d,
                       double *Cfull) {
  if ((int64_t)r * ns <= 0) return;
  scatter_rows_kernel<<<gridn((int64_t)r * ns), 256, 0, st>>>(Cr, r, ns, perm, d, Cfull);
  RFDD_CHECK_LAUNCH();
}


// G[c][r] = G[r][c] for r in [r0, r1), c in [c0, c1)  (k x k row-major)
__global__ void mirror_block_kernel(double *G, int64_t k, int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
  const int64_t w = c1 - c0, total = (r1 - r0) * w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = r0 + e / w, c = c0 + e % w;
    G[c * k + r] = G[r * k + c];
  }
}
void mirror_block(cudaStream_t st, double *G, int64_t k, int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
  if (r1 <= r0 || c1 <= c0) return;
  mirror_block_kernel<<<gridn((r1 - r0) * (c1 - c0)), 256, 0, st>>>(G, k, r0, r1, c0, c1);
  RFDD_CHECK_LAUNCH();
}

}  // namespace rfdd
