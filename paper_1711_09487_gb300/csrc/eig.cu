// Dense symmetric eigensolver used by the Rayleigh-Ritz steps (Alg. 3 step 7 and the
// completion passes).  Textbook algorithms: Householder reduction to tridiagonal form, implicit
// QL iteration with Wilkinson-type shifts on the tridiagonal matrix, back-transformation.
#include "eig.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>

namespace rfdd {

constexpr int EIG_MAXB = 64;

struct SymBatchP {
  SymItem it[EIG_MAXB];
};

__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < nw; ++q) s += red[q];
  return s;
}

// Step i, part 1: Householder vector for row i (columns i+1..n-1), LAPACK convention
// H_i = I - tau v v^T with v[0] = 1, H_i x = beta e_1.
__global__ void house_kernel(SymBatchP b, int i) {
  SymItem it = b.it[blockIdx.x];
  const int n = it.n;
  if (i >= n) return;
  double *row = it.H + (int64_t)i * it.ld;
  __shared__ double red[32];
  if (i >= n - 1) {
    if (threadIdx.x == 0) { it.d[i] = row[i]; it.tau[i] = 0.0; }
    return;
  }
  const int len = n - i - 1;
  double *x = row + i + 1;
  double ss = 0.0;
  for (int k = 1 + threadIdx.x; k < len; k += blockDim.x) ss = fma(x[k], x[k], ss);
  const double sig = block_sum(ss, red);
  const double alpha = x[0];
  __shared__ double scale_s, beta_s, tau_s;
  if (threadIdx.x == 0) {
    it.d[i] = row[i];
    if (sig == 0.0) {
      tau_s = 0.0;
      beta_s = alpha;
      scale_s = 0.0;
    } else {
      const double nrm = sqrt(alpha * alpha + sig);
      const double beta = alpha <= 0.0 ? nrm : -nrm;
      tau_s = (beta - alpha) / beta;
      scale_s = 1.0 / (alpha - beta);
      beta_s = beta;
    }
    it.e[i] = beta_s;
    it.tau[i] = tau_s;
  }
  __syncthreads();
  const double sc = scale_s;
  for (int k = 1 + threadIdx.x; k < len; k += blockDim.x) x[k] *= sc;
  if (threadIdx.x == 0) x[0] = 1.0;
}

// Step i, part 2: p = tau * H_t v (H_t = trailing block), warp per row.
__global__ void symv_kernel(SymBatchP b, int i) {
  SymItem it = b.it[blockIdx.y];
  const int n = it.n;
  if (i >= n - 2) return;
  const int len = n - i - 1;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (r >= len) return;
  const double *v = it.H + (int64_t)i * it.ld + i + 1;
  const double *h = it.H + (int64_t)(i + 1 + r) * it.ld + i + 1;
  double s = 0.0;
  for (int c = lane; c < len; c += 32) s = fma(h[c], v[c], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) it.work[r] = it.tau[i] * s;
}

// Step i, part 3: H_t -= v q^T + q v^T, q = p - (tau/2)(p^T v) v.  Each CTA recomputes p^T v.
// Products are rounded separately so that H_t stays exactly symmetric.
__global__ void rank2_kernel(SymBatchP b, int i) {
  SymItem it = b.it[blockIdx.y];
  const int n = it.n;
  if (i >= n - 2) return;
  const int len = n - i - 1;
  const double *v = it.H + (int64_t)i * it.ld + i + 1;
  __shared__ double red[32];
  double s = 0.0;
  for (int c = threadIdx.x; c < len; c += blockDim.x) s = fma(it.work[c], v[c], s);
  const double K = 0.5 * it.tau[i] * block_sum(s, red);
  const int64_t total = (int64_t)len * len;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / len), c = (int)(e % len);
    const double qr = it.work[r] - K * v[r];
    const double qc = it.work[c] - K * v[c];
    const double t = __dadd_rn(__dmul_rn(v[r], qc), __dmul_rn(qr, v[c]));
    double *h = it.H + (int64_t)(i + 1 + r) * it.ld + i + 1 + c;
    *h = *h - t;
  }
}

// Implicit QL on the tridiagonal matrix.  The scalar recurrence is sequential; it runs on one
// thread per matrix and logs every QL sweep's rotations (first index m, count, then the (c, s)
// pairs).  A second kernel applies the logged rotations to the eigenvector matrix: every row of
// Z (one component of all eigenvectors) evolves independently under the same rotation sequence,
// so rows are spread over many CTAs and kept in shared memory.
struct RotLog {
  double *cs;       // cap pairs (c, s) per matrix
  int *sweeps;      // cap_sw pairs (m, nrot) per matrix
  int *nsweeps;     // one counter per matrix
  int64_t cap, cap_sw;
};

__global__ void tql_scalar_kernel(SymBatchP b, RotLog lg, int *status) {
  SymItem it = b.it[blockIdx.x];
  const int n = it.n;
  double *d = it.d, *e = it.e;
  double *cs = lg.cs + (int64_t)blockIdx.x * lg.cap * 2;
  int *sw = lg.sweeps + (int64_t)blockIdx.x * lg.cap_sw * 2;
  if (threadIdx.x == 0) {
    if (n > 0) e[n - 1] = 0.0;
    const double eps = 2.220446049250313e-16;
    // global scale for the splitting test: an off-diagonal at the rounding level of the whole
    // matrix also splits (otherwise clusters of near-zero eigenvalues never deflate)
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) tnorm = fmax(tnorm, fabs(d[i]) + fabs(e[i]));
    int64_t used = 0, nsw = 0;
    bool overflow = false;
    for (int l = 0; l < n; ++l) {
      for (int iter = 0;; ++iter) {
        int m = l;
        for (; m < n - 1; ++m) {
          const double dd = fabs(d[m]) + fabs(d[m + 1]);
          if (fabs(e[m]) <= eps * dd || fabs(e[m]) <= 0.5 * eps * tnorm) break;
        }
        if (m == l) break;
        if (iter >= 100) {
          atomicOr(status, DS_NONFINITE);
          break;
        }
        double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
        double r = hypot(g, 1.0);
        g = d[m] - d[l] + e[l] / (g + (g >= 0 ? fabs(r) : -fabs(r)));
        double s = 1.0, c = 1.0, p = 0.0;
        bool early = false;
        int nrot = 0;
        const int64_t base = used;
        for (int i = m - 1; i >= l; --i) {
          const double f = s * e[i];
          const double bb = c * e[i];
          r = hypot(f, g);
          e[i + 1] = r;
          if (r == 0.0) {
            d[i + 1] -= p;
            e[m] = 0.0;
            early = true;
            break;
          }
          s = f / r;
          c = g / r;
          g = d[i + 1] - p;
          r = (d[i] - g) * s + 2.0 * c * bb;
          p = s * r;
          d[i + 1] = g + p;
          g = c * r - bb;
          if (!overflow && base + nrot < lg.cap) {
            cs[2 * (base + nrot)] = c;
            cs[2 * (base + nrot) + 1] = s;
          }
          ++nrot;
        }
        if (!early) {
          d[l] -= p;
          e[l] = g;
          e[m] = 0.0;
        }
        if (nrot > 0 && !overflow) {
          if (base + nrot > lg.cap || nsw >= lg.cap_sw) {
            overflow = true;
            atomicOr(status, DS_BAD_SIZE);
          } else {
            sw[2 * nsw] = m;
            sw[2 * nsw + 1] = nrot;
            ++nsw;
            used += nrot;
          }
        }
      }
    }
    lg.nsweeps[blockIdx.x] = (int)nsw;
  }
  __syncthreads();
  // rank sort (ties by index): perm[rank] = k, eigenvalues ascending into d
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double v = d[k];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double u = d[j];
      rank += (u < v) || (u == v && j < k);
    }
    it.perm[rank] = k;
    it.work[rank] = v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) d[k] = it.work[k];
}

// rows [row0, row0 + blockDim.x) of Z (Z = I initially) under the logged rotations; the
// result is written transposed: Zt[i][k] = Z[k][i] (row i of Zt = eigenvector i)
__global__ void tql_apply_kernel(SymBatchP b, RotLog lg, int rows_per_cta) {
  const SymItem it = b.it[blockIdx.y];
  const int n = it.n;
  const int k = blockIdx.x * rows_per_cta + threadIdx.x;
  if (blockIdx.x * rows_per_cta >= n) return;
  extern __shared__ double zs[];
  const int pitch = n | 1;
  double *z = zs + (int64_t)threadIdx.x * pitch;
  const bool live = k < n && threadIdx.x < rows_per_cta;
  if (live)
    for (int i = 0; i < n; ++i) z[i] = (i == k) ? 1.0 : 0.0;
  const double *cs = lg.cs + (int64_t)blockIdx.y * lg.cap * 2;
  const int *sw = lg.sweeps + (int64_t)blockIdx.y * lg.cap_sw * 2;
  const int nsw = lg.nsweeps[blockIdx.y];
  if (live) {
    int64_t off = 0;
    for (int q = 0; q < nsw; ++q) {
      const int m = sw[2 * q], nrot = sw[2 * q + 1];
      double carry = z[m];
      for (int t = 0; t < nrot; ++t) {
        const int i = m - 1 - t;
        const double c = __ldg(cs + 2 * (off + t)), s = __ldg(cs + 2 * (off + t) + 1);
        const double zi = z[i];
        z[i + 1] = s * zi + c * carry;
        carry = c * zi - s * carry;
      }
      z[m - nrot] = carry;
      off += nrot;
    }
    for (int i = 0; i < n; ++i) it.Zt[(int64_t)i * n + k] = z[i];
  }
}

void sym_eig_values(cudaStream_t st, const std::vector<SymItem> &items, int *status) {
  for (size_t s0 = 0; s0 < items.size(); s0 += EIG_MAXB) {
    SymBatchP b;
    memset(&b, 0, sizeof(b));
    const int cnt = (int)std::min<size_t>(EIG_MAXB, items.size() - s0);
    int nmax = 0;
    for (int i = 0; i < cnt; ++i) { b.it[i] = items[s0 + i]; nmax = std::max(nmax, b.it[i].n); }
    if (nmax == 0) continue;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    const bool timing = getenv("RFDD_LOG") && getenv("RFDD_LOG")[0] && getenv("RFDD_LOG")[0] != '0';
    if (timing) {
      cudaEventCreate(&ev0);
      cudaEventCreate(&ev1);
      cudaEventCreate(&ev2);
      cudaEventRecord(ev0, st);
    }
    for (int i = 0; i < nmax; ++i) {
      house_kernel<<<cnt, 256, 0, st>>>(b, i);
      RFDD_CHECK_LAUNCH();
      const int len = nmax - i - 1;
      if (i < nmax - 2) {
        symv_kernel<<<dim3(ceil_div((int64_t)len * 32, 256), cnt), 256, 0, st>>>(b, i);
        RFDD_CHECK_LAUNCH();
        const int blocks = std::max(1, std::min(1024, ceil_div((int64_t)len * len, 256 * 8)));
        rank2_kernel<<<dim3(blocks, cnt), 256, 0, st>>>(b, i);
        RFDD_CHECK_LAUNCH();
      }
    }
    RotLog lg;
    lg.cap = 2 * (int64_t)nmax * nmax + 64;
    lg.cap_sw = 40 * (int64_t)nmax + 64;
    RFDD_CUDA(cudaMallocAsync((void **)&lg.cs, (size_t)cnt * lg.cap * 2 * sizeof(double), st));
    RFDD_CUDA(cudaMallocAsync((void **)&lg.sweeps, (size_t)cnt * lg.cap_sw * 2 * sizeof(int), st));
    RFDD_CUDA(cudaMallocAsync((void **)&lg.nsweeps, (size_t)cnt * sizeof(int), st));
    if (timing) cudaEventRecord(ev1, st);
    tql_scalar_kernel<<<cnt, 256, 0, st>>>(b, lg, status);
    RFDD_CHECK_LAUNCH();
    if (timing) cudaEventRecord(ev2, st);
    const int pitch = nmax | 1;
    int rows = (int)std::min<int64_t>(64, (200 * 1024) / ((int64_t)pitch * sizeof(double)));
    RFDD_REQUIRE(rows >= 1, RFDD_EINVAL, "sym_eig: order too large");
    const size_t smem = (size_t)rows * pitch * sizeof(double);
    RFDD_CUDA(cudaFuncSetAttribute(tql_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tql_apply_kernel<<<dim3(ceil_div(nmax, rows), cnt), rows, smem, st>>>(b, lg, rows);
    RFDD_CHECK_LAUNCH();
    if (timing) {
      cudaEvent_t ev3;
      cudaEventCreate(&ev3);
      cudaEventRecord(ev3, st);
      cudaEventSynchronize(ev3);
      float a = 0, bb = 0, c = 0;
      cudaEventElapsedTime(&a, ev0, ev1);
      cudaEventElapsedTime(&bb, ev1, ev2);
      cudaEventElapsedTime(&c, ev2, ev3);
      fprintf(stderr, "[rfdd]     sym_eig n=%d x%d: tridiag %.2f ms, QL scalar %.2f ms, QL apply %.2f ms\n", nmax, cnt,
              a, bb, c);
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
      cudaEventDestroy(ev2);
      cudaEventDestroy(ev3);
    }
    RFDD_CUDA(cudaFreeAsync(lg.cs, st));
    RFDD_CUDA(cudaFreeAsync(lg.sweeps, st));
    RFDD_CUDA(cudaFreeAsync(lg.nsweeps, st));
  }
}

// x = H_0 H_1 ... H_{n-3} z for the selected eigenvectors z of the tridiagonal matrix; one CTA
// per output vector, the vector in shared memory.
struct BackBatchP {
  SymItem s[EIG_MAXB];
  const int *sel[EIG_MAXB];
  double *out[EIG_MAXB];
  int nsel[EIG_MAXB];
  int ld_out[EIG_MAXB];
};

__global__ void back_kernel(BackBatchP b) {
  const int bi = blockIdx.y;
  const int r = blockIdx.x;
  if (r >= b.nsel[bi]) return;
  const SymItem it = b.s[bi];
  const int n = it.n;
  extern __shared__ double x[];
  __shared__ double red[32];
  const int row = it.perm[b.sel[bi][r]];
  for (int k = threadIdx.x; k < n; k += blockDim.x) x[k] = it.Zt[(int64_t)row * n + k];
  __syncthreads();
  for (int i = n - 3; i >= 0; --i) {
    const double tau = it.tau[i];
    if (tau == 0.0) continue;
    const double *v = it.H + (int64_t)i * it.ld + i + 1;
    const int len = n - i - 1;
    double s = 0.0;
    for (int k = threadIdx.x; k < len; k += blockDim.x) s = fma(v[k], x[i + 1 + k], s);
    const double t = tau * block_sum(s, red);
    for (int k = threadIdx.x; k < len; k += blockDim.x) x[i + 1 + k] -= t * v[k];
    __syncthreads();
  }
  double *o = b.out[bi] + (int64_t)r * b.ld_out[bi];
  for (int k = threadIdx.x; k < n; k += blockDim.x) o[k] = x[k];
}

void sym_eig_vectors(cudaStream_t st, const std::vector<BackItem> &items) {
  for (size_t s0 = 0; s0 < items.size(); s0 += EIG_MAXB) {
    BackBatchP b;
    memset(&b, 0, sizeof(b));
    const int cnt = (int)std::min<size_t>(EIG_MAXB, items.size() - s0);
    int nmax = 1, selmax = 0;
    for (int i = 0; i < cnt; ++i) {
      const BackItem &it = items[s0 + i];
      b.s[i] = *it.s;
      b.sel[i] = it.sel;
      b.out[i] = it.out;
      b.nsel[i] = it.nsel;
      b.ld_out[i] = it.ld_out;
      nmax = std::max(nmax, it.s->n);
      selmax = std::max(selmax, it.nsel);
    }
    if (selmax == 0) continue;
    const size_t smem = (size_t)nmax * sizeof(double);
    RFDD_REQUIRE(smem <= 200 * 1024, RFDD_EINVAL, "sym_eig: order too large");
    RFDD_CUDA(cudaFuncSetAttribute(back_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    back_kernel<<<dim3(selmax, cnt), 256, smem, st>>>(b);
    RFDD_CHECK_LAUNCH();
  }
}

}  // namespace rfdd
