// Dense symmetric eigensolver used by the Rayleigh-Ritz steps (Alg. 3 step 7 and the
// completion passes).  Textbook algorithms: Householder reduction to tridiagonal form,
// bisection on Sturm counts for the eigenvalues of the tridiagonal matrix, inverse iteration
// with Gram-Schmidt inside clusters of close eigenvalues, back-transformation.
#include "eig.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>

namespace rfdd {

constexpr int EIG_MAXB = 64;

struct SymBatchP {
  SymItem it[EIG_MAXB];
};

// Block-wide sum, the same value in every thread.  One thread adds the warp partials (FP64
// arithmetic is scarce on this GPU: every thread adding them would cost nw FP64 adds each).
__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < nw; ++q) s += red[q];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Householder tridiagonalisation, one pass over the trailing block per step.  Step i reflects row
// i (columns i+1..n-1) with H_i = I - tau v v^T, v[0] = 1, H_i x = beta e_1 (LAPACK convention;
// v is kept in row i for the back-transformation); the trailing block then takes the rank-2
// update -v q^T - q v^T with p = tau H_t v, q = p - (tau/2)(p^T v) v.  The update of step i-1 is
// applied lazily: house_kernel(i) forms q_{i-1} and applies it to row i only (O(n) work: on this
// GPU one SM's FP64 rate is far too low for more), and update_symv_kernel(i) applies it to rows
// and columns i+1..n-1 while forming p_i from the updated entries, so each step reads and writes
// the trailing block once.

// Step i, part 1 (one CTA per item): q_{i-1} into qbuf, row i updated by step i-1, then the
// Householder vector of row i.
__global__ void __launch_bounds__(512) house_kernel(SymBatchP b, int i, double *qbuf, int64_t qstride) {
  SymItem it = b.it[blockIdx.x];
  const int n = it.n;
  if (i >= n) return;
  double *q = qbuf + (int64_t)blockIdx.x * qstride;
  double *row = it.H + (int64_t)i * it.ld;
  __shared__ double red[33];
  const int ip = i - 1;
  if (ip >= 0 && ip < n - 2) {
    // p_{i-1} covers rows i..n-1 (work[0..len)); v_{i-1} is row i-1 from column i on
    const int len = n - i;
    const double *v = it.H + (int64_t)ip * it.ld + i;
    double ss = 0.0;
    for (int k = threadIdx.x; k < len; k += blockDim.x) ss = fma(it.work[k], v[k], ss);
    const double K = 0.5 * it.tau[ip] * block_sum(ss, red);
    for (int k = threadIdx.x; k < len; k += blockDim.x) q[i + k] = it.work[k] - K * v[k];
    __syncthreads();
    const double vi = v[0], qi = q[i];
    for (int k = threadIdx.x; k < len; k += blockDim.x) row[i + k] = fma(-qi, v[k], fma(-vi, q[i + k], row[i + k]));
    __syncthreads();
  }
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

// Step i, part 2 (TRD_WPR warps per row r of the trailing block i+1..n-1): apply step i-1's rank-2
// update as two FMAs (the FP64 pipes bound this kernel; the block stays symmetric to rounding, a
// backward perturbation of the order of the update's rounding), then p_i[r] = tau_i (H_t v_i)[r]
// into work.  Runs for i <= n-2 (at i = n-2 only the pending update is left).
constexpr int TRD_WPR = 2;
__global__ void __launch_bounds__(256) update_symv_kernel(SymBatchP b, int i, const double *qbuf, int64_t qstride) {
  SymItem it = b.it[blockIdx.y];
  const int n = it.n;
  if (i > n - 2) return;
  const int len = n - i - 1;
  constexpr int TPR = 32 * TRD_WPR;                 // threads per row
  const int rloc = threadIdx.x / TPR, tr = threadIdx.x % TPR;
  const int r = blockIdx.x * (256 / TPR) + rloc;
  __shared__ double part[256 / 32];
  const int c0 = i + 1;
  const bool upd = i >= 1 && i - 1 < n - 2;
  const bool sym = i < n - 2;
  double s = 0.0;
  if (r < len) {
    double *h = it.H + (int64_t)(c0 + r) * it.ld + c0;
    const double *v = it.H + (int64_t)i * it.ld + c0;         // v_i (row i)
    const double *vp = it.H + (int64_t)(i - 1) * it.ld + c0;  // v_{i-1} from column i+1 on
    const double *q = qbuf + (int64_t)blockIdx.y * qstride + c0;
    const double vr = upd ? vp[r] : 0.0, qr = upd ? q[r] : 0.0;
    for (int c = tr; c < len; c += TPR) {
      double h0 = h[c];
      if (upd) {
        h0 = fma(-qr, vp[c], fma(-vr, q[c], h0));
        h[c] = h0;
      }
      s = fma(h0, v[c], s);
    }
  }
  if (!sym) return;  // uniform over the block
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (tr == 0 && r < len) {
    double t = 0.0;
    for (int w = 0; w < TRD_WPR; ++w) t += part[rloc * TRD_WPR + w];
    it.work[r] = it.tau[i] * t;
  }
}

// --------------------------------------------------------------------------------------
// Eigenvalues of the tridiagonal matrix by multisection on Sturm counts.  The Sturm count of x is
// the number of negative pivots of the LDL^T factorisation of T - x I (Sylvester's law).
// --------------------------------------------------------------------------------------
__device__ inline int sturm_count(const double *d, const double *e, int n, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int k = 1; k < n; ++k) {
    q = d[k] - x - e[k - 1] * e[k - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// 1/q by the hardware's approximate reciprocal refined with one Newton-Raphson step
// (r <- r + r (1 - q r)), which doubles the number of correct bits: relative error about 2^-44,
// far below what a Sturm count needs (it is a tiny backward perturbation of e_k^2).  |q| >= pivmin
// keeps q a normal number.
__device__ inline double recip_nr(double q) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(q));
  return fma(r, fma(-q, r, 1.0), r);
}

__device__ inline int sturm_count_nr(const double *__restrict__ d, const double *__restrict__ e, int n, double x,
                                     double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int k = 1; k < n; ++k) {
    const double ek = e[k - 1];
    q = fma(-ek * ek, recip_nr(q), d[k] - x);
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// BIS_G lanes per eigenvalue: each round the lanes take the Sturm counts at BIS_G points that cut
// [lo, hi] into BIS_G + 1 equal parts, and the part holding eigenvalue i becomes the new interval
// (log2(BIS_G + 1) bits per round instead of one, at BIS_G times the counting work).
constexpr int BIS_G = 8;

__global__ void __launch_bounds__(256) bisect_kernel(SymBatchP b) {
  const SymItem it = b.it[blockIdx.y];
  const int n = it.n;
  const int g = threadIdx.x % BIS_G;                                   // lane within the group
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) / BIS_G;       // eigenvalue index
  const unsigned gmask = ((1u << BIS_G) - 1u) << ((threadIdx.x & 31) & ~(BIS_G - 1));
  if (i >= n) return;  // the lanes of a group share i, so a group leaves together
  const double *d = it.d, *e = it.e;
  double gl = d[0], gu = d[0], emax2 = 0.0;
  for (int k = 0; k < n; ++k) {
    const double r = (k > 0 ? fabs(e[k - 1]) : 0.0) + (k < n - 1 ? fabs(e[k]) : 0.0);
    gl = fmin(gl, d[k] - r);
    gu = fmax(gu, d[k] + r);
    if (k < n - 1) emax2 = fmax(emax2, e[k] * e[k]);
  }
  const double eps = 2.220446049250313e-16;
  const double pivmin = 2.2250738585072014e-308 * fmax(1.0, emax2);
  const double span = fmax(fabs(gl), fabs(gu));
  double lo = gl - 2.0 * eps * span * n - pivmin, hi = gu + 2.0 * eps * span * n + pivmin;
  for (int round = 0; round < 100; ++round) {
    if (hi - lo <= 2.0 * eps * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin) break;
    const double step = (hi - lo) / (BIS_G + 1);
    const double x = lo + step * (g + 1);
    const bool above = (x > lo && x < hi) ? sturm_count_nr(d, e, n, x, pivmin) > i : (x >= hi);
    // the first cut point whose count exceeds i bounds the eigenvalue from above
    const unsigned m = __ballot_sync(gmask, above) & gmask;
    const int base = (threadIdx.x & 31) & ~(BIS_G - 1);
    const int first = m ? (__ffs(m) - 1 - base) : BIS_G;
    const double nlo = first > 0 ? lo + step * first : lo;
    const double nhi = first < BIS_G ? lo + step * (first + 1) : hi;
    if (!(nlo > lo || nhi < hi)) break;  // no progress in floating point
    lo = nlo;
    hi = nhi;
  }
  if (g == 0) it.lam[i] = 0.5 * (lo + hi);
}

// Householder reduction of every item of the batch to tridiagonal form (d, e)
static void tridiagonalize(cudaStream_t st, const SymBatchP &b, int cnt, int nmax) {
  double *qbuf = nullptr;
  RFDD_CUDA(cudaMallocAsync((void **)&qbuf, (size_t)cnt * std::max(nmax, 1) * sizeof(double), st));
  for (int i = 0; i < nmax; ++i) {
    house_kernel<<<cnt, 512, 0, st>>>(b, i, qbuf, nmax);
    RFDD_CHECK_LAUNCH();
    if (i <= nmax - 2) {
      const int len = nmax - i - 1;
      update_symv_kernel<<<dim3(ceil_div((int64_t)len * 32 * TRD_WPR, 256), cnt), 256, 0, st>>>(b, i, qbuf, nmax);
      RFDD_CHECK_LAUNCH();
    }
  }
  RFDD_CUDA(cudaFreeAsync(qbuf, st));
}

// counts[i] = number of eigenvalues of item i's tridiagonal matrix below shift (Sturm count)
__global__ void sturm_count_kernel(SymBatchP b, int cnt, double shift, long long *counts) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnt) return;
  const SymItem it = b.it[q];
  const int n = it.n;
  if (n <= 0) {
    counts[q] = 0;
    return;
  }
  double emax2 = 0.0;
  for (int k = 0; k + 1 < n; ++k) emax2 = fmax(emax2, it.e[k] * it.e[k]);
  const double pivmin = 2.2250738585072014e-308 * fmax(1.0, emax2);
  counts[q] = sturm_count(it.d, it.e, n, shift, pivmin);
}

void sym_negative_counts(cudaStream_t st, const std::vector<SymItem> &items, double shift, long long *counts_dev) {
  for (size_t s0 = 0; s0 < items.size(); s0 += EIG_MAXB) {
    SymBatchP b;
    memset(&b, 0, sizeof(b));
    const int cnt = (int)std::min<size_t>(EIG_MAXB, items.size() - s0);
    int nmax = 0;
    for (int i = 0; i < cnt; ++i) { b.it[i] = items[s0 + i]; nmax = std::max(nmax, b.it[i].n); }
    if (nmax > 0) tridiagonalize(st, b, cnt, nmax);
    sturm_count_kernel<<<1, 64, 0, st>>>(b, cnt, shift, counts_dev + s0);
    RFDD_CHECK_LAUNCH();
  }
}

void sym_eig_values(cudaStream_t st, const std::vector<SymItem> &items, int *status) {
  (void)status;
  for (size_t s0 = 0; s0 < items.size(); s0 += EIG_MAXB) {
    SymBatchP b;
    memset(&b, 0, sizeof(b));
    const int cnt = (int)std::min<size_t>(EIG_MAXB, items.size() - s0);
    int nmax = 0;
    for (int i = 0; i < cnt; ++i) { b.it[i] = items[s0 + i]; nmax = std::max(nmax, b.it[i].n); }
    if (nmax == 0) continue;
    tridiagonalize(st, b, cnt, nmax);
    // e[n-1] = 0 for every item (house_kernel leaves it undefined)
    // BIS_G lanes per eigenvalue, 256 / BIS_G eigenvalues per block
    bisect_kernel<<<dim3(ceil_div((int64_t)nmax * BIS_G, 256), cnt), 256, 0, st>>>(b);
    RFDD_CHECK_LAUNCH();
  }
}

// --------------------------------------------------------------------------------------
// Eigenvectors of the tridiagonal matrix by inverse iteration, one CTA per cluster.  Thread 0
// factors T - lambda I with partial pivoting (rows k, k+1 swapped when |sub| > |diagonal|) and
// runs the triangular solves; all threads share the Gram-Schmidt against the cluster's earlier
// vectors and the normalisation.
// --------------------------------------------------------------------------------------
struct Cluster {
  int item;   // index into the batch
  int first;  // position in the item's selection list
  int size;
};
struct InvIterP {
  SymItem it[EIG_MAXB];
  const int *sel[EIG_MAXB];   // device copies of the selections
};

__global__ void __launch_bounds__(256) inviter_kernel(InvIterP p, const Cluster *__restrict__ cl, double *scratch,
                                                      int64_t scratch_per_cta, double ctol) {
  const Cluster c = cl[blockIdx.x];
  const SymItem it = p.it[c.item];
  const int *sel = p.sel[c.item];
  const int n = it.n;
  const double *d = it.d, *e = it.e;
  double *u1 = scratch + (int64_t)blockIdx.x * scratch_per_cta;
  double *u2 = u1 + n, *u3 = u2 + n, *ml = u3 + n, *pv = ml + n, *x = pv + n, *ru = x + n;
  __shared__ double red[33];
  __shared__ double tnorm_s;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < n; ++k) t = fmax(t, fabs(d[k]) + (k > 0 ? fabs(e[k - 1]) : 0.0) + (k < n - 1 ? fabs(e[k]) : 0.0));
    tnorm_s = t;
  }
  __syncthreads();
  const double eps = 2.220446049250313e-16;
  const double delta = eps * fmax(tnorm_s, 1e-300);
  for (int q = 0; q < c.size; ++q) {
    const int row = c.first + q;  // output row in Zt
    const double lam = it.lam[sel[row]];
    // start vector: counter-based hash of (eigen index, component)
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      uint64_t z = (uint64_t)(sel[row] + 1) * 0x9E3779B97F4A7C15ull + (uint64_t)(k + 1) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      x[k] = (double)(z >> 11) * 0x1p-53 + 0.5;
    }
    if (threadIdx.x == 0) {
      double cd = d[0] - lam, ce1 = n > 1 ? e[0] : 0.0, ce2 = 0.0;
      for (int k = 0; k < n - 1; ++k) {
        const double sub = e[k];
        const double an = d[k + 1] - lam;
        const double bn = (k + 1 < n - 1) ? e[k + 1] : 0.0;
        if (fabs(cd) >= fabs(sub)) {
          if (cd == 0.0) cd = delta;
          const double l = sub / cd;
          u1[k] = cd;
          u2[k] = ce1;
          u3[k] = ce2;
          pv[k] = 0.0;
          ml[k] = l;
          cd = an - l * ce1;
          ce1 = bn - l * ce2;
          ce2 = 0.0;
        } else {
          const double l = cd / sub;
          u1[k] = sub;
          u2[k] = an;
          u3[k] = bn;
          pv[k] = 1.0;
          ml[k] = l;
          const double nd = ce1 - l * an;
          const double ne1 = ce2 - l * bn;
          cd = nd;
          ce1 = ne1;
          ce2 = 0.0;
        }
      }
      u1[n - 1] = (fabs(cd) < delta) ? (cd < 0 ? -delta : delta) : cd;
    }
    __syncthreads();
    // reciprocals of the pivots, once, by all threads: the solves below then multiply
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const double u = (k < n - 1 && fabs(u1[k]) < delta) ? (u1[k] < 0 ? -delta : delta) : u1[k];
      ru[k] = 1.0 / u;
    }
    __syncthreads();
    for (int iter = 0; iter < 3; ++iter) {
      if (threadIdx.x == 0) {
        for (int k = 0; k < n - 1; ++k) {
          if (pv[k] != 0.0) {
            const double t = x[k];
            x[k] = x[k + 1];
            x[k + 1] = t;
          }
          x[k + 1] -= ml[k] * x[k];
        }
        x[n - 1] *= ru[n - 1];
        if (n > 1) x[n - 2] = (x[n - 2] - u2[n - 2] * x[n - 1]) * ru[n - 2];
        for (int k = n - 3; k >= 0; --k) x[k] = (x[k] - u2[k] * x[k + 1] - u3[k] * x[k + 2]) * ru[k];
      }
      __syncthreads();
      // scale to unit max-norm first so that the dot products below cannot overflow
      double mx = 0.0;
      for (int k = threadIdx.x; k < n; k += blockDim.x) mx = fmax(mx, fabs(x[k]));
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
      __syncthreads();
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
      __syncthreads();
      double m2 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmax(m2, red[w]);
      const double inv = m2 > 0.0 ? 1.0 / m2 : 1.0;
      for (int k = threadIdx.x; k < n; k += blockDim.x) x[k] *= inv;
      __syncthreads();
      // Gram-Schmidt against the earlier vectors of the cluster (twice)
      for (int pass = 0; pass < 2; ++pass)
        for (int pq = 0; pq < q; ++pq) {
          const double *v = it.Zt + (int64_t)(c.first + pq) * n;
          double s = 0.0;
          for (int k = threadIdx.x; k < n; k += blockDim.x) s = fma(x[k], v[k], s);
          const double dot = block_sum(s, red);
          for (int k = threadIdx.x; k < n; k += blockDim.x) x[k] -= dot * v[k];
          __syncthreads();
        }
      double s = 0.0;
      for (int k = threadIdx.x; k < n; k += blockDim.x) s = fma(x[k], x[k], s);
      const double nrm = sqrt(block_sum(s, red));
      const double sc = nrm > 0.0 ? 1.0 / nrm : 0.0;
      for (int k = threadIdx.x; k < n; k += blockDim.x) x[k] *= sc;
      __syncthreads();
    }
    double *out = it.Zt + (int64_t)row * n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) out[k] = x[k];
    __syncthreads();
  }
  (void)ctol;
}

// x = H_0 H_1 ... H_{n-3} z for each tridiagonal eigenvector z (row of Zt); one CTA per vector,
// the vector in shared memory.
struct BackBatchP {
  SymItem s[EIG_MAXB];
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
  __shared__ double red[33];
  for (int k = threadIdx.x; k < n; k += blockDim.x) x[k] = it.Zt[(int64_t)r * n + k];
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

void sym_eig_vectors(cudaStream_t st, const std::vector<BackItem> &items, double ctol) {
  for (size_t s0 = 0; s0 < items.size(); s0 += EIG_MAXB) {
    const int cnt = (int)std::min<size_t>(EIG_MAXB, items.size() - s0);
    InvIterP ip;
    memset(&ip, 0, sizeof(ip));
    BackBatchP bb;
    memset(&bb, 0, sizeof(bb));
    std::vector<Cluster> clusters;
    std::vector<int> allsel;
    std::vector<size_t> seloff(cnt);
    int nmax = 1, selmax = 0;
    for (int i = 0; i < cnt; ++i) {
      const BackItem &bi = items[s0 + i];
      const SymItem &it = *bi.s;
      ip.it[i] = it;
      bb.s[i] = it;
      bb.out[i] = bi.out;
      bb.nsel[i] = (int)bi.sel.size();
      bb.ld_out[i] = bi.ld_out;
      nmax = std::max(nmax, it.n);
      selmax = std::max(selmax, (int)bi.sel.size());
      seloff[i] = allsel.size();
      allsel.insert(allsel.end(), bi.sel.begin(), bi.sel.end());
      if (bi.sel.empty()) continue;
      // clusters of close selected eigenvalues (needs the eigenvalues and the matrix scale)
      std::vector<double> lam(it.n), dd(it.n), ee(it.n);
      RFDD_CUDA(cudaMemcpyAsync(lam.data(), it.lam, it.n * sizeof(double), cudaMemcpyDeviceToHost, st));
      RFDD_CUDA(cudaMemcpyAsync(dd.data(), it.d, it.n * sizeof(double), cudaMemcpyDeviceToHost, st));
      RFDD_CUDA(cudaMemcpyAsync(ee.data(), it.e, it.n * sizeof(double), cudaMemcpyDeviceToHost, st));
      RFDD_CUDA(cudaStreamSynchronize(st));
      double tnorm = 0.0;
      for (int k = 0; k < it.n; ++k)
        tnorm = std::max(tnorm, std::fabs(dd[k]) + (k > 0 ? std::fabs(ee[k - 1]) : 0.0) +
                                    (k < it.n - 1 ? std::fabs(ee[k]) : 0.0));
      int start = 0;
      for (int q = 1; q <= (int)bi.sel.size(); ++q) {
        if (q == (int)bi.sel.size() || lam[bi.sel[q]] - lam[bi.sel[q - 1]] > ctol * tnorm) {
          clusters.push_back({i, start, q - start});
          start = q;
        }
      }
    }
    if (clusters.empty()) continue;
    int *sel_dev = nullptr;
    Cluster *cl_dev = nullptr;
    double *scratch = nullptr;
    const int64_t per = (int64_t)7 * nmax;
    RFDD_CUDA(cudaMallocAsync((void **)&sel_dev, allsel.size() * sizeof(int), st));
    RFDD_CUDA(cudaMallocAsync((void **)&cl_dev, clusters.size() * sizeof(Cluster), st));
    RFDD_CUDA(cudaMallocAsync((void **)&scratch, (size_t)clusters.size() * per * sizeof(double), st));
    RFDD_CUDA(cudaMemcpyAsync(sel_dev, allsel.data(), allsel.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    RFDD_CUDA(cudaMemcpyAsync(cl_dev, clusters.data(), clusters.size() * sizeof(Cluster), cudaMemcpyHostToDevice, st));
    for (int i = 0; i < cnt; ++i) ip.sel[i] = sel_dev + seloff[i];
    inviter_kernel<<<(unsigned)clusters.size(), 256, 0, st>>>(ip, cl_dev, scratch, per, ctol);
    RFDD_CHECK_LAUNCH();
    const size_t smem = (size_t)nmax * sizeof(double);
    RFDD_REQUIRE(smem <= 200 * 1024, RFDD_EINVAL, "sym_eig: order too large");
    RFDD_CUDA(cudaFuncSetAttribute(back_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    back_kernel<<<dim3(selmax, cnt), 256, smem, st>>>(bb);
    RFDD_CHECK_LAUNCH();
    RFDD_CUDA(cudaFreeAsync(sel_dev, st));
    RFDD_CUDA(cudaFreeAsync(cl_dev, st));
    RFDD_CUDA(cudaFreeAsync(scratch, st));
    // host vectors referenced by async copies must outlive them
    RFDD_CUDA(cudaStreamSynchronize(st));
  }
}

}  // namespace rfdd
