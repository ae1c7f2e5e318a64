// Sparse products, block assembly, Schur scatter and elementwise kernels.
#include "ops.cuh"

namespace rfdd {

namespace {

template <typename T>
struct Shift;
template <typename R>
struct Shift<cx<R>> {
  __device__ static cx<R> make(double a, double m, cx<double> z) {
    return cx<R>((R)(a - z.re * m), (R)(-z.im * m));
  }
};
template <>
struct Shift<float> {
  __device__ static float make(double a, double m, cx<double> z) { return (float)(a - z.re * m); }
};
template <>
struct Shift<double> {
  __device__ static double make(double a, double m, cx<double> z) { return a - z.re * m; }
};

}  // namespace

// --------------------------------------------------------------------------------------
// real SpMM, warp per row, lanes over columns
// --------------------------------------------------------------------------------------
__global__ void spmm_f64_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                const double *__restrict__ vals, int64_t r0, int64_t r1, int64_t qlo, int64_t qhi,
                                const double *__restrict__ X, int64_t ldx, double *__restrict__ Y, int64_t ldy,
                                int64_t b, int acc) {
  const int64_t r = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (r >= r1) return;
  const int64_t e0 = rp[r], e1 = rp[r + 1];
  for (int64_t c0 = 0; c0 < b; c0 += 32) {
    const int64_t c = c0 + lane;
    double s = 0.0;
    if (c < b)
      for (int64_t e = e0; e < e1; ++e) {
        const int64_t q = col[e];
        if (q < qlo || q >= qhi) continue;
        s = fma(vals[e], X[(q - qlo) * ldx + c], s);
      }
    if (c < b) {
      double *y = Y + (r - r0) * ldy + c;
      *y = acc ? *y + s : s;
    }
  }
}
__global__ void combine_values_kernel(const double *__restrict__ a, const double *__restrict__ m, double ca, double cm,
                                      int64_t nnz, double *__restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = ca * a[e] + cm * m[e];
}
void spmm_f64(cudaStream_t st, const DevPencil &P, int64_t r0, int64_t r1, int64_t qlo, int64_t qhi, double ca,
              double cm, const double *X, int64_t ldx, double *Y, int64_t ldy, int64_t b, bool accumulate) {
  if (r1 <= r0 || b <= 0) return;
  // the coefficient ca*a + cm*m of each entry, formed once (FP64 is the bound of this kernel)
  const double *vals = nullptr;
  double *comb = nullptr;
  if (ca == 1.0 && cm == 0.0) {
    vals = P.a;
  } else if (ca == 0.0 && cm == 1.0) {
    vals = P.m;
  } else {
    RFDD_CUDA(cudaMallocAsync((void **)&comb, (size_t)std::max<int64_t>(1, P.nnz) * sizeof(double), st));
    combine_values_kernel<<<std::min(4096, ceil_div(std::max<int64_t>(1, P.nnz), 256)), 256, 0, st>>>(P.a, P.m, ca, cm,
                                                                                                    P.nnz, comb);
    RFDD_CHECK_LAUNCH();
    vals = comb;
  }
  const int64_t warps = r1 - r0;
  spmm_f64_kernel<<<ceil_div(warps * 32, 256), 256, 0, st>>>(P.rowptr, P.col, vals, r0, r1, qlo, qhi, X, ldx, Y, ldy,
                                                               b, accumulate ? 1 : 0);
  RFDD_CHECK_LAUNCH();
  if (comb) RFDD_CUDA(cudaFreeAsync(comb, st));
}

// --------------------------------------------------------------------------------------
// complex coupling products (E(z) y and E(z)^T t) in the factor precision
// --------------------------------------------------------------------------------------
template <typename T>
__global__ void couple_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const double *__restrict__ av, const double *__restrict__ mv, int64_t r0, int64_t r1,
                              int64_t qlo, int64_t qhi, const cx<double> *__restrict__ zz, const T *__restrict__ X,
                              int64_t ldx, int64_t strideX, T *__restrict__ Y, int64_t ldy, int64_t strideY, int64_t b,
                              double sign, int acc) {
  using R = typename ST<T>::real;
  const int64_t r = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.y;
  if (r >= r1) return;
  const cx<double> z = zz[l];
  const T *Xl = X + l * strideX;
  T *Yl = Y + l * strideY;
  const int64_t e0 = rp[r], e1 = rp[r + 1];
  for (int64_t c0 = 0; c0 < b; c0 += 32) {
    const int64_t c = c0 + lane;
    if (c >= b) break;
    T s = ST<T>::zero();
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t q = col[e];
      if (q < qlo || q >= qhi) continue;
      const T v = Shift<T>::make(av[e], mv[e], z);
      s = ST<T>::fma(v, Xl[(q - qlo) * ldx + c], s);
    }
    T *y = Yl + (r - r0) * ldy + c;
    T out = (R)sign * s;
    *y = acc ? *y + out : out;
  }
}

template <typename T>
void couple(cudaStream_t st, const DevPencil &P, int64_t r0, int64_t r1, int64_t qlo, int64_t qhi,
            const cx<double> *z_dev, int nnodes, const T *X, int64_t ldx, int64_t strideX, T *Y, int64_t ldy,
            int64_t strideY, int64_t b, double sign, bool accumulate) {
  if (r1 <= r0 || b <= 0 || nnodes <= 0) return;
  dim3 grid(ceil_div((r1 - r0) * 32, 256), nnodes);
  couple_kernel<T><<<grid, 256, 0, st>>>(P.rowptr, P.col, P.a, P.m, r0, r1, qlo, qhi, z_dev, X, ldx, strideX, Y, ldy,
                                         strideY, b, sign, accumulate ? 1 : 0);
  RFDD_CHECK_LAUNCH();
}

// --------------------------------------------------------------------------------------
// FP64 shifted residual R = V - (A - zM) X (complex)
// --------------------------------------------------------------------------------------
__global__ void shifted_residual_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                        const double *__restrict__ av, const double *__restrict__ mv, int64_t n,
                                        const cx<double> *__restrict__ zz, const cx<double> *__restrict__ V,
                                        int64_t strideV, const cx<double> *__restrict__ X, cx<double> *__restrict__ Rr,
                                        int64_t stride, int64_t b) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.y;
  if (r >= n) return;
  const cx<double> z = zz[l];
  const cx<double> *Xl = X + l * stride;
  const int64_t e0 = rp[r], e1 = rp[r + 1];
  for (int64_t c0 = 0; c0 < b; c0 += 32) {
    const int64_t c = c0 + lane;
    if (c >= b) break;
    // (A x) and (M x) with real coefficients (4 FP64 FMAs per entry), then A x - z M x
    double ar = 0.0, ai = 0.0, mr = 0.0, mi = 0.0;
    for (int64_t e = e0; e < e1; ++e) {
      const cx<double> x = Xl[(int64_t)col[e] * b + c];
      const double a = av[e], m = mv[e];
      ar = fma(a, x.re, ar);
      ai = fma(a, x.im, ai);
      mr = fma(m, x.re, mr);
      mi = fma(m, x.im, mi);
    }
    const double sr = ar - (z.re * mr - z.im * mi);
    const double si = ai - (z.re * mi + z.im * mr);
    const cx<double> v = V[l * strideV + r * b + c];
    Rr[l * stride + r * b + c] = cx<double>(v.re - sr, v.im - si);
  }
}

void shifted_residual(cudaStream_t st, const DevPencil &P, const cx<double> *z_dev, int nnodes,
                      const cx<double> *V, int64_t strideV, const cx<double> *X, cx<double> *R, int64_t stride,
                      int64_t b) {
  dim3 grid(ceil_div(P.n * 32, 256), nnodes);
  shifted_residual_kernel<<<grid, 256, 0, st>>>(P.rowptr, P.col, P.a, P.m, P.n, z_dev, V, strideV, X, R, stride, b);
  RFDD_CHECK_LAUNCH();
}

// Double-FP32 variant.  The residual only has to resolve a scaled backward error a little
// below the refinement target (1e-12 of (||A|| + |z| ||M||) ||x|| by default); split operands
// (x = hi + lo, |x - hi - lo| <= 2^-48 |x|), error-free products (FMA) and compensated sums
// give about 2^-46 of sum |a||x| per product sum at FP32 throughput, instead of the FP64
// pipes that bound the FP64 kernel above.
__device__ __forceinline__ void df_mac(float &s, float &c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);
  const float t = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
  const float s1 = __fadd_rn(s, p);
  const float bb = __fsub_rn(s1, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bb)), __fsub_rn(p, bb));
  s = s1;
  c = __fadd_rn(c, __fadd_rn(err, t));
}
__device__ __forceinline__ void split_d(double v, float &hi, float &lo) {
  hi = __double2float_rn(v);
  lo = __double2float_rn(v - (double)hi);
}
__global__ void split_pencil_kernel(const double *__restrict__ a, const double *__restrict__ m, int64_t nnz,
                                    float4 *__restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    float4 w;
    split_d(a[e], w.x, w.y);
    split_d(m[e], w.z, w.w);
    out[e] = w;
  }
}
void split_pencil(cudaStream_t st, DevPencil &P, float4 *out) {
  if (P.nnz > 0) {
    split_pencil_kernel<<<std::min(4096, ceil_div(P.nnz, 256)), 256, 0, st>>>(P.a, P.m, P.nnz, out);
    RFDD_CHECK_LAUNCH();
  }
  P.am_split = out;
}
__global__ void split_c64_kernel(const cx<double> *__restrict__ X, float4 *__restrict__ Xs, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const cx<double> x = X[e];
    float4 w;
    split_d(x.re, w.x, w.y);
    split_d(x.im, w.z, w.w);
    Xs[e] = w;
  }
}
void split_c64(cudaStream_t st, const cx<double> *X, float4 *Xs, int64_t count) {
  if (count <= 0) return;
  split_c64_kernel<<<(unsigned)std::min<int64_t>(16384, ceil_div(count, 256)), 256, 0, st>>>(X, Xs, count);
  RFDD_CHECK_LAUNCH();
}
__global__ void shifted_residual_df_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                           const float4 *__restrict__ am, int64_t n, const cx<double> *__restrict__ zz,
                                           const cx<double> *__restrict__ V, int64_t strideV,
                                           const float4 *__restrict__ Xs, cx<double> *__restrict__ Rr, int64_t stride,
                                           int64_t b) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.y;
  if (r >= n) return;
  const cx<double> z = zz[l];
  const float4 *Xl = Xs + l * stride;
  const int64_t e0 = rp[r], e1 = rp[r + 1];
  for (int64_t c0 = 0; c0 < b; c0 += 32) {
    const int64_t c = c0 + lane;
    if (c >= b) break;
    // (A x) and (M x), real and imaginary parts, each as an unevaluated pair (s, t); the loads of
    // four entries are issued before their products (the column index, then the operand, is a
    // chain of two dependent loads per entry), the products are formed in entry order
    float s0 = 0.f, t0 = 0.f, s1 = 0.f, t1 = 0.f, s2 = 0.f, t2 = 0.f, s3 = 0.f, t3 = 0.f;
    int64_t e = e0;
    for (; e + 4 <= e1; e += 4) {
      int32_t q[4];
      float4 x[4], w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = col[e + u];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[u] = Xl[(int64_t)q[u] * b + c];
        w[u] = am[e + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        df_mac(s0, t0, w[u].x, w[u].y, x[u].x, x[u].y);
        df_mac(s1, t1, w[u].x, w[u].y, x[u].z, x[u].w);
        df_mac(s2, t2, w[u].z, w[u].w, x[u].x, x[u].y);
        df_mac(s3, t3, w[u].z, w[u].w, x[u].z, x[u].w);
      }
    }
    for (; e < e1; ++e) {
      const float4 x = Xl[(int64_t)col[e] * b + c];
      const float4 w = am[e];
      df_mac(s0, t0, w.x, w.y, x.x, x.y);
      df_mac(s1, t1, w.x, w.y, x.z, x.w);
      df_mac(s2, t2, w.z, w.w, x.x, x.y);
      df_mac(s3, t3, w.z, w.w, x.z, x.w);
    }
    const double ar = (double)s0 + (double)t0, ai = (double)s1 + (double)t1;
    const double mr = (double)s2 + (double)t2, mi = (double)s3 + (double)t3;
    const double sr = ar - (z.re * mr - z.im * mi);
    const double si = ai - (z.re * mi + z.im * mr);
    const cx<double> v = V[l * strideV + r * b + c];
    Rr[l * stride + r * b + c] = cx<double>(v.re - sr, v.im - si);
  }
}
// (A X, M X) for a real FP64 block X (n x b, ld b): products in double-FP32 on split operands
__global__ void split_f64_kernel(const double *__restrict__ X, float2 *__restrict__ Xs, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    float2 w;
    split_d(X[e], w.x, w.y);
    Xs[e] = w;
  }
}
__global__ void spmm_am_df_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                  const float4 *__restrict__ am, int64_t n, const float2 *__restrict__ Xs,
                                  double *__restrict__ YA, double *__restrict__ YM, int64_t b) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  const int64_t e0 = rp[r], e1 = rp[r + 1];
  for (int64_t c0 = 0; c0 < b; c0 += 32) {
    const int64_t c = c0 + lane;
    if (c >= b) break;
    float sa = 0.f, ta = 0.f, sm = 0.f, tm = 0.f;
    for (int64_t e = e0; e < e1; ++e) {
      const float2 x = Xs[(int64_t)col[e] * b + c];
      const float4 w = am[e];
      df_mac(sa, ta, w.x, w.y, x.x, x.y);
      df_mac(sm, tm, w.z, w.w, x.x, x.y);
    }
    YA[r * b + c] = (double)sa + (double)ta;
    YM[r * b + c] = (double)sm + (double)tm;
  }
}
void spmm_am_df(cudaStream_t st, const DevPencil &P, const double *X, double *YA, double *YM, int64_t b) {
  RFDD_REQUIRE(P.am_split != nullptr, RFDD_ESTATE, "split pencil values missing");
  if (P.n <= 0 || b <= 0) return;
  float2 *Xs = nullptr;
  const int64_t count = P.n * b;
  RFDD_CUDA(cudaMallocAsync((void **)&Xs, (size_t)count * sizeof(float2), st));
  split_f64_kernel<<<(unsigned)std::min<int64_t>(16384, ceil_div(count, 256)), 256, 0, st>>>(X, Xs, count);
  RFDD_CHECK_LAUNCH();
  spmm_am_df_kernel<<<ceil_div(P.n * 32, 256), 256, 0, st>>>(P.rowptr, P.col, P.am_split, P.n, Xs, YA, YM, b);
  RFDD_CHECK_LAUNCH();
  RFDD_CUDA(cudaFreeAsync(Xs, st));
}
void shifted_residual_df(cudaStream_t st, const DevPencil &P, const cx<double> *z_dev, int nnodes,
                         const cx<double> *V, int64_t strideV, const float4 *Xs, cx<double> *R, int64_t stride,
                         int64_t b) {
  RFDD_REQUIRE(P.am_split != nullptr, RFDD_ESTATE, "split pencil values missing");
  dim3 grid(ceil_div(P.n * 32, 256), nnodes);
  shifted_residual_df_kernel<<<grid, 256, 0, st>>>(P.rowptr, P.col, P.am_split, P.n, z_dev, V, strideV, Xs, R, stride,
                                                   b);
  RFDD_CHECK_LAUNCH();
}

// --------------------------------------------------------------------------------------
// a2: assemble dense (bordered) shifted blocks; warp per row
// --------------------------------------------------------------------------------------
template <typename T>
__global__ void assemble_blocks_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                       const double *__restrict__ av, const double *__restrict__ mv, int p,
                                       int64_t dsum, int64_t s, const int64_t *__restrict__ off,
                                       const int32_t *__restrict__ sidx, const int64_t *__restrict__ sidx_off,
                                       const int32_t *__restrict__ posmap, const int64_t *__restrict__ Doff,
                                       int64_t total_rows, const int64_t *__restrict__ boff,
                                       const cx<double> *__restrict__ zz, T *__restrict__ base, int border) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.y;
  if (g >= total_rows) return;
  int lo = 0, hi = p;  // find j with Doff[j] <= g < Doff[j+1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (Doff[mid] <= g) lo = mid; else hi = mid;
  }
  const int j = lo;
  const int64_t dj = off[j + 1] - off[j];
  const int64_t sj = sidx_off[j + 1] - sidx_off[j];
  const int64_t Dj = border ? dj + sj : dj;
  const int64_t i = g - Doff[j];
  T *row = base + boff[(int64_t)l * p + j] + i * Dj;
  const cx<double> z = zz[l];
  for (int64_t c = lane; c < Dj; c += 32) row[c] = ST<T>::zero();
  __syncwarp();
  const int32_t *pm = posmap + (int64_t)j * s;
  if (i < dj) {
    const int64_t r = off[j] + i;
    for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += 32) {
      const int64_t q = col[e];
      if (q < dsum) {
        row[q - off[j]] = Shift<T>::make(av[e], mv[e], z);
      } else if (border) {
        const int pos = pm[q - dsum];
        row[dj + pos] = Shift<T>::make(av[e], mv[e], z);
      }
    }
  } else {
    const int64_t a = sidx[sidx_off[j] + (i - dj)];
    const int64_t r = dsum + a;
    for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += 32) {
      const int64_t q = col[e];
      if (q >= off[j] && q < off[j + 1]) row[q - off[j]] = Shift<T>::make(av[e], mv[e], z);
    }
  }
}

template <typename T>
void assemble_blocks(cudaStream_t st, const DevPencil &P, const DevDD &dd, const int64_t *dev_D_off,
                     int64_t total_rows, const int64_t *dev_boff, const cx<double> *z_dev, int nnodes, T *base,
                     bool border) {
  if (total_rows <= 0) return;
  dim3 grid(ceil_div(total_rows * 32, 256), nnodes);
  assemble_blocks_kernel<T><<<grid, 256, 0, st>>>(P.rowptr, P.col, P.a, P.m, dd.p, dd.dsum, dd.s, dd.off, dd.sidx,
                                                  dd.sidx_off, dd.posmap, dev_D_off, total_rows, dev_boff, z_dev, base,
                                                  border ? 1 : 0);
  RFDD_CHECK_LAUNCH();
}

template <typename T>
__global__ void assemble_interface_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                          const double *__restrict__ av, const double *__restrict__ mv,
                                          int64_t dsum, int64_t s, const cx<double> *__restrict__ zz,
                                          T *__restrict__ S) {
  const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.y;
  if (a >= s) return;
  T *row = S + (int64_t)l * s * s + a * s;
  for (int64_t c = lane; c < s; c += 32) row[c] = ST<T>::zero();
  __syncwarp();
  const cx<double> z = zz[l];
  const int64_t r = dsum + a;
  for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += 32) {
    const int64_t q = col[e];
    if (q >= dsum) row[q - dsum] = Shift<T>::make(av[e], mv[e], z);
  }
}

template <typename T>
void assemble_interface(cudaStream_t st, const DevPencil &P, const DevDD &dd, const cx<double> *z_dev,
                        int nnodes, T *S) {
  dim3 grid(ceil_div(dd.s * 32, 256), nnodes);
  assemble_interface_kernel<T><<<grid, 256, 0, st>>>(P.rowptr, P.col, P.a, P.m, dd.dsum, dd.s, z_dev, S);
  RFDD_CHECK_LAUNCH();
}

template <typename T>
__global__ void scatter_schur_kernel(const int32_t *__restrict__ sidx_j, int p, int j, int dj, int sj, int64_t s,
                                     const int64_t *__restrict__ boff, const T *__restrict__ base,
                                     T *__restrict__ S) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int l = blockIdx.y;
  if (e >= (int64_t)sj * sj) return;
  const int a = (int)(e / sj), b = (int)(e % sj);
  const int64_t Dj = (int64_t)dj + sj;
  const T *trail = base + boff[(int64_t)l * p + j] + (int64_t)dj * Dj + dj;
  T *dst = S + (int64_t)l * s * s + (int64_t)sidx_j[a] * s + sidx_j[b];
  *dst = *dst + trail[(int64_t)a * Dj + b];
}

template <typename T>
void scatter_schur(cudaStream_t st, const DevDD &dd, int j, int dj, int sj, int64_t sidx_start,
                   const int64_t *dev_boff, const T *base, int nnodes, T *S) {
  if (sj <= 0) return;
  dim3 grid(ceil_div((int64_t)sj * sj, 256), nnodes);
  scatter_schur_kernel<T><<<grid, 256, 0, st>>>(dd.sidx + sidx_start, dd.p, j, dj, sj, dd.s, dev_boff, base, S);
  RFDD_CHECK_LAUNCH();
}

// --------------------------------------------------------------------------------------
// elementwise
// --------------------------------------------------------------------------------------
template <typename TO, typename TI>
__global__ void convert_kernel(const TI *__restrict__ x, TO *__restrict__ y, int64_t n);

#define RFDD_CONV_RR(TO, TI)                                                                           \
  template <>                                                                                          \
  __global__ void convert_kernel<TO, TI>(const TI *__restrict__ x, TO *__restrict__ y, int64_t n) {    \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) \
      y[i] = (TO)x[i];                                                                                 \
  }
#define RFDD_CONV_CC(RO, RI)                                                                           \
  template <>                                                                                          \
  __global__ void convert_kernel<cx<RO>, cx<RI>>(const cx<RI> *__restrict__ x, cx<RO> *__restrict__ y, int64_t n) { \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) \
      y[i] = cx<RO>((RO)x[i].re, (RO)x[i].im);                                                         \
  }
RFDD_CONV_RR(float, double)
RFDD_CONV_RR(double, float)
RFDD_CONV_RR(double, double)
RFDD_CONV_RR(float, float)
RFDD_CONV_CC(float, double)
RFDD_CONV_CC(double, float)
RFDD_CONV_CC(double, double)
RFDD_CONV_CC(float, float)

static int grid_for(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 152 * 32); }

template <typename TO, typename TI>
void convert(cudaStream_t st, const TI *x, TO *y, int64_t n) {
  if (n <= 0) return;
  convert_kernel<TO, TI><<<grid_for(n), 256, 0, st>>>(x, y, n);
  RFDD_CHECK_LAUNCH();
}
template void convert<float, double>(cudaStream_t, const double *, float *, int64_t);
template void convert<double, float>(cudaStream_t, const float *, double *, int64_t);
template void convert<double, double>(cudaStream_t, const double *, double *, int64_t);
template void convert<float, float>(cudaStream_t, const float *, float *, int64_t);
template void convert<cx<float>, cx<double>>(cudaStream_t, const cx<double> *, cx<float> *, int64_t);
template void convert<cx<double>, cx<float>>(cudaStream_t, const cx<float> *, cx<double> *, int64_t);
template void convert<cx<double>, cx<double>>(cudaStream_t, const cx<double> *, cx<double> *, int64_t);
template void convert<cx<float>, cx<float>>(cudaStream_t, const cx<float> *, cx<float> *, int64_t);

template <typename T>
__global__ void real_to_complex_kernel(const double *__restrict__ x, T *__restrict__ y, int64_t n, int nrep,
                                       int64_t stride) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T v = ST<T>::from_re(x[i]);
    for (int r = 0; r < nrep; ++r) y[r * stride + i] = v;
  }
}
template <typename T>
void real_to_complex(cudaStream_t st, const double *x, T *y, int64_t n, int nrep, int64_t stride) {
  if (n <= 0) return;
  real_to_complex_kernel<T><<<grid_for(n), 256, 0, st>>>(x, y, n, nrep, stride);
  RFDD_CHECK_LAUNCH();
}

template <typename T>
__global__ void weighted_real_sum_kernel(const T *__restrict__ Y, int64_t strideY, const cx<double> *__restrict__ w,
                                         int nnodes, double scale, double *__restrict__ W, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < nnodes; ++l) {
      const T y = Y[l * strideY + i];
      acc += w[l].re * (double)y.re - w[l].im * (double)y.im;
    }
    W[i] = scale * acc;
  }
}
template <typename T>
void weighted_real_sum(cudaStream_t st, const T *Y, int64_t strideY, const cx<double> *w_dev, int nnodes,
                       double scale, double *W, int64_t count) {
  if (count <= 0) return;
  weighted_real_sum_kernel<T><<<grid_for(count), 256, 0, st>>>(Y, strideY, w_dev, nnodes, scale, W, count);
  RFDD_CHECK_LAUNCH();
}

__global__ void axpy_f64_kernel(double a, const double *__restrict__ x, double *__restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}
void axpy_f64(cudaStream_t st, double a, const double *x, double *y, int64_t n) {
  if (n <= 0) return;
  axpy_f64_kernel<<<grid_for(n), 256, 0, st>>>(a, x, y, n);
  RFDD_CHECK_LAUNCH();
}
__global__ void axpy_c64_kernel(const cx<double> *__restrict__ x, cx<double> *__restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = y[i] + x[i];
}
void axpy_c64(cudaStream_t st, const cx<double> *x, cx<double> *y, int64_t n) {
  if (n <= 0) return;
  axpy_c64_kernel<<<grid_for(n), 256, 0, st>>>(x, y, n);
  RFDD_CHECK_LAUNCH();
}

__global__ void scale_cols_kernel(double *X, int64_t n, int64_t b, int64_t ld, const double *__restrict__ s) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * b; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / b, c = e % b;
    X[i * ld + c] *= s[c];
  }
}
void scale_cols_f64(cudaStream_t st, double *X, int64_t n, int64_t b, int64_t ld, const double *s) {
  if (n * b <= 0) return;
  scale_cols_kernel<<<grid_for(n * b), 256, 0, st>>>(X, n, b, ld, s);
  RFDD_CHECK_LAUNCH();
}

// SplitMix64 (Vigna): value i of stream `stream` is mix(seed + (stream*2^32 + i + 1)*golden),
// mapped to (mix >> 11) * 2^-52 - 1 in [-1, 1).
__global__ void counter_uniform_kernel(uint64_t seed, uint64_t stream, double *x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t c = (stream << 32) + (uint64_t)i + 1ull;
    uint64_t z = seed + c * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    x[i] = (double)(z >> 11) * 0x1p-52 - 1.0;
  }
}
void counter_uniform_dev(cudaStream_t st, uint64_t seed, uint64_t stream, double *x, int64_t n) {
  if (n <= 0) return;
  counter_uniform_kernel<<<grid_for(n), 256, 0, st>>>(seed, stream, x, n);
  RFDD_CHECK_LAUNCH();
}

// column dots: one CTA per column, fixed-order tree reduction (reproducible)
__global__ void col_dots_kernel(const double *__restrict__ X, int64_t ldx, const double *__restrict__ Y, int64_t ldy,
                                int64_t n, double *out) {
  const int64_t c = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(X[i * ldx + c], Y[i * ldy + c], s);
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}
void col_dots(cudaStream_t st, const double *X, int64_t ldx, const double *Y, int64_t ldy, int64_t n, int64_t b,
              double *out) {
  if (b <= 0) return;
  col_dots_kernel<<<(unsigned)b, 256, 0, st>>>(X, ldx, Y, ldy, n, out);
  RFDD_CHECK_LAUNCH();
}

__global__ void col_norms2_c64_kernel(const cx<double> *__restrict__ R, int64_t n, int64_t b, int64_t stride,
                                      double *out) {
  const int64_t c = blockIdx.x;
  const int l = blockIdx.y;
  const cx<double> *Rl = R + l * stride;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const cx<double> v = Rl[i * b + c];
    s = fma(v.re, v.re, fma(v.im, v.im, s));
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(int64_t)l * b + c] = red[0];
}
void col_norms2_c64(cudaStream_t st, const cx<double> *R, int64_t n, int64_t b, int nnodes, int64_t stride,
                    double *out) {
  if (b <= 0 || nnodes <= 0) return;
  col_norms2_c64_kernel<<<dim3((unsigned)b, nnodes), 256, 0, st>>>(R, n, b, stride, out);
  RFDD_CHECK_LAUNCH();
}

__global__ void copy_rows_kernel(const double *__restrict__ src, int64_t lds, double *__restrict__ dst, int64_t ldd,
                                 int64_t nrows, int64_t ncols) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nrows * ncols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ncols, c = e % ncols;
    dst[i * ldd + c] = src[i * lds + c];
  }
}
void copy_rows_f64(cudaStream_t st, const double *src, int64_t lds, double *dst, int64_t ldd, int64_t nrows,
                   int64_t ncols) {
  if (nrows * ncols <= 0) return;
  copy_rows_kernel<<<grid_for(nrows * ncols), 256, 0, st>>>(src, lds, dst, ldd, nrows, ncols);
  RFDD_CHECK_LAUNCH();
}

__global__ void gather_rows_kernel(const double *__restrict__ src, int64_t lds, const int64_t *__restrict__ idx,
                                   double *__restrict__ dst, int64_t ldd, int64_t nrows, int64_t ncols) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nrows * ncols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ncols, c = e % ncols;
    dst[i * ldd + c] = src[idx[i] * lds + c];
  }
}
void gather_rows_f64(cudaStream_t st, const double *src, int64_t lds, const int64_t *idx, double *dst,
                     int64_t ldd, int64_t nrows, int64_t ncols) {
  if (nrows * ncols <= 0) return;
  gather_rows_kernel<<<grid_for(nrows * ncols), 256, 0, st>>>(src, lds, idx, dst, ldd, nrows, ncols);
  RFDD_CHECK_LAUNCH();
}

__global__ void gather_rows_cols_kernel(const double *__restrict__ src, int64_t lds, const int64_t *__restrict__ ridx,
                                        const int64_t *__restrict__ cidx, double *__restrict__ dst, int64_t ldd,
                                        int64_t nrows, int64_t ncols) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nrows * ncols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ncols, c = e % ncols;
    dst[i * ldd + c] = src[ridx[i] * lds + cidx[c]];
  }
}
void gather_rows_cols_f64(cudaStream_t st, const double *src, int64_t lds, const int64_t *ridx, const int64_t *cidx,
                          double *dst, int64_t ldd, int64_t nrows, int64_t ncols) {
  if (nrows * ncols <= 0) return;
  gather_rows_cols_kernel<<<grid_for(nrows * ncols), 256, 0, st>>>(src, lds, ridx, cidx, dst, ldd, nrows, ncols);
  RFDD_CHECK_LAUNCH();
}

#define RFDD_INST_OPS(T)                                                                                     \
  template void assemble_blocks<T>(cudaStream_t, const DevPencil &, const DevDD &, const int64_t *, int64_t, \
                                   const int64_t *, const cx<double> *, int, T *, bool);
RFDD_INST_OPS(float)
RFDD_INST_OPS(double)
RFDD_INST_OPS(cx<float>)
RFDD_INST_OPS(cx<double>)

#define RFDD_INST_OPSC(T)                                                                                         \
  template void assemble_interface<T>(cudaStream_t, const DevPencil &, const DevDD &, const cx<double> *, int, T *); \
  template void scatter_schur<T>(cudaStream_t, const DevDD &, int, int, int, int64_t, const int64_t *, const T *, int, T *);    \
  template void couple<T>(cudaStream_t, const DevPencil &, int64_t, int64_t, int64_t, int64_t, const cx<double> *,  \
                          int, const T *, int64_t, int64_t, T *, int64_t, int64_t, int64_t, double, bool);           \
  template void real_to_complex<T>(cudaStream_t, const double *, T *, int64_t, int, int64_t);                        \
  template void weighted_real_sum<T>(cudaStream_t, const T *, int64_t, const cx<double> *, int, double, double *,   \
                                     int64_t);
RFDD_INST_OPSC(cx<float>)
RFDD_INST_OPSC(cx<double>)
// real shift (inertia counts)
template void assemble_interface<double>(cudaStream_t, const DevPencil &, const DevDD &, const cx<double> *, int,
                                         double *);
template void scatter_schur<double>(cudaStream_t, const DevDD &, int, int, int, int64_t, const int64_t *,
                                    const double *, int, double *);


// ---------------------------------------------------------------------------------------
// Interface gather / ordered scatter for the bordered-factor DD solve
// ---------------------------------------------------------------------------------------
// Yj_l[a][c] = G_l[sidx_j[a]][c]  for all nodes l
template <typename T>
__global__ void gather_iface_kernel(const int32_t *__restrict__ sidx_j, int sj, int64_t m, const T *__restrict__ G,
                                    int64_t strideG, T *__restrict__ Y, int64_t strideY) {
  const int l = blockIdx.y;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)sj * m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / m, c = e % m;
    Y[l * strideY + e] = G[l * strideG + (int64_t)sidx_j[a] * m + c];
  }
}
template <typename T>
void gather_iface(cudaStream_t st, const int32_t *sidx_j, int sj, int64_t m, const T *G, int64_t strideG, T *Y,
                  int64_t strideY, int nnodes) {
  if (sj <= 0 || m <= 0) return;
  gather_iface_kernel<T><<<dim3(std::min(4096, ceil_div((int64_t)sj * m, 256)), nnodes), 256, 0, st>>>(
      sidx_j, sj, m, G, strideG, Y, strideY);
  RFDD_CHECK_LAUNCH();
}
// G_l[sidx_j[a]][c] -= Rj_l[a][c]; called for j = 0..p-1 in order (reproducible sums)
template <typename T>
__global__ void scatter_sub_iface_kernel(const int32_t *__restrict__ sidx_j, int sj, int64_t m, const T *__restrict__ Rj,
                                         int64_t strideR, T *__restrict__ G, int64_t strideG) {
  const int l = blockIdx.y;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)sj * m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / m, c = e % m;
    T *g = G + l * strideG + (int64_t)sidx_j[a] * m + c;
    *g = *g - Rj[l * strideR + e];
  }
}
template <typename T>
void scatter_sub_iface(cudaStream_t st, const int32_t *sidx_j, int sj, int64_t m, const T *Rj, int64_t strideR, T *G,
                       int64_t strideG, int nnodes) {
  if (sj <= 0 || m <= 0) return;
  scatter_sub_iface_kernel<T><<<dim3(std::min(4096, ceil_div((int64_t)sj * m, 256)), nnodes), 256, 0, st>>>(
      sidx_j, sj, m, Rj, strideR, G, strideG);
  RFDD_CHECK_LAUNCH();
}
template void gather_iface<cx<float>>(cudaStream_t, const int32_t *, int, int64_t, const cx<float> *, int64_t,
                                      cx<float> *, int64_t, int);
template void gather_iface<cx<double>>(cudaStream_t, const int32_t *, int, int64_t, const cx<double> *, int64_t,
                                       cx<double> *, int64_t, int);
template void scatter_sub_iface<cx<float>>(cudaStream_t, const int32_t *, int, int64_t, const cx<float> *, int64_t,
                                           cx<float> *, int64_t, int);
template void scatter_sub_iface<cx<double>>(cudaStream_t, const int32_t *, int, int64_t, const cx<double> *, int64_t,
                                            cx<double> *, int64_t, int);


// ---------------------------------------------------------------------------------------
// Two-level interface factorisation: assembly of the level storage of each node
// (S2 = level-2 block s2 x s2 at offset 0, then one bordered block per group)
// ---------------------------------------------------------------------------------------
// L_l[edst[e]] = (a - z_l m) of interface CSR entry e0 + e, for entries with edst[e] >= 0
template <typename T>
__global__ void assemble_iface_levels_kernel(const double *__restrict__ av, const double *__restrict__ mv, int64_t e0,
                                             int64_t ne, const int64_t *__restrict__ edst,
                                             const cx<double> *__restrict__ zz, T *__restrict__ L, int64_t tsz) {
  const int l = blockIdx.y;
  const cx<double> z = zz[l];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = edst[e];
    if (d >= 0) L[(int64_t)l * tsz + d] = Shift<T>::make(av[e0 + e], mv[e0 + e], z);
  }
}
template <typename T>
void assemble_iface_levels(cudaStream_t st, const DevPencil &P, int64_t e0, int64_t ne, const int64_t *edst,
                           const cx<double> *z_dev, int nnodes, T *L, int64_t tsz) {
  if (ne <= 0) return;
  assemble_iface_levels_kernel<T><<<dim3(std::min<int64_t>(4096, ceil_div(ne, 256)), nnodes), 256, 0, st>>>(
      P.a, P.m, e0, ne, edst, z_dev, L, tsz);
  RFDD_CHECK_LAUNCH();
}

// Trailing block of subdomain j's bordered factor into the level storage: entry (t, u) goes to
// S2[r[t]][r[u]] when both are level 2, else to the group block at (q[t], q[u]).
template <typename T>
__global__ void scatter_schur_levels_kernel(int p, int j, int dj, int sj, const int32_t *__restrict__ q,
                                            const int32_t *__restrict__ r, int64_t s2, int64_t gbase, int64_t Dg,
                                            const int64_t *__restrict__ boff, const T *__restrict__ base,
                                            T *__restrict__ L, int64_t tsz) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int l = blockIdx.y;
  if (e >= (int64_t)sj * sj) return;
  const int t = (int)(e / sj), u = (int)(e % sj);
  const int64_t Dj = (int64_t)dj + sj;
  const T v = base[boff[(int64_t)l * p + j] + (int64_t)dj * Dj + dj + (int64_t)t * Dj + u];
  const int rt = r[t], ru = r[u];
  T *dst = L + (int64_t)l * tsz + ((rt >= 0 && ru >= 0) ? (int64_t)rt * s2 + ru : gbase + (int64_t)q[t] * Dg + q[u]);
  *dst = *dst + v;
}
template <typename T>
void scatter_schur_levels(cudaStream_t st, int p, int j, int dj, int sj, const int32_t *q_j, const int32_t *r_j,
                          int64_t s2, int64_t gbase, int64_t Dg, const int64_t *dev_boff, const T *base, int nnodes,
                          T *L, int64_t tsz) {
  if (sj <= 0) return;
  scatter_schur_levels_kernel<T><<<dim3(ceil_div((int64_t)sj * sj, 256), nnodes), 256, 0, st>>>(
      p, j, dj, sj, q_j, r_j, s2, gbase, Dg, dev_boff, base, L, tsz);
  RFDD_CHECK_LAUNCH();
}

// Trailing block of group g's bordered factor (n2 x n2 at gbase + n1 (Dg + 1), ld Dg) added to
// S2 at the level-2 positions i2g[0..n2)
template <typename T>
__global__ void scatter_trail_levels_kernel(const int32_t *__restrict__ i2g, int n1, int n2, int64_t gbase,
                                            int64_t s2, T *__restrict__ L, int64_t tsz) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int l = blockIdx.y;
  if (e >= (int64_t)n2 * n2) return;
  const int t = (int)(e / n2), u = (int)(e % n2);
  const int64_t Dg = (int64_t)n1 + n2;
  T *Ll = L + (int64_t)l * tsz;
  const T v = Ll[gbase + (int64_t)n1 * Dg + n1 + (int64_t)t * Dg + u];
  T *dst = Ll + (int64_t)i2g[t] * s2 + i2g[u];
  *dst = *dst + v;
}
template <typename T>
void scatter_trail_levels(cudaStream_t st, const int32_t *i2g, int n1, int n2, int64_t gbase, int64_t s2, int nnodes,
                          T *L, int64_t tsz) {
  if (n2 <= 0) return;
  scatter_trail_levels_kernel<T><<<dim3(ceil_div((int64_t)n2 * n2, 256), nnodes), 256, 0, st>>>(i2g, n1, n2, gbase,
                                                                                                  s2, L, tsz);
  RFDD_CHECK_LAUNCH();
}

#define RFDD_INST_LEVELS(T)                                                                                      \
  template void assemble_iface_levels<T>(cudaStream_t, const DevPencil &, int64_t, int64_t, const int64_t *,    \
                                         const cx<double> *, int, T *, int64_t);                                \
  template void scatter_schur_levels<T>(cudaStream_t, int, int, int, int, const int32_t *, const int32_t *,     \
                                        int64_t, int64_t, int64_t, const int64_t *, const T *, int, T *, int64_t); \
  template void scatter_trail_levels<T>(cudaStream_t, const int32_t *, int, int, int64_t, int64_t, int, T *, int64_t);
RFDD_INST_LEVELS(cx<float>)
RFDD_INST_LEVELS(cx<double>)

}  // namespace rfdd
