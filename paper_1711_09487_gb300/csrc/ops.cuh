// Sparse, assembly and elementwise kernels of the RF-DDES path (host launchers).
#pragma once
#include "common.cuh"

namespace rfdd {

// Pencil on the interior-first ordering as one CSR holding both values per entry (union of the
// patterns of A and M).
struct DevPencil {
  int64_t n = 0, nnz = 0;
  int64_t *rowptr = nullptr;  // n+1
  int32_t *col = nullptr;     // nnz
  double *a = nullptr;        // A values
  double *m = nullptr;        // M values
  float4 *am_split = nullptr; // per entry (hi(a), lo(a), hi(m), lo(m)): double-FP32 copies
};

// Subdomain geometry on the device.
struct DevDD {
  int p = 0;
  int64_t dsum = 0, s = 0;
  int64_t *off = nullptr;       // p+1 interior offsets
  int32_t *sidx = nullptr;      // concatenated sidx_j (interface indices coupled to subdomain j)
  int64_t *sidx_off = nullptr;  // p+1 offsets into sidx
  int32_t *posmap = nullptr;    // p x s: position of interface index in sidx_j, or -1
};

// Y[r][c] (=|+=) sum over entries (r, q) of the pencil with q in [qlo, qhi) of
//   (ca*a + cm*m) * X[q - qlo][c],  rows r in [r0, r1); X, Y real row-major with b columns.
void spmm_f64(cudaStream_t st, const DevPencil &P, int64_t r0, int64_t r1, int64_t qlo, int64_t qhi, double ca,
              double cm, const double *X, int64_t ldx, double *Y, int64_t ldy, int64_t b, bool accumulate);

// Complex coupling product in the factor precision:
//   Y[r - r0][c] = beta_y * Y[...] + sign * sum_{q in [qlo,qhi)} (a - z m)(r, q) * X[q - qlo][c]
// for all nodes l (z[l], X + l*strideX, Y + l*strideY).
template <typename T>
void couple(cudaStream_t st, const DevPencil &P, int64_t r0, int64_t r1, int64_t qlo, int64_t qhi,
            const cx<double> *z_dev, int nnodes, const T *X, int64_t ldx, int64_t strideX, T *Y, int64_t ldy,
            int64_t strideY, int64_t b, double sign, bool accumulate);

// R_l = V_l - (A - z_l M) X_l  (complex FP64, all rows, all nodes); V may have stride 0.
// P.am_split <- the double-FP32 split of the pencil's values (x = hi + lo, hi = fl32(x))
void split_pencil(cudaStream_t st, DevPencil &P, float4 *out);
// Xs[i] = (hi(re), lo(re), hi(im), lo(im)) of X[i], count elements
void split_c64(cudaStream_t st, const cx<double> *X, float4 *Xs, int64_t count);
// shifted_residual with the products in double-FP32 arithmetic on split operands (P.am_split
// and Xs); the combination with z_l and the difference with V stay FP64
void shifted_residual_df(cudaStream_t st, const DevPencil &P, const cx<double> *z_dev, int nnodes,
                         const cx<double> *V, int64_t strideV, const float4 *Xs, cx<double> *R, int64_t stride,
                         int64_t b);
// YA = A X and YM = M X for a real FP64 block X (n x b, row-major, ld b), all rows, with the
// products in double-FP32 arithmetic (about 2^-46 of sum |a||x|) on P.am_split and a split of X
void spmm_am_df(cudaStream_t st, const DevPencil &P, const double *X, double *YA, double *YM, int64_t b);
void shifted_residual(cudaStream_t st, const DevPencil &P, const cx<double> *z_dev, int nnodes,
                      const cx<double> *V, int64_t strideV, const cx<double> *X, cx<double> *R, int64_t stride,
                      int64_t b);

// a2: bordered shifted blocks.  For node l and subdomain j the D_j x D_j matrix at
// base + boff[l*p + j] (ld = D_j, D_j = d_j + s_j if border else d_j) receives
// [[B_j - z_l M_B^(j), E^_j(z_l)], [E^_j(z_l)^T, 0]]  (only the leading block if !border).
// For real T the shift's imaginary part must be zero.
template <typename T>
void assemble_blocks(cudaStream_t st, const DevPencil &P, const DevDD &dd, const int64_t *dev_D_off,
                     int64_t total_rows, const int64_t *dev_boff, const cx<double> *z_dev, int nnodes, T *base,
                     bool border);
// S_l = C - z_l M_C (dense s x s at S + l*s*s).
template <typename T>
void assemble_interface(cudaStream_t st, const DevPencil &P, const DevDD &dd, const cx<double> *z_dev,
                        int nnodes, T *S);
// For subdomain j: S_l[sidx_j[a]][sidx_j[b]] += T_l[a][b], T_l = trailing s_j x s_j block of the
// bordered factor (base + boff[l*p+j] + d_j*(D_j+1), ld D_j).  Called for j = 0..p-1 in order, so
// the sums are reproducible.
template <typename T>
void scatter_schur(cudaStream_t st, const DevDD &dd, int j, int dj, int sj, int64_t sidx_start,
                   const int64_t *dev_boff, const T *base, int nnodes, T *S);

// Two-level interface factorisation (storage per node: S2 (s2 x s2) at 0, then the bordered
// block of each group; tsz elements per node, node l at L + l*tsz).
// L_l[edst[e]] = a - z_l m for the interface CSR entries e0 + e, e < ne, with edst[e] >= 0.
template <typename T>
void assemble_iface_levels(cudaStream_t st, const DevPencil &P, int64_t e0, int64_t ne, const int64_t *edst,
                           const cx<double> *z_dev, int nnodes, T *L, int64_t tsz);
// Adds the trailing s_j x s_j block of subdomain j's bordered factor: entry (t, u) to
// S2[r_j[t]][r_j[u]] if both are >= 0, else to the group block at gbase (ld Dg), (q_j[t], q_j[u]).
// Called for j = 0..p-1 in order (reproducible sums).
template <typename T>
void scatter_schur_levels(cudaStream_t st, int p, int j, int dj, int sj, const int32_t *q_j, const int32_t *r_j,
                          int64_t s2, int64_t gbase, int64_t Dg, const int64_t *dev_boff, const T *base, int nnodes,
                          T *L, int64_t tsz);
// S2[i2g[t]][i2g[u]] += trailing n2 x n2 block of the group block at gbase (n1 + n2 square).
template <typename T>
void scatter_trail_levels(cudaStream_t st, const int32_t *i2g, int n1, int n2, int64_t gbase, int64_t s2, int nnodes,
                          T *L, int64_t tsz);

template <typename TO, typename TI>
void convert(cudaStream_t st, const TI *x, TO *y, int64_t n);
// copy a real block into complex (imag 0), possibly replicated for several nodes
template <typename T>
void real_to_complex(cudaStream_t st, const double *x, T *y, int64_t n, int nrep, int64_t stride);
// W = scale * sum_l Re(w_l * Y_l)   (Y_l complex, count elements each, FP64 accumulation)
template <typename T>
void weighted_real_sum(cudaStream_t st, const T *Y, int64_t strideY, const cx<double> *w_dev, int nnodes,
                       double scale, double *W, int64_t count);
void axpy_f64(cudaStream_t st, double a, const double *x, double *y, int64_t n);
void axpy_c64(cudaStream_t st, const cx<double> *x, cx<double> *y, int64_t n);   // y += x
void scale_cols_f64(cudaStream_t st, double *X, int64_t n, int64_t b, int64_t ld, const double *s);
void counter_uniform_dev(cudaStream_t st, uint64_t seed, uint64_t stream, double *x, int64_t n);
// out[c] = sum_i X[i][c] * Y[i][c]   (n x b, ld), FP64, deterministic
void col_dots(cudaStream_t st, const double *X, int64_t ldx, const double *Y, int64_t ldy, int64_t n, int64_t b,
              double *out);
// out[l*b + c] = sum_i |R_l[i][c]|^2 (complex), deterministic
void col_norms2_c64(cudaStream_t st, const cx<double> *R, int64_t n, int64_t b, int nnodes, int64_t stride,
                    double *out);
// gather/scatter of row blocks between a tall block and a strided sub-block
void copy_rows_f64(cudaStream_t st, const double *src, int64_t lds, double *dst, int64_t ldd, int64_t nrows,
                   int64_t ncols);
// X[i][c] -> X[perm[i]][c] style row permutation: dst[i] = src[idx[i]]
void gather_rows_f64(cudaStream_t st, const double *src, int64_t lds, const int64_t *idx, double *dst,
                     int64_t ldd, int64_t nrows, int64_t ncols);
// dst[i][c] = src[ridx[i]][cidx[c]]  (nrows x ncols)
void gather_rows_cols_f64(cudaStream_t st, const double *src, int64_t lds, const int64_t *ridx, const int64_t *cidx,
                          double *dst, int64_t ldd, int64_t nrows, int64_t ncols);

// Y_l (s_j x m) = rows sidx_j of G_l ; G_l rows sidx_j -= R_l (ordered, call for j = 0..p-1)
template <typename T>
void gather_iface(cudaStream_t st, const int32_t *sidx_j, int sj, int64_t m, const T *G, int64_t strideG, T *Y,
                  int64_t strideY, int nnodes);
template <typename T>
void scatter_sub_iface(cudaStream_t st, const int32_t *sidx_j, int sj, int64_t m, const T *Rj, int64_t strideR, T *G,
                       int64_t strideG, int nnodes);

}  // namespace rfdd
