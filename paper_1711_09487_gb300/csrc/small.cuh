// Small dense FP64 helpers (one CTA per matrix): Cholesky with drop tolerance and the inverse
// of the triangular factor, used for block orthonormalisation (Cholesky-QR).
#pragma once
#include "common.cuh"

namespace rfdd {

struct CholItem {
  double *G;     // b x b Gram matrix (row-major, ld = b); overwritten by R (upper, G = R^T R)
  double *Rinv;  // b x b output: R^{-1} (columns of dropped pivots are zero)
  int *dead;     // b flags: 1 where the pivot fell below tol * max diagonal
  int b;
};
void chol_inv_batched(cudaStream_t st, const std::vector<CholItem> &items, double tol);

// C = D A D elementwise for a k x k matrix with diagonal scaling vector d
void scale_sym(cudaStream_t st, double *A, int64_t k, const double *d);
// out[q][c] = U[q][c] * d[c] * f[q]   (r x k)
void scale_rows_cols(cudaStream_t st, const double *U, int64_t r, int64_t k, const double *d, const double *f,
                     double *out);
// d[c] = G[c][c] > 0 ? 1/sqrt(G[c][c]) : 0
void inv_sqrt_diag(cudaStream_t st, const double *G, int64_t k, double *d);
// f[q] = 1/sqrt(lam[q0 + q])
void inv_sqrt_vec(cudaStream_t st, const double *lam, int64_t r, double *f);
// residual norms: res[c] = ||AX_c - theta_c MX_c|| / (|theta_c| ||MX_c||)
void ritz_residuals(cudaStream_t st, const double *AX, const double *MX, const double *theta, int64_t n, int64_t b,
                    double *res);
// out[c] = sum_i X[i][c] Y[i][c] for n x b row-major blocks
void col_dots(cudaStream_t st, const double *X, const double *Y, int64_t n, int64_t b, double *out);
// y[i] -= x[i] for generic element type
template <typename T>
void sub_inplace(cudaStream_t st, const T *x, T *y, int64_t n);

}  // namespace rfdd

namespace rfdd {
// Pivoted Cholesky of the k x k symmetric G (full storage, in place); returns the rank (pivots
// > tol), perm (device, k) the column order; R is the leading rank x rank upper triangle.
int pivoted_cholesky(cudaStream_t st, double *G, int k, int *perm, double tol, int *rank_dev);
void gather_sym(cudaStream_t st, const double *K, int k, const int *perm, int r, double *out);
void unit_lower_from_upper(cudaStream_t st, const double *R, int ldr, int r, double *Lt);
void scale_rows_by_rdiag(cudaStream_t st, const double *in, int r, bool trans, const double *R, int ldr, double *out);
void symmetrize(cudaStream_t st, const double *A, int r, double *out);
void transpose(cudaStream_t st, const double *in, int a, int b, double *out);
void scatter_rows_perm(cudaStream_t st, const double *Cr, int r, int ns, const int *perm, const double *d,
                       double *Cfull);
// G[c][r] = G[r][c] for r in [r0, r1), c in [c0, c1)  (k x k row-major)
void mirror_block(cudaStream_t st, double *G, int64_t k, int64_t r0, int64_t r1, int64_t c0, int64_t c1);
}  // namespace rfdd
