// Dense symmetric eigensolver (FP64) for the Rayleigh-Ritz steps: Householder
// tridiagonalisation, implicit-shift QL on the tridiagonal with rotation accumulation, and
// back-transformation of selected eigenvectors.  Batched over matrices of uneven order.
#pragma once
#include "common.cuh"

namespace rfdd {

struct SymItem {
  double *H;      // n x n symmetric, row-major (ld); overwritten by Householder vectors
  int n, ld;
  double *d;      // n: diagonal -> eigenvalues (ascending after sym_eig_values)
  double *e;      // n: sub-diagonal
  double *tau;    // n
  double *work;   // n
  double *Zt;     // n x n: row j = eigenvector j of the tridiagonal matrix
  int *perm;      // n: sorted position -> row of Zt
};

// Tridiagonalise every H, then diagonalise the tridiagonal matrices; on return d holds the
// eigenvalues in ascending order and perm maps sorted index -> row of Zt.  status gets
// DS_NONFINITE if QL did not converge within 60 iterations for some eigenvalue.
void sym_eig_values(cudaStream_t st, const std::vector<SymItem> &items, int *status);

// out_b (nsel_b x n_b, row-major, ld_out) row r = eigenvector for sorted index sel_b[r] of H_b.
struct BackItem {
  const SymItem *s;
  const int *sel;  // device, nsel entries (sorted-order indices)
  int nsel;
  double *out;
  int ld_out;
};
void sym_eig_vectors(cudaStream_t st, const std::vector<BackItem> &items);

}  // namespace rfdd
