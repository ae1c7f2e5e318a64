// Dense symmetric eigensolver (FP64) for the Rayleigh-Ritz steps: Householder
// tridiagonalisation, eigenvalues of the tridiagonal matrix by bisection on Sturm counts (one
// thread per eigenvalue), eigenvectors of selected eigenvalues by inverse iteration (one CTA per
// cluster of close eigenvalues, Gram-Schmidt within the cluster), back-transformation.
#pragma once
#include "common.cuh"

namespace rfdd {

struct SymItem {
  double *H;      // n x n symmetric, row-major (ld); overwritten by Householder vectors
  int n, ld;
  double *d;      // n: diagonal of the tridiagonal matrix
  double *e;      // n: its off-diagonal (e[i] couples i and i+1; e[n-1] = 0)
  double *tau;    // n: Householder scalars
  double *work;   // n: scratch
  double *lam;    // n: eigenvalues, ascending (output of sym_eig_values)
  double *Zt;     // >= nsel x n scratch: eigenvectors of the tridiagonal matrix (rows)
};

// Tridiagonalise every H and compute all its eigenvalues into lam (ascending).
void sym_eig_values(cudaStream_t st, const std::vector<SymItem> &items, int *status);

// Number of eigenvalues below shift of every H (Householder tridiagonalisation, which keeps the
// inertia, then a Sturm count of the tridiagonal matrix); H is overwritten.  counts_dev: device
// array, one entry per item.
void sym_negative_counts(cudaStream_t st, const std::vector<SymItem> &items, double shift, long long *counts_dev);

// Eigenvectors for the ascending sorted indices sel of each item: out row r (ld_out) = unit
// eigenvector of H for lam[sel[r]].  Eigenvalues closer than ctol * ||T|| to a neighbouring
// selected one form a cluster whose vectors are orthogonalised against each other.
struct BackItem {
  const SymItem *s;
  std::vector<int> sel;   // host, ascending
  double *out;
  int ld_out;
};
void sym_eig_vectors(cudaStream_t st, const std::vector<BackItem> &items, double ctol);

}  // namespace rfdd
