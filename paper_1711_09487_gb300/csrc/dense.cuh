// Batched dense kernels (host-side launchers): GEMM, blocked LU with tournament pivoting on
// bordered matrices, LU solves.  Every routine works on a batch of independent matrices of
// uneven sizes and is instantiated for float, double, cx<float>, cx<double>.
#pragma once
#include "common.cuh"

namespace rfdd {

// SM count of the current device (cached per device)
int sm_count();

constexpr int MAXB = 64;      // matrices per launch (descriptors travel as kernel parameters)
constexpr int LU_NB = 32;     // tournament panel width (pivot columns per inner step)

// C = beta*C + alpha*op(A) op(B); row-major, op(X) = X or X^T (stored transposed).
template <typename T>
struct GemmItem {
  const T *A;
  const T *B;
  T *C;
  int m, n, k;
  int lda, ldb, ldc;
};

template <typename T>
void gemm_batched(cudaStream_t st, const std::vector<GemmItem<T>> &items, bool ta, bool tb,
                  double alpha, double beta);
// FP64 operands and result, double-FP32 arithmetic (relative error near 2^-46 of sum |a b|):
// for products on eigenvector bases.  sym[i] != 0 marks a square product known to be symmetric
// (A^T P A with P symmetric): only its upper tiles are formed and mirrored.
void gemm_f64x2_batched(cudaStream_t st, const std::vector<GemmItem<double>> &items, bool ta, bool tb, double alpha,
                        double beta, const std::vector<char> &sym = {});
// the CUDA-core kernel only (no tensor-core dispatch); sym as for gemm_f64x2_batched (real T)
template <typename T>
void gemm_simt_batched(cudaStream_t st, const std::vector<GemmItem<T>> &items, bool ta, bool tb,
                       double alpha, double beta, const std::vector<char> &sym = {});

// One bordered matrix for LU: D x D (row-major, leading dimension ld), of which the first dp
// rows/columns are eliminated with pivoting restricted to rows < dp.  After the factorisation
// the trailing (D-dp) x (D-dp) block holds C~ - E^T B^{-1} E (the Schur complement of the
// leading block).  piv: int32[dp], LAPACK-style sequence of row interchanges (row t <-> piv[t]).
template <typename T>
struct LuItem {
  T *A;
  int *piv;
  int dp, D, ld;
};

struct LuWork {
  int *cand = nullptr;   // candidate buffers (2 x MAXB x stride ints)
  void *top = nullptr;   // MAXB x NB x NB scratch
  size_t cand_ints = 0, top_bytes = 0;
};

// nbo: outer block (trailing-update depth), a multiple of LU_NB.
template <typename T>
void lu_batched(cudaStream_t st, const std::vector<LuItem<T>> &items, int nbo, int *dev_status);

// Solve with LU factors: X <- U^{-1} L^{-1} P X for the leading dp x dp block of each item.
// Optional: inverses of the nbi x nbi diagonal blocks of L (unit lower) and U (upper), block b
// at Linv + b * nbi * nbi (leading dimension nbi; the last block uses its leading w x w part).
// When every item of a triangular solve carries them and nbi equals the solve's block size, the
// diagonal blocks are applied as matrix products (tensor cores for complex FP32) instead of by
// substitution.
template <typename T>
struct SolveItem {
  const T *LU;
  const int *piv;
  int n, ld;       // order of the factored block and its leading dimension
  T *X;
  int ldx, ncols;
  const T *Linv = nullptr, *Uinv = nullptr;
  int nbi = 0;
  // Optional tensor-core tile copies (complex FP32 only, see tc_pack_a_batched): of the n x n
  // factor (LUp, packed as an n x n operand) and of the inverse blocks (one nbi x nbi operand per
  // block, block b at Linvp/Uinvp + b * tc_packed_a_floats(nbi, nbi)).  Used as the A operands of
  // the block-inverse solves instead of packing the same factor again on every solve.
  const float *LUp_hi = nullptr, *LUp_lo = nullptr;
  const float *Linvp_hi = nullptr, *Linvp_lo = nullptr, *Uinvp_hi = nullptr, *Uinvp_lo = nullptr;
};
// Elements of the inverse-block storage of one n x n factor.
inline int64_t block_inverse_elems(int64_t n, int nbi) { return (int64_t)((n + nbi - 1) / nbi) * nbi * nbi; }
// Linv[i] / Uinv[i] <- inverses of the diagonal nbi-blocks of items[i]'s L and U (either may be
// null to skip it); computed by substitution against identity blocks.
template <typename T>
void lu_block_inverses(cudaStream_t st, const std::vector<SolveItem<T>> &items, int nbi, const std::vector<T *> &Linv,
                       const std::vector<T *> &Uinv);
template <typename T>
void lu_solve_batched(cudaStream_t st, const std::vector<SolveItem<T>> &items, int nbo);

// Building blocks exposed for the tests of individual steps.
template <typename T>
void apply_pivots(cudaStream_t st, const std::vector<SolveItem<T>> &items);
template <typename T>
void trsm_lower_unit(cudaStream_t st, const std::vector<SolveItem<T>> &items, int nbo);
template <typename T>
void trsm_upper(cudaStream_t st, const std::vector<SolveItem<T>> &items, int nbo);

}  // namespace rfdd
