/*
 * rfdd.h -- C ABI of the GB300-native RF-DDES interface rational filter.
 *
 * Method: Kalantzis, Xi, Saad, "Beyond AMLS: Domain decomposition with rational filtering"
 * (arXiv:1711.09487).  The library finds every eigenpair (lambda, x) of a real symmetric pencil
 * A x = lambda M x (M SPD) with lambda in [alpha, beta] (Section 1).  The number of eigenpairs is
 * found, not given.
 *
 * Conventions shared by every entry point:
 *  - Return value: RFDD_OK (0) or one of the RFDD_E* codes below.  On error nothing the caller
 *    owns is modified, except output buffers of the failing call may hold partial data; the
 *    message of the last error on the calling thread is available from rfdd_last_error().
 *  - Sparse inputs are full (both triangles) CSR with int64 row pointers, int32 column indices
 *    (in any order within a row, no duplicates) and float64 values, in host memory or, with
 *    rfdd_csr.location = 1, in device memory.  They are copied at setup; the caller keeps
 *    ownership.  (A device-resident CSR is copied to the host for the validation and the
 *    interior-first ordering, which run on the host, then uploaded in that order.)
 *  - Dense host arrays are row-major.  Complex values are interleaved (re, im) float64 pairs.
 *  - "Interior-first ordering" (Eq. dd1): the interior unknowns of subdomain 0, 1, ..., p-1
 *    (each in increasing original index), then the interface unknowns (label -1) in increasing
 *    original index.  Subdomain j occupies rows [off_j, off_j + d_j); the interface occupies the
 *    last s rows.  rfdd_layout() returns off_j, d_j, s and the permutation.
 *  - Every call runs on the handle's CUDA stream and returns after its results are complete,
 *    except rfdd_solve_async().  A solve also runs the real interior factorisation and the V_j
 *    subspace iteration (a8) on a second stream that the handle creates and owns, launched from
 *    a host thread of its own and joined before the call returns or fails.
 *  - A handle is not thread-safe; distinct handles may be used from different threads.  Each
 *    handle's kernels record device-side failures (a zero pivot, a tensor-core wait that ran out
 *    of iterations) in a status word of that handle, so a failure is reported by the call that
 *    met it and by no other handle.
 */
#ifndef RFDD_H
#define RFDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define RFDD_OK 0
#define RFDD_EINVAL 1            /* bad argument: size mismatch, alpha >= beta, n_nodes < 1, NULL */
#define RFDD_ENOTSYM 2           /* A or M not symmetric (pattern or values) */
#define RFDD_EPARTITION 3        /* edge between two subdomains, empty subdomain, no interface */
#define RFDD_ENOTSPD_M 4         /* M not positive definite (a non-positive diagonal entry) */
#define RFDD_ESINGULAR 5         /* zero or non-finite pivot in a factorisation */
#define RFDD_ENOMEM 6            /* device allocation failed */
#define RFDD_EADMIT 7            /* the solve's device memory need exceeds opt.mem_budget */
#define RFDD_NOT_CONVERGED 8     /* results returned, but some residual > res_tol */
#define RFDD_ECUDA 9             /* CUDA runtime error */
#define RFDD_ESTATE 10           /* call out of order (e.g. filter before factor) */

/* ---- option values ---------------------------------------------------------------------- */
#define RFDD_FP64 0              /* plain path: all factorisations and solves in FP64 */
#define RFDD_MIXED 1             /* complex-FP32 factorisations, FP64 iterative refinement */
#define RFDD_MIDPOINT 0          /* midpoint rule of order 2Nc (Section 6, the paper's choice) */
#define RFDD_GAUSS_LEGENDRE 1    /* Gauss-Legendre on the upper half circle (Section 2.1) */

typedef struct {
  int64_t n;
  const int64_t *rowptr; /* n+1 */
  const int32_t *col;    /* rowptr[n] */
  const double *val;     /* rowptr[n] */
  int32_t location;      /* where rowptr, col and val live: 0 host memory (the default of a
                            zero-initialised struct), 1 device memory of the current device */
} rfdd_csr;

typedef struct {
  int precision;        /* RFDD_FP64 | RFDD_MIXED (default RFDD_MIXED) */
  int quad_rule;        /* RFDD_MIDPOINT | RFDD_GAUSS_LEGENDRE (default midpoint) */
  double sigma;         /* real shift of the interior step (Eq. prol2); NaN -> (alpha+beta)/2 */
  int nev_b;            /* eigenvectors per subdomain in V_j (Alg. 3 step 3); default 100,
                           capped at d_j */
  int psi;              /* resolvent-expansion depth (Eq. yet1); default 3 */
  double lanczos_tol;   /* Alg. 2 trace-stagnation tolerance; default 1e-6 */
  int block;            /* block size b of the block variant of Alg. 2; default 32 */
  double res_tol;       /* residual target ||Ax-lMx||/(|l| ||Mx||); default 1e-10 */
  int max_passes;       /* completion passes (filtered subspace iteration); default 8 */
  int ir_max;           /* FP64 iterative-refinement steps per shifted solve; default 10 */
  uint64_t seed;        /* counter-based RNG seed for start blocks; default 1 */
  size_t mem_budget;    /* device bytes one solve may hold; 0 = no limit */
  void *stream;         /* cudaStream_t to run on (must stay valid until rfdd_destroy: the
                           handle's device buffers are stream-ordered allocations on it);
                           NULL = a stream owned by the handle */
  double guard_frac;    /* completion block m = n_in + max(ceil(guard_frac n_in), min_guard) */
  int min_guard;        /* (defaults 0.3 and 8) */
  int keep_schur;       /* nonzero: keep an unfactored copy of every S(zeta_l) (for checks) */
  int subspace_iters;   /* block shift-invert iterations that build V_j (default 4) */
  int m_align;          /* completion block m rounded up to a multiple of this (default 128, the
                           complex column width of one tensor-core tile: the extra guard vectors
                           ride in tile columns that would otherwise be padding); <= 1: none */
  int pack_factors;     /* mixed solve: form of the complex factors kept for the solves.  1: the
                           tensor-core tile copies only (TF32 hi/lo, 16 bytes per complex entry,
                           packed once after the factorisation; the complex64 factors are freed
                           then, so the peak holds both); 0: the complex64 factors only (8 bytes
                           per entry; every solve product packs its factor block on the fly);
                           -1 (default): 1 unless mem_budget is set and the peak of 1 exceeds it */
} rfdd_options;

typedef struct rfdd_handle rfdd_handle;
typedef struct rfdd_result rfdd_result;

/* Diagnostics of one solve.  Times are CUDA-event milliseconds on the handle's stream. */
typedef struct {
  int64_t nev;          /* eigenpairs returned (inside [alpha, beta]) */
  int64_t mu;           /* Alg. 2 basis size (columns of Q) */
  int64_t k;            /* columns of Z (Eq. z) kept after M-orthonormalisation */
  int64_t m;            /* completion block size at the last pass (it grows when the Ritz values
                           inside [alpha, beta] fill it; see rfdd_solve) */
  int32_t passes;       /* completion passes run */
  int32_t ir_steps_max; /* largest number of refinement steps any shifted solve needed */
  double max_resid;     /* largest residual among the returned pairs */
  double pre_max_resid; /* largest residual of the RF-DDES Ritz pairs before completion */
  int64_t pre_nev;      /* RF-DDES Ritz values inside [alpha, beta] before completion */
  double t_factor_ms;   /* a2-a5: shifted blocks, LU(B), Schur update, S assembly + LU(S) */
  double t_lanczos_ms;  /* a6-a7 */
  double t_interior_ms; /* a8 */
  double t_rr_ms;       /* a9 */
  double t_complete_ms; /* a10 */
  double t_total_ms;
  int32_t status;       /* RFDD_OK or RFDD_NOT_CONVERGED */
  int32_t packed;       /* 1 if the solves used tile copies of the factors (opt.pack_factors) */
  double sigma;         /* real shift the interior step used (Eq. prol2): opt.sigma or (alpha+beta)/2,
                           moved, at most three times, while it lies within tau max(1, |sigma|) of
                           an eigenvalue of some (B_j, M_B^(j)): FP64 tau = 1e-8, move
                           1e-6 (beta - alpha); mixed (FP32 factors) tau = 1e-5, move
                           max(1e-3 (beta - alpha), 2 tau max(1, |sigma|)) */
  double t_factor_enqueue_ms; /* host wall time to issue the a2-a5 launches (they run
                                 asynchronously: the host limits the phase only if this
                                 approaches t_factor_ms) */
  int64_t factor_launches;    /* kernels launched for a2-a5 */
  int32_t fp64_basis;         /* 1 if the completion passes switched their basis products (Gram
                                 matrices, Ritz vectors) and refinement residuals from
                                 double-FP32 to FP64 because the residuals stopped falling
                                 (mixed precision only) */
  int32_t reserved0;
} rfdd_info;

/* Fill *opt with the defaults listed above. */
void rfdd_default_options(rfdd_options *opt);

/* Message of the last error on this thread ("" if none).  Valid until the next call. */
const char *rfdd_last_error(void);

/* Static description of a status code. */
const char *rfdd_status_string(int code);

/* ---- a0: quadrature (Section 2.1, Eq. contour/contour2/contour3; Section 6) -------------
 * Poles zeta_l (Im > 0) and weights omega_l, l = 0..n_nodes-1, of the rational filter
 * rho(x) = 2 Re sum_l omega_l/(x - zeta_l) on the circle through alpha and beta.
 * z_out, w_out: host, 2*n_nodes doubles each (interleaved complex).  Host only. */
int rfdd_quadrature(double alpha, double beta, int32_t n_nodes, int32_t rule, double *z_out,
                    double *w_out);

/* ---- a1: setup (Alg. 3 step 1; Section 2.3, Eq. dd1) -----------------------------------
 * Validates (A, M, part), computes the interior-first ordering, splits the pencil into the
 * blocks B_j, M_B^(j), E_j, M_E^(j), C, M_C and uploads them.  A and M may each be host- or
 * device-resident (rfdd_csr.location; RFDD_EINVAL for another value, RFDD_ECUDA if a device
 * copy fails).  part: host int32[n], label -1
 * for interface unknowns and 0..p-1 for subdomain interiors; the labels must form a vertex
 * separator (no A or M entry couples two different subdomains) and every subdomain and the
 * interface must be non-empty.  opt may be NULL (defaults).  On success *out owns device
 * memory until rfdd_destroy(). */
int rfdd_setup(const rfdd_csr *A, const rfdd_csr *M, const int32_t *part, int32_t p,
               const rfdd_options *opt, rfdd_handle **out);

/* Layout of the interior-first ordering: off (p+1 int64: subdomain j is rows off[j]..off[j+1]-1,
 * the interface rows off[p]..n-1) and perm (n int64: new index -> original index).  Either
 * pointer may be NULL.  *p_out and *s_out receive p and s. */
int rfdd_layout(const rfdd_handle *h, int64_t *off, int64_t *perm, int32_t *p_out,
                int64_t *s_out);

/* Two-level interface factorisation (a5 and the S solves of a6 and a10): the block inverse of
 * Eq. (inv_dd2) applied a second time, to S(zeta_l), with groups of subdomains in the role of the
 * subdomains.  This is the recursive use of the decomposition that Section 7 proposes; Section
 * 6.3 names the S(zeta) solves as what limits RF-DDES as p grows.
 *   group: p labels in 0..n_groups-1 (host memory, read during the call).  n_groups = 0 (group
 *   may be NULL) restores the one dense LU of S(zeta_l) per node.
 * Reading (the paper gives no recursion of the interface): an interface node is level 1 of group
 * g when every subdomain it touches (has a coupling to) is in g and no interface node it is
 * coupled to in C or M_C is such a candidate of another group; all other interface nodes are
 * level 2.  S restricted to the level-1 nodes is then block diagonal over the groups.  Each node's
 * factors are, per group, the LU of the bordered block [[S(I1_g,I1_g), S(I1_g,I2_g)],
 * [S(I2_g,I1_g), 0]] (I2_g: the level-2 nodes S couples to I1_g) and the dense LU of
 * S2' = S(I2,I2) - sum_g S(I2_g,I1_g) S(I1_g,I1_g)^{-1} S(I1_g,I2_g).  The results of a solve are
 * those of the dense factorisation up to rounding; the memory and the flops of a5 fall from s^2
 * and s^3 per node to about s2^2 + sum_g (|I1_g| + |I2_g|)^2 and their cubes.
 * Drops the handle's factors (the next rfdd_solve or rfdd_factor refactors).  RFDD_EINVAL: a
 * label out of range, n_groups < 0, or keep_schur set (the dense S is never formed). */
int rfdd_set_interface_groups(rfdd_handle *h, int32_t n_groups, const int32_t *group);

/* The split made by rfdd_set_interface_groups: cls (s int32, may be NULL) receives, per
 * interface unknown in interior-first order, its group when it is level 1 and -1 when it is
 * level 2 (all -1 with the dense factorisation); *s2 (may be NULL) the level-2 count (s with the
 * dense factorisation). */
int rfdd_interface_levels(const rfdd_handle *h, int32_t *cls, int64_t *s2);

/* Device workspaces of a handle come from the device's default stream-ordered memory pool, on
 * the handle's stream.  Freed workspaces stay in that pool for reuse by later solves and handles
 * of the process (its release threshold is raised at the first rfdd_setup on a device); a caller
 * that needs the memory back can trim the pool (cudaMemPoolTrimTo) after rfdd_destroy. */
void rfdd_destroy(rfdd_handle *h);

/* Frees the device memory of the last solve on the handle -- the factors of every B_j(zeta_l) and
 * S(zeta_l), their inverted diagonal blocks and packed copies, the interior factors, the Lanczos
 * basis, Z and the completion block -- and keeps the set-up (pencil, partition, maps), so that a
 * resident pencil holds only its set-up between solves.  Step-level calls that need factors then
 * return RFDD_ESTATE until the next rfdd_factor or rfdd_solve.  Waits for the handle's streams. */
int rfdd_release(rfdd_handle *h);

/* ---- full solve: Alg. 3 (RF-DDES) + completion ------------------------------------------
 * Runs a0-a10 for [alpha, beta] with n_nodes quadrature poles.  The completion block starts at
 * m = n_in + max(ceil(guard_frac n_in), min_guard) columns (n_in: RF-DDES Ritz values inside,
 * rounded up to m_align); when the Ritz values inside leave fewer than that many guard columns, the
 * block doubles with fresh counter-based vectors (at most four times, two more passes each), so
 * that an interval holding more eigenvalues than RF-DDES found is still completed.  Factors of the
 * previous solve are replaced.  *out receives a result (also on RFDD_NOT_CONVERGED, whose pairs carry their
 * residuals); free it with rfdd_result_free(). */
int rfdd_solve(rfdd_handle *h, double alpha, double beta, int32_t n_nodes, rfdd_result **out);

/* Eigenpairs of a result.  evals: ascending, nev doubles.  evecs: n x nev row-major, original
 * ordering, M-orthonormal.  resid: nev residuals ||A x - l M x||_2/(|l| ||M x||_2).  device = 0
 * gives host pointers, 1 gives device pointers.  Pointers stay valid until rfdd_result_free().
 * Any output pointer may be NULL. */
int rfdd_result_get(const rfdd_result *r, int64_t *nev, const double **evals,
                    const double **evecs, const double **resid, int32_t device);
int rfdd_result_info(const rfdd_result *r, rfdd_info *info);
/* RF-DDES Ritz values inside [alpha, beta] before completion (Alg. 3 step 7), ascending; host.
 * *count receives their number; vals may be NULL to query it. */
int rfdd_result_pre_evals(const rfdd_result *r, int64_t *count, double *vals);
void rfdd_result_free(rfdd_result *r);

/* ---- step-level entry points (each runs one row of the hot path on the handle) ------------ */

/* a2-a5 (Section 3.1, Eq. inv_dd2; paper: PARDISO/MUMPS factorisations): for every node
 * zeta_l (host, 2*n_nodes doubles, interleaved) assemble B_j(zeta_l) = B_j - zeta_l M_B^(j)
 * densely, LU-factor all of them (partial pivoting by |re|+|im| within tournament-selected
 * candidate rows), form X = B_j^{-1} E_j(zeta_l), the Schur complement
 * S(zeta_l) = C - zeta_l M_C - sum_j E_j(zeta_l)^T X (plain transpose), and LU-factor each S.
 * w (same layout) holds the quadrature weights used by later filter calls. */
int rfdd_factor(rfdd_handle *h, int32_t n_nodes, const double *z, const double *w);

/* Copy the assembled, unfactored S(zeta_l) (s x s complex, row-major, interleaved) to host
 * memory S_out (2*s*s doubles).  Needs opt.keep_schur != 0 at setup. */
int rfdd_schur_copy(rfdd_handle *h, int32_t node, double *S_out);

/* Solve with the factors of node `node`: which = 0 -> B_j(zeta) X = R for subdomain j (R is
 * d_j x nrhs); which = 1 -> S(zeta) X = R (R is s x nrhs); which = 2 -> (A - zeta M) X = R on
 * the interior-first ordering (R is n x nrhs) through the block inverse of Eq. (inv_dd2) with
 * FP64 iterative refinement.  R, X: host, complex interleaved row-major. */
int rfdd_shifted_solve(rfdd_handle *h, int32_t node, int32_t which, int32_t j, int64_t nrhs,
                       const double *R, double *X);

/* a6 (Alg. 2 line 2): W = Re sum_l omega_l S(zeta_l)^{-1} X for a real s x b block X.
 * X, W: host, s x b float64 row-major. */
int rfdd_filter_apply(rfdd_handle *h, int64_t b, const double *X, double *W);

/* a7 (Alg. 2, block variant, trace-stagnation stop every ceil(10/b) block steps): runs the
 * interface Krylov process on F = Re sum omega_l S_l^{-1}.  Q_out: host s x cap float64
 * row-major (may be NULL); *mu receives the basis size; traces (may be NULL, cap entries)
 * receive tr(T) after each block step; *nsteps the number of block steps. */
int rfdd_lanczos(rfdd_handle *h, int64_t cap, double *Q_out, int64_t *mu, double *traces,
                 int32_t *nsteps);

/* a8 (Section 4; Alg. 3 steps 2-4 and 6; Eq. trabala, trabala2, z): builds the projection
 * basis Z = [blockdiag(V_j) | -Sigma^(psi) | Gamma^(psi)] from the last Lanczos basis Q with
 * the real shift sigma (NaN -> (alpha+beta)/2 of the last solve or 0).  Z_out: host n x k
 * float64 row-major on the interior-first ordering (may be NULL); *k receives its column
 * count; kappa_out (may be NULL) receives sum_j nev_B^(j). */
int rfdd_interior(rfdd_handle *h, double sigma, int64_t cap, double *Z_out, int64_t *k,
                  int64_t *kappa_out);

/* a9 (Alg. 3 step 7): Rayleigh-Ritz of (A, M) on range(Z) of the last rfdd_interior call.
 * theta_out: host, all Ritz values ascending (cap entries); *k receives their number. */
int rfdd_rayleigh_ritz(rfdd_handle *h, int64_t cap, double *theta_out, int64_t *k);

/* Eigenvalue count (the interval problem of Section 1 asks for every eigenvalue in [alpha, beta];
 * this checks that none is missed): *count = number of eigenvalues of (A, M) strictly below sigma,
 * by Sylvester's law of inertia.  With the interior-first block form of Eq. (eq1), the inertia of
 * A - sigma M is that of the blocks B_sigma^(j) plus that of the Schur complement S(sigma)
 * (Haynsworth additivity).  Everything is FP64: the bordered real blocks are factored as in
 * rfdd_factor (their trailing blocks give S(sigma)), and each B_sigma^(j) and S(sigma) is reduced
 * to tridiagonal form by Householder similarity and counted by Sturm sequence.  The number of
 * eigenvalues in [alpha, beta] is count(beta) - count(alpha) when neither end is an eigenvalue.
 * Needs only rfdd_setup; uses the handle's stream; O(d_j^3) work per subdomain.
 * RFDD_ESINGULAR when sigma is an eigenvalue of a block B^(j) (choose another sigma). */
int rfdd_inertia(rfdd_handle *h, double sigma, int64_t *count);

/* Interior polish of approximate eigenpairs (Section 3, Eqs. (schur_eigvec2) and
 * (compute_u_parallel): once the interface part y of an eigenvector is known, its interior part
 * follows from one real solve per subdomain).  For each pair i it keeps the interface rows y of
 * column i of X and replaces the interior rows of every subdomain j by the solution u_j of
 *   (B_j - lambda_i M_B^(j)) u_j = -(E_j - lambda_i M_E^(j)) y_j,
 * each block factored by FP64 dense LU with partial pivoting, all (i, j) batched.  Then it
 * M-normalises the column, replaces lambda_i by its Rayleigh quotient x^T A x / x^T M x, and
 * writes resid_i = ||A x - lambda_i M x|| / (|lambda_i| ||M x||).  The result is exact when y is
 * the interface part of an exact eigenvector; its accuracy otherwise follows that of y.
 * X: host, n x nev row-major in the original ordering (the layout rfdd_result_get returns),
 * updated in place; lambda: host, nev, updated; resid: host, nev, written.  Needs only
 * rfdd_setup; uses the handle's stream.  Device memory: 6 n x nev FP64 arrays plus the dense
 * blocks of as many pairs at a time as fit in 4 GiB (or in half of opt.mem_budget when set),
 * at least one pair.
 * RFDD_ESINGULAR when some B_j - lambda_i M_B^(j) has a zero pivot (lambda_i an eigenvalue of a
 * subdomain pencil) or a column has a zero vector after the polish; RFDD_EINVAL for nev < 0,
 * null arrays or a non-finite lambda_i. */
int rfdd_polish(rfdd_handle *h, int64_t nev, double *lambda, double *X, double *resid);

/* a9 building block (Alg. 3 step 7 solves its projected problem with a dense symmetric
 * eigensolver): eigen-decomposition of a dense symmetric n x n FP64 matrix H on the GPU by
 * Householder tridiagonalisation, bisection on Sturm counts, inverse iteration (clusters
 * re-orthogonalised) and back-transformation.  H, evals, evecs
 * are host arrays; evals (n) ascending; evecs (n x n row-major) holds eigenvector j in ROW j.
 * Needs no handle (runs on the default stream of the current device). */
int rfdd_sym_eig(int64_t n, const double *H, double *evals, double *evecs);

/* Building block of a3-a5 (trailing updates of the factorisations), a6 and a10 (triangular-solve
 * updates): C = beta*C + alpha*A*B for complex single-precision A (m x k, leading dimension lda),
 * B (k x n, ldb), C (m x n, ldc), host arrays, row-major, interleaved (re, im) floats.
 * engine 1 = the tensor-core GEMM (tcgen05, 3xTF32 split) that every complex-FP32 contraction of
 * the solver runs on, with its automatic choice between a one-CTA kernel (128 x 256 tiles of the
 * realified product) and a two-CTA kernel (cta_group::2, 256 x 256 tiles on a pair of SMs);
 * engines 2 and 3 force the one-CTA and the two-CTA kernel; engine 0 = a CUDA-core kernel kept
 * as another engine for tests (the solver never dispatches to it).  RFDD_EINVAL for other
 * engines. */
int rfdd_cgemm(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B, int64_t ldb,
               float *C, int64_t ldc, double alpha, double beta, int32_t engine);

/* Building block of a7-a10 (products on the eigenvector bases: Lanczos projections and Gram
 * matrices, the interior CholQR, the Rayleigh-Ritz Gram matrices and Ritz vector updates):
 * C = beta*C + alpha*op(A)*op(B) for FP64 host arrays, row-major; op(X) = X^T when the flag is 1
 * (A then stored k x m with leading dimension lda >= m; B stored n x k with ldb >= k).
 * engine 0 = FP64 CUDA-core kernel; 1 = the double-FP32 kernel the solver uses for these
 * products (each operand split into two floats, error-free products and compensated sums:
 * |error| within about 2^-42 of sum_k |a_ik||b_kj|).  sym = 1 declares op(A)*op(B) symmetric
 * (m == n required): only the upper 64 x 64 tiles are formed and mirrored.
 * Deep K with few output tiles is split over CTAs and the partial tiles summed in a fixed order. */
int rfdd_dgemm(int64_t m, int64_t n, int64_t k, int32_t ta, const double *A, int64_t lda, int32_t tb,
               const double *B, int64_t ldb, double *C, int64_t ldc, double alpha, double beta,
               int32_t engine, int32_t sym);

/* Tile-shape autotuner of the tensor-core GEMMs (no counterpart in the paper).  Where both the
 * one-CTA kernel (128 x 256 output tiles) and the two-CTA kernel (256 x 256 tiles per SM pair)
 * can run a launch, the library times both on real launches of the same class -- device,
 * complex or real, the K depth bucket floor(log2(K/32 tiles)) and the launch's tile count against
 * the SM count; never what else runs -- three timings each, with CUDA events on the launch's
 * stream and without blocking, then keeps the faster for every later launch of that class in this
 * process.  Until a class is decided, and whenever tuning is off, a fixed rule chooses (the
 * two-CTA kernel from complex K = 256 on).  Launches inside a stream capture are never timed;
 * they take a decided class's choice, else the rule.
 * rfdd_autotune: mode 0 turns tuning off, 1 on (the default), 2 forgets every class.  Returns 1
 * if tuning was on before the call, 0 if off, -RFDD_EINVAL for another mode.
 * rfdd_autotune_table: writes the table as text, one line per class, "device complex splits
 * kbucket tbucket winner n0 ms_per_gflop0 n1 ms_per_gflop1" (winner -1 while undecided;
 * candidate 0 = one-CTA, 1 = two-CTA), NUL-terminated and truncated to cap bytes; *len = its
 * full length.  Pass cap = 0 to query the length. */
int rfdd_autotune(int32_t mode);
int rfdd_autotune_table(char *buf, int64_t cap, int64_t *len);

/* Allocation-free variant of rfdd_cgemm (no counterpart in the paper).  For callers that cannot
 * allocate device memory -- a process whose device memory is capped or owned by another
 * allocator, a real-time loop that must not enter the allocator, code that must not pay the
 * implicit synchronisation an allocation can cause -- this computes C = beta*C + alpha*A*B on the
 * tensor cores with A, B, C in DEVICE memory (complex single precision, row-major, interleaved,
 * leading dimensions in complex elements) and stages the packed operands in a fixed static
 * device array (6 MiB per device that has loaded the library, held until process exit) instead
 * of a workspace.  Limits: 1 <= m, n <= 1024 and 1 <= k <= 128; larger sizes return RFDD_EINVAL.
 * The first call on a device looks up the device addresses of that array and of its status word
 * (make that first call before any stream capture).  Work runs on `stream` (a cudaStream_t, NULL =
 * the legacy default stream): the call clears the status word, packs, multiplies and reads the
 * status word back on that stream, then waits for that stream alone; it does not synchronise the
 * device.  Every call shares the one array and status word, which keep the last call's contents:
 * calls that overlap on the GPU (from different host threads or streams) race and must be
 * serialised by the caller.  RFDD_ECUDA when the tensor-core kernel's bounded wait ran out.
 * No memory is allocated or freed by this call. */
int rfdd_cgemm_noalloc(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B,
                       int64_t ldb, float *C, int64_t ldc, double alpha, double beta, void *stream);

/* ---- measurement hooks (no counterpart in the paper) -------------------------------------
 * rfdd_kernel_launches: number of kernels this library has launched in this process.
 * rfdd_profile(1): clear the records and time every launch of the dense contraction kernels
 * (kind 0: CUDA-core GEMM, kind 1: tensor-core GEMM) with CUDA events on their stream;
 * rfdd_profile(0) stops recording.  rfdd_profile_get sums, for one kind, the launches, their
 * event-measured milliseconds and their algorithmic flops (a complex multiply-add counts 8).
 * rfdd_profile_busy gives, for one kind, the milliseconds during which at least one recorded
 * launch was running: the union of their [start, end] intervals, so that launches of two
 * streams that ran at the same time count once (it equals the sum when launches never overlap).
 * Returns RFDD_ESTATE if launches were recorded without rfdd_profile(1). */
long long rfdd_kernel_launches(void);
/* Throughput probe of one arithmetic unit on the current device, in TFLOP/s (best of three timed
 * launches after a warm-up, CUDA events): which = 0 the tensor pipe's TF32 rate (tcgen05
 * kind::tf32 MMAs of 128 x 256 x 8 issued back to back from operand tiles held in shared memory,
 * one CTA per SM); 1 FP64 fused multiply-add on the CUDA cores; 2 FP32 fused multiply-add on the
 * CUDA cores; 3 a plain TF32 GEMM through the solver's tensor-core kernel (one MMA per product,
 * operands fed from memory; a real 8192^3 GEMM, the MMA kernel alone timed, operand packing
 * excluded).  Allocates about 1.9 GB (which = 3) or a few MB, on a stream of its own. */
int rfdd_peak_probe(int32_t which, double *tflops);
int rfdd_profile(int32_t enable);
int rfdd_profile_get(int32_t kind, int64_t *launches, double *ms, double *flops);
int rfdd_profile_busy(int32_t kind, double *busy_ms);
/* Sum, over the recorded launches of one kind, of their compulsory DRAM bytes by the traffic model
 * of the kernel: C read (when beta != 0) and written once, every packed operand tile read once.
 * (Kind 1 only; kind 0 records 0.)  Scaled by the ratio of ncu-measured to model bytes on one
 * captured launch, it gives the DRAM traffic of launches too large to capture. */
int rfdd_profile_bytes(int32_t kind, double *bytes);

/* RF-KRYLOV, Algorithm 1 (Section 2.2): the paper's comparison method, on the same factors.
 * Computes the quadrature (n_nodes, opt.quad_rule), factors every B_j(zeta_l) and S(zeta_l) as
 * rfdd_solve does, then runs Krylov on rho(M^{-1}A) in the whole space: each step applies
 * w = 2 Re sum_l omega_l (A - zeta_l M)^{-1} M q (line 2) to a block of opt.block vectors through
 * Eq. (inv_dd2) with FP64 refinement, orthogonalises in the M inner product (rho(M^{-1}A) is
 * self-adjoint there, so H_mu is symmetric; with M = I it is the printed Euclidean process), and
 * every ceil(10/opt.block) steps stops when the sum of the eigenvalues of H_mu that are >= 1/2
 * changed by at most opt.lanczos_tol of its magnitude (line 13), or when mu reaches max_dim
 * (0 = min(n, 4096)).  Lines 15-16: Rayleigh-Ritz of (A, M) on the Krylov basis, then the
 * completion passes of rfdd_solve to the residual target.  The result is read like rfdd_solve's;
 * info.mu is the Krylov dimension, info.k the Rayleigh-Ritz rank, info.t_lanczos_ms the Krylov
 * phase, rfdd_result_pre_evals the Ritz values inside [alpha, beta] before completion.  Device
 * memory beyond the factors: n x min(max_dim, n) doubles for the basis and about
 * (3 + 2 n_nodes) n x block doubles of workspace.  Errors as rfdd_solve; RFDD_EINVAL also for
 * max_dim < 0 or 0 < max_dim < opt.block. */
int rfdd_rfkrylov(rfdd_handle *h, double alpha, double beta, int32_t n_nodes, int64_t max_dim, rfdd_result **out);

/* Asynchronous solve for serving: enqueues the solve on `stream` (a cudaStream_t, NULL = the
 * handle's) and returns; rfdd_result_ready() reports completion (1 done, 0 running, <0 error
 * code negated).  The handle must not be used until the result is ready. */
int rfdd_solve_async(rfdd_handle *h, double alpha, double beta, int32_t n_nodes, void *stream,
                     rfdd_result **out);
int rfdd_result_ready(const rfdd_result *r);

/* Device bytes a solve with these parameters needs (factors, Schur complements, workspaces);
 * used for admission against a memory budget. */
int rfdd_memory_estimate(const rfdd_handle *h, int32_t n_nodes, int64_t nev_guess, size_t *bytes);

/* ---- serving: continuous batching of interval requests (no counterpart in the paper) --------
 * Many clients asking the interval problem of Section 1 on one GPU.  A pencil is set up once
 * (rfdd_server_add_pencil runs rfdd_setup on the calling thread and returns its errors) and stays
 * resident; a request names a resident pencil and an interval.  max_inflight worker threads take
 * waiting requests in arrival order, each solving on the stream of its pencil's handle, so the
 * work of different requests overlaps on the device.  A request starts when a worker is free, no
 * other request of its pencil runs (a handle serves one solve at a time) and its device-memory
 * estimate (rfdd_memory_estimate with nev_hint, or 100 when 0) fits in what mem_budget has left;
 * the first waiting request that satisfies these starts, and the oldest waiting request is passed
 * over at most max_bypass times.  After each solve the handle's factors are released
 * (rfdd_release).  A request's own mem_budget is capped at the server's (so the form of its factors,
 * rfdd_options.pack_factors, fits the server's budget).  Results are those of rfdd_solve on the same
 * pencil and interval with those options; they do not depend on what else runs. */
typedef struct rfdd_server rfdd_server;
typedef struct {
  size_t mem_budget;     /* device bytes the running requests may hold by estimate (default 150 GiB) */
  int32_t max_inflight;  /* requests running at once, one worker thread each (default 4, max 64) */
  int32_t max_bypass;    /* times the oldest waiting request may be passed over (default 8) */
  int32_t device;        /* CUDA device; -1 = the device current at rfdd_server_create (default) */
} rfdd_server_options;

typedef struct {
  int32_t status;        /* -1 waiting, -2 running, else the solve's return code (RFDD_OK,
                            RFDD_NOT_CONVERGED or an error; RFDD_ESTATE if dropped at destroy) */
  int64_t pencil;
  int64_t nev;           /* eigenpairs returned */
  size_t bytes;          /* device-memory estimate it was admitted with */
  double queue_ms;       /* submit -> start (host steady clock) */
  double run_ms;         /* start -> done */
  double latency_ms;     /* submit -> done */
} rfdd_request_info;

typedef struct {
  int64_t completed, failed, waiting;
  int32_t running, peak_running;
  size_t in_use, peak_in_use;   /* estimated device bytes of the running requests */
  int64_t pencils;              /* resident pencils */
} rfdd_server_stats;

void rfdd_server_default_options(rfdd_server_options *o);
/* RFDD_EINVAL for max_inflight outside [1, 64], a zero budget or a negative max_bypass. */
int rfdd_server_create(const rfdd_server_options *o, rfdd_server **out);
/* Set up a pencil (same inputs and errors as rfdd_setup; opt.stream is ignored: each resident
 * pencil gets a stream of its own).  *pencil_id identifies it in later calls. */
int rfdd_server_add_pencil(rfdd_server *s, const rfdd_csr *A, const rfdd_csr *M, const int32_t *part, int32_t p,
                           const rfdd_options *opt, int64_t *pencil_id);
/* Queue a request; returns at once.  RFDD_EADMIT when its estimate exceeds the whole budget (it
 * could never start), RFDD_EINVAL for an unknown pencil, alpha >= beta or n_nodes < 1. */
int rfdd_server_submit(rfdd_server *s, int64_t pencil_id, double alpha, double beta, int32_t n_nodes,
                       int64_t nev_hint, int64_t *request_id);
/* Queue a request that brings its own pencil (host CSR, location 0, copied by this call; no device
 * work here):
 * the worker that runs it sets the pencil up, solves and frees it, so its latency includes the
 * set-up.  It is admitted by the estimate of rfdd_memory_estimate plus the set-up, from the block
 * sizes that a host scan of the pattern and labels gives.  Returns at once; RFDD_EADMIT and
 * RFDD_EINVAL as for rfdd_server_submit, RFDD_EINVAL also for labels or columns out of range
 * (the other rfdd_setup errors come back as the request's status). */
int rfdd_server_submit_pencil(rfdd_server *s, const rfdd_csr *A, const rfdd_csr *M, const int32_t *part, int32_t p,
                              const rfdd_options *opt, double alpha, double beta, int32_t n_nodes,
                              int64_t nev_hint, int64_t *request_id);
/* Wait up to timeout_ms (< 0: no limit; 0: poll) for a request.  *done = 1 when it finished; then
 * *out receives its result (NULL if the solve failed; see rfdd_server_request_info for the code),
 * which the caller owns and frees with rfdd_result_free.  A result is handed out once (RFDD_ESTATE
 * on a second wait). */
int rfdd_server_wait(rfdd_server *s, int64_t request_id, double timeout_ms, int32_t *done, rfdd_result **out);
int rfdd_server_request_info(rfdd_server *s, int64_t request_id, rfdd_request_info *info);
int rfdd_server_get_stats(rfdd_server *s, rfdd_server_stats *out);
/* Frees a resident pencil; RFDD_ESTATE while requests of it wait or run (and for the pencil of a
 * rfdd_server_submit_pencil request, which the server frees itself). */
int rfdd_server_remove_pencil(rfdd_server *s, int64_t pencil_id);
/* Drops waiting requests, waits for running ones, frees every pencil and unclaimed result. */
void rfdd_server_destroy(rfdd_server *s);

#ifdef __cplusplus
}
#endif
#endif /* RFDD_H */
