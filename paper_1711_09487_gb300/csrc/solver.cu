// RF-DDES orchestration on one GPU and the C ABI (include/rfdd.h).
//
// Algorithm 3 of the paper (RF-DDES) with its interface step Algorithm 2, in the
// interior-first ordering of Eq. (dd1):
//   a0 quadrature -> a1 setup -> a2 dense shifted (bordered) blocks -> a3/a4 batched LU of
//   [[B_j(z), E_j(z)], [E_j(z)^T, 0]] (the trailing block becomes -E^T B^{-1} E) -> a5 S(z)
//   assembly + LU -> a6/a7 block Lanczos on F = Re sum w S^{-1} -> a8 interior basis
//   (V_j, Sigma, Gamma) -> a9 Rayleigh-Ritz on Z -> a10 completion passes with the DD
//   resolvent of Eq. (inv_dd2) and FP64 iterative refinement.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <functional>
#include <cmath>
#include <exception>
#include <memory>
#include <mutex>
#include <limits>
#include <numeric>
#include <system_error>
#include <thread>
#include <tuple>

#include "dense.cuh"
#include "eig.cuh"
#include "ops.cuh"
#include "probe.cuh"
#include "small.cuh"
#include "tc_gemm.cuh"

using namespace rfdd;

namespace rfdd {
std::atomic<long long> g_kernel_launches{0};
thread_local long long g_thread_launches = 0;
namespace {
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};  // read by every launching host thread
std::vector<ProfileRec> g_prof;
std::vector<cudaEvent_t> g_prof_pool;
cudaEvent_t g_prof_ref = nullptr;  // completed before any recorded launch started
}  // namespace
bool profiling_enabled() { return g_prof_on; }
cudaEvent_t profile_event() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
void profile_push(cudaEvent_t a, cudaEvent_t b, double flops, int kind, double bytes) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.push_back({a, b, flops, kind, bytes});
}
}  // namespace rfdd

namespace {

thread_local std::string g_last_error;

// Diagnostics on stderr when the environment variable RFDD_LOG is set to a nonzero value.
bool log_on() {
  static int on = [] {
    const char *v = getenv("RFDD_LOG");
    return (v && v[0] && v[0] != '0') ? 1 : 0;
  }();
  return on != 0;
}
#define RFDD_LOGF(...)                    \
  do {                                    \
    if (log_on()) {                       \
      fprintf(stderr, "[rfdd] " __VA_ARGS__); \
      fputc('\n', stderr);                \
    }                                     \
  } while (0)

// ------------------------------------------------------------------------------------
// device buffers
// ------------------------------------------------------------------------------------
// Device buffers.  Inside an AllocScope (every entry point that works on a handle's stream)
// they come from the stream-ordered pool on that stream: allocation and release are ordered
// with the stream's work and never synchronise the device, as cudaFree would between the many
// short-lived workspaces of a solve.  Outside a scope, and for buffers that must outlive the
// handle's stream (results), plain cudaMalloc / cudaFree.
thread_local cudaStream_t g_alloc_stream = nullptr;
struct AllocScope {
  cudaStream_t prev;
  explicit AllocScope(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
  ~AllocScope() { g_alloc_stream = prev; }
  AllocScope(const AllocScope &) = delete;
  AllocScope &operator=(const AllocScope &) = delete;
};

struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaStream_t st_ = nullptr;
  bool async_ = false;
  bool sync_only = false;
  Buf() = default;
  explicit Buf(bool sync) : sync_only(sync) {}
  Buf(const Buf &) = delete;
  Buf &operator=(const Buf &) = delete;
  ~Buf() { release(); }
  void release() {
    if (p) {
      if (async_) cudaFreeAsync(p, st_);
      else cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
    async_ = false;
  }
  void alloc(size_t b) {
    release();
    if (b == 0) b = 16;
    cudaError_t e;
    if (g_alloc_stream && !sync_only) {
      e = cudaMallocAsync(&p, b, g_alloc_stream);
      async_ = e == cudaSuccess;
      st_ = g_alloc_stream;
    } else {
      e = cudaMalloc(&p, b);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      async_ = false;
      throw Error(RFDD_ENOMEM, "device allocation of " + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
    }
    bytes = b;
  }
  void ensure(size_t b) {
    if (b > bytes) alloc(b);
  }
  template <typename T>
  T *as() const { return reinterpret_cast<T *>(p); }
};

// Keep freed pool memory for reuse instead of returning it to the driver at every stream
// synchronisation (once per device; affects this process's default pool only).
void keep_pool_memory() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done.push_back(dev);
}

template <typename T>
void upload(Buf &b, const std::vector<T> &v, cudaStream_t st) {
  b.alloc(v.size() * sizeof(T));
  if (!v.empty()) RFDD_CUDA(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

// CUDA-event lap timer for the diagnostics log (no-op unless RFDD_LOG is set)
struct Lap {
  cudaStream_t st;
  cudaEvent_t e0 = nullptr;
  const char *what;
  Lap(cudaStream_t s, const char *w) : st(s), what(w) {
    if (log_on()) {
      cudaEventCreate(&e0);
      cudaEventRecord(e0, st);
    }
  }
  void mark(const char *label) {
    if (!log_on()) return;
    cudaEvent_t e1;
    cudaEventCreate(&e1);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    fprintf(stderr, "[rfdd]   %s/%s: %.3f ms\n", what, label, ms);
    cudaEventDestroy(e0);
    e0 = e1;
  }
  ~Lap() {
    if (e0) cudaEventDestroy(e0);
  }
};

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  double ms() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    return t;
  }
};

}  // namespace

// ------------------------------------------------------------------------------------
// handle and result
// ------------------------------------------------------------------------------------
struct rfdd_result {
  int64_t n = 0, nev = 0;
  std::vector<double> evals, resid, pre_evals;
  std::vector<double> evecs_host;  // filled on demand
  bool host_ready = false;
  Buf evecs{true}, evals_dev{true}, resid_dev{true};  // outlive the handle's stream
  rfdd_info info{};
  std::atomic<int> ready{1};
  std::thread worker;
  cudaStream_t st = nullptr;
  ~rfdd_result() {
    if (worker.joinable()) worker.join();
  }
};

struct rfdd_handle {
  rfdd_options opt;
  int64_t n = 0, s = 0, dsum = 0, nnz = 0;
  int p = 0;
  std::vector<int64_t> off, perm, iperm, d, sidx_off, D;
  std::vector<int32_t> sidx;
  double normA = 0.0, normM = 0.0;  // max absolute row sums
  double gershM = 0.0;              // min over rows of M_ii - sum_{j != i} |M_ij| (a lower bound of M's
                                    // spectrum when positive)
  bool has_me = false;              // M_E != 0 (the Gamma block of Z is needed)
  std::vector<int64_t> host_rp;
  std::vector<int32_t> host_cl, host_posmap;
  std::vector<double> host_av, host_mv;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  // device copies
  Buf amsplit;  // double-FP32 split of the pencil values (mixed-precision residuals)
  Buf rowptr, col, aval, mval, off_dev, sidx_dev, sidx_off_dev, posmap, iperm_dev, status;
  DevPencil P;
  DevDD dd;
  // factors (a2-a5)
  int nnodes = 0;
  std::vector<cx<double>> z, w;
  Buf z_dev, w_dev, fac, boff_dev, Doff_dev, pivB, Sfac, pivS, Skeep;
  // inverses of the NBO-blocks on the diagonals of the B and S factors (triangular solves)
  Buf BLinv, BUinv, SLinv, SUinv;
  std::vector<int64_t> binvoff;  // (node, subdomain) -> offset into BLinv / BUinv
  int64_t sinv_elems = 0;        // per node in SLinv / SUinv
  // Mixed solve: tensor-core tile copies (TF32 hi/lo) of the factor operands the solves multiply
  // by, packed once per factorisation.  Per B factor (node, subdomain) and per S factor (node):
  // the leading LU, the inverse diagonal blocks of L and of U, and (B only) the border blocks L21
  // and U12.  Float offsets of each hi array into Pk; its lo array follows it.
  Buf Pk;
  struct PkOff { int64_t lu = -1, li = -1, ui = -1, l21 = -1, u12 = -1; };
  std::vector<PkOff> pkB, pkS;
  // Real factorisation of the B_sigma^(j) (a8), started on a second stream at the beginning of a
  // solve so that it overlaps the complex factorisations and the Lanczos process; interior_impl
  // waits for it through ev_join.
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  Buf IBs, Ipiv, IRLinv, IRUinv, I_doff, I_boffr_dev, I_zs, I_status;
  // V_j of the same shift (Alg. 3 step 3), computed right after the B_sigma factorisation on the
  // same stream: the M_B-orthonormal subspace basis X (dsum x I_mw), the selected eigenvectors of
  // its Rayleigh-Ritz problem (rows of I_Gt, p blocks of I_mw x I_mw) and the smallest
  // |delta - sigma| seen (the shift guard's test)
  Buf IVX, IVGt;
  int64_t I_mw = 0;
  double I_gap = 0.0;
  std::vector<int64_t> I_boffr, I_rinvoff;
  double I_sigma = 0.0;
  size_t I_tsize = 0;
  bool I_ready = false, I_forked = false;
  std::thread I_thread;       // host thread launching the started factorisation
  std::exception_ptr I_exc;   // its error, rethrown by interior_join
  std::vector<int64_t> boff, pivBoff;
  bool have_factors = false;
  bool basis_fp64 = false;         // the completion's basis products in FP64 (see complete)
  double factor_enqueue_ms = 0.0;  // host time to issue the last factorisation's launches
  long long factor_launches = 0;   // kernels it launched
  double alpha = 0, beta = 0;
  bool have_interval = false;
  // Lanczos (a7)
  Buf Q;
  int64_t mu = 0, qcap = 0;
  std::vector<double> traces;
  // interior (a8)
  Buf Zb;
  int64_t kz = 0, kappa = 0;
  std::vector<int64_t> voff;  // V_j occupies Z columns [voff[j], voff[j+1])
  double sigma_used = 0.0;
  double interior_gap = 0.0;  // min over subdomains of |delta - sigma| seen by the last interior step
  // Rayleigh-Ritz (a9)
  std::vector<double> rr_theta;
  Buf X0;
  int64_t m0 = 0;
  // Interface rows of the union CSR, kept for the two-level split: per interface row a, entries
  // [if_rp[a], if_rp[a+1]) (relative to the first interface row's first entry), their column in
  // interface numbering (-1: an interior column) and whether A or M is nonzero there.
  int64_t if_e0 = 0;  // union-CSR index of the first interface row's first entry
  std::vector<int64_t> if_rp;
  std::vector<int32_t> if_cl;
  std::vector<char> if_nz;
  // Two-level interface factorisation (rfdd_set_interface_groups): the block inverse of
  // Eq. (inv_dd2) applied to S(z) with groups of subdomains as its subdomains.
  struct Levels {
    int G = 0;                           // groups; 0 = one dense S per node
    std::vector<int32_t> group;          // group of each subdomain
    std::vector<int32_t> cls;            // per interface node: its group if level 1, else -1
    int64_t s1 = 0, s2 = 0;              // level-1 and level-2 node counts
    std::vector<int64_t> n1, n2, g1off;  // per group |I1_g|, |I2_g|, first level-order row of I1_g
    std::vector<int64_t> goff;           // per group: element offset of its block in a node's storage
    std::vector<int64_t> poff, ioff;     // per group: pivot and inverse-block offsets within a node
    int64_t tsz = 0, psz = 0, isz = 0;   // per node: storage, pivot and inverse-block elements
    std::vector<int32_t> lorder, lpos;   // level order -> interface index, and its inverse
    std::vector<int32_t> i2g;            // I2_g as level-2 positions, concatenated over groups
    std::vector<int64_t> i2g_off;        // G + 1 offsets into i2g
    std::vector<int64_t> edst;           // per interface CSR entry: offset in a node's storage or -1
    std::vector<int32_t> q, r;           // per sidx entry: position in the group block / level-2 position
    Buf lorder_dev, lpos_dev, i2g_dev, edst_dev, q_dev, r_dev;
    void clear() {
      G = 0;
      s1 = s2 = tsz = psz = isz = 0;
      for (auto *v : {&group, &cls, &lorder, &lpos, &i2g, &q, &r}) v->clear();
      for (auto *v : {&n1, &n2, &g1off, &goff, &poff, &ioff, &i2g_off, &edst}) v->clear();
      for (Buf *b : {&lorder_dev, &lpos_dev, &i2g_dev, &edst_dev, &q_dev, &r_dev}) b->release();
    }
  } lv;
  Buf Lfac, pivL, LLinv, LUinv;          // two-level factors, nc nodes x (tsz, psz, isz)
  std::vector<PkOff> pkG;                // packed operands of the group blocks (node, group)
};

namespace {

inline bool is_mixed(const rfdd_handle *h) { return h->opt.precision == RFDD_MIXED; }

// Waits for the handle's stream, then raises what the device recorded in the status word w
// (h->status unless given; the tensor-core GEMMs of the handle record their wait time-outs in the
// same word); a nonzero word is cleared.
void sync_status(rfdd_handle *h, const char *where, Buf *w = nullptr) {
  RFDD_CUDA(cudaStreamSynchronize(h->st));
  if (!w) w = &h->status;
  int s = 0;
  RFDD_CUDA(cudaMemcpyAsync(&s, w->p, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  RFDD_CUDA(cudaStreamSynchronize(h->st));
  if (s != 0) {
    RFDD_CUDA(cudaMemsetAsync(w->p, 0, sizeof(int), h->st));
    RFDD_CUDA(cudaStreamSynchronize(h->st));
    if (s & DS_WAIT_TIMEOUT)
      throw Error(RFDD_ECUDA, std::string(where) + ": a tensor-core GEMM timed out waiting for its operands");
    if (s & (DS_ZERO_PIVOT | DS_NONFINITE))
      throw Error(RFDD_ESINGULAR, std::string(where) + ": zero or non-finite pivot (device status " +
                                      std::to_string(s) + ")");
    throw Error(RFDD_ECUDA, std::string(where) + ": device status " + std::to_string(s));
  }
}

// ------------------------------------------------------------------------------------
// a0: quadrature (Section 2.1; midpoint rule of Section 6)
// ------------------------------------------------------------------------------------
void quadrature(double alpha, double beta, int nc, int rule, std::vector<cx<double>> &z,
                std::vector<cx<double>> &w) {
  RFDD_REQUIRE(beta > alpha && nc >= 1, RFDD_EINVAL, "quadrature: need alpha < beta and n_nodes >= 1");
  const double c = 0.5 * (alpha + beta), r = 0.5 * (beta - alpha);
  z.resize(nc);
  w.resize(nc);
  if (rule == RFDD_MIDPOINT) {
    for (int l = 0; l < nc; ++l) {
      const double th = (2.0 * (l + 1) - 1.0) * M_PI / (2.0 * nc);
      const double er = std::cos(th), ei = std::sin(th);
      z[l] = cx<double>(c + r * er, r * ei);
      w[l] = cx<double>(-r * er / (2.0 * nc), -r * ei / (2.0 * nc));
    }
  } else if (rule == RFDD_GAUSS_LEGENDRE) {
    // Gauss-Legendre nodes by Newton iteration on P_nc from Chebyshev starting points
    std::vector<double> t(nc), wt(nc);
    for (int i = 0; i < nc; ++i) {
      double x = std::cos(M_PI * (i + 0.75) / (nc + 0.5));
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= nc; ++k) {
          const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        double pn = nc == 1 ? x : p1, pm = nc == 1 ? 1.0 : p0;
        const double dp = nc * (x * pn - pm) / (x * x - 1.0);
        const double dx = pn / dp;
        x -= dx;
        if (std::fabs(dx) < 1e-16) break;
      }
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= nc; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = nc == 1 ? x : p1, pm = nc == 1 ? 1.0 : p0;
      const double dp = nc * (x * pn - pm) / (x * x - 1.0);
      t[i] = x;
      wt[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    {  // ascending nodes t (theta increasing)
      std::vector<int> o(nc);
      std::iota(o.begin(), o.end(), 0);
      std::sort(o.begin(), o.end(), [&](int a, int b) { return t[a] < t[b]; });
      std::vector<double> t2(nc), w2(nc);
      for (int i = 0; i < nc; ++i) { t2[i] = t[o[i]]; w2[i] = wt[o[i]]; }
      t.swap(t2);
      wt.swap(w2);
    }
    for (int l = 0; l < nc; ++l) {
      const double th = 0.5 * M_PI * (1.0 + t[l]);
      const double er = std::cos(th), ei = std::sin(th);
      z[l] = cx<double>(c + r * er, r * ei);
      w[l] = cx<double>(-0.25 * r * wt[l] * er, -0.25 * r * wt[l] * ei);
    }
  } else {
    throw Error(RFDD_EINVAL, "quadrature: unknown rule");
  }
}

// ------------------------------------------------------------------------------------
// a1: setup (validation, interior-first ordering, union CSR, interface maps)
// ------------------------------------------------------------------------------------
void validate_csr(const rfdd_csr *A, const char *name) {
  RFDD_REQUIRE(A && A->rowptr && A->col && A->val && A->n > 0, RFDD_EINVAL, std::string(name) + ": NULL or empty");
  const int64_t n = A->n;
  RFDD_REQUIRE(A->rowptr[0] == 0, RFDD_EINVAL, std::string(name) + ": rowptr[0] != 0");
  for (int64_t i = 0; i < n; ++i) {
    RFDD_REQUIRE(A->rowptr[i + 1] >= A->rowptr[i], RFDD_EINVAL, std::string(name) + ": rowptr not monotone");
    for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      RFDD_REQUIRE(A->col[e] >= 0 && A->col[e] < n, RFDD_EINVAL, std::string(name) + ": column out of range");
      RFDD_REQUIRE(std::isfinite(A->val[e]), RFDD_EINVAL, std::string(name) + ": non-finite value");
    }
  }
}

// A CSR given in device memory (rfdd_csr.location = 1) copied to host vectors; a host CSR is
// returned as it is.
struct HostCsrCopy {
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  rfdd_csr view{};
};
const rfdd_csr *on_host(const rfdd_csr *X, HostCsrCopy &c, const char *name) {
  if (!X || X->location == 0) return X;
  RFDD_REQUIRE(X->location == 1, RFDD_EINVAL, std::string(name) + ": location must be 0 (host) or 1 (device)");
  RFDD_REQUIRE(X->rowptr && X->col && X->val && X->n > 0, RFDD_EINVAL, std::string(name) + ": NULL or empty");
  c.rowptr.resize(X->n + 1);
  RFDD_CUDA(cudaMemcpy(c.rowptr.data(), X->rowptr, (X->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
  const int64_t nnz = c.rowptr[X->n];
  RFDD_REQUIRE(c.rowptr[0] == 0 && nnz >= 0, RFDD_EINVAL, std::string(name) + ": bad row pointers");
  c.col.resize(nnz);
  c.val.resize(nnz);
  if (nnz > 0) {
    RFDD_CUDA(cudaMemcpy(c.col.data(), X->col, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
    RFDD_CUDA(cudaMemcpy(c.val.data(), X->val, nnz * sizeof(double), cudaMemcpyDeviceToHost));
  }
  c.view = rfdd_csr{X->n, c.rowptr.data(), c.col.data(), c.val.data(), 0};
  return &c.view;
}

// symmetric in pattern and value: compare with the transpose built by counting sort
// Host work over rows split into contiguous chunks, one thread per chunk (results do not depend
// on the number of threads).
template <typename F>
void parallel_rows(int64_t n, F &&f) {
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(std::thread::hardware_concurrency(), (n + 4095) / 4096));
  if (nt <= 1) {
    f(0, n, 0);
    return;
  }
  std::vector<std::thread> th;
  for (int64_t t = 0; t < nt; ++t) th.emplace_back([&, t] { f(n * t / nt, n * (t + 1) / nt, (int)t); });
  for (auto &x : th) x.join();
}

void check_symmetric(const rfdd_csr *A, const char *name) {
  const int64_t n = A->n, nnz = A->rowptr[n];
  // rows with strictly increasing columns: look every entry's mirror up by binary search
  std::atomic<int> unsorted{0};
  parallel_rows(n, [&](int64_t r0, int64_t r1, int) {
    for (int64_t i = r0; i < r1; ++i)
      for (int64_t e = A->rowptr[i] + 1; e < A->rowptr[i + 1]; ++e)
        if (A->col[e] <= A->col[e - 1]) {
          unsorted = 1;
          return;
        }
  });
  if (!unsorted) {
    std::atomic<int> bad{0};  // 1: pattern, 2: values
    parallel_rows(n, [&](int64_t r0, int64_t r1, int) {
      for (int64_t i = r0; i < r1 && !bad.load(std::memory_order_relaxed); ++i)
        for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
          const int64_t j = A->col[e];
          const int32_t *b = A->col + A->rowptr[j], *en = A->col + A->rowptr[j + 1];
          const int32_t *f = std::lower_bound(b, en, (int32_t)i);
          if (f == en || *f != i) {
            bad = 1;
            return;
          }
          const double a = A->val[e], c = A->val[A->rowptr[j] + (f - b)];
          if (!(std::fabs(a - c) <= 1e-14 * std::max(std::fabs(a), std::fabs(c)))) {
            bad = 2;
            return;
          }
        }
    });
    RFDD_REQUIRE(bad != 1, RFDD_ENOTSYM, std::string(name) + " is not symmetric (pattern)");
    RFDD_REQUIRE(bad != 2, RFDD_ENOTSYM, std::string(name) + " is not symmetric (values)");
    return;
  }
  std::vector<int64_t> cnt(n + 1, 0);
  for (int64_t e = 0; e < nnz; ++e) cnt[A->col[e] + 1]++;
  for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
  std::vector<int64_t> trow(nnz);
  std::vector<double> tval(nnz);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      const int64_t q = pos[A->col[e]]++;
      trow[q] = i;
      tval[q] = A->val[e];
    }
  // row i of A^T: entries (trow, tval) in [cnt[i], cnt[i+1]), already in increasing row order;
  // compare with row i of A as sorted sets
  std::atomic<int> bad{0};  // 1: pattern, 2: values, 3: a column twice in one row
  parallel_rows(n, [&](int64_t r0, int64_t r1, int) {
    std::vector<std::pair<int64_t, double>> ra;
    for (int64_t i = r0; i < r1 && !bad.load(std::memory_order_relaxed); ++i) {
      ra.clear();
      for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) ra.push_back({A->col[e], A->val[e]});
      if (!std::is_sorted(ra.begin(), ra.end(), [](auto &x, auto &y) { return x.first < y.first; }))
        std::sort(ra.begin(), ra.end());
      for (size_t k = 1; k < ra.size(); ++k)
        if (ra[k].first == ra[k - 1].first) {
          bad = 3;
          return;
        }
      if ((int64_t)ra.size() != cnt[i + 1] - cnt[i]) {
        bad = 1;
        return;
      }
      for (size_t k = 0; k < ra.size(); ++k) {
        const int64_t q = cnt[i] + (int64_t)k;
        if (ra[k].first != trow[q]) {
          bad = 1;
          return;
        }
        const double a = ra[k].second, b = tval[q];
        if (!(std::fabs(a - b) <= 1e-14 * std::max(std::fabs(a), std::fabs(b)))) {
          bad = 2;
          return;
        }
      }
    }
  });
  RFDD_REQUIRE(bad != 3, RFDD_EINVAL, std::string(name) + ": a column appears twice in one row");
  RFDD_REQUIRE(bad != 1, RFDD_ENOTSYM, std::string(name) + " is not symmetric (pattern)");
  RFDD_REQUIRE(bad != 2, RFDD_ENOTSYM, std::string(name) + " is not symmetric (values)");
}
void do_setup(rfdd_handle *h, const rfdd_csr *A, const rfdd_csr *M, const int32_t *part, int32_t p) {
  validate_csr(A, "A");
  validate_csr(M, "M");
  RFDD_REQUIRE(A->n == M->n, RFDD_EINVAL, "A and M differ in size");
  RFDD_REQUIRE(part != nullptr && p >= 1, RFDD_EINVAL, "partition: NULL or p < 1");
  check_symmetric(A, "A");
  check_symmetric(M, "M");
  const int64_t n = A->n;
  for (int64_t i = 0; i < n; ++i) {
    bool diag = false;
    for (int64_t e = M->rowptr[i]; e < M->rowptr[i + 1]; ++e)
      if (M->col[e] == i) {
        RFDD_REQUIRE(M->val[e] > 0.0, RFDD_ENOTSPD_M, "M has a non-positive diagonal entry");
        diag = true;
      }
    RFDD_REQUIRE(diag, RFDD_ENOTSPD_M, "M has a zero diagonal entry");
  }
  std::vector<int64_t> count(p + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    RFDD_REQUIRE(part[i] >= -1 && part[i] < p, RFDD_EPARTITION, "partition label out of range");
    count[part[i] + 1]++;
  }
  RFDD_REQUIRE(count[0] > 0, RFDD_EPARTITION, "partition has no interface unknowns");
  for (int j = 0; j < p; ++j) RFDD_REQUIRE(count[j + 1] > 0, RFDD_EPARTITION, "empty subdomain");
  for (const rfdd_csr *X : {A, M})
    for (int64_t i = 0; i < n; ++i)
      for (int64_t e = X->rowptr[i]; e < X->rowptr[i + 1]; ++e) {
        const int a = part[i], b = part[X->col[e]];
        RFDD_REQUIRE(!(a >= 0 && b >= 0 && a != b), RFDD_EPARTITION,
                     "partition is not a vertex separator (two subdomains are coupled)");
      }
  h->n = n;
  h->p = p;
  h->d.assign(p, 0);
  for (int j = 0; j < p; ++j) h->d[j] = count[j + 1];
  h->s = count[0];
  h->off.assign(p + 1, 0);
  for (int j = 0; j < p; ++j) h->off[j + 1] = h->off[j] + h->d[j];
  h->dsum = h->off[p];
  h->perm.resize(n);
  h->iperm.resize(n);
  {
    std::vector<int64_t> cur(h->off.begin(), h->off.end());
    int64_t ci = h->dsum;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t r = part[i] >= 0 ? cur[part[i]]++ : ci++;
      h->perm[r] = i;
      h->iperm[i] = r;
    }
  }
  // union CSR in the new ordering: rows merged in parallel chunks, then concatenated in order
  std::vector<int64_t> rp(n + 1, 0);
  std::vector<int32_t> cl;
  std::vector<double> av, mv;
  const int64_t nt_max = std::max<int64_t>(1, std::thread::hardware_concurrency());
  std::vector<std::vector<int32_t>> ccl(nt_max);
  std::vector<std::vector<double>> cav(nt_max), cmv(nt_max);
  std::vector<double> cna(nt_max, 0.0), cnm(nt_max, 0.0), cgm(nt_max, std::numeric_limits<double>::infinity());
  std::vector<int64_t> cr0(nt_max, -1);
  std::vector<int64_t> rowlen(n, 0);
  parallel_rows(n, [&](int64_t r0, int64_t r1, int t) {
    // thread-local buffers (vector headers of different threads would share cache lines)
    std::vector<std::pair<int64_t, std::pair<double, double>>> row;
    std::vector<int32_t> c;
    std::vector<double> a, m;
    double na = 0.0, nm = 0.0, gm = std::numeric_limits<double>::infinity();
    int64_t est = 0;
    for (int64_t r = r0; r < r1; ++r) {
      const int64_t i = h->perm[r];
      est += (A->rowptr[i + 1] - A->rowptr[i]) + (M->rowptr[i + 1] - M->rowptr[i]);
    }
    c.reserve(est);
    a.reserve(est);
    m.reserve(est);
    for (int64_t r = r0; r < r1; ++r) {
      const int64_t i = h->perm[r];
      row.clear();
      double sa = 0, sm = 0;
      for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
        row.push_back({h->iperm[A->col[e]], {A->val[e], 0.0}});
        sa += std::fabs(A->val[e]);
      }
      double mdiag = 0.0;
      for (int64_t e = M->rowptr[i]; e < M->rowptr[i + 1]; ++e) {
        row.push_back({h->iperm[M->col[e]], {0.0, M->val[e]}});
        sm += std::fabs(M->val[e]);
        if (M->col[e] == i) mdiag += M->val[e];
      }
      na = std::max(na, sa);
      nm = std::max(nm, sm);
      gm = std::min(gm, 2.0 * mdiag - sm);
      // equal columns are summed below; each entry holds only one of (a, m), so their order is free
      std::sort(row.begin(), row.end(), [](auto &x, auto &y) { return x.first < y.first; });
      const size_t before = c.size();
      for (size_t k = 0; k < row.size(); ++k) {
        if (c.size() > before && c.back() == row[k].first) {
          a.back() += row[k].second.first;
          m.back() += row[k].second.second;
        } else {
          c.push_back((int32_t)row[k].first);
          a.push_back(row[k].second.first);
          m.push_back(row[k].second.second);
        }
      }
      rowlen[r] = (int64_t)(c.size() - before);
    }
    cr0[t] = r0;
    cna[t] = na;
    cnm[t] = nm;
    cgm[t] = gm;
    ccl[t] = std::move(c);
    cav[t] = std::move(a);
    cmv[t] = std::move(m);
  });
  for (int64_t r = 0; r < n; ++r) rp[r + 1] = rp[r] + rowlen[r];
  h->normA = h->normM = 0.0;
  h->gershM = std::numeric_limits<double>::infinity();
  for (int64_t t = 0; t < nt_max; ++t) {
    h->normA = std::max(h->normA, cna[t]);
    h->normM = std::max(h->normM, cnm[t]);
    h->gershM = std::min(h->gershM, cgm[t]);
  }
  cl.resize(rp[n]);
  av.resize(rp[n]);
  mv.resize(rp[n]);
  for (int64_t t = 0; t < nt_max; ++t) {
    if (cr0[t] < 0) continue;
    const int64_t o = rp[cr0[t]];
    std::copy(ccl[t].begin(), ccl[t].end(), cl.begin() + o);
    std::copy(cav[t].begin(), cav[t].end(), av.begin() + o);
    std::copy(cmv[t].begin(), cmv[t].end(), mv.begin() + o);
  }
  h->nnz = rp[n];
  // interface coupling sets sidx_j
  const int64_t s = h->s, dsum = h->dsum;
  std::vector<int32_t> posmap((size_t)p * s, -1);
  h->sidx.clear();
  h->sidx_off.assign(p + 1, 0);
  for (int j = 0; j < p; ++j) {
    std::vector<int32_t> touched;
    for (int64_t r = h->off[j]; r < h->off[j + 1]; ++r)
      for (int64_t e = rp[r]; e < rp[r + 1]; ++e)
        if (cl[e] >= dsum) touched.push_back((int32_t)(cl[e] - dsum));
    std::sort(touched.begin(), touched.end());
    touched.erase(std::unique(touched.begin(), touched.end()), touched.end());
    for (size_t k = 0; k < touched.size(); ++k) posmap[(size_t)j * s + touched[k]] = (int32_t)k;
    h->sidx.insert(h->sidx.end(), touched.begin(), touched.end());
    h->sidx_off[j + 1] = (int64_t)h->sidx.size();
  }
  h->D.resize(p);
  for (int j = 0; j < p; ++j) h->D[j] = h->d[j] + (h->sidx_off[j + 1] - h->sidx_off[j]);
  h->host_rp = std::move(rp);
  h->host_cl = std::move(cl);
  h->host_av = std::move(av);
  h->host_mv = std::move(mv);
  h->host_posmap = std::move(posmap);
}

void do_upload(rfdd_handle *h) {
  const int p = h->p;
  const int64_t n = h->n, s = h->s, dsum = h->dsum;
  auto &rp = h->host_rp;
  auto &cl = h->host_cl;
  auto &av = h->host_av;
  auto &mv = h->host_mv;
  auto &posmap = h->host_posmap;
  cudaStream_t st = h->st;
  upload(h->rowptr, rp, st);
  upload(h->col, cl, st);
  upload(h->aval, av, st);
  upload(h->mval, mv, st);
  upload(h->off_dev, h->off, st);
  upload(h->sidx_dev, h->sidx, st);
  upload(h->sidx_off_dev, h->sidx_off, st);
  upload(h->posmap, posmap, st);
  upload(h->iperm_dev, h->iperm, st);
  h->status.alloc(sizeof(int));
  RFDD_CUDA(cudaMemsetAsync(h->status.p, 0, sizeof(int), st));
  RFDD_CUDA(cudaStreamSynchronize(st));
  h->P.n = n;
  h->P.nnz = h->nnz;
  h->P.rowptr = h->rowptr.as<int64_t>();
  h->P.col = h->col.as<int32_t>();
  h->P.a = h->aval.as<double>();
  h->P.m = h->mval.as<double>();
  h->amsplit.alloc((size_t)std::max<int64_t>(1, h->nnz) * sizeof(float4));
  split_pencil(st, h->P, h->amsplit.as<float4>());
  h->dd.p = p;
  h->dd.dsum = dsum;
  h->dd.s = s;
  h->dd.off = h->off_dev.as<int64_t>();
  h->dd.sidx = h->sidx_dev.as<int32_t>();
  h->dd.sidx_off = h->sidx_off_dev.as<int64_t>();
  h->dd.posmap = h->posmap.as<int32_t>();
  // interface rows, for the two-level split of the interface
  h->if_e0 = rp[dsum];
  h->if_rp.assign(s + 1, 0);
  h->if_cl.clear();
  h->if_nz.clear();
  for (int64_t a = 0; a < s; ++a) {
    for (int64_t e = rp[dsum + a]; e < rp[dsum + a + 1]; ++e) {
      h->if_cl.push_back(cl[e] >= dsum ? (int32_t)(cl[e] - dsum) : -1);
      h->if_nz.push_back(av[e] != 0.0 || mv[e] != 0.0);
    }
    h->if_rp[a + 1] = (int64_t)h->if_cl.size();
  }
  // M_E != 0 iff some interior row has a nonzero M entry in an interface column
  h->has_me = false;
  for (int64_t r = 0; r < dsum && !h->has_me; ++r)
    for (int64_t e = rp[r]; e < rp[r + 1]; ++e)
      if (cl[e] >= dsum && mv[e] != 0.0) { h->has_me = true; break; }
  rp.clear(); cl.clear(); av.clear(); mv.clear(); posmap.clear();
  rp.shrink_to_fit(); cl.shrink_to_fit(); av.shrink_to_fit(); mv.shrink_to_fit(); posmap.shrink_to_fit();
}

constexpr int NBO_LU = 256;  // outer block (trailing-update depth) of the factorisations
constexpr int NBO = 256;     // outer block of the triangular solves

// Two-level split of the interface for a grouping of the subdomains (rfdd_set_interface_groups).
// S(z)[a][b] can be nonzero only when interface nodes a and b touch a common subdomain (a term
// of E^T B^{-1} E) or are coupled in C or M_C.  Node a is level 1 of group g when every
// subdomain it touches is in g (at least one) and no node it is coupled to in C or M_C is such a
// candidate of another group; all other nodes are level 2.  S restricted to the level-1 nodes is
// then block diagonal over the groups, and I2_g (the level-2 nodes S can couple to I1_g) are the
// level-2 nodes touched by a subdomain of g or coupled in C / M_C to a node of I1_g.
void build_levels(rfdd_handle *h, int G, const int32_t *group) {
  auto &L = h->lv;
  L.clear();
  if (G <= 0) return;
  const int p = h->p;
  const int64_t s = h->s;
  L.G = G;
  L.group.assign(group, group + p);
  std::vector<int32_t> touch(s, -2);  // -2 none, -1 several groups, else the one group
  for (int j = 0; j < p; ++j)
    for (int64_t t = h->sidx_off[j]; t < h->sidx_off[j + 1]; ++t) {
      const int32_t a = h->sidx[t];
      touch[a] = touch[a] == -2 ? group[j] : (touch[a] == group[j] ? touch[a] : -1);
    }
  L.cls.assign(s, -1);
  for (int64_t a = 0; a < s; ++a) {
    if (touch[a] < 0) continue;
    bool ok = true;
    for (int64_t e = h->if_rp[a]; e < h->if_rp[a + 1] && ok; ++e) {
      const int32_t b = h->if_cl[e];
      if (b >= 0 && h->if_nz[e] && touch[b] >= 0 && touch[b] != touch[a]) ok = false;
    }
    if (ok) L.cls[a] = touch[a];
  }
  // level order: I1_0, I1_1, ..., I2 (each ascending)
  L.n1.assign(G, 0);
  L.n2.assign(G, 0);
  L.g1off.assign(G + 1, 0);
  std::vector<int32_t> pos1(s, -1), pos2(s, -1);  // index in I1_g, index in I2
  for (int64_t a = 0; a < s; ++a)
    if (L.cls[a] >= 0) pos1[a] = (int32_t)L.n1[L.cls[a]]++;
    else pos2[a] = (int32_t)L.s2++;
  for (int g = 0; g < G; ++g) L.g1off[g + 1] = L.g1off[g] + L.n1[g];
  L.s1 = L.g1off[G];
  L.lorder.assign(s, 0);
  L.lpos.assign(s, 0);
  for (int64_t a = 0; a < s; ++a) {
    const int64_t q = L.cls[a] >= 0 ? L.g1off[L.cls[a]] + pos1[a] : L.s1 + pos2[a];
    L.lorder[q] = (int32_t)a;
    L.lpos[a] = (int32_t)q;
  }
  // I2_g, and each group block's position of its level-2 nodes
  std::vector<std::vector<int32_t>> i1(G);
  for (int64_t a = 0; a < s; ++a)
    if (L.cls[a] >= 0) i1[L.cls[a]].push_back((int32_t)a);
  L.i2g_off.assign(G + 1, 0);
  std::vector<int32_t> gpos2(s, -1);  // index of a level-2 node in I2_g of the group at hand
  L.edst.assign(h->if_cl.size(), -1);
  L.q.assign(h->sidx.size(), -1);
  L.r.assign(h->sidx.size(), -1);
  L.goff.assign(G, 0);
  L.poff.assign(G, 0);
  L.ioff.assign(G, 0);
  int64_t tot = L.s2 * L.s2, ptot = L.s2, itot = block_inverse_elems(L.s2, NBO);
  for (int g = 0; g < G; ++g) {
    std::vector<char> near(s, 0);
    for (int j = 0; j < p; ++j)
      if (group[j] == g)
        for (int64_t t = h->sidx_off[j]; t < h->sidx_off[j + 1]; ++t) near[h->sidx[t]] = 1;
    for (int32_t a : i1[g])
      for (int64_t e = h->if_rp[a]; e < h->if_rp[a + 1]; ++e)
        if (h->if_cl[e] >= 0 && h->if_nz[e]) near[h->if_cl[e]] = 1;
    std::vector<int32_t> j2;
    for (int64_t b = 0; b < s; ++b)
      if (near[b] && L.cls[b] < 0) j2.push_back((int32_t)b);
    L.n2[g] = (int64_t)j2.size();
    for (size_t k = 0; k < j2.size(); ++k) {
      gpos2[j2[k]] = (int32_t)k;
      L.i2g.push_back(pos2[j2[k]]);
    }
    L.i2g_off[g + 1] = (int64_t)L.i2g.size();
    const int64_t n1 = L.n1[g], Dg = n1 + L.n2[g];
    L.goff[g] = tot;
    L.poff[g] = ptot;
    L.ioff[g] = itot;
    tot += Dg * Dg;
    ptot += n1;
    itot += block_inverse_elems(n1, NBO);
    // position of node x in group g's bordered block (-1: not in it)
    auto gp = [&](int32_t x) -> int64_t {
      if (L.cls[x] == g) return pos1[x];
      if (L.cls[x] < 0 && gpos2[x] >= 0) return n1 + gpos2[x];
      return -1;
    };
    // C - z M_C entries in the group block: rows of I1_g, and rows of I2_g at columns of I1_g
    for (int32_t a : i1[g])
      for (int64_t e = h->if_rp[a]; e < h->if_rp[a + 1]; ++e) {
        const int32_t b = h->if_cl[e];
        if (b < 0) continue;
        const int64_t cb = gp(b);
        if (cb >= 0) L.edst[e] = L.goff[g] + (int64_t)pos1[a] * Dg + cb;
      }
    for (int32_t a : j2)
      for (int64_t e = h->if_rp[a]; e < h->if_rp[a + 1]; ++e) {
        const int32_t b = h->if_cl[e];
        if (b >= 0 && L.cls[b] == g) L.edst[e] = L.goff[g] + (n1 + gpos2[a]) * Dg + pos1[b];
      }
    for (int j = 0; j < p; ++j)
      if (group[j] == g)
        for (int64_t t = h->sidx_off[j]; t < h->sidx_off[j + 1]; ++t) {
          const int32_t a = h->sidx[t];
          L.q[t] = (int32_t)gp(a);
          L.r[t] = L.cls[a] < 0 ? pos2[a] : -1;
        }
    for (int32_t b : j2) gpos2[b] = -1;
  }
  // level-2 rows at level-2 columns go to S2
  for (int64_t a = 0; a < s; ++a)
    if (L.cls[a] < 0)
      for (int64_t e = h->if_rp[a]; e < h->if_rp[a + 1]; ++e) {
        const int32_t b = h->if_cl[e];
        if (b >= 0 && L.cls[b] < 0) L.edst[e] = (int64_t)pos2[a] * L.s2 + pos2[b];
      }
  L.tsz = tot;
  L.psz = ptot;
  L.isz = itot;
  cudaStream_t st = h->st;
  upload(L.lorder_dev, L.lorder, st);
  upload(L.lpos_dev, L.lpos, st);
  if (!L.i2g.empty()) upload(L.i2g_dev, L.i2g, st);
  if (!L.edst.empty()) upload(L.edst_dev, L.edst, st);
  upload(L.q_dev, L.q, st);
  upload(L.r_dev, L.r, st);
  RFDD_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------------------------
// precision-dependent parts
// ------------------------------------------------------------------------------------

}  // namespace

// Device bytes of the factors of one solve at their peak (a2-a5 storage, inverted diagonal
// blocks, pivots; with tile copies, the copies too: the complex64 factors are freed only after
// they have been packed).
static size_t factor_bytes_impl(const SolveShape &g, int nc, bool packed) {
  const bool mixed = g.precision == RFDD_MIXED;
  const size_t scal = mixed ? sizeof(cx<float>) : sizeof(cx<double>);
  size_t e = 0;
  for (int j = 0; j < g.p; ++j) e += (size_t)g.D[j] * g.D[j];
  size_t b = (size_t)nc * e * scal;
  // interface factors: one dense S, or S2' and the bordered group blocks
  size_t se = (size_t)g.s * g.s, sinv = (size_t)block_inverse_elems(g.s, 256), spk = se + 2 * sinv;
  if (g.lv_groups > 0) {
    se = (size_t)g.lv_s2 * g.lv_s2;
    sinv = (size_t)block_inverse_elems(g.lv_s2, 256);
    spk = se + 2 * sinv;
    for (int k = 0; k < g.lv_groups; ++k) {
      const size_t n1 = (size_t)g.lv_n1[k], n2 = (size_t)g.lv_n2[k], bi = (size_t)block_inverse_elems(n1, 256);
      se += (n1 + n2) * (n1 + n2);
      sinv += bi;
      spk += n1 * n1 + 2 * n1 * n2 + 2 * bi;
    }
  }
  b += (size_t)nc * se * scal * (g.keep_schur ? 2 : 1);
  size_t inv = sinv;  // inverted diagonal blocks of L and U
  for (int j = 0; j < g.p; ++j) inv += (size_t)block_inverse_elems(g.d[j], 256);
  b += 2 * (size_t)nc * inv * scal;
  if (mixed && packed) {  // packed tensor-core copies of the solve operands (hi + lo)
    size_t pk = spk;
    for (int j = 0; j < g.p; ++j)
      pk += (size_t)g.D[j] * g.D[j] - (size_t)(g.D[j] - g.d[j]) * (g.D[j] - g.d[j]) +
            2 * (size_t)block_inverse_elems(g.d[j], 256);
    b += (size_t)nc * pk * 2 * scal;
  }
  int64_t dsum = 0;
  for (int j = 0; j < g.p; ++j) dsum += g.d[j];
  b += (size_t)nc * (dsum + g.s) * sizeof(int);
  return b;
}

bool rfdd::packed_factors(const SolveShape &g, int nc) {
  if (g.precision != RFDD_MIXED || g.pack_factors == 0) return false;
  if (g.pack_factors == 1 || g.mem_budget == 0) return true;
  return factor_bytes_impl(g, nc, true) <= g.mem_budget;
}

size_t rfdd::factor_bytes_of(const SolveShape &g, int nc) { return factor_bytes_impl(g, nc, packed_factors(g, nc)); }

// Device bytes a solve holds at its peak: the factors, the completion blocks for about nev_guess
// pairs, the Lanczos basis; plus, when with_setup, the resident set-up (union CSR with both
// values, its double-FP32 split, maps).
size_t rfdd::solve_bytes_of(const SolveShape &g, int nc, int64_t nev_guess, bool with_setup) {
  const size_t scal = g.precision == RFDD_MIXED ? sizeof(cx<float>) : sizeof(cx<double>);
  size_t b = factor_bytes_of(g, nc);
  int64_t m = nev_guess + std::max<int64_t>((int64_t)std::ceil(g.guard_frac * nev_guess), g.min_guard);
  if (g.m_align > 1) m = (m + g.m_align - 1) / g.m_align * g.m_align;
  b += (size_t)nc * g.n * m * (sizeof(cx<double>) * 4 + scal * 2);  // completion blocks
  b += (size_t)nc * g.n * m * scal;  // triangular solves: full-height block products
  b += (size_t)g.s * g.s * sizeof(double);                           // Lanczos basis
  if (with_setup) b += (size_t)g.nnz * (4 + 8 + 8 + 16) + (size_t)g.n * 64;
  return b;
}

namespace {

rfdd::SolveShape shape_of(const rfdd_handle *h) {
  rfdd::SolveShape g;
  g.n = h->n;
  g.s = h->s;
  g.p = h->p;
  g.nnz = h->nnz;
  g.d = h->d.data();
  g.D = h->D.data();
  g.precision = h->opt.precision;
  g.keep_schur = h->opt.keep_schur;
  g.guard_frac = h->opt.guard_frac;
  g.min_guard = h->opt.min_guard;
  g.m_align = h->opt.m_align;
  g.pack_factors = h->opt.pack_factors;
  g.mem_budget = h->opt.mem_budget;
  g.lv_groups = h->lv.G;
  g.lv_s2 = h->lv.s2;
  g.lv_n1 = h->lv.n1.data();
  g.lv_n2 = h->lv.n2.data();
  return g;
}

size_t factor_bytes(const rfdd_handle *h, int nc) { return rfdd::factor_bytes_of(shape_of(h), nc); }

void pack_factor_operands(rfdd_handle *h);
template <typename Tf>
void factor_levels(rfdd_handle *h, const Tf *base);

template <typename Tf>
void factor_impl(rfdd_handle *h) {
  const auto host0 = std::chrono::steady_clock::now();
  const long long launches0 = g_thread_launches;
  cudaStream_t st = h->st;
  const int nc = h->nnodes, p = h->p;
  const int64_t s = h->s;
  // a2: bordered blocks for all (node, subdomain)
  h->boff.assign((size_t)nc * p, 0);
  int64_t tot = 0;
  for (int l = 0; l < nc; ++l)
    for (int j = 0; j < p; ++j) {
      h->boff[(size_t)l * p + j] = tot;
      tot += h->D[j] * h->D[j];
    }
  std::vector<int64_t> Doff(p + 1, 0);
  for (int j = 0; j < p; ++j) Doff[j + 1] = Doff[j] + h->D[j];
  h->fac.alloc((size_t)tot * sizeof(Tf));
  upload(h->boff_dev, h->boff, st);
  upload(h->Doff_dev, Doff, st);
  h->pivBoff.assign((size_t)nc * p, 0);
  int64_t pt = 0;
  for (int l = 0; l < nc; ++l)
    for (int j = 0; j < p; ++j) {
      h->pivBoff[(size_t)l * p + j] = pt;
      pt += h->d[j];
    }
  h->pivB.alloc((size_t)pt * sizeof(int));
  Tf *base = h->fac.as<Tf>();
  assemble_blocks<Tf>(st, h->P, h->dd, h->Doff_dev.as<int64_t>(), Doff[p], h->boff_dev.as<int64_t>(),
                      h->z_dev.as<cx<double>>(), nc, base, true);
  // a3 + a4: LU of the bordered blocks (pivots restricted to the B rows)
  std::vector<LuItem<Tf>> items;
  for (int l = 0; l < nc; ++l)
    for (int j = 0; j < p; ++j) {
      LuItem<Tf> it;
      it.A = base + h->boff[(size_t)l * p + j];
      it.piv = h->pivB.as<int>() + h->pivBoff[(size_t)l * p + j];
      it.dp = (int)h->d[j];
      it.D = (int)h->D[j];
      it.ld = (int)h->D[j];
      items.push_back(it);
    }
  lu_batched<Tf>(st, items, NBO_LU, h->status.as<int>());
  {  // inverted diagonal blocks of every B_j(z_l) factor, for the triangular solves
    h->binvoff.assign((size_t)nc * p, 0);
    int64_t bt = 0;
    for (int l = 0; l < nc; ++l)
      for (int j = 0; j < p; ++j) {
        h->binvoff[(size_t)l * p + j] = bt;
        bt += block_inverse_elems(h->d[j], NBO);
      }
    h->BLinv.alloc((size_t)bt * sizeof(Tf));
    h->BUinv.alloc((size_t)bt * sizeof(Tf));
    std::vector<SolveItem<Tf>> fi;
    std::vector<Tf *> li, ui;
    for (int l = 0; l < nc; ++l)
      for (int j = 0; j < p; ++j) {
        SolveItem<Tf> x;
        x.LU = base + h->boff[(size_t)l * p + j];
        x.piv = nullptr;
        x.n = (int)h->d[j];
        x.ld = (int)h->D[j];
        x.X = nullptr;
        x.ldx = x.ncols = 0;
        fi.push_back(x);
        li.push_back(h->BLinv.as<Tf>() + h->binvoff[(size_t)l * p + j]);
        ui.push_back(h->BUinv.as<Tf>() + h->binvoff[(size_t)l * p + j]);
      }
    lu_block_inverses<Tf>(st, fi, NBO, li, ui);
  }
  // a5: S(z) = C - z M_C + sum_j trailing_j, then LU (two levels when the subdomains are grouped)
  if (h->lv.G > 0) factor_levels<Tf>(h, base);
  else {
  h->Sfac.alloc((size_t)nc * s * s * sizeof(Tf));
  h->pivS.alloc((size_t)nc * s * sizeof(int));
  Tf *S = h->Sfac.as<Tf>();
  assemble_interface<Tf>(st, h->P, h->dd, h->z_dev.as<cx<double>>(), nc, S);
  for (int j = 0; j < p; ++j) {
    const int sj = (int)(h->sidx_off[j + 1] - h->sidx_off[j]);
    scatter_schur<Tf>(st, h->dd, j, (int)h->d[j], sj, h->sidx_off[j], h->boff_dev.as<int64_t>(), base, nc, S);
  }
  if (h->opt.keep_schur) {
    h->Skeep.alloc((size_t)nc * s * s * sizeof(Tf));
    RFDD_CUDA(cudaMemcpyAsync(h->Skeep.p, S, (size_t)nc * s * s * sizeof(Tf), cudaMemcpyDeviceToDevice, st));
  }
  std::vector<LuItem<Tf>> sit;
  for (int l = 0; l < nc; ++l) {
    LuItem<Tf> it;
    it.A = S + (int64_t)l * s * s;
    it.piv = h->pivS.as<int>() + (int64_t)l * s;
    it.dp = it.D = it.ld = (int)s;
    sit.push_back(it);
  }
  lu_batched<Tf>(st, sit, NBO_LU, h->status.as<int>());
  {
    h->sinv_elems = block_inverse_elems(s, NBO);
    h->SLinv.alloc((size_t)nc * h->sinv_elems * sizeof(Tf));
    h->SUinv.alloc((size_t)nc * h->sinv_elems * sizeof(Tf));
    std::vector<SolveItem<Tf>> fi;
    std::vector<Tf *> li, ui;
    for (int l = 0; l < nc; ++l) {
      SolveItem<Tf> x;
      x.LU = S + (int64_t)l * s * s;
      x.piv = nullptr;
      x.n = x.ld = (int)s;
      x.X = nullptr;
      x.ldx = x.ncols = 0;
      fi.push_back(x);
      li.push_back(h->SLinv.as<Tf>() + (int64_t)l * h->sinv_elems);
      ui.push_back(h->SUinv.as<Tf>() + (int64_t)l * h->sinv_elems);
    }
    lu_block_inverses<Tf>(st, fi, NBO, li, ui);
  }
  }
  if constexpr (std::is_same<Tf, cx<float>>::value) {
    if (rfdd::packed_factors(shape_of(h), h->nnodes)) {
      // the solves read only the tile copies (and the inverted diagonal blocks): one copy of each
      // factor stays
      pack_factor_operands(h);
      h->fac.release();  // stream-ordered: after the packing kernels
      h->Sfac.release();
      h->Lfac.release();
    }
  }
  // how long the host took to issue the phase, against its device time (t_factor_ms): the
  // launches are asynchronous, so the host only limits the phase if it takes as long
  h->factor_enqueue_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - host0).count();
  h->factor_launches = g_thread_launches - launches0;
  sync_status(h, "factor");
  h->have_factors = true;
}

// packed (hi, lo) pointers of one operand in h->Pk; (nullptr, nullptr) when absent
std::pair<const float *, const float *> pk_ptrs(const rfdd_handle *h, int64_t off, int64_t floats) {
  if (off < 0 || !h->Pk.p) return {nullptr, nullptr};
  const float *hi = h->Pk.as<float>() + off;
  return {hi, hi + floats};
}
template <typename Tf>
void attach_packed(const rfdd_handle *h, SolveItem<Tf> &x, const rfdd_handle::PkOff &o, int64_t n) {
  if (!h->Pk.p) return;
  const int64_t nblk = (n + NBO - 1) / NBO, bf = tc_packed_a_floats(NBO, NBO);
  std::tie(x.LUp_hi, x.LUp_lo) = pk_ptrs(h, o.lu, tc_packed_a_floats(n, n));
  std::tie(x.Linvp_hi, x.Linvp_lo) = pk_ptrs(h, o.li, nblk * bf);
  std::tie(x.Uinvp_hi, x.Uinvp_lo) = pk_ptrs(h, o.ui, nblk * bf);
}

// the inverted diagonal blocks of factor (node l, subdomain j), when present
template <typename Tf>
void attach_binv(const rfdd_handle *h, SolveItem<Tf> &x, int l, int j) {
  if (!h->BLinv.p) return;
  const int64_t o = h->binvoff[(size_t)l * h->p + j];
  x.Linv = h->BLinv.as<Tf>() + o;
  x.Uinv = h->BUinv.as<Tf>() + o;
  x.nbi = NBO;
  if (!h->pkB.empty()) attach_packed(h, x, h->pkB[(size_t)l * h->p + j], h->d[j]);
}

// Mixed solve: pack the factor operands of the later solves once (see rfdd_handle::Pk)
void pack_factor_operands(rfdd_handle *h) {
  cudaStream_t st = h->st;
  const int nc = h->nnodes, p = h->p;
  const int64_t s = h->s, bf = tc_packed_a_floats(NBO, NBO);
  h->pkB.assign((size_t)nc * p, {});
  h->pkS.assign((size_t)nc, {});
  h->pkG.assign((size_t)nc * h->lv.G, {});
  int64_t tot = 0;
  auto take = [&](int64_t floats) {
    const int64_t o = tot;
    tot += 2 * floats;
    return o;
  };
  for (int l = 0; l < nc; ++l) {
    for (int j = 0; j < p; ++j) {
      const int64_t dj = h->d[j], sj = h->D[j] - dj, nblk = (dj + NBO - 1) / NBO;
      auto &o = h->pkB[(size_t)l * p + j];
      o.lu = take(tc_packed_a_floats(dj, dj));
      o.li = take(nblk * bf);
      o.ui = take(nblk * bf);
      if (sj > 0) {
        o.l21 = take(tc_packed_a_floats(sj, dj));
        o.u12 = take(tc_packed_a_floats(dj, sj));
      }
    }
    auto &o = h->pkS[l];
    const int64_t sS = h->lv.G > 0 ? h->lv.s2 : s;  // two levels: S2' takes the place of S
    const int64_t nblk = (sS + NBO - 1) / NBO;
    if (sS > 0) {
      o.lu = take(tc_packed_a_floats(sS, sS));
      o.li = take(nblk * bf);
      o.ui = take(nblk * bf);
    }
    for (int g = 0; g < h->lv.G; ++g) {
      const int64_t n1 = h->lv.n1[g], n2 = h->lv.n2[g], nb1 = (n1 + NBO - 1) / NBO;
      auto &og = h->pkG[(size_t)l * h->lv.G + g];
      if (n1 == 0) continue;
      og.lu = take(tc_packed_a_floats(n1, n1));
      og.li = take(nb1 * bf);
      og.ui = take(nb1 * bf);
      if (n2 > 0) {
        og.l21 = take(tc_packed_a_floats(n2, n1));
        og.u12 = take(tc_packed_a_floats(n1, n2));
      }
    }
  }
  h->Pk.alloc((size_t)tot * sizeof(float));
  float *P = h->Pk.as<float>();
  std::vector<TcPackJob> jobs;
  auto job = [&](const cx<float> *A, int64_t lda, int64_t m, int64_t k, int64_t off) {
    if (off < 0 || m <= 0 || k <= 0) return;
    jobs.push_back({A, lda, m, k, P + off, P + off + tc_packed_a_floats(m, k)});
  };
  auto blocks = [&](const cx<float> *inv, int64_t n, int64_t off) {
    const int64_t nblk = (n + NBO - 1) / NBO;
    for (int64_t b = 0; b < nblk; ++b)
      jobs.push_back({inv + b * NBO * NBO, NBO, NBO, NBO, P + off + b * bf, P + off + nblk * bf + b * bf});
  };
  cx<float> *base = h->fac.as<cx<float>>();
  for (int l = 0; l < nc; ++l) {
    for (int j = 0; j < p; ++j) {
      const int64_t dj = h->d[j], Dj = h->D[j], sj = Dj - dj;
      const auto &o = h->pkB[(size_t)l * p + j];
      const cx<float> *A = base + h->boff[(size_t)l * p + j];
      job(A, Dj, dj, dj, o.lu);
      job(A + dj * Dj, Dj, sj, dj, o.l21);
      job(A + dj, Dj, dj, sj, o.u12);
      blocks(h->BLinv.as<cx<float>>() + h->binvoff[(size_t)l * p + j], dj, o.li);
      blocks(h->BUinv.as<cx<float>>() + h->binvoff[(size_t)l * p + j], dj, o.ui);
    }
    const auto &o = h->pkS[l];
    if (h->lv.G == 0) {
      job(h->Sfac.as<cx<float>>() + (int64_t)l * s * s, s, s, s, o.lu);
      blocks(h->SLinv.as<cx<float>>() + (int64_t)l * h->sinv_elems, s, o.li);
      blocks(h->SUinv.as<cx<float>>() + (int64_t)l * h->sinv_elems, s, o.ui);
      continue;
    }
    const auto &L = h->lv;
    const cx<float> *T = h->Lfac.as<cx<float>>() + (int64_t)l * L.tsz;
    const cx<float> *Li = h->LLinv.as<cx<float>>() + (int64_t)l * L.isz, *Ui = h->LUinv.as<cx<float>>() + (int64_t)l * L.isz;
    if (L.s2 > 0) {
      job(T, L.s2, L.s2, L.s2, o.lu);
      blocks(Li, L.s2, o.li);
      blocks(Ui, L.s2, o.ui);
    }
    for (int g = 0; g < L.G; ++g) {
      const int64_t n1 = L.n1[g], n2 = L.n2[g], Dg = n1 + n2;
      if (n1 == 0) continue;
      const auto &og = h->pkG[(size_t)l * L.G + g];
      const cx<float> *Bg = T + L.goff[g];
      job(Bg, Dg, n1, n1, og.lu);
      job(Bg + n1 * Dg, Dg, n2, n1, og.l21);
      job(Bg + n1, Dg, n1, n2, og.u12);
      blocks(Li + L.ioff[g], n1, og.li);
      blocks(Ui + L.ioff[g], n1, og.ui);
    }
  }
  tc_pack_a_batched(st, jobs);
}

// B_j(z_l) solves on a tall block F (n x m per node, stride fs): interior rows only
template <typename Tf>
void solve_B(rfdd_handle *h, Tf *F, int64_t ldf, int64_t fs, int64_t m, const std::vector<int> &nodes,
             int64_t row_base_shift = 0) {
  std::vector<SolveItem<Tf>> it;
  Tf *base = h->fac.as<Tf>();
  for (int l : nodes)
    for (int j = 0; j < h->p; ++j) {
      SolveItem<Tf> x;
      x.LU = base + h->boff[(size_t)l * h->p + j];
      x.piv = h->pivB.as<int>() + h->pivBoff[(size_t)l * h->p + j];
      x.n = (int)h->d[j];
      x.ld = (int)h->D[j];
      x.X = F + (int64_t)l * fs + (h->off[j] - row_base_shift) * ldf;
      x.ldx = (int)ldf;
      x.ncols = (int)m;
      attach_binv(h, x, l, j);
      it.push_back(x);
    }
  lu_solve_batched<Tf>(h->st, it, NBO);
}

template <typename Tf>
void solve_S_levels(rfdd_handle *h, Tf *G, int64_t gs, int64_t m, const std::vector<int> &nodes);

template <typename Tf>
void solve_S(rfdd_handle *h, Tf *G, int64_t ldg, int64_t gs, int64_t m, const std::vector<int> &nodes) {
  if (h->lv.G > 0) {
    RFDD_REQUIRE(ldg == m, RFDD_EINVAL, "two-level interface solve needs ldg == m");
    solve_S_levels<Tf>(h, G, gs, m, nodes);
    return;
  }
  std::vector<SolveItem<Tf>> it;
  for (int l : nodes) {
    SolveItem<Tf> x;
    x.LU = h->Sfac.as<Tf>() + (int64_t)l * h->s * h->s;
    x.piv = h->pivS.as<int>() + (int64_t)l * h->s;
    x.n = (int)h->s;
    x.ld = (int)h->s;
    x.X = G + (int64_t)l * gs;
    x.ldx = (int)ldg;
    x.ncols = (int)m;
    if (h->SLinv.p) {
      x.Linv = h->SLinv.as<Tf>() + (int64_t)l * h->sinv_elems;
      x.Uinv = h->SUinv.as<Tf>() + (int64_t)l * h->sinv_elems;
      x.nbi = NBO;
      if (!h->pkS.empty()) attach_packed(h, x, h->pkS[l], h->s);
    }
    it.push_back(x);
  }
  lu_solve_batched<Tf>(h->st, it, NBO);
}

template <typename Tf>
void border_gemm(cudaStream_t st, const std::vector<GemmItem<Tf>> &g, const std::vector<TcPackedA> &pa, double alpha,
                 double beta);

// ------------------------------------------------------------------------------------
// Two-level interface factorisation (rfdd_set_interface_groups): Eq. (inv_dd2) applied to S(z)
// with the subdomain groups as its subdomains.  Per node the level storage holds S2 (level-2
// block, s2 x s2) and, per group g, the bordered block [[S(I1_g, I1_g), S(I1_g, I2_g)],
// [S(I2_g, I1_g), 0]].  The bordered LU of each group block leaves -S21 S11^{-1} S12 in its
// trailing block; their ordered sum into S2 gives S2' = S22 - sum_g S21 S11^{-1} S12, which is
// factored densely.
// ------------------------------------------------------------------------------------
template <typename Tf>
void factor_levels(rfdd_handle *h, const Tf *base) {
  auto &L = h->lv;
  cudaStream_t st = h->st;
  const int nc = h->nnodes, p = h->p, G = L.G;
  h->Lfac.alloc((size_t)nc * L.tsz * sizeof(Tf));
  h->pivL.alloc((size_t)nc * std::max<int64_t>(L.psz, 1) * sizeof(int));
  Tf *T = h->Lfac.as<Tf>();
  RFDD_CUDA(cudaMemsetAsync(T, 0, (size_t)nc * L.tsz * sizeof(Tf), st));
  assemble_iface_levels<Tf>(st, h->P, h->if_e0, (int64_t)L.edst.size(), L.edst_dev.as<int64_t>(),
                            h->z_dev.as<cx<double>>(), nc, T, L.tsz);
  for (int j = 0; j < p; ++j) {
    const int g = L.group[j];
    const int sj = (int)(h->sidx_off[j + 1] - h->sidx_off[j]);
    scatter_schur_levels<Tf>(st, p, j, (int)h->d[j], sj, L.q_dev.as<int32_t>() + h->sidx_off[j],
                             L.r_dev.as<int32_t>() + h->sidx_off[j], L.s2, L.goff[g], L.n1[g] + L.n2[g],
                             h->boff_dev.as<int64_t>(), base, nc, T, L.tsz);
  }
  int *piv = h->pivL.as<int>();
  std::vector<LuItem<Tf>> items;
  for (int l = 0; l < nc; ++l)
    for (int g = 0; g < G; ++g) {
      if (L.n1[g] == 0) continue;
      LuItem<Tf> it;
      it.A = T + (int64_t)l * L.tsz + L.goff[g];
      it.piv = piv + (int64_t)l * L.psz + L.poff[g];
      it.dp = (int)L.n1[g];
      it.D = it.ld = (int)(L.n1[g] + L.n2[g]);
      items.push_back(it);
    }
  if (!items.empty()) lu_batched<Tf>(st, items, NBO_LU, h->status.as<int>());
  for (int g = 0; g < G; ++g)
    if (L.n1[g] > 0)
      scatter_trail_levels<Tf>(st, L.i2g_dev.as<int32_t>() + L.i2g_off[g], (int)L.n1[g], (int)L.n2[g], L.goff[g],
                               L.s2, nc, T, L.tsz);
  if (L.s2 > 0) {
    items.clear();
    for (int l = 0; l < nc; ++l) {
      LuItem<Tf> it;
      it.A = T + (int64_t)l * L.tsz;
      it.piv = piv + (int64_t)l * L.psz;
      it.dp = it.D = it.ld = (int)L.s2;
      items.push_back(it);
    }
    lu_batched<Tf>(st, items, NBO_LU, h->status.as<int>());
  }
  // inverted diagonal blocks of every level factor, for the triangular solves
  h->LLinv.alloc((size_t)nc * L.isz * sizeof(Tf));
  h->LUinv.alloc((size_t)nc * L.isz * sizeof(Tf));
  std::vector<SolveItem<Tf>> fi;
  std::vector<Tf *> li, ui;
  for (int l = 0; l < nc; ++l)
    for (int g = -1; g < G; ++g) {
      const int64_t n = g < 0 ? L.s2 : L.n1[g];
      if (n == 0) continue;
      SolveItem<Tf> x;
      x.LU = T + (int64_t)l * L.tsz + (g < 0 ? 0 : L.goff[g]);
      x.piv = nullptr;
      x.n = (int)n;
      x.ld = (int)(g < 0 ? L.s2 : L.n1[g] + L.n2[g]);
      x.X = nullptr;
      x.ldx = x.ncols = 0;
      fi.push_back(x);
      const int64_t o = (int64_t)l * L.isz + (g < 0 ? 0 : L.ioff[g]);
      li.push_back(h->LLinv.as<Tf>() + o);
      ui.push_back(h->LUinv.as<Tf>() + o);
    }
  if (!fi.empty()) lu_block_inverses<Tf>(st, fi, NBO, li, ui);
}

// factor of level block g (-1: S2) of node l as a solve item on X (ld m)
template <typename Tf>
SolveItem<Tf> level_item(const rfdd_handle *h, int l, int g, Tf *X, int64_t m) {
  const auto &L = h->lv;
  SolveItem<Tf> x;
  x.LU = h->Lfac.as<Tf>() + (int64_t)l * L.tsz + (g < 0 ? 0 : L.goff[g]);
  x.piv = h->pivL.as<int>() + (int64_t)l * L.psz + (g < 0 ? 0 : L.poff[g]);
  x.n = (int)(g < 0 ? L.s2 : L.n1[g]);
  x.ld = (int)(g < 0 ? L.s2 : L.n1[g] + L.n2[g]);
  x.X = X;
  x.ldx = (int)m;
  x.ncols = (int)m;
  if (h->LLinv.p) {
    const int64_t o = (int64_t)l * L.isz + (g < 0 ? 0 : L.ioff[g]);
    x.Linv = h->LLinv.as<Tf>() + o;
    x.Uinv = h->LUinv.as<Tf>() + o;
    x.nbi = NBO;
    if (g < 0 && !h->pkS.empty()) attach_packed(h, x, h->pkS[l], L.s2);
    if (g >= 0 && !h->pkG.empty()) attach_packed(h, x, h->pkG[(size_t)l * L.G + g], L.n1[g]);
  }
  return x;
}

// Y = S(z_l)^{-1} Y through the level factors: with the rows in level order (u),
//   w_g = L11_g^{-1} P_g u[I1_g];  u[I2] -= sum_g scatter(L21_g w_g);  u[I2] = S2'^{-1} u[I2];
//   w_g -= U12_g u[I2_g];  u[I1_g] = U11_g^{-1} w_g.
// G rows are interface-ordered, ld m; node list position i reads G + i * gs.
template <typename Tf>
void solve_S_levels_run(rfdd_handle *h, Tf *G, int64_t gs, int64_t m, const std::vector<int> &nl) {
  const auto &L = h->lv;
  cudaStream_t st = h->st;
  const int64_t s = h->s, s1 = L.s1;
  const int nn = (int)nl.size(), NG = L.G;
  int64_t n2max = 1;
  for (int g = 0; g < NG; ++g) n2max = std::max(n2max, L.n2[g]);
  const int64_t us = s * m, hs = (int64_t)NG * n2max * m;
  Buf U, Ht;
  U.alloc((size_t)nn * us * sizeof(Tf));
  Ht.alloc((size_t)nn * hs * sizeof(Tf));
  Tf *u = U.as<Tf>(), *ht = Ht.as<Tf>();
  gather_iface<Tf>(st, L.lorder_dev.as<int32_t>(), (int)s, m, G, gs, u, us, nn);
  std::vector<SolveItem<Tf>> it;
  for (int i = 0; i < nn; ++i)
    for (int g = 0; g < NG; ++g)
      if (L.n1[g] > 0) it.push_back(level_item<Tf>(h, nl[i], g, u + i * us + L.g1off[g] * m, m));
  if (!it.empty()) {
    apply_pivots<Tf>(st, it);
    trsm_lower_unit<Tf>(st, it, NBO);
  }
  auto border = [&](bool lower) {
    std::vector<GemmItem<Tf>> gi;
    std::vector<TcPackedA> pa;
    for (int i = 0; i < nn; ++i)
      for (int g = 0; g < NG; ++g) {
        const int64_t n1 = L.n1[g], n2 = L.n2[g], Dg = n1 + n2;
        if (n1 == 0 || n2 == 0) continue;
        const Tf *blk = h->Lfac.as<Tf>() + (int64_t)nl[i] * L.tsz + L.goff[g];
        Tf *w = u + i * us + L.g1off[g] * m, *hh = ht + i * hs + (int64_t)g * n2max * m;
        const auto *pk = h->pkG.empty() ? nullptr : &h->pkG[(size_t)nl[i] * NG + g];
        if (lower) {
          gi.push_back({blk + n1 * Dg, w, hh, (int)n2, (int)m, (int)n1, (int)Dg, (int)m, (int)m});
          const auto pp = pk ? pk_ptrs(h, pk->l21, tc_packed_a_floats(n2, n1))
                             : std::pair<const float *, const float *>{nullptr, nullptr};
          pa.push_back(TcPackedA{pp.first, pp.second, tc_packed_a_ktiles(n1)});
        } else {
          gi.push_back({blk + n1, hh, w, (int)n1, (int)m, (int)n2, (int)Dg, (int)m, (int)m});
          const auto pp = pk ? pk_ptrs(h, pk->u12, tc_packed_a_floats(n1, n2))
                             : std::pair<const float *, const float *>{nullptr, nullptr};
          pa.push_back(TcPackedA{pp.first, pp.second, tc_packed_a_ktiles(n2)});
        }
      }
    if (!gi.empty()) border_gemm<Tf>(st, gi, pa, lower ? 1.0 : -1.0, lower ? 0.0 : 1.0);
  };
  border(true);
  for (int g = 0; g < NG; ++g)
    if (L.n1[g] > 0 && L.n2[g] > 0)
      scatter_sub_iface<Tf>(st, L.i2g_dev.as<int32_t>() + L.i2g_off[g], (int)L.n2[g], m, ht + (int64_t)g * n2max * m,
                            hs, u + s1 * m, us, nn);
  if (L.s2 > 0) {
    std::vector<SolveItem<Tf>> si;
    for (int i = 0; i < nn; ++i) si.push_back(level_item<Tf>(h, nl[i], -1, u + i * us + s1 * m, m));
    lu_solve_batched<Tf>(st, si, NBO);
  }
  for (int g = 0; g < NG; ++g)
    if (L.n1[g] > 0 && L.n2[g] > 0)
      gather_iface<Tf>(st, L.i2g_dev.as<int32_t>() + L.i2g_off[g], (int)L.n2[g], m, u + s1 * m, us,
                       ht + (int64_t)g * n2max * m, hs, nn);
  border(false);
  if (!it.empty()) trsm_upper<Tf>(st, it, NBO);
  gather_iface<Tf>(st, L.lpos_dev.as<int32_t>(), (int)s, m, u, us, G, gs, nn);
}

template <typename Tf>
void solve_S_levels(rfdd_handle *h, Tf *G, int64_t gs, int64_t m, const std::vector<int> &nodes) {
  bool all = (int)nodes.size() == h->nnodes;
  for (size_t i = 0; i < nodes.size() && all; ++i) all = nodes[i] == (int)i;
  if (all) {
    solve_S_levels_run<Tf>(h, G, gs, m, nodes);
    return;
  }
  for (int l : nodes) solve_S_levels_run<Tf>(h, G + (int64_t)l * gs, 0, m, std::vector<int>{l});
}

// Products on the eigenvector bases (Lanczos blocks, interior CholQR, Rayleigh-Ritz Gram
// matrices, Ritz-vector updates): double-FP32 arithmetic in the mixed-precision solve, FP64 in
// the plain FP64 solve.
void basis_gemm_on(const rfdd_handle *h, cudaStream_t st, const std::vector<GemmItem<double>> &g, bool ta, bool tb,
                   double alpha, double beta, const std::vector<char> &sym = {}) {
  if (h->opt.precision == RFDD_FP64 || h->basis_fp64) gemm_simt_batched<double>(st, g, ta, tb, alpha, beta, sym);
  else gemm_f64x2_batched(st, g, ta, tb, alpha, beta, sym);
}
void basis_gemm(const rfdd_handle *h, const std::vector<GemmItem<double>> &g, bool ta, bool tb, double alpha,
                double beta, const std::vector<char> &sym = {}) {
  basis_gemm_on(h, h->st, g, ta, tb, alpha, beta, sym);
}

std::vector<int> all_nodes(const rfdd_handle *h) {
  std::vector<int> v(h->nnodes);
  std::iota(v.begin(), v.end(), 0);
  return v;
}

// a6: W = scale * Re sum_l w_l S_l^{-1} X  (X, W: s x b FP64 device)
template <typename Tf>
void filter_impl(rfdd_handle *h, const double *X, double *W, int64_t b, double scale) {
  const int64_t s = h->s;
  const int nc = h->nnodes;
  Buf rhs;
  rhs.alloc((size_t)nc * s * b * sizeof(Tf));
  real_to_complex<Tf>(h->st, X, rhs.as<Tf>(), s * b, nc, s * b);
  solve_S<Tf>(h, rhs.as<Tf>(), b, s * b, b, all_nodes(h));
  weighted_real_sum<Tf>(h->st, rhs.as<Tf>(), s * b, h->w_dev.as<cx<double>>(), nc, scale, W, s * b);
}

// a border product of the DD solve, with the packed border block when there is one
template <typename Tf>
void border_gemm(cudaStream_t st, const std::vector<GemmItem<Tf>> &g, const std::vector<TcPackedA> &pa, double alpha,
                 double beta) {
  if constexpr (std::is_same<Tf, cx<float>>::value) {
    tc_gemm_complex_pa(st, g, pa, alpha, beta);
    return;
  }
  gemm_batched<Tf>(st, g, false, false, alpha, beta);
}

// DD resolvent (Eq. inv_dd2) in the factor precision for all nodes:
// X_l = (A - z_l M)^{-1} R_l,  R, X: complex FP64, n x m per node (stride n*m).
// The bordered factorisation P[B_j E_j] = L[U U12], [E_j^T 0] = L21[U U12] + [0 T_j] holds the
// block LU of (A - z M) restricted to subdomain j, so with w_j = L^{-1} P f_j:
//   S y = g - sum_j L21_j w_j,     u_j = U^{-1} (w_j - U12_j y[sidx_j]),
// one forward and one backward triangular solve per block plus two border products.
// R_l = R + l * strideR (strideR = 0: one right-hand side shared by all nodes).
template <typename Tf>
void dd_solve(rfdd_handle *h, const cx<double> *R, int64_t strideR, cx<double> *X, int64_t m, Buf &F, Buf &Ht) {
  cudaStream_t st = h->st;
  const int nc = h->nnodes, p = h->p;
  const int64_t n = h->n, dsum = h->dsum;
  const int64_t fs = n * m;
  int64_t smax = 1;
  for (int j = 0; j < p; ++j) smax = std::max<int64_t>(smax, h->sidx_off[j + 1] - h->sidx_off[j]);
  F.ensure((size_t)nc * fs * sizeof(Tf));
  Ht.ensure((size_t)nc * p * smax * m * sizeof(Tf));
  Tf *f = F.as<Tf>(), *ht = Ht.as<Tf>();
  Tf *base = h->fac.as<Tf>();
  const int64_t hs = (int64_t)p * smax * m;  // per-node stride of the border scratch
  Lap lap(st, "dd");
  for (int l = 0; l < nc; ++l) convert<Tf, cx<double>>(st, R + l * strideR, f + l * fs, fs);
  // w = L^{-1} P f for every (node, subdomain)
  {
    std::vector<SolveItem<Tf>> it;
    for (int l = 0; l < nc; ++l)
      for (int j = 0; j < p; ++j) {
        SolveItem<Tf> x;
        x.LU = base + h->boff[(size_t)l * p + j];
        x.piv = h->pivB.as<int>() + h->pivBoff[(size_t)l * p + j];
        x.n = (int)h->d[j];
        x.ld = (int)h->D[j];
        x.X = f + (int64_t)l * fs + h->off[j] * m;
        x.ldx = (int)m;
        x.ncols = (int)m;
        attach_binv(h, x, l, j);
        it.push_back(x);
      }
    apply_pivots<Tf>(st, it);
    trsm_lower_unit<Tf>(st, it, NBO);
  }
  lap.mark("forward");
  // g -= sum_j L21_j w_j  (s_j x d_j times d_j x m, then an ordered scatter)
  {
    std::vector<GemmItem<Tf>> g;
    std::vector<TcPackedA> pa;
    for (int l = 0; l < nc; ++l)
      for (int j = 0; j < p; ++j) {
        const int sj = (int)(h->sidx_off[j + 1] - h->sidx_off[j]);
        if (sj == 0) continue;
        const int64_t Dj = h->D[j], dj = h->d[j];
        g.push_back({base + h->boff[(size_t)l * p + j] + dj * Dj, f + (int64_t)l * fs + h->off[j] * m,
                     ht + l * hs + (int64_t)j * smax * m, sj, (int)m, (int)dj, (int)Dj, (int)m, (int)m});
        const auto pp = h->pkB.empty() ? std::pair<const float *, const float *>{nullptr, nullptr}
                                       : pk_ptrs(h, h->pkB[(size_t)l * p + j].l21, tc_packed_a_floats(sj, dj));
        pa.push_back(TcPackedA{pp.first, pp.second, tc_packed_a_ktiles(dj)});
      }
    border_gemm<Tf>(st, g, pa, 1.0, 0.0);
    for (int j = 0; j < p; ++j) {
      const int sj = (int)(h->sidx_off[j + 1] - h->sidx_off[j]);
      scatter_sub_iface<Tf>(st, h->dd.sidx + h->sidx_off[j], sj, m, ht + (int64_t)j * smax * m, hs, f + dsum * m, fs,
                            nc);
    }
  }
  lap.mark("border L21");
  solve_S<Tf>(h, f + dsum * m, m, fs, m, all_nodes(h));  // y = S^{-1} g'
  lap.mark("S solve");
  // w_j -= U12_j y[sidx_j], then u_j = U^{-1} w_j
  {
    for (int j = 0; j < p; ++j) {
      const int sj = (int)(h->sidx_off[j + 1] - h->sidx_off[j]);
      gather_iface<Tf>(st, h->dd.sidx + h->sidx_off[j], sj, m, f + dsum * m, fs, ht + (int64_t)j * smax * m, hs, nc);
    }
    std::vector<GemmItem<Tf>> g;
    std::vector<TcPackedA> pa;
    std::vector<SolveItem<Tf>> it;
    for (int l = 0; l < nc; ++l)
      for (int j = 0; j < p; ++j) {
        const int sj = (int)(h->sidx_off[j + 1] - h->sidx_off[j]);
        const int64_t Dj = h->D[j], dj = h->d[j];
        if (sj > 0) {
          g.push_back({base + h->boff[(size_t)l * p + j] + dj, ht + l * hs + (int64_t)j * smax * m,
                       f + (int64_t)l * fs + h->off[j] * m, (int)dj, (int)m, sj, (int)Dj, (int)m, (int)m});
          const auto pp = h->pkB.empty() ? std::pair<const float *, const float *>{nullptr, nullptr}
                                         : pk_ptrs(h, h->pkB[(size_t)l * p + j].u12, tc_packed_a_floats(dj, sj));
          pa.push_back(TcPackedA{pp.first, pp.second, tc_packed_a_ktiles(sj)});
        }
        SolveItem<Tf> x;
        x.LU = base + h->boff[(size_t)l * p + j];
        x.piv = nullptr;
        x.n = (int)dj;
        x.ld = (int)Dj;
        x.X = f + (int64_t)l * fs + h->off[j] * m;
        x.ldx = (int)m;
        x.ncols = (int)m;
        attach_binv(h, x, l, j);
        it.push_back(x);
      }
    border_gemm<Tf>(st, g, pa, -1.0, 1.0);
    lap.mark("border U12");
    trsm_upper<Tf>(st, it, NBO);
  }
  lap.mark("backward");
  convert<cx<double>, Tf>(st, f, X, nc * fs);
}

// Shifted solves with FP64 iterative refinement (Section 3.1 block inverse as the approximate
// solver, FP64 sparse residuals): X_l = (A - z_l M)^{-1} V for all nodes; V real (n x m).
// Refinement stops once every shifted residual satisfies
//   ||r|| <= tol * (||A|| + |z| ||M||) ||x||   (tol >= 1e-14), or after ir_max steps.
template <typename Tf>
int refined_solve(rfdd_handle *h, const double *V, cx<double> *X, int64_t m, double tol, bool fp64_residual = false) {
  cudaStream_t st = h->st;
  const int nc = h->nnodes;
  const int64_t n = h->n;
  Buf Vc, Rr, Dx, F, Ht, nr, nx;
  Vc.alloc((size_t)n * m * sizeof(cx<double>));
  real_to_complex<cx<double>>(st, V, Vc.as<cx<double>>(), n * m, 1, 0);
  dd_solve<Tf>(h, Vc.as<cx<double>>(), 0, X, m, F, Ht);
  const int irmax = std::is_same<Tf, cx<double>>::value ? std::min(1, h->opt.ir_max) : h->opt.ir_max;
  Rr.alloc((size_t)nc * n * m * sizeof(cx<double>));
  Dx.alloc((size_t)nc * n * m * sizeof(cx<double>));
  nr.alloc((size_t)nc * m * sizeof(double));
  nx.alloc((size_t)nc * m * sizeof(double));
  std::vector<double> hr(nc * m), hx(nc * m);
  int steps = 0;
  Buf Xs;
  // mixed solve: double-FP32 residual products unless the caller needs FP64 ones
  const bool df = std::is_same<Tf, cx<float>>::value && !fp64_residual;
  if (df) Xs.alloc((size_t)nc * n * m * sizeof(float4));
  for (int it = 0; it <= irmax; ++it) {
    if (df) {
      split_c64(st, X, Xs.as<float4>(), (int64_t)nc * n * m);
      shifted_residual_df(st, h->P, h->z_dev.as<cx<double>>(), nc, Vc.as<cx<double>>(), 0, Xs.as<float4>(),
                          Rr.as<cx<double>>(), n * m, m);
    } else {
      shifted_residual(st, h->P, h->z_dev.as<cx<double>>(), nc, Vc.as<cx<double>>(), 0, X, Rr.as<cx<double>>(),
                       n * m, m);
    }
    col_norms2_c64(st, Rr.as<cx<double>>(), n, m, nc, n * m, nr.as<double>());
    col_norms2_c64(st, X, n, m, nc, n * m, nx.as<double>());
    RFDD_CUDA(cudaMemcpyAsync(hr.data(), nr.p, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    RFDD_CUDA(cudaMemcpyAsync(hx.data(), nx.p, hx.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    RFDD_CUDA(cudaStreamSynchronize(st));
    bool ok = true;
    for (int l = 0; l < nc && ok; ++l) {
      const double zn = std::sqrt(h->z[l].re * h->z[l].re + h->z[l].im * h->z[l].im);
      const double scale = (h->normA + zn * h->normM);
      for (int64_t c = 0; c < m; ++c)
        if (std::sqrt(hr[l * m + c]) > tol * scale * std::sqrt(hx[l * m + c]) + 1e-300) { ok = false; break; }
    }
    if (log_on()) {
      double worst = 0.0;
      for (int l = 0; l < nc; ++l) {
        const double zn = std::sqrt(h->z[l].re * h->z[l].re + h->z[l].im * h->z[l].im);
        for (int64_t c = 0; c < m; ++c)
          worst = std::max(worst, std::sqrt(hr[l * m + c]) / ((h->normA + zn * h->normM) *
                                                               std::sqrt(hx[l * m + c]) + 1e-300));
      }
      RFDD_LOGF("  refinement step %d: worst scaled residual %.3e", it, worst);
    }
    if (ok || it == irmax) break;
    dd_solve<Tf>(h, Rr.as<cx<double>>(), n * m, Dx.as<cx<double>>(), m, F, Ht);
    axpy_c64(st, Dx.as<cx<double>>(), X, (int64_t)nc * n * m);
    ++steps;
  }
  return steps;
}

// ------------------------------------------------------------------------------------
// M-orthonormal Rayleigh-Ritz on range(Y) for a tall FP64 block Y (n x k, row-major):
// Gram G = Y^T M Y and K = Y^T A Y, unit-diagonal scaling D, pivoted Cholesky
// P^T (D G D) P = R^T R that drops directions whose pivot falls below `drop` (Y's columns may
// be linearly dependent), projected H = R^{-T} P^T (D K D) P R^{-1}, and its eigenpairs.
// Returns all Ritz values (ascending) and, for the selected sorted indices, the coefficient block
// C (k x nsel) such that the Ritz vectors are Y C.
// ------------------------------------------------------------------------------------
struct RRout {
  std::vector<double> theta;  // all Ritz values (ascending)
  int64_t r = 0;              // dimension kept
};

// vstruct: the leading kappa columns of Y are blockdiag(V_j) (subdomain j's rows only, columns
// voff[j]..voff[j+1]); their Gram blocks are then formed per subdomain (exactly zero between
// different subdomains), and only the remaining columns need full-length products.
RRout rayleigh_ritz_coeffs(rfdd_handle *h, const double *Y, int64_t k, double drop, double ctol,
                           const std::function<std::vector<int>(const std::vector<double> &)> &select,
                           Buf &Cout, std::vector<int> &sel_out, bool vstruct = false) {
  auto gram = [&](const std::vector<GemmItem<double>> &g, const std::vector<char> &sym) {
    basis_gemm(h, g, true, false, 1.0, 0.0, sym);
  };
  cudaStream_t st = h->st;
  const int64_t n = h->n;
  Lap lap(st, "rr");
  Buf MY, AY, G, K;
  MY.alloc((size_t)n * k * sizeof(double));
  AY.alloc((size_t)n * k * sizeof(double));
  if (is_mixed(h) && !h->basis_fp64) {  // the basis products' precision (basis_gemm)
    spmm_am_df(st, h->P, Y, AY.as<double>(), MY.as<double>(), k);
  } else {
    spmm_f64(st, h->P, 0, n, 0, n, 0.0, 1.0, Y, k, MY.as<double>(), k, k, false);
    spmm_f64(st, h->P, 0, n, 0, n, 1.0, 0.0, Y, k, AY.as<double>(), k, k, false);
  }
  lap.mark("spmm");
  G.alloc((size_t)k * k * sizeof(double));
  K.alloc((size_t)k * k * sizeof(double));
  const int64_t kap = vstruct ? h->kappa : 0;
  if (kap > 0) {
    const int64_t ks = k - kap;
    RFDD_CUDA(cudaMemsetAsync(G.p, 0, (size_t)k * k * sizeof(double), st));
    RFDD_CUDA(cudaMemsetAsync(K.p, 0, (size_t)k * k * sizeof(double), st));
    std::vector<GemmItem<double>> g;
    std::vector<char> sym;
    for (int q = 0; q < 2; ++q) {  // q = 0: M (Gram), q = 1: A
      const double *PY = q == 0 ? MY.as<double>() : AY.as<double>();
      double *Out = q == 0 ? G.as<double>() : K.as<double>();
      if (ks > 0) {  // S^T (P S)
        g.push_back({Y + kap, PY + kap, Out + kap * k + kap, (int)ks, (int)ks, (int)n, (int)k, (int)k, (int)k});
        sym.push_back(1);
      }
      for (int j = 0; j < h->p; ++j) {
        const int64_t v0 = h->voff[j], nv = h->voff[j + 1] - h->voff[j];
        if (nv <= 0) continue;
        const int64_t r0 = h->off[j], dj = h->d[j];
        // V_j^T (P V_j) and V_j^T (P S) over subdomain j's rows
        g.push_back({Y + r0 * k + v0, PY + r0 * k + v0, Out + v0 * k + v0, (int)nv, (int)nv, (int)dj, (int)k, (int)k,
                     (int)k});
        sym.push_back(1);
        if (ks > 0) {
          g.push_back({Y + r0 * k + v0, PY + r0 * k + kap, Out + v0 * k + kap, (int)nv, (int)ks, (int)dj, (int)k,
                       (int)k, (int)k});
          sym.push_back(0);
        }
      }
    }
    gram(g, sym);
    if (ks > 0) {
      mirror_block(st, G.as<double>(), k, 0, kap, kap, k);  // (S, V) blocks from (V, S)
      mirror_block(st, K.as<double>(), k, 0, kap, kap, k);
    }
  } else {
    std::vector<GemmItem<double>> g = {
        {Y, MY.as<double>(), G.as<double>(), (int)k, (int)k, (int)n, (int)k, (int)k, (int)k},
        {Y, AY.as<double>(), K.as<double>(), (int)k, (int)k, (int)n, (int)k, (int)k, (int)k}};
    gram(g, {1, 1});
  }
  MY.release();
  AY.release();
  lap.mark("gram");
  Buf dsc, perm, rankd;
  dsc.alloc((size_t)k * sizeof(double));
  perm.alloc((size_t)k * sizeof(int));
  rankd.alloc(sizeof(int));
  inv_sqrt_diag(st, G.as<double>(), k, dsc.as<double>());
  scale_sym(st, G.as<double>(), k, dsc.as<double>());
  scale_sym(st, K.as<double>(), k, dsc.as<double>());
  const int r = pivoted_cholesky(st, G.as<double>(), (int)k, perm.as<int>(), drop, rankd.as<int>());
  lap.mark("pivoted cholesky");
  RFDD_REQUIRE(r > 0, RFDD_ESINGULAR, "Rayleigh-Ritz: basis has no independent direction");
  // H = R^{-T} Kp R^{-1}: with Lt = (D_R^{-1} R^T) unit lower, R^{-T} B = Lt^{-1} D_R^{-1} B
  Buf Kp, Lt, B, H;
  Kp.alloc((size_t)r * r * sizeof(double));
  Lt.alloc((size_t)r * r * sizeof(double));
  B.alloc((size_t)r * r * sizeof(double));
  H.alloc((size_t)r * r * sizeof(double));
  gather_sym(st, K.as<double>(), (int)k, perm.as<int>(), r, Kp.as<double>());
  unit_lower_from_upper(st, G.as<double>(), (int)k, r, Lt.as<double>());
  scale_rows_by_rdiag(st, Kp.as<double>(), r, false, G.as<double>(), (int)k, B.as<double>());
  SolveItem<double> tri;
  tri.LU = Lt.as<double>();
  tri.piv = nullptr;
  tri.n = r;
  tri.ld = r;
  tri.X = B.as<double>();
  tri.ldx = r;
  tri.ncols = r;
  trsm_lower_unit<double>(st, {tri}, 128);                                   // B = R^{-T} Kp
  scale_rows_by_rdiag(st, B.as<double>(), r, true, G.as<double>(), (int)k, Kp.as<double>());
  tri.X = Kp.as<double>();
  trsm_lower_unit<double>(st, {tri}, 128);                                   // Kp = R^{-T} B^T = H^T
  symmetrize(st, Kp.as<double>(), r, H.as<double>());
  K.release();
  Kp.release();
  B.release();
  lap.mark("projected H");
  Buf hd, he, ht, hw, hl, hZ;
  hd.alloc(r * sizeof(double));
  he.alloc(r * sizeof(double));
  ht.alloc(r * sizeof(double));
  hw.alloc(r * sizeof(double));
  hl.alloc(r * sizeof(double));
  SymItem hi{H.as<double>(), r, r, hd.as<double>(), he.as<double>(), ht.as<double>(), hw.as<double>(), hl.as<double>(),
             nullptr};
  sym_eig_values(st, {hi}, h->status.as<int>());
  RRout out;
  out.r = r;
  out.theta.resize(r);
  RFDD_CUDA(cudaMemcpyAsync(out.theta.data(), hl.p, r * sizeof(double), cudaMemcpyDeviceToHost, st));
  RFDD_CUDA(cudaStreamSynchronize(st));
  lap.mark("H eigenvalues");
  sel_out = select(out.theta);
  const int64_t ns = (int64_t)sel_out.size();
  if (ns > 0) {
    Buf Yt, Ct;
    hZ.alloc((size_t)ns * r * sizeof(double));
    hi.Zt = hZ.as<double>();
    Yt.alloc((size_t)ns * r * sizeof(double));
    BackItem bi{&hi, sel_out, Yt.as<double>(), r};
    sym_eig_vectors(st, {bi}, ctol);
    // C_r = R^{-1} Y_sel^T (r x ns), then rows back to the original column order with D
    Ct.alloc((size_t)r * ns * sizeof(double));
    transpose(st, Yt.as<double>(), (int)ns, r, Ct.as<double>());
    SolveItem<double> up;
    up.LU = G.as<double>();
    up.piv = nullptr;
    up.n = r;
    up.ld = (int)k;
    up.X = Ct.as<double>();
    up.ldx = (int)ns;
    up.ncols = (int)ns;
    trsm_upper<double>(st, {up}, 128);
    Cout.alloc((size_t)k * ns * sizeof(double));
    RFDD_CUDA(cudaMemsetAsync(Cout.p, 0, (size_t)k * ns * sizeof(double), st));
    scatter_rows_perm(st, Ct.as<double>(), r, (int)ns, perm.as<int>(), dsc.as<double>(), Cout.as<double>());
  }
  lap.mark("eigenvectors + coefficients");
  sync_status(h, "rayleigh-ritz");
  return out;
}

// Ritz values (sorted) -> the m indices nearest [alpha, beta] (distance 0 inside), sorted
std::vector<int> select_nearest(const std::vector<double> &th, double a, double b, int64_t m) {
  std::vector<int> idx(th.size());
  std::iota(idx.begin(), idx.end(), 0);
  const double c = 0.5 * (a + b);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
    const double dx = std::max(std::max(a - th[x], th[x] - b), 0.0);
    const double dy = std::max(std::max(a - th[y], th[y] - b), 0.0);
    if (dx != dy) return dx < dy;
    return std::fabs(th[x] - c) < std::fabs(th[y] - c);
  });
  if ((int64_t)idx.size() > m) idx.resize(m);
  std::sort(idx.begin(), idx.end());
  return idx;
}

// ------------------------------------------------------------------------------------
// a7: block Lanczos on F (Alg. 2) with CGS2 against all previous blocks
// ------------------------------------------------------------------------------------
template <typename Tf>
void lanczos_impl(rfdd_handle *h) {
  cudaStream_t st = h->st;
  const int64_t s = h->s;
  const int64_t b = std::max<int64_t>(1, std::min<int64_t>(h->opt.block, s));
  const int64_t qld = s;  // mu <= s columns
  h->qcap = qld;
  h->Q.alloc((size_t)s * qld * sizeof(double));
  double *Q = h->Q.as<double>();
  RFDD_CUDA(cudaMemsetAsync(Q, 0, (size_t)s * qld * sizeof(double), st));
  Buf W, Wraw, Xb, Cb, Gb, Rinv, dead, Bprev, Amu, tmp;
  W.alloc((size_t)s * b * sizeof(double));
  Wraw.alloc((size_t)s * b * sizeof(double));
  Xb.alloc((size_t)s * b * sizeof(double));
  Cb.alloc((size_t)qld * b * sizeof(double));
  Gb.alloc((size_t)b * b * sizeof(double));
  Rinv.alloc((size_t)b * b * sizeof(double));
  dead.alloc((size_t)b * sizeof(int));
  Bprev.alloc((size_t)b * b * sizeof(double));
  Amu.alloc((size_t)b * b * sizeof(double));
  tmp.alloc((size_t)s * b * sizeof(double));
  std::vector<int> hdead(b);
  uint64_t stream_id = 0;
  auto project_out = [&](double *Wp, int64_t bw, int64_t ncols_prev) {  // W -= Q (Q^T W)
    if (ncols_prev <= 0) return;
    basis_gemm(h, {{Q, Wp, Cb.as<double>(), (int)ncols_prev, (int)bw, (int)s, (int)qld, (int)bw, (int)bw}},
                         true, false, 1.0, 0.0);
    basis_gemm(h, {{Q, Cb.as<double>(), Wp, (int)s, (int)bw, (int)ncols_prev, (int)qld, (int)bw, (int)bw}},
                         false, false, -1.0, 1.0);
  };
  // Lines 4-12 of Alg. 2 for a block of bw columns (row stride bw): two classical Gram-Schmidt
  // passes against Q[:, 0:ncols_prev], Cholesky-QR, one more projection and Cholesky-QR; columns
  // that vanish (breakdown, line 8) are replaced by fresh random vectors (line 9).
  auto orthonormalize = [&](double *Wp, int64_t bw, int64_t ncols_prev) {
    for (int attempt = 0; attempt < 4; ++attempt) {
      project_out(Wp, bw, ncols_prev);
      project_out(Wp, bw, ncols_prev);
      bool any_dead = false;
      for (int q = 0; q < 2; ++q) {
        basis_gemm(h, {{Wp, Wp, Gb.as<double>(), (int)bw, (int)bw, (int)s, (int)bw, (int)bw, (int)bw}}, true,
                           false, 1.0, 0.0, {1});
        chol_inv_batched(st, {CholItem{Gb.as<double>(), Rinv.as<double>(), dead.as<int>(), (int)bw}}, 1e-24);
        basis_gemm(h, {{Wp, Rinv.as<double>(), tmp.as<double>(), (int)s, (int)bw, (int)bw, (int)bw, (int)bw,
                                   (int)bw}},
                             false, false, 1.0, 0.0);
        RFDD_CUDA(cudaMemcpyAsync(Wp, tmp.p, (size_t)s * bw * sizeof(double), cudaMemcpyDeviceToDevice, st));
        RFDD_CUDA(cudaMemcpyAsync(hdead.data(), dead.p, bw * sizeof(int), cudaMemcpyDeviceToHost, st));
        RFDD_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < bw; ++c) any_dead |= hdead[c] != 0;
        if (any_dead) break;
        if (q == 0) project_out(Wp, bw, ncols_prev);  // "twice is enough" after normalisation
      }
      if (!any_dead) return;
      Buf fresh;
      fresh.alloc((size_t)s * bw * sizeof(double));
      counter_uniform_dev(st, h->opt.seed, 1000 + (++stream_id), fresh.as<double>(), s * bw);
      std::vector<double> hw((size_t)s * bw), hf((size_t)s * bw);
      RFDD_CUDA(cudaMemcpyAsync(hw.data(), Wp, hw.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      RFDD_CUDA(cudaMemcpyAsync(hf.data(), fresh.p, hf.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      RFDD_CUDA(cudaStreamSynchronize(st));
      for (int64_t i = 0; i < s; ++i)
        for (int c = 0; c < bw; ++c)
          if (hdead[c]) hw[i * bw + c] = hf[i * bw + c];
      RFDD_CUDA(cudaMemcpyAsync(Wp, hw.data(), hw.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    throw Error(RFDD_ESINGULAR, "lanczos: could not extend the basis");
  };
  // line 0: start block
  int64_t bc = b, bprev = 0, col = 0;  // current block width, previous width, first column
  counter_uniform_dev(st, h->opt.seed, 0, W.as<double>(), s * bc);
  orthonormalize(W.as<double>(), bc, 0);
  copy_rows_f64(st, W.as<double>(), bc, Q, qld, s, bc);
  h->traces.clear();
  double trace = 0.0, last_check = 0.0;
  const int check_every = (int)std::max<int64_t>(1, (10 + b - 1) / b);
  int64_t nblk = 0;
  std::vector<double> ha(b * b);
  while (true) {
    double *Qmu = Q + col;
    copy_rows_f64(st, Qmu, qld, Xb.as<double>(), bc, s, bc);
    Lap lap(st, "lanczos");
    filter_impl<Tf>(h, Xb.as<double>(), W.as<double>(), bc, 1.0);  // line 2: F q
    lap.mark("filter");
    if (nblk > 0)  // ... - Q_{mu-1} B_mu^T
      basis_gemm(h, {{Q + col - bprev, Bprev.as<double>(), W.as<double>(), (int)s, (int)bc, (int)bprev,
                                 (int)qld, (int)bprev, (int)bc}},
                           false, true, -1.0, 1.0);
    // line 3: A_mu = Q_mu^T W
    basis_gemm(h, {{Xb.as<double>(), W.as<double>(), Amu.as<double>(), (int)bc, (int)bc, (int)s, (int)bc,
                               (int)bc, (int)bc}},
                         true, false, 1.0, 0.0);
    RFDD_CUDA(cudaMemcpyAsync(ha.data(), Amu.p, bc * bc * sizeof(double), cudaMemcpyDeviceToHost, st));
    RFDD_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < bc; ++c) trace += ha[c * bc + c];
    h->traces.push_back(trace);
    ++nblk;
    const int64_t mu_now = col + bc;
    if (mu_now >= s) break;  // the space is exhausted (mu = s)
    if (nblk % check_every == 0) {  // line 13
      if (std::fabs(trace - last_check) <= h->opt.lanczos_tol * std::fabs(trace)) break;
      last_check = trace;
    }
    // lines 4-12 for the next block (width bn), B_{mu+1} = Q_{mu+1}^T W
    const int64_t bn = std::min<int64_t>(b, s - mu_now);
    if (bn < bc)  // keep the leading bn columns of W (row stride bc -> bn)
      copy_rows_f64(st, W.as<double>(), bc, tmp.as<double>(), bn, s, bn);
    else
      RFDD_CUDA(cudaMemcpyAsync(tmp.p, W.p, (size_t)s * bc * sizeof(double), cudaMemcpyDeviceToDevice, st));
    RFDD_CUDA(cudaMemcpyAsync(Wraw.p, W.p, (size_t)s * bc * sizeof(double), cudaMemcpyDeviceToDevice, st));
    RFDD_CUDA(cudaMemcpyAsync(W.p, tmp.p, (size_t)s * bn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    orthonormalize(W.as<double>(), bn, mu_now);
    lap.mark("orthonormalize");
    // B (bn x bc) = Q_next^T W_raw
    basis_gemm(h, {{W.as<double>(), Wraw.as<double>(), Bprev.as<double>(), (int)bn, (int)bc, (int)s, (int)bn,
                               (int)bc, (int)bc}},
                         true, false, 1.0, 0.0);
    copy_rows_f64(st, W.as<double>(), bn, Q + mu_now, qld, s, bn);
    bprev = bc;
    col = mu_now;
    bc = bn;
  }
  h->mu = col + bc;
  RFDD_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------------------------
// a8: interior basis and Z (Eq. trabala, trabala2, z)
// ------------------------------------------------------------------------------------
// Waits for an interior factorisation started on the second stream: joins the host thread that
// launched it and orders the handle's stream after its kernels.  Its error, if any, is rethrown
// when the caller is about to use the factors (rethrow), else dropped with the factors.
void interior_join(rfdd_handle *h, bool rethrow = true) {
  if (h->I_thread.joinable()) h->I_thread.join();
  if (h->I_forked) {
    RFDD_CUDA(cudaStreamWaitEvent(h->st, h->ev_join, 0));
    h->I_forked = false;
  }
  if (h->I_exc) {
    std::exception_ptr e = h->I_exc;
    h->I_exc = nullptr;
    h->I_ready = false;
    if (rethrow) std::rethrow_exception(e);
  }
}

// X (dsum x m FP64, all subdomains, row-major) <- B_sigma^{-1} X on stream st, through the real
// factors of the interior step (LU and inverted diagonal blocks)
template <typename Tr>
void bsig_solve(const rfdd_handle *h, cudaStream_t st, double *X, int64_t m) {
  const int p = h->p;
  const int64_t dsum = h->dsum;
  Buf t;
  t.alloc((size_t)dsum * m * sizeof(Tr));
  convert<Tr, double>(st, X, t.as<Tr>(), dsum * m);
  std::vector<SolveItem<Tr>> si;
  for (int j = 0; j < p; ++j) {
    SolveItem<Tr> x;
    x.LU = h->IBs.as<Tr>() + h->I_boffr[j];
    x.piv = h->Ipiv.as<int>() + h->off[j];
    x.n = x.ld = (int)h->d[j];
    x.X = t.as<Tr>() + h->off[j] * m;
    x.ldx = (int)m;
    x.ncols = (int)m;
    x.Linv = h->IRLinv.as<Tr>() + h->I_rinvoff[j];
    x.Uinv = h->IRUinv.as<Tr>() + h->I_rinvoff[j];
    x.nbi = NBO;
    si.push_back(x);
  }
  lu_solve_batched<Tr>(st, si, NBO);
  convert<double, Tr>(st, t.as<Tr>(), X, dsum * m);
}

// nev_B^(j) = min(nev_b, d_j) eigenvectors per subdomain, from a subspace of mb_j columns
void vj_sizes(const rfdd_handle *h, std::vector<int64_t> &nvb, std::vector<int64_t> &mb, int64_t &mw) {
  const int p = h->p;
  nvb.assign(p, 0);
  mb.assign(p, 0);
  mw = 0;
  for (int j = 0; j < p; ++j) {
    nvb[j] = std::min<int64_t>(h->opt.nev_b, h->d[j]);
    mb[j] = std::min<int64_t>(h->d[j], nvb[j] + std::max<int64_t>(8, nvb[j] / 5));
    mw = std::max(mw, mb[j]);
  }
}

// V_j (Alg. 3 step 3): block shift-invert subspace iteration on B_sigma^{-1} M_B with
// M_B-orthonormalisation (Cholesky-QR twice), then a Rayleigh-Ritz step for (B_sigma, M_B) on each
// span(X_j) that keeps the nev_B eigenvectors with the smallest |delta - sigma|.  Runs on stream
// st after the B_sigma factors; leaves X in h->IVX, the selected eigenvectors of the projected
// problems in h->IVGt and the smallest |delta - sigma| in h->I_gap.  The two buffers are
// allocated by the caller's thread on the handle's stream.
template <typename Tr>
void interior_vj(rfdd_handle *h, cudaStream_t st, int *status, double sigma) {
  const int p = h->p;
  const int64_t dsum = h->dsum;
  std::vector<int64_t> nvb, mb;
  int64_t mw = 0;
  vj_sizes(h, nvb, mb, mw);
  double *X = h->IVX.as<double>();
  Buf Y, G, Rinv, dead, T;
  Y.alloc((size_t)dsum * mw * sizeof(double));
  T.alloc((size_t)dsum * mw * sizeof(double));
  G.alloc((size_t)p * mw * mw * sizeof(double));
  Rinv.alloc((size_t)p * mw * mw * sizeof(double));
  dead.alloc((size_t)p * mw * sizeof(int));
  RFDD_CUDA(cudaMemsetAsync(T.p, 0, (size_t)dsum * mw * sizeof(double), st));
  counter_uniform_dev(st, h->opt.seed, 500, X, dsum * mw);
  auto m_orth = [&](double *Xp) {  // M_B-orthonormalise each subdomain block (CholQR, twice)
    for (int pass = 0; pass < 2; ++pass) {
      spmm_f64(st, h->P, 0, dsum, 0, dsum, 0.0, 1.0, Xp, mw, Y.as<double>(), mw, mw, false);
      std::vector<GemmItem<double>> g;
      std::vector<CholItem> ch;
      for (int j = 0; j < p; ++j) {
        g.push_back({Xp + h->off[j] * mw, Y.as<double>() + h->off[j] * mw, G.as<double>() + (int64_t)j * mw * mw,
                     (int)mb[j], (int)mb[j], (int)h->d[j], (int)mw, (int)mw, (int)mb[j]});
        ch.push_back({G.as<double>() + (int64_t)j * mw * mw, Rinv.as<double>() + (int64_t)j * mw * mw,
                      dead.as<int>() + j * mw, (int)mb[j]});
      }
      basis_gemm_on(h, st, g, true, false, 1.0, 0.0, std::vector<char>(g.size(), 1));
      chol_inv_batched(st, ch, 1e-28);
      std::vector<GemmItem<double>> g2;
      for (int j = 0; j < p; ++j)
        g2.push_back({Xp + h->off[j] * mw, Rinv.as<double>() + (int64_t)j * mw * mw, T.as<double>() + h->off[j] * mw,
                      (int)h->d[j], (int)mb[j], (int)mb[j], (int)mw, (int)mb[j], (int)mw});
      basis_gemm_on(h, st, g2, false, false, 1.0, 0.0);
      RFDD_CUDA(cudaMemcpyAsync(Xp, T.p, (size_t)dsum * mw * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
  };
  m_orth(X);
  const int iters = std::max(1, h->opt.subspace_iters);
  for (int it = 0; it < iters; ++it) {
    spmm_f64(st, h->P, 0, dsum, 0, dsum, 0.0, 1.0, X, mw, Y.as<double>(), mw, mw, false);  // M_B X
    bsig_solve<Tr>(h, st, Y.as<double>(), mw);
    RFDD_CUDA(cudaMemcpyAsync(X, Y.p, (size_t)dsum * mw * sizeof(double), cudaMemcpyDeviceToDevice, st));
    m_orth(X);
  }
  // Rayleigh-Ritz for (B_sigma, M_B) on span(X_j): H_j = X_j^T B_sigma X_j (X_j is M_B-orthonormal)
  spmm_f64(st, h->P, 0, dsum, 0, dsum, 1.0, -sigma, X, mw, Y.as<double>(), mw, mw, false);
  {
    std::vector<GemmItem<double>> g;
    for (int j = 0; j < p; ++j)
      g.push_back({X + h->off[j] * mw, Y.as<double>() + h->off[j] * mw, G.as<double>() + (int64_t)j * mw * mw,
                   (int)mb[j], (int)mb[j], (int)h->d[j], (int)mw, (int)mw, (int)mb[j]});
    basis_gemm_on(h, st, g, true, false, 1.0, 0.0, std::vector<char>(g.size(), 1));
  }
  Buf ed, ee, et, ew, el, eZ;
  ed.alloc((size_t)p * mw * sizeof(double));
  ee.alloc((size_t)p * mw * sizeof(double));
  et.alloc((size_t)p * mw * sizeof(double));
  ew.alloc((size_t)p * mw * sizeof(double));
  el.alloc((size_t)p * mw * sizeof(double));
  eZ.alloc((size_t)p * mw * mw * sizeof(double));
  std::vector<SymItem> si;
  for (int j = 0; j < p; ++j)
    si.push_back({G.as<double>() + (int64_t)j * mw * mw, (int)mb[j], (int)mb[j], ed.as<double>() + j * mw,
                  ee.as<double>() + j * mw, et.as<double>() + j * mw, ew.as<double>() + j * mw,
                  el.as<double>() + j * mw, eZ.as<double>() + (int64_t)j * mw * mw});
  sym_eig_values(st, si, status);
  std::vector<double> ev((size_t)p * mw);
  RFDD_CUDA(cudaMemcpyAsync(ev.data(), el.p, ev.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  RFDD_CUDA(cudaStreamSynchronize(st));
  // Ritz values of (B_sigma, M_B) on span X_j: delta - sigma for the delta nearest sigma
  double gap = std::numeric_limits<double>::infinity();
  for (int j = 0; j < p; ++j)
    for (int64_t c = 0; c < mb[j]; ++c) gap = std::min(gap, std::fabs(ev[j * mw + c]));
  std::vector<BackItem> bi;
  for (int j = 0; j < p; ++j) {
    std::vector<int> idx(mb[j]);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int b) { return std::fabs(ev[j * mw + a]) < std::fabs(ev[j * mw + b]); });
    idx.resize(nvb[j]);
    std::sort(idx.begin(), idx.end());
    bi.push_back({&si[j], idx, h->IVGt.as<double>() + (int64_t)j * mw * mw, (int)mb[j]});
  }
  sym_eig_vectors(st, bi, 1e-6);
  h->I_gap = gap;
}

// B_sigma^(j) dense (real) blocks, their LU and inverted diagonal blocks.  Buffers are allocated
// and the small tables uploaded on the handle's stream.  With on == h->st the kernels follow
// there and record into h->status.  Otherwise a host thread launches them on `on` after ev_fork
// (so that their thousands of small launches do not hold up the launches of the complex
// factorisations), records the pivot status in I_status and signals ev_join; interior_join
// waits for it.
template <typename Tr>
void interior_factor_start(rfdd_handle *h, double sigma, cudaStream_t on) {
  cudaStream_t st = h->st;
  h->I_ready = false;
  interior_join(h, false);  // an earlier start that was never consumed (a solve that failed after it)
  const int p = h->p;
  const int64_t dsum = h->dsum;
  std::vector<int64_t> doff(p + 1, 0);
  h->I_boffr.assign(p, 0);
  h->I_rinvoff.assign(p + 1, 0);
  int64_t tot = 0;
  for (int j = 0; j < p; ++j) {
    doff[j + 1] = doff[j] + h->d[j];
    h->I_boffr[j] = tot;
    tot += h->d[j] * h->d[j];
    h->I_rinvoff[j + 1] = h->I_rinvoff[j] + block_inverse_elems(h->d[j], NBO);
  }
  h->IBs.alloc((size_t)tot * sizeof(Tr));
  h->Ipiv.alloc((size_t)std::max<int64_t>(1, dsum) * sizeof(int));
  h->IRLinv.alloc((size_t)h->I_rinvoff[p] * sizeof(Tr));
  h->IRUinv.alloc((size_t)h->I_rinvoff[p] * sizeof(Tr));
  upload(h->I_doff, doff, st);
  upload(h->I_boffr_dev, h->I_boffr, st);
  std::vector<cx<double>> zsig = {cx<double>(sigma, 0.0)};
  upload(h->I_zs, zsig, st);
  {
    std::vector<int64_t> nvb, mb;
    vj_sizes(h, nvb, mb, h->I_mw);
    h->IVX.alloc((size_t)std::max<int64_t>(1, dsum * h->I_mw) * sizeof(double));
    h->IVGt.alloc((size_t)std::max<int64_t>(1, (int64_t)p * h->I_mw * h->I_mw) * sizeof(double));
  }
  int *status = h->status.as<int>();
  if (on != st) {
    if (!h->I_status.p) h->I_status.alloc(sizeof(int));
    RFDD_CUDA(cudaMemsetAsync(h->I_status.p, 0, sizeof(int), st));
    status = h->I_status.as<int>();
    RFDD_CUDA(cudaEventRecord(h->ev_fork, st));
  }
  Tr *Bs = h->IBs.as<Tr>();
  std::vector<LuItem<Tr>> items;
  std::vector<SolveItem<Tr>> fi;
  std::vector<Tr *> li, ui;
  for (int j = 0; j < p; ++j) {
    LuItem<Tr> it;
    it.A = Bs + h->I_boffr[j];
    it.piv = h->Ipiv.as<int>() + h->off[j];
    it.dp = it.D = it.ld = (int)h->d[j];
    items.push_back(it);
    SolveItem<Tr> x;
    x.LU = Bs + h->I_boffr[j];
    x.piv = nullptr;
    x.n = x.ld = (int)h->d[j];
    x.X = nullptr;
    x.ldx = x.ncols = 0;
    fi.push_back(x);
    li.push_back(h->IRLinv.as<Tr>() + h->I_rinvoff[j]);
    ui.push_back(h->IRUinv.as<Tr>() + h->I_rinvoff[j]);
  }
  const DevPencil P = h->P;
  const DevDD dd = h->dd;
  const int64_t *doff_dev = h->I_doff.as<int64_t>(), *boffr_dev = h->I_boffr_dev.as<int64_t>();
  const cx<double> *zs = h->I_zs.as<cx<double>>();
  auto launch = [=](cudaStream_t s) {
    TcStatusScope ts(status);  // tensor-core time-outs of these launches land in their status word
    // assemble_blocks without border: D_j = d_j, and the same row mapping
    assemble_blocks<Tr>(s, P, dd, doff_dev, dsum, boffr_dev, zs, 1, Bs, false);
    lu_batched<Tr>(s, items, NBO_LU, status);
    // inverted diagonal blocks for the many solves of the subspace iteration and the chains
    lu_block_inverses<Tr>(s, fi, NBO, li, ui);
    // V_j needs only these factors: on the second stream it overlaps the complex factorisations
    // and the Lanczos process too
    interior_vj<Tr>(h, s, status, sigma);
  };
  if (on == st) {
    launch(st);
  } else {
    int device = 0;
    RFDD_CUDA(cudaGetDevice(&device));
    h->I_forked = true;
    try {
      h->I_thread = std::thread([h, on, device, launch] {
        try {
          RFDD_CUDA(cudaSetDevice(device));
          AllocScope scope(on);  // this thread's workspaces are stream-ordered on its stream
          RFDD_CUDA(cudaStreamWaitEvent(on, h->ev_fork, 0));
          launch(on);
        } catch (...) {
          h->I_exc = std::current_exception();
        }
        // recorded even after an error, so that interior_join never waits on a stale event
        cudaEventRecord(h->ev_join, on);
      });
    } catch (const std::system_error &) {  // no thread to be had: the same launches from here
      AllocScope scope(on);
      RFDD_CUDA(cudaStreamWaitEvent(on, h->ev_fork, 0));
      launch(on);
      RFDD_CUDA(cudaEventRecord(h->ev_join, on));
    }
  }
  h->I_sigma = sigma;
  h->I_tsize = sizeof(Tr);
  h->I_ready = true;
}

template <typename Tr>
void interior_impl(rfdd_handle *h, double sigma) {
  cudaStream_t st = h->st;
  const int p = h->p;
  const int64_t n = h->n, dsum = h->dsum, s = h->s, mu = h->mu;
  const int psi = std::max(1, h->opt.psi);
  RFDD_REQUIRE(mu > 0, RFDD_ESTATE, "interior: run the Lanczos step first");
  h->sigma_used = sigma;
  // B_sigma^(j) dense (real), its LU and inverted diagonal blocks: started at the beginning of
  // the solve on the second stream, or computed here
  // factors started on the second stream are used when they are for this shift and type; only
  // then does their launch error or pivot status concern this call
  const bool use_forked = h->I_forked && h->I_ready && h->I_sigma == sigma && h->I_tsize == sizeof(Tr);
  interior_join(h, use_forked);
  Lap lap(st, "interior");
  if (!(h->I_ready && h->I_sigma == sigma && h->I_tsize == sizeof(Tr))) interior_factor_start<Tr>(h, sigma, st);
  h->I_ready = false;  // consumed: the next solve factors again
  sync_status(h, "interior LU");
  if (use_forked && h->I_status.p) sync_status(h, "interior LU", &h->I_status);
  lap.mark("join");
  // V_j (computed with the factors, see interior_vj): sizes and column offsets in Z
  std::vector<int64_t> nvb, mb, voff(p + 1, 0);
  int64_t mw = 0;
  vj_sizes(h, nvb, mb, mw);
  for (int j = 0; j < p; ++j) voff[j + 1] = voff[j] + nvb[j];
  RFDD_REQUIRE(mw == h->I_mw, RFDD_ESTATE, "interior: V_j buffers of another size");
  h->kappa = voff[p];
  h->voff = voff;
  h->interior_gap = h->I_gap;
  // Z = [blockdiag(V_j) | -Sigma^(psi) | Gamma^(psi)] (n x k), interface rows [0 | Q 0 | 0]
  const bool with_gamma = h->has_me;
  const int64_t kz = h->kappa + (int64_t)psi * mu * (with_gamma ? 2 : 1);
  h->kz = kz;
  h->Zb.alloc((size_t)n * kz * sizeof(double));
  double *Z = h->Zb.as<double>();
  RFDD_CUDA(cudaMemsetAsync(Z, 0, (size_t)n * kz * sizeof(double), st));
  {
    // V_j = X_j * Gt_j^T  (d_j x nvb_j) into Z rows off_j, columns voff_j
    std::vector<GemmItem<double>> g;
    for (int j = 0; j < p; ++j)
      g.push_back({h->IVX.as<double>() + h->off[j] * mw, h->IVGt.as<double>() + (int64_t)j * mw * mw,
                   Z + h->off[j] * kz + voff[j], (int)h->d[j], (int)nvb[j], (int)mb[j], (int)mw, (int)mb[j], (int)kz});
    basis_gemm(h, g, false, true, 1.0, 0.0);
  }
  h->IVX.release();
  h->IVGt.release();
  lap.mark("V_j");
  // Phi = (E - sigma M_E) Q, Psi = M_E Q  (all interior rows, d x mu), side by side in one block
  // [Phi | Psi]: both chains apply the same B_sigma^{-1} M_B, so each step is one product and one
  // solve on nch * mu columns (Eq. trabala, trabala2)
  const int nch = with_gamma ? 2 : 1;
  const int64_t wc = (int64_t)nch * mu;
  Buf PP, tmp, neg;
  PP.alloc((size_t)dsum * wc * sizeof(double));
  tmp.alloc((size_t)dsum * wc * sizeof(double));
  spmm_f64(st, h->P, 0, dsum, dsum, n, 1.0, -sigma, h->Q.as<double>(), h->qcap, PP.as<double>(), wc, mu, false);
  if (with_gamma)
    spmm_f64(st, h->P, 0, dsum, dsum, n, 0.0, 1.0, h->Q.as<double>(), h->qcap, PP.as<double>() + mu, wc, mu, false);
  const std::vector<double> negv((size_t)mu, -1.0);
  upload(neg, negv, st);
  for (int t = 0; t < psi; ++t) {
    if (t > 0) {
      spmm_f64(st, h->P, 0, dsum, 0, dsum, 0.0, 1.0, PP.as<double>(), wc, tmp.as<double>(), wc, wc, false);  // M_B X
      RFDD_CUDA(cudaMemcpyAsync(PP.p, tmp.p, (size_t)dsum * wc * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    bsig_solve<Tr>(h, st, PP.as<double>(), wc);
    // Z[0:dsum, kappa + t*mu : +mu] = -Sigma step t;  Z[0:dsum, kappa + psi*mu + t*mu : +mu] = Gamma step t
    const int64_t cs = h->kappa + (int64_t)t * mu;
    copy_rows_f64(st, PP.as<double>(), wc, Z + cs, kz, dsum, mu);
    scale_cols_f64(st, Z + cs, dsum, mu, kz, neg.as<double>());
    if (with_gamma) copy_rows_f64(st, PP.as<double>() + mu, wc, Z + h->kappa + (int64_t)psi * mu + t * mu, kz, dsum, mu);
  }
  // interface rows: Q under the first mu columns of the Sigma block
  copy_rows_f64(st, h->Q.as<double>(), h->qcap, Z + dsum * kz + h->kappa, kz, s, mu);
  lap.mark("chains");
  sync_status(h, "interior");
}

// ------------------------------------------------------------------------------------
// a9 + a10
// ------------------------------------------------------------------------------------
struct SolveState {
  double *X = nullptr;
};

template <typename Tf>
void rr_on_Z(rfdd_handle *h, double alpha, double beta, rfdd_result *res) {
  cudaStream_t st = h->st;
  const int64_t n = h->n, kz = h->kz;
  Buf C;
  std::vector<int> sel;
  int64_t m_sel = 0;
  // pivots below this (on the unit-diagonal Gram matrix) mark linearly dependent columns of Z
  const double drop = 1e-12;
  RRout rr = rayleigh_ritz_coeffs(
      h, h->Zb.as<double>(), kz, drop, 1e-9,
      [&](const std::vector<double> &th) {
        int64_t nin = 0;
        for (double t : th) nin += (t >= alpha && t <= beta);
        int64_t m = nin + std::max<int64_t>((int64_t)std::ceil(h->opt.guard_frac * nin), h->opt.min_guard);
        if (h->opt.m_align > 1) m = (m + h->opt.m_align - 1) / h->opt.m_align * h->opt.m_align;
        m = std::min<int64_t>((int64_t)th.size(), m);
        m_sel = m;
        return select_nearest(th, alpha, beta, m);
      },
      C, sel, true);
  h->rr_theta = rr.theta;
  h->m0 = (int64_t)sel.size();
  h->X0.alloc((size_t)n * std::max<int64_t>(1, h->m0) * sizeof(double));
  if (h->m0 > 0)
    basis_gemm(h, {{h->Zb.as<double>(), C.as<double>(), h->X0.as<double>(), (int)n, (int)h->m0, (int)kz,
                             (int)kz, (int)h->m0, (int)h->m0}},
                       false, false, 1.0, 0.0);
  if (res) {
    res->pre_evals.clear();
    for (double t : rr.theta)
      if (t >= alpha && t <= beta) res->pre_evals.push_back(t);
    res->info.k = rr.r;
  }
  RFDD_CUDA(cudaStreamSynchronize(st));
}

// Condition bound of the shifted systems when M's Gershgorin bound is positive:
// ||(A - z M)^{-1}|| <= 1 / (|Im z| lambda_min(M)), so kappa(A - z M) <= (||A|| + |z| ||M||) /
// (|Im z| gershM).  A solve refined to scaled backward error eta has forward error up to kappa eta.
// 0 when no bound is known.
double shifted_kappa_bound(const rfdd_handle *h) {
  double kappa = 0.0;
  if (h->gershM > 0.0 && std::isfinite(h->gershM))
    for (const auto &zl : h->z) {
      const double zn = std::hypot(zl.re, zl.im);
      kappa = std::max(kappa, (h->normA + zn * h->normM) / (std::fabs(zl.im) * h->gershM));
    }
  return kappa;
}

template <typename Tf>
void complete(rfdd_handle *h, double alpha, double beta, rfdd_result *res) {
  cudaStream_t st = h->st;
  const int64_t n = h->n;
  const int nc = h->nnodes;
  int64_t m = h->m0;
  Buf X;
  X.alloc((size_t)n * m * sizeof(double));
  RFDD_CUDA(cudaMemcpyAsync(X.p, h->X0.p, (size_t)n * m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  // residuals of the RF-DDES Ritz pairs before completion (diagnostic)
  auto residuals_of = [&](const double *Xp, int64_t mm, const std::vector<double> &th, std::vector<double> &out) {
    Buf AX, MX, thd, rs;
    AX.alloc((size_t)n * mm * sizeof(double));
    MX.alloc((size_t)n * mm * sizeof(double));
    spmm_f64(st, h->P, 0, n, 0, n, 1.0, 0.0, Xp, mm, AX.as<double>(), mm, mm, false);
    spmm_f64(st, h->P, 0, n, 0, n, 0.0, 1.0, Xp, mm, MX.as<double>(), mm, mm, false);
    upload(thd, th, st);
    rs.alloc(mm * sizeof(double));
    ritz_residuals(st, AX.as<double>(), MX.as<double>(), thd.as<double>(), n, mm, rs.as<double>());
    out.resize(mm);
    RFDD_CUDA(cudaMemcpyAsync(out.data(), rs.p, mm * sizeof(double), cudaMemcpyDeviceToHost, st));
    RFDD_CUDA(cudaStreamSynchronize(st));
  };
  {
    // Ritz values of the selected X0 columns (sorted-by-value selection of rr_theta)
    std::vector<double> th0 = h->rr_theta;
    std::vector<int> idx = select_nearest(th0, alpha, beta, m);
    std::vector<double> ths;
    for (int i : idx) ths.push_back(th0[i]);
    std::vector<double> r0;
    if (m > 0) residuals_of(X.as<double>(), m, ths, r0);
    double mx = 0.0;
    int64_t nin = 0;
    for (int64_t c = 0; c < m; ++c)
      if (ths[c] >= alpha && ths[c] <= beta) { mx = std::max(mx, r0[c]); ++nin; }
    res->info.pre_max_resid = mx;
    res->info.pre_nev = nin;
    RFDD_LOGF("rf-ddes: mu=%lld kz=%lld r=%zu m0=%lld inside=%lld max_res_inside=%.3e", (long long)h->mu,
              (long long)h->kz, h->rr_theta.size(), (long long)m, (long long)nin, mx);
  }
  int64_t count_prev = res->info.pre_nev;
  double res_level = std::max(res->info.pre_max_resid, 1e-300);
  const double kappa = shifted_kappa_bound(h);
  // The double-FP32 refinement residual is accurate to about 2^-46 of sum |a||x|; when kappa times
  // that exceeds 1/100 of the residual target, the residual is formed with FP64 products.
  bool fp64_res = kappa * 0x1p-46 > 1e-2 * h->opt.res_tol;
  // The double-FP32 basis products (Gram matrices, Ritz vectors) leave an error of about 2^-46
  // relative in each Ritz vector; a residual relative to |lambda| then cannot fall below about
  // 2^-46 ||A|| / |lambda|, which is above the target for eigenvalues far smaller than ||A||.
  // When the largest residual of the unconverged inside pairs shrinks by less than 10x over a
  // pass, the remaining passes form those products, and the refinement residuals, in FP64.
  struct BasisPrecision {
    rfdd_handle *h;
    ~BasisPrecision() { h->basis_fp64 = false; }
  } basis_precision{h};
  h->basis_fp64 = false;
  double unconv_prev = -1.0;
  Buf V, Xc, C, Xprev;
  std::vector<double> theta, resid, theta_prev, resid_prev;
  std::vector<int64_t> keep;  // Ritz pairs returned: inside [alpha, beta], converged, not spurious
  int passes = 0, irmax = 0, grown = 0, pass_limit = h->opt.max_passes;
  bool converged = false, from_prev = false;
  // A pass whose inside Ritz pairs have all converged except some with large residuals, while
  // the number of converged ones did not change, leaves those pairs "suspect": the next filter
  // application measures the filter's Rayleigh quotient at each of them (gain, rho(lambda) for an
  // eigenvector and >= 1/2 on [alpha, beta]).  Suspects with gain below 1/4 are spurious: mixtures
  // of eigenvectors from both sides of the interval with equal small filter values (the midpoint
  // filter is symmetric about the centre), whose Rayleigh quotient falls inside.  They are
  // dropped and the converged pairs of that pass are the result.
  bool suspect = false;
  int64_t nin = 0, good_prev = -1;
  for (passes = 1; passes <= pass_limit; ++passes) {
    // X <- 2 Re sum w_l (A - z_l M)^{-1} M X   (Eq. rhoAM through Eq. inv_dd2)
    V.ensure((size_t)n * m * sizeof(double));
    spmm_f64(st, h->P, 0, n, 0, n, 0.0, 1.0, X.as<double>(), m, V.as<double>(), m, m, false);
    if (suspect) {
      Xprev.alloc((size_t)n * m * sizeof(double));
      RFDD_CUDA(cudaMemcpyAsync(Xprev.p, X.p, (size_t)n * m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    Xc.ensure((size_t)nc * n * m * sizeof(cx<double>));
    // the filter only has to be as accurate as the subspace it acts on: refine the shifted
    // solves to a small fraction of the current residual level, and no further than a small
    // fraction (1/100) of the residual target; where the condition bound is known, kappa times
    // the backward error stays below those fractions
    double ir_tol = 1e-6 * res_level;
    if (kappa > 0.0) ir_tol = std::min(ir_tol, 1e-2 * res_level / kappa);
    ir_tol = std::max(std::max(1e-15, 1e-2 * h->opt.res_tol / std::max(1.0, kappa)), ir_tol);
    irmax = std::max(irmax, refined_solve<Tf>(h, V.as<double>(), Xc.as<cx<double>>(), m, ir_tol, fp64_res));
    weighted_real_sum<cx<double>>(st, Xc.as<cx<double>>(), n * m, h->w_dev.as<cx<double>>(), nc, 2.0, X.as<double>(),
                                  n * m);
    if (suspect) {
      // gains of the last pass's Ritz vectors x (M-orthonormal): x^T M rho(A) x
      Buf g;
      g.alloc((size_t)m * sizeof(double));
      col_dots(st, V.as<double>(), X.as<double>(), n, m, g.as<double>());
      std::vector<double> gain(m);
      RFDD_CUDA(cudaMemcpyAsync(gain.data(), g.p, m * sizeof(double), cudaMemcpyDeviceToHost, st));
      RFDD_CUDA(cudaStreamSynchronize(st));
      bool all_spurious = true;
      int64_t spurious = 0;
      for (int64_t c = 0; c < m; ++c)
        if (theta_prev[c] >= alpha && theta_prev[c] <= beta && resid_prev[c] > h->opt.res_tol) {
          if (gain[c] < 0.25) ++spurious;
          else all_spurious = false;
        }
      RFDD_LOGF("pass %d: %lld suspect Ritz pairs of the last pass are spurious (all: %d)", passes,
                (long long)spurious, (int)all_spurious);
      if (all_spurious) {
        keep.clear();
        for (int64_t c = 0; c < m; ++c)
          if (theta_prev[c] >= alpha && theta_prev[c] <= beta && resid_prev[c] <= h->opt.res_tol) keep.push_back(c);
        theta = theta_prev;
        resid = resid_prev;
        nin = (int64_t)keep.size();
        converged = true;
        from_prev = true;
        break;
      }
    }
    // Rayleigh-Ritz on range(X), all Ritz pairs kept
    std::vector<int> sel;
    RRout rr = rayleigh_ritz_coeffs(
        h, X.as<double>(), m, 1e-12, 1e-5,
        [&](const std::vector<double> &th) {
          std::vector<int> all(th.size());
          std::iota(all.begin(), all.end(), 0);
          return all;
        },
        C, sel);
    const int64_t r = rr.r;
    Buf Xn;
    Xn.alloc((size_t)n * r * sizeof(double));
    basis_gemm(h, {{X.as<double>(), C.as<double>(), Xn.as<double>(), (int)n, (int)r, (int)m, (int)m,
                             (int)r, (int)r}},
                       false, false, 1.0, 0.0);
    theta = rr.theta;
    residuals_of(Xn.as<double>(), r, theta, resid);
    X.alloc((size_t)n * r * sizeof(double));
    RFDD_CUDA(cudaMemcpyAsync(X.p, Xn.p, (size_t)n * r * sizeof(double), cudaMemcpyDeviceToDevice, st));
    m = r;
    keep.clear();
    int64_t inside = 0, good = 0;
    double mx = 0.0;
    for (int64_t c = 0; c < r; ++c)
      if (theta[c] >= alpha && theta[c] <= beta) {
        ++inside;
        keep.push_back(c);
        mx = std::max(mx, resid[c]);
        good += resid[c] <= h->opt.res_tol;
      }
    nin = inside;
    RFDD_LOGF("pass %d: m=%lld inside=%lld converged=%lld (prev inside %lld, prev converged %lld) max_res_inside=%.3e "
              "ir_steps=%d", passes, (long long)m, (long long)inside, (long long)good, (long long)count_prev,
              (long long)good_prev, mx, irmax);
    // the residual level the next refinement targets: the median over the inside pairs (spurious
    // pairs never converge and would hold the level of the others up), and that of the converged
    // pairs when only suspects remain above it
    double mx_good = 0.0;
    std::vector<double> rin;
    for (int64_t c : keep) {
      rin.push_back(resid[c]);
      if (resid[c] <= h->opt.res_tol) mx_good = std::max(mx_good, resid[c]);
    }
    if (!rin.empty()) {
      std::nth_element(rin.begin(), rin.begin() + rin.size() / 2, rin.end());
      res_level = rin[rin.size() / 2];
    } else {
      res_level = 1.0;
    }
    // The block must hold every eigenvalue inside plus guard vectors.  When the Ritz values inside
    // leave fewer than the guard count of columns outside, the interval may hold more eigenvalues
    // than the block (the RF-DDES count it was sized from was short), and subspace iteration
    // cannot converge there: the filter is nearly flat inside the interval.  The block then grows
    // to twice its size with fresh counter-based vectors, and the passes continue.
    const int64_t guard = std::max<int64_t>((int64_t)std::ceil(h->opt.guard_frac * inside), h->opt.min_guard);
    if (inside > 0 && r - inside < guard && grown < 4 && r < n) {
      int64_t mn = std::max<int64_t>(2 * r, inside + 2 * guard);
      if (h->opt.m_align > 1) mn = (mn + h->opt.m_align - 1) / h->opt.m_align * h->opt.m_align;
      mn = std::min<int64_t>(mn, n);
      if (mn > r) {
        Buf Xg, Tr;
        Xg.alloc((size_t)n * mn * sizeof(double));
        Tr.alloc((size_t)n * (mn - r) * sizeof(double));
        copy_rows_f64(st, X.as<double>(), r, Xg.as<double>(), mn, n, r);
        counter_uniform_dev(st, h->opt.seed, 5000 + (uint64_t)grown, Tr.as<double>(), n * (mn - r));
        copy_rows_f64(st, Tr.as<double>(), mn - r, Xg.as<double>() + r, mn, n, mn - r);
        X.alloc((size_t)n * mn * sizeof(double));
        RFDD_CUDA(cudaMemcpyAsync(X.p, Xg.p, (size_t)n * mn * sizeof(double), cudaMemcpyDeviceToDevice, st));
        RFDD_LOGF("pass %d: %lld Ritz values inside a block of %lld: block grown to %lld", passes, (long long)inside,
                  (long long)r, (long long)mn);
        m = mn;
        ++grown;
        pass_limit = std::min(h->opt.max_passes + 10, pass_limit + 2);  // passes for the grown block
        count_prev = -1;
        good_prev = -1;
        suspect = false;
        continue;
      }
    }
    if (inside == count_prev && (inside == 0 || mx <= h->opt.res_tol)) {
      converged = true;
      break;
    }
    {
      double unconv = 0.0;
      for (int64_t c : keep)
        if (resid[c] > h->opt.res_tol) unconv = std::max(unconv, resid[c]);
      if (is_mixed(h) && !h->basis_fp64 && unconv > 0.0 && unconv_prev > 0.0 && unconv > 0.1 * unconv_prev) {
        h->basis_fp64 = true;
        fp64_res = true;
        res->info.fp64_basis = 1;
        RFDD_LOGF("pass %d: unconverged residuals %.3e after %.3e: basis products in FP64 from here on", passes,
                  unconv, unconv_prev);
      }
      unconv_prev = unconv;
    }
    suspect = good > 0 && good < inside && good == good_prev;
    if (suspect) {
      theta_prev = theta;
      resid_prev = resid;
      res_level = mx_good;
      // the test needs one more filter application (the passes stay bounded: max_passes + 10)
      pass_limit = std::min(h->opt.max_passes + 10, std::max(pass_limit, passes + 1));
    }
    count_prev = inside;
    good_prev = good;
  }
  if (passes > pass_limit) passes = pass_limit;
  // results in the original ordering: evecs[i_orig][c] = X[iperm[i_orig]][keep[c]]
  res->n = n;
  res->nev = nin;
  res->evals.clear();
  res->resid.clear();
  for (int64_t c : keep) {
    res->evals.push_back(theta[c]);
    res->resid.push_back(resid[c]);
  }
  res->evecs.alloc((size_t)n * std::max<int64_t>(1, nin) * sizeof(double));
  if (nin > 0) {
    Buf keep_dev;
    upload(keep_dev, keep, st);
    gather_rows_cols_f64(st, (from_prev ? Xprev : X).as<double>(), m, h->iperm_dev.as<int64_t>(),
                         keep_dev.as<int64_t>(), res->evecs.as<double>(), nin, n, nin);
    RFDD_CUDA(cudaStreamSynchronize(st));
  }
  upload(res->evals_dev, res->evals, st);
  upload(res->resid_dev, res->resid, st);
  RFDD_CUDA(cudaStreamSynchronize(st));
  res->info.nev = nin;
  res->info.m = m;
  res->info.passes = passes;
  res->info.ir_steps_max = irmax;
  res->info.max_resid = 0.0;
  for (double v : res->resid) res->info.max_resid = std::max(res->info.max_resid, v);
  res->info.status = converged ? RFDD_OK : RFDD_NOT_CONVERGED;
}

// ------------------------------------------------------------------------------------
// Interior polish (Section 3, Eqs. (schur_eigvec2) and (compute_u_parallel)): an eigenvector's
// interior part follows from its interface part y by one real solve per subdomain,
// (B_j - lambda M_B^(j)) u_j = -(E_j - lambda M_E^(j)) y_j.  Applied to approximate pairs it
// replaces the interior rows, then M-normalises and takes the Rayleigh quotient.  FP64.
// ------------------------------------------------------------------------------------
void polish_impl(rfdd_handle *h, int64_t nev, double *lam, double *Xh, double *resid) {
  cudaStream_t st = h->st;
  const int p = h->p;
  const int64_t n = h->n, dsum = h->dsum;
  for (int64_t c = 0; c < nev; ++c)
    RFDD_REQUIRE(std::isfinite(lam[c]), RFDD_EINVAL, "polish: non-finite eigenvalue");
  // interior-first ordering: Xi[k][c] = X[perm[k]][c]
  Buf Xo, Xi, permd, lamd, R;
  Xo.alloc((size_t)n * nev * sizeof(double));
  Xi.alloc((size_t)n * nev * sizeof(double));
  RFDD_CUDA(cudaMemcpyAsync(Xo.p, Xh, (size_t)n * nev * sizeof(double), cudaMemcpyHostToDevice, st));
  upload(permd, h->perm, st);
  gather_rows_f64(st, Xo.as<double>(), nev, permd.as<int64_t>(), Xi.as<double>(), nev, n, nev);
  std::vector<double> lv(lam, lam + nev);
  upload(lamd, lv, st);
  // right-hand sides of every subdomain at once (interior rows): lambda_c M_E y_c - E y_c
  R.alloc((size_t)std::max<int64_t>(1, dsum) * nev * sizeof(double));
  const double *Y = Xi.as<double>() + dsum * nev;
  spmm_f64(st, h->P, 0, dsum, dsum, n, 0.0, 1.0, Y, nev, R.as<double>(), nev, nev, false);
  scale_cols_f64(st, R.as<double>(), dsum, nev, nev, lamd.as<double>());
  spmm_f64(st, h->P, 0, dsum, dsum, n, -1.0, 0.0, Y, nev, R.as<double>(), nev, nev, true);
  // shifted dense blocks, LU and one solve per (pair, subdomain), in chunks of pairs
  int64_t per_pair = 0;
  std::vector<int64_t> doff(p + 1, 0), bo(p, 0);
  for (int j = 0; j < p; ++j) {
    doff[j + 1] = doff[j] + h->d[j];
    bo[j] = per_pair;
    per_pair += h->d[j] * h->d[j];
  }
  size_t cap = (size_t)4 << 30;  // dense-block bytes per chunk
  if (h->opt.mem_budget > 0) cap = std::min(cap, h->opt.mem_budget / 2);
  const int64_t chunk =
      std::max<int64_t>(1, std::min<int64_t>({nev, (int64_t)(cap / ((size_t)per_pair * sizeof(double))), 65535}));
  Buf doff_dev, boff_dev, zs, Bs, piv;
  upload(doff_dev, doff, st);
  std::vector<int64_t> boff((size_t)chunk * p);
  for (int64_t l = 0; l < chunk; ++l)
    for (int j = 0; j < p; ++j) boff[l * p + j] = l * per_pair + bo[j];
  upload(boff_dev, boff, st);
  Bs.alloc((size_t)chunk * per_pair * sizeof(double));
  piv.alloc((size_t)chunk * std::max<int64_t>(1, dsum) * sizeof(int));
  for (int64_t c0 = 0; c0 < nev; c0 += chunk) {
    const int64_t cnt = std::min(chunk, nev - c0);
    std::vector<cx<double>> z(cnt);
    for (int64_t l = 0; l < cnt; ++l) z[l] = cx<double>(lam[c0 + l], 0.0);
    upload(zs, z, st);
    assemble_blocks<double>(st, h->P, h->dd, doff_dev.as<int64_t>(), dsum, boff_dev.as<int64_t>(),
                            zs.as<cx<double>>(), (int)cnt, Bs.as<double>(), false);
    std::vector<LuItem<double>> items;
    std::vector<SolveItem<double>> si;
    for (int64_t l = 0; l < cnt; ++l)
      for (int j = 0; j < p; ++j) {
        LuItem<double> it;
        it.A = Bs.as<double>() + boff[l * p + j];
        it.piv = piv.as<int>() + l * dsum + h->off[j];
        it.dp = it.D = it.ld = (int)h->d[j];
        items.push_back(it);
        SolveItem<double> x;
        x.LU = it.A;
        x.piv = it.piv;
        x.n = x.ld = (int)h->d[j];
        x.X = R.as<double>() + h->off[j] * nev + (c0 + l);
        x.ldx = (int)nev;
        x.ncols = 1;
        si.push_back(x);
      }
    lu_batched<double>(st, items, NBO_LU, h->status.as<int>());
    lu_solve_batched<double>(st, si, NBO);
  }
  sync_status(h, "polish LU");
  copy_rows_f64(st, R.as<double>(), nev, Xi.as<double>(), nev, dsum, nev);
  // M-normalise, Rayleigh quotients and residuals
  Buf AX, MX, dA, dM, scd, thd, rs;
  AX.alloc((size_t)n * nev * sizeof(double));
  MX.alloc((size_t)n * nev * sizeof(double));
  spmm_f64(st, h->P, 0, n, 0, n, 1.0, 0.0, Xi.as<double>(), nev, AX.as<double>(), nev, nev, false);
  spmm_f64(st, h->P, 0, n, 0, n, 0.0, 1.0, Xi.as<double>(), nev, MX.as<double>(), nev, nev, false);
  dA.alloc(nev * sizeof(double));
  dM.alloc(nev * sizeof(double));
  col_dots(st, Xi.as<double>(), nev, AX.as<double>(), nev, n, nev, dA.as<double>());
  col_dots(st, Xi.as<double>(), nev, MX.as<double>(), nev, n, nev, dM.as<double>());
  std::vector<double> xax(nev), xmx(nev), sc(nev), th(nev);
  RFDD_CUDA(cudaMemcpyAsync(xax.data(), dA.p, nev * sizeof(double), cudaMemcpyDeviceToHost, st));
  RFDD_CUDA(cudaMemcpyAsync(xmx.data(), dM.p, nev * sizeof(double), cudaMemcpyDeviceToHost, st));
  RFDD_CUDA(cudaStreamSynchronize(st));
  for (int64_t c = 0; c < nev; ++c) {
    RFDD_REQUIRE(xmx[c] > 0.0 && std::isfinite(xmx[c]), RFDD_ESINGULAR,
                 "polish: vector " + std::to_string(c) + " has no M-norm (zero interface part?)");
    sc[c] = 1.0 / std::sqrt(xmx[c]);
    th[c] = xax[c] / xmx[c];
  }
  upload(scd, sc, st);
  upload(thd, th, st);
  scale_cols_f64(st, Xi.as<double>(), n, nev, nev, scd.as<double>());
  scale_cols_f64(st, AX.as<double>(), n, nev, nev, scd.as<double>());
  scale_cols_f64(st, MX.as<double>(), n, nev, nev, scd.as<double>());
  rs.alloc(nev * sizeof(double));
  ritz_residuals(st, AX.as<double>(), MX.as<double>(), thd.as<double>(), n, nev, rs.as<double>());
  // back to the input ordering: X[o][c] = Xi[iperm[o]][c]
  gather_rows_f64(st, Xi.as<double>(), nev, h->iperm_dev.as<int64_t>(), Xo.as<double>(), nev, n, nev);
  RFDD_CUDA(cudaMemcpyAsync(Xh, Xo.p, (size_t)n * nev * sizeof(double), cudaMemcpyDeviceToHost, st));
  RFDD_CUDA(cudaMemcpyAsync(resid, rs.p, nev * sizeof(double), cudaMemcpyDeviceToHost, st));
  RFDD_CUDA(cudaStreamSynchronize(st));
  std::copy(th.begin(), th.end(), lam);
}

// ------------------------------------------------------------------------------------
// Eigenvalue count below sigma (Sylvester's law of inertia, in FP64).  With M SPD the number
// of eigenvalues of (A, M) below sigma is the number of negative eigenvalues of A - sigma M.
// In the interior-first block form of Eq. (eq1) with B_sigma nonsingular, the inertia of
// A - sigma M is the sum of the inertias of the blocks B_sigma^(j) and of the Schur
// complement S(sigma) (Haynsworth).  The bordered real blocks are factored as in the complex
// path (their trailing blocks give S(sigma)); each B_sigma^(j) and S(sigma) is reduced to
// tridiagonal form by Householder similarity, which keeps the inertia, and counted by Sturm.
// ------------------------------------------------------------------------------------
int64_t inertia_impl(rfdd_handle *h, double sigma) {
  cudaStream_t st = h->st;
  const int p = h->p;
  const int64_t s = h->s;
  std::vector<int64_t> boff(p, 0), Doff(p + 1, 0), hoff(p + 1, 0);
  int64_t tot = 0;
  for (int j = 0; j < p; ++j) {
    boff[j] = tot;
    tot += h->D[j] * h->D[j];
    Doff[j + 1] = Doff[j] + h->D[j];
    hoff[j + 1] = hoff[j] + h->d[j] * h->d[j];
  }
  Buf Bb, boff_dev, Doff_dev, zs, piv, Hs, dbuf, cnt;
  Bb.alloc((size_t)tot * sizeof(double));
  upload(boff_dev, boff, st);
  upload(Doff_dev, Doff, st);
  std::vector<cx<double>> zv = {cx<double>(sigma, 0.0)};
  upload(zs, zv, st);
  assemble_blocks<double>(st, h->P, h->dd, Doff_dev.as<int64_t>(), Doff[p], boff_dev.as<int64_t>(),
                          zs.as<cx<double>>(), 1, Bb.as<double>(), true);
  // the B_sigma^(j) blocks are counted from copies (the LU overwrites them); S(sigma) after them
  Hs.alloc((size_t)(hoff[p] + s * s) * sizeof(double));
  for (int j = 0; j < p; ++j)
    copy_rows_f64(st, Bb.as<double>() + boff[j], h->D[j], Hs.as<double>() + hoff[j], h->d[j], h->d[j], h->d[j]);
  piv.alloc((size_t)std::max<int64_t>(1, h->dsum) * sizeof(int));
  std::vector<LuItem<double>> items;
  for (int j = 0; j < p; ++j) {
    LuItem<double> it;
    it.A = Bb.as<double>() + boff[j];
    it.piv = piv.as<int>() + h->off[j];
    it.dp = (int)h->d[j];
    it.D = it.ld = (int)h->D[j];
    items.push_back(it);
  }
  lu_batched<double>(st, items, NBO_LU, h->status.as<int>());
  double *S = Hs.as<double>() + hoff[p];
  if (s > 0) {
    assemble_interface<double>(st, h->P, h->dd, zs.as<cx<double>>(), 1, S);
    for (int j = 0; j < p; ++j) {
      const int sj = (int)(h->sidx_off[j + 1] - h->sidx_off[j]);
      scatter_schur<double>(st, h->dd, j, (int)h->d[j], sj, h->sidx_off[j], boff_dev.as<int64_t>(), Bb.as<double>(), 1,
                            S);
    }
  }
  sync_status(h, "inertia: B_sigma factorisation");
  Bb.release();
  int64_t nmax = s;
  for (int j = 0; j < p; ++j) nmax = std::max(nmax, h->d[j]);
  const int nitems = p + (s > 0 ? 1 : 0);
  dbuf.alloc((size_t)nitems * 4 * std::max<int64_t>(1, nmax) * sizeof(double));
  std::vector<SymItem> si;
  for (int q = 0; q < nitems; ++q) {
    const int64_t nq = q < p ? h->d[q] : s;
    double *w = dbuf.as<double>() + (int64_t)q * 4 * nmax;
    si.push_back({q < p ? Hs.as<double>() + hoff[q] : S, (int)nq, (int)nq, w, w + nmax, w + 2 * nmax, w + 3 * nmax,
                  nullptr, nullptr});
  }
  cnt.alloc((size_t)nitems * sizeof(long long));
  sym_negative_counts(st, si, 0.0, cnt.as<long long>());
  std::vector<long long> hc(nitems);
  RFDD_CUDA(cudaMemcpyAsync(hc.data(), cnt.p, nitems * sizeof(long long), cudaMemcpyDeviceToHost, st));
  RFDD_CUDA(cudaStreamSynchronize(st));
  int64_t total = 0;
  for (long long c : hc) total += c;
  return total;
}

// ------------------------------------------------------------------------------------
// precision dispatch
// ------------------------------------------------------------------------------------
void set_nodes(rfdd_handle *h, int nc, const double *z, const double *w) {
  h->nnodes = nc;
  h->z.resize(nc);
  h->w.resize(nc);
  for (int l = 0; l < nc; ++l) {
    h->z[l] = cx<double>(z[2 * l], z[2 * l + 1]);
    h->w[l] = cx<double>(w[2 * l], w[2 * l + 1]);
    RFDD_REQUIRE(std::isfinite(h->z[l].re) && std::isfinite(h->z[l].im) && h->z[l].im != 0.0, RFDD_EINVAL,
                 "quadrature poles must be finite and off the real axis");
  }
  upload(h->z_dev, h->z, h->st);
  upload(h->w_dev, h->w, h->st);
}

void factor(rfdd_handle *h) {
  if (h->opt.mem_budget > 0) {
    const size_t need = factor_bytes(h, h->nnodes);
    RFDD_REQUIRE(need <= h->opt.mem_budget, RFDD_EADMIT,
                 "factorisation needs " + std::to_string(need) + " bytes, budget " + std::to_string(h->opt.mem_budget));
  }
  h->have_factors = false;
  h->fac.release();
  h->Sfac.release();
  h->Skeep.release();
  h->BLinv.release();
  h->BUinv.release();
  h->SLinv.release();
  h->SUinv.release();
  h->Pk.release();
  h->pkB.clear();
  h->pkS.clear();
  h->pkG.clear();
  h->Lfac.release();
  h->pivL.release();
  h->LLinv.release();
  h->LUinv.release();
  if (is_mixed(h)) factor_impl<cx<float>>(h);
  else factor_impl<cx<double>>(h);
}

// ------------------------------------------------------------------------------------
// Algorithm 1 (RF-KRYLOV, Section 2.2): Krylov on rho(M^{-1}A) in the whole space
// ------------------------------------------------------------------------------------
// Block Krylov with full orthogonalisation in the M inner product (rho(M^{-1}A) is self-adjoint
// there, so H_mu = Q^T M rho Q is symmetric; with M = I this is the printed Euclidean process):
//   line 2:     W = 2 Re sum_l w_l (A - z_l M)^{-1} M Q_t through Eq. (inv_dd2) with the same
//               factors as the RF-DDES solve and FP64 refinement;
//   lines 3-6:  two classical Gram-Schmidt passes in the M inner product against Q; their
//               coefficients are the block column t of H;
//   lines 7-12: M-Cholesky-QR of the new block (twice, with one more projection between);
//               columns that vanish are replaced by counter-based vectors (streams 7001, ...);
//   line 13:    every ceil(10/b) block steps, stop when the sum of the eigenvalues >= 1/2 of H_mu
//               changed by at most lanczos_tol of its magnitude since the previous check, or
//               when mu reaches the column cap;
//   lines 15-16: Rayleigh-Ritz of (A, M) on range(Q_mu); then the completion passes as in
//               rfdd_solve.
// The start block is counter-based (stream 7000).
template <typename Tf>
void rfkrylov_impl(rfdd_handle *h, double alpha, double beta, int64_t max_dim, rfdd_result *res) {
  cudaStream_t st = h->st;
  const int64_t n = h->n;
  const int nc = h->nnodes;
  const int64_t b = std::max<int64_t>(1, std::min<int64_t>(h->opt.block, n));
  const int64_t cap = std::min<int64_t>(n, max_dim > 0 ? max_dim : 4096);
  RFDD_REQUIRE(cap >= b, RFDD_EINVAL, "rf-krylov: max_dim below the block size");
  Buf Qb, W, MW, Xb, V, Xc, Cb, Gb, Rinv, dead, tmp;
  Qb.alloc((size_t)n * cap * sizeof(double));
  double *Q = Qb.as<double>();
  W.alloc((size_t)n * b * sizeof(double));
  MW.alloc((size_t)n * b * sizeof(double));
  Xb.alloc((size_t)n * b * sizeof(double));
  V.alloc((size_t)n * b * sizeof(double));
  Xc.alloc((size_t)nc * n * b * sizeof(cx<double>));
  Cb.alloc((size_t)cap * b * sizeof(double));
  Gb.alloc((size_t)b * b * sizeof(double));
  Rinv.alloc((size_t)b * b * sizeof(double));
  dead.alloc((size_t)b * sizeof(int));
  tmp.alloc((size_t)n * b * sizeof(double));
  const double kappa = shifted_kappa_bound(h);
  const bool fp64_res = kappa * 0x1p-46 > 1e-2 * h->opt.res_tol;
  // the filter is applied as accurately as the completion passes finish: 1/100 of the residual
  // target, divided by the condition bound where it is known
  const double ir_tol = std::max(1e-15, 1e-2 * h->opt.res_tol / std::max(1.0, kappa));
  std::vector<double> U((size_t)cap * cap, 0.0);  // blocks of H on and above the diagonal
  std::vector<double> hc((size_t)cap * b), hdiag(b);
  std::vector<int> hdead(b);
  double hmax = 0.0;
  // W -= Q C, C = Q[:, :ncols]^T M W (twice); with `acc` the coefficients are added to H's
  // block column starting at column c0
  auto mproj = [&](double *Wp, int64_t bw, int64_t ncols, bool acc, int64_t c0) {
    if (ncols <= 0) return;
    for (int pass = 0; pass < 2; ++pass) {
      spmm_f64(st, h->P, 0, n, 0, n, 0.0, 1.0, Wp, bw, MW.as<double>(), bw, bw, false);
      basis_gemm(h, {{Q, MW.as<double>(), Cb.as<double>(), (int)ncols, (int)bw, (int)n, (int)cap, (int)bw, (int)bw}},
                 true, false, 1.0, 0.0);
      basis_gemm(h, {{Q, Cb.as<double>(), Wp, (int)n, (int)bw, (int)ncols, (int)cap, (int)bw, (int)bw}}, false,
                 false, -1.0, 1.0);
      if (acc) {
        RFDD_CUDA(cudaMemcpyAsync(hc.data(), Cb.p, (size_t)ncols * bw * sizeof(double), cudaMemcpyDeviceToHost, st));
        RFDD_CUDA(cudaStreamSynchronize(st));
        for (int64_t r = 0; r < ncols; ++r)
          for (int64_t c = 0; c < bw; ++c) {
            U[(size_t)r * cap + c0 + c] += hc[(size_t)r * bw + c];
            hmax = std::max(hmax, std::fabs(U[(size_t)r * cap + c0 + c]));
          }
      }
    }
  };
  uint64_t extra = 0;
  // M-Cholesky-QR of Wp (n x bw) against Q[:, :ncols]; dead columns replaced and redone
  auto morth = [&](double *Wp, int64_t bw, int64_t ncols) {
    for (int attempt = 0; attempt < 4; ++attempt) {
      bool any_dead = false;
      for (int q = 0; q < 2 && !any_dead; ++q) {
        spmm_f64(st, h->P, 0, n, 0, n, 0.0, 1.0, Wp, bw, MW.as<double>(), bw, bw, false);
        basis_gemm(h, {{Wp, MW.as<double>(), Gb.as<double>(), (int)bw, (int)bw, (int)n, (int)bw, (int)bw, (int)bw}},
                   true, false, 1.0, 0.0, {1});
        std::vector<double> g((size_t)bw * bw);
        RFDD_CUDA(cudaMemcpyAsync(g.data(), Gb.p, g.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        chol_inv_batched(st, {CholItem{Gb.as<double>(), Rinv.as<double>(), dead.as<int>(), (int)bw}}, 1e-24);
        RFDD_CUDA(cudaMemcpyAsync(hdead.data(), dead.p, bw * sizeof(int), cudaMemcpyDeviceToHost, st));
        RFDD_CUDA(cudaStreamSynchronize(st));
        // a column whose M norm is at most 1e-14 max|H| is dead even when all are that small
        const double floor2 = (1e-14 * hmax) * (1e-14 * hmax);
        for (int64_t c = 0; c < bw; ++c) {
          if (!(g[(size_t)c * bw + c] > floor2)) hdead[c] = 1;
          any_dead |= hdead[c] != 0;
        }
        if (any_dead) break;
        basis_gemm(h, {{Wp, Rinv.as<double>(), tmp.as<double>(), (int)n, (int)bw, (int)bw, (int)bw, (int)bw, (int)bw}},
                   false, false, 1.0, 0.0);
        RFDD_CUDA(cudaMemcpyAsync(Wp, tmp.p, (size_t)n * bw * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (q == 0 && ncols > 0) mproj(Wp, bw, ncols, false, 0);  // one more pass after normalising
      }
      if (!any_dead) return;
      Buf fresh;
      fresh.alloc((size_t)n * sizeof(double));
      for (int64_t c = 0; c < bw; ++c)
        if (hdead[c]) {
          counter_uniform_dev(st, h->opt.seed, 7001 + extra++, fresh.as<double>(), n);
          copy_rows_f64(st, fresh.as<double>(), 1, Wp + c, bw, n, 1);
        }
      mproj(Wp, bw, ncols, false, 0);
    }
    throw Error(RFDD_ESINGULAR, "rf-krylov: could not extend the basis");
  };
  // eigenvalues of the symmetric H_mu (mu x mu) on the GPU
  auto h_eigs = [&](int64_t mu) {
    std::vector<double> H((size_t)mu * mu);
    for (int64_t r = 0; r < mu; ++r)
      for (int64_t c = 0; c < mu; ++c) {
        const double up = r <= c ? U[(size_t)r * cap + c] : U[(size_t)c * cap + r];
        H[(size_t)r * mu + c] = up;
      }
    // diagonal blocks: symmetric part (the coefficients of a block on itself)
    for (int64_t r = 0; r < mu; ++r)
      for (int64_t c = r + 1; c < mu; ++c)
        if (r / b == c / b) {
          const double v = 0.5 * (U[(size_t)r * cap + c] + U[(size_t)c * cap + r]);
          H[(size_t)r * mu + c] = H[(size_t)c * mu + r] = v;
        }
    Buf Hd, d, e, t, wk, lam;
    upload(Hd, H, st);
    d.alloc(mu * sizeof(double));
    e.alloc(mu * sizeof(double));
    t.alloc(mu * sizeof(double));
    wk.alloc(mu * sizeof(double));
    lam.alloc(mu * sizeof(double));
    SymItem si{Hd.as<double>(), (int)mu, (int)mu, d.as<double>(), e.as<double>(), t.as<double>(), wk.as<double>(),
               lam.as<double>(), nullptr};
    sym_eig_values(st, {si}, h->status.as<int>());
    std::vector<double> ev(mu);
    RFDD_CUDA(cudaMemcpyAsync(ev.data(), lam.p, mu * sizeof(double), cudaMemcpyDeviceToHost, st));
    RFDD_CUDA(cudaStreamSynchronize(st));
    return ev;
  };
  // line 0
  counter_uniform_dev(st, h->opt.seed, 7000, W.as<double>(), n * b);
  hmax = 1.0;
  morth(W.as<double>(), b, 0);
  hmax = 0.0;
  copy_rows_f64(st, W.as<double>(), b, Q, cap, n, b);
  int64_t col = 0, bc = b, steps = 0;
  const int64_t per_check = std::max<int64_t>(1, (10 + b - 1) / b);
  double last = NAN;
  std::vector<double> sums;
  int irmax = 0;
  while (true) {
    copy_rows_f64(st, Q + col, cap, Xb.as<double>(), bc, n, bc);
    spmm_f64(st, h->P, 0, n, 0, n, 0.0, 1.0, Xb.as<double>(), bc, V.as<double>(), bc, bc, false);
    irmax = std::max(irmax, refined_solve<Tf>(h, V.as<double>(), Xc.as<cx<double>>(), bc, ir_tol, fp64_res));
    weighted_real_sum<cx<double>>(st, Xc.as<cx<double>>(), n * bc, h->w_dev.as<cx<double>>(), nc, 2.0,
                                  W.as<double>(), n * bc);                                      // line 2
    const int64_t mu = col + bc;
    mproj(W.as<double>(), bc, mu, true, col);                                                   // lines 3-6
    ++steps;
    if (steps % per_check == 0 || mu >= cap) {                                                  // line 13
      const std::vector<double> ev = h_eigs(mu);
      double cur = 0.0;
      for (double x : ev)
        if (x >= 0.5) cur += x;
      sums.push_back(cur);
      RFDD_LOGF("rf-krylov: mu=%lld sum of eigenvalues >= 1/2 of H: %.12g", (long long)mu, cur);
      if (!std::isnan(last) && std::fabs(cur - last) <= h->opt.lanczos_tol * std::fabs(cur)) break;
      last = cur;
    }
    if (mu >= cap) break;
    const int64_t bn = std::min<int64_t>(b, cap - mu);                                          // lines 7-12
    if (bn < bc) {
      copy_rows_f64(st, W.as<double>(), bc, tmp.as<double>(), bn, n, bn);
      RFDD_CUDA(cudaMemcpyAsync(W.p, tmp.p, (size_t)n * bn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    morth(W.as<double>(), bn, mu);
    copy_rows_f64(st, W.as<double>(), bn, Q + mu, cap, n, bn);
    col = mu;
    bc = bn;
  }
  const int64_t mu = col + bc;
  h->mu = mu;
  res->info.mu = mu;
  res->info.ir_steps_max = std::max(res->info.ir_steps_max, irmax);
  h->traces = sums;
  // lines 15-16: Rayleigh-Ritz of (A, M) on range(Q_mu)
  Buf Y, C;
  Y.alloc((size_t)n * mu * sizeof(double));
  copy_rows_f64(st, Q, cap, Y.as<double>(), mu, n, mu);
  Qb.release();
  std::vector<int> sel;
  RRout rr = rayleigh_ritz_coeffs(
      h, Y.as<double>(), mu, 1e-12, 1e-9,
      [&](const std::vector<double> &th) {
        int64_t nin = 0;
        for (double x : th) nin += (x >= alpha && x <= beta);
        int64_t m = nin + std::max<int64_t>((int64_t)std::ceil(h->opt.guard_frac * nin), h->opt.min_guard);
        if (h->opt.m_align > 1) m = (m + h->opt.m_align - 1) / h->opt.m_align * h->opt.m_align;
        m = std::min<int64_t>((int64_t)th.size(), m);
        return select_nearest(th, alpha, beta, m);
      },
      C, sel);
  h->rr_theta = rr.theta;
  h->m0 = (int64_t)sel.size();
  h->X0.alloc((size_t)n * std::max<int64_t>(1, h->m0) * sizeof(double));
  if (h->m0 > 0)
    basis_gemm(h, {{Y.as<double>(), C.as<double>(), h->X0.as<double>(), (int)n, (int)h->m0, (int)mu, (int)mu,
                    (int)h->m0, (int)h->m0}},
               false, false, 1.0, 0.0);
  res->pre_evals.clear();
  for (double t : rr.theta)
    if (t >= alpha && t <= beta) res->pre_evals.push_back(t);
  res->info.k = rr.r;
  RFDD_CUDA(cudaStreamSynchronize(st));
}

void run_rfkrylov(rfdd_handle *h, double alpha, double beta, int nc, int64_t max_dim, rfdd_result *res) {
  RFDD_REQUIRE(beta > alpha && nc >= 1, RFDD_EINVAL, "rf-krylov: need alpha < beta and n_nodes >= 1");
  RFDD_REQUIRE(max_dim >= 0, RFDD_EINVAL, "rf-krylov: max_dim must be >= 0");
  Timer total(h->st);
  std::vector<cx<double>> z, w;
  quadrature(alpha, beta, nc, h->opt.quad_rule, z, w);
  if (h->opt.mem_budget > 0) {
    const size_t need = factor_bytes(h, nc);
    RFDD_REQUIRE(need <= h->opt.mem_budget, RFDD_EADMIT,
                 "rf-krylov needs " + std::to_string(need) + " bytes of factors, budget " +
                     std::to_string(h->opt.mem_budget));
  }
  std::vector<double> zz(2 * nc), ww(2 * nc);
  for (int l = 0; l < nc; ++l) {
    zz[2 * l] = z[l].re;
    zz[2 * l + 1] = z[l].im;
    ww[2 * l] = w[l].re;
    ww[2 * l + 1] = w[l].im;
  }
  set_nodes(h, nc, zz.data(), ww.data());
  h->alpha = alpha;
  h->beta = beta;
  h->have_interval = true;
  {
    Timer t(h->st);
    factor(h);
    res->info.t_factor_ms = t.ms();
    res->info.t_factor_enqueue_ms = h->factor_enqueue_ms;
    res->info.factor_launches = h->factor_launches;
    res->info.packed = h->pkB.empty() ? 0 : 1;
  }
  {
    Timer t(h->st);
    if (is_mixed(h)) rfkrylov_impl<cx<float>>(h, alpha, beta, max_dim, res);
    else rfkrylov_impl<cx<double>>(h, alpha, beta, max_dim, res);
    res->info.t_lanczos_ms = t.ms();
  }
  {
    Timer t(h->st);
    if (is_mixed(h)) complete<cx<float>>(h, alpha, beta, res);
    else complete<cx<double>>(h, alpha, beta, res);
    res->info.t_complete_ms = t.ms();
  }
  res->info.sigma = NAN;
  res->info.t_total_ms = total.ms();
}

void run_solve(rfdd_handle *h, double alpha, double beta, int nc, rfdd_result *res) {
  RFDD_REQUIRE(beta > alpha && nc >= 1, RFDD_EINVAL, "solve: need alpha < beta and n_nodes >= 1");
  Timer total(h->st);
  std::vector<cx<double>> z, w;
  quadrature(alpha, beta, nc, h->opt.quad_rule, z, w);
  if (h->opt.mem_budget > 0) {  // admission before any device work of the solve
    const size_t need = factor_bytes(h, nc);
    RFDD_REQUIRE(need <= h->opt.mem_budget, RFDD_EADMIT,
                 "solve needs " + std::to_string(need) + " bytes of factors, budget " +
                     std::to_string(h->opt.mem_budget));
  }
  std::vector<double> zz(2 * nc), ww(2 * nc);
  for (int l = 0; l < nc; ++l) {
    zz[2 * l] = z[l].re;
    zz[2 * l + 1] = z[l].im;
    ww[2 * l] = w[l].re;
    ww[2 * l + 1] = w[l].im;
  }
  set_nodes(h, nc, zz.data(), ww.data());
  h->alpha = alpha;
  h->beta = beta;
  h->have_interval = true;
  const double sigma = std::isnan(h->opt.sigma) ? 0.5 * (alpha + beta) : h->opt.sigma;
  {
    // the real B_sigma factorisation needs neither the complex factors nor the Lanczos basis:
    // start it on the second stream so that it fills the gaps of the next two steps
    if (!h->st2) {
      RFDD_CUDA(cudaStreamCreateWithFlags(&h->st2, cudaStreamNonBlocking));
      RFDD_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
      RFDD_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    }
    if (is_mixed(h)) interior_factor_start<float>(h, sigma, h->st2);
    else interior_factor_start<double>(h, sigma, h->st2);
  }
  {
    Timer t(h->st);
    factor(h);
    res->info.t_factor_ms = t.ms();
    res->info.t_factor_enqueue_ms = h->factor_enqueue_ms;
    res->info.factor_launches = h->factor_launches;
    res->info.packed = h->pkB.empty() ? 0 : 1;
  }
  {
    Timer t(h->st);
    if (is_mixed(h)) lanczos_impl<cx<float>>(h);
    else lanczos_impl<cx<double>>(h);
    res->info.t_lanczos_ms = t.ms();
    res->info.mu = h->mu;
  }
  {
    Timer t(h->st);
    // Guard on the shift: sigma at, or within tau max(1, |sigma|) of, an eigenvalue of some
    // pencil (B_j, M_B^(j)) leaves B_sigma (nearly) singular.  The shift then moves and the
    // interior step is redone, at most three times.  FP64 factors: tau = 1e-8, move
    // 1e-6 (beta - alpha).  FP32 factors (mixed) resolve B_sigma only to about 1e-7 relative, so
    // there tau = 1e-5 and the move is max(1e-3 (beta - alpha), 2 tau max(1, |sigma|)).
    const double tau = is_mixed(h) ? 1e-5 : 1e-8;
    double sig = sigma;
    for (int attempt = 0;; ++attempt) {
      bool near = false;
      try {
        if (is_mixed(h)) interior_impl<float>(h, sig);
        else interior_impl<double>(h, sig);
        near = h->interior_gap < tau * std::max(1.0, std::fabs(sig));
      } catch (const Error &e) {
        if (e.code != RFDD_ESINGULAR || attempt >= 3) throw;
        near = true;
      }
      if (!near || attempt >= 3) break;
      RFDD_LOGF("interior: sigma %.17g within %.3e of a subdomain eigenvalue, moved", sig, h->interior_gap);
      sig += is_mixed(h) ? std::max(1e-3 * (beta - alpha), 2.0 * tau * std::max(1.0, std::fabs(sig)))
                         : 1e-6 * (beta - alpha);
    }
    res->info.sigma = sig;
    res->info.t_interior_ms = t.ms();
  }
  {
    Timer t(h->st);
    if (is_mixed(h)) rr_on_Z<cx<float>>(h, alpha, beta, res);
    else rr_on_Z<cx<double>>(h, alpha, beta, res);
    res->info.t_rr_ms = t.ms();
  }
  {
    Timer t(h->st);
    if (is_mixed(h)) complete<cx<float>>(h, alpha, beta, res);
    else complete<cx<double>>(h, alpha, beta, res);
    res->info.t_complete_ms = t.ms();
  }
  res->info.t_total_ms = total.ms();
}

template <typename F>
int guarded(F &&f) {
  try {
    g_last_error.clear();
    f();
    return RFDD_OK;
  } catch (const Error &e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return RFDD_ENOMEM;
  } catch (const std::exception &e) {
    g_last_error = e.what();
    return RFDD_ECUDA;
  } catch (...) {  // nothing may unwind through the C ABI
    g_last_error = "unknown error";
    return RFDD_ECUDA;
  }
}

}  // namespace

// ======================================================================================
// C ABI
// ======================================================================================
extern "C" {

void rfdd_default_options(rfdd_options *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = RFDD_MIXED;
  o->quad_rule = RFDD_MIDPOINT;
  o->sigma = NAN;
  o->nev_b = 100;
  o->psi = 3;
  o->lanczos_tol = 1e-6;
  o->block = 32;
  o->res_tol = 1e-10;
  o->max_passes = 8;
  o->ir_max = 10;
  o->seed = 1;
  o->mem_budget = 0;
  o->stream = nullptr;
  o->guard_frac = 0.3;
  o->min_guard = 8;
  o->m_align = 128;
  o->pack_factors = -1;
  o->keep_schur = 0;
  o->subspace_iters = 4;
}

const char *rfdd_last_error(void) { return g_last_error.c_str(); }

const char *rfdd_status_string(int code) {
  switch (code) {
    case RFDD_OK: return "ok";
    case RFDD_EINVAL: return "invalid argument";
    case RFDD_ENOTSYM: return "matrix not symmetric";
    case RFDD_EPARTITION: return "invalid partition";
    case RFDD_ENOTSPD_M: return "M not positive definite";
    case RFDD_ESINGULAR: return "singular factorisation";
    case RFDD_ENOMEM: return "out of device memory";
    case RFDD_EADMIT: return "memory budget exceeded";
    case RFDD_NOT_CONVERGED: return "not converged";
    case RFDD_ECUDA: return "CUDA error";
    case RFDD_ESTATE: return "call out of order";
    default: return "unknown status";
  }
}

int rfdd_quadrature(double alpha, double beta, int32_t n_nodes, int32_t rule, double *z_out, double *w_out) {
  return guarded([&] {
    RFDD_REQUIRE(z_out && w_out, RFDD_EINVAL, "quadrature: NULL output");
    std::vector<cx<double>> z, w;
    quadrature(alpha, beta, n_nodes, rule, z, w);
    for (int l = 0; l < n_nodes; ++l) {
      z_out[2 * l] = z[l].re;
      z_out[2 * l + 1] = z[l].im;
      w_out[2 * l] = w[l].re;
      w_out[2 * l + 1] = w[l].im;
    }
  });
}

int rfdd_setup(const rfdd_csr *A, const rfdd_csr *M, const int32_t *part, int32_t p, const rfdd_options *opt,
               rfdd_handle **out) {
  if (!out) return RFDD_EINVAL;
  *out = nullptr;
  rfdd_handle *h = new (std::nothrow) rfdd_handle();
  if (!h) return RFDD_ENOMEM;
  HostCsrCopy hostA, hostM;
  int rc = guarded([&] {
    A = on_host(A, hostA, "A");
    M = on_host(M, hostM, "M");
    if (opt) h->opt = *opt;
    else rfdd_default_options(&h->opt);
    RFDD_REQUIRE(h->opt.precision == RFDD_FP64 || h->opt.precision == RFDD_MIXED, RFDD_EINVAL, "bad precision");
    RFDD_REQUIRE(h->opt.block >= 1 && h->opt.block <= 64, RFDD_EINVAL, "block must be in [1, 64]");
    RFDD_REQUIRE(h->opt.psi >= 1 && h->opt.nev_b >= 1, RFDD_EINVAL, "psi and nev_b must be >= 1");
    const auto t0 = std::chrono::steady_clock::now();
    do_setup(h, A, M, part, p);  // host-side validation and ordering (no CUDA calls)
    RFDD_LOGF("setup: host validation and ordering %.1f ms",
              std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
    if (h->opt.stream) {
      h->st = (cudaStream_t)h->opt.stream;
    } else {
      RFDD_CUDA(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
      h->own_stream = true;
    }
    keep_pool_memory();
    AllocScope scope(h->st);
    do_upload(h);
  });
  if (rc != RFDD_OK) {
    rfdd_destroy(h);
    return rc;
  }
  *out = h;
  return RFDD_OK;
}

int rfdd_layout(const rfdd_handle *h, int64_t *off, int64_t *perm, int32_t *p_out, int64_t *s_out) {
  if (!h) return RFDD_EINVAL;
  if (off) std::copy(h->off.begin(), h->off.end(), off);
  if (perm) std::copy(h->perm.begin(), h->perm.end(), perm);
  if (p_out) *p_out = h->p;
  if (s_out) *s_out = h->s;
  return RFDD_OK;
}

int rfdd_set_interface_groups(rfdd_handle *h, int32_t n_groups, const int32_t *group) {
  if (!h || n_groups < 0 || (n_groups > 0 && !group)) return RFDD_EINVAL;
  return guarded([&] {
    AllocScope scope(h->st);
    if (n_groups > 0) {
      RFDD_REQUIRE(!h->opt.keep_schur, RFDD_EINVAL, "keep_schur needs the dense interface factorisation");
      for (int j = 0; j < h->p; ++j)
        RFDD_REQUIRE(group[j] >= 0 && group[j] < n_groups, RFDD_EINVAL, "group label out of range");
    }
    interior_join(h, false);
    RFDD_CUDA(cudaStreamSynchronize(h->st));
    // the factors of the previous split are no longer valid
    for (Buf *b : {&h->fac, &h->pivB, &h->Sfac, &h->pivS, &h->Skeep, &h->BLinv, &h->BUinv, &h->SLinv, &h->SUinv,
                   &h->Pk, &h->Lfac, &h->pivL, &h->LLinv, &h->LUinv})
      b->release();
    h->pkB.clear();
    h->pkS.clear();
    h->pkG.clear();
    h->have_factors = false;
    build_levels(h, n_groups, group);
  });
}

int rfdd_interface_levels(const rfdd_handle *h, int32_t *cls, int64_t *s2) {
  if (!h) return RFDD_EINVAL;
  if (cls) {
    if (h->lv.G > 0) std::copy(h->lv.cls.begin(), h->lv.cls.end(), cls);
    else std::fill(cls, cls + h->s, -1);
  }
  if (s2) *s2 = h->lv.G > 0 ? h->lv.s2 : h->s;
  return RFDD_OK;
}

void rfdd_destroy(rfdd_handle *h) {
  if (!h) return;
  if (h->I_thread.joinable()) h->I_thread.join();
  if (h->st2) {
    cudaStreamSynchronize(h->st2);
    cudaStreamDestroy(h->st2);
    h->st2 = nullptr;
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->st) cudaStreamSynchronize(h->st);
  cudaStream_t st = h->st;
  bool own = h->own_stream;
  delete h;                            // enqueues the stream-ordered frees of its buffers on st
  if (st) cudaStreamSynchronize(st);
  if (own && st) cudaStreamDestroy(st);
}

int rfdd_release(rfdd_handle *h) {
  if (!h) return RFDD_EINVAL;
  return guarded([&] {
    interior_join(h, false);  // a started interior factorisation finishes before its buffers go
    RFDD_CUDA(cudaStreamSynchronize(h->st));
    if (h->st2) RFDD_CUDA(cudaStreamSynchronize(h->st2));
    for (Buf *b : {&h->fac, &h->boff_dev, &h->Doff_dev, &h->pivB, &h->Sfac, &h->pivS, &h->Skeep, &h->BLinv,
                   &h->BUinv, &h->SLinv, &h->SUinv, &h->Pk, &h->Lfac, &h->pivL, &h->LLinv, &h->LUinv, &h->IBs, &h->Ipiv, &h->IRLinv, &h->IRUinv, &h->I_doff,
                   &h->I_boffr_dev, &h->I_zs, &h->IVX, &h->IVGt, &h->Q, &h->Zb, &h->X0})
      b->release();
    h->have_factors = false;
    h->I_ready = false;
    h->mu = h->kz = h->kappa = h->m0 = 0;
    h->rr_theta.clear();
    RFDD_CUDA(cudaStreamSynchronize(h->st));
  });
}

int rfdd_factor(rfdd_handle *h, int32_t n_nodes, const double *z, const double *w) {
  if (!h || !z || !w || n_nodes < 1) return RFDD_EINVAL;
  return guarded([&] {
    AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
    set_nodes(h, n_nodes, z, w);
    factor(h);
  });
}

int rfdd_schur_copy(rfdd_handle *h, int32_t node, double *S_out) {
  if (!h || !S_out) return RFDD_EINVAL;
  return guarded([&] {
    AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
    RFDD_REQUIRE(h->have_factors && h->opt.keep_schur, RFDD_ESTATE, "schur_copy needs keep_schur and rfdd_factor");
    RFDD_REQUIRE(node >= 0 && node < h->nnodes, RFDD_EINVAL, "node out of range");
    const int64_t s = h->s;
    if (is_mixed(h)) {
      Buf t;
      t.alloc((size_t)s * s * sizeof(cx<double>));
      convert<cx<double>, cx<float>>(h->st, h->Skeep.as<cx<float>>() + (int64_t)node * s * s, t.as<cx<double>>(), s * s);
      RFDD_CUDA(cudaMemcpyAsync(S_out, t.p, (size_t)s * s * sizeof(cx<double>), cudaMemcpyDeviceToHost, h->st));
      RFDD_CUDA(cudaStreamSynchronize(h->st));
    } else {
      RFDD_CUDA(cudaMemcpyAsync(S_out, h->Skeep.as<cx<double>>() + (int64_t)node * s * s,
                                (size_t)s * s * sizeof(cx<double>), cudaMemcpyDeviceToHost, h->st));
      RFDD_CUDA(cudaStreamSynchronize(h->st));
    }
  });
}

int rfdd_shifted_solve(rfdd_handle *h, int32_t node, int32_t which, int32_t j, int64_t nrhs, const double *R,
                       double *X) {
  if (!h || !R || !X || nrhs < 1) return RFDD_EINVAL;
  return guarded([&] {
    AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
    RFDD_REQUIRE(h->have_factors, RFDD_ESTATE, "shifted_solve needs rfdd_factor");
    RFDD_REQUIRE(node >= 0 && node < h->nnodes, RFDD_EINVAL, "node out of range");
    cudaStream_t st = h->st;
    int64_t rows;
    if (which == 0) {
      RFDD_REQUIRE(j >= 0 && j < h->p, RFDD_EINVAL, "subdomain out of range");
      rows = h->d[j];
    } else if (which == 1) {
      rows = h->s;
    } else if (which == 2) {
      rows = h->n;
    } else {
      throw Error(RFDD_EINVAL, "which must be 0, 1 or 2");
    }
    Buf r64;
    r64.alloc((size_t)rows * nrhs * sizeof(cx<double>));
    RFDD_CUDA(cudaMemcpyAsync(r64.p, R, (size_t)rows * nrhs * sizeof(cx<double>), cudaMemcpyHostToDevice, st));
    auto go = [&](auto tag) {
      using Tf = decltype(tag);
      if (which == 2) {
        // (A - z_l M) X = R through the block inverse with FP64 refinement; every node is
        // solved on replicated input and node l is returned
        const int nc = h->nnodes;
        Buf Rall, Xall, Rr, Dx, F, Ht;
        Rall.alloc((size_t)nc * rows * nrhs * sizeof(cx<double>));
        for (int l = 0; l < nc; ++l)
          RFDD_CUDA(cudaMemcpyAsync(Rall.as<cx<double>>() + (int64_t)l * rows * nrhs, r64.p,
                                    (size_t)rows * nrhs * sizeof(cx<double>), cudaMemcpyDeviceToDevice, st));
        Xall.alloc((size_t)nc * rows * nrhs * sizeof(cx<double>));
        Rr.alloc((size_t)nc * rows * nrhs * sizeof(cx<double>));
        Dx.alloc((size_t)nc * rows * nrhs * sizeof(cx<double>));
        dd_solve<Tf>(h, Rall.as<cx<double>>(), rows * nrhs, Xall.as<cx<double>>(), nrhs, F, Ht);
        for (int it = 0; it < h->opt.ir_max; ++it) {
          shifted_residual(st, h->P, h->z_dev.as<cx<double>>(), nc, Rall.as<cx<double>>(), rows * nrhs,
                           Xall.as<cx<double>>(), Rr.as<cx<double>>(), rows * nrhs, nrhs);
          dd_solve<Tf>(h, Rr.as<cx<double>>(), rows * nrhs, Dx.as<cx<double>>(), nrhs, F, Ht);
          axpy_c64(st, Dx.as<cx<double>>(), Xall.as<cx<double>>(), (int64_t)nc * rows * nrhs);
        }
        RFDD_CUDA(cudaMemcpyAsync(X, Xall.as<cx<double>>() + (int64_t)node * rows * nrhs,
                                  (size_t)rows * nrhs * sizeof(cx<double>), cudaMemcpyDeviceToHost, st));
        RFDD_CUDA(cudaStreamSynchronize(st));
        return;
      }
      Buf t;
      t.alloc((size_t)rows * nrhs * sizeof(Tf));
      convert<Tf, cx<double>>(st, r64.as<cx<double>>(), t.as<Tf>(), rows * nrhs);
      std::vector<SolveItem<Tf>> si(1);
      if (which == 0) {
        si[0].LU = h->fac.as<Tf>() + h->boff[(size_t)node * h->p + j];
        si[0].piv = h->pivB.as<int>() + h->pivBoff[(size_t)node * h->p + j];
        si[0].n = (int)h->d[j];
        si[0].ld = (int)h->D[j];
        attach_binv(h, si[0], node, j);
        si[0].X = t.as<Tf>();
        si[0].ldx = (int)nrhs;
        si[0].ncols = (int)nrhs;
        lu_solve_batched<Tf>(st, si, NBO);
      } else {
        solve_S<Tf>(h, t.as<Tf>(), nrhs, 0, nrhs, std::vector<int>{(int)node});
      }
      convert<cx<double>, Tf>(st, t.as<Tf>(), r64.as<cx<double>>(), rows * nrhs);
      RFDD_CUDA(cudaMemcpyAsync(X, r64.p, (size_t)rows * nrhs * sizeof(cx<double>), cudaMemcpyDeviceToHost, st));
      RFDD_CUDA(cudaStreamSynchronize(st));
    };
    if (is_mixed(h)) go(cx<float>());
    else go(cx<double>());
  });
}

int rfdd_filter_apply(rfdd_handle *h, int64_t b, const double *X, double *W) {
  if (!h || !X || !W || b < 1) return RFDD_EINVAL;
  return guarded([&] {
    AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
    RFDD_REQUIRE(h->have_factors, RFDD_ESTATE, "filter_apply needs rfdd_factor");
    const int64_t s = h->s;
    Buf x, wv;
    x.alloc((size_t)s * b * sizeof(double));
    wv.alloc((size_t)s * b * sizeof(double));
    RFDD_CUDA(cudaMemcpyAsync(x.p, X, (size_t)s * b * sizeof(double), cudaMemcpyHostToDevice, h->st));
    if (is_mixed(h)) filter_impl<cx<float>>(h, x.as<double>(), wv.as<double>(), b, 1.0);
    else filter_impl<cx<double>>(h, x.as<double>(), wv.as<double>(), b, 1.0);
    RFDD_CUDA(cudaMemcpyAsync(W, wv.p, (size_t)s * b * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    RFDD_CUDA(cudaStreamSynchronize(h->st));
  });
}

int rfdd_lanczos(rfdd_handle *h, int64_t cap, double *Q_out, int64_t *mu, double *traces, int32_t *nsteps) {
  if (!h) return RFDD_EINVAL;
  return guarded([&] {
    AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
    RFDD_REQUIRE(h->have_factors, RFDD_ESTATE, "lanczos needs rfdd_factor");
    if (is_mixed(h)) lanczos_impl<cx<float>>(h);
    else lanczos_impl<cx<double>>(h);
    if (mu) *mu = h->mu;
    if (nsteps) *nsteps = (int32_t)h->traces.size();
    if (traces)
      for (int64_t i = 0; i < (int64_t)h->traces.size() && i < cap; ++i) traces[i] = h->traces[i];
    if (Q_out) {
      RFDD_REQUIRE(cap >= h->mu, RFDD_EINVAL, "lanczos: cap smaller than the basis");
      Buf q;
      q.alloc((size_t)h->s * h->mu * sizeof(double));
      copy_rows_f64(h->st, h->Q.as<double>(), h->qcap, q.as<double>(), h->mu, h->s, h->mu);
      std::vector<double> tmp((size_t)h->s * h->mu);
      RFDD_CUDA(cudaMemcpyAsync(tmp.data(), q.p, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      RFDD_CUDA(cudaStreamSynchronize(h->st));
      for (int64_t i = 0; i < h->s; ++i)
        std::copy(tmp.begin() + i * h->mu, tmp.begin() + (i + 1) * h->mu, Q_out + i * cap);
    }
  });
}

int rfdd_interior(rfdd_handle *h, double sigma, int64_t cap, double *Z_out, int64_t *k, int64_t *kappa_out) {
  if (!h) return RFDD_EINVAL;
  return guarded([&] {
    AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
    RFDD_REQUIRE(h->mu > 0, RFDD_ESTATE, "interior needs rfdd_lanczos");
    double sg = sigma;
    if (std::isnan(sg)) sg = h->have_interval ? 0.5 * (h->alpha + h->beta) : 0.0;
    if (is_mixed(h)) interior_impl<float>(h, sg);
    else interior_impl<double>(h, sg);
    if (k) *k = h->kz;
    if (kappa_out) *kappa_out = h->kappa;
    if (Z_out) {
      RFDD_REQUIRE(cap >= h->kz, RFDD_EINVAL, "interior: cap smaller than the number of columns");
      std::vector<double> tmp((size_t)h->n * h->kz);
      RFDD_CUDA(cudaMemcpyAsync(tmp.data(), h->Zb.p, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      RFDD_CUDA(cudaStreamSynchronize(h->st));
      for (int64_t i = 0; i < h->n; ++i)
        std::copy(tmp.begin() + i * h->kz, tmp.begin() + (i + 1) * h->kz, Z_out + i * cap);
    }
  });
}

int rfdd_rayleigh_ritz(rfdd_handle *h, int64_t cap, double *theta_out, int64_t *k) {
  if (!h) return RFDD_EINVAL;
  return guarded([&] {
    AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
    RFDD_REQUIRE(h->kz > 0, RFDD_ESTATE, "rayleigh_ritz needs rfdd_interior");
    const double a = h->have_interval ? h->alpha : -INFINITY, b = h->have_interval ? h->beta : INFINITY;
    if (is_mixed(h)) rr_on_Z<cx<float>>(h, a, b, nullptr);
    else rr_on_Z<cx<double>>(h, a, b, nullptr);
    if (k) *k = (int64_t)h->rr_theta.size();
    if (theta_out)
      for (int64_t i = 0; i < (int64_t)h->rr_theta.size() && i < cap; ++i) theta_out[i] = h->rr_theta[i];
  });
}

int rfdd_inertia(rfdd_handle *h, double sigma, int64_t *count) {
  if (!h || !count || !std::isfinite(sigma)) return RFDD_EINVAL;
  return guarded([&] {
    AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
    *count = inertia_impl(h, sigma);
  });
}

int rfdd_polish(rfdd_handle *h, int64_t nev, double *lambda, double *X, double *resid) {
  if (!h || nev < 0 || (nev > 0 && (!lambda || !X || !resid))) return RFDD_EINVAL;
  if (nev == 0) return RFDD_OK;
  return guarded([&] {
    AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
    interior_join(h, false);  // nothing of a failed solve may still be running on the second stream
    polish_impl(h, nev, lambda, X, resid);
  });
}

int rfdd_solve(rfdd_handle *h, double alpha, double beta, int32_t n_nodes, rfdd_result **out) {
  if (!h || !out) return RFDD_EINVAL;
  *out = nullptr;
  rfdd_result *r = new (std::nothrow) rfdd_result();
  if (!r) return RFDD_ENOMEM;
  int rc = guarded([&] {
    AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
    run_solve(h, alpha, beta, n_nodes, r);
  });
  if (rc != RFDD_OK) {
    delete r;
    return rc;
  }
  *out = r;
  return r->info.status;
}

int rfdd_rfkrylov(rfdd_handle *h, double alpha, double beta, int32_t n_nodes, int64_t max_dim, rfdd_result **out) {
  if (!h || !out) return RFDD_EINVAL;
  *out = nullptr;
  rfdd_result *r = new (std::nothrow) rfdd_result();
  if (!r) return RFDD_ENOMEM;
  int rc = guarded([&] {
    AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
    run_rfkrylov(h, alpha, beta, n_nodes, max_dim, r);
  });
  if (rc != RFDD_OK) {
    delete r;
    return rc;
  }
  *out = r;
  return r->info.status;
}

int rfdd_solve_async(rfdd_handle *h, double alpha, double beta, int32_t n_nodes, void *stream, rfdd_result **out) {
  if (!h || !out) return RFDD_EINVAL;
  *out = nullptr;
  if (!(beta > alpha) || n_nodes < 1) return RFDD_EINVAL;
  rfdd_result *r = new (std::nothrow) rfdd_result();
  if (!r) return RFDD_ENOMEM;
  if (stream) h->st = (cudaStream_t)stream;
  r->ready.store(0);
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    device = 0;
  }
  r->worker = std::thread([h, alpha, beta, n_nodes, r, device] {
    int rc = guarded([&] {
      RFDD_CUDA(cudaSetDevice(device));
      AllocScope scope(h->st);
    TcStatusScope tcs(h->status.as<int>());
      run_solve(h, alpha, beta, n_nodes, r);
    });
    if (rc != RFDD_OK) r->ready.store(-rc);
    else r->ready.store(1);
  });
  *out = r;
  return RFDD_OK;
}

int rfdd_result_ready(const rfdd_result *r) {
  if (!r) return -RFDD_EINVAL;
  return r->ready.load();
}

int rfdd_result_get(const rfdd_result *r_, int64_t *nev, const double **evals, const double **evecs,
                    const double **resid, int32_t device) {
  rfdd_result *r = const_cast<rfdd_result *>(r_);
  if (!r) return RFDD_EINVAL;
  if (r->ready.load() != 1) return r->ready.load() < 0 ? -r->ready.load() : RFDD_ESTATE;
  return guarded([&] {
    if (nev) *nev = r->nev;
    if (device) {
      if (evals) *evals = r->evals_dev.as<double>();
      if (evecs) *evecs = r->evecs.as<double>();
      if (resid) *resid = r->resid_dev.as<double>();
    } else {
      if (evecs && !r->host_ready) {
        r->evecs_host.resize((size_t)r->n * r->nev);
        if (!r->evecs_host.empty())
          RFDD_CUDA(cudaMemcpy(r->evecs_host.data(), r->evecs.p, r->evecs_host.size() * sizeof(double),
                               cudaMemcpyDeviceToHost));
        r->host_ready = true;
      }
      if (evals) *evals = r->evals.data();
      if (evecs) *evecs = r->evecs_host.data();
      if (resid) *resid = r->resid.data();
    }
  });
}

int rfdd_result_info(const rfdd_result *r, rfdd_info *info) {
  if (!r || !info) return RFDD_EINVAL;
  *info = r->info;
  return RFDD_OK;
}

int rfdd_result_pre_evals(const rfdd_result *r, int64_t *count, double *vals) {
  if (!r || !count) return RFDD_EINVAL;
  *count = (int64_t)r->pre_evals.size();
  if (vals) std::copy(r->pre_evals.begin(), r->pre_evals.end(), vals);
  return RFDD_OK;
}

void rfdd_result_free(rfdd_result *r) { delete r; }

int rfdd_sym_eig(int64_t n, const double *H, double *evals, double *evecs) {
  if (n < 1 || !H || !evals || !evecs) return RFDD_EINVAL;
  return guarded([&] {
    cudaStream_t st = 0;
    Buf Hd, d, e, t, w, lam, Z, out, status;
    Hd.alloc((size_t)n * n * sizeof(double));
    RFDD_CUDA(cudaMemcpy(Hd.p, H, (size_t)n * n * sizeof(double), cudaMemcpyHostToDevice));
    d.alloc(n * sizeof(double));
    e.alloc(n * sizeof(double));
    t.alloc(n * sizeof(double));
    w.alloc(n * sizeof(double));
    lam.alloc(n * sizeof(double));
    Z.alloc((size_t)n * n * sizeof(double));
    status.alloc(sizeof(int));
    RFDD_CUDA(cudaMemset(status.p, 0, sizeof(int)));
    SymItem si{Hd.as<double>(), (int)n, (int)n, d.as<double>(), e.as<double>(), t.as<double>(), w.as<double>(),
               lam.as<double>(), Z.as<double>()};
    sym_eig_values(st, {si}, status.as<int>());
    std::vector<int> all(n);
    std::iota(all.begin(), all.end(), 0);
    out.alloc((size_t)n * n * sizeof(double));
    sym_eig_vectors(st, {BackItem{&si, all, out.as<double>(), (int)n}}, 1e-5);
    RFDD_CUDA(cudaStreamSynchronize(st));
    int stt = 0;
    RFDD_CUDA(cudaMemcpy(&stt, status.p, sizeof(int), cudaMemcpyDeviceToHost));
    RFDD_REQUIRE(stt == 0, RFDD_ESINGULAR, "sym_eig: eigensolver reported a failure");
    RFDD_CUDA(cudaMemcpy(evals, lam.p, n * sizeof(double), cudaMemcpyDeviceToHost));
    RFDD_CUDA(cudaMemcpy(evecs, out.p, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToHost));
  });
}

int rfdd_cgemm(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B, int64_t ldb, float *C,
               int64_t ldc, double alpha, double beta, int32_t engine) {
  if (m < 1 || n < 1 || k < 1 || !A || !B || !C || lda < k || ldb < n || ldc < n) return RFDD_EINVAL;
  if (engine < 0 || engine > 3) return RFDD_EINVAL;
  return guarded([&] {
    cudaStream_t st = 0;
    Buf a, b, c;
    a.alloc((size_t)m * lda * sizeof(cx<float>));
    b.alloc((size_t)k * ldb * sizeof(cx<float>));
    c.alloc((size_t)m * ldc * sizeof(cx<float>));
    RFDD_CUDA(cudaMemcpy(a.p, A, (size_t)m * lda * sizeof(cx<float>), cudaMemcpyHostToDevice));
    RFDD_CUDA(cudaMemcpy(b.p, B, (size_t)k * ldb * sizeof(cx<float>), cudaMemcpyHostToDevice));
    RFDD_CUDA(cudaMemcpy(c.p, C, (size_t)m * ldc * sizeof(cx<float>), cudaMemcpyHostToDevice));
    std::vector<GemmItem<cx<float>>> it = {{a.as<cx<float>>(), b.as<cx<float>>(), c.as<cx<float>>(), (int)m, (int)n,
                                            (int)k, (int)lda, (int)ldb, (int)ldc}};
    Buf status;
    status.alloc(sizeof(int));
    RFDD_CUDA(cudaMemset(status.p, 0, sizeof(int)));
    if (engine >= 1 && engine <= 3) {
      TcStatusScope tcs(status.as<int>());
      TcEngineScope eng(engine == 2 ? 1 : engine == 3 ? 2 : 0);
      tc_gemm_complex(st, it, alpha, beta);
    } else {
      gemm_simt_batched<cx<float>>(st, it, false, false, alpha, beta);
    }
    RFDD_CUDA(cudaStreamSynchronize(st));
    int stt = 0;
    RFDD_CUDA(cudaMemcpy(&stt, status.p, sizeof(int), cudaMemcpyDeviceToHost));
    RFDD_REQUIRE(stt == 0, RFDD_ECUDA, "tensor-core GEMM reported a time-out");
    RFDD_CUDA(cudaMemcpy(C, c.p, (size_t)m * ldc * sizeof(cx<float>), cudaMemcpyDeviceToHost));
  });
}

int rfdd_dgemm(int64_t m, int64_t n, int64_t k, int32_t ta, const double *A, int64_t lda, int32_t tb, const double *B,
               int64_t ldb, double *C, int64_t ldc, double alpha, double beta, int32_t engine, int32_t sym) {
  if (m < 1 || n < 1 || k < 1 || !A || !B || !C || ldc < n) return RFDD_EINVAL;
  if (lda < (ta ? m : k) || ldb < (tb ? k : n)) return RFDD_EINVAL;
  if (sym && m != n) return RFDD_EINVAL;
  return guarded([&] {
    cudaStream_t st = 0;
    const size_t na = (size_t)(ta ? k : m) * lda, nb = (size_t)(tb ? n : k) * ldb, ncm = (size_t)m * ldc;
    Buf a, b, c;
    a.alloc(na * sizeof(double));
    b.alloc(nb * sizeof(double));
    c.alloc(ncm * sizeof(double));
    RFDD_CUDA(cudaMemcpy(a.p, A, na * sizeof(double), cudaMemcpyHostToDevice));
    RFDD_CUDA(cudaMemcpy(b.p, B, nb * sizeof(double), cudaMemcpyHostToDevice));
    RFDD_CUDA(cudaMemcpy(c.p, C, ncm * sizeof(double), cudaMemcpyHostToDevice));
    std::vector<GemmItem<double>> it = {
        {a.as<double>(), b.as<double>(), c.as<double>(), (int)m, (int)n, (int)k, (int)lda, (int)ldb, (int)ldc}};
    if (engine == 1) gemm_f64x2_batched(st, it, ta != 0, tb != 0, alpha, beta, {(char)(sym != 0)});
    else gemm_simt_batched<double>(st, it, ta != 0, tb != 0, alpha, beta, {(char)(sym != 0)});
    RFDD_CUDA(cudaStreamSynchronize(st));
    RFDD_CUDA(cudaMemcpy(C, c.p, ncm * sizeof(double), cudaMemcpyDeviceToHost));
  });
}

int rfdd_autotune(int32_t mode) {
  if (mode < 0 || mode > 2) return -RFDD_EINVAL;
  return tc_autotune(mode);
}

int rfdd_autotune_table(char *buf, int64_t cap, int64_t *len) {
  if (!len || cap < 0 || (cap > 0 && !buf)) return RFDD_EINVAL;
  return guarded([&] {
    const std::string t = tc_autotune_table();
    *len = (int64_t)t.size();
    if (cap > 0) {
      const size_t c = std::min<size_t>((size_t)cap - 1, t.size());
      memcpy(buf, t.data(), c);
      buf[c] = 0;
    }
  });
}

int rfdd_cgemm_noalloc(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B, int64_t ldb,
                       float *C, int64_t ldc, double alpha, double beta, void *stream) {
  if (!A || !B || !C || lda < k || ldb < n || ldc < n) return RFDD_EINVAL;
  return guarded([&] {
    cudaStream_t st = (cudaStream_t)stream;
    const int stt = tc_gemm_complex_noalloc(
        st, reinterpret_cast<const cx<float> *>(A), lda, reinterpret_cast<const cx<float> *>(B), ldb,
        reinterpret_cast<cx<float> *>(C), ldc, (int)std::min<int64_t>(m, INT32_MAX),
        (int)std::min<int64_t>(n, INT32_MAX), (int)std::min<int64_t>(k, INT32_MAX), alpha, beta);
    RFDD_REQUIRE(stt == 0, RFDD_ECUDA, "tensor-core GEMM reported a time-out");
  });
}

int rfdd_peak_probe(int32_t which, double *tflops) {
  if (!tflops) return RFDD_EINVAL;
  return guarded([&] { *tflops = peak_probe(which); });
}

long long rfdd_kernel_launches(void) { return g_kernel_launches.load(); }

int rfdd_profile(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto &r : g_prof) {
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof.clear();
  if (enable) {
    // time origin for rfdd_profile_busy: recorded and completed before any launch that follows
    return guarded([&] {
      if (!g_prof_ref) RFDD_CUDA(cudaEventCreate(&g_prof_ref));
      RFDD_CUDA(cudaEventRecord(g_prof_ref, 0));
      RFDD_CUDA(cudaEventSynchronize(g_prof_ref));
      g_prof_on = true;
    });
  }
  g_prof_on = false;
  return RFDD_OK;
}

int rfdd_profile_busy(int32_t kind, double *busy_ms) {
  if (!busy_ms) return RFDD_EINVAL;
  return guarded([&] {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    *busy_ms = 0.0;
    std::vector<std::pair<double, double>> iv;
    for (auto &r : g_prof) {
      if (r.kind != kind) continue;
      RFDD_REQUIRE(g_prof_ref, RFDD_ESTATE, "profile_busy: no recording started");
      RFDD_CUDA(cudaEventSynchronize(r.b));
      float a = 0.f, b = 0.f;
      RFDD_CUDA(cudaEventElapsedTime(&a, g_prof_ref, r.a));
      RFDD_CUDA(cudaEventElapsedTime(&b, g_prof_ref, r.b));
      iv.push_back({(double)a, (double)std::max(a, b)});
    }
    std::sort(iv.begin(), iv.end());
    double lo = 0.0, hi = -1.0;  // the current merged interval
    for (auto &x : iv) {
      if (x.first > hi) {
        if (hi > lo) *busy_ms += hi - lo;
        lo = x.first;
        hi = x.second;
      } else {
        hi = std::max(hi, x.second);
      }
    }
    if (hi > lo) *busy_ms += hi - lo;
  });
}

int rfdd_profile_get(int32_t kind, int64_t *launches, double *ms, double *flops) {
  if (!launches || !ms || !flops) return RFDD_EINVAL;
  return guarded([&] {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    *launches = 0;
    *ms = 0.0;
    *flops = 0.0;
    for (auto &r : g_prof) {
      if (r.kind != kind) continue;
      RFDD_CUDA(cudaEventSynchronize(r.b));
      float t = 0.f;
      RFDD_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
      *launches += 1;
      *ms += t;
      *flops += r.flops;
    }
  });
}

int rfdd_profile_bytes(int32_t kind, double *bytes) {
  if (!bytes) return RFDD_EINVAL;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  *bytes = 0.0;
  for (auto &r : g_prof)
    if (r.kind == kind) *bytes += r.bytes;
  return RFDD_OK;
}

int rfdd_memory_estimate(const rfdd_handle *h, int32_t n_nodes, int64_t nev_guess, size_t *bytes) {
  if (!h || !bytes || n_nodes < 1 || nev_guess < 0) return RFDD_EINVAL;
  *bytes = rfdd::solve_bytes_of(shape_of(h), n_nodes, nev_guess, false);
  return RFDD_OK;
}

}  // extern "C"
