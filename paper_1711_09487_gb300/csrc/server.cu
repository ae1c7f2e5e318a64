// Serving loop: continuous batching of eigenvalue-interval requests on one GPU.
//
// The interval problem of Section 1 (every eigenpair of A x = lambda M x in [alpha, beta]) asked
// by many clients at once.  Pencils are set up once and stay resident on the device (their
// ordering, blocks and maps: rfdd_setup); requests name a resident pencil and an interval.  A
// fixed set of worker threads, each solving on the stream of the pencil's handle, takes waiting
// requests as slots and device memory free up (serve_policy.h): work of different requests
// overlaps on the device, and a request that arrives while others run starts as soon as its
// memory estimate (rfdd_memory_estimate) fits in the budget.  After a solve the handle's factors
// are released (rfdd_release), so a resident pencil holds only its set-up between requests.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "serve_policy.h"

using Clock = std::chrono::steady_clock;

namespace {

struct HostCsr {
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  void copy(const rfdd_csr &a) {
    rowptr.assign(a.rowptr, a.rowptr + a.n + 1);
    col.assign(a.col, a.col + rowptr.back());
    val.assign(a.val, a.val + rowptr.back());
  }
  rfdd_csr view() const { return rfdd_csr{(int64_t)rowptr.size() - 1, rowptr.data(), col.data(), val.data(), 0}; }
};

struct SPencil {
  rfdd_handle *h = nullptr;
  bool busy = false;    // a request of this pencil is running (a handle serves one solve at a time)
  int pending = 0;      // requests waiting or running
  // a pencil that came with its request (rfdd_server_submit_pencil): host copies, set up by the
  // worker that runs the request and destroyed after it
  bool one_shot = false;
  HostCsr A, M;
  std::vector<int32_t> part;
  int32_t p = 0;
  rfdd_options opt{};
};

// Sizes of the interior-first blocks of a pencil from its host CSR (d_j, s, s_j), for the
// admission estimate of a request whose pencil is not set up yet.  RFDD_EINVAL on labels or
// columns out of range.
int shape_from_csr(const rfdd_csr &A, const rfdd_csr &M, const int32_t *part, int32_t p, std::vector<int64_t> &d,
                   std::vector<int64_t> &D, int64_t &s, int64_t &nnz) {
  const int64_t n = A.n;
  if (n < 1 || M.n != n || p < 1 || !A.rowptr || !A.col || !M.rowptr || !M.col || !part) return RFDD_EINVAL;
  d.assign(p, 0);
  s = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (part[i] < -1 || part[i] >= p) return RFDD_EINVAL;
    if (part[i] < 0) ++s;
    else ++d[part[i]];
  }
  std::vector<std::vector<int64_t>> adj(p);
  for (const rfdd_csr *X : {&A, &M})
    for (int64_t i = 0; i < n; ++i) {
      if (part[i] < 0) continue;
      for (int64_t e = X->rowptr[i]; e < X->rowptr[i + 1]; ++e) {
        const int64_t c = X->col[e];
        if (c < 0 || c >= n) return RFDD_EINVAL;
        if (part[c] < 0) adj[part[i]].push_back(c);
      }
    }
  D.assign(p, 0);
  for (int j = 0; j < p; ++j) {
    std::sort(adj[j].begin(), adj[j].end());
    D[j] = d[j] + (int64_t)(std::unique(adj[j].begin(), adj[j].end()) - adj[j].begin());
  }
  nnz = A.rowptr[n] + M.rowptr[n];
  return RFDD_OK;
}

constexpr int32_t REQ_WAITING = -1, REQ_RUNNING = -2;

struct SRequest {
  int64_t pencil = -1;
  double alpha = 0, beta = 0;
  int32_t nc = 0;
  size_t bytes = 0;
  int32_t status = REQ_WAITING;
  rfdd_result *res = nullptr;
  bool taken = false;
  int64_t nev = 0;
  Clock::time_point t_submit, t_start, t_done;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct rfdd_server {
  rfdd_server_options opt{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<int64_t, SPencil> pencils;
  std::map<int64_t, SRequest> reqs;
  std::deque<int64_t> queue;  // waiting request ids in arrival order
  rfdd::serve::State st;
  std::vector<std::thread> workers;
  bool stop = false;
  int64_t next_pencil = 0, next_req = 0;
  int64_t completed = 0, failed = 0;
  int peak_running = 0;
  size_t peak_in_use = 0;

  void worker_loop();
};

void rfdd_server::worker_loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    int64_t rid = -1;
    while (!stop) {
      std::vector<rfdd::serve::Waiting> w;
      w.reserve(queue.size());
      for (int64_t id : queue) w.push_back({id, reqs[id].pencil, reqs[id].bytes});
      const int i = rfdd::serve::pick_next(w, st, [&](int64_t pid) { return pencils[pid].busy; });
      if (i >= 0) {
        rid = w[i].id;
        queue.erase(queue.begin() + i);
        break;
      }
      cv_work.wait(lk);
    }
    if (rid < 0) return;  // stopping
    SRequest &r = reqs[rid];
    SPencil &pc = pencils[r.pencil];
    pc.busy = true;
    r.status = REQ_RUNNING;
    r.t_start = Clock::now();
    st.in_use += r.bytes;
    st.running += 1;
    peak_running = std::max(peak_running, st.running);
    peak_in_use = std::max(peak_in_use, st.in_use);
    rfdd_handle *h = pc.h;
    const bool one_shot = pc.one_shot;
    const double a = r.alpha, b = r.beta;
    const int32_t nc = r.nc;
    lk.unlock();
    rfdd_result *res = nullptr;
    int rc = RFDD_OK;
    if (one_shot) {  // the pencil's set-up is part of this request
      const rfdd_csr Av = pc.A.view(), Mv = pc.M.view();
      rc = rfdd_setup(&Av, &Mv, pc.part.data(), pc.p, &pc.opt, &h);
    }
    if (rc == RFDD_OK) {
      rc = rfdd_solve(h, a, b, nc, &res);
      if (one_shot) rfdd_destroy(h);
      else rfdd_release(h);  // the factors go; the pencil's set-up stays resident
    }
    int64_t nev = 0;
    if (res) rfdd_result_get(res, &nev, nullptr, nullptr, nullptr, 0);
    lk.lock();
    SRequest &rr = reqs[rid];
    rr.status = rc;
    rr.res = res;
    rr.nev = nev;
    rr.t_done = Clock::now();
    SPencil &pp = pencils[rr.pencil];
    pp.busy = false;
    pp.pending -= 1;
    if (pp.one_shot) pencils.erase(rr.pencil);
    st.in_use -= rr.bytes;
    st.running -= 1;
    if (rc == RFDD_OK || rc == RFDD_NOT_CONVERGED) completed += 1;
    else failed += 1;
    cv_work.notify_all();
    cv_done.notify_all();
  }
}

extern "C" {

void rfdd_server_default_options(rfdd_server_options *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->mem_budget = (size_t)150 << 30;
  o->max_inflight = 4;
  o->max_bypass = 8;
  o->device = -1;
}

int rfdd_server_create(const rfdd_server_options *o, rfdd_server **out) {
  if (!out) return RFDD_EINVAL;
  *out = nullptr;
  rfdd_server_options opt;
  if (o) opt = *o;
  else rfdd_server_default_options(&opt);
  if (opt.max_inflight < 1 || opt.max_inflight > 64 || opt.mem_budget == 0 || opt.max_bypass < 0)
    return RFDD_EINVAL;
  rfdd_server *s = new (std::nothrow) rfdd_server();
  if (!s) return RFDD_ENOMEM;
  s->opt = opt;
  if (opt.device >= 0) {
    s->device = opt.device;
  } else if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return RFDD_ECUDA;
  }
  s->st.budget = opt.mem_budget;
  s->st.max_inflight = opt.max_inflight;
  s->st.max_bypass = opt.max_bypass;
  try {
    for (int i = 0; i < opt.max_inflight; ++i) s->workers.emplace_back([s] { s->worker_loop(); });
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    delete s;
    return RFDD_ENOMEM;
  }
  *out = s;
  return RFDD_OK;
}

int rfdd_server_add_pencil(rfdd_server *s, const rfdd_csr *A, const rfdd_csr *M, const int32_t *part, int32_t p,
                           const rfdd_options *opt, int64_t *pencil_id) {
  if (!s || !pencil_id) return RFDD_EINVAL;
  rfdd_options o;
  if (opt) o = *opt;
  else rfdd_default_options(&o);
  o.stream = nullptr;  // every resident pencil solves on a stream of its own handle
  // a request may hold at most the server's budget: its factor form follows from that (pack_factors)
  if (o.mem_budget == 0 || o.mem_budget > s->opt.mem_budget) o.mem_budget = s->opt.mem_budget;
  if (cudaSetDevice(s->device) != cudaSuccess) {
    cudaGetLastError();
    return RFDD_ECUDA;
  }
  rfdd_handle *h = nullptr;
  const int rc = rfdd_setup(A, M, part, p, &o, &h);
  if (rc != RFDD_OK) return rc;
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t id = s->next_pencil++;
  s->pencils[id].h = h;
  *pencil_id = id;
  return RFDD_OK;
}

int rfdd_server_submit(rfdd_server *s, int64_t pencil_id, double alpha, double beta, int32_t n_nodes, int64_t nev_hint,
                       int64_t *request_id) {
  if (!s || !request_id || !(beta > alpha) || n_nodes < 1 || nev_hint < 0) return RFDD_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->pencils.find(pencil_id);
  if (it == s->pencils.end()) return RFDD_EINVAL;
  size_t bytes = 0;
  const int rc = rfdd_memory_estimate(it->second.h, n_nodes, nev_hint > 0 ? nev_hint : 100, &bytes);
  if (rc != RFDD_OK) return rc;
  if (bytes > s->st.budget) return RFDD_EADMIT;  // could never start
  const int64_t id = s->next_req++;
  SRequest &r = s->reqs[id];
  r.pencil = pencil_id;
  r.alpha = alpha;
  r.beta = beta;
  r.nc = n_nodes;
  r.bytes = bytes;
  r.t_submit = Clock::now();
  it->second.pending += 1;
  s->queue.push_back(id);
  *request_id = id;
  lk.unlock();
  s->cv_work.notify_all();
  return RFDD_OK;
}

int rfdd_server_submit_pencil(rfdd_server *s, const rfdd_csr *A, const rfdd_csr *M, const int32_t *part, int32_t p,
                              const rfdd_options *opt, double alpha, double beta, int32_t n_nodes, int64_t nev_hint,
                              int64_t *request_id) {
  if (!s || !A || !M || !request_id || !(beta > alpha) || n_nodes < 1 || nev_hint < 0) return RFDD_EINVAL;
  if (A->location != 0 || M->location != 0) return RFDD_EINVAL;  // requests bring host copies
  rfdd_options o;
  if (opt) o = *opt;
  else rfdd_default_options(&o);
  o.stream = nullptr;
  if (o.mem_budget == 0 || o.mem_budget > s->opt.mem_budget) o.mem_budget = s->opt.mem_budget;
  std::vector<int64_t> d, D;
  int64_t sz = 0, nnz = 0;
  int rc = shape_from_csr(*A, *M, part, p, d, D, sz, nnz);
  if (rc != RFDD_OK) return rc;
  rfdd::SolveShape g;
  g.n = A->n;
  g.s = sz;
  g.p = p;
  g.nnz = nnz;
  g.d = d.data();
  g.D = D.data();
  g.precision = o.precision;
  g.keep_schur = o.keep_schur;
  g.guard_frac = o.guard_frac;
  g.min_guard = o.min_guard;
  g.m_align = o.m_align;
  g.pack_factors = o.pack_factors;
  g.mem_budget = o.mem_budget;
  const size_t bytes = rfdd::solve_bytes_of(g, n_nodes, nev_hint > 0 ? nev_hint : 100, true);
  if (bytes > s->opt.mem_budget) return RFDD_EADMIT;  // could never start
  SPencil pc;
  pc.one_shot = true;
  pc.A.copy(*A);
  pc.M.copy(*M);
  pc.part.assign(part, part + A->n);
  pc.p = p;
  pc.opt = o;
  std::unique_lock<std::mutex> lk(s->mu);
  const int64_t pid = s->next_pencil++;
  SPencil &stored = s->pencils[pid];
  stored = std::move(pc);
  stored.pending = 1;
  const int64_t id = s->next_req++;
  SRequest &r = s->reqs[id];
  r.pencil = pid;
  r.alpha = alpha;
  r.beta = beta;
  r.nc = n_nodes;
  r.bytes = bytes;
  r.t_submit = Clock::now();
  s->queue.push_back(id);
  *request_id = id;
  lk.unlock();
  s->cv_work.notify_all();
  return RFDD_OK;
}

int rfdd_server_wait(rfdd_server *s, int64_t request_id, double timeout_ms, int32_t *done, rfdd_result **out) {
  if (!s || !done || !out) return RFDD_EINVAL;
  *done = 0;
  *out = nullptr;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return RFDD_EINVAL;
  auto finished = [&] { return it->second.status != REQ_WAITING && it->second.status != REQ_RUNNING; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, finished);
  } else if (!finished()) {
    s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), finished);
  }
  if (!finished()) return RFDD_OK;
  if (it->second.taken) return RFDD_ESTATE;  // its result was handed out already
  *done = 1;
  *out = it->second.res;
  it->second.res = nullptr;
  it->second.taken = true;
  return RFDD_OK;
}

int rfdd_server_request_info(rfdd_server *s, int64_t request_id, rfdd_request_info *info) {
  if (!s || !info) return RFDD_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return RFDD_EINVAL;
  const SRequest &r = it->second;
  memset(info, 0, sizeof(*info));
  info->status = r.status;
  info->pencil = r.pencil;
  info->nev = r.nev;
  info->bytes = r.bytes;
  const auto now = Clock::now();
  const bool started = r.status != REQ_WAITING, finished = started && r.status != REQ_RUNNING;
  info->queue_ms = ms_between(r.t_submit, started ? r.t_start : now);
  info->run_ms = started ? ms_between(r.t_start, finished ? r.t_done : now) : 0.0;
  info->latency_ms = ms_between(r.t_submit, finished ? r.t_done : now);
  return RFDD_OK;
}

int rfdd_server_get_stats(rfdd_server *s, rfdd_server_stats *out) {
  if (!s || !out) return RFDD_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->completed = s->completed;
  out->failed = s->failed;
  out->waiting = (int64_t)s->queue.size();
  out->running = s->st.running;
  out->peak_running = s->peak_running;
  out->in_use = s->st.in_use;
  out->peak_in_use = s->peak_in_use;
  out->pencils = (int64_t)s->pencils.size();
  return RFDD_OK;
}

int rfdd_server_remove_pencil(rfdd_server *s, int64_t pencil_id) {
  if (!s) return RFDD_EINVAL;
  rfdd_handle *h = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->pencils.find(pencil_id);
    if (it == s->pencils.end()) return RFDD_EINVAL;
    if (it->second.pending > 0 || it->second.one_shot) return RFDD_ESTATE;  // still in use
    h = it->second.h;
    s->pencils.erase(it);
  }
  rfdd_destroy(h);
  return RFDD_OK;
}

void rfdd_server_destroy(rfdd_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;  // waiting requests are dropped; running ones finish
    for (int64_t id : s->queue) {
      s->reqs[id].status = RFDD_ESTATE;
      s->pencils[s->reqs[id].pencil].pending -= 1;
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (auto &t : s->workers) t.join();
  for (auto &kv : s->reqs)
    if (kv.second.res) rfdd_result_free(kv.second.res);
  for (auto &kv : s->pencils)
    if (kv.second.h) rfdd_destroy(kv.second.h);
  delete s;
}

}  // extern "C"
