// Online autotuner of the tensor-core tile shape (host logic only, no CUDA): for each class of
// GEMM launch it times both tile shapes on real launches of that class, a few times each, and
// then keeps the faster one for every later launch of the class.  Kept apart from the launcher so
// that it can be compiled and tested on a host without a GPU.
//
// Candidates: 0 = one-CTA kernel, 128 x 256 output tiles; 1 = two-CTA kernel (cta_group::2),
// 256 x 256 tiles per SM pair.  A class is keyed by the launch's own sizes only (never by what
// else runs): device, complex or real, split count, the K depth bucket floor(log2(K tiles)), and
// the size bucket of the launch's one-CTA tile count relative to the SM count.  While a class is
// exploring, its launches alternate between the candidates (the one launched fewest times goes
// next); each timed launch reports milliseconds per GFLOP; once every candidate has `samples`
// timings, the one with the lower mean wins (ties to the one-CTA kernel) and the class is fixed
// for the life of the process.  Launches whose timings are still outstanding take the fixed
// rule's choice, as do all launches when tuning is off.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <tuple>

namespace rfdd {
namespace tune {

constexpr int NCAND = 2;

struct Key {
  int device = 0, cplx = 1, splits = 3, kbucket = 0, tbucket = 0;
  bool operator<(const Key &o) const {
    return std::tie(device, cplx, splits, kbucket, tbucket) <
           std::tie(o.device, o.cplx, o.splits, o.kbucket, o.tbucket);
  }
};

// floor(log2(nkt)), clamped to [0, 12]
inline int k_bucket(int64_t nkt) {
  int b = 0;
  while (b < 12 && (int64_t(2) << b) <= nkt) ++b;
  return b;
}

// launch size against the SM count: < 1/2, < 1, < 2, < 4, < 8, < 16, >= 16 waves of tiles
inline int t_bucket(int64_t tiles, int nsm) {
  const double r = (double)tiles / (double)(nsm > 0 ? nsm : 1);
  int b = 0;
  double edge = 0.5;
  while (b < 6 && r >= edge) {
    ++b;
    edge *= 2.0;
  }
  return b;
}

struct Stats {
  int launched[NCAND] = {0, 0};  // timed launches issued
  int done[NCAND] = {0, 0};      // timings received
  double sum[NCAND] = {0.0, 0.0};  // sum of ms per GFLOP
  int winner = -1;
};

struct Choice {
  int cand;      // candidate to launch
  bool measure;  // time this launch and report it with record()
};

class Tuner {
 public:
  bool enabled = true;
  int samples = 3;

  // The candidate for the next launch of class k; `rule` is the fixed rule's choice.
  Choice choose(const Key &k, int rule) {
    if (!enabled) return {rule, false};
    Stats &s = table_[k];
    if (s.winner >= 0) return {s.winner, false};
    int c = 0;
    for (int i = 1; i < NCAND; ++i)
      if (s.launched[i] < s.launched[c]) c = i;
    if (s.launched[c] < samples) {
      ++s.launched[c];
      return {c, true};
    }
    return {rule, false};  // every candidate issued; timings outstanding
  }

  // A timing of a launch that choose() asked to measure.
  void record(const Key &k, int cand, double ms_per_gflop) {
    auto it = table_.find(k);
    if (it == table_.end() || cand < 0 || cand >= NCAND) return;
    Stats &s = it->second;
    if (s.winner >= 0 || !(ms_per_gflop > 0.0) || !std::isfinite(ms_per_gflop)) return;
    ++s.done[cand];
    s.sum[cand] += ms_per_gflop;
    for (int i = 0; i < NCAND; ++i)
      if (s.done[i] < samples) return;
    int w = 0;
    for (int i = 1; i < NCAND; ++i)
      if (s.sum[i] / s.done[i] < s.sum[w] / s.done[w]) w = i;
    s.winner = w;
  }

  // A launch that was to be measured but could not be timed: it no longer counts as issued.
  void forget(const Key &k, int cand) {
    auto it = table_.find(k);
    if (it != table_.end() && cand >= 0 && cand < NCAND && it->second.launched[cand] > it->second.done[cand])
      --it->second.launched[cand];
  }

  void clear() { table_.clear(); }
  const std::map<Key, Stats> &table() const { return table_; }

  // One line per class: "dev cplx splits kbucket tbucket winner n0 mean0 n1 mean1\n" (means in
  // ms per GFLOP, 0 when no timing).
  std::string dump() const {
    std::string out;
    char line[256];
    for (const auto &e : table_) {
      const Key &k = e.first;
      const Stats &s = e.second;
      std::snprintf(line, sizeof(line), "%d %d %d %d %d %d %d %.6g %d %.6g\n", k.device, k.cplx, k.splits,
                    k.kbucket, k.tbucket, s.winner, s.done[0], s.done[0] ? s.sum[0] / s.done[0] : 0.0,
                    s.done[1], s.done[1] ? s.sum[1] / s.done[1] : 0.0);
      out += line;
    }
    return out;
  }

 private:
  std::map<Key, Stats> table_;
};

}  // namespace tune
}  // namespace rfdd
