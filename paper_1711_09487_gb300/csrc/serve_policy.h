// Admission policy of the serving loop (host logic only, no CUDA): which waiting request starts
// next.  Kept apart from the server so that it can be compiled and tested on a host without a GPU.
//
// Requests wait in arrival order.  A request may start when (1) fewer than max_inflight requests
// run, (2) its pencil has no request running (a handle serves one solve at a time), and (3) its
// device-memory estimate fits in what the budget has left.  The first waiting request that
// satisfies all three starts (first fit in arrival order), so small requests fill the memory a
// large one leaves free.  To keep a large request from waiting forever, the oldest waiting
// request may be passed over at most max_bypass times; after that nothing else starts until it
// does.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace rfdd {
namespace serve {

struct Waiting {
  int64_t id;        // request id (arrival order)
  int64_t pencil;    // pencil id
  size_t bytes;      // device-memory estimate the request is admitted with
};

struct State {
  size_t budget = 0;          // device bytes all running requests may hold
  size_t in_use = 0;          // bytes of the running requests
  int running = 0;            // requests running
  int max_inflight = 1;
  int max_bypass = 8;
  int head_bypassed = 0;      // times the oldest waiting request was passed over
  int64_t head_id = -1;       // which request head_bypassed counts for
};

// Index into `queue` (arrival order) of the request to start now, or -1.  `busy(pencil)` tells
// whether a pencil has a request running.  Updates the bypass count of the oldest request.
template <typename Busy>
int pick_next(const std::vector<Waiting> &queue, State &st, Busy &&busy) {
  if (queue.empty() || st.running >= st.max_inflight) return -1;
  if (queue[0].id != st.head_id) {
    st.head_id = queue[0].id;
    st.head_bypassed = 0;
  }
  auto fits = [&](const Waiting &w) { return !busy(w.pencil) && st.in_use + w.bytes <= st.budget; };
  if (fits(queue[0])) return 0;
  if (st.head_bypassed >= st.max_bypass) return -1;  // the oldest request has waited long enough
  for (size_t i = 1; i < queue.size(); ++i) {
    if (fits(queue[i])) {
      ++st.head_bypassed;
      return (int)i;
    }
  }
  return -1;
}

}  // namespace serve
}  // namespace rfdd
