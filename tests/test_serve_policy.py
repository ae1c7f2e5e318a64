"""Admission policy of the serving loop (csrc/serve_policy.h), compiled on the host with g++ and
driven through the cases it must get right: arrival order when everything fits, the in-flight
limit, first fit past a request whose memory does not fit, one solve at a time per pencil, and
the bound on how often the oldest request is passed over."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1711_09487_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <set>
#include "serve_policy.h"
using namespace rfdd::serve;
#define CHECK(c) do { if (!(c)) { std::printf("FAILED line %d: %s\n", __LINE__, #c); return 1; } } while (0)
int main() {
  std::set<long long> busy;
  auto isbusy = [&](long long p) { return busy.count(p) > 0; };
  {  // everything fits: arrival order
    State st; st.budget = 100; st.max_inflight = 4;
    std::vector<Waiting> q = {{0, 0, 10}, {1, 1, 10}};
    CHECK(pick_next(q, st, isbusy) == 0);
  }
  {  // in-flight limit
    State st; st.budget = 100; st.max_inflight = 2; st.running = 2;
    std::vector<Waiting> q = {{0, 0, 10}};
    CHECK(pick_next(q, st, isbusy) == -1);
  }
  {  // the head does not fit: first fit behind it, at most max_bypass times
    State st; st.budget = 100; st.in_use = 60; st.max_inflight = 8; st.max_bypass = 2;
    std::vector<Waiting> q = {{5, 0, 50}, {6, 1, 30}, {7, 2, 45}, {8, 3, 20}};
    CHECK(pick_next(q, st, isbusy) == 1);          // 30 fits, 45 does not
    CHECK(st.head_bypassed == 1 && st.head_id == 5);
    q.erase(q.begin() + 1); st.in_use += 30;       // 90 in use
    CHECK(pick_next(q, st, isbusy) == -1);          // nothing fits in 10
    st.in_use = 70;                                 // something finished: 30 free
    CHECK(pick_next(q, st, isbusy) == 2);           // request 8 (20) passes the head again
    CHECK(st.head_bypassed == 2);
    q.erase(q.begin() + 2); st.in_use = 50;         // 50 free: the head (50) fits now
    CHECK(pick_next(q, st, isbusy) == 0);
    st.in_use = 80;
    std::vector<Waiting> q2 = {{5, 0, 50}, {9, 4, 5}};
    CHECK(pick_next(q2, st, isbusy) == -1);         // passed over twice already: the head waits
    std::vector<Waiting> q3 = {{9, 4, 5}};
    CHECK(pick_next(q3, st, isbusy) == 0 && st.head_id == 9 && st.head_bypassed == 0);  // new head
  }
  {  // a pencil with a running request is skipped; its next request waits
    State st; st.budget = 100; st.max_inflight = 4;
    busy.insert(0);
    std::vector<Waiting> q = {{0, 0, 10}, {1, 0, 10}, {2, 1, 10}};
    CHECK(pick_next(q, st, isbusy) == 2);
    busy.clear();
  }
  {  // a request larger than the whole budget never starts (the server refuses it at submit)
    State st; st.budget = 100; st.max_inflight = 4;
    std::vector<Waiting> q = {{0, 0, 101}};
    CHECK(pick_next(q, st, isbusy) == -1);
  }
  std::printf("ok\n");
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_admission_policy(tmp_path):
    src = tmp_path / "policy_test.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "policy_test"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
