"""Tile-shape autotuner (csrc/tc_tune.h), compiled on the host with g++ and driven with made-up
timings: the buckets of the class key, alternation while a class explores, the fixed rule while
timings are outstanding, the winner by mean time (ties to the one-CTA kernel), a decided class
never changing, classes kept apart, untimed launches forgotten, tuning off, and the table text."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1711_09487_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstring>
#include "tc_tune.h"
using namespace rfdd::tune;
#define CHECK(c) do { if (!(c)) { std::printf("FAILED line %d: %s\n", __LINE__, #c); return 1; } } while (0)
int main() {
  // buckets
  CHECK(k_bucket(1) == 0 && k_bucket(2) == 1 && k_bucket(15) == 3 && k_bucket(16) == 4 && k_bucket(1 << 20) == 12);
  CHECK(t_bucket(10, 152) == 0 && t_bucket(76, 152) == 1 && t_bucket(151, 152) == 1 && t_bucket(152, 152) == 2);
  CHECK(t_bucket(304, 152) == 3 && t_bucket(152 * 16, 152) == 6 && t_bucket(152 * 100, 152) == 6);
  Key a; a.kbucket = 4; a.tbucket = 3;
  Key b = a; b.tbucket = 4;
  {  // explore: alternate, starting with candidate 0; then the rule while timings are outstanding
    Tuner t;
    int seq[6];
    for (int i = 0; i < 6; ++i) { Choice c = t.choose(a, 1); CHECK(c.measure); seq[i] = c.cand; }
    CHECK(seq[0] == 0 && seq[1] == 1 && seq[2] == 0 && seq[3] == 1 && seq[4] == 0 && seq[5] == 1);
    Choice c = t.choose(a, 1);
    CHECK(!c.measure && c.cand == 1);                 // rule's choice, nothing timed
    CHECK(t.choose(a, 0).cand == 0);
    // timings: the two-CTA kernel is faster on average
    t.record(a, 0, 1.00); t.record(a, 1, 0.90); t.record(a, 0, 1.10); t.record(a, 1, 1.20);
    CHECK(t.table().at(a).winner == -1);              // not all timings in
    t.record(a, 0, 1.00); t.record(a, 1, 0.95);
    CHECK(t.table().at(a).winner == 1);               // means 1.033 vs 1.017
    for (int i = 0; i < 4; ++i) { Choice d = t.choose(a, 0); CHECK(d.cand == 1 && !d.measure); }
    t.record(a, 0, 0.01);                             // a late timing does not reopen the class
    CHECK(t.table().at(a).winner == 1);
    // another class is independent
    Choice e = t.choose(b, 1);
    CHECK(e.measure && e.cand == 0 && t.table().at(b).winner == -1);
  }
  {  // ties go to the one-CTA kernel; bad timings are ignored
    Tuner t; t.samples = 1;
    t.choose(a, 1); t.choose(a, 1);
    t.record(a, 1, -1.0); t.record(a, 1, 0.0 / 0.0 + 0.0 * 0.0);
    CHECK(t.table().at(a).winner == -1);
    t.record(a, 0, 2.0); t.record(a, 1, 2.0);
    CHECK(t.table().at(a).winner == 0);
  }
  {  // a launch that could not be timed is issued again
    Tuner t; t.samples = 1;
    CHECK(t.choose(a, 0).cand == 0);
    t.forget(a, 0);
    Choice c = t.choose(a, 0);
    CHECK(c.cand == 0 && c.measure);
    CHECK(t.choose(a, 0).cand == 1);
  }
  {  // tuning off: the rule, no timing, no table entry
    Tuner t; t.enabled = false;
    Choice c = t.choose(a, 1);
    CHECK(c.cand == 1 && !c.measure && t.table().empty());
  }
  {  // table text
    Tuner t; t.samples = 1;
    t.choose(a, 0); t.choose(a, 0); t.record(a, 0, 0.5); t.record(a, 1, 0.25);
    std::string s = t.dump();
    CHECK(s == "0 1 3 4 3 1 1 0.5 1 0.25\n");
  }
  std::printf("ok\n");
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_tile_shape_tuner(tmp_path):
    src = tmp_path / "tune_test.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "tune_test"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
