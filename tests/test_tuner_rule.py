"""The autotuner's selection rule and cache (paper_2306_00271_gb300/csrc/tuner.h), compiled with the
host C++ compiler and run on the CPU: the earliest (cheapest) candidate wins unless a later one
is faster by more than the margin, failed probes never win, choices are cached per shape key, and
a call's time is extrapolated from probes of two step counts."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "paper_2306_00271_gb300", "csrc")

DRIVER = r"""
#include "tuner.h"
#include <cmath>
#include <cstdio>
#include <thread>
#include <vector>
using namespace trh::tune;
int main() {
  const float nan = std::nanf("");
  { const float m[2] = {1.0f, 0.99f}; std::printf("%d\n", pick(m, 2, 0.02f)); }   // 0: within margin
  { const float m[2] = {1.0f, 0.90f}; std::printf("%d\n", pick(m, 2, 0.02f)); }   // 1: faster
  { const float m[2] = {-1.0f, 2.0f}; std::printf("%d\n", pick(m, 2, 0.02f)); }   // 1: probe 0 failed
  { const float m[2] = {nan, nan}; std::printf("%d\n", pick(m, 2, 0.02f)); }      // 0: all failed
  { const float m[3] = {0.5f, 0.6f, 0.4f}; std::printf("%d\n", pick(m, 3, 0.0f)); } // 2
  { const float m[2] = {1.0f, 1.0f}; std::printf("%d\n", pick(m, 2, 0.0f)); }     // 0: tie
  { const float m[3] = {1.0f, 0.5f, 0.49f}; std::printf("%d\n", pick(m, 3, 0.05f)); } // 1
  Cache c;
  int v = -1;
  const Key a{kColumnSplit, 1, 61, 0, 60, 2000}, b{kColumnSplit, 1, 61, 0, 120, 2000},
      t{kWideTile, 0, 61, 0, 60, 2000}, a400{kColumnSplit, 1, 61, 0, 60, 400};
  std::printf("%d\n", (int)c.find(a, &v));                                        // 0
  c.put(a, 1);
  c.put(t, 32);
  { const int f = c.find(a, &v); std::printf("%d %d\n", f, v); }                // 1 1
  std::printf("%d\n", (int)c.find(b, &v));                                        // 0: other pair count
  std::printf("%d\n", (int)c.find(a400, &v));                                     // 0: other step count
  { const int f = c.find(t, &v); std::printf("%d %d\n", f, v); }                // 1 32
  std::vector<std::thread> th;
  for (int i = 0; i < 8; ++i)
    th.emplace_back([&c, i] { for (int k = 0; k < 1000; ++k) c.put(Key{kWideTile, i, k, 0, 1, 1}, k); });
  for (auto& x : th) x.join();
  std::printf("%zu\n", c.size());                                                 // 8002
  // a probe of 2 and 12 steps, the call 2000 steps: overhead 1.0 ms, 0.1 ms a step
  std::printf("%.1f\n", extrapolate(1.2f, 2, 2.2f, 12, 2000));                    // 201.0
  std::printf("%.1f\n", extrapolate(1.2f, 2, -1.0f, 12, 2000));                   // 1.2: failed probe
  return 0;
}
"""


def test_selection_rule_and_cache(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "tuner_driver.cpp"
    exe = tmp_path / "tuner_driver"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I", HEADER_DIR, str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    assert out[:7] == ["0", "1", "1", "0", "2", "0", "1"]
    assert out[7:13] == ["0", "1 1", "0", "0", "1 32", "8002"]
    assert out[13:15] == ["201.0", "1.2"]
