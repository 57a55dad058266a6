"""The integer digit extraction of the reverse sweep's tensor-core contraction
(paper_2306_00271_gb300/csrc/fixed_digits.cuh), compiled as host code and run on the CPU: the
scale exponent is the smallest power of two at or above |x|, the 31-bit fixed-point value is x
scaled and rounded to the nearest integer, and the four balanced base-256 digits are exact in BF16,
bounded by 128 and add up to that value exactly. The device build compiles the same source."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "paper_2306_00271_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

DRIVER = r"""
#include "fixed_digits.cuh"
#include <cmath>
#include <cstdio>
using namespace trh::fixed;

static unsigned long long state = 0x9E3779B97F4A7C15ull;
static unsigned long long next64() {   // splitmix64
  unsigned long long z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double uniform() { return (double)(next64() >> 11) * 0x1.0p-53; }
static int decode(uint16_t b) {        // BF16 pattern -> the integer it holds
  const float f = float_of_bits((uint32_t)b << 16);
  return (int)f;
}

int main() {
  long long fails = 0, checked = 0;
  for (int d = -256; d <= 256; ++d)
    if (decode(bf16_of_int(d)) != d || (bits_of_float((float)d) >> 16) != bf16_of_int(d)) ++fails;
  const double specials[] = {0.0, -0.0, 1.0, -1.0, 0.5, 0x1.fffffffffffffp-1, 0x1.0000000000001p0,
                             -0x1.0p-60, 0x1.8p+40, 4.9e-324, -2.2e-308};
  for (int row = 0; row < 4000; ++row) {
    double x[65];
    const double mag = std::ldexp(1.0, (int)(next64() % 200) - 100);
    for (int k = 0; k < 64; ++k) x[k] = (2.0 * uniform() - 1.0) * mag * std::ldexp(1.0, -(int)(next64() % 40));
    x[64] = specials[row % 11] * (row % 3 == 0 ? 1.0 : mag);
    if (row % 5 == 0) x[next64() % 64] = std::ldexp(1.0, (int)(next64() % 200) - 100);  // exact power
    int E = INT_MIN;
    for (int k = 0; k < 65; ++k) {
      const int e = ceil_exp(x[k]);
      if (x[k] != 0.0 && std::fpclassify(x[k]) == FP_NORMAL) {
        // smallest e with |x| <= 2^e
        if (!(std::fabs(x[k]) <= std::ldexp(1.0, e) && std::fabs(x[k]) > std::ldexp(1.0, e - 1))) ++fails;
      }
      if (x[k] == 0.0 && e != INT_MIN) ++fails;
      if (e > E) E = e;
    }
    if (E == INT_MIN) E = 0;
    if (E < -126) E = -126;
    if (E > 127) continue;                 // outside the FP32 scale range: not used
    if (pow2f(E) != std::ldexp(1.0f, E)) ++fails;
    for (int k = 0; k < 65; ++k) {
      const long long V = fixed31(x[k], E);
      const double exact = std::ldexp(x[k], 31 - E);
      if (std::fpclassify(x[k]) == FP_NORMAL && std::fabs(exact - (double)V) > 0.5) ++fails;
      if (V > (1ll << 31) || V < -(1ll << 31)) ++fails;
      uint16_t b[4];
      digits_of(V, b);
      long long sum = 0;
      for (int i = 0; i < 4; ++i) {
        const int d = decode(b[i]);
        if (d > 128 || d < -128) ++fails;
        sum = sum * 256 + d;
      }
      if (sum != V) ++fails;
      ++checked;
    }
  }
  std::printf("%lld %lld\n", checked, fails);
  return 0;
}
"""


def test_fixed_point_digits(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("no host C++ compiler or CUDA headers")
    src = tmp_path / "fixed_driver.cpp"
    exe = tmp_path / "fixed_driver"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", HEADER_DIR, "-I", CUDA_INC, str(src), "-o",
                    str(exe)], check=True)
    checked, fails = map(int, subprocess.run([str(exe)], check=True, capture_output=True,
                                             text=True).stdout.split())
    assert checked > 200000 and fails == 0, (checked, fails)
