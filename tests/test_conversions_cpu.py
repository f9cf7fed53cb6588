"""The integer-pipe fp64 <-> fp32 conversions of the device code (f32_of,
f64_of in csrc/common.cuh; used by the operand slicing and the split-K
reduction) against the IEEE 754 conversions of the host compiler.

The functions are __host__ __device__, so a host program compiled by nvcc
runs the same source on the CPU. Checked: 2e6 random bit patterns (every
class: normal, subnormal, zero, inf, NaN), values around each fp32 exponent
including exact rounding ties, and the documented flush to zero below the
fp32 normal range.
"""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2607_15158_gb300", "csrc")

PROGRAM = r"""
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include "common.cuh"
using namespace ctm;
static unsigned fb(float f) { unsigned u; memcpy(&u, &f, 4); return u; }
static unsigned long long db(double d) { unsigned long long u; memcpy(&u, &d, 8); return u; }
int main() {
  long bad = 0, n = 0;
  auto check = [&](double x) {
    ++n;
    const float ref = (float)x, got = f32_of(x);
    bool ok = fb(ref) == fb(got) || (std::isnan(ref) && std::isnan(got));
    if (!ok && std::fabs(x) < FLT_MIN) ok = got == 0.0f && std::signbit(got) == std::signbit(x);
    const double r2 = (double)ref, g2 = f64_of(ref);
    bool ok2 = db(r2) == db(g2) || (std::isnan(r2) && std::isnan(g2));
    if (!ok2 && std::fabs(ref) < FLT_MIN) ok2 = g2 == 0.0;
    if (!(ok && ok2)) {
      if (bad < 5) printf("mismatch x=%a f32 ref=%a got=%a f64 ref=%a got=%a\n", x, ref, got, r2, g2);
      ++bad;
    }
  };
  std::mt19937_64 rng(7);
  for (long i = 0; i < 2000000; ++i) {
    unsigned long long b = rng();
    double x;
    memcpy(&x, &b, 8);
    check(x);
  }
  for (int e = -130; e < 130; ++e)
    for (unsigned m = 0; m < 64; ++m) {
      const double base = std::ldexp(1.0, e);
      const double x = base * (1.0 + std::ldexp((double)m, -23)) + ((m & 1) ? std::ldexp(base, -24) : 0.0);
      check(x); check(-x); check(std::nextafter(x, 0.0)); check(std::nextafter(x, 1e300));
    }
  const double special[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, DBL_MAX, FLT_MAX,
                            (double)FLT_MAX * (1 + 1e-8), FLT_MIN, FLT_MIN * 0.5, DBL_MIN, 1.0, -1.0};
  for (double x : special) check(x);
  printf("%ld checks, %ld mismatches\n", n, bad);
  return bad ? 1 : 0;
}
"""


def test_integer_pipe_conversions_match_ieee(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "conv.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "conv"
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "0 mismatches" in run.stdout
