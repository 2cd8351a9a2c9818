"""The mixed path's forces leave the fixed-point accumulators through an
integer-only conversion (x * 2^-32 rounded to nearest even, built from the bits);
it must give exactly the bits of (double)x * 2^-32.  The device helper is also a
host function: compiled here into a small host program and checked on powers of
two and their neighbours, halfway cases of the rounding, and random values."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2212_14446_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include "pod_common.cuh"
int main() {
  std::mt19937_64 g(11);
  long long bad = 0, n = 0;
  auto check = [&](long long x) {
    const double a = fastpod::fixed_to_double(x, -32), b = (double)x * 0x1p-32;
    ++n;
    if (std::memcmp(&a, &b, 8)) ++bad;
  };
  check(0);
  for (int k = 0; k < 63; ++k) {
    const long long p = 1LL << k;
    for (long long d = -3; d <= 3; ++d) { check(p + d); check(-(p + d)); }
    if (k > 53) {
      const long long h = 1LL << (k - 53);
      for (long long base : {p, p + 2 * h, p + 6 * h}) {
        check(base + h); check(base + h - 1); check(base + h + 1); check(-(base + h));
        check(base + 3 * h); check(-(base + 3 * h));
      }
    }
  }
  for (int i = 0; i < 2000000; ++i) {
    long long x = (long long)(g() >> (g() % 64));
    check((g() & 1) ? -x : x);
  }
  std::printf("%lld %lld\n", n, bad);
  return bad != 0;
}
"""


def test_integer_conversion_matches_the_fp64_conversion():
    nvcc = os.environ.get("NVCC") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc")
                                      else shutil.which("nvcc"))
    if not nvcc:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cu")
        exe = os.path.join(d, "t")
        with open(src, "w") as f:
            f.write(PROGRAM)
        subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, src, "-o", exe], check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True)
        n, bad = (int(v) for v in out.stdout.split())
        assert out.returncode == 0 and bad == 0 and n > 2000000
