"""The integer-arithmetic FP64 -> FP32 conversion the kernels use
(csrc/ras_convert.h) against the C conversion, bit for bit, on the host:
random bit patterns over every exponent, every rounding case at the 29
dropped bits (below, at and above one half, ties with an even and an odd
kept bit), the ends of the binary32 normal range, carries into the next
binade and to infinity, zeros, subnormals, infinities and NaN."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_2003_05361_gb300", "csrc", "ras_convert.h")

PROGRAM = r"""
#include <stdio.h>
#include <stdint.h>
#include <string.h>
#include "ras_convert.h"

static uint64_t state = 0x2003053610000001ull;
static uint64_t next(void) {  /* SplitMix64 */
  uint64_t z = (state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static long tested = 0, bad = 0;
static void check_d(uint64_t u) {
  double v; memcpy(&v, &u, 8);
  float a = ras::f64_to_f32_rn(v), b = (float)v;
  uint32_t ua, ub; memcpy(&ua, &a, 4); memcpy(&ub, &b, 4);
  ++tested;
  if (ua != ub) { if (bad < 5) printf("d2f %016llx: %08x vs %08x\n", (unsigned long long)u, ua, ub); ++bad; }
}
int main(void) {
  for (int i = 0; i < 2000000; ++i) check_d(next());
  /* every binary64 exponent, with the dropped bits below / at / above half */
  const uint64_t rests[] = {0, 1, 0x0fffffffull, 0x10000000ull, 0x10000001ull, 0x1fffffffull};
  for (uint64_t e = 0; e < 2048; ++e)
    for (int s = 0; s < 2; ++s)
      for (uint64_t r : rests)
        for (int k = 0; k < 64; ++k) {
          /* the 23 kept fraction bits: all ones (a carry into the next
             binade), zero, or random (even and odd last kept bits) */
          const uint64_t kept = k == 0 ? 0x7fffffull : k == 1 ? 0 : (next() & 0x7fffffull);
          check_d(((uint64_t)s << 63) | (e << 52) | (kept << 29) | r);
        }
  printf("%ld %ld\n", tested, bad);
  return 0;
}
"""


def test_conversion_matches_c_cast(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "convert_check.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "convert_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off",
                    "-I" + os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    tested, bad = map(int, out.split()[-2:])
    assert tested > 3_000_000
    assert bad == 0, out
