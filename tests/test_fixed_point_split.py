"""The arithmetic behind the sorted deposit's exactness, restated in C and
checked against exact rounding (CPU; gcc with contraction off, C99 fmaf):

* the push's split of a scaled contribution v (|v| < 2^38) into
  h = rne(v / 2^16) and r = v - 2^16 h (exact, |r| <= 2^15), both rounded to
  integers by adding 1.5 * 2^23 and reading the bits: 2^16 h + rne(r) must be
  rne(v), the value whose 64-bit sum is order-independent;
* the E update's conversion of a 64-bit fixed-point sum n to FP32 times a
  power-of-two scale s: n = a 2^24 + b (0 <= b < 2^24), fma(a, 2^24 s, b s)
  must be the correctly rounded n s while |n| < 2^48.
"""
import os
import shutil
import subprocess

import pytest

SRC = r"""
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

static int bits(float x) { int i; memcpy(&i, &x, 4); return i; }

/* the split: returns 2^16 h + rne(r) */
static long long split(float v) {
  const float M = 12582912.0f;
  float hs = fmaf(v, 1.52587890625e-05f, M);
  float h = hs - M;
  float r = fmaf(-h, 65536.0f, v);
  int lo = bits(r + M) - 0x4B400000;
  int hh = bits(hs) - 0x4B400000;
  return (long long)hh * 65536LL + lo;
}

static float to_float(long long n, float s) {
  float a = (float)(int)(n >> 24);
  float b = (float)(int)(n & 0xFFFFFFLL);
  return fmaf(a, 16777216.0f * s, b * s);
}

int main(void) {
  uint64_t st = 88172645463325252ULL;
  long bad = 0, n = 0;
  for (int e = -30; e <= 37; ++e)
    for (int k = 0; k < 100000; ++k) {
      st ^= st << 13; st ^= st >> 7; st ^= st << 17;
      float m = (float)(st >> 40) / 16777216.0f;
      float v = ldexpf(1.0f + m, e - 1);
      if (st & 1) v = -v;
      if (fabsf(v) >= ldexpf(1.0f, 38)) continue;
      if (split(v) != llrintf(v)) ++bad;
      ++n;
    }
  for (int e = 0; e < 48; ++e)
    for (int k = 0; k < 100000; ++k) {
      st ^= st << 13; st ^= st >> 7; st ^= st << 17;
      long long q = e ? (long long)(st >> 16) & ((1LL << e) - 1) : (long long)(st >> 63);
      if (st & 2) q = -q;
      float s = ldexpf(1.0f, -(int)((st >> 8) % 60));
      float ref = (float)((long double)q * (long double)s);
      if (to_float(q, s) != ref) ++bad;
      ++n;
    }
  printf("%ld %ld\n", n, bad);
  return bad != 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_fixed_point_split_and_conversion_are_exact(tmp_path):
    src = os.path.join(tmp_path, "split.c")
    exe = os.path.join(tmp_path, "split")
    open(src, "w").write(SRC)
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", src, "-o", exe, "-lm"], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    n, bad = map(int, out.stdout.split())
    assert n > 10_000_000 and bad == 0, out.stdout
