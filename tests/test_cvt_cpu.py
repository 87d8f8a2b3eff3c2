"""The integer-pipe conversions between binary64 and binary32 (csrc/cvt.cuh) against the host's
IEEE 754 casts, bit for bit: every binary32 pattern for FP32 -> FP64, and for FP64 -> FP32
random patterns over the whole exponent range together with the cases a rounding slip would
miss (ties to even with an even and an odd kept bit, just above and below the tie, mantissa
carries into the exponent, the largest finite results and the overflow to infinity, the
smallest normal results, zeros, subnormals, infinities, NaNs).  The header is plain C++, so the
same source the kernels use is compiled here with g++."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1805_06557_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include <cstring>
#include "cvt.cuh"

static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t next() {  // splitmix64
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double d_of(uint64_t u) { double d; memcpy(&d, &u, 8); return d; }
static uint32_t u_of(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static uint64_t u_of(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }

static long bad = 0, n64 = 0;
static void check64(uint64_t u) {
  const double d = d_of(u);
  const uint32_t a = u_of(cvt::f64_to_f32(d)), b = u_of((float)d);
  ++n64;
  if (a != b && bad++ < 5) printf("f64_to_f32 %016llx: %08x vs %08x\n", (unsigned long long)u, a, b);
}

int main() {
  // FP32 -> FP64: every pattern
  long n32 = 0;
  for (uint64_t v = 0; v <= 0xffffffffull; ++v) {
    float f; const uint32_t w = (uint32_t)v; memcpy(&f, &w, 4);
    const uint64_t a = u_of(cvt::f32_to_f64(f)), b = u_of((double)f);
    ++n32;
    if (a != b && bad++ < 5) printf("f32_to_f64 %08x: %016llx vs %016llx\n", w, (unsigned long long)a, (unsigned long long)b);
  }
  // FP64 -> FP32: random patterns, and random patterns with the exponent in and around the
  // fast path's range
  for (long i = 0; i < 100000000; ++i) check64(next());
  for (long i = 0; i < 100000000; ++i) {
    const uint64_t r = next();
    const uint64_t e = 860 + (r >> 54) % 330;  // e11 in [860, 1189]
    check64((r & 0x800FFFFFFFFFFFFFull) | (e << 52));
  }
  // constructed cases at every exponent: the 29 dropped bits at 0, 1, tie - 1, tie, tie + 1,
  // all ones, with kept mantissas 0, 1, 2, odd / even, all ones (carry)
  const uint64_t drops[] = {0, 1, 0x0fffffffull, 0x10000000ull, 0x10000001ull, 0x1fffffffull};
  const uint64_t keeps[] = {0, 1, 2, 3, 0x3ffffeull, 0x3fffffull, 0x7ffffeull, 0x7fffffull, 0x400000ull};
  for (uint64_t e = 0; e < 2048; ++e)
    for (uint64_t sg = 0; sg < 2; ++sg)
      for (uint64_t k : keeps)
        for (uint64_t dr : drops) check64((sg << 63) | (e << 52) | (k << 29) | dr);
  printf("checked %ld binary32 and %ld binary64 inputs, %ld mismatches\n", n32, n64, bad);
  return bad ? 1 : 0;
}
"""


def test_conversions_match_host_casts(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "cvt_test.cpp"
    exe = tmp_path / "cvt_test"
    src.write_text(HARNESS)
    # -ffp-contract=off and no fast-math: the host casts must be the IEEE ones
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 mismatches" in r.stdout
