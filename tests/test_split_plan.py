"""Host check of the K split of the FP64 grouped GEMM (csrc/lrt_fp64_tile.h, split_segments).

A long output (phase 2 of sigma sums dozens of block products along one K axis) has its
tiles cut along the segment list into K parts that run on separate CTAs, their partial
tiles added in order afterwards.  The result is right only if the parts cover the segment
list exactly once, in order, as runs of whole segments, and it stays bit-identical across
calls only if the cut depends on the segment list alone.  This test compiles the rule as
plain C++ and checks, on random segment lists, that the parts are contiguous, non-empty and
cover every segment once; that their K adds up; that there are at most `want` of them; and
that none holds more than ktot / want plus one segment's K.  It needs no GPU.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1311_1646_gb300", "csrc")

CHECKER = r"""
#include "lrt_fp64_tile.h"
#include <cstdio>
#include <vector>
using namespace lrt;

static unsigned long long st = 0x2545F4914F6CDD1Dull;
static int rnd(int n) { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (int)(st % (unsigned long long)n); }

int main() {
  int cases = 0;
  for (int it = 0; it < 20000; ++it) {
    const int nseg = 1 + rnd(it % 3 == 0 ? 8 : 200);
    std::vector<int> k(nseg);
    long long ktot = 0;
    int kmax = 0;
    for (int q = 0; q < nseg; ++q) {
      k[q] = rnd(5) == 0 ? 0 : 1 + rnd(it % 2 ? 40 : 600);   // zero-K segments too
      ktot += k[q];
      kmax = k[q] > kmax ? k[q] : kmax;
    }
    const int want = 1 + rnd(nseg);
    std::vector<int> sb, se;
    std::vector<long long> kp;
    const int n = split_segments(k.data(), nseg, ktot, want, [&](int a, int b, long long c) {
      sb.push_back(a);
      se.push_back(b);
      kp.push_back(c);
    });
    if (n != (int)sb.size() || n < 1 || n > want) { printf("count %d (want %d)\n", n, want); return 1; }
    int next = 0;
    long long sum = 0;
    for (int j = 0; j < n; ++j) {
      if (sb[j] != next || se[j] <= sb[j]) { printf("not contiguous at part %d\n", j); return 1; }
      long long s = 0;
      for (int q = sb[j]; q < se[j]; ++q) s += k[q];
      if (s != kp[j]) { printf("K of part %d\n", j); return 1; }
      if (ktot > 0 && kp[j] * want > ktot + (long long)want * kmax) { printf("part %d too long\n", j); return 1; }
      sum += kp[j];
      next = se[j];
    }
    if (next != nseg || sum != ktot) { printf("coverage\n"); return 1; }
    // the same list cut again: the same parts
    int m = 0;
    bool same = true;
    split_segments(k.data(), nseg, ktot, want, [&](int a, int b, long long) {
      same = same && m < n && sb[m] == a && se[m] == b;
      ++m;
    });
    if (!same || m != n) { printf("not deterministic\n"); return 1; }
    ++cases;
  }
  printf("ok %d\n", cases);
  return 0;
}
"""


def test_k_split_covers_each_segment_once_in_order(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    src = tmp_path / "split_check.cpp"
    exe = tmp_path / "split_check"
    src.write_text(CHECKER)
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")
