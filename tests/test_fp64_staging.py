"""Host check of the FP64 grouped GEMM's staging plan (csrc/lrt_fp64_tile.h).

The sigma phases sum, per output tile, many short block products (Eqs. hzero_sb,
hleft_sb: one product per operator pair of the "x" summation).  The kernel packs
their contracted indices along one K axis and stages 32 positions at a time; the
plan decides which thread copies which element.  This test compiles the plan as
plain C++ and checks, for random segment lists, tile shapes, storage orders and vector
blockings (a tile spanning the same product for several trial vectors),
that every element of every staged chunk is copied exactly once, from the right
address, and that nothing outside the chunk is written.  It needs no GPU.
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
#include <cstdlib>
#include <vector>
using namespace lrt;

static unsigned long long st = 0x9E3779B97F4A7C15ull;
static int rnd(int n) { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (int)(st % (unsigned long long)n); }

int main() {
  int cases = 0;
  for (int it = 0; it < 3000; ++it) {
    const int nb = 1 + rnd(GEMM_SEGB);
    const int mt = 1 + rnd(GEMM_TILE_M), nt = 1 + rnd(GEMM_TILE_N);
    const int m0 = rnd(3) * GEMM_TILE_M, n0 = rnd(3) * GEMM_TILE_N;
    std::vector<std::vector<double>> store(2 * nb);
    SegS sd[GEMM_SEGB];
    int kst[GEMM_SEGB + 1];
    kst[0] = 0;
    for (int q = 0; q < nb; ++q) {
      const int k = rnd(6) == 0 ? 0 : 1 + rnd(40);
      SegS s;
      s.transA = rnd(2);
      s.transB = rnd(2);
      s.scale = 1.0;
      // vector blocking in half the cases: rows of A (columns of B) in blocks of avr (bvc),
      // block v of the operand at v * avs (v * bvs)
      s.avr = rnd(2) ? 1 + rnd(20) : 0;
      s.bvc = rnd(2) ? 1 + rnd(12) : 0;
      const int arows = s.avr ? s.avr : m0 + mt, bcols = s.bvc ? s.bvc : n0 + nt;
      const int nva = s.avr ? (m0 + mt + s.avr - 1) / s.avr : 1, nvb = s.bvc ? (n0 + nt + s.bvc - 1) / s.bvc : 1;
      // A is (m0 + mt) x k, B is k x (n0 + nt) (per vector block); leading dimensions padded at random
      const int ar = s.transA ? k : arows, ac = s.transA ? arows : k;
      const int br = s.transB ? bcols : k, bc = s.transB ? k : bcols;
      s.lda = ac + rnd(4);
      s.ldb = bc + rnd(4);
      s.avs = (int64_t)ar * s.lda + rnd(5);
      s.bvs = (int64_t)br * s.ldb + rnd(5);
      store[2 * q].assign((size_t)(nva * s.avs) + 1, 0.0);
      store[2 * q + 1].assign((size_t)(nvb * s.bvs) + 1, 0.0);
      s.A = store[2 * q].data();
      s.B = store[2 * q + 1].data();
      sd[q] = s;
      kst[q + 1] = kst[q] + k;
    }
    for (int q = nb; q < GEMM_SEGB; ++q) kst[q + 1] = kst[nb];
    const int Kb = kst[nb];
    for (int p0 = 0; p0 < Kb; p0 += GEMM_KC) {
      const int kc = Kb - p0 < GEMM_KC ? Kb - p0 : GEMM_KC;
      const double* a_src[GEMM_TILE_M][GEMM_KC] = {};
      const double* b_src[GEMM_KC][GEMM_TILE_N] = {};
      int a_n[GEMM_TILE_M][GEMM_KC] = {}, b_n[GEMM_KC][GEMM_TILE_N] = {};
      bool bad = false;
      for (int tid = 0; tid < GEMM_THREADS; ++tid)
        stage_chunk(tid, sd, kst, Kb, p0, m0, mt, n0, nt, [&](int which, int r, int c, const double* src) {
          if (which == 0) {
            if (r < 0 || r >= mt || c < 0 || c >= kc) { bad = true; return; }
            a_src[r][c] = src; a_n[r][c]++;
          } else {
            if (r < 0 || r >= kc || c < 0 || c >= nt) { bad = true; return; }
            b_src[r][c] = src; b_n[r][c]++;
          }
        });
      if (bad) { printf("write outside the chunk: case %d p0 %d\n", it, p0); return 1; }
      for (int kk = 0; kk < kc; ++kk) {
        const int p = p0 + kk;
        int q = 0;
        while (kst[q + 1] <= p) ++q;
        const SegS& s = sd[q];
        const int kl = p - kst[q];
        for (int i = 0; i < mt; ++i) {
          // independent statement of the address: vector block and row inside it
          const int gr = m0 + i, va = s.avr ? gr / s.avr : 0, ra = s.avr ? gr % s.avr : gr;
          const double* base = s.A + (size_t)va * (size_t)s.avs;
          const double* want = s.transA ? base + (size_t)kl * s.lda + ra : base + (size_t)ra * s.lda + kl;
          if (a_n[i][kk] != 1 || a_src[i][kk] != want) {
            printf("A element (%d, %d) copied %d times, case %d\n", i, kk, a_n[i][kk], it);
            return 1;
          }
        }
        for (int j = 0; j < nt; ++j) {
          const int gc = n0 + j, vb = s.bvc ? gc / s.bvc : 0, cb = s.bvc ? gc % s.bvc : gc;
          const double* base = s.B + (size_t)vb * (size_t)s.bvs;
          const double* want = s.transB ? base + (size_t)cb * s.ldb + kl : base + (size_t)kl * s.ldb + cb;
          if (b_n[kk][j] != 1 || b_src[kk][j] != want) {
            printf("B element (%d, %d) copied %d times, case %d\n", kk, j, b_n[kk][j], it);
            return 1;
          }
        }
      }
      ++cases;
    }
  }
  printf("ok %d chunks\n", cases);
  return 0;
}
"""


def test_fp64_staging_plan_copies_every_element_once(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "check.cpp"
    src.write_text(CHECKER)
    exe = tmp_path / "check"
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")
