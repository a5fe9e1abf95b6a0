// Staging plan of one output tile of the grouped FP64 GEMM (gemm_fp64_kernel).
//
// An output tile sums, over its segments q, scale_q * op(A_q) op(B_q).  The segments'
// contracted index ranges are concatenated into one K axis; a batch of up to
// GEMM_SEGB segments has the prefix kst[0..nb] (kst[q] = first K position of
// segment q, kst[nb] = Kb).  The K axis is staged GEMM_KC positions at a time, so
// several short segments share one chunk:
//
//   As[i][kk] = op(A_q)(m0 + i, p - kst[q]),  Bs[kk][j] = op(B_q)(p - kst[q], n0 + j),
//   p = p0 + kk < Kb, q the segment holding p.
//
// Each element is copied by exactly one thread.  Which thread depends on the storage of
// the segment's operand, so a warp's 32 lanes always read consecutive addresses: lanes
// run along K where the operand is K-contiguous, along the rows (A) or columns (B)
// otherwise.  The functions are host-callable so the coverage can be checked on a CPU.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define LRT_HD __host__ __device__ __forceinline__
#else
#define LRT_HD inline
#endif

namespace lrt {

constexpr int GEMM_KC = 32;        // K positions per staged chunk
constexpr int GEMM_SEGB = 32;      // segment descriptors staged per batch (one per lane of warp 0)
constexpr int GEMM_THREADS = 128;
constexpr int GEMM_WARPS = GEMM_THREADS / 32;
constexpr int GEMM_TILE_M = 64;    // equal to GEMM_TM / GEMM_TN of lrt_kernels.h
constexpr int GEMM_TILE_N = 32;

// a segment with its relative pointers resolved.  Vector blocking: when avr > 0 the rows of
// op(A) come in blocks of avr, block v starting at A + v * avs (the same block product for
// the v-th trial vector); when bvc > 0 the columns of op(B) come in blocks of bvc, block v
// starting at B + v * bvs.  A tile then spans the products of several vectors at once.
struct SegS {
  const double* A;
  const double* B;
  int lda, ldb;
  int transA, transB;
  double scale;
  int avr, bvc;
  int64_t avs, bvs;
};

// address of op(A)(row, kl) and op(B)(kl, col) of a segment
LRT_HD const double* seg_a(const SegS& s, int row, int kl) {
  const double* a = s.A;
  if (s.avr > 0) {
    const int v = row / s.avr;
    a += (int64_t)v * s.avs;
    row -= v * s.avr;
  }
  return s.transA ? a + (int64_t)kl * s.lda + row : a + (int64_t)row * s.lda + kl;
}
LRT_HD const double* seg_b(const SegS& s, int kl, int col) {
  const double* b = s.B;
  if (s.bvc > 0) {
    const int v = col / s.bvc;
    b += (int64_t)v * s.bvs;
    col -= v * s.bvc;
  }
  return s.transB ? b + (int64_t)col * s.ldb + kl : b + (int64_t)kl * s.ldb + col;
}

// K parts of an output whose segments have K k[0..nseg) (total ktot): at most `want` runs
// of whole segments, cut after segment q once the K so far reaches (parts + 1) / want of
// ktot, the last run taking whatever remains (zero-K segments included);
// emit(sb, se, kp) for segments [sb, se) with K kp.  Depends on the segment list only.
template <class F>
LRT_HD int split_segments(const int* k, int nseg, long long ktot, int want, F&& emit) {
  int parts = 0, sb = 0;
  long long acc = 0, kp = 0;
  for (int q = 0; q < nseg; ++q) {
    acc += k[q];
    kp += k[q];
    if (q + 1 == nseg || (parts + 1 < want && acc * want >= ktot * (parts + 1))) {
      emit(sb, q + 1, kp);
      ++parts;
      sb = q + 1;
      kp = 0;
    }
  }
  return parts;
}

// the segment holding K position p (p < kst[nb]), searching forward from q
LRT_HD int seg_at(const int* kst, int p, int q) {
  while (kst[q + 1] <= p) ++q;
  return q;
}

// Copies of thread tid for the chunk starting at p0: f(0, i, kk, src) for As[i][kk] and
// f(1, kk, j, src) for Bs[kk][j].
template <class F>
LRT_HD void stage_chunk(int tid, const SegS* sd, const int* kst, int Kb, int p0, int m0, int mt, int n0, int nt,
                        F&& f) {
  static_assert(GEMM_THREADS % 64 == 0 && GEMM_KC == 32 && GEMM_TILE_M == 64 && GEMM_TILE_N == 32,
                "the lane mappings below assume whole pairs of warps, 32-wide chunks and 64 x 32 tiles");
  const int lane = tid & 31, warp = tid >> 5;
  // lanes along K: A and B stored K-contiguous (A row-major, B transposed)
  {
    const int p = p0 + lane;
    if (p < Kb) {
      const int q = seg_at(kst, p, 0);
      const SegS& s = sd[q];
      const int kl = p - kst[q];
      if (!s.transA)
        for (int i = warp; i < mt; i += GEMM_WARPS) f(0, i, lane, seg_a(s, m0 + i, kl));
      if (s.transB)
        for (int j = warp; j < nt; j += GEMM_WARPS) f(1, lane, j, seg_b(s, kl, n0 + j));
    }
  }
  // lanes along the rows of A stored transposed (K-major)
  {
    const int i = tid & 63;
    int q = 0;
    if (i < mt)
      for (int kk = tid >> 6; kk < GEMM_KC; kk += GEMM_THREADS / 64) {
        const int p = p0 + kk;
        if (p >= Kb) break;
        q = seg_at(kst, p, q);
        const SegS& s = sd[q];
        if (s.transA) f(0, i, kk, seg_a(s, m0 + i, p - kst[q]));
      }
  }
  // lanes along the columns of B stored row-major (K-major)
  {
    const int j = lane;
    int q = 0;
    if (j < nt)
      for (int kk = warp; kk < GEMM_KC; kk += GEMM_WARPS) {
        const int p = p0 + kk;
        if (p >= Kb) break;
        q = seg_at(kst, p, q);
        const SegS& s = sd[q];
        if (!s.transB) f(1, kk, j, seg_b(s, p - kst[q], n0 + j));
      }
  }
}

}  // namespace lrt
