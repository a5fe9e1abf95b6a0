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

// a segment with its relative pointers resolved
struct SegS {
  const double* A;
  const double* B;
  int lda, ldb;
  int transA, transB;
  double scale;
};

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
        for (int i = warp; i < mt; i += GEMM_WARPS) f(0, i, lane, s.A + (int64_t)(m0 + i) * s.lda + kl);
      if (s.transB)
        for (int j = warp; j < nt; j += GEMM_WARPS) f(1, lane, j, s.B + (int64_t)(n0 + j) * s.ldb + kl);
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
        if (s.transA) f(0, i, kk, s.A + (int64_t)(p - kst[q]) * s.lda + m0 + i);
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
        if (!s.transB) f(1, kk, j, s.B + (int64_t)(p - kst[q]) * s.ldb + n0 + j);
      }
  }
}

}  // namespace lrt
