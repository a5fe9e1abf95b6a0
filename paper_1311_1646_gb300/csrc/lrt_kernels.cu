// FP64 kernels of the sigma / renormalization path.
//
//  gather:    scaled, optionally transposed block copies summed into destination
//             sub-blocks (building enlarged-block operators, the "x h_i" of
//             Eq. lopr1st); HBM-bound, 32x32 tiles staged through shared memory.
//  gemm_fp64: grouped GEMM whose output tiles each loop over a list of
//             (A, B, scale) products (K-concatenation), so all contributions to
//             one output block are summed in registers without atomics.
//  diag:      outer products of operator diagonals (preconditioner of Eq. error).
#include "lrt_kernels.h"

namespace lrt {

// ---------------------------------------------------------------------------
// gather
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) gather_kernel(const GatherTask* __restrict__ tasks,
                                                     const GatherSrc* __restrict__ srcs,
                                                     const int3* __restrict__ tiles, int ntiles) {
  __shared__ double tile[GATHER_TILE][GATHER_TILE + 1];
  const int w = blockIdx.x;
  if (w >= ntiles) return;
  const int3 wi = tiles[w];
  const GatherTask t = tasks[wi.x];
  const int r0 = wi.y * GATHER_TILE, c0 = wi.z * GATHER_TILE;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int s = 0; s < t.src_count; ++s) {
    const GatherSrc g = srcs[t.src_begin + s];
    if (!g.trans) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty + 8 * i, c = c0 + tx;
        if (r < t.rows && c < t.cols) acc[i] += g.scale * g.src[(int64_t)r * g.ld + c];
      }
    } else {
      // dst(r, c) = src(c, r): stage src rows c0.. (cols r0..) coalesced, read transposed
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int cc = ty + 8 * i;          // src row offset (= dst col)
        const int rr = tx;                  // src col offset (= dst row)
        const int c = c0 + cc, r = r0 + rr;
        tile[cc][rr] = (c < t.cols && r < t.rows) ? g.src[(int64_t)c * g.ld + r] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int rr = ty + 8 * i, cc = tx;
        acc[i] += g.scale * tile[cc][rr];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 8 * i, c = c0 + tx;
    if (r < t.rows && c < t.cols) t.dst[(int64_t)r * t.ld_dst + c] += acc[i];
  }
}

void launch_gather(const GatherTask* tasks, const GatherSrc* srcs, const int3* tiles, int ntiles,
                   cudaStream_t st) {
  if (ntiles <= 0) return;
  gather_kernel<<<ntiles, dim3(32, 8), 0, st>>>(tasks, srcs, tiles, ntiles);
}

// ---------------------------------------------------------------------------
// grouped FP64 GEMM with K-concatenated segments
//
// GB300 issues about 2 FP64 FMA per clock per SM, so the kernel is bound by the
// number of DFMA warp instructions, not by operand bandwidth.  Register tiling
// is therefore pointless and padding is the enemy: each lane owns individual
// output elements of a <= GEMM_TM x GEMM_TN tile (flattened, so only the last
// warp of a tile is partly idle) and the K loop runs the exact trip count.
// ---------------------------------------------------------------------------
constexpr int KC = 16;
constexpr int GEMM_THREADS = 128;
constexpr int GEMM_MAXE = GEMM_TM * GEMM_TN / GEMM_THREADS;   // outputs per thread

__global__ void __launch_bounds__(GEMM_THREADS) gemm_fp64_kernel(const GemmOut* __restrict__ outs,
                                                                 const GemmSeg* __restrict__ segs,
                                                                 const int3* __restrict__ tiles, int ntiles,
                                                                 const double* __restrict__ xbase,
                                                                 double* __restrict__ ybase,
                                                                 double* __restrict__ tbase) {
  __shared__ double As[GEMM_TM][KC + 1];
  __shared__ double Bs[KC][GEMM_TN + 1];
  const int w = blockIdx.x;
  if (w >= ntiles) return;
  const int3 wi = tiles[w];
  const GemmOut o = outs[wi.x];
  const int m0 = wi.y * GEMM_TM, n0 = wi.z * GEMM_TN;
  const int mt = min(GEMM_TM, o.m - m0), nt = min(GEMM_TN, o.n - n0);
  const int ne = mt * nt;
  const int tid = threadIdx.x;
  int ri[GEMM_MAXE], ci[GEMM_MAXE];
  double acc[GEMM_MAXE];
#pragma unroll
  for (int j = 0; j < GEMM_MAXE; ++j) {
    const int e = tid + GEMM_THREADS * j;
    ri[j] = e < ne ? e / nt : 0;
    ci[j] = e < ne ? e % nt : 0;
    acc[j] = 0.0;
  }
  const int cnt = ne > tid ? (ne - tid + GEMM_THREADS - 1) / GEMM_THREADS : 0;

  for (int s = 0; s < o.seg_count; ++s) {
    GemmSeg g = segs[o.seg_begin + s];
    if (g.a_rel) g.A = (g.a_rel == 1 ? xbase : tbase) + g.a_off;
    if (g.b_rel) g.B = (g.b_rel == 1 ? xbase : tbase) + g.b_off;
    for (int k0 = 0; k0 < g.k; k0 += KC) {
      const int kc = min(KC, g.k - k0);
      for (int e = tid; e < mt * kc; e += GEMM_THREADS) {
        int i, kk;
        if (!g.transA) { i = e / kc; kk = e % kc; } else { kk = e / mt; i = e % mt; }
        const int gi = m0 + i, gk = k0 + kk;
        As[i][kk] = g.scale * (g.transA ? g.A[(int64_t)gk * g.lda + gi] : g.A[(int64_t)gi * g.lda + gk]);
      }
      for (int e = tid; e < kc * nt; e += GEMM_THREADS) {
        int j, kk;
        if (!g.transB) { kk = e / nt; j = e % nt; } else { j = e / kc; kk = e % kc; }
        const int gj = n0 + j, gk = k0 + kk;
        Bs[kk][j] = g.transB ? g.B[(int64_t)gj * g.ldb + gk] : g.B[(int64_t)gk * g.ldb + gj];
      }
      __syncthreads();
      for (int kk = 0; kk < kc; ++kk) {
#pragma unroll
        for (int j = 0; j < GEMM_MAXE; ++j)
          if (j < cnt) acc[j] = fma(As[ri[j]][kk], Bs[kk][ci[j]], acc[j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int j = 0; j < GEMM_MAXE; ++j) {
    if (j >= cnt) break;
    double* c = (o.c_rel ? (o.c_rel == 1 ? ybase : tbase) + o.c_off : o.C) + (int64_t)(m0 + ri[j]) * o.ldc +
                (n0 + ci[j]);
    *c = o.accumulate ? (*c + acc[j]) : acc[j];
  }
}

void launch_gemm_fp64(const GemmOut* outs, const GemmSeg* segs, const int3* tiles, int ntiles,
                      const double* xbase, double* ybase, double* tbase, cudaStream_t st) {
  if (ntiles <= 0) return;
  gemm_fp64_kernel<<<ntiles, GEMM_THREADS, 0, st>>>(outs, segs, tiles, ntiles, xbase, ybase, tbase);
}

// ---------------------------------------------------------------------------
// diagonal of H_eff
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) diag_kernel(const DiagOut* __restrict__ outs,
                                                   const DiagTerm* __restrict__ terms,
                                                   double* __restrict__ dbase) {
  const DiagOut o = outs[blockIdx.x];
  const int n = o.rows * o.cols;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int i = e / o.cols, j = e % o.cols;
    double acc = 0.0;
    for (int t = 0; t < o.term_count; ++t) {
      const DiagTerm d = terms[o.term_begin + t];
      const double xv = d.x ? d.x[(int64_t)i * d.xs] : 1.0;
      const double yv = d.y ? d.y[(int64_t)j * d.ys] : 1.0;
      acc += d.scale * xv * yv;
    }
    dbase[o.d_off + e] = acc;
  }
}

void launch_diag(const DiagOut* outs, const DiagTerm* terms, int nouts, double* dbase,
                 cudaStream_t st) {
  if (nouts <= 0) return;
  diag_kernel<<<nouts, 256, 0, st>>>(outs, terms, dbase);
}

}  // namespace lrt
