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
// ---------------------------------------------------------------------------
constexpr int KC = 16;

__global__ void __launch_bounds__(256) gemm_fp64_kernel(const GemmOut* __restrict__ outs,
                                                        const GemmSeg* __restrict__ segs,
                                                        const int3* __restrict__ tiles, int ntiles,
                                                        const double* __restrict__ xbase,
                                                        double* __restrict__ ybase) {
  __shared__ double As[KC][GEMM_TILE + 2];
  __shared__ double Bs[KC][GEMM_TILE + 2];
  const int w = blockIdx.x;
  if (w >= ntiles) return;
  const int3 wi = tiles[w];
  const GemmOut o = outs[wi.x];
  const int m0 = wi.y * GEMM_TILE, n0 = wi.z * GEMM_TILE;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int s = 0; s < o.seg_count; ++s) {
    GemmSeg g = segs[o.seg_begin + s];
    if (g.a_rel) g.A = xbase + g.a_off;
    if (g.b_rel) g.B = xbase + g.b_off;
    for (int k0 = 0; k0 < g.k; k0 += KC) {
      // A tile: op(A)(m0 + i, k0 + kk) -> As[kk][i]
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int idx = tid + 256 * e;
        int i, kk;
        if (!g.transA) { i = idx / KC; kk = idx % KC; } else { kk = idx / GEMM_TILE; i = idx % GEMM_TILE; }
        const int gi = m0 + i, gk = k0 + kk;
        double v = 0.0;
        if (gi < o.m && gk < g.k)
          v = g.transA ? g.A[(int64_t)gk * g.lda + gi] : g.A[(int64_t)gi * g.lda + gk];
        As[kk][i] = v * g.scale;
      }
      // B tile: op(B)(k0 + kk, n0 + j) -> Bs[kk][j]
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int idx = tid + 256 * e;
        int j, kk;
        if (!g.transB) { kk = idx / GEMM_TILE; j = idx % GEMM_TILE; } else { j = idx / KC; kk = idx % KC; }
        const int gj = n0 + j, gk = k0 + kk;
        double v = 0.0;
        if (gj < o.n && gk < g.k)
          v = g.transB ? g.B[(int64_t)gj * g.ldb + gk] : g.B[(int64_t)gk * g.ldb + gj];
        Bs[kk][j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = m0 + ty + 16 * i;
    if (gi >= o.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = n0 + tx + 16 * j;
      if (gj >= o.n) continue;
      double* c = (o.c_rel ? ybase + o.c_off : o.C) + (int64_t)gi * o.ldc + gj;
      *c = o.accumulate ? (*c + acc[i][j]) : acc[i][j];
    }
  }
}

void launch_gemm_fp64(const GemmOut* outs, const GemmSeg* segs, const int3* tiles, int ntiles,
                      const double* xbase, double* ybase, cudaStream_t st) {
  if (ntiles <= 0) return;
  gemm_fp64_kernel<<<ntiles, 256, 0, st>>>(outs, segs, tiles, ntiles, xbase, ybase);
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
