// FP64 kernels of the sigma / renormalization path.
//
//  gather:    scaled, optionally transposed block copies summed into destination
//             sub-blocks (building enlarged-block operators, the "x h_i" of
//             Eq. lopr1st); 32x32 tiles, source descriptors staged in shared memory.
//  gemm_fp64: grouped GEMM whose output tiles each loop over a list of
//             (A, B, scale) products (K-concatenation), so all contributions to
//             one output block are summed in registers without atomics.
//  diag:      outer products of operator diagonals (preconditioner of Eq. error).
#include "lrt_kernels.h"
#include "lrt_fp64_tile.h"

#include <algorithm>
#include <atomic>

namespace lrt {

// ---------------------------------------------------------------------------
// gather
// ---------------------------------------------------------------------------
// The sources of a task (a dozen on average for an enlarged operator set, most of them
// blocks of a few tens of rows) are staged as descriptors in shared memory, and their
// loads are unrolled so that several are in flight: a tile costs a few memory round trips
// instead of two per source.  Transposed sources are read straight from global memory;
// the CTA's reads of one source block stay in L1.
// A work item is a chunk of GATHER_CHUNK consecutive elements of the task's row-major
// destination (thread t owns elements t, t + 256, ...): blocks only a few columns wide
// still fill every lane, where square 32 x 32 tiles left most of them idle.  Each
// element sums its sources in the order they are listed.
constexpr int GATHER_SRC_STAGE = 64;
constexpr int GATHER_PER_THREAD = GATHER_CHUNK / 256;

__device__ __forceinline__ void gather_item(const GatherTask* __restrict__ tasks, const GatherSrc* __restrict__ srcs,
                                            const int3 wi, double* dbase, const double* sbase1,
                                            const double* sbase2, GatherSrc* sd) {
  GatherTask t = tasks[wi.x];
  if (dbase) t.dst = dbase + t.dst_off;
  const int tid = threadIdx.x;
  const int64_t n = (int64_t)t.rows * t.cols;
  const int64_t e0 = (int64_t)wi.y * GATHER_CHUNK + tid;
  int rr[GATHER_PER_THREAD], cc[GATHER_PER_THREAD];
  double acc[GATHER_PER_THREAD];
#pragma unroll
  for (int i = 0; i < GATHER_PER_THREAD; ++i) {
    const int64_t e = e0 + 256 * i;
    rr[i] = e < n ? (int)(e / t.cols) : -1;
    cc[i] = e < n ? (int)(e - (int64_t)rr[i] * t.cols) : 0;
    acc[i] = 0.0;
  }
  for (int s0 = 0; s0 < t.src_count; s0 += GATHER_SRC_STAGE) {
    const int ns = min(GATHER_SRC_STAGE, t.src_count - s0);
    __syncthreads();   // the previous descriptors are no longer read
    if (tid < ns) {
      GatherSrc g = srcs[t.src_begin + s0 + tid];
      if (g.rel) g.src = (g.rel == 1 ? sbase1 : sbase2) + g.src_off;
      sd[tid] = g;
    }
    __syncthreads();
#pragma unroll 4
    for (int s = 0; s < ns; ++s) {
      const double* src = sd[s].src;
      const int64_t ld = sd[s].ld;
      const double sc = sd[s].scale;
      const bool tr = sd[s].trans != 0;
#pragma unroll
      for (int i = 0; i < GATHER_PER_THREAD; ++i)
        if (rr[i] >= 0) acc[i] += sc * (tr ? src[(int64_t)cc[i] * ld + rr[i]] : src[(int64_t)rr[i] * ld + cc[i]]);
    }
  }
#pragma unroll
  for (int i = 0; i < GATHER_PER_THREAD; ++i)
    if (rr[i] >= 0) t.dst[(int64_t)rr[i] * t.ld_dst + cc[i]] += acc[i];
}

__global__ void __launch_bounds__(256) gather_kernel(const GatherTask* __restrict__ tasks,
                                                     const GatherSrc* __restrict__ srcs,
                                                     const int3* __restrict__ tiles, int ntiles,
                                                     double* __restrict__ dbase,
                                                     const double* __restrict__ sbase1,
                                                     const double* __restrict__ sbase2) {
  __shared__ GatherSrc sd[GATHER_SRC_STAGE];
  if ((int)blockIdx.x >= ntiles) return;
  gather_item(tasks, srcs, tiles[blockIdx.x], dbase, sbase1, sbase2, sd);
}

__global__ void __launch_bounds__(256) gather_inst_kernel(const GatherTask* __restrict__ tasks,
                                                          const GatherSrc* __restrict__ srcs,
                                                          const int3* __restrict__ tiles, int ntiles,
                                                          const __grid_constant__ GatherInstSet P, int ninst) {
  __shared__ GatherSrc sd[GATHER_SRC_STAGE];
  const int w = blockIdx.x / ninst;
  if (w >= ntiles) return;
  const GatherBases* b = &P.b[blockIdx.x % ninst];
  gather_item(tasks, srcs, tiles[w], b->d, b->s1, b->s2, sd);
}

void launch_gather(const GatherTask* tasks, const GatherSrc* srcs, const int3* tiles, int ntiles,
                   cudaStream_t st, double* dbase, const double* sbase1, const double* sbase2) {
  if (ntiles <= 0) return;
  gather_kernel<<<ntiles, 256, 0, st>>>(tasks, srcs, tiles, ntiles, dbase, sbase1, sbase2);
}

void launch_gather_inst(const GatherTask* tasks, const GatherSrc* srcs, const int3* tiles, int ntiles,
                        const GatherInstSet& bases, int ninst, cudaStream_t st) {
  // the caller checks 1 <= ninst <= 64 and ntiles * ninst < 2^31
  if (ntiles <= 0 || ninst <= 0) return;
  gather_inst_kernel<<<(unsigned)((long long)ntiles * ninst), 256, 0, st>>>(tasks, srcs, tiles, ntiles, bases, ninst);
}

// ---------------------------------------------------------------------------
// grouped FP64 GEMM with K-concatenated segments
//
// GB300 issues about 2 FP64 FMA per clock per SM, so the kernel is bound by the
// number of DFMA warp instructions once its operands arrive in time.  Padding is
// the enemy: each lane owns individual output elements of a <= GEMM_TM x GEMM_TN
// tile (flattened, so only the last warp of a tile is partly idle).  The segments
// of a tile (often a dozen or more, each contracting only ~8 indices) are packed
// along one K axis and staged GEMM_KC positions at a time with cp.async into a
// double buffer, so a chunk's copies are all in flight at once and overlap the
// previous chunk's FMAs (the staging plan is in lrt_fp64_tile.h).
// ---------------------------------------------------------------------------
constexpr int GEMM_MAXE = GEMM_TM * GEMM_TN / GEMM_THREADS;   // outputs per thread
constexpr int GEMM_CTAS = 4;                                   // resident CTAs per SM (registers, shared memory)
static_assert(GEMM_TM == GEMM_TILE_M && GEMM_TN == GEMM_TILE_N, "tile shape of the staging plan");

struct GemmSmem {
  double As[2][GEMM_TM][GEMM_KC + 1];
  double Bs[2][GEMM_KC][GEMM_TN + 1];
  double sc[2][GEMM_KC];          // scale of the segment holding each K position of a chunk
  SegS sd[GEMM_SEGB];
  int kst[GEMM_SEGB + 1];
  int unit[2];                    // every scale of the chunk is 1
};

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// extra base i of a launch (a switch, so the parameter block is not copied to local memory)
__device__ __forceinline__ double* extra_base(const GemmExtra& ex, int i) {
  switch (i) {
    case 0: return ex.p[0];
    case 1: return ex.p[1];
    case 2: return ex.p[2];
    case 3: return ex.p[3];
    case 4: return ex.p[4];
    case 5: return ex.p[5];
    case 6: return ex.p[6];
    default: return ex.p[7];
  }
}

// acc[j] += sum_kk As[row_j][kk] Bs[kk][col_j] over a staged chunk, for the first N outputs
template <int N>
__device__ __forceinline__ void fma_chunk(double (&acc)[GEMM_MAXE], const uint32_t (&rc)[GEMM_MAXE],
                                          const double* __restrict__ As, const double* __restrict__ Bs, int kc) {
  for (int kk = 0; kk < kc; ++kk) {
#pragma unroll
    for (int j = 0; j < N; ++j)
      acc[j] = fma(As[(rc[j] >> 16) * (GEMM_KC + 1) + kk], Bs[kk * (GEMM_TN + 1) + (rc[j] & 0xFFFFu)], acc[j]);
  }
}

// the FMA loop is dispatched by a switch (one indirect branch) over these output counts;
// a chain of compares measured ~10% slower on the small tiles of phase 1
static_assert(GEMM_MAXE == 16, "the switch below lists the output counts 1..16");

// one tile of the grouped GEMM; extra(i) resolves extra base i of the tile's instance
template <class Extra>
__device__ __forceinline__ void gemm_fp64_tile(const GemmOut* __restrict__ outs, const GemmSeg* __restrict__ segs,
                                               const int3 wi, const double* xbase, double* ybase, double* tbase,
                                               double* wbase, const GemmOut& o, const Extra& extra) {
  extern __shared__ __align__(16) unsigned char gemm_smem_raw[];
  GemmSmem& S = *reinterpret_cast<GemmSmem*>(gemm_smem_raw);
  const int m0 = wi.y >> 8, mt = wi.y & 255, n0 = wi.z >> 8, nt = wi.z & 255;
  const int ne = mt * nt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t rc[GEMM_MAXE];        // (row << 16) | col of each owned output element
  double acc[GEMM_MAXE];
#pragma unroll
  for (int j = 0; j < GEMM_MAXE; ++j) {
    const int e = tid + GEMM_THREADS * j;
    rc[j] = e < ne ? ((uint32_t)(e / nt) << 16) | (uint32_t)(e % nt) : 0u;
    acc[j] = 0.0;
  }
  const int cnt = ne > tid ? (ne - tid + GEMM_THREADS - 1) / GEMM_THREADS : 0;
  // outputs of lane 0, the most of any lane of the warp; the other lanes' extra slots
  // accumulate (0, 0)-element products that are never stored
  const int cntw = ne > 32 * warp ? (ne - 32 * warp + GEMM_THREADS - 1) / GEMM_THREADS : 0;

  for (int b0 = 0; b0 < o.seg_count; b0 += GEMM_SEGB) {
    const int nb = min(GEMM_SEGB, o.seg_count - b0);
    __syncthreads();   // the previous batch's descriptors and buffers are no longer read
    if (warp == 0) {
      int k = 0;
      if (lane < nb) {
        GemmSeg g = segs[o.seg_begin + b0 + lane];
        if (g.a_rel) g.A = (g.a_rel == 1 ? xbase : g.a_rel == 2 ? tbase : extra(g.a_rel - 3)) + g.a_off;
        if (g.b_rel) g.B = (g.b_rel == 1 ? xbase : g.b_rel == 2 ? tbase : extra(g.b_rel - 3)) + g.b_off;
        S.sd[lane] = SegS{g.A, g.B, g.lda, g.ldb, g.transA, g.transB, g.scale, g.a_vr, g.b_vc, g.a_vs, g.b_vs};
        k = g.k;
      }
      int incl = k;   // inclusive prefix of k over the lanes
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
      }
      S.kst[lane + 1] = incl;
      if (lane == 0) S.kst[0] = 0;
    }
    __syncthreads();
    const int Kb = S.kst[nb];
    const int nch = (Kb + GEMM_KC - 1) / GEMM_KC;

    auto issue = [&](int c, int buf) {
      const int p0 = c * GEMM_KC;
      stage_chunk(tid, S.sd, S.kst, Kb, p0, m0, mt, n0, nt, [&](int which, int r, int col, const double* src) {
        if (which == 0) cp_async8(&S.As[buf][r][col], src);
        else cp_async8(&S.Bs[buf][r][col], src);
      });
      if (warp == 0) {
        const int p = p0 + lane;
        const double s = p < Kb ? S.sd[seg_at(S.kst, p, 0)].scale : 1.0;
        S.sc[buf][lane] = s;
        const bool u = __all_sync(0xffffffffu, s == 1.0);
        if (lane == 0) S.unit[buf] = u ? 1 : 0;
      }
      cp_async_commit();
    };

    if (nch > 0) issue(0, 0);
    for (int c = 0; c < nch; ++c) {
      const int buf = c & 1;
      if (c + 1 < nch) {
        issue(c + 1, buf ^ 1);   // buffer buf ^ 1 was last read before the previous iteration's barrier
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();           // chunk c has landed for every thread
      const int kc = min(GEMM_KC, Kb - c * GEMM_KC);
      if (!S.unit[buf]) {        // scale row kk of B by its segment's scale
        if (lane < nt)
          for (int kk = warp; kk < kc; kk += GEMM_WARPS) S.Bs[buf][kk][lane] *= S.sc[buf][kk];
        __syncthreads();
      }
      const double* As = &S.As[buf][0][0];
      const double* Bs = &S.Bs[buf][0][0];
      switch (cntw) {            // warp-uniform trip count: no predicated-off DFMA occupies the pipe
#define LRT_FMA_CASE(N) \
  case N: fma_chunk<N>(acc, rc, As, Bs, kc); break;
        LRT_FMA_CASE(1) LRT_FMA_CASE(2) LRT_FMA_CASE(3) LRT_FMA_CASE(4) LRT_FMA_CASE(5) LRT_FMA_CASE(6)
        LRT_FMA_CASE(7) LRT_FMA_CASE(8) LRT_FMA_CASE(9) LRT_FMA_CASE(10) LRT_FMA_CASE(11) LRT_FMA_CASE(12)
        LRT_FMA_CASE(13) LRT_FMA_CASE(14) LRT_FMA_CASE(15) LRT_FMA_CASE(16)
#undef LRT_FMA_CASE
        default: break;
      }
      __syncthreads();           // buffer buf is free for chunk c + 2
    }
  }
  double* cbase = o.c_rel == GEMM_C_SPLIT ? wbase + o.c_off
                 : o.c_rel ? (o.c_rel == 1 ? ybase : o.c_rel == 2 ? tbase : extra(o.c_rel - 3)) + o.c_off : o.C;
#pragma unroll
  for (int j = 0; j < GEMM_MAXE; ++j) {
    if (j >= cnt) break;
    int r = m0 + (int)(rc[j] >> 16), col = n0 + (int)(rc[j] & 0xFFFFu);
    double* c = cbase;
    if (o.c_vr > 0) {            // row blocks of the vectors
      const int v = r / o.c_vr;
      c += (int64_t)v * o.c_vs;
      r -= v * o.c_vr;
    } else if (o.c_vc > 0) {     // column blocks of the vectors
      const int v = col / o.c_vc;
      c += (int64_t)v * o.c_vs;
      col -= v * o.c_vc;
    }
    c += (int64_t)r * o.ldc + col;
    *c = o.accumulate ? (*c + acc[j]) : acc[j];
  }
}

// Per-device state: a process may drive several GPUs (one context per device), and a
// function attribute set with cudaFuncSetAttribute applies to the current device only.
constexpr int MAX_DEVICES = 64;

int gemm_fp64_slots() {
  static std::atomic<int> slots[MAX_DEVICES];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return GEMM_CTAS;
  int n = slots[dev].load(std::memory_order_acquire);
  if (!n) {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    n = std::max(1, nsm) * GEMM_CTAS;
    slots[dev].store(n, std::memory_order_release);
  }
  return n;
}

// Opt the FP64 GEMM into its dynamic shared memory on the current device, once per device.
// On failure the attribute stays unset, the error is the runtime's last error, and the
// caller's launch check reports it.
__global__ void __launch_bounds__(GEMM_THREADS, GEMM_CTAS) gemm_fp64_kernel(const GemmOut* __restrict__ outs,
                                                                    const GemmSeg* __restrict__ segs,
                                                                    const int3* __restrict__ tiles, int ntiles,
                                                                    const double* __restrict__ xbase,
                                                                    double* __restrict__ ybase,
                                                                    double* __restrict__ tbase,
                                                                    const GemmBases* __restrict__ multi,
                                                                    const GemmExtra ex, double* __restrict__ wbase) {
  const int w = blockIdx.x;
  if (w >= ntiles) return;
  const int3 wi = tiles[w];
  const GemmOut o = outs[wi.x];
  if (multi) {
    const GemmBases b = multi[o.inst];
    xbase = b.x;
    ybase = b.y;
    tbase = b.t;
  }
  gemm_fp64_tile(outs, segs, wi, xbase, ybase, tbase, wbase, o, [&](int i) { return extra_base(ex, i); });
}

__global__ void __launch_bounds__(GEMM_THREADS, GEMM_CTAS) gemm_fp64_inst_kernel(const GemmOut* __restrict__ outs,
                                                                         const GemmSeg* __restrict__ segs,
                                                                         const int3* __restrict__ tiles,
                                                                         int ntiles,
                                                                         const __grid_constant__ GemmInstSet P,
                                                                         int ninst) {
  const int w = blockIdx.x / ninst;
  if (w >= ntiles) return;
  const GemmInst* b = &P.b[blockIdx.x % ninst];
  const int3 wi = tiles[w];
  const GemmOut o = outs[wi.x];
  gemm_fp64_tile(outs, segs, wi, b->x, b->y, b->t, nullptr, o, [&](int i) { return b->e[i]; });
}

static cudaError_t gemm_fp64_smem_attr() {
  static std::atomic<int> done[MAX_DEVICES];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  for (const void* f : {(const void*)gemm_fp64_kernel, (const void*)gemm_fp64_inst_kernel}) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GemmSmem));
    if (e != cudaSuccess) return e;
    // all of the unified L1 as shared memory, so GEMM_CTAS CTAs fit on an SM
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
  }
  done[dev].store(1, std::memory_order_release);   // concurrent first calls set the same values
  return cudaSuccess;
}

void launch_gemm_fp64(const GemmOut* outs, const GemmSeg* segs, const int3* tiles, int ntiles,
                      const double* xbase, double* ybase, double* tbase, cudaStream_t st, const GemmExtra* extra,
                      double* wbase) {
  if (ntiles <= 0) return;
  if (gemm_fp64_smem_attr() != cudaSuccess) return;
  const GemmExtra ex = extra ? *extra : GemmExtra{};
  gemm_fp64_kernel<<<ntiles, GEMM_THREADS, sizeof(GemmSmem), st>>>(outs, segs, tiles, ntiles, xbase, ybase, tbase,
                                                                  nullptr, ex, wbase);
}

// One CTA per split tile: each element sums its parts in part order (deterministic), then
// lands where the tile's output puts it, vector blocking included, as in the GEMM epilogue.
__global__ void __launch_bounds__(256) split_reduce_kernel(const GemmOut* __restrict__ outs,
                                                           const SplitTile* __restrict__ tiles,
                                                           const double* __restrict__ wbase,
                                                           double* __restrict__ ybase, double* __restrict__ tbase) {
  const SplitTile t = tiles[blockIdx.x];
  const GemmOut o = outs[t.o];
  double* cbase = o.c_rel == 1 ? ybase + o.c_off : o.c_rel == 2 ? tbase + o.c_off : o.C;
  const int ne = t.mt * t.nt;
  const double* w = wbase + t.ws_off;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < t.nparts; ++p) s += w[(int64_t)p * ne + e];
    int r = t.m0 + e / t.nt, col = t.n0 + e % t.nt;
    double* c = cbase;
    if (o.c_vr > 0) {
      const int v = r / o.c_vr;
      c += (int64_t)v * o.c_vs;
      r -= v * o.c_vr;
    } else if (o.c_vc > 0) {
      const int v = col / o.c_vc;
      c += (int64_t)v * o.c_vs;
      col -= v * o.c_vc;
    }
    c += (int64_t)r * o.ldc + col;
    *c = o.accumulate ? (*c + s) : s;
  }
}

void launch_split_reduce(const GemmOut* outs, const SplitTile* tiles, int ntiles, const double* wbase, double* ybase,
                         double* tbase, cudaStream_t st) {
  if (ntiles <= 0) return;
  split_reduce_kernel<<<ntiles, 256, 0, st>>>(outs, tiles, wbase, ybase, tbase);
}

void launch_gemm_fp64_inst(const GemmOut* outs, const GemmSeg* segs, const int3* tiles, int ntiles,
                           const GemmInstSet& bases, int ninst, cudaStream_t st) {
  // the caller checks 1 <= ninst <= GEMM_MAX_INST and ntiles * ninst < 2^31
  if (ntiles <= 0 || ninst <= 0) return;
  if (gemm_fp64_smem_attr() != cudaSuccess) return;
  gemm_fp64_inst_kernel<<<(unsigned)((long long)ntiles * ninst), GEMM_THREADS, sizeof(GemmSmem), st>>>(
      outs, segs, tiles, ntiles, bases, ninst);
}

void launch_gemm_fp64_multi(const GemmOut* outs, const GemmSeg* segs, const int3* tiles, int ntiles,
                            const GemmBases* bases, cudaStream_t st) {
  if (ntiles <= 0) return;
  if (gemm_fp64_smem_attr() != cudaSuccess) return;
  gemm_fp64_kernel<<<ntiles, GEMM_THREADS, sizeof(GemmSmem), st>>>(outs, segs, tiles, ntiles, nullptr, nullptr,
                                                                  nullptr, bases, GemmExtra{}, nullptr);
}

// ---------------------------------------------------------------------------
// diagonal of H_eff
// ---------------------------------------------------------------------------
// One CTA per output block; term diagonals are staged through shared memory in
// chunks so each element reads them from there instead of from global memory.
constexpr int DIAG_CHUNK = 16;
constexpr int DIAG_MAXD = 128;     // rows and columns of a block staged per chunk (32 KB of shared memory)

__global__ void __launch_bounds__(256) diag_kernel(const DiagOut* __restrict__ outs,
                                                   const DiagTerm* __restrict__ terms,
                                                   double* __restrict__ dbase) {
  __shared__ double xs[DIAG_CHUNK][DIAG_MAXD];   // scale_t * x_t, so one DFMA per term and element
  __shared__ double ys[DIAG_CHUNK][DIAG_MAXD];
  const DiagOut o = outs[blockIdx.x];
  for (int r0 = 0; r0 < o.rows; r0 += DIAG_MAXD)
    for (int c0 = 0; c0 < o.cols; c0 += DIAG_MAXD) {
      const int rt = min(DIAG_MAXD, o.rows - r0), ct = min(DIAG_MAXD, o.cols - c0);
      const int n = rt * ct;
      // each thread keeps up to 8 partial sums in registers, more are revisited below
      for (int base = 0; base < n; base += 8 * blockDim.x) {
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int t0 = 0; t0 < o.term_count; t0 += DIAG_CHUNK) {
          const int tc = min(DIAG_CHUNK, o.term_count - t0);
          __syncthreads();
          for (int e = threadIdx.x; e < tc * (rt + ct); e += blockDim.x) {
            const int t = e / (rt + ct), u = e % (rt + ct);
            const DiagTerm d = terms[o.term_begin + t0 + t];
            if (u < rt) xs[t][u] = d.x ? d.scale * d.x[(int64_t)(r0 + u) * d.xs] : d.scale;
            else ys[t][u - rt] = d.y ? d.y[(int64_t)(c0 + u - rt) * d.ys] : 1.0;
          }
          __syncthreads();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int e = base + threadIdx.x + j * blockDim.x;
            if (e < n) {
              const int i = e / ct, jj = e % ct;
              double a = acc[j];
              for (int t = 0; t < tc; ++t) a = fma(xs[t][i], ys[t][jj], a);
              acc[j] = a;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int e = base + threadIdx.x + j * blockDim.x;
          if (e < n) dbase[o.d_off + (int64_t)(r0 + e / ct) * o.cols + (c0 + e % ct)] = acc[j];
        }
      }
    }
}

void launch_diag(const DiagOut* outs, const DiagTerm* terms, int nouts, double* dbase,
                 cudaStream_t st) {
  if (nouts <= 0) return;
  diag_kernel<<<nouts, 256, 0, st>>>(outs, terms, dbase);
}

}  // namespace lrt

// ---------------------------------------------------------------------------
// Davidson vector operations
// ---------------------------------------------------------------------------
namespace lrt {

__global__ void __launch_bounds__(256) dots_kernel(const double* __restrict__ V, int64_t ld, int m,
                                                   const double* __restrict__ w, int64_t n,
                                                   double* __restrict__ out) {
  __shared__ double red[256];
  const int j = blockIdx.x;
  if (j >= m) return;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc = fma(V[j * ld + e], w[e], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

void launch_dots(const double* V, int64_t ld, int m, const double* w, int64_t n, double* out, cudaStream_t st) {
  if (m <= 0) return;
  dots_kernel<<<m, 256, 0, st>>>(V, ld, m, w, n, out);
}

// out[a * nb + b] = A[a] . B[b] for vectors given by pointer arrays (one block per pair)
__global__ void __launch_bounds__(256) pair_dots_kernel(const double* const* __restrict__ A,
                                                        const double* const* __restrict__ B, int nb, int64_t n,
                                                        double* __restrict__ out) {
  __shared__ double red[256];
  const int a = blockIdx.x / nb, b = blockIdx.x % nb;
  const double* x = A[a];
  const double* y = B[b];
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc = fma(x[e], y[e], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

void launch_pair_dots(const double* const* A, const double* const* B, int na, int nb, int64_t n, double* out,
                      cudaStream_t st) {
  if (na <= 0 || nb <= 0) return;
  pair_dots_kernel<<<na * nb, 256, 0, st>>>(A, B, nb, n, out);
}

__global__ void __launch_bounds__(256) lincomb_kernel(const double* __restrict__ V, int64_t ld, int m,
                                                      const double* __restrict__ coef, int64_t n,
                                                      double* __restrict__ out, double beta) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = beta == 0.0 ? 0.0 : beta * out[e];
    for (int j = 0; j < m; ++j) acc = fma(coef[j], V[j * ld + e], acc);
    out[e] = acc;
  }
}

void launch_lincomb(const double* V, int64_t ld, int m, const double* coef, int64_t n, double* out, double beta,
                    cudaStream_t st) {
  if (n <= 0) return;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  lincomb_kernel<<<grid, 256, 0, st>>>(V, ld, m, coef, n, out, beta);
}

__global__ void __launch_bounds__(256) precond_kernel(const double* __restrict__ r, const double* __restrict__ d,
                                                      double theta, int64_t n, double* __restrict__ t) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double den = d[e] - theta;
    if (fabs(den) < 1e-4) den = den < 0.0 ? -1e-4 : 1e-4;
    t[e] = -r[e] / den;
  }
}

void launch_precond(const double* r, const double* d, double theta, int64_t n, double* t, cudaStream_t st) {
  if (n <= 0) return;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  precond_kernel<<<grid, 256, 0, st>>>(r, d, theta, n, t);
}

// ---------------------------------------------------------------------------
// batched vector operations of the TDA sweeps
// ---------------------------------------------------------------------------
static int vec_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 4)); }

__global__ void __launch_bounds__(256) rank1_batch_kernel(const double* __restrict__ w, int64_t ldw,
                                                          const double* __restrict__ coef, double alpha, int nv,
                                                          double* __restrict__ V, int64_t ld, int64_t n) {
  const int v = blockIdx.y;
  const double c = coef ? alpha * coef[v] : alpha;
  if (c == 0.0) return;
  double* x = V + (int64_t)v * ld;
  const double* y = w + (int64_t)v * ldw;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] = fma(c, y[e], x[e]);
}

void launch_rank1_batch(const double* w, int64_t ldw, const double* coef, double alpha, int nv, double* V,
                        int64_t ld, int64_t n, cudaStream_t st) {
  if (nv <= 0 || n <= 0) return;
  rank1_batch_kernel<<<dim3(vec_grid(n), nv), 256, 0, st>>>(w, ldw, coef, alpha, nv, V, ld, n);
}

// one thread per element and up to ROT_MU outputs at a time: every old vector is read once
// per group of ROT_MU new vectors
constexpr int ROT_MU = 16;
__global__ void __launch_bounds__(256) rotate_kernel(const double* __restrict__ Vold, int64_t ld_old, int lold,
                                                     const double* __restrict__ a, int m, int mu0, int mcnt,
                                                     double* __restrict__ Vnew, int64_t ld_new, int64_t n) {
  __shared__ double sa[JACOBI_MAXN * ROT_MU];
  for (int t = threadIdx.x; t < lold * mcnt; t += blockDim.x) sa[t] = a[(t / mcnt) * m + mu0 + t % mcnt];
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double acc[ROT_MU];
#pragma unroll
    for (int q = 0; q < ROT_MU; ++q) acc[q] = 0.0;
    for (int j = 0; j < lold; ++j) {
      const double x = Vold[(int64_t)j * ld_old + e];
#pragma unroll
      for (int q = 0; q < ROT_MU; ++q)
        if (q < mcnt) acc[q] = fma(sa[j * mcnt + q], x, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < ROT_MU; ++q)
      if (q < mcnt) Vnew[(int64_t)(mu0 + q) * ld_new + e] = acc[q];
  }
}

void launch_rotate(const double* Vold, int64_t ld_old, int lold, const double* a, int m, double* Vnew,
                   int64_t ld_new, int64_t n, cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  if (lold <= 0) {
    for (int mu = 0; mu < m; ++mu) cudaMemsetAsync(Vnew + (int64_t)mu * ld_new, 0, (size_t)n * sizeof(double), st);
    return;
  }
  for (int mu0 = 0; mu0 < m; mu0 += ROT_MU)
    rotate_kernel<<<vec_grid(n), 256, 0, st>>>(Vold, ld_old, lold, a, m, mu0, std::min(ROT_MU, m - mu0), Vnew,
                                               ld_new, n);
}

__global__ void __launch_bounds__(256) precond_batch_kernel(const double* __restrict__ R, int64_t ldr,
                                                            const double* __restrict__ d,
                                                            const double* __restrict__ theta, int64_t n,
                                                            double* __restrict__ Z, int64_t ldz, double sign) {
  const int v = blockIdx.y;
  const double th = theta[v];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double den = d[e] - th;
    if (fabs(den) < 1e-4) den = den < 0.0 ? -1e-4 : 1e-4;
    Z[(int64_t)v * ldz + e] = -sign * R[(int64_t)v * ldr + e] / den;
  }
}

__global__ void __launch_bounds__(256) precond_abs_kernel(const double* __restrict__ R, const double* __restrict__ d,
                                                          double shift, int64_t n, double* __restrict__ Z) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    Z[e] = R[e] / fmax(fabs(d[e] - shift), 1e-4);
}

void launch_precond_abs(const double* R, const double* d, double shift, int64_t n, double* Z, cudaStream_t st) {
  if (n <= 0) return;
  precond_abs_kernel<<<vec_grid(n), 256, 0, st>>>(R, d, shift, n, Z);
}

void launch_precond_batch(const double* R, int64_t ldr, const double* d, const double* theta, int nv, int64_t n,
                          double* Z, int64_t ldz, double sign, cudaStream_t st) {
  if (nv <= 0 || n <= 0) return;
  precond_batch_kernel<<<dim3(vec_grid(n), nv), 256, 0, st>>>(R, ldr, d, theta, n, Z, ldz, sign);
}

// first pass: CTA (pair p, chunk c) sums its share of the elements of pair p
__device__ __forceinline__ double block_sum256(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  return red[0];
}

__global__ void __launch_bounds__(256) vdots_part_kernel(const double* __restrict__ A, int64_t lda,
                                                         const double* __restrict__ B, int64_t ldb, int nb,
                                                         int64_t n, int pairs_mode, double* __restrict__ work) {
  __shared__ double red[256];
  const int p = blockIdx.y, c = blockIdx.x;
  const int a = pairs_mode ? p / nb : p;
  const int b = pairs_mode ? p % nb : p;
  const double* x = A + (int64_t)a * lda;
  const double* y = B + (int64_t)b * ldb;
  const int64_t per = (n + DOT_CHUNKS - 1) / DOT_CHUNKS;
  const int64_t e0 = (int64_t)c * per, e1 = min(n, e0 + per);
  double acc = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) acc = fma(x[e], y[e], acc);
  const double s = block_sum256(acc, red);
  if (threadIdx.x == 0) work[(int64_t)p * DOT_CHUNKS + c] = s;
}

__global__ void vdots_sum_kernel(const double* __restrict__ work, int np, double* __restrict__ out, int accumulate) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double s = 0.0;
  for (int c = 0; c < DOT_CHUNKS; ++c) s += work[(int64_t)p * DOT_CHUNKS + c];
  out[p] = accumulate ? out[p] + s : s;
}

void launch_vdots(const double* A, int64_t lda, const double* B, int64_t ldb, int nv, int64_t n, double* out,
                  bool accumulate, double* work, cudaStream_t st) {
  if (nv <= 0) return;
  vdots_part_kernel<<<dim3(DOT_CHUNKS, nv), 256, 0, st>>>(A, lda, B, ldb, 1, n, 0, work);
  vdots_sum_kernel<<<(nv + 127) / 128, 128, 0, st>>>(work, nv, out, accumulate ? 1 : 0);
}

void launch_pair_dots_strided(const double* A, int64_t lda, int na, const double* B, int64_t ldb, int nb, int64_t n,
                              double* out, double* work, cudaStream_t st) {
  if (na <= 0 || nb <= 0) return;
  vdots_part_kernel<<<dim3(DOT_CHUNKS, na * nb), 256, 0, st>>>(A, lda, B, ldb, nb, n, 1, work);
  vdots_sum_kernel<<<(na * nb + 127) / 128, 128, 0, st>>>(work, na * nb, out, 0);
}

__global__ void gather_sum_kernel(const double* __restrict__ src, const int* __restrict__ beg,
                                  const int* __restrict__ idx, const double* __restrict__ coef, int nout,
                                  double* __restrict__ out) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nout) return;
  double s = 0.0;
  for (int j = beg[d]; j < beg[d + 1]; ++j) s = fma(coef[j], src[idx[j]], s);
  out[d] += s;
}

void launch_gather_sum(const double* src, const int* beg, const int* idx, const double* coef, int nout, double* out,
                       cudaStream_t st) {
  if (nout <= 0) return;
  gather_sum_kernel<<<(nout + 127) / 128, 128, 0, st>>>(src, beg, idx, coef, nout, out);
}

__global__ void reduced_acc_kernel(const double* __restrict__ D1, const double* __restrict__ D2,
                                   const double* __restrict__ D3, int l, double* __restrict__ Hr,
                                   double* __restrict__ Sr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= l * l) return;
  const int a = t / l, b = t % l;
  Hr[t] += D1[t] + D2[t] + D2[b * l + a];
  Sr[t] += D3[t];
}

void launch_reduced_acc(const double* D1, const double* D2, const double* D3, int l, double* Hr, double* Sr,
                        cudaStream_t st) {
  if (l <= 0) return;
  reduced_acc_kernel<<<(l * l + 127) / 128, 128, 0, st>>>(D1, D2, D3, l, Hr, Sr);
}

// Cyclic Jacobi eigenvalue iteration for a small symmetric matrix held in shared
// memory (n <= JACOBI_MAXN = 48): each rotation zeroes A[p][q]; sweeps stop when the off-diagonal norm is
// below 1e-15 of the Frobenius norm, or after a fixed number of sweeps.
__global__ void __launch_bounds__(256) jacobi_kernel(double* __restrict__ Ag, int n, double* __restrict__ w,
                                                     double* __restrict__ Zg) {
  __shared__ double A[JACOBI_MAXN][JACOBI_MAXN + 1];
  __shared__ double Z[JACOBI_MAXN][JACOBI_MAXN + 1];
  __shared__ double cs[2];
  __shared__ double off;
  __shared__ int order[JACOBI_MAXN];
  const int tid = threadIdx.x;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    A[i][j] = 0.5 * (Ag[i * n + j] + Ag[j * n + i]);
    Z[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) {
      double o = 0.0, f = 0.0;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          f += A[i][j] * A[i][j];
          if (i != j) o += A[i][j] * A[i][j];
        }
      off = (o <= 1e-30 * f) ? -1.0 : o;
    }
    __syncthreads();
    if (off < 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (tid == 0) {
          const double apq = A[p][q];
          double c = 1.0, s = 0.0;
          if (apq != 0.0) {
            const double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
          cs[0] = c;
          cs[1] = s;
        }
        __syncthreads();
        const double c = cs[0], s = cs[1];
        if (s != 0.0) {
          // rotate columns p, q of A and Z
          for (int i = tid; i < n; i += blockDim.x) {
            const double aip = A[i][p], aiq = A[i][q];
            A[i][p] = c * aip - s * aiq;
            A[i][q] = s * aip + c * aiq;
            const double zip = Z[i][p], ziq = Z[i][q];
            Z[i][p] = c * zip - s * ziq;
            Z[i][q] = s * zip + c * ziq;
          }
          __syncthreads();
          // rotate rows p, q of A
          for (int j = tid; j < n; j += blockDim.x) {
            const double apj = A[p][j], aqj = A[q][j];
            A[p][j] = c * apj - s * aqj;
            A[q][j] = s * apj + c * aqj;
          }
        }
        __syncthreads();
      }
  }
  if (tid == 0) {
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int i = 1; i < n; ++i) {       // insertion sort by eigenvalue
      const int v = order[i];
      int j = i - 1;
      while (j >= 0 && A[order[j]][order[j]] > A[v][v]) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = v;
    }
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    Zg[i * n + j] = Z[i][order[j]];
  }
  for (int i = tid; i < n; i += blockDim.x) w[i] = A[order[i]][order[i]];
}

void launch_jacobi_eigh(double* A, int n, double* w, double* Z, cudaStream_t st) {
  if (n <= 0) return;
  jacobi_kernel<<<1, 64, 0, st>>>(A, n, w, Z);
}

}  // namespace lrt
