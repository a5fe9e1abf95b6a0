// Split-TF32 tensor-core GEMM (tcgen05, sm_103a) for the mixed-precision path.
//
// Same task structure as gemm_fp64_kernel: every output tile (128 rows x 64
// columns) sums K-concatenated products scale_s * op(A_s) op(B_s).  Operands are
// held as TF32 pairs x = hi + lo (hi = rna(x), lo = rna(x - hi) of the FP32-rounded
// value), split once per operator set and once per input vector, and the product is
// accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi (lo*lo is below FP32 resolution).
// Each product (segment) accumulates in FP32 in tensor memory; the running sum over
// the segments of a tile is a compensated (two-sum) FP32 pair in registers, folded
// in once per finished segment, so plain FP32 accumulation spans only the K of one
// block product.  No FP64 arithmetic runs in the loop: on this GPU the FP64 pipe is
// the scarcest resource.
//
// Persistent, warp-specialised kernel (one CTA per SM, tiles dealt round-robin in
// the host's longest-first order; 8 warps, so two per SM sub-partition and up to 255
// registers a thread for the epilogue's 128 running-sum registers):
//   warps 4-6  producers: copy K chunks of 32 of the four operand tiles from global
//              memory into a 4-stage ring in shared memory, 128-byte-swizzled K-major
//              (the layout tcgen05 reads with SWIZZLE_128B descriptors), zero-filling
//              the K tail; arrive on full[stage].
//   warp 7     one thread issues 3 x (K / 8) tcgen05.mma per chunk into one of two
//              TMEM accumulators (64 columns each), commits the stage back to its
//              producers and, after the last chunk of a product, commits the
//              accumulator to the epilogue.
//   warps 0-3  epilogue: thread = tile row = TMEM lane; folds each finished product
//              into the compensated sum, releases the accumulator, stores the tile.
// The block products are small (rows and columns of a few tens), so instead of TMA
// (one tensor map per operand would be needed) the producers gather with coalesced
// loads: along K for K-contiguous operands (one row of 32 per warp instruction, a
// conflict-free 128-byte shared store) and along M/N for transposed ones (32 rows per
// instruction, four K values per thread packed into one 16-byte store).
//
// Every wait is bounded by the global timer and also ends when another role has
// failed: on expiry the kernel records an error code, stops issuing work, waits (with
// a bound) for its own MMAs in flight, releases its tensor memory and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lrt_kernels.h"

namespace lrt {

namespace {

constexpr int TC_M = 128;               // rows of an output tile (one TMEM lane per row)
constexpr int TC_N = 64;                // columns of an output tile (TMEM columns)
constexpr int TC_K = 32;                // K elements per stage (one 128-byte swizzle row)
constexpr int STAGES = 4;
constexpr int EPI_WARPS = 4, PROD_WARPS = 3;
constexpr int TC_THREADS = 32 * (EPI_WARPS + PROD_WARPS + 1);
constexpr int A_BYTES = TC_M * TC_K * 4;    // one TF32 operand tile of A (16 KB)
constexpr int B_BYTES = TC_N * TC_K * 4;    // 8 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr uint32_t TMEM_COLS = 2 * TC_N;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s per wait

static_assert(STAGE_BYTES % 1024 == 0 && A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0,
              "swizzle atoms must stay 1024-byte aligned");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) of a 128-byte-swizzled K-major tile with TC_K = 32
// columns: row r occupies bytes [128 r, 128 r + 128); its 16-byte chunk c (elements
// 4c..4c+3) sits at chunk position c XOR (r mod 8).
__device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
  return (uint32_t)((row << 7) + ((((k >> 2) ^ row) & 7) << 4) + ((k & 3) << 2));
}

// shared-memory matrix descriptor, K-major, SWIZZLE_128B: 8-row groups 1024 bytes
// apart (SBO), LBO unused for swizzled K-major layouts (set to 1)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;                 // descriptor version for this architecture
  d |= (uint64_t)2 << 61;                 // layout: 128-byte swizzle
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = TC_N
__host__ __device__ constexpr uint32_t make_idesc() {
  return (1u << 4)                        // D format F32
         | (2u << 7)                      // A format TF32
         | (2u << 10)                     // B format TF32
         | ((uint32_t)(TC_N >> 3) << 17)  // N / 8
         | ((uint32_t)(TC_M >> 4) << 24); // M / 16
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  uint64_t state;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(smem_u32(bar)) : "memory");
  (void)state;
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(a), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait for the phase with the given parity; false on expiry or when another
// role has already failed (then the caller stops)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* failed, int* err) {
  const uint32_t a = smem_u32(bar);
  if (mbar_try(a, parity)) return true;
  const uint64_t t0 = now_ns();
  for (;;) {
    if (mbar_try(a, parity)) return true;
    if (*failed) return false;
    if (now_ns() - t0 > WAIT_NS) {
      *failed = 1;
      if (err) atomicExch(err, 1);
      return false;
    }
  }
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void ld_16cols(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// One operand as the producers see it: tile row r (output row for A, output column
// for B) against K.  A segment's transA matches `trans`; its transB is the opposite
// (transB = 1 stores B as N x K, i.e. K-contiguous).
struct Operand {
  const float* hi;
  const float* lo;
  int64_t ld;
  int trans;      // 0: element (r, k) at r * ld + k (K-contiguous); 1: at k * ld + r
};

// 4-byte asynchronous global -> shared copy; src_bytes = 0 writes a zero and reads nothing
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// Issue the copies of rows [0, nr) x K [k0, k0 + kc) of an operand into a swizzled
// tile pair, zero-filling K in [kc, kpad).  Executed by the PROD_WARPS producer warps;
// rows >= nr are left as they are (they only reach output rows/columns never stored).
__device__ __forceinline__ void stage_operand(const Operand& op, int r0, int nr, int k0, int kc, int kpad,
                                              uint32_t shi, uint32_t slo, int pw, int lane) {
  if (!op.trans) {
    // lane = k: one tile row per warp instruction, 128 contiguous bytes of the source
    const int kk = lane;
    if (kk >= kpad) return;
    const uint32_t nb = kk < kc ? 4u : 0u;
    const int ks = kk < kc ? kk : 0;
    for (int r = pw; r < nr; r += PROD_WARPS) {
      const int64_t idx = (int64_t)(r0 + r) * op.ld + (k0 + ks);
      const uint32_t off = sw128_offset(r, kk);
      cp_async4(shi + off, op.hi + idx, nb);
      cp_async4(slo + off, op.lo + idx, nb);
    }
  } else {
    // lane = (row mod 8, k mod 4): 8 rows x 4 K per warp instruction, four 32-byte
    // source sectors and 32 distinct shared-memory banks
    const int rr = lane & 7, q = lane >> 3;
    const int ngroups = (nr + 7) >> 3;
    const int nchunks = kpad >> 2;
    for (int item = pw; item < ngroups * nchunks; item += PROD_WARPS) {
      const int grp = item / nchunks, c = item - grp * nchunks;
      const int r = grp * 8 + rr, kk = 4 * c + q;
      if (r >= nr) continue;
      const uint32_t nb = kk < kc ? 4u : 0u;
      const int64_t idx = (int64_t)(k0 + (kk < kc ? kk : 0)) * op.ld + (r0 + r);
      const uint32_t off = sw128_offset(r, kk);
      cp_async4(shi + off, op.hi + idx, nb);
      cp_async4(slo + off, op.lo + idx, nb);
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(TC_THREADS, 1) gemm_tf32x3_kernel(const GemmOut* __restrict__ outs,
                                                                     const TcSeg* __restrict__ segs,
                                                                     const int3* __restrict__ tiles, int ntiles,
                                                                     TcBases bases, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2], tempty_bar[2], drain_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed_s;
  volatile int* failed = &failed_s;
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 32 * PROD_WARPS);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull_bar[a], 1);
      mbar_init(&tempty_bar[a], 32 * EPI_WARPS);
    }
    mbar_init(&drain_bar, 1);
    failed_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp >= EPI_WARPS && warp < EPI_WARPS + PROD_WARPS) {
    // ---------------- producers
    // Copies of chunk `it` are one cp.async group; the group LAG chunks older is
    // waited for, fenced to the async proxy and announced on its full barrier, so
    // LAG + 1 chunks of copies are in flight per thread.
    constexpr int LAG = 2;
    static_assert(LAG < STAGES, "the producer must not wait on a stage it has not announced");
    const int pw = warp - EPI_WARPS;
    uint32_t it = 0;
    const uint32_t sbase = smem_u32(sm);
    for (int w = blockIdx.x; w < ntiles && !*failed; w += gridDim.x) {
      const int3 wi = tiles[w];
      const GemmOut o = outs[wi.x];
      const int m0 = wi.y * TC_M, n0 = wi.z * TC_N;
      const int mt = min(TC_M, o.m - m0), nt = min(TC_N, o.n - n0);
      for (int s = 0; s < o.seg_count && !*failed; ++s) {
        const TcSeg g = segs[o.seg_begin + s];
        if (g.k <= 0) continue;
        Operand A{g.a_rel ? (g.a_rel == 1 ? bases.xhi : bases.thi) + g.a_off : g.Ahi,
                  g.a_rel ? (g.a_rel == 1 ? bases.xlo : bases.tlo) + g.a_off : g.Alo, g.lda, g.transA};
        Operand B{g.b_rel ? (g.b_rel == 1 ? bases.xhi : bases.thi) + g.b_off : g.Bhi,
                  g.b_rel ? (g.b_rel == 1 ? bases.xlo : bases.tlo) + g.b_off : g.Blo, g.ldb, !g.transB};
        for (int k0 = 0; k0 < g.k; k0 += TC_K, ++it) {
          const int kc = min(TC_K, g.k - k0), kpad = (kc + 7) & ~7;
          const uint32_t stage = it % STAGES, round = it / STAGES;
          if (round > 0 && !mbar_wait(&empty_bar[stage], (round - 1) & 1, failed, err)) break;
          const uint32_t st = sbase + stage * STAGE_BYTES;
          stage_operand(A, m0, mt, k0, kc, kpad, st, st + A_BYTES, pw, lane);
          stage_operand(B, n0, nt, k0, kc, kpad, st + 2 * A_BYTES, st + 2 * A_BYTES + B_BYTES, pw, lane);
          asm volatile("cp.async.commit_group;" ::: "memory");
          if (it >= (uint32_t)LAG) {
            asm volatile("cp.async.wait_group %0;" ::"n"(LAG) : "memory");
            // generic-proxy writes -> visible to the tensor core's async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&full_bar[(it - LAG) % STAGES]);
          }
        }
      }
    }
    // announce the chunks still in flight
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!*failed)
      for (uint32_t j = (it > (uint32_t)LAG ? it - LAG : 0u); j < it; ++j) mbar_arrive(&full_bar[j % STAGES]);
  } else if (warp == EPI_WARPS + PROD_WARPS) {
    // ---------------- MMA issuer (one thread)
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc();
      uint32_t it = 0, sg = 0;
      bool any = false;
      for (int w = blockIdx.x; w < ntiles && !*failed; w += gridDim.x) {
        const GemmOut o = outs[tiles[w].x];
        for (int s = 0; s < o.seg_count && !*failed; ++s) {
          const int k = segs[o.seg_begin + s].k;
          if (k <= 0) continue;
          const uint32_t a = sg & 1, u = sg >> 1;
          if (u > 0 && !mbar_wait(&tempty_bar[a], (u - 1) & 1, failed, err)) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dt = tmem + a * TC_N;
          bool first = true;
          for (int k0 = 0; k0 < k; k0 += TC_K, ++it) {
            const int nks = (min(TC_K, k - k0) + 7) >> 3;
            const uint32_t stage = it % STAGES, round = it / STAGES;
            if (!mbar_wait(&full_bar[stage], round & 1, failed, err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(sm + stage * STAGE_BYTES);
            const uint32_t ah = base, al = base + A_BYTES, bh = base + 2 * A_BYTES, bl = bh + B_BYTES;
            for (int ks = 0; ks < nks; ++ks) {
              const uint32_t step = (uint32_t)ks * 32u;     // 8 TF32 = 32 bytes along K
              mma_tf32(dt, make_desc(ah + step), make_desc(bh + step), idesc, first ? 0u : 1u);
              mma_tf32(dt, make_desc(ah + step), make_desc(bl + step), idesc, 1u);
              mma_tf32(dt, make_desc(al + step), make_desc(bh + step), idesc, 1u);
              first = false;
            }
            mma_commit(&empty_bar[stage]);
            any = true;
          }
          if (*failed) break;
          mma_commit(&tfull_bar[a]);
          ++sg;
        }
      }
      if (*failed && any) {
        // let the MMAs already issued finish before the tensor memory is released
        mma_commit(&drain_bar);
        const uint32_t da = smem_u32(&drain_bar);
        const uint64_t t0 = now_ns();
        while (!mbar_try(da, 0) && now_ns() - t0 < WAIT_NS) {
        }
      }
    }
  } else {
    // ---------------- epilogue: thread = tile row = TMEM lane
    const int row = tid;
    uint32_t sg = 0;
    for (int w = blockIdx.x; w < ntiles && !*failed; w += gridDim.x) {
      const int3 wi = tiles[w];
      const GemmOut o = outs[wi.x];
      const int m0 = wi.y * TC_M, n0 = wi.z * TC_N;
      const int mt = min(TC_M, o.m - m0), nt = min(TC_N, o.n - n0);
      float sum[TC_N], cmp[TC_N];
#pragma unroll
      for (int c = 0; c < TC_N; ++c) sum[c] = cmp[c] = 0.0f;
      for (int s = 0; s < o.seg_count; ++s) {
        const TcSeg g = segs[o.seg_begin + s];
        if (g.k <= 0) continue;
        const uint32_t a = sg & 1, u = sg >> 1;
        // the warp stays converged for the .sync.aligned tensor-memory loads
        const bool ok = mbar_wait(&tfull_bar[a], u & 1, failed, err);
        if (!__all_sync(0xffffffffu, ok)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + a * TC_N;
#pragma unroll
        for (int c0 = 0; c0 < TC_N; c0 += 16) {
          float v[16];
          ld_16cols(taddr + (uint32_t)c0, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float y = g.scale * v[i] - cmp[c0 + i];
            const float t = sum[c0 + i] + y;
            cmp[c0 + i] = (t - sum[c0 + i]) - y;
            sum[c0 + i] = t;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&tempty_bar[a]);
        ++sg;
      }
      if (*failed) break;
      if (row < mt) {
        if (o.c_rel == 2) {
          // intermediate: keep it as a TF32 pair for the next phase
#pragma unroll
          for (int c = 0; c < TC_N; ++c) {
            if (c < nt) {
              const float v = sum[c] - cmp[c];
              uint32_t hi, lo;
              split_tf32(v, hi, lo);
              const int64_t idx = o.c_off + (int64_t)(m0 + row) * o.ldc + (n0 + c);
              bases.thi[idx] = __uint_as_float(hi);
              bases.tlo[idx] = __uint_as_float(lo);
            }
          }
        } else {
          double* C = (o.c_rel == 1 ? bases.y + o.c_off : o.C);
#pragma unroll
          for (int c = 0; c < TC_N; ++c) {
            if (c < nt) {
              const double v = (double)sum[c] - (double)cmp[c];
              double* p = C + (int64_t)(m0 + row) * o.ldc + (n0 + c);
              *p = o.accumulate ? (*p + v) : v;
            }
          }
        }
      }
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

__global__ void __launch_bounds__(256) split_tf32_kernel(const double* __restrict__ src, int64_t n,
                                                         float* __restrict__ hi, float* __restrict__ lo) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h, l;
    split_tf32((float)src[e], h, l);
    hi[e] = __uint_as_float(h);
    lo[e] = __uint_as_float(l);
  }
}

void launch_split_tf32(const double* src, int64_t n, float* hi, float* lo, cudaStream_t st) {
  if (n <= 0) return;
  const int grid = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
  split_tf32_kernel<<<grid, 256, 0, st>>>(src, n, hi, lo);
}

int tc_tile_m() { return TC_M; }
int tc_tile_n() { return TC_N; }

void launch_gemm_tf32x3(const GemmOut* outs, const TcSeg* segs, const int3* tiles, int ntiles, TcBases b,
                        int* err, cudaStream_t st) {
  if (ntiles <= 0) return;
  static int nsm = 0;
  if (!nsm) {
    cudaFuncSetAttribute(gemm_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  const int grid = std::min(ntiles, nsm);
  gemm_tf32x3_kernel<<<grid, TC_THREADS, SMEM_BYTES, st>>>(outs, segs, tiles, ntiles, b, err);
}

}  // namespace lrt
