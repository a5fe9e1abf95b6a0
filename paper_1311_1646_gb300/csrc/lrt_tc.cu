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
// Persistent, warp-specialised kernel (one CTA per SM, 6 warps).  The host hands
// every CTA a linear stream of items (tile header, then the tile's block products),
// so only the producer touches global metadata, a few items ahead; the other roles
// get theirs through shared memory:
//   warp 4     producer (one thread): per K chunk of 32, four bulk copies
//              (cp.async.bulk, completion counted in bytes on the stage's mbarrier)
//              of the A and B TC-matrix rows of the tile, hi and lo planes, into a
//              3-stage ring; the packed layout already is the 128-byte-swizzled
//              K-major image with zero K padding.  Each chunk carries a record (K
//              steps, first/last of its product); each product and each tile end a
//              record for the epilogue in a ring.
//   warp 5     one thread issues 3 x (K / 8) tcgen05.mma per chunk into one of four
//              TMEM accumulators (64 columns each), commits the stage back to the
//              producer and, after the last chunk of a product, commits the
//              accumulator to the epilogue.
//   warps 0-3  epilogue: thread = tile row = TMEM lane; folds each finished product
//              into the compensated sum, releases the accumulator, and at a tile end
//              stages the tile in shared memory so that a warp stores whole rows:
//              FP64 into y, or TF32 pairs into the TC matrix of an intermediate.
//
// Every wait is bounded by the global timer and also ends when another role has
// failed: on expiry the kernel records an error code, stops issuing work, waits (with
// a bound) for its own MMAs and copies in flight, releases its tensor memory and
// returns.
#include <cuda_runtime.h>

#include <atomic>
#include <stdint.h>

#include <algorithm>

#include "lrt_kernels.h"

namespace lrt {

namespace {

constexpr int TC_M = 128;               // rows of an output tile (one TMEM lane per row)
constexpr int TC_K = 32;                // K elements per stage (one 128-byte swizzle row)
constexpr int STAGES = 3;
constexpr int NINFO = 16;               // epilogue record ring
constexpr int EPI_WARPS = 4, PROD_WARPS = 1;
constexpr int TC_THREADS = 32 * (EPI_WARPS + PROD_WARPS + 1);
constexpr int A_BYTES = TC_M * TC_K * 4;    // one TF32 operand tile of A (16 KB)
constexpr int NACC = 4;                 // TMEM accumulators (product ring to the epilogue)
constexpr uint64_t WAIT_NS = TC_WAIT_NS;  // drains of copies and MMAs already issued

// Sizes that follow from the tile width TN (output columns = TMEM columns of one
// accumulator): 32 or 64, chosen per launch by the host's autotuner.
template <int TN>
struct Tile {
  static constexpr int B_BYTES = TN * TC_K * 4;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int STG_LD = TN + 1;                  // 8-byte words per staged output row (padded)
  static constexpr int STG_WARP_BYTES = 32 * STG_LD * 8;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + EPI_WARPS * STG_WARP_BYTES + 1024;
  static constexpr uint32_t TMEM_COLS = NACC * TN;
  static_assert(STAGE_BYTES % 1024 == 0 && A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0,
                "swizzle atoms must stay 1024-byte aligned");
  static_assert(2 * (TN / 32) * 32 * 128 <= STG_WARP_BYTES, "TC-matrix staging fits the warp's buffer");
  static_assert(TMEM_COLS >= 32 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "TMEM allocation: power of two >= 32");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
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

// instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = TN
template <int TN>
__host__ __device__ constexpr uint32_t make_idesc() {
  return (1u << 4)                        // D format F32
         | (2u << 7)                      // A format TF32
         | (2u << 10)                     // B format TF32
         | ((uint32_t)(TN >> 3) << 17)    // N / 8
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
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* failed, int* err,
                                          uint64_t lim) {
  const uint32_t a = smem_u32(bar);
  if (mbar_try(a, parity)) return true;
  const uint64_t t0 = now_ns();
  for (uint32_t n = 1;; ++n) {
    if (mbar_try(a, parity)) return true;
    if ((n & 255u) == 0u) {
      if (*failed) return false;
      if (now_ns() - t0 > lim) {
        *failed = 1;
        if (err) atomicExch(err, 1);
        return false;
      }
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

// 16 consecutive TMEM columns of this warp's 32 lanes; completes at tcgen05.wait::ld
__device__ __forceinline__ void ld_16cols_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// global -> shared bulk copy whose completion is counted (in bytes) on an mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// per-stage record from the producers to the MMA thread
constexpr int META_FIRST = 1, META_LAST = 2, META_END = 4;
struct StageMeta {
  int nks;     // K steps of 8
  int flags;
};
// ring record from the producers to the epilogue
constexpr int INFO_MMA = 1, INFO_TILE_END = 2, INFO_END = 4, INFO_FIRST = 8;
struct EpiInfo {
  int flags;
  float scale;
  TcTileHdr t;
};

__device__ __forceinline__ TcItem load_item(const TcItem* p) {
  TcItem r;
  const int4* q = reinterpret_cast<const int4*>(p);
  int4* d = reinterpret_cast<int4*>(&r);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(TcItem) / 16); ++i) d[i] = __ldg(q + i);
  return r;
}

}  // namespace

static_assert(sizeof(TcItem) % 16 == 0, "items are read as 16-byte vectors");

template <int TN>
__global__ void __launch_bounds__(TC_THREADS, 1) gemm_tf32x3_kernel(const TcItem* __restrict__ items,
                                                                     const int* __restrict__ cta_begin,
                                                                     TcOut out, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[NACC], tempty_bar[NACC], drain_bar;
  __shared__ uint64_t info_full[NINFO], info_empty[NINFO];
  __shared__ StageMeta meta[STAGES];
  __shared__ EpiInfo info[NINFO];
  __shared__ uint32_t tmem_base;
  __shared__ int failed_s;
  volatile int* failed = &failed_s;
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(Tile<TN>::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);   // the producer's arrive (with the expected bytes)
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(&tfull_bar[a], 1);
      mbar_init(&tempty_bar[a], 32 * EPI_WARPS);
    }
    for (int q = 0; q < NINFO; ++q) {
      mbar_init(&info_full[q], 1);
      mbar_init(&info_empty[q], 32 * EPI_WARPS);
    }
    mbar_init(&drain_bar, 1);
    failed_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint64_t lim = out.wait_ns ? out.wait_ns : WAIT_NS;   // every progress wait

  if (warp == EPI_WARPS) {
    // ---------------- producer (one thread)
    if (lane == 0) {
      const uint32_t sbase = smem_u32(sm);
      uint32_t it = 0, ei = 0;
      bool ok = true;
      // the epilogue record ring
      auto post = [&](const EpiInfo& rec) -> bool {
        const uint32_t slot = ei % NINFO, use = ei / NINFO;
        if (use > 0 && !mbar_wait(&info_empty[slot], (use - 1) & 1, failed, err, lim)) return false;
        info[slot] = rec;
        mbar_arrive(&info_full[slot]);
        ++ei;
        return true;
      };
      const int p0 = cta_begin[blockIdx.x], p1 = cta_begin[blockIdx.x + 1];
      bool have_tile = false, first_seg = true;
      TcTileHdr hdr{};
      TcPieceRec pieces[TC_MAX_PIECES];
      int npieces = 0;
      TcItem cur, nx1, nx2;
      if (p0 < p1) cur = load_item(items + p0);
      if (p0 + 1 < p1) nx1 = load_item(items + p0 + 1);
      for (int p = p0; p < p1 && ok && !*failed; ++p) {
        if (p + 2 < p1) nx2 = load_item(items + p + 2);
        if (cur.type == TC_ITEM_TILE) {
          if (have_tile) ok = post(EpiInfo{INFO_TILE_END, 0.0f, hdr});
          hdr = cur.t;
          have_tile = true;
          first_seg = true;
          npieces = 0;
        } else if (cur.type == TC_ITEM_PIECE) {
          if (npieces < TC_MAX_PIECES) pieces[npieces++] = cur.p;
        } else if (cur.s.k > 0) {
          const TcSegRec& g = cur.s;
          ok = post(EpiInfo{INFO_MMA | (first_seg ? INFO_FIRST : 0), g.scale, hdr});
          first_seg = false;
          // rows of the two matrices this tile reads (multiples of 8: whole swizzle atoms)
          uint32_t ra = (uint32_t)min(TC_M, g.a_rp - hdr.m0);
          if (hdr.c_rel == 3 || hdr.c_rel == 4) {
            ra = 0;
            for (int j = 0; j < npieces; ++j) ra += (uint32_t)pieces[j].nrows;
          } else if (hdr.c_rel == 5) {
            ra = (uint32_t)(hdr.vslots * g.a_rp);   // row slots: all rows of each vector's A
          }
          // vector slots: hdr.accumulate slots of hdr.ldc rows, each all of one vector's B
          const bool slots = hdr.c_rel == 4;
          const uint32_t rb = slots ? (uint32_t)(hdr.accumulate * hdr.ldc) : (uint32_t)min(TN, g.b_rp - hdr.n0);
          const uint32_t bytes = 2u * 128u * (ra + rb);
          for (int k0 = 0, q = 0; k0 < g.k && ok; k0 += TC_K, ++q, ++it) {
            const uint32_t stage = it % STAGES, round = it / STAGES;
            if (round > 0 && !mbar_wait(&empty_bar[stage], (round - 1) & 1, failed, err, lim)) {
              ok = false;
              break;
            }
            const int kc = min(TC_K, g.k - k0);
            meta[stage] = StageMeta{(kc + 7) >> 3, (k0 == 0 ? META_FIRST : 0) | (k0 + TC_K >= g.k ? META_LAST : 0)};
            const uint32_t st = sbase + stage * Tile<TN>::STAGE_BYTES;
            const int64_t ao = ((int64_t)q * g.a_rp + hdr.m0) * TC_K, bo = ((int64_t)q * g.b_rp + hdr.n0) * TC_K;
            mbar_arrive_tx(&full_bar[stage], bytes);
            if (hdr.c_rel == 5) {
              for (int j = 0; j < hdr.vslots; ++j) {
                const int64_t vo = (int64_t)j * g.a_vstride + (int64_t)q * g.a_rp * TC_K;
                const uint32_t so = (uint32_t)(j * g.a_rp) * 128u;
                bulk_g2s(st + so, g.a_hi + vo, 128u * (uint32_t)g.a_rp, &full_bar[stage]);
                bulk_g2s(st + A_BYTES + so, g.a_lo + vo, 128u * (uint32_t)g.a_rp, &full_bar[stage]);
              }
            } else if (hdr.c_rel >= 3) {
              for (int j = 0; j < npieces; ++j) {
                const TcPieceRec& pc = pieces[j];
                const int64_t po = ((int64_t)q * pc.a_rp + pc.a_row0) * TC_K;
                const uint32_t so = (uint32_t)pc.smem_row * 128u;
                bulk_g2s(st + so, pc.a_hi + po, 128u * (uint32_t)pc.nrows, &full_bar[stage]);
                bulk_g2s(st + A_BYTES + so, pc.a_lo + po, 128u * (uint32_t)pc.nrows, &full_bar[stage]);
              }
            } else {
              bulk_g2s(st, g.a_hi + ao, 128u * ra, &full_bar[stage]);
              bulk_g2s(st + A_BYTES, g.a_lo + ao, 128u * ra, &full_bar[stage]);
            }
            if (slots) {
              for (int j = 0; j < hdr.accumulate; ++j) {
                const int64_t vo = (int64_t)j * g.b_vstride + (int64_t)q * g.b_rp * TC_K;
                const uint32_t so = (uint32_t)(j * hdr.ldc) * 128u;
                bulk_g2s(st + 2 * A_BYTES + so, g.b_hi + vo, 128u * (uint32_t)hdr.ldc, &full_bar[stage]);
                bulk_g2s(st + 2 * A_BYTES + Tile<TN>::B_BYTES + so, g.b_lo + vo, 128u * (uint32_t)hdr.ldc,
                         &full_bar[stage]);
              }
            } else {
              bulk_g2s(st + 2 * A_BYTES, g.b_hi + bo, 128u * rb, &full_bar[stage]);
              bulk_g2s(st + 2 * A_BYTES + Tile<TN>::B_BYTES, g.b_lo + bo, 128u * rb, &full_bar[stage]);
            }
          }
        }
        cur = nx1;
        nx1 = nx2;
      }
      if (ok && !*failed) {
        if (have_tile) ok = post(EpiInfo{INFO_TILE_END, 0.0f, hdr});
        ok = ok && post(EpiInfo{INFO_END, 0.0f, hdr});
        // end-of-stream record for the MMA thread, in a stage of its own
        const uint32_t stage = it % STAGES, round = it / STAGES;
        if (ok && !(round > 0 && !mbar_wait(&empty_bar[stage], (round - 1) & 1, failed, err, lim))) {
          meta[stage] = StageMeta{0, META_END};
          mbar_arrive(&full_bar[stage]);
        }
      }
      if (*failed) {
        // copies already issued must land before the CTA's shared memory goes away:
        // wait (bounded) for every stage that was filled after its last release
        for (uint32_t j = (it > (uint32_t)STAGES ? it - STAGES : 0u); j < it; ++j) {
          const uint32_t fa = smem_u32(&full_bar[j % STAGES]);
          const uint64_t t0 = now_ns();
          while (!mbar_try(fa, (j / STAGES) & 1) && now_ns() - t0 < WAIT_NS) {
          }
        }
      }
    }
  } else if (warp == EPI_WARPS + PROD_WARPS) {
    // ---------------- MMA issuer (one thread)
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc<TN>();
      uint32_t sg = 0;
      bool any = false;
      // test hook: a wait on a barrier nothing arrives at (its phase never completes),
      // which ends the launch through the expired-wait path below
      if (out.stall && blockIdx.x == 0) mbar_wait(&drain_bar, 0, failed, err, lim);
      for (uint32_t it = 0; !*failed; ++it) {
        const uint32_t stage = it % STAGES, round = it / STAGES;
        if (!mbar_wait(&full_bar[stage], round & 1, failed, err, lim)) break;
        const StageMeta m = meta[stage];
        if (m.flags & META_END) break;
        const uint32_t a = sg % NACC;
        if (m.flags & META_FIRST) {
          const uint32_t u = sg / NACC;
          if (u > 0 && !mbar_wait(&tempty_bar[a], (u - 1) & 1, failed, err, lim)) break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dt = tmem + a * TN;
        const uint32_t base = smem_u32(sm + stage * Tile<TN>::STAGE_BYTES);
        const uint32_t ah = base, al = base + A_BYTES, bh = base + 2 * A_BYTES, bl = bh + Tile<TN>::B_BYTES;
        for (int ks = 0; ks < m.nks; ++ks) {
          const uint32_t step = (uint32_t)ks * 32u;     // 8 TF32 = 32 bytes along K
          const uint32_t acc = ((m.flags & META_FIRST) && ks == 0) ? 0u : 1u;
          mma_tf32(dt, make_desc(ah + step), make_desc(bh + step), idesc, acc);
          mma_tf32(dt, make_desc(ah + step), make_desc(bl + step), idesc, 1u);
          mma_tf32(dt, make_desc(al + step), make_desc(bh + step), idesc, 1u);
        }
        mma_commit(&empty_bar[stage]);
        any = true;
        if (m.flags & META_LAST) {
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
    uint8_t* stg = sm + STAGES * Tile<TN>::STAGE_BYTES + warp * Tile<TN>::STG_WARP_BYTES;   // this warp's 32 rows
    uint32_t sg = 0;
    bool tile_has_mma = false;
    float sum[TN], cmp[TN];
#pragma unroll
    for (int c = 0; c < TN; ++c) sum[c] = cmp[c] = 0.0f;
    for (uint32_t ei = 0;; ++ei) {
      const uint32_t slot = ei % NINFO;
      // the warp stays converged for the .sync.aligned tensor-memory loads
      const bool got = mbar_wait(&info_full[slot], (ei / NINFO) & 1, failed, err, lim);
      if (!__all_sync(0xffffffffu, got)) break;
      const EpiInfo rec = info[slot];
      mbar_arrive(&info_empty[slot]);
      if (rec.flags & INFO_END) break;
      if (rec.flags & INFO_MMA) {
        const uint32_t a = sg % NACC, u = sg / NACC;
        const bool ok = mbar_wait(&tfull_bar[a], u & 1, failed, err, lim);
        if (!__all_sync(0xffffffffu, ok)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + a * TN;
#pragma unroll
        for (int c0 = 0; c0 < TN; c0 += 32) {
          uint32_t v[32];
          ld_16cols_async(taddr + (uint32_t)c0, v);
          ld_16cols_async(taddr + (uint32_t)c0 + 16u, v + 16);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (rec.flags & INFO_FIRST) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              sum[c0 + i] = rec.scale * __uint_as_float(v[i]);
              cmp[c0 + i] = 0.0f;
            }
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const float y = rec.scale * __uint_as_float(v[i]) - cmp[c0 + i];
              const float t = sum[c0 + i] + y;
              cmp[c0 + i] = (t - sum[c0 + i]) - y;
              sum[c0 + i] = t;
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&tempty_bar[a]);
        ++sg;
        tile_has_mma = true;
      }
      if (rec.flags & INFO_TILE_END) {
        const TcTileHdr& t = rec.t;
        if (!tile_has_mma) {
#pragma unroll
          for (int c = 0; c < TN; ++c) sum[c] = cmp[c] = 0.0f;
        }
        tile_has_mma = false;
        const int rr = lane;
        const int rbase = warp * 32;
        const int nrows = min(32, t.mt - rbase);
        // the staging buffer may still be read by this warp's previous bulk stores
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncwarp();
        if (t.c_rel == 4) {
          // Vector slots: each thread writes its row of every slot straight into the
          // piece's intermediate of that vector (TC-matrix image, 16-byte groups permuted
          // by row mod 8).  A slot is at most one chunk wide; positions past it keep the
          // zeros the intermediate was cleared to.
          const int r = rbase + lane;
          if (r < t.mt) {
            const TcItem* pit = reinterpret_cast<const TcItem*>(t.C);
            for (int j = 0; j < t.inst; ++j) {
              const TcItem pe = load_item(pit + j);
              if (r < pe.p.smem_row || r >= pe.p.smem_row + pe.p.nrows) continue;
              const int64_t trow = pe.p.t_row0 + (r - pe.p.smem_row);
#pragma unroll
              for (int g = 0; g < TN / 4; ++g) {
                const int c = 4 * g;
                const int slot = c / t.ldc;
                if (slot < t.accumulate) {
                  const int pg = (c - slot * t.ldc) >> 2;
                  uint32_t h[4], l[4];
#pragma unroll
                  for (int e = 0; e < 4; ++e) split_tf32(sum[c + e] - cmp[c + e], h[e], l[e]);
                  const int64_t o = (int64_t)slot * t.c_off + trow * 32 + (((pg ^ (int)trow) & 7) << 2);
                  *(uint4*)(pe.p.t_hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
                  *(uint4*)(pe.p.t_lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
                }
              }
              break;
            }
          }
        } else if (t.c_rel == 2 || t.c_rel == 3) {
          // Intermediate: this warp's rows as a TC-matrix image (two chunks of 32
          // columns, hi and lo planes; row r's 16-byte groups permuted by r mod 8),
          // then one bulk store per chunk and plane: rows [m0 + 32 w, + nrows) of a
          // chunk are contiguous in the matrix.  Columns past the output are zeros.
#pragma unroll
          for (int q = 0; q < TN / 32; ++q)
#pragma unroll
            for (int g4 = 0; g4 < 8; ++g4) {
              uint32_t h[4], l[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int c = 32 * q + 4 * g4 + e;
                h[e] = l[e] = 0u;
                if (c < t.nt) split_tf32(sum[c] - cmp[c], h[e], l[e]);
              }
              const uint32_t o = (uint32_t)(((q * 32 + rr) << 7) + (((g4 ^ rr) & 7) << 4));
              *(uint4*)(stg + o) = make_uint4(h[0], h[1], h[2], h[3]);
              *(uint4*)(stg + (TN / 32) * 32 * 128 + o) = make_uint4(l[0], l[1], l[2], l[3]);
            }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          // one bulk store per chunk and plane of a run of rows that is contiguous both
          // here and in its intermediate
          auto store_rows = [&](float* th, float* tl, int trp, int64_t trow, int r0, int nr) {
            for (int q = 0; q < TN / 32; ++q) {
              const int cq = t.n0 + 32 * q;
              if (cq >= t.t_k) break;
              const int64_t go = ((int64_t)(cq >> 5) * trp + trow) * 32;
              const uint32_t so = smem_u32(stg) + (uint32_t)(q * 32 * 128) + (uint32_t)r0 * 128u;
              asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(th + go), "r"(so),
                           "r"((uint32_t)nr * 128u)
                           : "memory");
              asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(tl + go),
                           "r"(so + (uint32_t)(TN / 32) * 32u * 128u), "r"((uint32_t)nr * 128u)
                           : "memory");
            }
          };
          if (lane == 0) {
            if (t.c_rel == 2) {
              if (nrows > 0) store_rows(t.t_hi, t.t_lo, t.t_rp, t.m0 + rbase, 0, nrows);
            } else {
              // stacked tile: the pieces that overlap this warp's 32 rows
              const TcItem* pit = reinterpret_cast<const TcItem*>(t.C);
              for (int j = 0; j < t.inst; ++j) {
                const TcItem pe = load_item(pit + j);
                const int s0 = pe.p.smem_row, s1 = s0 + pe.p.nrows;
                const int lo = max(s0, rbase), hi = min(s1, rbase + 32);
                if (lo < hi) store_rows(pe.p.t_hi, pe.p.t_lo, pe.p.t_rp, pe.p.t_row0 + (lo - s0), lo - rbase, hi - lo);
              }
            }
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          }
        } else {
          // FP64 output: stage the rows, then the warp stores row by row (coalesced)
#pragma unroll
          for (int c = 0; c < TN; ++c)
            *(double*)(stg + (rr * Tile<TN>::STG_LD + c) * 8) = (double)sum[c] - (double)cmp[c];
          __syncwarp();
          double* C = (t.c_rel != 0 ? (out.ys ? out.ys[t.inst] : out.y) + t.c_off : t.C);
          for (int r = 0; r < nrows; ++r) {
            int R = t.m0 + rbase + r;
            double* dst = C;
            if (t.c_rel == 5) {
              // row slots: slot j is vector v0 + j, its padding rows are not written
              const int j = R / t.vrows;
              R -= j * t.vrows;
              if (j >= t.vslots || R >= t.vvalid) continue;
              dst += (int64_t)j * t.vstride;
            }
            dst += (int64_t)R * t.ldc + t.n0;
            for (int c = lane; c < t.nt; c += 32) {
              const double v = *(const double*)(stg + (r * Tile<TN>::STG_LD + c) * 8);
              dst[c] = t.accumulate ? dst[c] + v : v;
            }
          }
        }
        __syncwarp();
      }
    }
  }

  if (warp < EPI_WARPS && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Tile<TN>::TMEM_COLS));
  }
}

// Packing into TC matrices: block x = descriptor, block y = vector; a warp writes one
// 128-byte row of a chunk (lane = position in the chunk), rows and chunks strided
// over the block's warps.
__global__ void __launch_bounds__(256) tc_pack_kernel(const TcPack* __restrict__ d, const double* base,
                                                      int64_t src_stride, float* __restrict__ hi,
                                                      float* __restrict__ lo, int64_t dst_stride) {
  const TcPack p = d[blockIdx.x];
  const double* src = (base ? base + (int64_t)blockIdx.y * src_stride + p.src_off : p.src);
  const int64_t dst = p.dst_off + (int64_t)blockIdx.y * dst_stride;
  const int nch = (p.K + 31) >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int w = warp; w < nch * p.Rp; w += blockDim.x >> 5) {
    const int q = w / p.Rp, r = w - q * p.Rp;
    const int k = 32 * q + lane;
    float v = 0.0f;
    if (r < p.R && k < p.K) v = (float)(p.trans ? src[(int64_t)k * p.ld + r] : src[(int64_t)r * p.ld + k]);
    uint32_t h, l;
    split_tf32(v, h, l);
    const int64_t o = dst + ((int64_t)q * p.Rp + r) * 32 + ((((lane >> 2) ^ r) & 7) << 2) + (lane & 3);
    hi[o] = __uint_as_float(h);
    lo[o] = __uint_as_float(l);
  }
}

void launch_tc_pack(const TcPack* d, int n, const double* base, int64_t src_stride, float* dst_hi, float* dst_lo,
                    int64_t dst_stride, int nvec, cudaStream_t st) {
  if (n <= 0 || nvec <= 0) return;
  tc_pack_kernel<<<dim3((unsigned)n, (unsigned)nvec), 256, 0, st>>>(d, base, src_stride, dst_hi, dst_lo, dst_stride);
}

int tc_tile_m() { return TC_M; }

// Per-device state: a process may drive several GPUs (one context per device), and a
// function attribute set with cudaFuncSetAttribute applies to the current device only.
constexpr int TC_MAX_DEVICES = 64;

static int sm_count() {
  static std::atomic<int> count[TC_MAX_DEVICES];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TC_MAX_DEVICES) return 1;
  int nsm = count[dev].load(std::memory_order_acquire);
  if (!nsm) {
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
    count[dev].store(nsm, std::memory_order_release);
  }
  return nsm;
}

int tc_num_ctas(int ntiles) { return std::max(1, std::min(ntiles, sm_count())); }

template <int TN>
static void launch_tn(const TcItem* items, const int* cta_begin, int nctas, TcOut out, int* err, cudaStream_t st) {
  // opt into the dynamic shared memory once per device; on failure the error is the
  // runtime's last error and the caller's launch check reports it
  static std::atomic<int> attr[TC_MAX_DEVICES];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  if (dev < 0 || dev >= TC_MAX_DEVICES) return;
  if (!attr[dev].load(std::memory_order_acquire)) {
    if (cudaFuncSetAttribute(gemm_tf32x3_kernel<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Tile<TN>::SMEM_BYTES) != cudaSuccess)
      return;
    attr[dev].store(1, std::memory_order_release);
  }
  gemm_tf32x3_kernel<TN><<<nctas, TC_THREADS, Tile<TN>::SMEM_BYTES, st>>>(items, cta_begin, out, err);
}

void launch_gemm_tf32x3(const TcItem* items, const int* cta_begin, int nctas, int tile_n, TcOut out, int* err,
                        cudaStream_t st) {
  if (nctas <= 0) return;
  if (tile_n == 32)
    launch_tn<32>(items, cta_begin, nctas, out, err, st);
  else
    launch_tn<64>(items, cta_begin, nctas, out, err, st);
}

}  // namespace lrt
