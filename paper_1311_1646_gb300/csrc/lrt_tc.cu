// Split-TF32 tensor-core GEMM (tcgen05, sm_103a) for the mixed-precision path.
//
// Same task structure as gemm_fp64_kernel: every output tile (128 rows x 64
// columns) sums K-concatenated products scale_s * op(A_s) op(B_s).  Operands are
// held as TF32 pairs x = hi + lo (hi = rna(x), lo = rna(x - hi) of the FP32-rounded
// value), split once per operator set and once per input vector, and the product is
// accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi (lo*lo is below FP32 resolution).
// Each product (segment) accumulates in FP32 in tensor memory; the running sum over
// the segments of a tile is a compensated (two-sum) FP32 pair in registers, read
// back once per finished segment, so plain FP32 accumulation spans only the K of one
// block product.  No FP64 arithmetic runs in the loop: on this GPU the FP64 pipe is
// the scarcest resource.
//
// Per K chunk of 32: all 128 threads convert and store the four operand tiles in
// shared memory in the canonical no-swizzle K-major layout (8-row x 16-byte core
// matrices), one thread issues 3 x 4 tcgen05.mma (K = 8 each) and commits them to
// an mbarrier, and every thread waits on that barrier before the tiles are
// rewritten.  Every wait is bounded: on expiry the kernel records an error code,
// stops issuing work, releases its tensor memory and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lrt_kernels.h"

namespace lrt {

namespace {

constexpr int TC_M = 128;               // rows of an output tile (one TMEM lane per row)
constexpr int TC_N = 64;                // columns of an output tile (TMEM columns)
constexpr int TC_K = 32;                // K elements staged per chunk
constexpr int TC_THREADS = 128;
constexpr int A_BYTES = TC_M * TC_K * 4;    // one TF32 operand tile of A
constexpr int B_BYTES = TC_N * TC_K * 4;
constexpr int SMEM_BYTES = 2 * A_BYTES + 2 * B_BYTES + 1024;
constexpr uint32_t WAIT_LIMIT = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) of a K-major tile with TC_K columns:
// core matrix (row / 8, k / 4) at ((row / 8) * (TC_K / 4) + k / 4) * 128, inside it
// row (row % 8) at 16 bytes and element (k % 4) at 4 bytes.
__device__ __forceinline__ uint32_t kmajor_offset(int row, int k) {
  return (uint32_t)((((row >> 3) * (TC_K / 4) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}

// shared-memory matrix descriptor, no swizzle, K-major:
// LBO = 128 B (next core matrix along K), SBO = (TC_K / 4) * 128 B (next 8 rows)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((((TC_K / 4) * 128u) >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;                 // descriptor version for this architecture
  return d;                               // base offset 0, LBO mode 0, swizzle none (0)
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

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// bounded wait for the phase with the given parity; returns false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
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

}  // namespace

__global__ void __launch_bounds__(TC_THREADS, 1) gemm_tf32x3_kernel(const GemmOut* __restrict__ outs,
                                                                     const TcSeg* __restrict__ segs,
                                                                     const int3* __restrict__ tiles, int ntiles,
                                                                     TcBases bases, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int w = blockIdx.x;
  if (w >= ntiles) return;
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sAh = sm;
  uint8_t* sAl = sm + A_BYTES;
  uint8_t* sBh = sm + 2 * A_BYTES;
  uint8_t* sBl = sm + 2 * A_BYTES + B_BYTES;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TC_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  const int3 wi = tiles[w];
  const GemmOut o = outs[wi.x];
  const int m0 = wi.y * TC_M, n0 = wi.z * TC_N;
  const int mt = min(TC_M, o.m - m0), nt = min(TC_N, o.n - n0);
  constexpr uint32_t idesc = make_idesc();
  uint32_t phase = 0;
  const int row = warp * 32 + (tid & 31);
  float sum[TC_N], cmp[TC_N];     // compensated running sum of the tile row
#pragma unroll
  for (int c = 0; c < TC_N; ++c) sum[c] = cmp[c] = 0.0f;

  for (int s = 0; s < o.seg_count && !failed; ++s) {
    const TcSeg g = segs[o.seg_begin + s];
    const float* Ah = g.a_rel ? (g.a_rel == 1 ? bases.xhi : bases.thi) + g.a_off : g.Ahi;
    const float* Al = g.a_rel ? (g.a_rel == 1 ? bases.xlo : bases.tlo) + g.a_off : g.Alo;
    const float* Bh = g.b_rel ? (g.b_rel == 1 ? bases.xhi : bases.thi) + g.b_off : g.Bhi;
    const float* Bl = g.b_rel ? (g.b_rel == 1 ? bases.xlo : bases.tlo) + g.b_off : g.Blo;
    bool issued = false;
    for (int k0 = 0; k0 < g.k && !failed; k0 += TC_K) {
      const int kc = min(TC_K, g.k - k0);
      // A tile: op(A)(m0 + i, k0 + kk), zero outside
      for (int e = tid; e < TC_M * TC_K; e += TC_THREADS) {
        int i, kk;
        if (!g.transA) { i = e / TC_K; kk = e % TC_K; } else { kk = e / TC_M; i = e % TC_M; }
        uint32_t hi = 0u, lo = 0u;
        if (i < mt && kk < kc) {
          const int64_t idx = g.transA ? (int64_t)(k0 + kk) * g.lda + (m0 + i) : (int64_t)(m0 + i) * g.lda + (k0 + kk);
          hi = __float_as_uint(Ah[idx]);
          lo = __float_as_uint(Al[idx]);
        }
        const uint32_t off = kmajor_offset(i, kk);
        *(uint32_t*)(sAh + off) = hi;
        *(uint32_t*)(sAl + off) = lo;
      }
      // B tile stored N x K (K-major): element (j, kk) = op(B)(k0 + kk, n0 + j)
      for (int e = tid; e < TC_N * TC_K; e += TC_THREADS) {
        int j, kk;
        if (!g.transB) { kk = e / TC_N; j = e % TC_N; } else { j = e / TC_K; kk = e % TC_K; }
        uint32_t hi = 0u, lo = 0u;
        if (j < nt && kk < kc) {
          const int64_t idx = g.transB ? (int64_t)(n0 + j) * g.ldb + (k0 + kk) : (int64_t)(k0 + kk) * g.ldb + (n0 + j);
          hi = __float_as_uint(Bh[idx]);
          lo = __float_as_uint(Bl[idx]);
        }
        const uint32_t off = kmajor_offset(j, kk);
        *(uint32_t*)(sBh + off) = hi;
        *(uint32_t*)(sBl + off) = lo;
      }
      // make the generic-proxy stores visible to the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl), bh = smem_u32(sBh), bl = smem_u32(sBl);
#pragma unroll
        for (int ks = 0; ks < TC_K / 8; ++ks) {
          const uint32_t step = (uint32_t)ks * 256u;   // two 16-byte core-matrix columns
          const uint32_t acc0 = (issued || ks > 0) ? 1u : 0u;
          mma_tf32(tmem, make_desc(ah + step), make_desc(bh + step), idesc, acc0);
          mma_tf32(tmem, make_desc(ah + step), make_desc(bl + step), idesc, 1u);
          mma_tf32(tmem, make_desc(al + step), make_desc(bh + step), idesc, 1u);
        }
        mma_commit(&bar);
      }
      issued = true;
      if (!mbar_wait(&bar, phase)) {
        failed = 1;
        if (err) atomicExch(err, 1);
      }
      phase ^= 1u;
      __syncthreads();
    }
    if (issued && !failed) {
      // fold this product into the compensated running sum (two-sum in FP32)
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c0 = 0; c0 < TC_N; c0 += 16) {
        float v[16];
        ld_16cols(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float y = g.scale * v[i] - cmp[c0 + i];
          const float t = sum[c0 + i] + y;
          cmp[c0 + i] = (t - sum[c0 + i]) - y;
          sum[c0 + i] = t;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }

  if (!failed && row < mt) {
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
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N));
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
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(gemm_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr = true;
  }
  gemm_tf32x3_kernel<<<ntiles, TC_THREADS, SMEM_BYTES, st>>>(outs, segs, tiles, ntiles, b, err);
}

}  // namespace lrt
