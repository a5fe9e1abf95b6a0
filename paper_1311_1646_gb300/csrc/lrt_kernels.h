// Device work descriptors and kernel launchers of the DMRG sigma / renormalization path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lrt {

// dst (rows x cols, leading dimension ld_dst) = sum_s scale_s * op(src_s), op = transpose or not.
struct GatherTask {
  double* dst;
  int ld_dst;
  int rows, cols;
  int src_begin, src_count;
};
struct GatherSrc {
  const double* src;
  int ld;
  int trans;
  double scale;
};

// C (m x n, ldc) = [C +] sum_s scale_s * op(A_s) (m x k_s) * op(B_s) (k_s x n).
// Pointers flagged *_rel are offsets (in doubles) from a base pointer passed at
// launch: 1 = the caller's x (A, B) or y (C) buffer, 2 = the workspace of
// intermediates.  A plan therefore serves any caller buffers and workspace.
struct GemmOut {
  double* C;
  int64_t c_off;
  int ldc;
  int m, n;
  int seg_begin, seg_count;
  int accumulate;
  int c_rel;
};
struct GemmSeg {
  const double* A;
  const double* B;
  int64_t a_off, b_off;
  int lda, ldb;
  int k;
  int transA, transB;
  int a_rel, b_rel;
  double scale;
};

// diag (rows x cols block, row-major) += sum_t scale_t * x_t[i] * y_t[j]   (x_t, y_t strided diagonals)
struct DiagOut {
  int64_t d_off;     // offset of the output block from the base pointer passed at launch
  int rows, cols;
  int term_begin, term_count;
};
struct DiagTerm {
  const double* x;   // diagonal of the X block: x[i * xs], or NULL for the identity
  const double* y;   // diagonal of the Y block: y[j * ys], or NULL for the identity
  int xs, ys;
  double scale;
};

// work items: (task index, tile row, tile col) packed as int3
void launch_gather(const GatherTask* tasks, const GatherSrc* srcs, const int3* tiles, int ntiles,
                   cudaStream_t st);
void launch_gemm_fp64(const GemmOut* outs, const GemmSeg* segs, const int3* tiles, int ntiles,
                      const double* xbase, double* ybase, double* tbase, cudaStream_t st);
void launch_diag(const DiagOut* outs, const DiagTerm* terms, int nouts, double* dbase, cudaStream_t st);

// Split-TF32 tensor-core variant of the grouped GEMM.  Operands are pre-split TF32
// pairs (hi, lo) in FP32 storage.  The host lays out, for every CTA of the
// persistent launch, the work it will do as one linear stream of items: a tile
// header, then the tile's block products (segments) with operand pointers resolved.
// Outputs with c_rel == 2 are written as hi/lo pairs into the intermediates (thi,
// tlo at c_off), c_rel == 1 as FP64 into y at c_off, c_rel == 0 as FP64 into C.
struct TcTileHdr {
  double* C;
  int64_t c_off;
  int ldc, m0, n0, mt, nt, c_rel, accumulate, pad;
};
constexpr int TC_TRANS_A = 1;   // A element (i, k) at k * lda + i (else i * lda + k)
constexpr int TC_TRANS_B = 2;   // B element (k, j) at k * ldb + j (else j * ldb + k)
struct TcSegRec {
  const float* a_hi;
  const float* a_lo;
  const float* b_hi;
  const float* b_lo;
  int lda, ldb, k, trans;
  float scale;
  int pad;
};
constexpr int TC_ITEM_TILE = 1, TC_ITEM_SEG = 2;
struct TcItem {
  int type;
  int pad;
  union {
    TcTileHdr t;
    TcSegRec s;
  };
};
struct TcOut {
  float* thi;
  float* tlo;
  double* y;
};
// number of CTAs (one per SM) the tensor-core launch uses for ntiles tiles; CTA b
// takes tiles b, b + n, b + 2n, ... of the host's order
int tc_num_ctas(int ntiles);
// items[cta_begin[b] .. cta_begin[b + 1]) is the stream of CTA b, b < nctas
void launch_gemm_tf32x3(const TcItem* items, const int* cta_begin, int nctas, TcOut out, int* err,
                        cudaStream_t st);
// hi = rna_tf32((float)x), lo = rna_tf32((float)x - hi) elementwise
void launch_split_tf32(const double* src, int64_t n, float* hi, float* lo, cudaStream_t st);
int tc_tile_m();
int tc_tile_n();

constexpr int GATHER_TILE = 32;
constexpr int GEMM_TM = 64;   // output tile rows
constexpr int GEMM_TN = 32;   // output tile columns

}  // namespace lrt

namespace lrt {
// Davidson vector operations (FP64): V holds m vectors of length n with stride ld.
void launch_dots(const double* V, int64_t ld, int m, const double* w, int64_t n, double* out, cudaStream_t st);
void launch_lincomb(const double* V, int64_t ld, int m, const double* coef, int64_t n, double* out, double beta,
                    cudaStream_t st);
void launch_precond(const double* r, const double* d, double theta, int64_t n, double* t, cudaStream_t st);
// Eigen-decomposition of a small symmetric n x n matrix (n <= JACOBI_MAXN) by cyclic Jacobi
// rotations in one CTA: A (row-major, overwritten) -> eigenvalues w (ascending) and
// eigenvectors as the columns of Z (row-major n x n).
void launch_jacobi_eigh(double* A, int n, double* w, double* Z, cudaStream_t st);
constexpr int JACOBI_MAXN = 48;
}  // namespace lrt
