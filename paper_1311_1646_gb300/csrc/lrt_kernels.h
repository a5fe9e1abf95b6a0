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
// pairs (hi, lo) in FP32 storage: absolute pointers for operator data, or offsets from
// the hi/lo copies of x (rel 1) or of the intermediates (rel 2).  Outputs with
// c_rel == 2 are written as hi/lo pairs into the intermediates, others as FP64.
struct TcSeg {
  const float* Ahi;
  const float* Alo;
  const float* Bhi;
  const float* Blo;
  int64_t a_off, b_off;
  int lda, ldb;
  int k;
  int transA, transB;
  int a_rel, b_rel;
  float scale;
};
struct TcBases {
  const float* xhi;
  const float* xlo;
  float* thi;
  float* tlo;
  double* y;
};
void launch_gemm_tf32x3(const GemmOut* outs, const TcSeg* segs, const int3* tiles, int ntiles, TcBases b,
                        int* err, cudaStream_t st);
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
