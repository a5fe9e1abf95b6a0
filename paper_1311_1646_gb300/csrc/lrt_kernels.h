// Device work descriptors and kernel launchers of the DMRG sigma / renormalization path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lrt {

// dst (rows x cols, leading dimension ld_dst) += sum_s scale_s * op(src_s), op = transpose or not.
// A launch given base pointers reads dst as dbase + dst_off and a source with rel = 1 or 2
// as sbase1 / sbase2 + src_off (a template replayed for new data of the same layout).
struct GatherTask {
  double* dst;
  int ld_dst;
  int rows, cols;
  int src_begin, src_count;
  int64_t dst_off;
};
struct GatherSrc {
  const double* src;
  int ld;
  int trans;
  double scale;
  int64_t src_off;
  int rel;
};

// C (m x n, ldc) = [C +] sum_s scale_s * op(A_s) (m x k_s) * op(B_s) (k_s x n).
// Pointers flagged *_rel are offsets (in doubles) from a base pointer passed at
// launch: 1 = the caller's x (A, B) or y (C) buffer, 2 = the workspace of
// intermediates, 3.. = extra base rel - 3 (GemmExtra).  A plan therefore serves any
// caller buffers and workspace, and a plan kept as a template serves new operator data
// of the same layout.
// Vector blocking (several trial vectors in one output): with c_vr > 0 the output's rows
// come in blocks of c_vr, block v at C + v * c_vs; with c_vc > 0 its columns come in blocks
// of c_vc, block v at C + v * c_vs.  A segment's A rows (a_vr, a_vs) and B columns (b_vc,
// b_vs) are blocked the same way.  Zero: an ordinary dense operand.
struct GemmOut {
  double* C;
  int64_t c_off;
  int ldc;
  int m, n;
  int seg_begin, seg_count;
  int accumulate;
  int c_rel;
  int inst;      // batched launches: index of the instance whose bases the rel pointers use
  int c_vr, c_vc;
  int64_t c_vs;
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
  int a_vr, b_vc;
  int64_t a_vs, b_vs;
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

// gather work items: (task index, chunk of GATHER_CHUNK destination elements, 0) packed as int3
void launch_gather(const GatherTask* tasks, const GatherSrc* srcs, const int3* tiles, int ntiles,
                   cudaStream_t st, double* dbase = nullptr, const double* sbase1 = nullptr,
                   const double* sbase2 = nullptr);
// one gather plan over up to GEMM_MAX_INST instances: CTA b runs work item b / ninst with
// the bases of instance b % ninst (in the launch's parameter block)
struct GatherBases {
  double* d;
  const double* s1;
  const double* s2;
};
struct GatherInstSet {
  GatherBases b[64];
};
void launch_gather_inst(const GatherTask* tasks, const GatherSrc* srcs, const int3* tiles, int ntiles,
                        const GatherInstSet& bases, int ninst, cudaStream_t st);
// FP64 GEMM work items: output o, rows [m0, m0 + mt) and columns [n0, n0 + nt) of it,
// mt <= GEMM_TM, nt <= GEMM_TN, packed as (o, (m0 << 8) | mt, (n0 << 8) | nt)
inline int3 gemm_tile(int o, int m0, int mt, int n0, int nt) { return make_int3(o, (m0 << 8) | mt, (n0 << 8) | nt); }
// CTAs of the FP64 GEMM resident on the GPU at once (SMs x CTAs per SM)
int gemm_fp64_slots();
constexpr int GEMM_NEXTRA = 8;
struct GemmExtra {
  double* p[GEMM_NEXTRA];
};
void launch_gemm_fp64(const GemmOut* outs, const GemmSeg* segs, const int3* tiles, int ntiles,
                      const double* xbase, double* ybase, double* tbase, cudaStream_t st,
                      const GemmExtra* extra = nullptr, double* wbase = nullptr);
// Split K: an output tile whose segment list is long is cut into parts, each a contiguous
// run of its segments written as a partial tile (c_rel GEMM_C_SPLIT: wbase + c_off, row
// stride nt) into the plan's workspace; split_reduce then adds the parts in order and
// stores the sum where the output's own addressing puts it (c_rel 0, 1 or 2).
constexpr int GEMM_C_SPLIT = 15;
constexpr int GEMM_SPLIT_K = 512;   // K per part of a split tile
struct SplitTile {
  int64_t ws_off;     // part p of the tile at ws_off + p * mt * nt
  int o;              // the output the tile belongs to
  int nparts;
  int m0, mt, n0, nt;
};
void launch_split_reduce(const GemmOut* outs, const SplitTile* tiles, int ntiles, const double* wbase, double* ybase,
                         double* tbase, cudaStream_t st);
// batched form: the bases of output o are bases[o.inst] (device array)
struct GemmBases {
  const double* x;
  double* y;
  double* t;
};
void launch_gemm_fp64_multi(const GemmOut* outs, const GemmSeg* segs, const int3* tiles, int ntiles,
                            const GemmBases* bases, cudaStream_t st);
// One plan replayed over up to GEMM_MAX_INST instances in one launch: CTA b runs tile
// b / ninst of instance b % ninst, every base (x, y, t and the extra bases) taken from
// that instance's entry.  The entries travel in the launch's parameter block (no upload,
// no host synchronization); the instances' tiles interleave, so the plan's longest-first
// order holds across them.
constexpr int GEMM_MAX_INST = 64;
struct GemmInst {
  const double* x;
  double* y;
  double* t;
  double* e[GEMM_NEXTRA];
};
struct GemmInstSet {
  GemmInst b[GEMM_MAX_INST];
};
void launch_gemm_fp64_inst(const GemmOut* outs, const GemmSeg* segs, const int3* tiles, int ntiles,
                           const GemmInstSet& bases, int ninst, cudaStream_t st);
void launch_diag(const DiagOut* outs, const DiagTerm* terms, int nouts, double* dbase, cudaStream_t st);

// Split-TF32 tensor-core variant of the grouped GEMM.
//
// Operands live in "TC matrices": an R x K matrix (R = output rows or columns of
// the product, K = the contracted index) stored as TF32 pairs in two planes (hi, lo),
// each plane ceil(K / 32) chunks of Rp = roundup(R, 8) rows of 32 values, 128 bytes
// a row, the 16-byte groups of row r permuted by XOR (r mod 8): the image tcgen05
// reads with a 128-byte-swizzled K-major descriptor, so one bulk copy moves rows
// [r0, r0 + n) of a chunk.  Padding (K beyond the matrix, rows R..Rp) is zero.
//
// The host lays out, for every CTA of the persistent launch, the work it will do as
// one linear stream of items: a tile header, then the tile's block products.
struct TcTileHdr {
  double* C;          // FP64 output (c_rel 0); y + c_off when c_rel == 1
  float* t_hi;        // TC-matrix output (c_rel 2): planes of the intermediate
  float* t_lo;
  int64_t c_off;
  int ldc;
  int m0, n0, mt, nt; // tile origin and extent inside the output
  int c_rel;
  int accumulate;
  int t_rp, t_k;      // TC-matrix output: padded rows, valid K (= output columns)
  int inst;           // batched launches: instance whose y receives a c_rel == 1 output
  int vslots, vrows, vvalid, vstride;   // row slots (c_rel == 5)
};
struct TcSegRec {
  const float* a_hi;  // TC matrix A (rows = output rows) and B (rows = output columns)
  const float* a_lo;
  const float* b_hi;
  const float* b_lo;
  int a_rp, b_rp;     // padded rows of the two matrices
  int k;              // valid K
  float scale;
  int64_t b_vstride;  // c_rel 4: floats between the B matrices of consecutive vectors
  int64_t a_vstride;  // c_rel 5: floats between the A matrices of consecutive vectors
};
// Stacked tiles (c_rel == 3): the tile's 128 rows hold several short products that share
// their B operand and K; header.C points at the tile's piece items, header.inst counts
// them, and every piece names the rows of its A matrix, where they go in the tile (a
// multiple of 8, so the swizzle phase of the packed rows is kept) and the intermediate
// they produce.  The pieces are followed by one segment item (B, k, scale).
struct TcPieceRec {
  const float* a_hi;
  const float* a_lo;
  float* t_hi;
  float* t_lo;
  int a_rp, a_row0;   // A matrix: padded rows, first row of the piece
  int nrows;          // rows of the piece (multiple of 8)
  int smem_row;       // first row of the piece in the tile (multiple of 8)
  int t_rp, t_row0;   // intermediate: padded rows, first row written
};
// Vector-slot tiles (c_rel == 4): stacked pieces as for c_rel 3, and the tile's columns
// split into header.accumulate slots of header.ldc columns (a multiple of 8), slot j
// holding the product for vector v0 + j.  The producer copies slot j's B rows from
// b + j * b_vstride; the epilogue writes slot j into the piece's intermediate plus
// j * header.c_off floats.  Narrow products (a few columns per vector) thereby fill
// the tile's columns with the vectors of a block-Davidson step.
// Row-slot tiles (c_rel == 5): an FP64 output of few rows (phase 2 of sigma, y = sum
// T Y^T) takes header.vslots vectors in the tile's rows, slot j = rows [j vrows, (j + 1)
// vrows) holding vector v0 + j.  The producer copies slot j's A rows from a + j *
// a_vstride; the epilogue writes the slot's first vvalid rows to y + c_off + j * vstride.
// Every segment's A matrix has vrows padded rows and lies in a per-vector pool; B (an
// operator block) is shared by the vectors.
constexpr int TC_ITEM_TILE = 1, TC_ITEM_SEG = 2, TC_ITEM_PIECE = 3;
constexpr int TC_MAX_PIECES = 16;
struct TcItem {
  int type;
  int pad;
  union {
    TcTileHdr t;
    TcSegRec s;
    TcPieceRec p;
  };
};
struct TcOut {
  double* y;                // y of a single-instance launch
  double* const* ys;        // batched launches: y of instance i is ys[i] (device array), else NULL
  unsigned long long wait_ns;   // limit of every pipeline wait (0: TC_WAIT_NS)
  int stall;                // test hook: CTA 0's MMA thread first waits on a barrier nothing
                            // arrives at, so the launch ends through the expired-wait path
};
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;   // 2 s per pipeline wait
// number of CTAs (one per SM) the tensor-core launch uses for ntiles tiles; CTA b
// takes tiles b, b + n, b + 2n, ... of the host's order
int tc_num_ctas(int ntiles);
// items[cta_begin[b] .. cta_begin[b + 1]) is the stream of CTA b, b < nctas; tiles are
// 128 x tile_n (tile_n = 32 or 64, the value the stream was built for)
void launch_gemm_tf32x3(const TcItem* items, const int* cta_begin, int nctas, int tile_n, TcOut out, int* err,
                        cudaStream_t st);

// Packing into TC matrices: element (r, k) of the source is src[r * ld + k], or
// src[k * ld + r] when trans; source = base + src_off when base is given at launch.
struct TcPack {
  const double* src;
  int64_t src_off;
  int64_t ld;
  int64_t dst_off;    // float offset of the matrix in the destination planes
  int R, K, Rp, trans;
};
// packs descriptors [0, n) for each of nvec vectors: vector v reads base + v * src_stride
// (or src when base is null) and writes at dst + v * dst_stride
void launch_tc_pack(const TcPack* d, int n, const double* base, int64_t src_stride, float* dst_hi, float* dst_lo,
                    int64_t dst_stride, int nvec, cudaStream_t st);
int tc_tile_m();

constexpr int GATHER_CHUNK = 1024;   // destination elements per gather work item
constexpr int GEMM_TM = 64;   // output tile rows
constexpr int GEMM_TN = 32;   // output tile columns

}  // namespace lrt

namespace lrt {
// Davidson vector operations (FP64): V holds m vectors of length n with stride ld.
void launch_dots(const double* V, int64_t ld, int m, const double* w, int64_t n, double* out, cudaStream_t st);
// out[a * nb + b] = A[a] . B[b], a < na, b < nb (device arrays of device pointers, length n each)
void launch_pair_dots(const double* const* A, const double* const* B, int na, int nb, int64_t n, double* out,
                      cudaStream_t st);
void launch_lincomb(const double* V, int64_t ld, int m, const double* coef, int64_t n, double* out, double beta,
                    cudaStream_t st);
void launch_precond(const double* r, const double* d, double theta, int64_t n, double* t, cudaStream_t st);
// Eigen-decomposition of a small symmetric n x n matrix (n <= JACOBI_MAXN) by cyclic Jacobi
// rotations in one CTA: A (row-major, overwritten) -> eigenvalues w (ascending) and
// eigenvectors as the columns of Z (row-major n x n).
void launch_jacobi_eigh(double* A, int n, double* w, double* Z, cudaStream_t st);
constexpr int JACOBI_MAXN = 48;

// Batched forms for the sweeps of several trial vectors at once.  A batch holds nv
// vectors of length n with stride ld (doubles).
// V_v += alpha * coef[v] * W_v, W_v = w + v * ldw (ldw = 0: one w for all v); coef: device
// array of nv values, or NULL for 1
void launch_rank1_batch(const double* w, int64_t ldw, const double* coef, double alpha, int nv, double* V,
                        int64_t ld, int64_t n, cudaStream_t st);
// Vnew_mu = sum_j a[j * m + mu] Vold_j, mu < m, j < lold  (a: device, row-major lold x m)
void launch_rotate(const double* Vold, int64_t ld_old, int lold, const double* a, int m, double* Vnew,
                   int64_t ld_new, int64_t n, cudaStream_t st);
// Z_v = sign * (-R_v / (d - theta[v])), |d - theta| clamped to >= 1e-4 (Eq. error)
void launch_precond_batch(const double* R, int64_t ldr, const double* d, const double* theta, int nv, int64_t n,
                          double* Z, int64_t ldz, double sign, cudaStream_t st);
// Z = R / max(|d - shift|, 1e-4): a positive diagonal preconditioner (for MINRES on the
// indefinite shifted site equations)
void launch_precond_abs(const double* R, const double* d, double shift, int64_t n, double* Z, cudaStream_t st);
// Deterministic dot products in two passes (per-CTA partial sums in `work`, then a fixed-order
// sum), `work` holding at least DOT_WORK(npairs) doubles:
//   vdots: out[v] (+)= A_v . B_v  (ldb = 0: one B for all v)
//   pair_dots_strided: out[a * nb + b] = A_a . B_b
constexpr int DOT_CHUNKS = 64;
inline int64_t dot_work(int64_t npairs) { return npairs * DOT_CHUNKS; }
void launch_vdots(const double* A, int64_t lda, const double* B, int64_t ldb, int nv, int64_t n, double* out,
                  bool accumulate, double* work, cudaStream_t st);
void launch_pair_dots_strided(const double* A, int64_t lda, int na, const double* B, int64_t ldb, int nb, int64_t n,
                              double* out, double* work, cudaStream_t st);
// out[d] += sum_{j in [beg[d], beg[d + 1])} coef[j] * src[idx[j]], d < nout (one thread per
// output, terms in list order: deterministic)
void launch_gather_sum(const double* src, const int* beg, const int* idx, const double* coef, int nout, double* out,
                       cudaStream_t st);
// Hr[a * l + b] += D1[a * l + b] + D2[a * l + b] + D2[b * l + a];  Sr += D3  (Eqs. hleft2, sleft2)
void launch_reduced_acc(const double* D1, const double* D2, const double* D3, int l, double* Hr, double* Sr,
                        cudaStream_t st);
}  // namespace lrt
