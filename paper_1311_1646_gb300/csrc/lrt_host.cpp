// Host side of the DMRG sigma / renormalization library: context, operator-set
// planning and the C ABI declared in include/lrt.h.
//
// The Hamiltonian is split across every cut X | Y of the chain into renormalized
// normal and complementary operators (the "x" of Eqs. hzero_sb and lopr1st):
//
//   H = H^X + H^Y + sum_{x in X} (C_x S^Y_x - c_x S^Y_x^T) + sum_{y in Y} (S^X_y^T c_y - S^X_y C_y)
//     + [X normal] sum_{p<q in X} (A_pq P^Y_pq + A_pq^T P^Y_pq^T) + sum_{p,q in X} B_pq Q^Y_pq
//     | [Y normal] sum_{r<s in Y} (P^X_rs^T A_rs^T + P^X_rs A_rs) + sum_{u,w in Y} Q^X_uw B_uw
//
// with C_p = a+_p, c_p = a_p, A_pq = C_p C_q, B_pq = C_p c_q and, for a block Z,
//   S^Z_x = 1/2 sum_{q in Z} t_xq c_q + sum_{q,r,s in Z} v_xqrs C_q c_s c_r,
//   P^Z_pq = sum_{r,s in Z} v_pqrs c_s c_r,  Q^Z_pq = sum_{r,s in Z} (v_prqs - v_prsq) C_r c_s,
// v_pqrs = <pq|rs>.  A product X_op Y_op acts on |x>|y> with the sign
// (-1)^{parity(Y_op) N(x)}.  The normal side of cut b is the left one when 2b <= k.
//
// Blocks are enlarged by one site ("blocking") with formulas that express every
// operator of X (+) Y through operators of X and Y; a site is a 4-state space whose
// operators are built directly.  Enlarged operators live in a fused basis: the
// states of label Q are the sub-blocks n = 0..3 in order, each the states of the
// neighbouring bond sector Q -/+ n.
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/lrt.h"
#include "lrt_kernels.h"
#include "lrt_fp64_tile.h"

namespace lrt {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// Caching device allocator of a context: freed blocks are kept for reuse by the context
// that freed them, so the sweeps' thousands of temporaries cost neither a cudaMalloc nor
// the device synchronization of a cudaFree (size classes below).  Every ABI call makes
// its context's pool current for the calling thread; a context launches on one stream,
// so a reused block is ordered after the work that last used it.
struct DevPool {
  std::unordered_map<void*, size_t> live;      // pointer -> size class
  std::map<size_t, std::vector<void*>> cached; // size class -> free blocks
  size_t large_cached = 0;                     // bytes of cached blocks above POOL_MAX_BYTES
  void release() {
    for (auto& kv : cached)
      for (void* p : kv.second) cudaFree(p);
    cached.clear();
    large_cached = 0;
  }
  ~DevPool() { release(); }
};
static thread_local DevPool* t_pool = nullptr;
// Blocks up to POOL_MAX_BYTES are cached in power-of-two classes.  Larger blocks (operator
// sets, workspaces) are cached by size rounded up to POOL_LARGE_GRAIN: the sweeps free and
// allocate the same layouts over and over, and a cudaFree would synchronize the device.
// At most POOL_LARGE_CACHE bytes of them are kept; a failed allocation releases the cache.
constexpr size_t POOL_MAX_BYTES = (size_t)8 << 20;
constexpr size_t POOL_LARGE_GRAIN = (size_t)2 << 20;
constexpr size_t POOL_LARGE_CACHE = (size_t)32 << 30;

struct PoolScope {
  DevPool* prev;
  explicit PoolScope(DevPool* p) : prev(t_pool) { t_pool = p; }
  ~PoolScope() { t_pool = prev; }
};

static cudaError_t dev_alloc(void** p, size_t bytes) {
  DevPool* pool = t_pool;
  if (!pool) return cudaMalloc(p, bytes);
  size_t c;
  if (bytes <= POOL_MAX_BYTES) {
    c = 256;
    while (c < bytes) c <<= 1;
  } else {
    c = (bytes + POOL_LARGE_GRAIN - 1) / POOL_LARGE_GRAIN * POOL_LARGE_GRAIN;
  }
  auto it = pool->cached.find(c);
  if (it != pool->cached.end() && !it->second.empty()) {
    *p = it->second.back();
    it->second.pop_back();
    if (c > POOL_MAX_BYTES) pool->large_cached -= c;
    pool->live[*p] = c;
    return cudaSuccess;
  }
  cudaError_t e = cudaMalloc(p, c);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pool->release();
    e = cudaMalloc(p, c);
  }
  if (e == cudaSuccess) pool->live[*p] = c;
  return e;
}

// Freed blocks are reused by later allocations of the same context, whose work is
// ordered after the frees on the context's stream.
static void dev_free(void* p) {
  if (!p) return;
  if (DevPool* pool = t_pool) {
    auto it = pool->live.find(p);
    if (it != pool->live.end()) {
      const size_t c = it->second;
      pool->live.erase(it);
      if (c > POOL_MAX_BYTES) {
        if (pool->large_cached + c > POOL_LARGE_CACHE) {
          cudaFree(p);
          return;
        }
        pool->large_cached += c;
      }
      pool->cached[c].push_back(p);
      return;
    }
  }
  cudaFree(p);
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      throw Error(LRT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

static const int QNA[4] = {0, 1, 0, 1};
static const int QNB[4] = {0, 0, 1, 1};

// ---------------------------------------------------------------------------
// sector tables
// ---------------------------------------------------------------------------
struct Sectors {
  std::vector<int> a, b, d;
  std::unordered_map<int, int> idx;
  static int key(int qa, int qb) { return (qa + 512) * 2048 + (qb + 512); }
  int find(int qa, int qb) const {
    auto it = idx.find(key(qa, qb));
    return it == idx.end() ? -1 : it->second;
  }
  int add(int qa, int qb, int dim) {
    int i = (int)a.size();
    a.push_back(qa);
    b.push_back(qb);
    d.push_back(dim);
    idx[key(qa, qb)] = i;
    return i;
  }
  int n() const { return (int)a.size(); }
};

// fused (enlarged) basis of L (+) site (right = false) or site (+) R (right = true)
struct Fused {
  Sectors s;                        // fused labels and total dims
  std::vector<std::array<int, 4>> sub;   // source sector of sub-block n, or -1
  std::vector<std::array<int, 4>> off;   // row/col offset of sub-block n
  std::vector<std::array<int, 4>> dim;   // dimension of sub-block n (0 if absent)
};

static Fused fuse(const Sectors& src, bool right) {
  std::map<std::pair<int, int>, int> labels;
  for (int s = 0; s < src.n(); ++s)
    for (int n = 0; n < 4; ++n) {
      int qa = right ? src.a[s] - QNA[n] : src.a[s] + QNA[n];
      int qb = right ? src.b[s] - QNB[n] : src.b[s] + QNB[n];
      labels[{qa, qb}] = 1;
    }
  Fused f;
  for (auto& kv : labels) {
    std::array<int, 4> sub, off, dim;
    int tot = 0;
    for (int n = 0; n < 4; ++n) {
      int qa = right ? kv.first.first + QNA[n] : kv.first.first - QNA[n];
      int qb = right ? kv.first.second + QNB[n] : kv.first.second - QNB[n];
      int s = src.find(qa, qb);
      sub[n] = s;
      off[n] = tot;
      dim[n] = s >= 0 ? src.d[s] : 0;
      tot += dim[n];
    }
    if (tot == 0) continue;
    f.s.add(kv.first.first, kv.first.second, tot);
    f.sub.push_back(sub);
    f.off.push_back(off);
    f.dim.push_back(dim);
  }
  return f;
}

// ---------------------------------------------------------------------------
// integrals
// ---------------------------------------------------------------------------
struct Ints {
  int k = 0, nso = 0;
  std::vector<double> t;   // nso^2
  std::vector<double> v;   // nso^4, v[p,q,r,s] = <pq|rs>
  double e_core = 0.0;
  double T(int p, int q) const { return t[(size_t)p * nso + q]; }
  double V(int p, int q, int r, int s) const {
    return v[(((size_t)p * nso + q) * nso + r) * nso + s];
  }
};

static void build_ints(Ints& I, int k, const double* h, const double* eri, int nL, const double* B,
                       double e_core) {
  I.k = k;
  I.nso = 2 * k;
  const int n = I.nso;
  I.t.assign((size_t)n * n, 0.0);
  I.v.assign((size_t)n * n * n * n, 0.0);
  I.e_core = e_core;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j)
      for (int s = 0; s < 2; ++s) I.t[(size_t)(2 * i + s) * n + 2 * j + s] = h[i * k + j];
  std::vector<double> chem((size_t)k * k * k * k);
  if (eri) {
    std::memcpy(chem.data(), eri, chem.size() * sizeof(double));
  } else {
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j)
        for (int a = 0; a < k; ++a)
          for (int b = 0; b < k; ++b) {
            double acc = 0.0;
            for (int L = 0; L < nL; ++L) acc += B[((size_t)L * k + i) * k + j] * B[((size_t)L * k + a) * k + b];
            chem[(((size_t)i * k + j) * k + a) * k + b] = acc;
          }
  }
  // <pq|rs> = (pr|qs) with spin(p) = spin(r), spin(q) = spin(s)
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r) {
        if ((p & 1) != (r & 1)) continue;
        for (int s = 0; s < n; ++s) {
          if ((q & 1) != (s & 1)) continue;
          I.v[(((size_t)p * n + q) * n + r) * n + s] =
              chem[(((size_t)(p / 2) * k + r / 2) * k + q / 2) * k + s / 2];
        }
      }
}

// ---------------------------------------------------------------------------
// operator sets
// ---------------------------------------------------------------------------
enum Kind : int { KI = 0, KH, KC, KS, KA, KB, KP, KQ };

struct Key {
  int kind, p, q;
  bool operator<(const Key& o) const { return std::tie(kind, p, q) < std::tie(o.kind, o.p, o.q); }
};

static int kind_parity(int kind) { return (kind == KC || kind == KS) ? 1 : 0; }

// change of the block's own (N_a, N_b) caused by the operator
static void key_delta(const Key& k, int& da, int& db) {
  da = db = 0;
  auto add = [&](int p, int s) {
    if (p & 1) db += s; else da += s;
  };
  switch (k.kind) {
    case KC: add(k.p, +1); break;
    case KS: add(k.p, -1); break;
    case KA: add(k.p, +1); add(k.q, +1); break;
    case KB: add(k.p, +1); add(k.q, -1); break;
    case KP: add(k.p, -1); add(k.q, -1); break;
    case KQ: add(k.q, +1); add(k.p, -1); break;
    default: break;
  }
}

struct OpSet {
  Sectors basis;          // bond labels (left: own count; right: N - own count)
  bool right = false;
  std::vector<int> orbs;
  std::vector<char> in;
  char mode = 'N';
  std::vector<Key> keys;
  std::map<Key, int> index;
  std::vector<int> da, db, par;
  std::vector<int> bra;        // [op * ns + ket] -> bra sector or -1
  std::vector<int64_t> off;    // [op * ns + ket] -> offset (doubles) or -1
  int64_t total = 0;
  double* d = nullptr;
  std::unique_ptr<Fused> fused;   // for enlarged sets
  std::vector<uint16_t> mask;     // enlarged sets: nonzero sub-blocks (bit 4*n_bra + n_ket) per block
  std::vector<char> bnz;          // per block: not identically zero (structural zeros are skipped)
  std::vector<char> onz;          // per operator: some block not identically zero

  bool block_nz(int op, int ket) const { return bnz[(size_t)op * ns() + ket] != 0; }
  void finish_nz() {
    onz.assign(keys.size(), 0);
    for (size_t o = 0; o < keys.size(); ++o)
      for (int s = 0; s < ns(); ++s)
        if (bnz[o * ns() + s]) onz[o] = 1;
  }
  OpSet() = default;
  OpSet(const OpSet&) = delete;
  ~OpSet() {
    if (d) dev_free(d);
  }
  int ns() const { return basis.n(); }
  int find(const Key& k) const {
    auto it = index.find(k);
    return it == index.end() ? -1 : it->second;
  }
  int bra_of(int op, int ket) const { return bra[(size_t)op * ns() + ket]; }
  int64_t off_of(int op, int ket) const { return off[(size_t)op * ns() + ket]; }
};

static void make_keys(OpSet& S, const std::vector<int>& orbs, char mode, int nso) {
  S.orbs = orbs;
  S.in.assign(nso, 0);
  for (int p : orbs) S.in[p] = 1;
  S.mode = mode;
  std::vector<int> out;
  for (int p = 0; p < nso; ++p)
    if (!S.in[p]) out.push_back(p);
  auto push = [&](int kind, int p, int q) {
    Key k{kind, p, q};
    S.index[k] = (int)S.keys.size();
    S.keys.push_back(k);
  };
  push(KI, -1, -1);
  push(KH, -1, -1);
  for (int p : orbs) push(KC, p, -1);
  for (int z : out) push(KS, z, -1);
  const std::vector<int>& pr = (mode == 'N') ? orbs : out;
  const int A = (mode == 'N') ? KA : KP, B = (mode == 'N') ? KB : KQ;
  for (size_t i = 0; i < pr.size(); ++i)
    for (size_t j = i + 1; j < pr.size(); ++j) push(A, pr[i], pr[j]);
  for (size_t i = 0; i < pr.size(); ++i)
    for (size_t j = i; j < pr.size(); ++j) push(B, pr[i], pr[j]);
  const int nop = (int)S.keys.size();
  S.da.resize(nop);
  S.db.resize(nop);
  S.par.resize(nop);
  for (int o = 0; o < nop; ++o) {
    key_delta(S.keys[o], S.da[o], S.db[o]);
    S.par[o] = kind_parity(S.keys[o].kind);
  }
}

static void layout_blocks(OpSet& S) {
  const int ns = S.ns(), nop = (int)S.keys.size();
  const int sg = S.right ? -1 : 1;
  S.bra.assign((size_t)nop * ns, -1);
  S.off.assign((size_t)nop * ns, -1);
  S.bnz.assign((size_t)nop * ns, 0);
  S.total = 0;
  for (int o = 0; o < nop; ++o)
    for (int s = 0; s < ns; ++s) {
      int b = S.basis.find(S.basis.a[s] + sg * S.da[o], S.basis.b[s] + sg * S.db[o]);
      if (b < 0) continue;
      S.bra[(size_t)o * ns + s] = b;
      S.off[(size_t)o * ns + s] = S.total;
      S.total += (int64_t)S.basis.d[b] * S.basis.d[s];
    }
}

static void alloc_zero(OpSet& S, cudaStream_t st) {
  if (S.total <= 0) return;
  cudaError_t e = dev_alloc((void**)&S.d, (size_t)S.total * sizeof(double));
  if (e != cudaSuccess) throw Error(LRT_ENOMEM, "device allocation of an operator set failed");
  CK(cudaMemsetAsync(S.d, 0, (size_t)S.total * sizeof(double), st));
}

// ---------------------------------------------------------------------------
// single-site operators (4 x 4, basis |0>, |a>, |b>, |ab> = C_a C_b |0>)
// ---------------------------------------------------------------------------
struct Mat4 {
  double m[16];
  Mat4() { std::fill(m, m + 16, 0.0); }
  double& operator()(int i, int j) { return m[i * 4 + j]; }
  double operator()(int i, int j) const { return m[i * 4 + j]; }
  Mat4 operator*(const Mat4& o) const {
    Mat4 r;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        double s = 0.0;
        for (int l = 0; l < 4; ++l) s += m[i * 4 + l] * o.m[l * 4 + j];
        r.m[i * 4 + j] = s;
      }
    return r;
  }
  Mat4& axpy(double c, const Mat4& o) {
    for (int i = 0; i < 16; ++i) m[i] += c * o.m[i];
    return *this;
  }
  Mat4 T() const {
    Mat4 r;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) r.m[j * 4 + i] = m[i * 4 + j];
    return r;
  }
  bool zero() const {
    for (double x : m)
      if (x != 0.0) return false;
    return true;
  }
};

struct Site {
  int i;
  Mat4 ann[2], cre[2];   // local a_alpha, a_beta and their transposes
  explicit Site(int site) : i(site) {
    // a_alpha: |a> -> |0>, |ab> -> |b>;  a_beta: |b> -> |0>, |ab> = C_a C_b|0> -> -C_a|0> = -|a>
    ann[0](0, 1) = 1.0;
    ann[0](2, 3) = 1.0;
    ann[1](0, 2) = 1.0;
    ann[1](1, 3) = -1.0;
    cre[0] = ann[0].T();
    cre[1] = ann[1].T();
  }
  bool local(int p) const { return p / 2 == i; }
  const Mat4& C(int p) const { return cre[p & 1]; }
  const Mat4& c(int p) const { return ann[p & 1]; }
  Mat4 op(const Ints& I, int kind, int p, int q, int trans) const {
    Mat4 r;
    const int lo[2] = {2 * i, 2 * i + 1};
    switch (kind) {
      case KI:
        for (int a = 0; a < 4; ++a) r(a, a) = 1.0;
        break;
      case KH:
        for (int x : lo)
          for (int y : lo) r.axpy(I.T(x, y), C(x) * c(y));
        for (int pp : lo)
          for (int qq : lo)
            for (int rr : lo)
              for (int ss : lo) r.axpy(0.5 * I.V(pp, qq, rr, ss), C(pp) * C(qq) * c(ss) * c(rr));
        break;
      case KC:
        r = C(p);
        break;
      case KS:
        for (int x : lo) r.axpy(0.5 * I.T(p, x), c(x));
        for (int qq : lo)
          for (int rr : lo)
            for (int ss : lo) r.axpy(I.V(p, qq, rr, ss), C(qq) * c(ss) * c(rr));
        break;
      case KA:
        r = C(p) * C(q);
        break;
      case KB:
        r = C(p) * c(q);
        break;
      case KP:
        for (int rr : lo)
          for (int ss : lo) r.axpy(I.V(p, q, rr, ss), c(ss) * c(rr));
        break;
      case KQ:
        for (int rr : lo)
          for (int ss : lo) r.axpy(I.V(p, rr, q, ss) - I.V(p, rr, ss, q), C(rr) * c(ss));
        break;
    }
    return trans ? r.T() : r;
  }
};

// ---------------------------------------------------------------------------
// operator references: a requested operator as a combination of stored ones
// ---------------------------------------------------------------------------
struct Ref {
  int op;
  int t;
  double c;
};

static void get_refs(const OpSet& S, const Ints& I, int kind, int p, int q, int t, double c,
                     std::vector<Ref>& out) {
  auto stored = [&](int kk, int a, int b, int tt, double cc) {
    int o = S.find(Key{kk, a, b});
    if (o >= 0 && (S.onz.empty() || S.onz[o])) out.push_back(Ref{o, tt, cc});
  };
  switch (kind) {
    case KI: stored(KI, -1, -1, t, c); return;
    case KH: stored(KH, -1, -1, t, c); return;
    case KC: stored(KC, p, -1, t, c); return;
    case KS: stored(KS, p, -1, t, c); return;
    case KA:
      if (p == q) return;
      if (p < q) stored(KA, p, q, t, c); else stored(KA, q, p, t, -c);
      return;
    case KB:
      if (p <= q) stored(KB, p, q, t, c); else stored(KB, q, p, 1 - t, c);
      return;
    case KP:
      if (p == q) return;
      if (p > q) { get_refs(S, I, KP, q, p, t, -c, out); return; }
      if (S.mode == 'C') { stored(KP, p, q, t, c); return; }
      // P_pq = sum_{r<s in Z} (v_pqrs - v_pqsr) A_rs^T
      for (size_t i = 0; i < S.orbs.size(); ++i)
        for (size_t j = i + 1; j < S.orbs.size(); ++j) {
          const int r = S.orbs[i], s = S.orbs[j];
          const double w = I.V(p, q, r, s) - I.V(p, q, s, r);
          if (w != 0.0) stored(KA, r, s, 1 - t, c * w);
        }
      return;
    case KQ:
      if (p > q) { get_refs(S, I, KQ, q, p, 1 - t, c, out); return; }
      if (S.mode == 'C') { stored(KQ, p, q, t, c); return; }
      // Q_pq = sum_{r,s in Z} (v_prqs - v_prsq) B_rs
      for (int r : S.orbs)
        for (int s : S.orbs) {
          const double w = I.V(p, r, q, s) - I.V(p, r, s, q);
          if (w != 0.0) get_refs(S, I, KB, r, s, t, c * w, out);
        }
      return;
  }
}

// ---------------------------------------------------------------------------
// terms: (coef, X spec, Y spec)
// ---------------------------------------------------------------------------
struct Spec {
  int kind, p, q, t;
};
struct Term {
  double c;
  Spec x, y;
};

static void cross_terms(const std::vector<int>& X, const std::vector<int>& Y, bool x_normal,
                        std::vector<Term>& T) {
  for (int x : X) {
    T.push_back({1.0, {KC, x, -1, 0}, {KS, x, -1, 0}});
    T.push_back({-1.0, {KC, x, -1, 1}, {KS, x, -1, 1}});
  }
  for (int y : Y) {
    T.push_back({1.0, {KS, y, -1, 1}, {KC, y, -1, 1}});
    T.push_back({-1.0, {KS, y, -1, 0}, {KC, y, -1, 0}});
  }
  const std::vector<int>& N = x_normal ? X : Y;
  for (size_t i = 0; i < N.size(); ++i)
    for (size_t j = i + 1; j < N.size(); ++j) {
      const int p = N[i], q = N[j];
      if (x_normal) {
        T.push_back({1.0, {KA, p, q, 0}, {KP, p, q, 0}});
        T.push_back({1.0, {KA, p, q, 1}, {KP, p, q, 1}});
      } else {
        T.push_back({1.0, {KP, p, q, 1}, {KA, p, q, 1}});
        T.push_back({1.0, {KP, p, q, 0}, {KA, p, q, 0}});
      }
    }
  for (size_t i = 0; i < N.size(); ++i)
    for (size_t j = i; j < N.size(); ++j) {
      const int p = N[i], q = N[j];
      if (x_normal) {
        T.push_back({1.0, {KB, p, q, 0}, {KQ, p, q, 0}});
        if (p != q) T.push_back({1.0, {KB, p, q, 1}, {KQ, p, q, 1}});
      } else {
        T.push_back({1.0, {KQ, p, q, 0}, {KB, p, q, 0}});
        if (p != q) T.push_back({1.0, {KQ, p, q, 1}, {KB, p, q, 1}});
      }
    }
}

// terms of every operator of X (+) Y (X before Y), keyed like the new set
static std::vector<std::vector<Term>> blocking_terms(const OpSet& New, const std::vector<int>& X,
                                                      const std::vector<int>& Y, const Ints& I) {
  std::vector<char> inX(I.nso, 0), inY(I.nso, 0);
  for (int p : X) inX[p] = 1;
  for (int p : Y) inY[p] = 1;
  std::vector<std::vector<Term>> out(New.keys.size());
  for (size_t o = 0; o < New.keys.size(); ++o) {
    const Key& k = New.keys[o];
    std::vector<Term>& T = out[o];
    switch (k.kind) {
      case KI:
        T.push_back({1.0, {KI, -1, -1, 0}, {KI, -1, -1, 0}});
        break;
      case KH:
        T.push_back({1.0, {KH, -1, -1, 0}, {KI, -1, -1, 0}});
        T.push_back({1.0, {KI, -1, -1, 0}, {KH, -1, -1, 0}});
        cross_terms(X, Y, X.size() < Y.size(), T);
        break;
      case KC:
        if (inX[k.p]) T.push_back({1.0, {KC, k.p, -1, 0}, {KI, -1, -1, 0}});
        else T.push_back({1.0, {KI, -1, -1, 0}, {KC, k.p, -1, 0}});
        break;
      case KS: {
        const int z = k.p;
        T.push_back({1.0, {KS, z, -1, 0}, {KI, -1, -1, 0}});
        T.push_back({1.0, {KI, -1, -1, 0}, {KS, z, -1, 0}});
        for (int q : X) T.push_back({1.0, {KC, q, -1, 0}, {KP, z, q, 0}});
        for (int q : Y) T.push_back({1.0, {KP, z, q, 0}, {KC, q, -1, 0}});
        for (int w : Y) T.push_back({1.0, {KQ, z, w, 0}, {KC, w, -1, 1}});
        for (int u : X) T.push_back({1.0, {KC, u, -1, 1}, {KQ, z, u, 0}});
        break;
      }
      case KA:
        if (inX[k.p] && inX[k.q]) T.push_back({1.0, {KA, k.p, k.q, 0}, {KI, -1, -1, 0}});
        else if (inY[k.p] && inY[k.q]) T.push_back({1.0, {KI, -1, -1, 0}, {KA, k.p, k.q, 0}});
        else T.push_back({1.0, {KC, k.p, -1, 0}, {KC, k.q, -1, 0}});
        break;
      case KB:
        if (inX[k.p] && inX[k.q]) T.push_back({1.0, {KB, k.p, k.q, 0}, {KI, -1, -1, 0}});
        else if (inY[k.p] && inY[k.q]) T.push_back({1.0, {KI, -1, -1, 0}, {KB, k.p, k.q, 0}});
        else T.push_back({1.0, {KC, k.p, -1, 0}, {KC, k.q, -1, 1}});
        break;
      case KP: {
        const int p = k.p, q = k.q;
        T.push_back({1.0, {KP, p, q, 0}, {KI, -1, -1, 0}});
        T.push_back({1.0, {KI, -1, -1, 0}, {KP, p, q, 0}});
        for (int x : X)
          for (int y : Y) {
            const double w = I.V(p, q, y, x) - I.V(p, q, x, y);
            if (w != 0.0) T.push_back({w, {KC, x, -1, 1}, {KC, y, -1, 1}});
          }
        break;
      }
      case KQ: {
        const int p = k.p, q = k.q;
        T.push_back({1.0, {KQ, p, q, 0}, {KI, -1, -1, 0}});
        T.push_back({1.0, {KI, -1, -1, 0}, {KQ, p, q, 0}});
        for (int x : X)
          for (int y : Y) {
            const double w1 = I.V(p, x, q, y) - I.V(p, x, y, q);
            if (w1 != 0.0) T.push_back({w1, {KC, x, -1, 0}, {KC, y, -1, 1}});
            const double w2 = -(I.V(p, y, q, x) - I.V(p, y, x, q));
            if (w2 != 0.0) T.push_back({w2, {KC, x, -1, 1}, {KC, y, -1, 0}});
          }
        break;
      }
    }
  }
  return out;
}

// ---------------------------------------------------------------------------
// device upload helper
// ---------------------------------------------------------------------------
template <class T>
struct DevArray {
  T* p = nullptr;
  size_t n = 0;
  DevArray() = default;
  DevArray(const DevArray&) = delete;
  ~DevArray() {
    if (p) dev_free(p);
  }
  void swap(DevArray& o) {
    std::swap(p, o.p);
    std::swap(n, o.n);
  }
  void upload(const std::vector<T>& v, cudaStream_t st) {
    if (p) {
      dev_free(p);
      p = nullptr;
    }
    n = v.size();
    if (n == 0) return;
    if (dev_alloc((void**)&p, n * sizeof(T)) != cudaSuccess) throw Error(LRT_ENOMEM, "device allocation failed");
    CK(cudaMemcpyAsync(p, v.data(), n * sizeof(T), cudaMemcpyHostToDevice, st));
  }
};

struct DevBuf {
  double* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) {
    o.p = nullptr;
    o.n = 0;
  }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      if (p) dev_free(p);
      p = o.p;
      n = o.n;
      o.p = nullptr;
      o.n = 0;
    }
    return *this;
  }
  ~DevBuf() {
    if (p) dev_free(p);
  }
  double* ensure(size_t need) {
    if (need <= n && p) return p;
    if (p) dev_free(p);
    p = nullptr;
    n = 0;
    if (need == 0) need = 1;
    if (dev_alloc((void**)&p, need * sizeof(double)) != cudaSuccess) throw Error(LRT_ENOMEM, "device allocation (sweep)");
    n = need;
    return p;
  }
};

struct GatherPlan {
  DevArray<GatherTask> tasks;
  DevArray<GatherSrc> srcs;
  DevArray<int3> tiles;
  int ntiles = 0;
  void run(cudaStream_t st) const { launch_gather(tasks.p, srcs.p, tiles.p, ntiles, st); }
};

struct GemmPlan {
  DevArray<GemmOut> outs;    // the plan's outputs, then the K parts of split tiles
  DevArray<GemmSeg> segs;
  DevArray<int3> tiles;      // FP64 kernel tiles
  int ntiles = 0;
  int nbase = 0;             // outputs before the K parts
  DevArray<SplitTile> splits;
  int nsplit = 0;
  DevBuf ws;                 // partial tiles of the split tiles
  double flops = 0.0;
  void run(cudaStream_t st, const double* xb, double* yb, double* tb = nullptr, const GemmExtra* ex = nullptr) const {
    launch_gemm_fp64(outs.p, segs.p, tiles.p, ntiles, xb, yb, tb, st, ex, ws.p);
    if (nsplit > 0) launch_split_reduce(outs.p, splits.p, nsplit, ws.p, yb, tb, st);
  }
  int launches() const { return (ntiles > 0) + (nsplit > 0); }
};

static void build_gather(GatherPlan& P, std::vector<GatherTask>& tasks, std::vector<GatherSrc>& srcs,
                         cudaStream_t st) {
  std::vector<int3> tiles;
  for (size_t i = 0; i < tasks.size(); ++i) {
    const int64_t nch = ((int64_t)tasks[i].rows * tasks[i].cols + GATHER_CHUNK - 1) / GATHER_CHUNK;
    if (nch > INT32_MAX) throw Error(LRT_EINVAL, "gather: destination block too large");
    for (int64_t a = 0; a < nch; ++a) tiles.push_back(make_int3((int)i, (int)a, 0));
  }
  P.tasks.upload(tasks, st);
  P.srcs.upload(srcs, st);
  P.tiles.upload(tiles, st);
  P.ntiles = (int)tiles.size();
}

static void build_gemm(GemmPlan& P, const std::vector<GemmOut>& outs_in, const std::vector<GemmSeg>& segs,
                       cudaStream_t st, bool split = false) {
  // A tile costs its warps of outputs times its K chunks of DFMA issue, plus a fixed
  // cost per chunk.  Tiles far longer than an even share of the launch (an output with
  // many long K segments) would run on after all others finished.  With `split`, an
  // output that sums several segments (y or T outputs) and at least 2 GEMM_SPLIT_K of K
  // has each of its tiles cut along its segment list into K parts of about GEMM_SPLIT_K:
  // each part a partial tile in the workspace, added in order by the reduction launch.
  // The parts depend on the output's own segments only, so an element is summed in the
  // same grouping whichever call (vector count, batch) the output belongs to.  Otherwise
  // tiles above an even share are cut into row slices.  Then the longest go first.  (Row
  // slices of a quarter share were measured 2.5x slower on the k = 24 workload's phase 2:
  // every slice stages the whole K range of B for a few rows; a K part stages only its
  // own range.)
  std::vector<GemmOut> outs = outs_in;
  std::vector<int64_t> ktot(outs_in.size(), 0);
  double fl = 0.0;
  for (size_t i = 0; i < outs_in.size(); ++i)
    for (int s = 0; s < outs_in[i].seg_count; ++s) {
      ktot[i] += segs[outs_in[i].seg_begin + s].k;
      fl += 2.0 * outs_in[i].m * (double)outs_in[i].n * segs[outs_in[i].seg_begin + s].k;
    }
  auto cost = [](int64_t mt, int64_t nt, int64_t k) {
    return ((k + GEMM_KC - 1) / GEMM_KC) * (32 * ((mt * nt + 31) / 32) + 64) + 64;
  };
  int64_t total = 0;
  for (size_t i = 0; i < outs_in.size(); ++i)
    for (int m0 = 0; m0 < outs_in[i].m; m0 += GEMM_TM)
      for (int n0 = 0; n0 < outs_in[i].n; n0 += GEMM_TN)
        total += cost(std::min(GEMM_TM, outs_in[i].m - m0), std::min(GEMM_TN, outs_in[i].n - n0), ktot[i]);
  const int64_t cap = std::max<int64_t>(1, total / gemm_fp64_slots());
  std::vector<std::pair<int64_t, int3>> tl;
  std::vector<SplitTile> sp;
  int64_t wsz = 0;
  for (size_t i = 0; i < outs_in.size(); ++i) {
    const GemmOut& O = outs_in[i];
    for (int m0 = 0; m0 < O.m; m0 += GEMM_TM)
      for (int n0 = 0; n0 < O.n; n0 += GEMM_TN) {
        const int mt = std::min(GEMM_TM, O.m - m0), nt = std::min(GEMM_TN, O.n - n0);
        const int64_t c = cost(mt, nt, ktot[i]);
        const int want = (int)std::min<int64_t>(O.seg_count, ktot[i] / GEMM_SPLIT_K);
        if (split && want >= 2 && O.c_rel <= 2 && outs.size() < (size_t)INT32_MAX) {
          // contiguous runs of the segment list, each about ktot / want of K
          SplitTile t{wsz, (int)i, 0, m0, mt, n0, nt};
          std::vector<int> kseg(O.seg_count);
          for (int q = 0; q < O.seg_count; ++q) kseg[q] = segs[O.seg_begin + q].k;
          split_segments(kseg.data(), O.seg_count, ktot[i], want, [&](int sb, int se, long long kp) {
            GemmOut po = O;
            po.C = nullptr;
            po.c_rel = GEMM_C_SPLIT;
            po.c_off = wsz + (int64_t)t.nparts * mt * nt - ((int64_t)m0 * nt + n0);
            po.ldc = nt;
            po.accumulate = 0;
            po.c_vr = po.c_vc = 0;
            po.c_vs = 0;
            po.seg_begin = O.seg_begin + sb;
            po.seg_count = se - sb;
            outs.push_back(po);
            tl.push_back({cost(mt, nt, kp), gemm_tile((int)outs.size() - 1, m0, mt, n0, nt)});
            ++t.nparts;
          });
          wsz += (int64_t)t.nparts * mt * nt;
          sp.push_back(t);
          continue;
        }
        const int parts = (int)std::min<int64_t>(mt, (c + cap - 1) / cap);
        for (int p = 0, r = m0; p < parts; ++p) {
          const int rows = mt / parts + (p < mt % parts ? 1 : 0);
          tl.push_back({cost(rows, nt, ktot[i]), gemm_tile((int)i, r, rows, n0, nt)});
          r += rows;
        }
      }
  }
  std::stable_sort(tl.begin(), tl.end(), [](const std::pair<int64_t, int3>& a, const std::pair<int64_t, int3>& b) {
    return a.first > b.first;
  });
  std::vector<int3> tiles(tl.size());
  for (size_t t = 0; t < tl.size(); ++t) tiles[t] = tl[t].second;
  P.outs.upload(outs, st);
  P.segs.upload(segs, st);
  P.tiles.upload(tiles, st);
  P.ntiles = (int)tiles.size();
  P.nbase = (int)outs_in.size();
  P.splits.upload(sp, st);
  P.nsplit = (int)sp.size();
  if (wsz > 0) P.ws.ensure((size_t)wsz);
  P.flops = fl;
}

}  // namespace lrt

// ===========================================================================
// context
// ===========================================================================
namespace lrt {

struct SiteTensor {
  std::vector<int64_t> blk_off;     // per right-bond sector: start of its fused block (-1 if empty)
  std::vector<int> blk_rows;        // fused rows of that block
  // sub-block (q_l, n): offset of the D_l x D_r sub-block and its right sector
  std::vector<std::array<int64_t, 4>> sub_off;   // per left-bond sector
  std::vector<std::array<int, 4>> sub_qr;
  int64_t total = 0;
  double* d = nullptr;
  SiteTensor() = default;
  SiteTensor(SiteTensor&& o) noexcept
      : blk_off(std::move(o.blk_off)), blk_rows(std::move(o.blk_rows)), sub_off(std::move(o.sub_off)),
        sub_qr(std::move(o.sub_qr)), total(o.total), d(o.d) {
    o.d = nullptr;
  }
  SiteTensor(const SiteTensor&) = delete;
  SiteTensor& operator=(SiteTensor&& o) noexcept {
    if (this != &o) {
      if (d) dev_free(d);
      blk_off = std::move(o.blk_off);
      blk_rows = std::move(o.blk_rows);
      sub_off = std::move(o.sub_off);
      sub_qr = std::move(o.sub_qr);
      total = o.total;
      d = o.d;
      o.d = nullptr;
    }
    return *this;
  }
  ~SiteTensor() {
    if (d) dev_free(d);
  }
};

static void site_layout(SiteTensor& S, const Sectors& L, const Sectors& R) {
  S.blk_off.assign(R.n(), -1);
  S.blk_rows.assign(R.n(), 0);
  S.sub_off.assign(L.n(), {-1, -1, -1, -1});
  S.sub_qr.assign(L.n(), {-1, -1, -1, -1});
  int64_t off = 0;
  for (int r = 0; r < R.n(); ++r) {
    int rows = 0;
    const int64_t start = off;
    for (int n = 0; n < 4; ++n) {
      const int l = L.find(R.a[r] - QNA[n], R.b[r] - QNB[n]);
      if (l < 0) continue;
      S.sub_off[l][n] = start + (int64_t)rows * R.d[r];
      S.sub_qr[l][n] = r;
      rows += L.d[l];
    }
    if (rows > 0) {
      S.blk_off[r] = start;
      S.blk_rows[r] = rows;
    }
    off += (int64_t)rows * R.d[r];
  }
  S.total = off;
}

struct TdaState;

// Tensor-core twin of a sigma plan.  A TC matrix is R x K (R = output rows or
// columns of the product, K = contracted index), packed as ceil(K / 32) chunks of
// Rp = roundup(R, 8) rows of 32 TF32 pairs (see TcPack).
struct TcMat {
  int pool;
  int64_t off;     // float offset inside its pool (inside one vector's part for pools 1, 2)
  int R, Rp, K;
};
struct TcPlanSeg {
  int a, b;        // TC matrices
  int k;
  float scale;
};
struct TcPlanOut {
  int tmat;        // output TC matrix (intermediate), or -1 for an FP64 output
  int64_t c_off;   // FP64 output in y: offset and row stride
  int ldc;
  int m, n;
  int seg_begin, seg_count;
  double* C = nullptr;   // FP64 output at an absolute address instead of y (row stride ldc)
};
struct TcPlan {
  std::vector<TcMat> mats;
  int64_t pool_size[3] = {0, 0, 0};     // floats (per vector for pools 1, 2)
  std::vector<TcPack> pack0;            // operator sub-matrices (absolute sources)
  std::vector<TcPack> pack1;            // x-derived (sources relative to x)
  std::map<std::tuple<const double*, int64_t, int, int, int>, int> op_of;
  std::map<std::tuple<int64_t, int64_t, int, int, int>, int> x_of;
  std::vector<TcPlanOut> out1, out2;
  std::vector<TcPlanSeg> segs;
  static int64_t words(int Rp, int K) { return (int64_t)((K + 31) / 32) * Rp * 32; }
  int add(int pool, int R, int K) {
    TcMat m{pool, pool_size[pool], R, (R + 7) & ~7, K};
    pool_size[pool] += words(m.Rp, K);
    mats.push_back(m);
    return (int)mats.size() - 1;
  }
  // operator sub-matrix: element (r, k) = src[r * ld + k] (or src[k * ld + r] when trans)
  int op(const double* src, int64_t ld, int trans, int R, int K) {
    auto key = std::make_tuple(src, ld, trans, R, K);
    auto it = op_of.find(key);
    if (it != op_of.end()) return it->second;
    const int id = add(0, R, K);
    pack0.push_back(TcPack{src, 0, ld, mats[id].off, R, K, mats[id].Rp, trans});
    op_of[key] = id;
    return id;
  }
  // sub-matrix of x, source offset relative to the vector's start
  int x(int64_t src_off, int64_t ld, int trans, int R, int K) {
    auto key = std::make_tuple(src_off, ld, trans, R, K);
    auto it = x_of.find(key);
    if (it != x_of.end()) return it->second;
    const int id = add(1, R, K);
    pack1.push_back(TcPack{nullptr, src_off, ld, mats[id].off, R, K, mats[id].Rp, trans});
    x_of[key] = id;
    return id;
  }
};

struct SigmaPlan {
  uint64_t serial = 0;      // unique per plan (batched launches detect rebuilt plans by it)
  bool has_tc = false;      // the tensor-core twin was planned
  GemmPlan p1, p2;
  // operator sets of a plan built with relative addresses (X, Xrev, Y, Yrev at extra
  // bases 0..3); a kept plan serves new sets of the same layout by changing these
  GemmExtra ex{};
  DevArray<DiagOut> douts;
  DevArray<DiagTerm> dterms;
  int ndiag = 0;
  double* tbuf = nullptr;   // workspace of the phase-1 intermediates
  int64_t tsize = 0;        // its size in doubles
  int64_t nelem = 0;
  int n_terms = 0, n_products = 0;
  double op_bytes = 0.0;
  double flops_alg = 0.0;   // products of non-zero sub-blocks only
  // tensor-core twin of the two phases (host description; device streams built on
  // first mixed use): whole fused blocks, operands as TC matrices in three pools
  // (0: operator sub-matrices, 1: x-derived, per vector, 2: intermediates T, per vector)
  TcPlan tc;
  // mixed path (split TF32): segments with TF32 operand pointers and hi/lo workspaces
  bool tc_ready = false;
  DevArray<TcItem> tci1, tci2;    // per-CTA work streams of the two phases
  DevArray<int> tcb1, tcb2;
  int tcn1 = 0, tcn2 = 0;
  int tn1 = 64, tn2 = 64;         // tile widths chosen by the autotuner
  DevArray<TcPack> xpack;         // packing of x into pool 1 (every call)
  float* pool_hi[3] = {nullptr, nullptr, nullptr};
  float* pool_lo[3] = {nullptr, nullptr, nullptr};
  ~SigmaPlan() {
    if (tbuf) dev_free(tbuf);
    for (int q = 0; q < 3; ++q) {
      if (pool_hi[q]) dev_free(pool_hi[q]);
      if (pool_lo[q]) dev_free(pool_lo[q]);
    }
  }
};

}  // namespace lrt

namespace lrt {
struct BatchPlan;
}
struct lrt_ctx {
  lrt::DevPool pool;     // first member: destroyed last, after every buffer returned to it
  uint64_t id = 0;       // unique per context (batched launches identify instances by it)
  std::map<std::string, std::unique_ptr<lrt::BatchPlan>> batches;   // batched sigma led by this context
  int dev = 0;
  cudaStream_t st = nullptr;
  std::string err;
  bool have_ham = false;
  lrt::Ints I;
  bool have_mps = false;
  int k = 0, na = 0, nb = 0;
  std::vector<lrt::Sectors> bonds;
  std::vector<lrt::SiteTensor> sites;     // left-canonical (or only) form
  std::vector<lrt::SiteTensor> sites_r;   // right-canonical form, when given separately
  std::vector<std::unique_ptr<lrt::OpSet>> L, R, XL, YR;
  std::map<std::tuple<int, int, int>, std::unique_ptr<lrt::SigmaPlan>> plans;
  lrt_sigma_stats last{};
  int last_sweeps = 0;
  std::vector<std::pair<double, int>> sweep_log;   // last sweep_tda: seconds and mixed flag per sweep
  uint64_t tc_wait_ns = 0;   // limit of the tensor-core pipeline waits (0: the default)
  int tc_stall = 0;          // test hook: the next tensor-core launch stalls on a wait
  int* derr = nullptr;   // device flag set by a kernel whose bounded wait expired
  std::unique_ptr<lrt::TdaState> tda;
  // right-fused copy task lists per (bond, layout of site tensor and fused basis), relative
  // to the copy's buffer and the site tensor
  std::map<std::pair<int, uint64_t>, std::unique_ptr<lrt::GatherPlan>> rf_plans;
  ~lrt_ctx() {
    if (derr) lrt::dev_free(derr);
  }
};

namespace lrt {

// the output block of a tensor-core launch with the context's wait settings; a pending
// stall (test hook) is consumed by this launch
static TcOut tc_out(lrt_ctx* c, double* y, double* const* ys) {
  TcOut o{y, ys, (unsigned long long)c->tc_wait_ns, c->tc_stall};
  c->tc_stall = 0;
  return o;
}

static char left_mode(int b, int k) { return (2 * b <= k) ? 'N' : 'C'; }
static char right_mode(int b, int k) { return (2 * b <= k) ? 'C' : 'N'; }

static void drop_plans(lrt_ctx* c) { c->plans.clear(); }

static std::unique_ptr<OpSet> vacuum(lrt_ctx* c, bool right) {
  auto S = std::make_unique<OpSet>();
  S->right = right;
  const int b = right ? c->k : 0;
  const Sectors& bt = c->bonds[b];
  S->basis.add(bt.a[0], bt.b[0], 1);
  make_keys(*S, {}, right ? right_mode(b, c->k) : left_mode(b, c->k), c->I.nso);
  layout_blocks(*S);
  alloc_zero(*S, c->st);
  const double one = 1.0;
  const int iop = S->find(Key{KI, -1, -1});
  CK(cudaMemcpyAsync(S->d + S->off_of(iop, 0), &one, sizeof(double), cudaMemcpyHostToDevice, c->st));
  S->bnz[(size_t)iop * S->ns()] = 1;
  S->finish_nz();
  CK(cudaStreamSynchronize(c->st));
  return S;
}

static void reset_env(lrt_ctx* c) {
  drop_plans(c);
  c->L.clear();
  c->R.clear();
  c->XL.clear();
  c->YR.clear();
  if (!c->have_mps || !c->have_ham) return;
  c->L.resize(c->k + 1);
  c->R.resize(c->k + 1);
  c->XL.resize(c->k);
  c->YR.resize(c->k);
  c->L[0] = vacuum(c, false);
  c->R[c->k] = vacuum(c, true);
}

// L[b] (+) site b  (right = false)   or   site b (+) R[b+1]  (right = true)
// X (+) site b (right = false: X is a left block ending at bond b) or site b (+) X
// (right = true: X is a right block starting at bond b+1).  For a first-order
// (transition) set X, Xrev is its reverse set: a transposed reference reads it.
// The plan of one enlargement (layout of the enlarged set and its gather tasks, with
// addresses as offsets), reusable for any input set of the same layout and structure:
// the TDA enlarges the first-order sets of every trial vector at a site, all alike.
struct EnlTemplate {
  std::unique_ptr<OpSet> proto;        // layout of the enlarged set, no data
  std::unique_ptr<GatherPlan> gp;      // device task list: destinations relative to the new
                                       // set, sources relative to X (rel 1) or Xrev (rel 2)
  uint64_t sig = 0;
};

// layout and structure signature of an input (X, Xrev) pair
static uint64_t set_signature(const OpSet& X, const OpSet* Xr) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  for (const OpSet* S : {&X, Xr}) {
    if (!S) {
      mix(0x9E3779B97F4A7C15ull);
      continue;
    }
    mix((uint64_t)S->keys.size());
    mix((uint64_t)S->ns());
    mix((uint64_t)S->total);
    for (char b : S->bnz) mix((uint64_t)(unsigned char)b);
  }
  return h;
}

static std::unique_ptr<OpSet> layout_copy(const OpSet& t) {
  auto S = std::make_unique<OpSet>();
  S->basis = t.basis;
  S->right = t.right;
  S->orbs = t.orbs;
  S->in = t.in;
  S->mode = t.mode;
  S->keys = t.keys;
  S->index = t.index;
  S->da = t.da;
  S->db = t.db;
  S->par = t.par;
  S->bra = t.bra;
  S->off = t.off;
  S->total = t.total;
  S->bnz = t.bnz;
  S->onz = t.onz;
  S->mask = t.mask;
  if (t.fused) S->fused = std::make_unique<Fused>(*t.fused);
  return S;
}

static std::unique_ptr<OpSet> enlarge_set(lrt_ctx* c, const OpSet& X, const OpSet* Xrev, int b, bool right,
                                          EnlTemplate* tpl = nullptr) {
  const Ints& I = c->I;
  const Site site(b);
  auto E = std::make_unique<OpSet>();
  E->right = right;
  E->fused = std::make_unique<Fused>(fuse(X.basis, right));
  E->basis = E->fused->s;
  std::vector<int> sorbs = {2 * b, 2 * b + 1};
  std::vector<int> orbs;
  if (right) {
    orbs = sorbs;
    orbs.insert(orbs.end(), X.orbs.begin(), X.orbs.end());
  } else {
    orbs = X.orbs;
    orbs.insert(orbs.end(), sorbs.begin(), sorbs.end());
  }
  make_keys(*E, orbs, right ? right_mode(b, c->k) : left_mode(b + 1, c->k), I.nso);
  layout_blocks(*E);
  alloc_zero(*E, c->st);
  E->mask.assign(E->bra.size(), 0);
  const Fused& F = *E->fused;
  auto terms = right ? blocking_terms(*E, sorbs, X.orbs, I) : blocking_terms(*E, X.orbs, sorbs, I);

  std::vector<GatherTask> tasks;
  std::vector<std::vector<GatherSrc>> tsrc;
  std::vector<std::vector<std::pair<int64_t, char>>> tsrc_off;   // template: source offsets
  std::unordered_map<const double*, int> task_of;
  std::vector<Ref> refs;
  for (size_t o = 0; o < E->keys.size(); ++o) {
    std::map<std::pair<int, int>, Mat4> acc;
    for (const Term& t : terms[o]) {
      refs.clear();
      Mat4 e4;
      if (right) {
        e4 = site.op(I, t.x.kind, t.x.p, t.x.q, t.x.t);
        get_refs(X, I, t.y.kind, t.y.p, t.y.q, t.y.t, t.c, refs);
      } else {
        get_refs(X, I, t.x.kind, t.x.p, t.x.q, t.x.t, t.c, refs);
        e4 = site.op(I, t.y.kind, t.y.p, t.y.q, t.y.t);
      }
      if (e4.zero()) continue;
      for (const Ref& r : refs) acc[{r.op, r.t}].axpy(r.c, e4);
    }
    for (auto& kv : acc) {
      const int j = kv.first.first, tr = kv.first.second;
      const Mat4& e4 = kv.second;
      if (e4.zero()) continue;
      const OpSet& XS = (tr && Xrev) ? *Xrev : X;
      for (int s = 0; s < X.ns(); ++s) {
        const int sb = X.bra_of(j, s);
        if (sb < 0 || !XS.block_nz(j, s)) continue;
        const int be = tr ? s : sb, ke = tr ? sb : s;
        const double* src = XS.d + X.off_of(j, s);
        const int ld = X.basis.d[s];
        for (int n1 = 0; n1 < 4; ++n1)
          for (int n0 = 0; n0 < 4; ++n0) {
            const double e = e4(n1, n0);
            if (e == 0.0) continue;
            int fk, fb, sign;
            if (right) {
              fk = F.s.find(X.basis.a[ke] - QNA[n0], X.basis.b[ke] - QNB[n0]);
              fb = F.s.find(X.basis.a[be] - QNA[n1], X.basis.b[be] - QNB[n1]);
              sign = (X.par[j] && ((QNA[n0] + QNB[n0]) & 1)) ? -1 : 1;
            } else {
              fk = F.s.find(X.basis.a[ke] + QNA[n0], X.basis.b[ke] + QNB[n0]);
              fb = F.s.find(X.basis.a[be] + QNA[n1], X.basis.b[be] + QNB[n1]);
              const int sp = (QNA[n1] + QNB[n1] + QNA[n0] + QNB[n0]) & 1;
              sign = (sp && ((X.basis.a[ke] + X.basis.b[ke]) & 1)) ? -1 : 1;
            }
            if (fk < 0 || fb < 0 || E->bra_of((int)o, fk) != fb)
              throw Error(LRT_EINVAL, "internal: blocking term outside the operator's sector");
            const int ldd = F.s.d[fk];
            double* dst = E->d + E->off_of((int)o, fk) + (int64_t)F.off[fb][n1] * ldd + F.off[fk][n0];
            auto it = task_of.find(dst);
            int ti;
            if (it == task_of.end()) {
              ti = (int)tasks.size();
              task_of[dst] = ti;
              tasks.push_back(GatherTask{dst, ldd, X.basis.d[be], X.basis.d[ke], 0, 0});
              tsrc.emplace_back();
            } else {
              ti = it->second;
            }
            tsrc[ti].push_back(GatherSrc{src, ld, tr, sign * e});
            if (tpl) {
              tsrc_off.resize(tsrc.size());
              tsrc_off[ti].push_back({src - XS.d, (tr && Xrev) ? 1 : 0});
            }
            E->mask[(size_t)o * E->ns() + fk] |= (uint16_t)(1u << (4 * n1 + n0));
            E->bnz[(size_t)o * E->ns() + fk] = 1;
          }
      }
    }
  }
  std::vector<GatherSrc> srcs;
  for (size_t i = 0; i < tasks.size(); ++i) {
    tasks[i].src_begin = (int)srcs.size();
    tasks[i].src_count = (int)tsrc[i].size();
    srcs.insert(srcs.end(), tsrc[i].begin(), tsrc[i].end());
  }
  E->finish_nz();
  if (tpl) {
    // the same task list with addresses relative to the launch's bases, kept on the device
    tpl->proto = layout_copy(*E);
    tsrc_off.resize(tsrc.size());
    std::vector<GatherSrc> rsrcs;
    rsrcs.reserve(srcs.size());
    for (size_t i = 0; i < tasks.size(); ++i) {
      tasks[i].dst_off = tasks[i].dst - E->d;
      tasks[i].dst = nullptr;
      for (size_t j = 0; j < tsrc[i].size(); ++j) {
        GatherSrc g = tsrc[i][j];
        g.src = nullptr;
        g.src_off = tsrc_off[i][j].first;
        g.rel = tsrc_off[i][j].second ? 2 : 1;
        rsrcs.push_back(g);
      }
    }
    tpl->gp = std::make_unique<GatherPlan>();
    build_gather(*tpl->gp, tasks, rsrcs, c->st);
    launch_gather(tpl->gp->tasks.p, tpl->gp->srcs.p, tpl->gp->tiles.p, tpl->gp->ntiles, c->st, E->d, X.d,
                  Xrev ? Xrev->d : nullptr);
    CK(cudaGetLastError());
    return E;
  }
  GatherPlan gp;
  build_gather(gp, tasks, srcs, c->st);
  gp.run(c->st);
  CK(cudaGetLastError());
  return E;
}

// an enlargement replayed from its template for new input data of the same layout: one
// launch of the template's device task list with the new sets as bases
static std::unique_ptr<OpSet> enlarge_from(lrt_ctx* c, const EnlTemplate& t, const OpSet& X, const OpSet* Xrev) {
  auto E = layout_copy(*t.proto);
  alloc_zero(*E, c->st);
  launch_gather(t.gp->tasks.p, t.gp->srcs.p, t.gp->tiles.p, t.gp->ntiles, c->st, E->d, X.d, Xrev ? Xrev->d : nullptr);
  CK(cudaGetLastError());
  return E;
}

static std::unique_ptr<OpSet> enlarge(lrt_ctx* c, int b, bool right) {
  return enlarge_set(c, right ? *c->R[b + 1] : *c->L[b], nullptr, b, right);
}

static OpSet& enlarged(lrt_ctx* c, int b, bool right) {
  auto& slot = right ? c->YR[b] : c->XL[b];
  if (!slot) {
    if (right && !c->R[b + 1]) throw Error(LRT_ESTATE, "right block of bond " + std::to_string(b + 1) + " not built");
    if (!right && !c->L[b]) throw Error(LRT_ESTATE, "left block of bond " + std::to_string(b) + " not built");
    slot = enlarge(c, b, right);
  }
  return *slot;
}

// One contribution bra^T [E] ket to a renormalized block: E is an enlarged operator
// set, bra and ket are site tensors (the zeroth-order isometry, or a first-order
// one for the second bracket of Eqs. lopr1st / ropr1st).
struct RenTerm {
  const OpSet* E;
  const SiteTensor* bra;
  const SiteTensor* ket;
};

// right-fused copy of a site tensor between bonds b and b+1 (per left sector q:
// D_q x fused(q), sub-blocks n side by side); returns the per-sector offsets
static std::vector<int64_t> rfused_copy(lrt_ctx* c, int b, const SiteTensor& T, DevBuf& buf, const Fused& F);

static void run_two_phase_tc(lrt_ctx* c, const std::vector<GemmOut>& o1, const std::vector<GemmSeg>& s1,
                             const std::vector<GemmOut>& o2, const std::vector<GemmSeg>& s2);

// A renormalization kept for replay: its two grouped GEMMs with every address relative to
// launch bases, so new operator data and isometries of the same layout (the first-order
// sets of every TDA sweep) cost one pair of launches and no host planning.  Bases: term
// t's enlarged set, ket and bra at extra bases 3t, 3t + 1, 3t + 2, the new block at
// REN_BASE_OUT, the intermediates at the launch's workspace.
struct RenTemplate {
  std::unique_ptr<OpSet> proto;
  std::unique_ptr<GemmPlan> p1, p2;
  int64_t toff = 0;
  uint64_t sig = 0;
};
constexpr int REN_MAX_TERMS = 2, REN_BASE_OUT = 6;
static_assert(REN_BASE_OUT < GEMM_NEXTRA && 3 * REN_MAX_TERMS <= REN_BASE_OUT, "renormalization bases");

static uint64_t site_signature(const SiteTensor& T) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  mix((uint64_t)T.total);
  for (int64_t o : T.blk_off) mix((uint64_t)o);
  for (int r : T.blk_rows) mix((uint64_t)r);
  return h;
}
static uint64_t ren_signature(int b, bool right, const std::vector<RenTerm>& terms) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  mix((uint64_t)b);
  mix(right ? 1u : 0u);
  for (const RenTerm& t : terms) {
    mix(set_signature(*t.E, nullptr));
    mix(site_signature(*t.ket));
    mix(site_signature(*t.bra));
  }
  return h;
}

// the plan lists with addresses made absolute (extra bases resolved) and the workspace
// left as offsets, the form the tensor-core two-phase path takes
static void ren_absolute(std::vector<GemmOut>& o1, std::vector<GemmSeg>& s1, std::vector<GemmOut>& o2,
                         std::vector<GemmSeg>& s2, const GemmExtra& ex) {
  auto segs = [&](std::vector<GemmSeg>& v) {
    for (GemmSeg& g : v) {
      if (g.a_rel >= 3) g.A = ex.p[g.a_rel - 3] + g.a_off, g.a_off = 0, g.a_rel = 0;
      if (g.b_rel >= 3) g.B = ex.p[g.b_rel - 3] + g.b_off, g.b_off = 0, g.b_rel = 0;
      if (g.b_rel == 2) g.b_rel = 0;
    }
  };
  auto outs = [&](std::vector<GemmOut>& v) {
    for (GemmOut& o : v) {
      if (o.c_rel >= 3) o.C = ex.p[o.c_rel - 3] + o.c_off, o.c_off = 0, o.c_rel = 0;
      if (o.c_rel == 2) o.c_rel = 0;
    }
  };
  segs(s1);
  segs(s2);
  outs(o1);
  outs(o2);
}

// runs (and, given a template slot, keeps) a renormalization's two grouped GEMMs
static void ren_run(lrt_ctx* c, std::vector<GemmOut>& o1, std::vector<GemmSeg>& s1, std::vector<GemmOut>& o2,
                    std::vector<GemmSeg>& s2, int64_t toff, const GemmExtra& ex, int prec, RenTemplate* tpl,
                    const OpSet& N, uint64_t sig) {
  if (prec == LRT_MIXED) {
    ren_absolute(o1, s1, o2, s2, ex);
    run_two_phase_tc(c, o1, s1, o2, s2);
    return;
  }
  auto p1 = std::make_unique<GemmPlan>(), p2 = std::make_unique<GemmPlan>();
  build_gemm(*p1, o1, s1, c->st);
  build_gemm(*p2, o2, s2, c->st);
  double* tmp = nullptr;
  if (toff > 0 && dev_alloc((void**)&tmp, (size_t)toff * sizeof(double)) != cudaSuccess)
    throw Error(LRT_ENOMEM, "renormalize workspace");
  launch_gemm_fp64(p1->outs.p, p1->segs.p, p1->tiles.p, p1->ntiles, nullptr, nullptr, tmp, c->st, &ex);
  launch_gemm_fp64(p2->outs.p, p2->segs.p, p2->tiles.p, p2->ntiles, nullptr, nullptr, tmp, c->st, &ex);
  CK(cudaGetLastError());
  if (tmp) dev_free(tmp);
  if (tpl) {
    tpl->proto = layout_copy(N);
    tpl->p1 = std::move(p1);
    tpl->p2 = std::move(p2);
    tpl->toff = toff;
    tpl->sig = sig;
  }
}

// replay of a kept renormalization; false when the template does not match
static std::unique_ptr<OpSet> ren_replay(lrt_ctx* c, RenTemplate* tpl, uint64_t sig, GemmExtra ex, int prec) {
  if (!tpl || prec != LRT_FP64 || !tpl->p1 || tpl->sig != sig) return nullptr;
  auto N = layout_copy(*tpl->proto);
  alloc_zero(*N, c->st);
  ex.p[REN_BASE_OUT] = N->d;
  double* tmp = nullptr;
  if (tpl->toff > 0 && dev_alloc((void**)&tmp, (size_t)tpl->toff * sizeof(double)) != cudaSuccess)
    throw Error(LRT_ENOMEM, "renormalize workspace");
  const GemmPlan& p1 = *tpl->p1;
  const GemmPlan& p2 = *tpl->p2;
  launch_gemm_fp64(p1.outs.p, p1.segs.p, p1.tiles.p, p1.ntiles, nullptr, nullptr, tmp, c->st, &ex);
  launch_gemm_fp64(p2.outs.p, p2.segs.p, p2.tiles.p, p2.ntiles, nullptr, nullptr, tmp, c->st, &ex);
  CK(cudaGetLastError());
  if (tmp) dev_free(tmp);
  return N;
}

// left block of bond b+1 = sum_t bra_t^T E_t ket_t over the enlarged left block of bond b
// (prec LRT_MIXED: the two grouped GEMMs as split-TF32 tensor-core products)
static std::unique_ptr<OpSet> renorm_left_terms(lrt_ctx* c, int b, const std::vector<RenTerm>& terms,
                                                int prec = LRT_FP64, RenTemplate* tpl = nullptr) {
  if (terms.empty() || (int)terms.size() > REN_MAX_TERMS) throw Error(LRT_EINVAL, "renormalize: 1 or 2 terms");
  GemmExtra ex{};
  for (size_t t = 0; t < terms.size(); ++t) {
    ex.p[3 * t] = terms[t].E->d;
    ex.p[3 * t + 1] = terms[t].ket->d;
    ex.p[3 * t + 2] = terms[t].bra->d;
  }
  const uint64_t sig = tpl ? ren_signature(b, false, terms) : 0;
  if (auto R = ren_replay(c, tpl, sig, ex, prec)) return R;
  const OpSet& E0 = *terms[0].E;
  const Fused& F = *E0.fused;
  auto N = std::make_unique<OpSet>();
  N->right = false;
  N->basis = c->bonds[b + 1];
  make_keys(*N, E0.orbs, E0.mode, c->I.nso);
  layout_blocks(*N);
  alloc_zero(*N, c->st);
  ex.p[REN_BASE_OUT] = N->d;
  std::vector<GemmOut> o1, o2;
  std::vector<GemmSeg> s1, s2;
  int64_t toff = 0;
  for (size_t o = 0; o < N->keys.size(); ++o)
    for (int q = 0; q < N->ns(); ++q) {
      const int qb = N->bra_of((int)o, q);
      if (qb < 0) continue;
      const int fk = F.s.find(N->basis.a[q], N->basis.b[q]);
      const int fb = F.s.find(N->basis.a[qb], N->basis.b[qb]);
      if (fk < 0 || fb < 0) continue;
      const int Dq = N->basis.d[q], Dqb = N->basis.d[qb];
      const int rk = F.s.d[fk], rb = F.s.d[fb];
      GemmOut out{nullptr, N->off_of((int)o, q), Dq, Dqb, Dq, (int)s2.size(), 0, 0, 3 + REN_BASE_OUT};
      for (size_t ti = 0; ti < terms.size(); ++ti) {
        const RenTerm& t = terms[ti];
        const OpSet& E = *t.E;
        if (E.bra_of((int)o, fk) != fb || !E.block_nz((int)o, fk)) continue;
        const SiteTensor& K = *t.ket;
        const SiteTensor& Bt = *t.bra;
        if (K.blk_off[q] < 0 || Bt.blk_off[qb] < 0) continue;
        if (K.blk_rows[q] != rk || Bt.blk_rows[qb] != rb)
          throw Error(LRT_EINVAL, "site tensor rows do not match the enlarged basis");
        const int r0 = 3 + 3 * (int)ti;
        o1.push_back(GemmOut{nullptr, toff, Dq, rb, Dq, (int)s1.size(), 1, 0, 2});
        s1.push_back(GemmSeg{nullptr, nullptr, E.off_of((int)o, fk), K.blk_off[q], rk, Dq, rk, 0, 0, r0, r0 + 1, 1.0});
        s2.push_back(GemmSeg{nullptr, nullptr, Bt.blk_off[qb], toff, Dqb, Dq, rb, 1, 0, r0 + 2, 2, 1.0});
        ++out.seg_count;
        toff += (int64_t)rb * Dq;
      }
      if (out.seg_count > 0) {
        o2.push_back(out);
        N->bnz[o * N->ns() + q] = 1;
      }
    }
  N->finish_nz();
  ren_run(c, o1, s1, o2, s2, toff, ex, prec, tpl, *N, sig);
  return N;
}

// right block of bond b = sum_t R_bra,t [E_t] R_ket,t^T over the enlarged right block site b (+) R
static std::unique_ptr<OpSet> renorm_right_terms(lrt_ctx* c, int b, const std::vector<RenTerm>& terms,
                                                 int prec = LRT_FP64, RenTemplate* tpl = nullptr) {
  if (terms.empty() || (int)terms.size() > REN_MAX_TERMS) throw Error(LRT_EINVAL, "renormalize: 1 or 2 terms");
  const OpSet& E0 = *terms[0].E;
  const Fused& F = *E0.fused;
  const Sectors& Lb = c->bonds[b];
  // right-fused copies of every distinct site tensor
  std::map<const SiteTensor*, std::pair<std::unique_ptr<DevBuf>, std::vector<int64_t>>> rf;
  for (const RenTerm& t : terms)
    for (const SiteTensor* T : {t.bra, t.ket})
      if (!rf.count(T)) {
        auto buf = std::make_unique<DevBuf>();
        auto off = rfused_copy(c, b, *T, *buf, F);
        rf[T] = {std::move(buf), std::move(off)};
      }
  GemmExtra ex{};
  for (size_t t = 0; t < terms.size(); ++t) {
    ex.p[3 * t] = terms[t].E->d;
    ex.p[3 * t + 1] = rf.at(terms[t].ket).first->p;
    ex.p[3 * t + 2] = rf.at(terms[t].bra).first->p;
  }
  const uint64_t sig = tpl ? ren_signature(b, true, terms) : 0;
  if (auto R = ren_replay(c, tpl, sig, ex, prec)) return R;
  auto N = std::make_unique<OpSet>();
  N->right = true;
  N->basis = Lb;
  make_keys(*N, E0.orbs, E0.mode, c->I.nso);
  layout_blocks(*N);
  alloc_zero(*N, c->st);
  ex.p[REN_BASE_OUT] = N->d;
  std::vector<GemmOut> o1, o2;
  std::vector<GemmSeg> s1, s2;
  int64_t toff = 0;
  for (size_t o = 0; o < N->keys.size(); ++o)
    for (int q = 0; q < N->ns(); ++q) {
      const int qb = N->bra_of((int)o, q);
      if (qb < 0) continue;
      const int fk = F.s.find(Lb.a[q], Lb.b[q]);
      const int fb = F.s.find(Lb.a[qb], Lb.b[qb]);
      if (fk < 0 || fb < 0) continue;
      const int Dq = Lb.d[q], Dqb = Lb.d[qb];
      const int ck = F.s.d[fk], cb = F.s.d[fb];
      GemmOut out{nullptr, N->off_of((int)o, q), Dq, Dqb, Dq, (int)s2.size(), 0, 0, 3 + REN_BASE_OUT};
      for (size_t ti = 0; ti < terms.size(); ++ti) {
        const RenTerm& t = terms[ti];
        const OpSet& E = *t.E;
        if (E.bra_of((int)o, fk) != fb || !E.block_nz((int)o, fk)) continue;
        const auto& K = rf.at(t.ket);
        const auto& Bt = rf.at(t.bra);
        if (K.second[q] < 0 || Bt.second[qb] < 0) continue;
        const int r0 = 3 + 3 * (int)ti;
        o1.push_back(GemmOut{nullptr, toff, Dq, cb, Dq, (int)s1.size(), 1, 0, 2});
        s1.push_back(GemmSeg{nullptr, nullptr, E.off_of((int)o, fk), K.second[q], ck, ck, ck, 0, 1, r0, r0 + 1, 1.0});
        s2.push_back(GemmSeg{nullptr, nullptr, Bt.second[qb], toff, cb, Dq, cb, 0, 0, r0 + 2, 2, 1.0});
        ++out.seg_count;
        toff += (int64_t)cb * Dq;
      }
      if (out.seg_count > 0) {
        o2.push_back(out);
        N->bnz[o * N->ns() + q] = 1;
      }
    }
  N->finish_nz();
  ren_run(c, o1, s1, o2, s2, toff, ex, prec, tpl, *N, sig);
  return N;
}

static void renorm_left(lrt_ctx* c, int b, int prec = LRT_FP64) {
  OpSet& E = enlarged(c, b, false);
  c->L[b + 1] = renorm_left_terms(c, b, {RenTerm{&E, &c->sites[b], &c->sites[b]}}, prec);
  for (int x = b + 2; x <= c->k; ++x) c->L[x].reset();
  for (int x = b + 1; x < c->k; ++x) c->XL[x].reset();
  drop_plans(c);
}

static void renorm_right(lrt_ctx* c, int b, int prec = LRT_FP64) {
  OpSet& E = enlarged(c, b, true);
  const SiteTensor& T = c->sites_r.empty() ? c->sites[b] : c->sites_r[b];
  c->R[b] = renorm_right_terms(c, b, {RenTerm{&E, &T, &T}}, prec);
  for (int x = 0; x < b; ++x) c->R[x].reset();
  for (int x = 0; x < b; ++x) c->YR[x].reset();
  drop_plans(c);
}

// ---------------------------------------------------------------------------
// wavefunction layouts
// ---------------------------------------------------------------------------
struct WfnBlock {
  int label_a, label_b;
  int rows, cols;
  int64_t off;
};

static std::vector<WfnBlock> wfn_blocks(lrt_ctx* c, int site, int nsite) {
  std::vector<WfnBlock> out;
  int64_t off = 0;
  if (nsite == 1) {
    const SiteTensor& T = c->sites[site];
    const Sectors& R = c->bonds[site + 1];
    for (int r = 0; r < R.n(); ++r) {
      if (T.blk_rows[r] == 0) continue;
      out.push_back(WfnBlock{R.a[r], R.b[r], T.blk_rows[r], R.d[r], off});
      off += (int64_t)T.blk_rows[r] * R.d[r];
    }
    return out;
  }
  const Fused fl = fuse(c->bonds[site], false);
  const Fused fr = fuse(c->bonds[site + 2], true);
  for (int m = 0; m < fl.s.n(); ++m) {
    const int j = fr.s.find(fl.s.a[m], fl.s.b[m]);
    if (j < 0) continue;
    out.push_back(WfnBlock{fl.s.a[m], fl.s.b[m], fl.s.d[m], fr.s.d[j], off});
    off += (int64_t)fl.s.d[m] * fr.s.d[j];
  }
  return out;
}

// ---------------------------------------------------------------------------
// sigma planning: y = sum_terms coef * sign * X_t psi Y_t^T
// ---------------------------------------------------------------------------
static uint16_t transpose_mask(uint16_t m) {
  uint16_t r = 0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      if (m & (1u << (4 * a + b))) r |= (uint16_t)(1u << (4 * b + a));
  return r;
}

// Products are formed at sub-block granularity so that zero sub-blocks of the
// enlarged operators are never multiplied:
//   phase 1: T[t](rows n') = sum_{n : X_t(n',n) != 0} X_t(n',n) psi_Q(rows n)
//   phase 2: y_Q'(rows n' [, cols m']) = sum_t sign_t T[t](rows n' [, cols m]) Y_t(m',m)^T
// X: enlarged left block (L (+) site `site`); Y: the right block of bond site+1
// (nsite 1) or the enlarged right block site+1 (+) R (nsite 2).  Xrev / Yrev: reverse
// sets of first-order (transition) operator sets, read by transposed references.
static std::unique_ptr<SigmaPlan> plan_sigma_sets(lrt_ctx* c, const OpSet& X, const OpSet* Xrev, const OpSet& Y,
                                                  const OpSet* Yrev, int site, int nsite, int nvec, bool tc = true,
                                                  bool rel_ops = false) {
  if (rel_ops && tc) throw Error(LRT_EINVAL, "internal: relative operator addresses are FP64 only");
  const Ints& I = c->I;
  const int k = c->k;
  const Fused& XF = *X.fused;
  const Fused* YF = (nsite == 2) ? Y.fused.get() : nullptr;
  const std::vector<WfnBlock> wb = wfn_blocks(c, site, nsite);
  std::unordered_map<int, int> blk_of;   // label key -> wfn block
  for (size_t i = 0; i < wb.size(); ++i) blk_of[Sectors::key(wb[i].label_a, wb[i].label_b)] = (int)i;
  int64_t nelem = 0;
  for (auto& w : wb) nelem = std::max(nelem, w.off + (int64_t)w.rows * w.cols);

  std::vector<Term> terms;
  terms.push_back({1.0, {KH, -1, -1, 0}, {KI, -1, -1, 0}});
  terms.push_back({1.0, {KI, -1, -1, 0}, {KH, -1, -1, 0}});
  cross_terms(X.orbs, Y.orbs, 2 * (site + 1) <= k, terms);
  if (I.e_core != 0.0) terms.push_back({I.e_core, {KI, -1, -1, 0}, {KI, -1, -1, 0}});

  auto plan = std::make_unique<SigmaPlan>();
  static std::atomic<uint64_t> next_serial{0};   // plans are built from several threads in sweep_tda_batched
  plan->serial = ++next_serial;
  plan->nelem = nelem;
  plan->n_terms = (int)terms.size();

  // every sub-block of y is an output (written even when no product reaches it)
  struct OutSub { int blk, r, mcol; };
  std::vector<OutSub> osub;
  std::map<std::tuple<int, int, int>, int> out_of;
  for (size_t w = 0; w < wb.size(); ++w) {
    const int fx = XF.s.find(wb[w].label_a, wb[w].label_b);
    for (int r = 0; r < 4; ++r) {
      if (XF.dim[fx][r] == 0) continue;
      if (nsite == 1) {
        out_of[{(int)w, r, 0}] = (int)osub.size();
        osub.push_back({(int)w, r, 0});
      } else {
        const int fy = YF->s.find(wb[w].label_a, wb[w].label_b);
        for (int m = 0; m < 4; ++m) {
          if (YF->dim[fy][m] == 0) continue;
          out_of[{(int)w, r, m}] = (int)osub.size();
          osub.push_back({(int)w, r, m});
        }
      }
    }
  }
  std::vector<std::vector<GemmSeg>> seg2(osub.size());
  std::vector<std::vector<const OpSet*>> seg2set(osub.size());
  std::vector<GemmOut> o1;
  std::vector<GemmSeg> s1;
  std::vector<const OpSet*> s1set;
  // Tensor-core twin: whole fused blocks instead of 4 x 4 sub-blocks (structurally
  // zero sub-blocks are stored zeros), so that the products fill the 128-row tiles.
  // Phase 1: per T block and right column group m, T_m = op(O_X) x_m; phase 2: per
  // (y block, column group), sum of T_m (or x_m) times the Y sub-matrix.
  TcPlan& tcp = plan->tc;
  std::map<std::tuple<int, int, int>, std::array<int, 4>> tc_T;   // T key -> TC matrix per m
  std::map<std::pair<int, int>, std::vector<TcPlanSeg>> tc_y;     // (y block, column group) -> products
  struct TEntry { int64_t tp; uint16_t rows; };
  std::map<std::tuple<int, int, int>, TEntry> tcache;   // (X op, trans, X ket fused) -> T
  int64_t toff = 0;
  std::vector<std::vector<DiagTerm>> dterm(wb.size());
  std::vector<Ref> rx, ry;
  double op_bytes = 0.0, falg = 0.0;
  int nprod = 0;
  // The identity of a zeroth-order enlarged block is the unit matrix (orthonormal
  // basis), so its products use psi directly; the identity of a first-order set is the
  // transition overlap <l0|l1> and is multiplied like any other operator.
  const int Ikey = Xrev ? -1 : X.find(Key{KI, -1, -1});

  for (const Term& t : terms) {
    rx.clear();
    ry.clear();
    get_refs(X, I, t.x.kind, t.x.p, t.x.q, t.x.t, 1.0, rx);
    get_refs(Y, I, t.y.kind, t.y.p, t.y.q, t.y.t, 1.0, ry);
    for (const Ref& a : rx)
      for (const Ref& bref : ry) {
        const double coef = t.c * a.c * bref.c;
        const OpSet& XS = (a.t && Xrev) ? *Xrev : X;
        const OpSet& YS = (bref.t && Yrev) ? *Yrev : Y;
        for (int f = 0; f < X.ns(); ++f) {
          const int fb0 = X.bra_of(a.op, f);
          if (fb0 < 0 || !XS.block_nz(a.op, f)) continue;
          const int be = a.t ? f : fb0, ke = a.t ? fb0 : f;
          auto ik = blk_of.find(Sectors::key(X.basis.a[ke], X.basis.b[ke]));
          auto ib = blk_of.find(Sectors::key(X.basis.a[be], X.basis.b[be]));
          if (ik == blk_of.end() || ib == blk_of.end()) continue;
          const WfnBlock& wk = wb[ik->second];
          const WfnBlock& wbb = wb[ib->second];
          const int yk = Y.basis.find(wk.label_a, wk.label_b);
          const int ybb = Y.basis.find(wbb.label_a, wbb.label_b);
          if (yk < 0 || ybb < 0) continue;
          const double* Bp;
          int transB, ldb;
          uint16_t ymask = 1;   // stored blocks: one dense sub-block
          if (!bref.t) {
            if (Y.bra_of(bref.op, yk) != ybb || !YS.block_nz(bref.op, yk)) continue;
            Bp = YS.d + Y.off_of(bref.op, yk);
            transB = 1;
            ldb = Y.basis.d[yk];
            if (YF) ymask = YS.mask[(size_t)bref.op * Y.ns() + yk];
          } else {
            if (Y.bra_of(bref.op, ybb) != yk || !YS.block_nz(bref.op, ybb)) continue;
            Bp = YS.d + Y.off_of(bref.op, ybb);
            transB = 0;
            ldb = Y.basis.d[ybb];
            if (YF) ymask = transpose_mask(YS.mask[(size_t)bref.op * Y.ns() + ybb]);
          }
          const int sign = (Y.par[bref.op] && ((wk.label_a + wk.label_b) & 1)) ? -1 : 1;
          const double sc = coef * sign;
          ++nprod;
          op_bytes += 8.0 * ((double)Y.basis.d[yk] * Y.basis.d[ybb]);

          // ---- phase 1 (shared by every Y partner of this X block)
          uint16_t rows = 0;
          int64_t tp = -1;
          const bool ident = (a.op == Ikey);
          if (ident) {
            for (int r = 0; r < 4; ++r)
              if (XF.dim[be][r]) rows |= (uint16_t)(1u << r);
          } else {
            const auto key = std::make_tuple(a.op, a.t, f);
            auto it = tcache.find(key);
            if (it == tcache.end()) {
              uint16_t mx = XS.mask[(size_t)a.op * X.ns() + f];
              if (a.t) mx = transpose_mask(mx);
              tp = toff;
              toff += (int64_t)wbb.rows * wk.cols;
              const double* base = XS.d + X.off_of(a.op, f);
              const int ld = X.basis.d[f];
              op_bytes += 8.0 * ((double)wbb.rows * wk.rows);
              for (int r = 0; r < 4; ++r) {
                bool any = false;
                for (int cc = 0; cc < 4; ++cc)
                  if (mx & (1u << (4 * r + cc))) any = true;
                if (!any) continue;
                rows |= (uint16_t)(1u << r);
                GemmOut out{nullptr, tp + (int64_t)XF.off[be][r] * wk.cols, wk.cols, XF.dim[be][r], wk.cols,
                            (int)s1.size(), 0, 0, 0};
                for (int cc = 0; cc < 4; ++cc) {
                  if (!(mx & (1u << (4 * r + cc)))) continue;
                  GemmSeg g{};
                  if (!a.t) {
                    g.A = base + (int64_t)XF.off[be][r] * ld + XF.off[ke][cc];
                    g.transA = 0;
                  } else {
                    g.A = base + (int64_t)XF.off[ke][cc] * ld + XF.off[be][r];
                    g.transA = 1;
                  }
                  g.lda = ld;
                  g.b_rel = 1;
                  g.b_off = wk.off + (int64_t)XF.off[ke][cc] * wk.cols;
                  g.ldb = wk.cols;
                  g.k = XF.dim[ke][cc];
                  g.scale = 1.0;
                  s1.push_back(g);
                  s1set.push_back(&XS);
                  ++out.seg_count;
                  falg += 2.0 * XF.dim[be][r] * XF.dim[ke][cc] * wk.cols;
                }
                o1.push_back(out);
              }
              if (tc && rows) {
                const int A = tcp.op(base, ld, a.t ? 1 : 0, wbb.rows, wk.rows);
                std::array<int, 4> tm{-1, -1, -1, -1};
                for (int m = 0; m < (nsite == 1 ? 1 : 4); ++m) {
                  const int dim = nsite == 1 ? wk.cols : YF->dim[yk][m];
                  const int64_t coff = nsite == 1 ? 0 : YF->off[yk][m];
                  if (dim == 0) continue;
                  const int B = tcp.x(wk.off + coff, wk.cols, 1, dim, wk.rows);
                  tm[m] = tcp.add(2, wbb.rows, dim);
                  tcp.out1.push_back(TcPlanOut{tm[m], 0, 0, wbb.rows, dim, (int)tcp.segs.size(), 1});
                  tcp.segs.push_back(TcPlanSeg{A, B, wk.rows, 1.0f});
                }
                tc_T[key] = tm;
              }
              tcache[key] = TEntry{tp, rows};
            } else {
              tp = it->second.tp;
              rows = it->second.rows;
            }
          }
          // ---- phase 2
          for (int r = 0; r < 4; ++r) {
            if (!(rows & (1u << r))) continue;
            const int64_t arow = ident ? wk.off + (int64_t)XF.off[ke][r] * wk.cols
                                       : tp + (int64_t)XF.off[be][r] * wk.cols;
            if (nsite == 1) {
              GemmSeg g{};
              g.a_rel = ident ? 1 : 0;
              g.a_off = arow;
              g.lda = wk.cols;
              g.B = Bp;
              g.ldb = ldb;
              g.transB = transB;
              g.k = wk.cols;
              g.scale = sc;
              seg2[out_of.at({ib->second, r, 0})].push_back(g);
              seg2set[out_of.at({ib->second, r, 0})].push_back(&YS);
              falg += 2.0 * XF.dim[be][r] * wk.cols * wbb.cols;
            } else {
              for (int mp = 0; mp < 4; ++mp)
                for (int m = 0; m < 4; ++m) {
                  if (!(ymask & (1u << (4 * mp + m)))) continue;
                  GemmSeg g{};
                  g.a_rel = ident ? 1 : 0;
                  g.a_off = arow + YF->off[yk][m];
                  g.lda = wk.cols;
                  if (!bref.t) g.B = Bp + (int64_t)YF->off[ybb][mp] * ldb + YF->off[yk][m];
                  else g.B = Bp + (int64_t)YF->off[yk][m] * ldb + YF->off[ybb][mp];
                  g.ldb = ldb;
                  g.transB = transB;
                  g.k = YF->dim[yk][m];
                  g.scale = sc;
                  seg2[out_of.at({ib->second, r, mp})].push_back(g);
                  seg2set[out_of.at({ib->second, r, mp})].push_back(&YS);
                  falg += 2.0 * XF.dim[be][r] * YF->dim[yk][m] * YF->dim[ybb][mp];
                }
            }
          }
          if (tc && rows) {
            const std::array<int, 4>* tm = ident ? nullptr : &tc_T.at(std::make_tuple(a.op, a.t, f));
            if (nsite == 1) {
              const int A = ident ? tcp.x(wk.off, wk.cols, 0, wk.rows, wk.cols) : (*tm)[0];
              const int B = tcp.op(Bp, ldb, bref.t ? 1 : 0, Y.basis.d[ybb], Y.basis.d[yk]);
              tc_y[{ib->second, 0}].push_back(TcPlanSeg{A, B, wk.cols, (float)sc});
            } else {
              for (int mp = 0; mp < 4; ++mp)
                for (int m = 0; m < 4; ++m) {
                  if (!(ymask & (1u << (4 * mp + m)))) continue;
                  const int A = ident ? tcp.x(wk.off + YF->off[yk][m], wk.cols, 0, wk.rows, YF->dim[yk][m]) : (*tm)[m];
                  if (A < 0) throw Error(LRT_EINVAL, "tensor-core plan: missing intermediate");
                  const double* src = !bref.t ? Bp + (int64_t)YF->off[ybb][mp] * ldb + YF->off[yk][m]
                                              : Bp + (int64_t)YF->off[yk][m] * ldb + YF->off[ybb][mp];
                  const int B = tcp.op(src, ldb, bref.t ? 1 : 0, YF->dim[ybb][mp], YF->dim[yk][m]);
                  tc_y[{ib->second, mp}].push_back(TcPlanSeg{A, B, YF->dim[yk][m], (float)sc});
                }
            }
          }
          // ---- diagonal contribution
          if (be == ke && yk == ybb) {
            DiagTerm d{};
            d.x = ident ? nullptr : XS.d + X.off_of(a.op, f);
            d.xs = X.basis.d[f] + 1;
            d.y = Bp;
            d.ys = Y.basis.d[yk] + 1;
            d.scale = sc;
            dterm[ik->second].push_back(d);
          }
        }
      }
  }
  if (toff > 0 && dev_alloc((void**)&plan->tbuf, (size_t)toff * nvec * sizeof(double)) != cudaSuccess)
    throw Error(LRT_ENOMEM, "sigma workspace");
  std::vector<GemmOut> O1, O2;
  std::vector<GemmSeg> S1, S2;
  plan->tsize = toff * nvec;
  // operator pointers as offsets from the set they live in (extra bases 0..3)
  auto set_rel = [&](const OpSet* S) { return S == &X ? 3 : S == Xrev ? 4 : S == &Y ? 5 : 6; };
  if (rel_ops) {
    plan->ex.p[0] = X.d;
    plan->ex.p[1] = Xrev ? Xrev->d : nullptr;
    plan->ex.p[2] = Y.d;
    plan->ex.p[3] = Yrev ? Yrev->d : nullptr;
    for (size_t q = 0; q < s1.size(); ++q) {
      s1[q].a_off = s1[q].A - s1set[q]->d;
      s1[q].A = nullptr;
      s1[q].a_rel = set_rel(s1set[q]);
    }
    for (size_t u = 0; u < seg2.size(); ++u)
      for (size_t q = 0; q < seg2[u].size(); ++q) {
        GemmSeg& g = seg2[u][q];
        g.b_off = g.B - seg2set[u][q]->d;
        g.B = nullptr;
        g.b_rel = set_rel(seg2set[u][q]);
      }
  }
  // The vectors of a call share every operator block: phase 1 (T = X x) places them side by
  // side along the columns of one output (x's block of vector v at + v * nelem, T of vector v
  // at + v * toff), phase 2 (y = sum T Y^T) stacks them along the rows (the T or x rows of
  // vector v at + v * toff or + v * nelem, y of vector v at + v * nelem).  One output then
  // holds the same block product for every vector, which fills the GEMM's tiles.
  const bool vb = nvec > 1;
  for (const GemmOut& x : o1) {
    GemmOut y = x;
    y.C = nullptr;
    y.c_rel = 2;
    y.seg_begin = (int)S1.size();
    if (vb) {
      y.n = x.n * nvec;
      y.c_vc = x.n;
      y.c_vs = toff;
    }
    for (int q = 0; q < x.seg_count; ++q) {
      GemmSeg g = s1[x.seg_begin + q];
      if (vb) {
        g.b_vc = x.n;
        g.b_vs = nelem;
      }
      S1.push_back(g);
    }
    O1.push_back(y);
  }
  for (size_t u = 0; u < osub.size(); ++u) {
    const OutSub& os = osub[u];
    const WfnBlock& w = wb[os.blk];
    const int fx = XF.s.find(w.label_a, w.label_b);
    int64_t coff = w.off + (int64_t)XF.off[fx][os.r] * w.cols;
    int ncols = w.cols;
    if (nsite == 2) {
      const int fy = YF->s.find(w.label_a, w.label_b);
      coff += YF->off[fy][os.mcol];
      ncols = YF->dim[fy][os.mcol];
    }
    const int m1 = XF.dim[fx][os.r];
    GemmOut y{nullptr, coff, w.cols, m1 * nvec, ncols, (int)S2.size(), (int)seg2[u].size(), 0, 1};
    if (vb) {
      y.c_vr = m1;
      y.c_vs = nelem;
    }
    for (size_t q = 0; q < seg2[u].size(); ++q) {
      GemmSeg g = seg2[u][q];
      const int64_t vs = g.a_rel ? nelem : toff;
      if (!g.a_rel) g.a_rel = 2;
      if (vb) {
        g.a_vr = m1;
        g.a_vs = vs;
      }
      S2.push_back(g);
    }
    O2.push_back(y);
  }
  build_gemm(plan->p1, O1, S1, c->st);
  build_gemm(plan->p2, O2, S2, c->st, !rel_ops);   // kept relative plans are replayed over instances
  // tensor-core twin: phase-2 outputs, one per (y block, column group)
  plan->has_tc = tc;
  for (size_t w = 0; w < wb.size() && tc; ++w)
    for (int m = 0; m < (nsite == 1 ? 1 : 4); ++m) {
      const WfnBlock& wbk = wb[w];
      int64_t coff = wbk.off;
      int ncols = wbk.cols;
      if (nsite == 2) {
        const int fy = YF->s.find(wbk.label_a, wbk.label_b);
        if (YF->dim[fy][m] == 0) continue;
        coff += YF->off[fy][m];
        ncols = YF->dim[fy][m];
      }
      auto it = tc_y.find({(int)w, m});
      const int sb = (int)tcp.segs.size();
      if (it != tc_y.end()) tcp.segs.insert(tcp.segs.end(), it->second.begin(), it->second.end());
      tcp.out2.push_back(TcPlanOut{-1, coff, wbk.cols, wbk.rows, ncols, sb, (int)tcp.segs.size() - sb});
    }
  std::vector<DiagOut> dout;
  std::vector<DiagTerm> dts;
  for (size_t w = 0; w < wb.size(); ++w) {
    dout.push_back(DiagOut{wb[w].off, wb[w].rows, wb[w].cols, (int)dts.size(), (int)dterm[w].size()});
    dts.insert(dts.end(), dterm[w].begin(), dterm[w].end());
  }
  plan->douts.upload(dout, c->st);
  plan->dterms.upload(dts, c->st);
  plan->ndiag = (int)dout.size();
  plan->n_products = nprod;
  plan->op_bytes = op_bytes;
  plan->flops_alg = falg * nvec;
  CK(cudaStreamSynchronize(c->st));
  return plan;
}

static std::unique_ptr<SigmaPlan> plan_sigma(lrt_ctx* c, int site, int nsite, int nvec, bool tc) {
  OpSet& X = enlarged(c, site, false);
  OpSet* Yp;
  if (nsite == 1) {
    if (!c->R[site + 1]) throw Error(LRT_ESTATE, "right block of bond " + std::to_string(site + 1) + " not built");
    Yp = c->R[site + 1].get();
  } else {
    Yp = &enlarged(c, site + 1, true);
  }
  return plan_sigma_sets(c, X, nullptr, *Yp, nullptr, site, nsite, nvec, tc);
}

// Work stream of one tensor-core launch over one or several plans (instances): tiles
// of 128 x 64 of every output, vector and instance in longest-first order, CTA b takes
// the tiles b, b + n, b + 2n, ...; each tile is a header followed by its block products
// with TC-matrix operands resolved.
struct TcSource {
  const TcPlan* tp;
  const std::vector<TcPlanOut>* outs;
  float* const* phi;
  float* const* plo;
  int64_t nelem;
  int inst;
};
static void build_tc_stream(const std::vector<TcSource>& src, int nvec, int TN, DevArray<TcItem>& items,
                            DevArray<int>& begins, int& nctas, cudaStream_t st) {
  const int TM = tc_tile_m();
  // Stacking: single-product outputs into intermediates (phase 1) that share their B
  // operand, K and width have their last (partial) 128-row block packed with others into
  // one tile, rows rounded up to 8 (first fit, decreasing).
  // Vector slots: when such a product is narrow (its B matrix, one vector's block of x,
  // has at most half a tile of rows), the tile's columns hold the same product for
  // several vectors, each slot all of one vector's B rows.  Such outputs are stacked once
  // for all vectors, full 128-row blocks as single pieces.
  // Row slots: an FP64 output of at most half a tile of rows whose A operands are all
  // per-vector matrices of its own (padded) height and whose B operands are shared
  // operator blocks takes several vectors in the tile's rows (c_rel 5).
  struct Piece { int o, row0, nrows, srow; };
  struct Stack { int s, v, n, k, b; std::vector<Piece> pc; int nv = 0, wv = 0; };   // nv > 0: vector slots
  std::vector<Stack> stacks;
  struct Tile { int s, v, o, a, b; int64_t k; int stack; int rs; };   // rs > 0: vectors v .. v + rs - 1 in row slots
  std::vector<Tile> tiles;
  // vectors per row-slot tile: at most a tile's rows, fewer when that would leave too few
  // tiles to spread over the SMs (at least two per CTA)
  auto row_slots = [&](const TcPlan& tp, const TcPlanOut& o) -> int {
    if (nvec < 2 || o.tmat >= 0 || o.C || o.seg_count < 1) return 0;
    const int Rp = (o.m + 7) & ~7;
    if (2 * Rp > TM) return 0;
    for (int q = 0; q < o.seg_count; ++q) {
      const TcPlanSeg& g = tp.segs[o.seg_begin + q];
      const TcMat& A = tp.mats[g.a];
      const TcMat& B = tp.mats[g.b];
      if (A.pool == 0 || B.pool != 0 || A.Rp != Rp) return 0;
    }
    return std::min(TM / Rp, nvec);
  };
  int64_t rs_products = 0;
  for (const TcSource& sc : src)
    for (const TcPlanOut& o : *sc.outs)
      if (row_slots(*sc.tp, o)) rs_products += (int64_t)nvec * ((o.n + TN - 1) / TN);
  const int rs_cap = (int)std::max<int64_t>(1, rs_products / (2 * (int64_t)tc_num_ctas(1 << 30)));
  auto pack = [&](std::map<std::tuple<int, int, int>, std::vector<Piece>>& groups, int si, int v,
                  std::vector<Stack>& out) {
    for (auto& kv : groups) {
      std::vector<Piece>& pcs = kv.second;
      std::stable_sort(pcs.begin(), pcs.end(), [](const Piece& x, const Piece& y) { return x.nrows > y.nrows; });
      std::vector<Stack> bins;
      std::vector<int> used;
      for (const Piece& pc : pcs) {
        size_t j = 0;
        for (; j < bins.size(); ++j)
          if (used[j] + pc.nrows <= TM && (int)bins[j].pc.size() < TC_MAX_PIECES) break;
        if (j == bins.size()) {
          bins.push_back(Stack{si, v, std::get<1>(kv.first), std::get<2>(kv.first), std::get<0>(kv.first), {}});
          used.push_back(0);
        }
        Piece q = pc;
        q.srow = used[j];
        used[j] += pc.nrows;
        bins[j].pc.push_back(q);
      }
      for (Stack& b : bins) out.push_back(std::move(b));
    }
  };
  for (size_t si = 0; si < src.size(); ++si) {
    const TcPlan& tp = *src[si].tp;
    const std::vector<TcPlanOut>& outs = *src[si].outs;
    // slot width of an output (its B matrix's padded rows), 0 when it does not take slots
    auto slot_width = [&](const TcPlanOut& o) -> int {
      if (nvec < 2 || o.tmat < 0 || o.seg_count != 1) return 0;
      const TcPlanSeg& g = tp.segs[o.seg_begin];
      const TcMat& A = tp.mats[g.a];
      const TcMat& B = tp.mats[g.b];
      const TcMat& T = tp.mats[o.tmat];
      if (A.pool != 0 || B.pool != 1 || T.pool != 2 || 2 * B.Rp > TN || T.K > 32 || o.n > B.Rp) return 0;
      return B.Rp;
    };
    {
      std::map<std::tuple<int, int, int>, std::vector<Piece>> groups;
      std::vector<Stack> bins;
      for (size_t i = 0; i < outs.size(); ++i) {
        if (!slot_width(outs[i])) continue;
        const TcPlanSeg& g = tp.segs[outs[i].seg_begin];
        const int full = outs[i].m / TM, rem = outs[i].m - full * TM;
        for (int a = 0; a < full; ++a)
          bins.push_back(Stack{(int)si, 0, outs[i].n, g.k, g.b, {Piece{(int)i, a * TM, TM, 0}}});
        if (rem) groups[std::make_tuple(g.b, outs[i].n, g.k)].push_back(Piece{(int)i, full * TM, (rem + 7) & ~7, 0});
      }
      pack(groups, (int)si, 0, bins);
      for (const Stack& b : bins) {
        const int w = slot_width(outs[b.pc[0].o]);
        const int spt = TN / w;
        for (int v0 = 0; v0 < nvec; v0 += spt) {
          Stack S = b;
          S.v = v0;
          S.nv = std::min(spt, nvec - v0);
          S.wv = w;
          const int id = (int)stacks.size();
          stacks.push_back(std::move(S));
          tiles.push_back(Tile{(int)si, v0, stacks[id].pc[0].o, 0, 0, (int64_t)stacks[id].k, id, 0});
        }
      }
    }
    for (size_t i = 0; i < outs.size(); ++i) {
      const int rs = std::min(row_slots(tp, outs[i]), rs_cap);
      if (rs <= 0) continue;
      int64_t kt = 0;
      for (int q = 0; q < outs[i].seg_count; ++q) kt += tp.segs[outs[i].seg_begin + q].k;
      for (int v0 = 0; v0 < nvec; v0 += rs)
        for (int b = 0; b < (outs[i].n + TN - 1) / TN; ++b)
          tiles.push_back(Tile{(int)si, v0, (int)i, 0, b, kt, -1, std::min(rs, nvec - v0)});
    }
    for (int v = 0; v < nvec; ++v) {
      std::map<std::tuple<int, int, int>, std::vector<Piece>> groups;   // (B matrix, n, k) -> pieces
      for (size_t i = 0; i < outs.size(); ++i) {
        if (slot_width(outs[i]) || row_slots(tp, outs[i])) continue;
        int64_t kt = 0;
        for (int q = 0; q < outs[i].seg_count; ++q) kt += tp.segs[outs[i].seg_begin + q].k;
        const bool stackable = outs[i].tmat >= 0 && outs[i].seg_count == 1 && outs[i].m % TM != 0;
        const int full = outs[i].m / TM;
        for (int a = 0; a < (stackable ? full : (outs[i].m + TM - 1) / TM); ++a)
          for (int b = 0; b < (outs[i].n + TN - 1) / TN; ++b)
            tiles.push_back(Tile{(int)si, v, (int)i, a, b, kt, -1, 0});
        if (stackable) {
          const TcPlanSeg& g = tp.segs[outs[i].seg_begin];
          const int rem = outs[i].m - full * TM;
          groups[std::make_tuple(g.b, outs[i].n, g.k)].push_back(Piece{(int)i, full * TM, (rem + 7) & ~7, 0});
        }
      }
      std::vector<Stack> bins;
      pack(groups, (int)si, v, bins);
      for (Stack& b : bins) {
        const int id = (int)stacks.size();
        stacks.push_back(std::move(b));
        for (int nb = 0; nb < (stacks[id].n + TN - 1) / TN; ++nb)
          tiles.push_back(Tile{(int)si, v, stacks[id].pc[0].o, 0, nb, (int64_t)stacks[id].k, id, 0});
      }
    }
  }
  std::stable_sort(tiles.begin(), tiles.end(), [](const Tile& x, const Tile& y) { return x.k > y.k; });
  const int nt = (int)tiles.size();
  nctas = nt > 0 ? tc_num_ctas(nt) : 0;
  auto base = [&](const TcSource& sc, const TcMat& m, int v, bool hi) -> float* {
    float* p = (hi ? sc.phi : sc.plo)[m.pool];
    return p + (m.pool ? (int64_t)v * sc.tp->pool_size[m.pool] : 0) + m.off;
  };
  std::vector<TcItem> it;
  std::vector<int> beg;
  std::vector<std::pair<size_t, size_t>> fix;   // stacked header -> index of its first piece
  for (int b = 0; b < nctas; ++b) {
    beg.push_back((int)it.size());
    for (int w = b; w < nt; w += nctas) {
      const Tile& t = tiles[w];
      const TcSource& sc = src[t.s];
      const TcPlan& tp = *sc.tp;
      const TcPlanOut& o = (*sc.outs)[t.o];
      if (t.stack >= 0) {
        const Stack& S = stacks[t.stack];
        TcItem h{};
        h.type = TC_ITEM_TILE;
        h.t.c_rel = S.nv ? 4 : 3;
        h.t.m0 = 0;
        h.t.n0 = t.b * TN;
        h.t.nt = std::min(TN, S.n - h.t.n0);
        h.t.t_k = S.n;
        h.t.inst = (int)S.pc.size();
        if (S.nv) {
          // slots: the vectors v0 .. v0 + nv - 1 of pools 1 (B) and 2 (intermediates)
          h.t.n0 = 0;
          h.t.nt = S.nv * S.wv;
          h.t.ldc = S.wv;
          h.t.accumulate = S.nv;
          h.t.c_off = tp.pool_size[2];
          if (S.nv * S.wv > TN || S.wv % 8 != 0 || S.wv > 32)
            throw Error(LRT_EINVAL, "tensor-core plan: vector slots outside the tile");
        }
        int rows = 0;
        for (const Piece& pc : S.pc) rows += pc.nrows;
        h.t.mt = rows;
        fix.push_back({it.size(), it.size() + 1});
        it.push_back(h);
        const TcPlanSeg* g0 = nullptr;
        for (const Piece& pc : S.pc) {
          const TcPlanOut& po = (*sc.outs)[pc.o];
          const TcPlanSeg& g = tp.segs[po.seg_begin];
          g0 = &g;
          const TcMat& A = tp.mats[g.a];
          const TcMat& T = tp.mats[po.tmat];
          if (A.Rp < pc.row0 + pc.nrows || T.Rp < pc.row0 + pc.nrows || T.K != S.n)
            throw Error(LRT_EINVAL, "tensor-core plan: stacked piece outside its matrices");
          TcItem r{};
          r.type = TC_ITEM_PIECE;
          r.p.a_hi = base(sc, A, t.v, true);
          r.p.a_lo = base(sc, A, t.v, false);
          r.p.t_hi = base(sc, T, t.v, true);
          r.p.t_lo = base(sc, T, t.v, false);
          r.p.a_rp = A.Rp;
          r.p.a_row0 = pc.row0;
          r.p.nrows = pc.nrows;
          r.p.smem_row = pc.srow;
          r.p.t_rp = T.Rp;
          r.p.t_row0 = pc.row0;
          it.push_back(r);
        }
        const TcMat& A0 = tp.mats[g0->a];
        const TcMat& B = tp.mats[g0->b];
        TcItem r{};
        r.type = TC_ITEM_SEG;
        r.s.a_hi = base(sc, A0, t.v, true);
        r.s.a_lo = base(sc, A0, t.v, false);
        r.s.b_hi = base(sc, B, t.v, true);
        r.s.b_lo = base(sc, B, t.v, false);
        r.s.a_rp = A0.Rp;
        r.s.b_rp = B.Rp;
        r.s.k = S.k;
        r.s.scale = g0->scale;
        if (S.nv) {
          if (B.Rp != S.wv || B.pool != 1) throw Error(LRT_EINVAL, "tensor-core plan: slot width of B");
          r.s.b_vstride = tp.pool_size[1];
        }
        it.push_back(r);
        continue;
      }
      TcItem h{};
      h.type = TC_ITEM_TILE;
      h.t.m0 = t.a * TM;
      h.t.n0 = t.b * TN;
      h.t.mt = std::min(TM, o.m - h.t.m0);
      h.t.nt = std::min(TN, o.n - h.t.n0);
      h.t.inst = sc.inst;
      const int Rp = (o.m + 7) & ~7;
      if (t.rs > 0) {
        if (sc.nelem > INT32_MAX || t.rs * Rp > TM)
          throw Error(LRT_EINVAL, "tensor-core plan: row slots outside the tile");
        h.t.c_rel = 5;
        h.t.m0 = 0;
        h.t.mt = t.rs * Rp;
        h.t.vslots = t.rs;
        h.t.vrows = Rp;
        h.t.vvalid = o.m;
        h.t.vstride = (int)sc.nelem;
        h.t.c_off = o.c_off + (int64_t)t.v * sc.nelem;
        h.t.ldc = o.ldc;
      } else if (o.tmat >= 0) {
        const TcMat& m = tp.mats[o.tmat];
        h.t.c_rel = 2;
        h.t.t_hi = base(sc, m, t.v, true);
        h.t.t_lo = base(sc, m, t.v, false);
        h.t.t_rp = m.Rp;
        h.t.t_k = m.K;
      } else if (o.C) {
        h.t.c_rel = 0;
        h.t.C = o.C;
        h.t.ldc = o.ldc;
      } else {
        h.t.c_rel = 1;
        h.t.c_off = o.c_off + (int64_t)t.v * sc.nelem;
        h.t.ldc = o.ldc;
      }
      it.push_back(h);
      for (int q = 0; q < o.seg_count; ++q) {
        const TcPlanSeg& g = tp.segs[o.seg_begin + q];
        if (g.k <= 0) continue;
        const TcMat& A = tp.mats[g.a];
        const TcMat& B = tp.mats[g.b];
        // the kernel copies rows [m0, m0 + 128) of A and [n0, n0 + 64) of B, clipped to Rp
        if (A.R < o.m || B.R < o.n || A.K < g.k || B.K < g.k)
          throw Error(LRT_EINVAL, "tensor-core plan: operand smaller than its product");
        TcItem r{};
        r.type = TC_ITEM_SEG;
        r.s.a_hi = base(sc, A, t.v, true);
        r.s.a_lo = base(sc, A, t.v, false);
        r.s.b_hi = base(sc, B, t.v, true);
        r.s.b_lo = base(sc, B, t.v, false);
        r.s.a_rp = A.Rp;
        r.s.b_rp = B.Rp;
        r.s.k = g.k;
        r.s.scale = g.scale;
        if (t.rs > 0) {
          if (A.pool == 0 || A.Rp != Rp) throw Error(LRT_EINVAL, "tensor-core plan: row-slot operand");
          r.s.a_vstride = tp.pool_size[A.pool];
        }
        it.push_back(r);
      }
    }
  }
  beg.push_back((int)it.size());
  items.upload(it, st);
  if (!fix.empty()) {
    // stacked headers point at their pieces, in the uploaded stream
    for (const auto& f : fix) it[f.first].t.C = reinterpret_cast<double*>(items.p + f.second);
    CK(cudaMemcpyAsync(items.p, it.data(), it.size() * sizeof(TcItem), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  begins.upload(beg, st);
}

// Autotuner of the tensor-core tile width (128 x 32 or 128 x 64) for one launch.
// Launches with enough tiles to occupy the GPU several times are timed once with each
// width (second of two runs, CUDA events, outputs into scratch buffers); smaller ones
// take 32 when the work-weighted output width is at most 32.  Returns the width, with
// the matching stream in items/begins/nctas.
static int tune_tc_stream(lrt_ctx* c, const std::vector<TcSource>& src, int nvec, TcOut scratch,
                          DevArray<TcItem>& items, DevArray<int>& begins, int& nctas, bool timed = true) {
  cudaStream_t st = c->st;
  build_tc_stream(src, nvec, 64, items, begins, nctas, st);
  double wn = 0.0, w = 0.0;
  int64_t ntiles = 0;
  for (const TcSource& sc : src)
    for (const TcPlanOut& o : *sc.outs) {
      int64_t kt = 0;
      for (int q = 0; q < o.seg_count; ++q) kt += sc.tp->segs[o.seg_begin + q].k;
      wn += (double)kt * o.m * std::min(o.n, 64);
      w += (double)kt * o.m;
      ntiles += (int64_t)((o.m + 127) / 128) * ((o.n + 63) / 64) * nvec;
    }
  const int heuristic = (w > 0.0 && wn / w <= 32.0) ? 32 : 64;
  if (!timed || ntiles < 4 * (int64_t)tc_num_ctas(1 << 30)) {
    if (heuristic == 32) build_tc_stream(src, nvec, 32, items, begins, nctas, st);
    return heuristic;
  }
  if (!c->derr) {
    if (dev_alloc((void**)&c->derr, sizeof(int)) != cudaSuccess) throw Error(LRT_ENOMEM, "error flag");
    CK(cudaMemsetAsync(c->derr, 0, sizeof(int), st));
  }
  DevArray<TcItem> it32;
  DevArray<int> b32;
  int n32 = 0;
  build_tc_stream(src, nvec, 32, it32, b32, n32, st);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float t[2] = {0.0f, 0.0f};
  for (int v = 0; v < 2; ++v) {
    for (int rep = 0; rep < 2; ++rep) {
      CK(cudaEventRecord(e0, st));
      if (v == 0)
        launch_gemm_tf32x3(items.p, begins.p, nctas, 64, scratch, c->derr, st);
      else
        launch_gemm_tf32x3(it32.p, b32.p, n32, 32, scratch, c->derr, st);
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&t[v], e0, e1));
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c->derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flag) {
    CK(cudaMemsetAsync(c->derr, 0, sizeof(int), st));
    throw Error(LRT_ETIMEOUT, "tensor-core autotuning: a pipeline wait expired");
  }
  if (t[1] < t[0]) {
    items.swap(it32);
    begins.swap(b32);
    nctas = n32;
    return 32;
  }
  return 64;
}

// TC-matrix pools, packed operators and work streams of a plan (once per plan)
static void prepare_tc(lrt_ctx* c, SigmaPlan& p, int nvec) {
  if (p.tc_ready) return;
  TcPlan& tp = p.tc;
  for (int q = 0; q < 3; ++q) {
    const size_t n = (size_t)std::max<int64_t>(tp.pool_size[q] * (q ? nvec : 1), 1);
    if (dev_alloc((void**)&p.pool_hi[q], n * sizeof(float)) != cudaSuccess ||
        dev_alloc((void**)&p.pool_lo[q], n * sizeof(float)) != cudaSuccess)
      throw Error(LRT_ENOMEM, "tensor-core operand pools");
    if (q == 2) {
      CK(cudaMemsetAsync(p.pool_hi[q], 0, n * sizeof(float), c->st));
      CK(cudaMemsetAsync(p.pool_lo[q], 0, n * sizeof(float), c->st));
    }
  }
  {
    DevArray<TcPack> d0;
    d0.upload(tp.pack0, c->st);
    launch_tc_pack(d0.p, (int)tp.pack0.size(), nullptr, 0, p.pool_hi[0], p.pool_lo[0], 0, 1, c->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
  }
  p.xpack.upload(tp.pack1, c->st);
  {
    // tile widths chosen on this plan's own data (x pool zeroed, outputs into scratch)
    const size_t nx = (size_t)std::max<int64_t>(tp.pool_size[1] * nvec, 1);
    CK(cudaMemsetAsync(p.pool_hi[1], 0, nx * sizeof(float), c->st));
    CK(cudaMemsetAsync(p.pool_lo[1], 0, nx * sizeof(float), c->st));
    DevBuf ys;
    ys.ensure((size_t)std::max<int64_t>(p.nelem * nvec, 1));
    const TcOut scratch = tc_out(c, ys.p, nullptr);
    p.tn1 = tune_tc_stream(c, {TcSource{&tp, &tp.out1, p.pool_hi, p.pool_lo, p.nelem, 0}}, nvec, scratch, p.tci1,
                           p.tcb1, p.tcn1);
    p.tn2 = tune_tc_stream(c, {TcSource{&tp, &tp.out2, p.pool_hi, p.pool_lo, p.nelem, 0}}, nvec, scratch, p.tci2,
                           p.tcb2, p.tcn2);
    CK(cudaStreamSynchronize(c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  p.tc_ready = true;
}

// y = H_eff x through the split-TF32 tensor-core kernels (both phases), then a check
// of the kernels' error flag (a bounded pipeline wait that expired)
static void run_tc(lrt_ctx* ctx, SigmaPlan& p, const double* x_dev, double* y_dev, int nvec) {
  if (!ctx->derr) {
    if (dev_alloc((void**)&ctx->derr, sizeof(int)) != cudaSuccess) throw Error(LRT_ENOMEM, "error flag");
    CK(cudaMemsetAsync(ctx->derr, 0, sizeof(int), ctx->st));
  }
  prepare_tc(ctx, p, nvec);
  launch_tc_pack(p.xpack.p, (int)p.tc.pack1.size(), x_dev, p.nelem, p.pool_hi[1], p.pool_lo[1], p.tc.pool_size[1],
                 nvec, ctx->st);
  const TcOut to = tc_out(ctx, y_dev, nullptr);
  launch_gemm_tf32x3(p.tci1.p, p.tcb1.p, p.tcn1, p.tn1, to, ctx->derr, ctx->st);
  launch_gemm_tf32x3(p.tci2.p, p.tcb2.p, p.tcn2, p.tn2, to, ctx->derr, ctx->st);
  CK(cudaGetLastError());
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (flag) {
    CK(cudaMemsetAsync(ctx->derr, 0, sizeof(int), ctx->st));
    throw Error(LRT_ETIMEOUT, "sigma: a tensor-core pipeline wait expired; results are invalid");
  }
}

// The renormalization's two grouped GEMMs (phase 1: T_i = op(A) op(B), one product per
// output, into a workspace; phase 2: C = sum op(A) T_s with T_s read as B, no
// transpose) on the tensor cores: phase 1 computes T_i^T = op(B)^T op(A)^T straight into
// a TC matrix (rows = columns of T), which is the operand image phase 2 needs; phase 2
// writes the FP64 blocks of C.  Operands are packed once; tile widths by the heuristic.
static void run_two_phase_tc(lrt_ctx* c, const std::vector<GemmOut>& o1, const std::vector<GemmSeg>& s1,
                             const std::vector<GemmOut>& o2, const std::vector<GemmSeg>& s2) {
  TcPlan tp;
  std::map<int64_t, int> tmat_of;   // workspace offset of T_i -> TC matrix of T_i^T
  auto a_role = [&](const GemmSeg& g, int m) { return tp.op(g.A, g.lda, g.transA ? 1 : 0, m, g.k); };
  auto b_role = [&](const GemmSeg& g, int n) { return tp.op(g.B, g.ldb, g.transB ? 0 : 1, n, g.k); };
  for (const GemmOut& o : o1) {
    if (o.seg_count != 1) throw Error(LRT_EINVAL, "mixed renormalize: one product per intermediate expected");
    const GemmSeg& g = s1[o.seg_begin];
    const int A = b_role(g, o.n);       // rows = columns of T
    const int B = a_role(g, o.m);       // rows = rows of T
    const int t = tp.add(2, o.n, o.m);
    tmat_of[o.c_off] = t;
    tp.out1.push_back(TcPlanOut{t, 0, 0, o.n, o.m, (int)tp.segs.size(), 1});
    tp.segs.push_back(TcPlanSeg{A, B, g.k, (float)g.scale});
  }
  for (const GemmOut& o : o2) {
    const int sb = (int)tp.segs.size();
    for (int q = 0; q < o.seg_count; ++q) {
      const GemmSeg& g = s2[o.seg_begin + q];
      if (g.transB) throw Error(LRT_EINVAL, "mixed renormalize: transposed intermediate");
      auto it = tmat_of.find(g.b_off);
      if (it == tmat_of.end()) throw Error(LRT_EINVAL, "mixed renormalize: unknown intermediate");
      tp.segs.push_back(TcPlanSeg{a_role(g, o.m), it->second, g.k, (float)g.scale});
    }
    TcPlanOut out{-1, 0, o.ldc, o.m, o.n, sb, (int)tp.segs.size() - sb};
    out.C = o.C;
    tp.out2.push_back(out);
  }
  float* phi[3] = {nullptr, nullptr, nullptr};
  float* plo[3] = {nullptr, nullptr, nullptr};
  struct Pools {
    float** h;
    float** l;
    ~Pools() {
      for (int q = 0; q < 3; ++q) {
        dev_free(h[q]);
        dev_free(l[q]);
      }
    }
  } guard_pools{phi, plo};
  for (int q : {0, 2}) {
    const size_t nw = (size_t)std::max<int64_t>(tp.pool_size[q], 1);
    if (dev_alloc((void**)&phi[q], nw * sizeof(float)) != cudaSuccess ||
        dev_alloc((void**)&plo[q], nw * sizeof(float)) != cudaSuccess)
      throw Error(LRT_ENOMEM, "mixed renormalize: operand pools");
  }
  DevArray<TcPack> d0;
  d0.upload(tp.pack0, c->st);
  launch_tc_pack(d0.p, (int)tp.pack0.size(), nullptr, 0, phi[0], plo[0], 0, 1, c->st);
  if (!c->derr) {
    if (dev_alloc((void**)&c->derr, sizeof(int)) != cudaSuccess) throw Error(LRT_ENOMEM, "error flag");
    CK(cudaMemsetAsync(c->derr, 0, sizeof(int), c->st));
  }
  DevArray<TcItem> i1, i2;
  DevArray<int> b1, b2;
  int n1 = 0, n2 = 0;
  const TcOut none = tc_out(c, nullptr, nullptr);
  const int t1 = tune_tc_stream(c, {TcSource{&tp, &tp.out1, phi, plo, 0, 0}}, 1, none, i1, b1, n1, false);
  const int t2 = tune_tc_stream(c, {TcSource{&tp, &tp.out2, phi, plo, 0, 0}}, 1, none, i2, b2, n2, false);
  launch_gemm_tf32x3(i1.p, b1.p, n1, t1, none, c->derr, c->st);
  launch_gemm_tf32x3(i2.p, b2.p, n2, t2, none, c->derr, c->st);
  CK(cudaGetLastError());
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c->derr, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (flag) {
    CK(cudaMemsetAsync(c->derr, 0, sizeof(int), c->st));
    throw Error(LRT_ETIMEOUT, "renormalize: a tensor-core pipeline wait expired; results are invalid");
  }
}

static SigmaPlan* find_plan(lrt_ctx* c, int site, int nsite, int nvec) {
  auto it = c->plans.find(std::make_tuple(site, nsite, nvec));
  return it == c->plans.end() ? nullptr : it->second.get();
}

// the plan of (site, nsite, nvec); tc: with the tensor-core twin (replanned if missing)
static SigmaPlan& get_plan(lrt_ctx* c, int site, int nsite, int nvec, bool tc = false) {
  auto key = std::make_tuple(site, nsite, nvec);
  auto it = c->plans.find(key);
  if (it != c->plans.end() && (!tc || it->second->has_tc)) return *it->second;
  auto p = plan_sigma(c, site, nsite, nvec, tc);
  SigmaPlan& ref = *p;
  c->plans[key] = std::move(p);
  return ref;
}

}  // namespace lrt

// ===========================================================================
// ground-state sweeps: two-site Davidson (Eq. dmrg) and density-matrix
// decimation with the gauge shift of Eq. gauge-shift
// ===========================================================================
namespace lrt {

struct SolverHandle {
  cusolverDnHandle_t h = nullptr;
  ~SolverHandle() {
    if (h) cusolverDnDestroy(h);
  }
};

static double dev_dot(const double* a, const double* b, int64_t n, double* dtmp, cudaStream_t st) {
  launch_dots(a, n, 1, b, n, dtmp, st);
  double r = 0.0;
  CK(cudaMemcpyAsync(&r, dtmp, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return r;
}

static void upload_coef(double* dcoef, const std::vector<double>& c, cudaStream_t st) {
  if (!c.empty()) CK(cudaMemcpyAsync(dcoef, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, st));
}

// Lowest eigenpair of H_eff at a two-site position; psi (device) is the start vector
// and receives the eigenvector.  Returns the eigenvalue.
static double davidson_site(lrt_ctx* c, int i, int nsite, double* psi, const lrt_gs_params& P, int* iters_out) {
  SigmaPlan& plan = get_plan(c, i, nsite, 1);
  const int64_t n = plan.nelem;
  const int maxs = std::max(2, std::min(P.dav_max_space, JACOBI_MAXN));
  DevBuf V, AV, diag, r, t, u, au, small, coef, Hd, Wd, Zd;
  V.ensure((size_t)maxs * n);
  AV.ensure((size_t)maxs * n);
  diag.ensure(n);
  r.ensure(n);
  t.ensure(n);
  u.ensure(n);
  au.ensure(n);
  small.ensure(JACOBI_MAXN + 8);
  coef.ensure(JACOBI_MAXN + 8);
  Hd.ensure(JACOBI_MAXN * JACOBI_MAXN);
  Wd.ensure(JACOBI_MAXN);
  Zd.ensure(JACOBI_MAXN * JACOBI_MAXN);
  cudaStream_t st = c->st;
  launch_diag(plan.douts.p, plan.dterms.p, plan.ndiag, diag.p, st);
  CK(cudaMemcpyAsync(t.p, psi, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  std::vector<double> Hs((size_t)maxs * maxs, 0.0), hcol(maxs), w(maxs), Z((size_t)maxs * maxs);
  int m = 0;
  double theta = 0.0;
  int it = 0;
  for (; it < P.dav_max_iter; ++it) {
    // orthogonalize the new direction against the subspace (twice) and normalize
    for (int pass = 0; pass < 2 && m > 0; ++pass) {
      launch_dots(V.p, n, m, t.p, n, small.p, st);
      std::vector<double> cc(m);
      CK(cudaMemcpyAsync(cc.data(), small.p, m * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (double& x : cc) x = -x;
      upload_coef(coef.p, cc, st);
      launch_lincomb(V.p, n, m, coef.p, n, t.p, 1.0, st);
    }
    const double nt = std::sqrt(std::max(0.0, dev_dot(t.p, t.p, n, small.p, st)));
    if (nt < 1e-14) break;
    launch_lincomb(nullptr, n, 0, coef.p, n, t.p, 1.0 / nt, st);
    CK(cudaMemcpyAsync(V.p + (size_t)m * n, t.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    plan.p1.run(st, V.p + (size_t)m * n, AV.p + (size_t)m * n, plan.tbuf, &plan.ex);
    plan.p2.run(st, V.p + (size_t)m * n, AV.p + (size_t)m * n, plan.tbuf, &plan.ex);
    launch_dots(V.p, n, m + 1, AV.p + (size_t)m * n, n, small.p, st);
    CK(cudaMemcpyAsync(hcol.data(), small.p, (m + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int j = 0; j <= m; ++j) {
      Hs[(size_t)j * maxs + m] = hcol[j];
      Hs[(size_t)m * maxs + j] = hcol[j];
    }
    ++m;
    // subspace eigenproblem on the GPU
    std::vector<double> Hc((size_t)m * m);
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) Hc[(size_t)a * m + b] = Hs[(size_t)a * maxs + b];
    CK(cudaMemcpyAsync(Hd.p, Hc.data(), Hc.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_jacobi_eigh(Hd.p, m, Wd.p, Zd.p, st);
    CK(cudaMemcpyAsync(w.data(), Wd.p, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(Z.data(), Zd.p, (size_t)m * m * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    theta = w[0];
    std::vector<double> al(m);
    for (int a = 0; a < m; ++a) al[a] = Z[(size_t)a * m + 0];
    upload_coef(coef.p, al, st);
    launch_lincomb(V.p, n, m, coef.p, n, u.p, 0.0, st);
    launch_lincomb(AV.p, n, m, coef.p, n, au.p, 0.0, st);
    CK(cudaMemcpyAsync(r.p, au.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    std::vector<double> mt = {-theta};
    upload_coef(coef.p, mt, st);
    launch_lincomb(u.p, n, 1, coef.p, n, r.p, 1.0, st);
    const double rn = std::sqrt(std::max(0.0, dev_dot(r.p, r.p, n, small.p, st)));
    if (rn < P.dav_tol) {
      ++it;
      break;
    }
    launch_precond(r.p, diag.p, theta, n, t.p, st);
    if (m == maxs) {   // restart with the Ritz vector
      CK(cudaMemcpyAsync(V.p, u.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(AV.p, au.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      std::fill(Hs.begin(), Hs.end(), 0.0);
      Hs[0] = theta;
      m = 1;
    }
  }
  CK(cudaMemcpyAsync(psi, u.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  if (iters_out) *iters_out = it;
  return theta;
}

// right-fused copy (per left sector q: D_q x fused(q), sub-blocks n side by side) of site b
static std::vector<int64_t> site_rfused(lrt_ctx* c, int b, DevBuf& buf, const Fused& F) {
  return rfused_copy(c, b, c->sites[b], buf, F);
}

// the layout of a right-fused copy (offsets per left sector, total) and its kept gather plan
static const GatherPlan& rfused_plan(lrt_ctx* c, int b, const SiteTensor& T, const Fused& F, std::vector<int64_t>& off,
                                     int64_t& tot);

static std::vector<int64_t> rfused_copy(lrt_ctx* c, int b, const SiteTensor& T, DevBuf& buf, const Fused& F) {
  std::vector<int64_t> off;
  int64_t tot = 0;
  const GatherPlan& g = rfused_plan(c, b, T, F, off, tot);
  double* p = buf.ensure(tot);
  CK(cudaMemsetAsync(p, 0, (size_t)std::max<int64_t>(tot, 1) * sizeof(double), c->st));
  launch_gather(g.tasks.p, g.srcs.p, g.tiles.p, g.ntiles, c->st, p, T.d);
  CK(cudaGetLastError());
  return off;
}

static const GatherPlan& rfused_plan(lrt_ctx* c, int b, const SiteTensor& T, const Fused& F, std::vector<int64_t>& off,
                                     int64_t& tot) {
  const Sectors& Lb = c->bonds[b];
  off.assign(Lb.n(), -1);
  tot = 0;
  uint64_t h = site_signature(T);
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  for (int q = 0; q < Lb.n(); ++q) {
    const int f = F.s.find(Lb.a[q], Lb.b[q]);
    mix((uint64_t)(f + 1));
    if (f < 0) continue;
    off[q] = tot;
    tot += (int64_t)Lb.d[q] * F.s.d[f];
    for (int n = 0; n < 4; ++n) mix((uint64_t)F.off[f][n]);
    mix((uint64_t)F.s.d[f]);
  }
  const std::pair<int, uint64_t> key{b, h};
  auto it = c->rf_plans.find(key);
  if (it == c->rf_plans.end()) {
    if (c->rf_plans.size() > 4096) c->rf_plans.clear();   // layouts of earlier bond dimensions
    std::vector<GatherTask> tasks;
    std::vector<GatherSrc> srcs;
    for (int q = 0; q < Lb.n(); ++q) {
      if (off[q] < 0) continue;
      const int f = F.s.find(Lb.a[q], Lb.b[q]);
      for (int n = 0; n < 4; ++n) {
        if (T.sub_off[q][n] < 0) continue;
        const int Dr = c->bonds[b + 1].d[T.sub_qr[q][n]];
        GatherTask t{nullptr, F.s.d[f], Lb.d[q], Dr, (int)srcs.size(), 1};
        t.dst_off = off[q] + F.off[f][n];
        tasks.push_back(t);
        GatherSrc g{nullptr, Dr, 0, 1.0};
        g.src_off = T.sub_off[q][n];
        g.rel = 1;
        srcs.push_back(g);
      }
    }
    auto np = std::make_unique<GatherPlan>();
    build_gather(*np, tasks, srcs, c->st);
    it = c->rf_plans.emplace(key, std::move(np)).first;
  }
  return *it->second;
}

// theta(i) = site i (left-fused) x site i+1 (right-fused), in the two-site layout
static void form_theta(lrt_ctx* c, int i, double* psi, const std::vector<WfnBlock>& wb) {
  const Fused fr = fuse(c->bonds[i + 2], true);
  DevBuf rf;
  std::vector<int64_t> roff = site_rfused(c, i + 1, rf, fr);
  const SiteTensor& A = c->sites[i];
  const Sectors& mid = c->bonds[i + 1];
  int64_t n = 0;
  for (auto& w : wb) n = std::max(n, w.off + (int64_t)w.rows * w.cols);
  CK(cudaMemsetAsync(psi, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(double), c->st));
  std::vector<GemmOut> outs;
  std::vector<GemmSeg> segs;
  for (const WfnBlock& w : wb) {
    const int q = mid.find(w.label_a, w.label_b);
    if (q < 0 || A.blk_off[q] < 0 || roff[q] < 0) continue;
    if (A.blk_rows[q] != w.rows) throw Error(LRT_EINVAL, "internal: theta rows mismatch");
    outs.push_back(GemmOut{psi + w.off, 0, w.cols, w.rows, w.cols, (int)segs.size(), 1, 0, 0});
    segs.push_back(GemmSeg{A.d + A.blk_off[q], rf.p + roff[q], 0, 0, mid.d[q], w.cols, mid.d[q], 0, 0, 0, 0, 1.0});
  }
  GemmPlan gp;
  build_gemm(gp, outs, segs, c->st);
  gp.run(c->st, nullptr, nullptr);
  CK(cudaStreamSynchronize(c->st));
}

static void upload_site(lrt_ctx* c, int b, SiteTensor&& T) {
  c->sites[b] = std::move(T);
}

// Split theta at bond i+1 keeping the M largest density-matrix weights; dir = +1
// leaves site i left-orthonormal and the centre on site i+1, dir = -1 leaves site
// i+1 right-orthonormal and the centre on site i.  Returns the discarded weight.
static double decimate(lrt_ctx* c, int i, const double* psi, const std::vector<WfnBlock>& wb, int M,
                       double trunc_tol, int dir, SolverHandle& sh) {
  cudaStream_t st = c->st;
  if (!sh.h) {
    if (cusolverDnCreate(&sh.h) != CUSOLVER_STATUS_SUCCESS) throw Error(LRT_ECUDA, "cusolverDnCreate failed");
  }
  cusolverDnSetStream(sh.h, st);
  // density matrices, one per middle sector: rho = psi psi^T (dir +1) or psi^T psi (dir -1)
  std::vector<int64_t> roff(wb.size());
  std::vector<int> rdim(wb.size());
  int64_t rtot = 0;
  for (size_t w = 0; w < wb.size(); ++w) {
    rdim[w] = dir > 0 ? wb[w].rows : wb[w].cols;
    roff[w] = rtot;
    rtot += (int64_t)rdim[w] * rdim[w];
  }
  DevBuf rho, ev;
  rho.ensure(rtot);
  int64_t etot = 0;
  for (int d : rdim) etot += d;
  ev.ensure(etot);
  {
    std::vector<GemmOut> outs;
    std::vector<GemmSeg> segs;
    for (size_t w = 0; w < wb.size(); ++w) {
      const WfnBlock& b = wb[w];
      outs.push_back(GemmOut{rho.p + roff[w], 0, rdim[w], rdim[w], rdim[w], (int)segs.size(), 1, 0, 0});
      if (dir > 0)
        segs.push_back(GemmSeg{psi + b.off, psi + b.off, 0, 0, b.cols, b.cols, b.cols, 0, 1, 0, 0, 1.0});
      else
        segs.push_back(GemmSeg{psi + b.off, psi + b.off, 0, 0, b.cols, b.cols, b.rows, 1, 0, 0, 0, 1.0});
    }
    GemmPlan gp;
    build_gemm(gp, outs, segs, st);
    gp.run(st, nullptr, nullptr);
  }
  // eigen-decomposition per sector (cuSOLVER, FP64 on the device)
  int* dinfo = nullptr;
  if (dev_alloc((void**)&dinfo, sizeof(int)) != cudaSuccess) throw Error(LRT_ENOMEM, "cusolver info");
  DevBuf work;
  std::vector<int64_t> eoff(wb.size());
  int64_t eo = 0;
  for (size_t w = 0; w < wb.size(); ++w) {
    eoff[w] = eo;
    const int nn = rdim[w];
    eo += nn;
    if (nn == 0) continue;
    int lw = 0;
    if (cusolverDnDsyevd_bufferSize(sh.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, nn, rho.p + roff[w], nn,
                                    ev.p + eoff[w], &lw) != CUSOLVER_STATUS_SUCCESS)
      throw Error(LRT_ECUDA, "syevd buffer size failed");
    work.ensure(std::max(lw, 1));
    if (cusolverDnDsyevd(sh.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, nn, rho.p + roff[w], nn,
                         ev.p + eoff[w], work.p, lw, dinfo) != CUSOLVER_STATUS_SUCCESS)
      throw Error(LRT_ECUDA, "syevd failed");
  }
  std::vector<double> evh(etot);
  CK(cudaMemcpyAsync(evh.data(), ev.p, etot * sizeof(double), cudaMemcpyDeviceToHost, st));
  int info = 0;
  CK(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  dev_free(dinfo);
  if (info != 0) throw Error(LRT_ECUDA, "syevd reported info " + std::to_string(info));
  // keep the M largest weights over all sectors (ties: sector order, then index)
  struct W { double v; int w; int j; };
  std::vector<W> all;
  double vmax = 0.0;
  for (size_t w = 0; w < wb.size(); ++w)
    for (int j = 0; j < rdim[w]; ++j) {
      all.push_back({evh[eoff[w] + j], (int)w, j});
      vmax = std::max(vmax, evh[eoff[w] + j]);
    }
  std::stable_sort(all.begin(), all.end(), [](const W& a, const W& b) {
    if (a.v != b.v) return a.v > b.v;
    if (a.w != b.w) return a.w < b.w;
    return a.j > b.j;
  });
  std::vector<int> keep(wb.size(), 0);
  double disc = 0.0;
  int kept = 0;
  for (const W& x : all) {
    if (kept < M && x.v > trunc_tol * vmax) {
      ++keep[x.w];
      ++kept;
    } else {
      disc += std::max(0.0, x.v);
    }
  }
  // new bond table (bond i+1)
  Sectors nb;
  std::vector<int> wsec(wb.size(), -1);
  for (size_t w = 0; w < wb.size(); ++w)
    if (keep[w] > 0) wsec[w] = nb.add(wb[w].label_a, wb[w].label_b, keep[w]);
  // the kept eigenvectors of a sector are its last keep[w] rows (ascending eigenvalues)
  c->bonds[i + 1] = nb;
  SiteTensor Ti, Tj;
  site_layout(Ti, c->bonds[i], c->bonds[i + 1]);
  site_layout(Tj, c->bonds[i + 1], c->bonds[i + 2]);
  if (dev_alloc((void**)&Ti.d, (size_t)std::max<int64_t>(Ti.total, 1) * sizeof(double)) != cudaSuccess ||
      dev_alloc((void**)&Tj.d, (size_t)std::max<int64_t>(Tj.total, 1) * sizeof(double)) != cudaSuccess)
    throw Error(LRT_ENOMEM, "site tensors");
  CK(cudaMemsetAsync(Ti.d, 0, (size_t)std::max<int64_t>(Ti.total, 1) * sizeof(double), st));
  CK(cudaMemsetAsync(Tj.d, 0, (size_t)std::max<int64_t>(Tj.total, 1) * sizeof(double), st));
  const Fused fr = fuse(c->bonds[i + 2], true);
  // right-fused buffer for the new site i+1 (D' x fused_R)
  DevBuf rfb;
  std::vector<int64_t> rfo(wb.size(), -1);
  int64_t rft = 0;
  for (size_t w = 0; w < wb.size(); ++w)
    if (keep[w] > 0) {
      rfo[w] = rft;
      rft += (int64_t)keep[w] * wb[w].cols;
    }
  rfb.ensure(std::max<int64_t>(rft, 1));
  CK(cudaMemsetAsync(rfb.p, 0, (size_t)std::max<int64_t>(rft, 1) * sizeof(double), st));   // gather accumulates
  std::vector<GemmOut> outs;
  std::vector<GemmSeg> segs;
  std::vector<GatherTask> gt;
  std::vector<GatherSrc> gs;
  for (size_t w = 0; w < wb.size(); ++w) {
    if (keep[w] == 0) continue;
    const WfnBlock& b = wb[w];
    const int q = wsec[w], d = keep[w];
    const double* vecs = rho.p + roff[w] + (int64_t)(rdim[w] - d) * rdim[w];   // d rows of length rdim
    if (dir > 0) {
      // site i block (rows x d) = vecs^T ; centre (d x cols) = vecs psi
      gt.push_back(GatherTask{Ti.d + Ti.blk_off[q], d, b.rows, d, (int)gs.size(), 1});
      gs.push_back(GatherSrc{vecs, rdim[w], 1, 1.0});
      outs.push_back(GemmOut{rfb.p + rfo[w], 0, b.cols, d, b.cols, (int)segs.size(), 1, 0, 0});
      segs.push_back(GemmSeg{vecs, psi + b.off, 0, 0, rdim[w], b.cols, b.rows, 0, 0, 0, 0, 1.0});
    } else {
      // site i+1 right-fused block (d x cols) = vecs ; centre on site i (rows x d) = psi vecs^T
      gt.push_back(GatherTask{rfb.p + rfo[w], b.cols, d, b.cols, (int)gs.size(), 1});
      gs.push_back(GatherSrc{vecs, rdim[w], 0, 1.0});
      outs.push_back(GemmOut{Ti.d + Ti.blk_off[q], 0, d, b.rows, d, (int)segs.size(), 1, 0, 0});
      segs.push_back(GemmSeg{psi + b.off, vecs, 0, 0, b.cols, rdim[w], b.cols, 0, 1, 0, 0, 1.0});
    }
  }
  {
    GatherPlan gp;
    build_gather(gp, gt, gs, st);
    gp.run(st);
    GemmPlan mp;
    build_gemm(mp, outs, segs, st);
    mp.run(st, nullptr, nullptr);
  }
  // right-fused (d x fused_R) -> left-fused storage of site i+1
  {
    std::vector<GatherTask> t2;
    std::vector<GatherSrc> s2;
    for (size_t w = 0; w < wb.size(); ++w) {
      if (keep[w] == 0) continue;
      const int q = wsec[w];
      const int f = fr.s.find(wb[w].label_a, wb[w].label_b);
      for (int n = 0; n < 4; ++n) {
        if (Tj.sub_off[q][n] < 0) continue;
        const int Dr = c->bonds[i + 2].d[Tj.sub_qr[q][n]];
        t2.push_back(GatherTask{Tj.d + Tj.sub_off[q][n], Dr, keep[w], Dr, (int)s2.size(), 1});
        s2.push_back(GatherSrc{rfb.p + rfo[w] + fr.off[f][n], wb[w].cols, 0, 1.0});
      }
    }
    GatherPlan gp;
    build_gather(gp, t2, s2, st);
    gp.run(st);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  upload_site(c, i, std::move(Ti));
  upload_site(c, i + 1, std::move(Tj));
  return disc;
}

static double sweep_gs_impl(lrt_ctx* c, const lrt_gs_params& P, int* nsw) {
  const int k = c->k;
  if (k < 2) throw Error(LRT_EINVAL, "sweep_gs: needs at least two sites");
  c->sites_r.clear();
  drop_plans(c);
  for (int b = 0; b < k; ++b) {
    c->XL[b].reset();
    c->YR[b].reset();
  }
  for (int b = 1; b < k; ++b) c->L[b].reset();
  for (int b = 0; b < k; ++b) c->R[b].reset();
  for (int b = k - 1; b >= 1; --b) renorm_right(c, b);   // sites right-orthonormal, centre at 0
  SolverHandle sh;
  DevBuf psi;
  double E = 0.0, Eprev = 0.0;
  int sweep = 0;
  for (; sweep < P.max_sweeps; ++sweep) {
    const int si = std::min(sweep / std::max(1, P.sweeps_per_M), P.n_schedule - 1);
    const int M = P.M_schedule[si];
    for (int dir : {+1, -1}) {
      for (int step = 0; step < k - 1; ++step) {
        const int i = dir > 0 ? step : k - 2 - step;
        std::vector<WfnBlock> wb = wfn_blocks(c, i, 2);
        int64_t n = 0;
        for (auto& w : wb) n = std::max(n, w.off + (int64_t)w.rows * w.cols);
        psi.ensure(n);
        form_theta(c, i, psi.p, wb);
        int its = 0;
        E = davidson_site(c, i, 2, psi.p, P, &its);
        decimate(c, i, psi.p, wb, M, P.trunc_tol, dir, sh);
        drop_plans(c);
        if (dir > 0) {
          c->R[i + 1].reset();
          c->YR[i].reset();
          renorm_left(c, i);
        } else {
          c->L[i + 1].reset();
          c->XL[i + 1].reset();
          renorm_right(c, i + 1);
        }
      }
    }
    if (sweep > 0 && sweep / std::max(1, P.sweeps_per_M) >= P.n_schedule - 1 && std::fabs(E - Eprev) < P.e_tol) {
      ++sweep;
      break;
    }
    Eprev = E;
  }
  if (nsw) *nsw = sweep;
  return E;
}

}  // namespace lrt

// ===========================================================================
// DMRG-TDA sweep (Fig. alg:dmrgtda): block Davidson through forward and backward
// sweeps with first-order renormalized operators
// ===========================================================================
namespace lrt {

struct TdaState {
  std::vector<SiteTensor> C0;                 // C0_i, left-fused
  std::vector<std::vector<double>> lam;       // Schmidt values per bond, concatenated by sector
  bool loaded = false;
};

// dense bond matrices (one D x D block per sector of a bond)
struct BondMat {
  std::vector<int64_t> off;
  DevBuf buf;
};

static void bond_layout(const Sectors& S, BondMat& M, cudaStream_t st) {
  M.off.assign(S.n(), 0);
  int64_t t = 0;
  for (int q = 0; q < S.n(); ++q) {
    M.off[q] = t;
    t += (int64_t)S.d[q] * S.d[q];
  }
  M.buf.ensure(std::max<int64_t>(t, 1));
  CK(cudaMemsetAsync(M.buf.p, 0, (size_t)std::max<int64_t>(t, 1) * sizeof(double), st));
}

static SiteTensor new_site(lrt_ctx* c, int i) {
  SiteTensor T;
  site_layout(T, c->bonds[i], c->bonds[i + 1]);
  if (dev_alloc((void**)&T.d, (size_t)std::max<int64_t>(T.total, 1) * sizeof(double)) != cudaSuccess)
    throw Error(LRT_ENOMEM, "site tensor");
  CK(cudaMemsetAsync(T.d, 0, (size_t)std::max<int64_t>(T.total, 1) * sizeof(double), c->st));
  return T;
}

static void run_gemms(lrt_ctx* c, const std::vector<GemmOut>& o, const std::vector<GemmSeg>& g) {
  if (o.empty()) return;
  GemmPlan p;
  build_gemm(p, o, g, c->st);
  p.run(c->st, nullptr, nullptr);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
}

static double t_dot(lrt_ctx* c, const SiteTensor& A, const SiteTensor& B, DevBuf& tmp) {
  tmp.ensure(4);
  return dev_dot(A.d, B.d, A.total, tmp.p, c->st);
}

// Y = a X + b Y
static void t_axpby(lrt_ctx* c, double a, const SiteTensor& X, double b, SiteTensor& Y, DevBuf& tmp) {
  tmp.ensure(4);
  CK(cudaMemcpyAsync(tmp.p, &a, sizeof(double), cudaMemcpyHostToDevice, c->st));
  launch_lincomb(X.d, X.total, 1, tmp.p, Y.total, Y.d, b, c->st);
  CK(cudaStreamSynchronize(c->st));
}

// out_q = A_q^T B_q for every right sector q (bond i+1)
static void t_lc(lrt_ctx* c, int i, const SiteTensor& A, const SiteTensor& B, BondMat& out) {
  const Sectors& R = c->bonds[i + 1];
  bond_layout(R, out, c->st);
  std::vector<GemmOut> o;
  std::vector<GemmSeg> g;
  for (int q = 0; q < R.n(); ++q) {
    if (A.blk_off[q] < 0) continue;
    const int D = R.d[q];
    o.push_back(GemmOut{out.buf.p + out.off[q], 0, D, D, D, (int)g.size(), 1, 0, 0});
    g.push_back(GemmSeg{A.d + A.blk_off[q], B.d + B.blk_off[q], 0, 0, D, D, A.blk_rows[q], 1, 0, 0, 0, 1.0});
  }
  run_gemms(c, o, g);
}

// out = A X (X on the right bond i+1), or out += when acc
static void t_rmul(lrt_ctx* c, int i, const SiteTensor& A, const BondMat& X, SiteTensor& out, bool acc) {
  const Sectors& R = c->bonds[i + 1];
  std::vector<GemmOut> o;
  std::vector<GemmSeg> g;
  for (int q = 0; q < R.n(); ++q) {
    if (A.blk_off[q] < 0) continue;
    const int D = R.d[q];
    o.push_back(GemmOut{out.d + out.blk_off[q], 0, D, A.blk_rows[q], D, (int)g.size(), 1, acc ? 1 : 0, 0});
    g.push_back(GemmSeg{A.d + A.blk_off[q], X.buf.p + X.off[q], 0, 0, D, D, D, 0, 0, 0, 0, 1.0});
  }
  run_gemms(c, o, g);
}

// out_ql = sum_n A(ql, n) B(ql, n)^T for every left sector ql (bond i)
static void t_rc(lrt_ctx* c, int i, const SiteTensor& A, const SiteTensor& B, BondMat& out) {
  const Sectors& L = c->bonds[i];
  bond_layout(L, out, c->st);
  std::vector<GemmOut> o;
  std::vector<GemmSeg> g;
  for (int q = 0; q < L.n(); ++q) {
    const int D = L.d[q];
    GemmOut x{out.buf.p + out.off[q], 0, D, D, D, (int)g.size(), 0, 0, 0};
    for (int n = 0; n < 4; ++n) {
      if (A.sub_off[q][n] < 0) continue;
      const int Dr = c->bonds[i + 1].d[A.sub_qr[q][n]];
      g.push_back(GemmSeg{A.d + A.sub_off[q][n], B.d + B.sub_off[q][n], 0, 0, Dr, Dr, Dr, 0, 1, 0, 0, 1.0});
      ++x.seg_count;
    }
    if (x.seg_count) o.push_back(x);
  }
  run_gemms(c, o, g);
}

// out = X A (X on the left bond i), or out += when acc
static void t_lmul(lrt_ctx* c, int i, const BondMat& X, const SiteTensor& A, SiteTensor& out, bool acc) {
  const Sectors& L = c->bonds[i];
  std::vector<GemmOut> o;
  std::vector<GemmSeg> g;
  for (int q = 0; q < L.n(); ++q)
    for (int n = 0; n < 4; ++n) {
      if (A.sub_off[q][n] < 0) continue;
      const int D = L.d[q];
      const int Dr = c->bonds[i + 1].d[A.sub_qr[q][n]];
      o.push_back(GemmOut{out.d + A.sub_off[q][n], 0, Dr, D, Dr, (int)g.size(), 1, acc ? 1 : 0, 0});
      g.push_back(GemmSeg{X.buf.p + X.off[q], A.d + A.sub_off[q][n], 0, 0, D, Dr, D, 0, 0, 0, 0, 1.0});
    }
  run_gemms(c, o, g);
}

static void lam_mats(lrt_ctx* c, int b, const std::vector<double>& lam, double cut, BondMat& L, BondMat& Li) {
  const Sectors& S = c->bonds[b];
  bond_layout(S, L, c->st);
  bond_layout(S, Li, c->st);
  double smax = 0.0;
  for (double x : lam) smax = std::max(smax, x);
  std::vector<double> hl(L.buf.n, 0.0), hi(L.buf.n, 0.0);
  int64_t pos = 0;
  for (int q = 0; q < S.n(); ++q) {
    for (int a = 0; a < S.d[q]; ++a) {
      const double x = lam[pos + a];
      hl[L.off[q] + (int64_t)a * S.d[q] + a] = x;
      hi[L.off[q] + (int64_t)a * S.d[q] + a] = (x > cut * smax) ? 1.0 / x : 0.0;
    }
    pos += S.d[q];
  }
  CK(cudaMemcpyAsync(L.buf.p, hl.data(), hl.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(Li.buf.p, hi.data(), hi.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
}

// an operator set with the layout of `t` and zero data
static std::unique_ptr<OpSet> clone_layout(lrt_ctx* c, const OpSet& t) {
  auto S = std::make_unique<OpSet>();
  S->basis = t.basis;
  S->right = t.right;
  S->orbs = t.orbs;
  S->in = t.in;
  S->mode = t.mode;
  S->keys = t.keys;
  S->index = t.index;
  S->da = t.da;
  S->db = t.db;
  S->par = t.par;
  S->bra = t.bra;
  S->off = t.off;
  S->total = t.total;
  S->bnz = t.bnz;
  S->onz = t.onz;
  S->mask = t.mask;
  if (t.fused) S->fused = std::make_unique<Fused>(*t.fused);
  alloc_zero(*S, c->st);
  return S;
}

struct FirstOrder {           // a first-order operator set and its reverse set
  std::unique_ptr<OpSet> f, r;
  bool empty() const { return !f; }
};

static double splitmix_normal(uint64_t seed, uint64_t idx) {
  auto sm = [](uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const uint64_t g = 0x9E3779B97F4A7C15ull;
  const uint64_t z1 = sm(seed + (2 * idx + 1) * g), z2 = sm(seed + (2 * idx + 2) * g);
  const double u1 = ((double)(z1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((double)(z2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

// ---------------------------------------------------------------------------
// One-site ground-state sweeps (Eq. dmrg at one site, bond dimensions fixed), which
// make the reference a stationary point of the one-site manifold as the TDA assumes.
// Gauge shifts by per-sector SVDs (cuSOLVER Jacobi SVD): left to right
// C_i = L S V^T per right sector, L_i = L, C_{i+1} = (S V^T) R_{i+1}; right to left
// C_i = U S R per left sector (right-fused rows), R_i = R, C_{i-1} = L_{i-1} (U S).
// A sector with fewer fused states than bond states keeps zero singular values.
// ---------------------------------------------------------------------------
struct SvdWork {
  SolverHandle sh;
  gesvdjInfo_t params = nullptr;
  int* info = nullptr;
  DevBuf work, A, U, V, S;
  explicit SvdWork(cudaStream_t st) {
    if (cusolverDnCreate(&sh.h) != CUSOLVER_STATUS_SUCCESS) throw Error(LRT_ECUDA, "cusolverDnCreate failed");
    cusolverDnSetStream(sh.h, st);
    if (cusolverDnCreateGesvdjInfo(&params) != CUSOLVER_STATUS_SUCCESS) throw Error(LRT_ECUDA, "gesvdj info");
    if (dev_alloc((void**)&info, sizeof(int)) != cudaSuccess) throw Error(LRT_ENOMEM, "cusolver info");
  }
  ~SvdWork() {
    if (params) cusolverDnDestroyGesvdjInfo(params);
    dev_free(info);
  }
  // full SVD of the column-major m x n matrix at src (copied first): U (m x m), V (n x n)
  // left in U, V; returns the min(m, n) singular values (descending)
  std::vector<double> svd(const double* src, int m, int n, cudaStream_t st) {
    const int p = std::min(m, n);
    A.ensure((size_t)m * n);
    U.ensure((size_t)m * m);
    V.ensure((size_t)n * n);
    S.ensure(std::max(1, p));
    CK(cudaMemcpyAsync(A.p, src, (size_t)m * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int lwork = 0;
    if (cusolverDnDgesvdj_bufferSize(sh.h, CUSOLVER_EIG_MODE_VECTOR, 0, m, n, A.p, m, S.p, U.p, m, V.p, n, &lwork,
                                     params) != CUSOLVER_STATUS_SUCCESS)
      throw Error(LRT_ECUDA, "gesvdj buffer size");
    work.ensure(std::max(lwork, 1));
    if (cusolverDnDgesvdj(sh.h, CUSOLVER_EIG_MODE_VECTOR, 0, m, n, A.p, m, S.p, U.p, m, V.p, n, work.p, lwork, info,
                          params) != CUSOLVER_STATUS_SUCCESS)
      throw Error(LRT_ECUDA, "gesvdj");
    std::vector<double> s(p);
    int h = 0;
    CK(cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(s.data(), S.p, p * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h < 0) throw Error(LRT_ECUDA, "gesvdj: invalid argument " + std::to_string(-h));
    return s;
  }
};

static void run_gathers(lrt_ctx* c, std::vector<GatherTask>& t, std::vector<GatherSrc>& s) {
  if (t.empty()) return;
  GatherPlan gp;
  build_gather(gp, t, s, c->st);
  gp.run(c->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
}

// M = X diag(w) (X: D x D bond blocks; per sector the weights w in sector order)
static void scale_cols(lrt_ctx* c, int b, const BondMat& X, const std::vector<double>& w, BondMat& out) {
  BondMat Lm, Lmi;
  lam_mats(c, b, w, 0.0, Lm, Lmi);
  const Sectors& S = c->bonds[b];
  bond_layout(S, out, c->st);
  std::vector<GemmOut> o;
  std::vector<GemmSeg> g;
  for (int q = 0; q < S.n(); ++q) {
    const int D = S.d[q];
    if (D == 0) continue;
    o.push_back(GemmOut{out.buf.p + out.off[q], 0, D, D, D, (int)g.size(), 1, 0, 0});
    g.push_back(GemmSeg{X.buf.p + X.off[q], Lm.buf.p + Lm.off[q], 0, 0, D, D, D, 0, 0, 0, 0, 1.0});
  }
  run_gemms(c, o, g);
}

// centre psi at site i -> L_i and the new centre at site i+1
static void gauge_shift_right(lrt_ctx* c, int i, const double* psi, SvdWork& W) {
  const Sectors& Rb = c->bonds[i + 1];
  const SiteTensor& T = c->sites[i];
  SiteTensor L = new_site(c, i);
  BondMat UT;               // per sector: U_a^T (row a = right singular vector a), D x D
  bond_layout(Rb, UT, c->st);
  std::vector<double> lam;
  std::vector<GatherTask> tasks;
  std::vector<GatherSrc> srcs;
  std::vector<DevBuf> keepU, keepV;
  for (int q = 0; q < Rb.n(); ++q) {
    const int D = Rb.d[q];
    const int rows = T.blk_off[q] >= 0 ? T.blk_rows[q] : 0;
    if (D == 0) continue;
    if (rows == 0) {
      std::vector<double> I((size_t)D * D, 0.0);
      for (int a = 0; a < D; ++a) I[(size_t)a * D + a] = 1.0;
      CK(cudaMemcpyAsync(UT.buf.p + UT.off[q], I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
      CK(cudaStreamSynchronize(c->st));
      lam.insert(lam.end(), D, 0.0);
      continue;
    }
    // the row-major block M (rows x D) is the column-major D x rows matrix M^T = U_a S V_a^T
    const std::vector<double> sv = W.svd(psi + T.blk_off[q], D, rows, c->st);
    const int p = (int)sv.size();
    for (int a = 0; a < D; ++a) lam.push_back(a < p ? sv[a] : 0.0);
    keepU.emplace_back();
    keepV.emplace_back();
    DevBuf& u = keepU.back();
    DevBuf& v = keepV.back();
    u.ensure((size_t)D * D);
    v.ensure((size_t)rows * rows);
    CK(cudaMemcpyAsync(u.p, W.U.p, (size_t)D * D * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(v.p, W.V.p, (size_t)rows * rows * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    // L block (rows x D): columns a < p = V_a's columns; U_a^T row-major = U_a's memory
    tasks.push_back(GatherTask{L.d + L.blk_off[q], D, rows, p, (int)srcs.size(), 1});
    srcs.push_back(GatherSrc{v.p, rows, 1, 1.0});
    tasks.push_back(GatherTask{UT.buf.p + UT.off[q], D, D, D, (int)srcs.size(), 1});
    srcs.push_back(GatherSrc{u.p, D, 0, 1.0});
  }
  run_gathers(c, tasks, srcs);
  // S V^T of the block = diag(lam) U_a^T; the next centre = (diag(lam) U_a^T) R_{i+1}
  BondMat UTt, X;
  bond_layout(Rb, UTt, c->st);
  {
    std::vector<GatherTask> t2;
    std::vector<GatherSrc> s2;
    for (int q = 0; q < Rb.n(); ++q) {
      const int D = Rb.d[q];
      if (D == 0) continue;
      t2.push_back(GatherTask{UTt.buf.p + UTt.off[q], D, D, D, (int)s2.size(), 1});
      s2.push_back(GatherSrc{UT.buf.p + UT.off[q], D, 1, 1.0});
    }
    run_gathers(c, t2, s2);
  }
  scale_cols(c, i + 1, UTt, lam, X);          // X^T = U_a diag(lam)  ->  X = diag(lam) U_a^T
  BondMat Xs;
  bond_layout(Rb, Xs, c->st);
  {
    std::vector<GatherTask> t3;
    std::vector<GatherSrc> s3;
    for (int q = 0; q < Rb.n(); ++q) {
      const int D = Rb.d[q];
      if (D == 0) continue;
      t3.push_back(GatherTask{Xs.buf.p + Xs.off[q], D, D, D, (int)s3.size(), 1});
      s3.push_back(GatherSrc{X.buf.p + X.off[q], D, 1, 1.0});
    }
    run_gathers(c, t3, s3);
  }
  SiteTensor next = new_site(c, i + 1);
  t_lmul(c, i + 1, Xs, c->sites[i + 1], next, false);
  c->sites[i] = std::move(L);
  c->sites[i + 1] = std::move(next);
}

// centre psi at site i -> R_i and the new centre at site i-1
static void gauge_shift_left(lrt_ctx* c, int i, const double* psi, SvdWork& W) {
  const Sectors& Lb = c->bonds[i];
  const Sectors& Rb = c->bonds[i + 1];
  const SiteTensor& T = c->sites[i];
  SiteTensor R = new_site(c, i);
  BondMat Y;                 // per left sector: V_a (row-major), scaled by the singular values below
  bond_layout(Lb, Y, c->st);
  std::vector<double> lam;
  std::vector<DevBuf> keep;
  for (int q = 0; q < Lb.n(); ++q) {
    const int D = Lb.d[q];
    if (D == 0) continue;
    // right-fused block (D x Wd): the sub-blocks (q, n) side by side
    int Wd = 0;
    std::array<int, 4> coff{-1, -1, -1, -1};
    for (int n = 0; n < 4; ++n)
      if (T.sub_off[q][n] >= 0) {
        coff[n] = Wd;
        Wd += Rb.d[T.sub_qr[q][n]];
      }
    if (Wd == 0) {
      std::vector<double> I((size_t)D * D, 0.0);
      for (int a = 0; a < D; ++a) I[(size_t)a * D + a] = 1.0;
      CK(cudaMemcpyAsync(Y.buf.p + Y.off[q], I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
      CK(cudaStreamSynchronize(c->st));
      lam.insert(lam.end(), D, 0.0);
      continue;
    }
    DevBuf rf;
    rf.ensure((size_t)D * Wd);
    CK(cudaMemsetAsync(rf.p, 0, (size_t)D * Wd * sizeof(double), c->st));
    std::vector<GatherTask> tg;
    std::vector<GatherSrc> sg;
    for (int n = 0; n < 4; ++n)
      if (coff[n] >= 0) {
        const int Dr = Rb.d[T.sub_qr[q][n]];
        tg.push_back(GatherTask{rf.p + coff[n], Wd, D, Dr, (int)sg.size(), 1});
        sg.push_back(GatherSrc{psi + T.sub_off[q][n], Dr, 0, 1.0});
      }
    run_gathers(c, tg, sg);
    // row-major RF (D x Wd) = column-major Wd x D matrix RF^T = U_a S V_a^T, so RF = V_a S U_a^T
    const std::vector<double> sv = W.svd(rf.p, Wd, D, c->st);
    const int p = (int)sv.size();
    for (int a = 0; a < D; ++a) lam.push_back(a < p ? sv[a] : 0.0);
    // R rows a < p: U_a^T (row-major = U_a's memory, ld Wd), scattered back to the sub-blocks
    DevBuf rr;
    rr.ensure((size_t)D * Wd);
    CK(cudaMemsetAsync(rr.p, 0, (size_t)D * Wd * sizeof(double), c->st));
    std::vector<GatherTask> t1;
    std::vector<GatherSrc> s1;
    t1.push_back(GatherTask{rr.p, Wd, p, Wd, 0, 1});
    s1.push_back(GatherSrc{W.U.p, Wd, 0, 1.0});
    t1.push_back(GatherTask{Y.buf.p + Y.off[q], D, D, p, 1, 1});       // V_a (D x D), columns a < p
    s1.push_back(GatherSrc{W.V.p, D, 1, 1.0});
    run_gathers(c, t1, s1);
    std::vector<GatherTask> t2;
    std::vector<GatherSrc> s2;
    for (int n = 0; n < 4; ++n)
      if (coff[n] >= 0) {
        const int Dr = Rb.d[T.sub_qr[q][n]];
        t2.push_back(GatherTask{R.d + T.sub_off[q][n], Dr, D, Dr, (int)s2.size(), 1});
        s2.push_back(GatherSrc{rr.p + coff[n], Wd, 0, 1.0});
      }
    run_gathers(c, t2, s2);
  }
  BondMat US;
  scale_cols(c, i, Y, lam, US);                 // U S of the right-fused SVD
  SiteTensor prev = new_site(c, i - 1);
  t_rmul(c, i - 1, c->sites[i - 1], US, prev, false);
  c->sites[i] = std::move(R);
  c->sites[i - 1] = std::move(prev);
}

static double sweep_onesite_impl(lrt_ctx* c, const lrt_gs_params& P, int nsweeps) {
  const int k = c->k;
  SvdWork W(c->st);
  DevBuf psi;
  double E = 0.0;
  for (int sweep = 0; sweep < nsweeps; ++sweep) {
    for (int i = 0; i + 1 < k; ++i) {
      const SiteTensor& C = c->sites[i];
      psi.ensure((size_t)std::max<int64_t>(C.total, 1));
      CK(cudaMemcpyAsync(psi.p, C.d, (size_t)C.total * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      int its = 0;
      E = davidson_site(c, i, 1, psi.p, P, &its);
      gauge_shift_right(c, i, psi.p, W);
      drop_plans(c);
      c->R[i + 1].reset();
      c->YR[i].reset();
      renorm_left(c, i);
    }
    for (int i = k - 1; i >= 1; --i) {
      const SiteTensor& C = c->sites[i];
      psi.ensure((size_t)std::max<int64_t>(C.total, 1));
      CK(cudaMemcpyAsync(psi.p, C.d, (size_t)C.total * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      int its = 0;
      E = davidson_site(c, i, 1, psi.p, P, &its);
      gauge_shift_left(c, i, psi.p, W);
      drop_plans(c);
      c->L[i].reset();
      c->XL[i].reset();
      renorm_right(c, i);
    }
  }
  return E;
}

// ---------------------------------------------------------------------------
// batched site algebra of the TDA sweeps
// ---------------------------------------------------------------------------
// nv site tensors of one site's layout, contiguous (stride = the layout's size); capacity
// rounded up to whole blocks of `block` vectors, so multi-vector sigma calls can run on
// whole blocks (the padding vectors are zero)
struct SiteBatch {
  int nv = 0;
  int64_t stride = 0;
  DevBuf buf;
  double* v(int j) const { return buf.p + (int64_t)j * stride; }
};

static void batch_alloc(lrt_ctx* c, SiteBatch& B, int64_t stride, int nv, int block) {
  B.nv = nv;
  B.stride = std::max<int64_t>(stride, 1);
  const int cap = std::max(1, (nv + block - 1) / block * block);
  B.buf.ensure((size_t)cap * B.stride);
  CK(cudaMemsetAsync(B.buf.p, 0, (size_t)cap * B.stride * sizeof(double), c->st));
}

// nv dense bond matrices of one bond's layout (one D x D block per sector), contiguous
struct BondBatch {
  std::vector<int64_t> off;
  int64_t stride = 0;
  int nv = 0;
  DevBuf buf;
};

static void bond_batch(lrt_ctx* c, int b, BondBatch& B, int nv) {
  const Sectors& S = c->bonds[b];
  B.off.assign(S.n(), 0);
  int64_t t = 0;
  for (int q = 0; q < S.n(); ++q) {
    B.off[q] = t;
    t += (int64_t)S.d[q] * S.d[q];
  }
  B.stride = std::max<int64_t>(t, 1);
  B.nv = nv;
  B.buf.ensure((size_t)std::max(nv, 1) * B.stride);
  CK(cudaMemsetAsync(B.buf.p, 0, (size_t)std::max(nv, 1) * B.stride * sizeof(double), c->st));
}

// nv first-order operator sets of one bond (both directions), one layout each
struct SetBatch {
  std::unique_ptr<OpSet> fp, rp;   // layouts (no data)
  uint64_t sig = 0;                // set_signature(fp, rp)
  int64_t fs = 0, rs = 0;          // strides
  int nv = 0;
  DevBuf f, r;
  bool empty() const { return !fp; }
  double* fv(int j) const { return f.p + (int64_t)j * fs; }
  double* rv(int j) const { return r.p + (int64_t)j * rs; }
};

static void set_batch(lrt_ctx* c, SetBatch& B, const OpSet& f, const OpSet& r, int nv) {
  B.fp = layout_copy(f);
  B.rp = layout_copy(r);
  B.sig = set_signature(*B.fp, B.rp.get());
  B.fs = std::max<int64_t>(f.total, 1);
  B.rs = std::max<int64_t>(r.total, 1);
  B.nv = nv;
  B.f.ensure((size_t)std::max(nv, 1) * B.fs);
  B.r.ensure((size_t)std::max(nv, 1) * B.rs);
  CK(cudaMemsetAsync(B.f.p, 0, (size_t)std::max(nv, 1) * B.fs * sizeof(double), c->st));
  CK(cudaMemsetAsync(B.r.p, 0, (size_t)std::max(nv, 1) * B.rs * sizeof(double), c->st));
}

// a site tensor that borrows its data (a slot of a batch) and never frees it
struct SiteView {
  SiteTensor t;
  SiteView(const SiteTensor& lay, double* p) {
    t.blk_off = lay.blk_off;
    t.blk_rows = lay.blk_rows;
    t.sub_off = lay.sub_off;
    t.sub_qr = lay.sub_qr;
    t.total = lay.total;
    t.d = p;
  }
  ~SiteView() { t.d = nullptr; }
};

struct TdaRunner {
  lrt_ctx* c;
  int k;
  const lrt_tda_params& P;
  std::vector<BondMat> lam, ilam;
  std::vector<DevBuf> diag;
  std::vector<SiteTensor> lay;       // layout of every site (no data)
  std::vector<std::unique_ptr<SigmaPlan>> h0one;   // H_0^[i] plans for one vector
  std::map<std::pair<int, int>, std::unique_ptr<SigmaPlan>> h0blk;   // (site, block) plans
  DevBuf tmp;
  double E0 = 0.0;
  bool mixed = false;   // site products on the tensor cores (until the FP64 refinement)
  int blk = 1;          // vectors per multi-vector H_0 call (the number of roots)

  TdaRunner(lrt_ctx* cc, const lrt_tda_params& p) : c(cc), k(cc->k), P(p), mixed(p.precision == LRT_MIXED) {}

  const SiteTensor& L0(int i) { return c->sites[i]; }
  const SiteTensor& R0(int i) { return c->sites_r[i]; }
  const SiteTensor& C0(int i) { return c->tda->C0[i]; }
  int64_t T(int i) const { return lay[i].total; }

  void setup() {
    lam.resize(k + 1);
    ilam.resize(k + 1);
    for (int b = 0; b <= k; ++b) lam_mats(c, b, c->tda->lam[b], P.pinv_cut, lam[b], ilam[b]);
    // zeroth-order environments: left blocks from L0, right blocks from R0
    for (int b = 0; b + 1 < k; ++b) renorm_left(c, b);
    for (int b = k - 1; b >= 1; --b) renorm_right(c, b);
    for (int i = 0; i < k; ++i) {
      enlarged(c, i, false);
      if (i > 0) enlarged(c, i, true);
    }
    lay.resize(k);
    h0one.resize(k);
    diag.resize(k);
    for (int i = 0; i < k; ++i) {
      site_layout(lay[i], c->bonds[i], c->bonds[i + 1]);
      h0one[i] = plan_sigma_sets(c, *c->XL[i], nullptr, *c->R[i + 1], nullptr, i, 1, 1, false);
      diag[i].ensure(std::max<int64_t>(h0one[i]->nelem, 1));
      launch_diag(h0one[i]->douts.p, h0one[i]->dterms.p, h0one[i]->ndiag, diag[i].p, c->st);
    }
    SiteTensor y = new_site(c, 0);
    run_plan(*h0one[0], C0(0).d, y.d, 1, false);    // the reference energy is FP64
    E0 = t_dot(c, C0(0), y, tmp);
  }

  void run_plan(SigmaPlan& p, const double* x, double* y, int nvec, bool tc) {
    if (tc) {
      run_tc(c, p, x, y, nvec);
    } else {
      p.p1.run(c->st, x, y, p.tbuf, &p.ex);
      p.p2.run(c->st, x, y, p.tbuf, &p.ex);
      CK(cudaGetLastError());
    }
  }

  // Y = H_0^[i] X for the first nv vectors of a batch (Eq. hzero_sb), as multi-vector sigma
  // calls on whole blocks of `blk` vectors (the block-Davidson right-hand sides)
  void h0(int i, const SiteBatch& X, int nv, SiteBatch& Y) {
    auto& p = h0blk[{i, blk}];
    if (!p) p = plan_sigma_sets(c, *c->XL[i], nullptr, *c->R[i + 1], nullptr, i, 1, blk, mixed);
    if (mixed && !p->has_tc) p = plan_sigma_sets(c, *c->XL[i], nullptr, *c->R[i + 1], nullptr, i, 1, blk, true);
    for (int v0 = 0; v0 < nv; v0 += blk) run_plan(*p, X.v(v0), Y.v(v0), blk, mixed);
  }

  // ---- batched bond/site products: grouped GEMMs planned once per (kind, site, nv) with
  // every per-vector address relative to extra bases 0 (batched A), 1 (batched B) and 2
  // (output), replayed for new batches ----
  enum { K_LC, K_RMUL, K_RMULB, K_RC, K_LMUL, K_LMULB };
  std::map<std::tuple<int, int, int, int, int, const void*>, std::unique_ptr<GemmPlan>> bops;
  GemmPlan& bop(int kind, int i, int nv, bool acc, double scale, const void* fixed, int64_t sa, int64_t sb,
                int64_t so, const std::vector<int64_t>* boff) {
    const int sgn = scale < 0 ? -1 : 1;
    auto& p = bops[std::make_tuple(kind, i, nv, acc ? 1 : 0, sgn, fixed)];
    if (p) return *p;
    std::vector<GemmOut> o;
    std::vector<GemmSeg> g;
    const SiteTensor& L = lay[i];
    const int A0 = 3, B1 = 4, O2 = 5;
    for (int v = 0; v < nv; ++v) {
      if (kind == K_LC || kind == K_RMUL || kind == K_RMULB) {
        // per right sector q of bond i+1
        const Sectors& R = c->bonds[i + 1];
        for (int q = 0; q < R.n(); ++q) {
          if (L.blk_off[q] < 0) continue;
          const int D = R.d[q], rows = L.blk_rows[q];
          const int64_t bo = L.blk_off[q];
          if (kind == K_LC) {            // out_v = A^T B_v   (A fixed, B batched)
            const SiteTensor& A = *(const SiteTensor*)fixed;
            o.push_back(GemmOut{nullptr, (*boff)[q] + v * so, D, D, D, (int)g.size(), 1, acc ? 1 : 0, O2, 0});
            g.push_back(GemmSeg{A.d + bo, nullptr, 0, bo + v * sb, D, D, rows, 1, 0, 0, B1, scale});
          } else if (kind == K_RMUL) {   // out_v = A_v X     (X fixed bond matrices)
            const BondMat& X = *(const BondMat*)fixed;
            o.push_back(GemmOut{nullptr, bo + v * so, D, rows, D, (int)g.size(), 1, acc ? 1 : 0, O2, 0});
            g.push_back(GemmSeg{nullptr, X.buf.p + X.off[q], bo + v * sa, 0, D, D, D, 0, 0, A0, 0, scale});
          } else {                       // out_v = A X_v     (A fixed, X batched)
            const SiteTensor& A = *(const SiteTensor*)fixed;
            o.push_back(GemmOut{nullptr, bo + v * so, D, rows, D, (int)g.size(), 1, acc ? 1 : 0, O2, 0});
            g.push_back(GemmSeg{A.d + bo, nullptr, 0, (*boff)[q] + v * sb, D, D, D, 0, 0, 0, B1, scale});
          }
        }
      } else if (kind == K_RC) {         // out_v,ql = sum_n A_v(ql,n) B(ql,n)^T  (B fixed)
        const SiteTensor& Bf = *(const SiteTensor*)fixed;
        const Sectors& Lb = c->bonds[i];
        for (int q = 0; q < Lb.n(); ++q) {
          const int D = Lb.d[q];
          GemmOut x{nullptr, (*boff)[q] + v * so, D, D, D, (int)g.size(), 0, acc ? 1 : 0, O2, 0};
          for (int n = 0; n < 4; ++n) {
            if (L.sub_off[q][n] < 0) continue;
            const int Dr = c->bonds[i + 1].d[L.sub_qr[q][n]];
            g.push_back(GemmSeg{nullptr, Bf.d + L.sub_off[q][n], L.sub_off[q][n] + v * sa, 0, Dr, Dr, Dr, 0, 1, A0,
                                0, scale});
            ++x.seg_count;
          }
          if (x.seg_count) o.push_back(x);
        }
      } else {                           // per (ql, n) sub-block
        const Sectors& Lb = c->bonds[i];
        for (int q = 0; q < Lb.n(); ++q)
          for (int n = 0; n < 4; ++n) {
            if (L.sub_off[q][n] < 0) continue;
            const int D = Lb.d[q];
            const int Dr = c->bonds[i + 1].d[L.sub_qr[q][n]];
            const int64_t so_ = L.sub_off[q][n];
            o.push_back(GemmOut{nullptr, so_ + v * so, Dr, D, Dr, (int)g.size(), 1, acc ? 1 : 0, O2, 0});
            if (kind == K_LMUL) {        // out_v = X A_v   (X fixed bond matrices)
              const BondMat& X = *(const BondMat*)fixed;
              g.push_back(GemmSeg{X.buf.p + X.off[q], nullptr, 0, so_ + v * sb, D, Dr, D, 0, 0, 0, B1, scale});
            } else {                     // out_v = X_v A   (A fixed, X batched)
              const SiteTensor& A = *(const SiteTensor*)fixed;
              g.push_back(GemmSeg{nullptr, A.d + so_, (*boff)[q] + v * sa, 0, D, Dr, D, 0, 0, A0, 0, scale});
            }
          }
      }
    }
    p = std::make_unique<GemmPlan>();
    if (!o.empty()) build_gemm(*p, o, g, c->st);
    return *p;
  }
  void run_bop(GemmPlan& p, const double* a, const double* b, double* out) {
    if (p.ntiles == 0) return;
    GemmExtra ex{};
    ex.p[0] = const_cast<double*>(a);
    ex.p[1] = const_cast<double*>(b);
    ex.p[2] = out;
    p.run(c->st, nullptr, nullptr, nullptr, &ex);
    CK(cudaGetLastError());
  }
  // X_v = A^T B_v on bond i+1 (A a fixed site-i tensor)
  void b_lc(int i, const SiteTensor& A, const SiteBatch& B, int nv, BondBatch& X) {
    bond_batch(c, i + 1, X, nv);
    run_bop(bop(K_LC, i, nv, false, 1.0, &A, 0, B.stride, X.stride, &X.off), nullptr, B.buf.p, X.buf.p);
  }
  // out_v (+)= s A_v X (X fixed on bond i+1)
  void b_rmul(int i, const SiteBatch& A, int nv, const BondMat& X, SiteBatch& out, bool acc, double s = 1.0) {
    run_bop(bop(K_RMUL, i, nv, acc, s, &X, A.stride, 0, out.stride, nullptr), A.buf.p, nullptr, out.buf.p);
  }
  // out_v (+)= s A X_v (A a fixed site-i tensor, X batched on bond i+1)
  void b_rmulb(int i, const SiteTensor& A, const BondBatch& X, int nv, SiteBatch& out, bool acc, double s = 1.0) {
    run_bop(bop(K_RMULB, i, nv, acc, s, &A, 0, X.stride, out.stride, &X.off), nullptr, X.buf.p, out.buf.p);
  }
  // X_v,ql = sum_n A_v(ql,n) B(ql,n)^T on bond i (B a fixed site-i tensor)
  void b_rc(int i, const SiteBatch& A, int nv, const SiteTensor& B, BondBatch& X) {
    bond_batch(c, i, X, nv);
    run_bop(bop(K_RC, i, nv, false, 1.0, &B, A.stride, 0, X.stride, &X.off), A.buf.p, nullptr, X.buf.p);
  }
  // out_v (+)= s X A_v (X fixed on bond i)
  void b_lmul(int i, const BondMat& X, const SiteBatch& A, int nv, SiteBatch& out, bool acc, double s = 1.0) {
    run_bop(bop(K_LMUL, i, nv, acc, s, &X, 0, A.stride, out.stride, nullptr), nullptr, A.buf.p, out.buf.p);
  }
  // out_v (+)= s X_v A (X batched on bond i, A a fixed site-i tensor)
  void b_lmulb(int i, const BondBatch& X, int nv, const SiteTensor& A, SiteBatch& out, bool acc, double s = 1.0) {
    run_bop(bop(K_LMULB, i, nv, acc, s, &A, X.stride, 0, out.stride, &X.off), X.buf.p, nullptr, out.buf.p);
  }

  // ---- vector algebra on batches (no host synchronization) ----
  DevBuf dwork, dcoef;
  void b_copy(const SiteBatch& A, int a0, int nv, SiteBatch& B, int b0) {
    if (nv > 0 && A.stride > 0)
      CK(cudaMemcpy2DAsync(B.v(b0), B.stride * sizeof(double), A.v(a0), A.stride * sizeof(double),
                           A.stride * sizeof(double), nv, cudaMemcpyDeviceToDevice, c->st));
  }
  // Y_v += s X_v
  void b_axpy(double s, const SiteBatch& X, int x0, SiteBatch& Y, int y0, int nv) {
    launch_rank1_batch(X.v(x0), X.stride, nullptr, s, nv, Y.v(y0), Y.stride, Y.stride, c->st);
  }
  // Q^C X_v = X_v - C0 (C0 . X_v)   (Eq. param)
  void b_projC(int i, SiteBatch& X, int x0, int nv) {
    dwork.ensure((size_t)dot_work(nv));
    dcoef.ensure((size_t)std::max(nv, 1));
    launch_vdots(X.v(x0), X.stride, C0(i).d, 0, nv, T(i), dcoef.p, false, dwork.p, c->st);
    launch_rank1_batch(C0(i).d, 0, dcoef.p, -1.0, nv, X.v(x0), X.stride, T(i), c->st);
  }
  // Q^L X_v = X_v - L0 (L0^T X_v)   (Eq. cwfn1st)
  void b_projL(int i, const SiteBatch& X, int nv, SiteBatch& out) {
    BondBatch Y;
    b_lc(i, L0(i), X, nv, Y);
    b_copy(X, 0, nv, out, 0);
    b_rmulb(i, L0(i), Y, nv, out, true, -1.0);
  }
  // X_v Q^R = X_v - (X_v R0^T) R0   (Eq. right1st)
  void b_projR(int i, const SiteBatch& X, int nv, SiteBatch& out) {
    BondBatch Y;
    b_rc(i, X, nv, R0(i), Y);
    b_copy(X, 0, nv, out, 0);
    b_lmulb(i, Y, nv, R0(i), out, true, -1.0);
  }

  // ---- first-order objects, one vector at a time (template replays, asynchronous) ----
  struct Enl {
    std::unique_ptr<OpSet> f, r;
  };
  std::map<std::tuple<int, int, int>, EnlTemplate> enl_tpl;   // (site, right, reverse) -> template
  std::unique_ptr<OpSet> enl(int i, bool right, int rev, const OpSet& X, const OpSet* Xr) {
    EnlTemplate& t = enl_tpl[std::make_tuple(i, right ? 1 : 0, rev)];
    const uint64_t sig = set_signature(X, Xr);
    if (t.proto && t.sig == sig) return enlarge_from(c, t, X, Xr);
    t = EnlTemplate();
    t.sig = sig;
    return enlarge_set(c, X, Xr, i, right, &t);
  }
  // The first-order site products use sets that are new for every vector and sweep but
  // keep their layout, so their plans are built once per (site, side) with operator
  // addresses relative to the sets and replayed with the new sets as bases: two FP64
  // launches and no host planning.  (In the tensor-core form each call would first pack
  // the whole new set; these products run in FP64 in both precisions.)
  struct DhTpl {
    std::unique_ptr<SigmaPlan> plan;
    uint64_t sig = 0;
  };
  std::map<std::pair<int, int>, DhTpl> dh_tpl;
  SigmaPlan& dh_plan(int i, int side, const OpSet& X, const OpSet* Xr, uint64_t xsig, const OpSet& Y,
                     const OpSet* Yr, uint64_t ysig) {
    DhTpl& t = dh_tpl[{i, side}];
    const uint64_t sig = xsig ^ (ysig * 1099511628211ull);
    if (!t.plan || t.sig != sig) {
      t.plan = plan_sigma_sets(c, X, Xr, Y, Yr, i, 1, 1, false, true);
      t.sig = sig;
    }
    return *t.plan;
  }
  // y = [H_mu^{L_{i-1}} x h_i x H_0^{R_i}] C0_i  (Eq. hleft_sb on C0; y zeroed by the caller)
  void dh_left(int i, const Enl& XE, double* y) {
    if (!XE.f) return;
    const OpSet& Y = *c->R[i + 1];
    SigmaPlan& p = dh_plan(i, 0, *XE.f, XE.r.get(), set_signature(*XE.f, XE.r.get()), Y, nullptr,
                           set_signature(Y, nullptr));
    p.ex.p[0] = XE.f->d;
    p.ex.p[1] = XE.r ? XE.r->d : nullptr;
    p.ex.p[2] = Y.d;
    p.ex.p[3] = nullptr;
    run_plan(p, C0(i).d, y, 1, false);
  }
  // ---- the per-vector first-order work of all vectors at once ----
  // The enlargements, ΔH C0 products and first-order renormalizations of the l vectors of a
  // site share their layouts, so each is one kept plan replayed over the vectors as the
  // instances of one launch per phase (instance mu's bases: its own sets).  A template is
  // (re)built by the first vector whose layout it does not match (its own launch), and a
  // vector whose layout differs from the template's runs on its own.
  static void inst_check(int64_t ntiles, int n) {
    if (n < 1 || n > GEMM_MAX_INST || ntiles * n > INT32_MAX) throw Error(LRT_EINVAL, "batched replay: launch size");
  }
  // the enlarged sets of X[mu] (with reverse Xr[mu]) for every mu
  std::vector<std::unique_ptr<OpSet>> enl_batch(int i, bool right, int rev, const std::vector<const OpSet*>& X,
                                                const std::vector<const OpSet*>& Xr) {
    const int nv = (int)X.size();
    std::vector<std::unique_ptr<OpSet>> out(nv);
    EnlTemplate& t = enl_tpl[std::make_tuple(i, right ? 1 : 0, rev)];
    std::vector<int> batch;
    for (int mu = 0; mu < nv; ++mu) {
      const uint64_t sig = set_signature(*X[mu], Xr[mu]);
      if (t.proto && t.sig == sig) {
        batch.push_back(mu);
      } else if (batch.empty()) {
        out[mu] = enl(i, right, rev, *X[mu], Xr[mu]);   // builds the template
      } else {
        // another layout than the template's: build a separate set, keep the template
        EnlTemplate tmp;
        tmp.sig = sig;
        out[mu] = enlarge_set(c, *X[mu], Xr[mu], i, right, &tmp);
      }
    }
    const GatherPlan* gp = t.gp.get();
    for (size_t j0 = 0; j0 < batch.size(); j0 += GEMM_MAX_INST) {
      const int n = (int)std::min<size_t>(GEMM_MAX_INST, batch.size() - j0);
      inst_check(gp->ntiles, n);
      GatherInstSet B{};
      for (int j = 0; j < n; ++j) {
        const int mu = batch[j0 + j];
        out[mu] = layout_copy(*t.proto);
        alloc_zero(*out[mu], c->st);
        B.b[j] = GatherBases{out[mu]->d, X[mu]->d, Xr[mu] ? Xr[mu]->d : nullptr};
      }
      launch_gather_inst(gp->tasks.p, gp->srcs.p, gp->tiles.p, gp->ntiles, B, n, c->st);
      CK(cudaGetLastError());
    }
    return out;
  }
  std::vector<Enl> enlarge_left_batch(int i, const std::vector<FirstOrder>& HL) {
    std::vector<Enl> e(HL.size());
    std::vector<const OpSet*> f, r;
    std::vector<int> idx;
    for (size_t mu = 0; mu < HL.size(); ++mu)
      if (!HL[mu].empty()) {
        idx.push_back((int)mu);
        f.push_back(HL[mu].f.get());
        r.push_back(HL[mu].r.get());
      }
    if (idx.empty()) return e;
    auto ef = enl_batch(i, false, 0, f, r);
    auto er = enl_batch(i, false, 1, r, f);
    for (size_t j = 0; j < idx.size(); ++j) {
      e[idx[j]].f = std::move(ef[j]);
      e[idx[j]].r = std::move(er[j]);
    }
    return e;
  }
  DevBuf iws;   // per-instance workspaces of the batched replays
  // one kept two-phase plan over instances: per instance x, y, workspace offset and extras
  void run_inst(const GemmPlan& p1, const GemmPlan& p2, int n, const GemmInstSet& B) {
    inst_check(std::max(p1.ntiles, p2.ntiles), n);
    launch_gemm_fp64_inst(p1.outs.p, p1.segs.p, p1.tiles.p, p1.ntiles, B, n, c->st);
    launch_gemm_fp64_inst(p2.outs.p, p2.segs.p, p2.tiles.p, p2.ntiles, B, n, c->st);
    CK(cudaGetLastError());
  }
  // out.v(mu) = [H_mu^{L_{i-1}} x h_i x H_0^{R_i}] C0_i for every mu with a first-order set
  // (Eq. hleft_sb on C0; out zeroed by the caller)
  void dh_left_batch(int i, const std::vector<Enl>& XE, SiteBatch& out) {
    const OpSet& Y = *c->R[i + 1];
    const uint64_t ysig = set_signature(Y, nullptr);
    std::vector<int> batch;
    uint64_t sig0 = 0;
    for (size_t mu = 0; mu < XE.size(); ++mu) {
      if (!XE[mu].f) continue;
      const uint64_t sig = set_signature(*XE[mu].f, XE[mu].r.get());
      if (batch.empty()) {
        sig0 = sig;
        batch.push_back((int)mu);
      } else if (sig == sig0) {
        batch.push_back((int)mu);
      } else {
        dh_left(i, XE[mu], out.v((int)mu));   // another layout: on its own (after the batch's plan is used)
      }
    }
    if (batch.empty()) return;
    SigmaPlan& p = dh_plan(i, 0, *XE[batch[0]].f, XE[batch[0]].r.get(), sig0, Y, nullptr, ysig);
    const int64_t ts = std::max<int64_t>(p.tsize, 1);
    for (size_t j0 = 0; j0 < batch.size(); j0 += GEMM_MAX_INST) {
      const int n = (int)std::min<size_t>(GEMM_MAX_INST, batch.size() - j0);
      iws.ensure((size_t)ts * n);
      GemmInstSet B{};
      for (int j = 0; j < n; ++j) {
        const Enl& e = XE[batch[j0 + j]];
        GemmInst& b = B.b[j];
        b.x = C0(i).d;
        b.y = out.v(batch[j0 + j]);
        b.t = iws.p + (int64_t)j * ts;
        b.e[0] = e.f->d;
        b.e[1] = e.r ? e.r->d : nullptr;
        b.e[2] = Y.d;
      }
      run_inst(p.p1, p.p2, n, B);
    }
  }
  // y_mu = [H_0^{L_{i-1}} x h_i x H_mu^{R_i}] C0_i for mu < nv, H_mu^{R_i} slot mu of a set
  // batch (second line of Eq. sigv2; out zeroed by the caller)
  void dh_right_batch(int i, const SetBatch& HR, int nv, SiteBatch& out) {
    if (HR.empty() || nv <= 0) return;
    const OpSet& X = *c->XL[i];
    SigmaPlan& p = dh_plan(i, 1, X, nullptr, set_signature(X, nullptr), *HR.fp, HR.rp.get(), HR.sig);
    const int64_t ts = std::max<int64_t>(p.tsize, 1);
    for (int v0 = 0; v0 < nv; v0 += GEMM_MAX_INST) {
      const int n = std::min(GEMM_MAX_INST, nv - v0);
      iws.ensure((size_t)ts * n);
      GemmInstSet B{};
      for (int j = 0; j < n; ++j) {
        GemmInst& b = B.b[j];
        b.x = C0(i).d;
        b.y = out.v(v0 + j);
        b.t = iws.p + (int64_t)j * ts;
        b.e[0] = X.d;
        b.e[2] = HR.fv(v0 + j);
        b.e[3] = HR.rv(v0 + j);
      }
      run_inst(p.p1, p.p2, n, B);
    }
  }
  // kept renormalization over instances: terms[mu] for every mu in `batch`, the template
  // matching them all; returns the new blocks
  void ren_batch(RenTemplate* tp, const std::vector<std::vector<RenTerm>>& terms, const std::vector<int>& batch,
                 const std::vector<std::vector<double*>>& kets, const std::vector<std::vector<double*>>& bras,
                 std::vector<std::unique_ptr<OpSet>>& out) {
    const int64_t ts = std::max<int64_t>(tp->toff, 1);
    for (size_t j0 = 0; j0 < batch.size(); j0 += GEMM_MAX_INST) {
      const int n = (int)std::min<size_t>(GEMM_MAX_INST, batch.size() - j0);
      iws.ensure((size_t)ts * n);
      GemmInstSet B{};
      for (int j = 0; j < n; ++j) {
        const int mu = batch[j0 + j];
        out[mu] = layout_copy(*tp->proto);
        alloc_zero(*out[mu], c->st);
        GemmInst& b = B.b[j];
        b.t = iws.p + (int64_t)j * ts;
        for (size_t t = 0; t < terms[mu].size(); ++t) {
          b.e[3 * t] = terms[mu][t].E->d;
          b.e[3 * t + 1] = kets[mu][t];
          b.e[3 * t + 2] = bras[mu][t];
        }
        b.e[REN_BASE_OUT] = out[mu]->d;
      }
      run_inst(*tp->p1, *tp->p2, n, B);
    }
  }
  // first-order left sets at bond i+1 (Eq. lopr1st), both directions, for every vector
  std::vector<FirstOrder> grow_HL_batch(int i, const std::vector<Enl>& XE, const SiteBatch& L1, int nv) {
    std::vector<FirstOrder> res(nv);
    const OpSet& XL = *c->XL[i];
    std::deque<SiteView> views;   // site tensors borrowing the batch's slots (not movable)
    for (int mu = 0; mu < nv; ++mu) views.emplace_back(lay[i], L1.v(mu));
    for (int dir = 0; dir < 2; ++dir) {
      std::vector<std::vector<RenTerm>> terms(nv);
      std::vector<std::vector<double*>> kets(nv), bras(nv);
      for (int mu = 0; mu < nv; ++mu) {
        const SiteTensor& l1 = views[mu].t;
        const OpSet* E = XE[mu].f ? (dir == 0 ? XE[mu].f.get() : XE[mu].r.get()) : nullptr;
        if (E) terms[mu].push_back(RenTerm{E, &L0(i), &L0(i)});
        terms[mu].push_back(dir == 0 ? RenTerm{&XL, &L0(i), &l1} : RenTerm{&XL, &l1, &L0(i)});
        for (const RenTerm& t : terms[mu]) {
          kets[mu].push_back(t.ket->d);
          bras[mu].push_back(t.bra->d);
        }
      }
      std::vector<std::unique_ptr<OpSet>> out(nv);
      // vectors grouped by the number of terms (with or without a first-order set)
      for (int nt = 1; nt <= 2; ++nt) {
        RenTemplate* tp = rtpl(i, false, dir, nt);
        std::vector<int> batch;
        uint64_t sig0 = 0;
        for (int mu = 0; mu < nv; ++mu) {
          if ((int)terms[mu].size() != nt) continue;
          const uint64_t sig = ren_signature(i, false, terms[mu]);
          if (tp->p1 && tp->sig == sig && (batch.empty() || sig == sig0)) {
            sig0 = sig;
            batch.push_back(mu);
          } else if (batch.empty() && !(tp->p1 && tp->sig == sig)) {
            out[mu] = renorm_left_terms(c, i, terms[mu], LRT_FP64, tp);   // builds the template
          } else {
            out[mu] = renorm_left_terms(c, i, terms[mu], LRT_FP64, nullptr);
          }
        }
        ren_batch(tp, terms, batch, kets, bras, out);
      }
      for (int mu = 0; mu < nv; ++mu) (dir == 0 ? res[mu].f : res[mu].r) = std::move(out[mu]);
    }
    return res;
  }
  // first-order right sets at bond i (Eq. ropr1st), both directions, for every vector
  std::vector<FirstOrder> grow_HR_batch(int i, const std::vector<FirstOrder>& HR, const SiteBatch& R1, int nv) {
    std::vector<FirstOrder> res(nv);
    const OpSet& YR = *c->YR[i];
    // enlarged first-order sets site (+) H_mu^{R_{i+1}}
    std::vector<std::unique_ptr<OpSet>> Yf(nv), Yr(nv);
    {
      std::vector<const OpSet*> f, r;
      std::vector<int> idx;
      for (int mu = 0; mu < nv; ++mu)
        if (!HR[mu].empty()) {
          idx.push_back(mu);
          f.push_back(HR[mu].f.get());
          r.push_back(HR[mu].r.get());
        }
      if (!idx.empty()) {
        auto ef = enl_batch(i, true, 0, f, r);
        auto er = enl_batch(i, true, 1, r, f);
        for (size_t j = 0; j < idx.size(); ++j) {
          Yf[idx[j]] = std::move(ef[j]);
          Yr[idx[j]] = std::move(er[j]);
        }
      }
    }
    // right-fused copies of R0_i (once) and of every R1_mu (one batched gather)
    const Fused& F = *YR.fused;
    DevBuf rf0;
    const std::vector<int64_t> off0 = rfused_copy(c, i, R0(i), rf0, F);
    std::deque<SiteView> views;   // site tensors borrowing the batch's slots (not movable)
    for (int mu = 0; mu < nv; ++mu) views.emplace_back(lay[i], R1.v(mu));
    std::vector<int64_t> off1;
    int64_t tot1 = 0;
    const GatherPlan& gp = rfused_plan(c, i, views[0].t, F, off1, tot1);
    if (off1 != off0) throw Error(LRT_EINVAL, "first-order right set: R1 and R0 layouts differ");
    DevBuf rf1;
    const int64_t st1 = std::max<int64_t>(tot1, 1);
    rf1.ensure((size_t)st1 * nv);
    CK(cudaMemsetAsync(rf1.p, 0, (size_t)st1 * nv * sizeof(double), c->st));
    for (int v0 = 0; v0 < nv; v0 += GEMM_MAX_INST) {
      const int n = std::min(GEMM_MAX_INST, nv - v0);
      inst_check(gp.ntiles, n);
      GatherInstSet B{};
      for (int j = 0; j < n; ++j) B.b[j] = GatherBases{rf1.p + (int64_t)(v0 + j) * st1, R1.v(v0 + j), nullptr};
      launch_gather_inst(gp.tasks.p, gp.srcs.p, gp.tiles.p, gp.ntiles, B, n, c->st);
      CK(cudaGetLastError());
    }
    for (int dir = 0; dir < 2; ++dir) {
      std::vector<std::vector<RenTerm>> terms(nv);
      std::vector<std::vector<double*>> kets(nv), bras(nv);
      for (int mu = 0; mu < nv; ++mu) {
        const SiteTensor& r1 = views[mu].t;
        double* rf1mu = rf1.p + (int64_t)mu * st1;
        const OpSet* E = dir == 0 ? Yf[mu].get() : Yr[mu].get();
        if (E) {
          terms[mu].push_back(RenTerm{E, &R0(i), &R0(i)});
          kets[mu].push_back(rf0.p);
          bras[mu].push_back(rf0.p);
        }
        terms[mu].push_back(dir == 0 ? RenTerm{&YR, &R0(i), &r1} : RenTerm{&YR, &r1, &R0(i)});
        kets[mu].push_back(dir == 0 ? rf1mu : rf0.p);
        bras[mu].push_back(dir == 0 ? rf0.p : rf1mu);
      }
      std::vector<std::unique_ptr<OpSet>> out(nv);
      for (int nt = 1; nt <= 2; ++nt) {
        RenTemplate* tp = rtpl(i, true, dir, nt);
        std::vector<int> batch;
        uint64_t sig0 = 0;
        for (int mu = 0; mu < nv; ++mu) {
          if ((int)terms[mu].size() != nt) continue;
          const uint64_t sig = ren_signature(i, true, terms[mu]);
          if (tp->p1 && tp->sig == sig && (batch.empty() || sig == sig0)) {
            sig0 = sig;
            batch.push_back(mu);
          } else if (batch.empty() && !(tp->p1 && tp->sig == sig)) {
            out[mu] = renorm_right_terms(c, i, terms[mu], LRT_FP64, tp);   // builds the template
          } else {
            out[mu] = renorm_right_terms(c, i, terms[mu], LRT_FP64, nullptr);
          }
        }
        ren_batch(tp, terms, batch, kets, bras, out);
      }
      for (int mu = 0; mu < nv; ++mu) (dir == 0 ? res[mu].f : res[mu].r) = std::move(out[mu]);
    }
    return res;
  }

  // renormalizations kept for replay, per (site, right, direction, number of terms)
  std::map<std::tuple<int, int, int, int>, RenTemplate> ren_tpl;
  RenTemplate* rtpl(int i, bool right, int rev, int nterms) {
    return &ren_tpl[std::make_tuple(i, right ? 1 : 0, rev, nterms)];
  }
  // Initial trial vector mu at site i.  seed != 0: SplitMix64 Gaussians; seed == 0: the
  // unit vector on the mu-th lowest diagonal element of H_0^[i] among the components where
  // the reference is small (|C0| < 1/2), a single-site excitation.  Both projected by Q^C.
  void start_site(int i, int mu, double* out) {
    std::vector<double> h(T(i), 0.0);
    bool unit = false;
    if (P.seed == 0) {
      std::vector<double> d(T(i)), c0(T(i));
      CK(cudaMemcpyAsync(d.data(), diag[i].p, d.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaMemcpyAsync(c0.data(), C0(i).d, c0.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      std::vector<int64_t> idx;
      for (int64_t e = 0; e < T(i); ++e)
        if (std::fabs(c0[e]) < 0.5) idx.push_back(e);
      if (!idx.empty()) {
        std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return d[a] < d[b]; });
        h[idx[std::min<int64_t>(mu, (int64_t)idx.size() - 1)]] = 1.0;
        unit = true;
      }
    }
    if (!unit) {
      const uint64_t seed = P.seed * 7919ull + 1000ull * (uint64_t)mu + (uint64_t)i;
      for (int64_t e = 0; e < T(i); ++e) h[e] = splitmix_normal(seed, (uint64_t)e);
      if (P.start_shift > 0.0) {
        // damped by the diagonal energy above the reference: low-lying configurations first
        std::vector<double> d(T(i));
        CK(cudaMemcpyAsync(d.data(), diag[i].p, d.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        for (int64_t e = 0; e < T(i); ++e) h[e] /= std::fabs(d[e] - E0) + P.start_shift;
      }
    }
    if (T(i) > 0) CK(cudaMemcpyAsync(out, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
  }

  // small generalized eigenproblem H a = theta S a (S semi-definite), eigensolves on the GPU
  void solve_gep(const std::vector<double>& H, const std::vector<double>& S, int l, std::vector<double>& w,
                 std::vector<double>& U) {
    if (l > JACOBI_MAXN) throw Error(LRT_EINVAL, "sweep_tda: subspace larger than the eigensolver limit");
    DevBuf A, W, Z;
    A.ensure((size_t)l * l);
    W.ensure(l);
    Z.ensure((size_t)l * l);
    std::vector<double> s(l), Us((size_t)l * l);
    CK(cudaMemcpyAsync(A.p, S.data(), (size_t)l * l * sizeof(double), cudaMemcpyHostToDevice, c->st));
    launch_jacobi_eigh(A.p, l, W.p, Z.p, c->st);
    CK(cudaMemcpyAsync(s.data(), W.p, l * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(Us.data(), Z.p, (size_t)l * l * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    double smax = 0.0;
    for (double x : s) smax = std::max(smax, x);
    std::vector<int> keep;
    for (int j = 0; j < l; ++j)
      if (s[j] > 1e-12 * std::max(smax, 1e-300)) keep.push_back(j);
    const int r = (int)keep.size();
    std::vector<double> X((size_t)l * r);   // X = U_keep s^-1/2
    for (int a = 0; a < l; ++a)
      for (int j = 0; j < r; ++j) X[(size_t)a * r + j] = Us[(size_t)a * l + keep[j]] / std::sqrt(s[keep[j]]);
    std::vector<double> Hp((size_t)r * r, 0.0);
    for (int p = 0; p < r; ++p)
      for (int q = 0; q < r; ++q) {
        double acc = 0.0;
        for (int a = 0; a < l; ++a)
          for (int b2 = 0; b2 < l; ++b2)
            acc += X[(size_t)a * r + p] * 0.5 * (H[(size_t)a * l + b2] + H[(size_t)b2 * l + a]) * X[(size_t)b2 * r + q];
        Hp[(size_t)p * r + q] = acc;
      }
    std::vector<double> wr(r), Y((size_t)r * r);
    CK(cudaMemcpyAsync(A.p, Hp.data(), (size_t)r * r * sizeof(double), cudaMemcpyHostToDevice, c->st));
    launch_jacobi_eigh(A.p, r, W.p, Z.p, c->st);
    CK(cudaMemcpyAsync(wr.data(), W.p, r * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(Y.data(), Z.p, (size_t)r * r * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    w = wr;
    U.assign((size_t)l * r, 0.0);     // U = X Y  (l x r)
    for (int a = 0; a < l; ++a)
      for (int q = 0; q < r; ++q) {
        double acc = 0.0;
        for (int p2 = 0; p2 < r; ++p2) acc += X[(size_t)a * r + p2] * Y[(size_t)p2 * r + q];
        U[(size_t)a * r + q] = acc;
      }
  }

  // sum_i |Q^C (H_0^[i] - E0) C0_i|^2: the site components of <T|H|Psi0> (Eq. dmrg at
  // every site), zero at a stationary point of the one-site manifold
  double stationarity() {
    setup();
    double g2 = 0.0;
    for (int i = 0; i < k; ++i) {
      SiteTensor y = new_site(c, i);
      run_plan(*h0one[i], C0(i).d, y.d, 1, false);
      t_axpby(c, -E0, C0(i), 1.0, y, tmp);
      proj_C(i, y);
      g2 += t_dot(c, y, y, tmp);
    }
    return g2;
  }
  void proj_C(int i, SiteTensor& X) { t_axpby(c, -t_dot(c, C0(i), X, tmp), C0(i), 1.0, X, tmp); }

  // ---- one-particle transition densities of the roots (Sec. "Results", Table
  // site_excitation): gamma^mu_pq = <Psi^mu| sum_sigma a+_{p sigma} a_{q sigma} |Psi0> ----
  //
  // The tangent vector of root mu is split at the centre c = k/2 into pieces that touch one
  // site each: Q^L C1_i for i < c, C1_c, and C1_i Q^R for i > c (C1_i its mixed-canonical site
  // tensor, Q^L and Q^R the projectors of Eqs. cwfn1st and right1st).  The pieces sum to the
  // vector exactly and gamma_pq = sum_i <piece_i| E_pq |Psi0>, each term a contraction of the
  // piece with the block operators of site i's environment acting on C0_i.  A piece left of
  // c is orthogonal to every operator acting only on the right block (its fused rows avoid
  // the span of L0_i), a piece right of c to every operator acting only on the left block, so
  // the pair operators B_pq = a+_p a_q are needed only where the library keeps them: in the
  // left blocks up to c and the right blocks from c + 1 on (the normal sides).  Creation
  // operators exist in every block.  The contractions run densely per bond (sector blocks
  // scattered into M x M matrices, fermion signs as diagonal factors) on the FP64 GEMM.
  bool want_gamma = false;
  std::vector<SiteBatch> keepC;   // the roots' C1_i of the sweep whose residuals are reported

  struct DenseBond {
    int M = 0;
    std::vector<int64_t> off;
  };
  DenseBond dense_bond(int b) {
    DenseBond d;
    const Sectors& S = c->bonds[b];
    d.off.resize(S.n());
    for (int q = 0; q < S.n(); ++q) {
      d.off[q] = d.M;
      d.M += S.d[q];
    }
    return d;
  }
  // nv site tensors of site i (stride `stride`) into dense [v][n][Ml][Mr]; sub-blocks scaled by
  // (-1)^{N(q_l)} when signL
  void site_to_dense(int i, const double* src, int64_t stride, int nv, double* dst, const DenseBond& dl,
                     const DenseBond& dr, bool signL) {
    std::vector<GatherTask> t;
    std::vector<GatherSrc> s;
    const SiteTensor& L = lay[i];
    const Sectors& Lb = c->bonds[i];
    const int64_t ms = (int64_t)dl.M * dr.M;
    for (int v = 0; v < nv; ++v)
      for (int q = 0; q < Lb.n(); ++q)
        for (int n = 0; n < 4; ++n) {
          if (L.sub_off[q][n] < 0) continue;
          const int qr = L.sub_qr[q][n];
          const int Dl = Lb.d[q], Dr = c->bonds[i + 1].d[qr];
          const double sg = (signL && ((Lb.a[q] + Lb.b[q]) & 1)) ? -1.0 : 1.0;
          t.push_back(GatherTask{dst + (int64_t)v * 4 * ms + n * ms + dl.off[q] * dr.M + dr.off[qr], dr.M, Dl, Dr,
                                 (int)s.size(), 1, 0});
          s.push_back(GatherSrc{src + (int64_t)v * stride + L.sub_off[q][n], Dr, 0, sg, 0, 0});
        }
    run_gathers(c, t, s);
  }
  // operator o of set S (basis = the bond's sectors) into a dense M x M matrix
  void op_to_dense(const OpSet& S, int o, double* dst, const DenseBond& d, std::vector<GatherTask>& t,
                   std::vector<GatherSrc>& s) {
    for (int q = 0; q < S.ns(); ++q) {
      const int qb = S.bra_of(o, q);
      if (qb < 0 || !S.block_nz(o, q)) continue;
      t.push_back(GatherTask{dst + d.off[qb] * d.M + d.off[q], d.M, S.basis.d[qb], S.basis.d[q], (int)s.size(), 1, 0});
      s.push_back(GatherSrc{S.d + S.off_of(o, q), S.basis.d[q], 0, 1.0, 0, 0});
    }
  }

  void compute_gamma(int n, double* gamma_out) {
    const int cc = k / 2;
    const int64_t kk = (int64_t)k * k;
    DevBuf dg;
    dg.ensure((size_t)std::max<int64_t>(n * kk, 1));
    CK(cudaMemsetAsync(dg.p, 0, (size_t)n * kk * sizeof(double), c->st));
    static const int NEL[4] = {0, 1, 1, 2};
    static const double SGN[4] = {1.0, -1.0, -1.0, 1.0};
    // site annihilators a_sigma[n][n'] (basis |0>, |a>, |b>, |ab>), nonzero entries
    struct E { int n, m; double v; };
    const std::vector<E> ann[2] = {{{0, 1, 1.0}, {2, 3, 1.0}}, {{0, 2, 1.0}, {1, 3, -1.0}}};
    const std::vector<E> cre[2] = {{{1, 0, 1.0}, {3, 2, 1.0}}, {{2, 0, 1.0}, {3, 1, -1.0}}};
    for (int i = 0; i < k; ++i) {
      if (keepC[i].nv < n) throw Error(LRT_ESTATE, "transition density: no Ritz vectors kept");
      const DenseBond dl = dense_bond(i), dr = dense_bond(i + 1);
      const int Ml = dl.M, Mr = dr.M;
      const int64_t ms = (int64_t)Ml * Mr, ml2 = (int64_t)Ml * Ml, mr2 = (int64_t)Mr * Mr;
      // pieces of the centred decomposition
      SiteBatch P;
      batch_alloc(c, P, T(i), n, blk);
      if (i < cc) b_projL(i, keepC[i], n, P);
      else if (i == cc) b_copy(keepC[i], 0, n, P, 0);
      else b_projR(i, keepC[i], n, P);
      DevBuf Dd, C0d, C0P;
      Dd.ensure((size_t)std::max<int64_t>(n * 4 * ms, 1));
      C0d.ensure((size_t)std::max<int64_t>(4 * ms, 1));
      C0P.ensure((size_t)std::max<int64_t>(4 * ms, 1));
      CK(cudaMemsetAsync(Dd.p, 0, (size_t)n * 4 * ms * sizeof(double), c->st));
      CK(cudaMemsetAsync(C0d.p, 0, (size_t)4 * ms * sizeof(double), c->st));
      CK(cudaMemsetAsync(C0P.p, 0, (size_t)4 * ms * sizeof(double), c->st));
      site_to_dense(i, P.buf.p, P.stride, n, Dd.p, dl, dr, false);
      site_to_dense(i, C0(i).d, T(i), 1, C0d.p, dl, dr, false);
      site_to_dense(i, C0(i).d, T(i), 1, C0P.p, dl, dr, true);     // P_L C0
      auto Dn = [&](int mu, int nn) { return Dd.p + (int64_t)mu * 4 * ms + nn * ms; };
      auto C0n = [&](int nn) { return C0d.p + nn * ms; };
      auto CPn = [&](int nn) { return C0P.p + nn * ms; };
      // dense block operators: left C_x (x < 2i) and, up to the centre, B_xy of same spin;
      // right C_y (y >= 2(i+1)) and, from the centre on, B_xy of same spin
      const OpSet* Ls = c->L[i].get();
      const OpSet* Rs = c->R[i + 1].get();
      struct Op { int x, y; };              // y < 0: creation operator of x
      std::vector<Op> lops, rops;
      for (int x = 0; x < 2 * i; ++x) lops.push_back({x, -1});
      if (i <= cc)
        for (int p = 0; p < i; ++p)
          for (int q = p; q < i; ++q)
            for (int s = 0; s < 2; ++s) lops.push_back({2 * p + s, 2 * q + s});
      for (int y = 2 * (i + 1); y < 2 * k; ++y) rops.push_back({y, -1});
      if (i >= cc)
        for (int p = i + 1; p < k; ++p)
          for (int q = p; q < k; ++q)
            for (int s = 0; s < 2; ++s) rops.push_back({2 * p + s, 2 * q + s});
      auto key_of = [&](const Op& o) { return o.y < 0 ? Key{KC, o.x, -1} : Key{KB, o.x, o.y}; };
      DevBuf LO, RO;
      LO.ensure((size_t)std::max<int64_t>((int64_t)lops.size() * ml2, 1));
      RO.ensure((size_t)std::max<int64_t>((int64_t)rops.size() * mr2, 1));
      CK(cudaMemsetAsync(LO.p, 0, LO.n * sizeof(double), c->st));
      CK(cudaMemsetAsync(RO.p, 0, RO.n * sizeof(double), c->st));
      {
        std::vector<GatherTask> t;
        std::vector<GatherSrc> s;
        for (size_t a = 0; a < lops.size(); ++a) {
          const int o = Ls ? Ls->find(key_of(lops[a])) : -1;
          if (o < 0) throw Error(LRT_EINVAL, "transition density: left block operator missing");
          op_to_dense(*Ls, o, LO.p + (int64_t)a * ml2, dl, t, s);
        }
        for (size_t a = 0; a < rops.size(); ++a) {
          const int o = Rs ? Rs->find(key_of(rops[a])) : -1;
          if (o < 0) throw Error(LRT_EINVAL, "transition density: right block operator missing");
          op_to_dense(*Rs, o, RO.p + (int64_t)a * mr2, dr, t, s);
        }
        run_gathers(c, t, s);
      }
      const int nLC = 2 * i, nRC = 2 * (k - i - 1);
      // root-independent: Z_y = (P_L C0_n) C_y  and  Z'_x = (P_L C0_n) C_x^T  (Ml x Mr)
      DevBuf Z, Zt;
      Z.ensure((size_t)std::max<int64_t>((int64_t)nRC * 4 * ms, 1));
      Zt.ensure((size_t)std::max<int64_t>((int64_t)nRC * 4 * ms, 1));
      if (nRC > 0 && Ml > 0 && Mr > 0) {
        std::vector<GemmOut> o;
        std::vector<GemmSeg> g;
        for (int a = 0; a < nRC; ++a)
          for (int nn = 0; nn < 4; ++nn) {
            const double* Cy = RO.p + (int64_t)a * mr2;
            o.push_back(GemmOut{Z.p + ((int64_t)a * 4 + nn) * ms, 0, Mr, Ml, Mr, (int)g.size(), 1, 0, 0});
            g.push_back(GemmSeg{CPn(nn), Cy, 0, 0, Mr, Mr, Mr, 0, 0, 0, 0, 1.0});
            o.push_back(GemmOut{Zt.p + ((int64_t)a * 4 + nn) * ms, 0, Mr, Ml, Mr, (int)g.size(), 1, 0, 0});
            g.push_back(GemmSeg{CPn(nn), Cy, 0, 0, Mr, Mr, Mr, 0, 1, 0, 0, 1.0});
          }
        run_gemms(c, o, g);
      }
      // per root: the left (Ml x Ml) and right (Mr x Mr) reduced transition matrices
      //   left:  ML, MLT, N_a, N_b, N'T_a, N'T_b, K_y (y right), QT_x (x right)
      //   right: MR, MRT, UT_a, UT_b, V_a, V_b
      const int nLM = 6 + 2 * nRC, nRM = 6;
      DevBuf LM, RM;
      LM.ensure((size_t)std::max<int64_t>((int64_t)n * nLM * ml2, 1));
      RM.ensure((size_t)std::max<int64_t>((int64_t)n * nRM * mr2, 1));
      CK(cudaMemsetAsync(LM.p, 0, LM.n * sizeof(double), c->st));
      CK(cudaMemsetAsync(RM.p, 0, RM.n * sizeof(double), c->st));
      if (Ml > 0 && Mr > 0) {
        std::vector<GemmOut> o;
        std::vector<GemmSeg> g;
        auto out = [&](double* C, int ld, int m, int nn) { o.push_back(GemmOut{C, 0, ld, m, nn, (int)g.size(), 0, 0, 0}); };
        // seg: op(A) op(B), A and B dense Ml x Mr (row-major, ld Mr); tA / tB transpose
        auto seg = [&](const double* A, int tA, const double* B, int tB, int kdim, double s) {
          g.push_back(GemmSeg{A, B, 0, 0, Mr, Mr, kdim, tA, tB, 0, 0, s});
          o.back().seg_count++;
        };
        for (int mu = 0; mu < n; ++mu) {
          double* L0m = LM.p + (int64_t)mu * nLM * ml2;
          double* R0m = RM.p + (int64_t)mu * nRM * mr2;
          out(L0m + 0 * ml2, Ml, Ml, Ml);                              // ML = sum D_n C0_n^T
          for (int nn = 0; nn < 4; ++nn) seg(Dn(mu, nn), 0, C0n(nn), 1, Mr, 1.0);
          out(L0m + 1 * ml2, Ml, Ml, Ml);                              // MLT = sum C0_n D_n^T
          for (int nn = 0; nn < 4; ++nn) seg(C0n(nn), 0, Dn(mu, nn), 1, Mr, 1.0);
          for (int s = 0; s < 2; ++s) {
            out(L0m + (2 + s) * ml2, Ml, Ml, Ml);                      // N_s = sum a_s[n,n'] D_n (P C0_n')^T
            for (const E& e : ann[s]) seg(Dn(mu, e.n), 0, CPn(e.m), 1, Mr, e.v);
            out(L0m + (4 + s) * ml2, Ml, Ml, Ml);                      // N'T_s = sum c_s[n,n'] (P C0_n') D_n^T
            for (const E& e : cre[s]) seg(CPn(e.m), 0, Dn(mu, e.n), 1, Mr, e.v);
          }
          for (int a = 0; a < nRC; ++a) {
            out(L0m + (6 + a) * ml2, Ml, Ml, Ml);                      // K_y = sum s_n D_n Z_{y,n}^T
            for (int nn = 0; nn < 4; ++nn) seg(Dn(mu, nn), 0, Z.p + ((int64_t)a * 4 + nn) * ms, 1, Mr, SGN[nn]);
            out(L0m + (6 + nRC + a) * ml2, Ml, Ml, Ml);                // QT_x = sum s_n Z'_{x,n} D_n^T
            for (int nn = 0; nn < 4; ++nn) seg(Zt.p + ((int64_t)a * 4 + nn) * ms, 0, Dn(mu, nn), 1, Mr, SGN[nn]);
          }
          // right matrices: contractions over the left index (k = Ml), A and B transposed roles
          auto rseg = [&](const double* A, const double* B, double s) {   // A^T B, A and B Ml x Mr
            g.push_back(GemmSeg{A, B, 0, 0, Mr, Mr, Ml, 1, 0, 0, 0, s});
            o.back().seg_count++;
          };
          out(R0m + 0 * mr2, Mr, Mr, Mr);                              // MR = sum D_n^T C0_n
          for (int nn = 0; nn < 4; ++nn) rseg(Dn(mu, nn), C0n(nn), 1.0);
          out(R0m + 1 * mr2, Mr, Mr, Mr);                              // MRT = sum C0_n^T D_n
          for (int nn = 0; nn < 4; ++nn) rseg(C0n(nn), Dn(mu, nn), 1.0);
          for (int s = 0; s < 2; ++s) {
            out(R0m + (2 + s) * mr2, Mr, Mr, Mr);                      // UT_s = sum c_s[n,n'] s_n' C0_n'^T D_n
            for (const E& e : cre[s]) rseg(C0n(e.m), Dn(mu, e.n), e.v * SGN[e.m]);
            out(R0m + (4 + s) * mr2, Mr, Mr, Mr);                      // V_s = sum a_s[n,n'] s_n' D_n^T C0_n'
            for (const E& e : ann[s]) rseg(Dn(mu, e.n), C0n(e.m), e.v * SGN[e.m]);
          }
        }
        run_gemms(c, o, g);
      }
      // dot products: every left operator with every left matrix, every right operator with
      // every right matrix (per root), and the site-diagonal terms <D_n, C0_n>
      const int nl = (int)lops.size(), nr = (int)rops.size();
      const int64_t nres = (int64_t)n * (nl * nLM + nr * nRM + 4);
      DevBuf res;
      res.ensure((size_t)std::max<int64_t>(nres, 1));
      CK(cudaMemsetAsync(res.p, 0, (size_t)nres * sizeof(double), c->st));
      dwork.ensure((size_t)dot_work(std::max<int64_t>(std::max<int64_t>((int64_t)nl * nLM, (int64_t)nr * nRM), 4)));
      auto rL = [&](int mu, int a, int m) { return (int64_t)mu * (nl * nLM + nr * nRM + 4) + (int64_t)a * nLM + m; };
      auto rR = [&](int mu, int a, int m) {
        return (int64_t)mu * (nl * nLM + nr * nRM + 4) + (int64_t)nl * nLM + (int64_t)a * nRM + m;
      };
      auto rS = [&](int mu, int nn) { return (int64_t)mu * (nl * nLM + nr * nRM + 4) + (int64_t)nl * nLM + nr * nRM + nn; };
      for (int mu = 0; mu < n; ++mu) {
        if (nl > 0 && Ml > 0)
          launch_pair_dots_strided(LO.p, ml2, nl, LM.p + (int64_t)mu * nLM * ml2, ml2, nLM, ml2, res.p + rL(mu, 0, 0),
                                   dwork.p, c->st);
        if (nr > 0 && Mr > 0)
          launch_pair_dots_strided(RO.p, mr2, nr, RM.p + (int64_t)mu * nRM * mr2, mr2, nRM, mr2, res.p + rR(mu, 0, 0),
                                   dwork.p, c->st);
        if (ms > 0) launch_vdots(Dn(mu, 0), ms, C0d.p, ms, 4, ms, res.p + rS(mu, 0), false, dwork.p, c->st);
      }
      // gamma[mu][p][q] += sum of coefficient x result, lists per output entry
      std::vector<std::vector<std::pair<int64_t, double>>> terms((size_t)n * kk);
      auto add = [&](int mu, int p, int q, int64_t r, double v) { terms[(size_t)mu * kk + (size_t)p * k + q].push_back({r, v}); };
      for (int mu = 0; mu < n; ++mu) {
        for (int nn = 0; nn < 4; ++nn)
          if (NEL[nn]) add(mu, i, i, rS(mu, nn), NEL[nn]);
        for (int a = 0; a < nl; ++a) {
          const Op& op = lops[a];
          if (op.y >= 0) {                         // B_xy, both in the left block
            const int p = op.x / 2, q = op.y / 2;
            add(mu, p, q, rL(mu, a, 0), 1.0);
            if (p != q) add(mu, q, p, rL(mu, a, 1), 1.0);
            continue;
          }
          const int x = op.x, p = x / 2, s = x & 1;
          add(mu, p, i, rL(mu, a, 2 + s), 1.0);    // a+_x (left) a_(i s)
          add(mu, i, p, rL(mu, a, 4 + s), -1.0);   // a+_(i s) a_x (left)
          for (int b = 0; b < nRC; ++b) {
            const int y = 2 * (i + 1) + b;
            if ((y & 1) != s) continue;
            add(mu, p, y / 2, rL(mu, a, 6 + b), 1.0);          // a+_x (left) a_y (right)
            add(mu, y / 2, p, rL(mu, a, 6 + nRC + b), -1.0);   // a+_y (right) a_x (left)
          }
        }
        for (int a = 0; a < nr; ++a) {
          const Op& op = rops[a];
          if (op.y >= 0) {                         // B_xy, both in the right block
            const int p = op.x / 2, q = op.y / 2;
            add(mu, p, q, rR(mu, a, 0), 1.0);
            if (p != q) add(mu, q, p, rR(mu, a, 1), 1.0);
            continue;
          }
          const int y = op.x, q = y / 2, s = y & 1;
          add(mu, i, q, rR(mu, a, 2 + s), 1.0);    // a+_(i s) a_y (right)
          add(mu, q, i, rR(mu, a, 4 + s), -1.0);   // a+_y (right) a_(i s)
        }
      }
      std::vector<int> beg(1, 0), idx;
      std::vector<double> coef;
      for (auto& tl : terms) {
        for (auto& pr : tl) {
          idx.push_back((int)pr.first);
          coef.push_back(pr.second);
        }
        beg.push_back((int)idx.size());
      }
      DevArray<int> dbeg, didx;
      DevArray<double> dcf;
      dbeg.upload(beg, c->st);
      didx.upload(idx, c->st);
      dcf.upload(coef, c->st);
      launch_gather_sum(res.p, dbeg.p, didx.p, dcf.p, (int)(n * kk), dg.p, c->st);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(c->st));
    }
    CK(cudaMemcpyAsync(gamma_out, dg.p, (size_t)n * kk * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
  }

  // Fig. alg:dmrgtda.  The trial vectors of a sweep are processed together at every site:
  // their site tensors are contiguous batches, the bond and site products of the gauge
  // shifts and projections are grouped launches over all vectors, the H_0 products are
  // multi-vector sigma calls, and the reduced matrices and residual norms accumulate on the
  // device; the host synchronizes once per sweep (and in the first, for the start vectors).
  void run(int n, double* theta_out, double* resid_out, int* iters_out, double* gamma_out = nullptr) {
    setup();
    want_gamma = gamma_out != nullptr;
    if (want_gamma) {
      keepC.clear();
      keepC.resize(k);
    }
    const int N = P.max_space > 0 ? P.max_space : std::min(JACOBI_MAXN, std::max(8 * n, 24));
    if (N > JACOBI_MAXN || 2 * n > JACOBI_MAXN)
      throw Error(LRT_EINVAL, "sweep_tda: max_space and 2 nroots must not exceed " + std::to_string(JACOBI_MAXN));
    if (P.correction != LRT_CORR_SITE && P.correction != LRT_CORR_SWEEP)
      throw Error(LRT_EINVAL, "sweep_tda: unknown correction");
    // Ritz vectors kept at a restart (the paper's deflation keeps n)
    const int keep = std::max(n, std::min(P.keep > 0 ? P.keep : n, N - n));
    blk = n;
    // previous subspace: R1 per site, first-order right sets per bond (both directions)
    std::vector<SiteBatch> oldR1(k);
    std::vector<SetBatch> oldHR(k + 1);
    int lold = 0;
    std::vector<double> alpha, theta, Hr, Sr, r2(n, 0.0);
    DevBuf d_alpha, d_theta, d_H, d_S, d_D, d_r2, d_gs;
    std::vector<double> gsf(n, 0.0);
    bool any_gs = false;
    int m = 0, it = 0;
    bool first = true;
    c->sweep_log.clear();
    for (;;) {
      const auto t_sweep = std::chrono::steady_clock::now();
      const bool sweep_mixed = mixed;
      if (!first) {
        std::vector<double> w, U;
        solve_gep(Hr, Sr, lold, w, U);
        const int mcols = (int)w.size();
        m = std::min(m, mcols);
        // every root needs a Ritz vector: a subspace whose overlap matrix keeps fewer than
        // n directions above the cut cannot continue the sweep Davidson
        if (m < n)
          throw Error(LRT_EINVAL, "sweep_tda: the trial subspace spans fewer directions than roots (" +
                                      std::to_string(m) + " < " + std::to_string(n) + ")");
        alpha.assign((size_t)lold * m, 0.0);
        for (int a = 0; a < lold; ++a)
          for (int j = 0; j < m; ++j) alpha[(size_t)a * m + j] = U[(size_t)a * mcols + j];
        theta.assign(w.begin(), w.begin() + m);
        d_alpha.ensure(alpha.size());
        d_theta.ensure(n);
        CK(cudaMemcpyAsync(d_alpha.p, alpha.data(), alpha.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
        CK(cudaMemcpyAsync(d_theta.p, theta.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->st));
        // the sweep correction, per root, once the root's last residual is below the gate
        any_gs = false;
        if (P.correction == LRT_CORR_SWEEP && it > 0) {
          const double gate = P.corr_tol > 0.0 ? P.corr_tol : 1.0;
          for (int mu = 0; mu < n; ++mu) {
            gsf[mu] = r2[mu] < gate ? 1.0 : 0.0;
            any_gs = any_gs || gsf[mu] != 0.0;
          }
          d_gs.ensure(n);
          CK(cudaMemcpyAsync(d_gs.p, gsf.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->st));
        }
      }
      const int l = m + n;
      d_H.ensure((size_t)l * l);
      d_S.ensure((size_t)l * l);
      d_D.ensure((size_t)3 * l * l);
      d_r2.ensure(n);
      CK(cudaMemsetAsync(d_H.p, 0, (size_t)l * l * sizeof(double), c->st));
      CK(cudaMemsetAsync(d_S.p, 0, (size_t)l * l * sizeof(double), c->st));
      CK(cudaMemsetAsync(d_r2.p, 0, n * sizeof(double), c->st));
      dwork.ensure((size_t)dot_work((int64_t)l * l));
      // ---------------- forward sweep ----------------
      SiteBatch Cprev;
      std::vector<FirstOrder> HL(l);
      std::vector<SiteBatch> L1(k);
      for (int i = 0; i < k; ++i) {
        SiteBatch C1;
        batch_alloc(c, C1, T(i), l, blk);
        SetBatch HRrot;
        if (m > 0) {
          // Eq. ritzrot2 at this site: R1 and the first-order right sets of bond i+1
          SiteBatch R1;
          batch_alloc(c, R1, T(i), m, blk);
          launch_rotate(oldR1[i].buf.p, oldR1[i].stride, lold, d_alpha.p, m, R1.buf.p, R1.stride, T(i), c->st);
          if (i + 1 < k && !oldHR[i + 1].empty()) {
            const SetBatch& O = oldHR[i + 1];
            set_batch(c, HRrot, *O.fp, *O.rp, m);
            launch_rotate(O.f.p, O.fs, lold, d_alpha.p, m, HRrot.f.p, HRrot.fs, O.fp->total, c->st);
            launch_rotate(O.r.p, O.rs, lold, d_alpha.p, m, HRrot.r.p, HRrot.rs, O.rp->total, c->st);
          }
          // Eq. gauge_fwd: C1_i = (L0_{i-1}^T C1_{i-1}) R0_i + Lambda_i R1_i
          if (i > 0) {
            BondBatch X;
            b_lc(i - 1, L0(i - 1), Cprev, m, X);
            b_lmulb(i, X, m, R0(i), C1, false);
            b_lmul(i, lam[i], R1, m, C1, true);
          } else {
            b_lmul(i, lam[0], R1, m, C1, false);
          }
        }
        if (want_gamma && m > 0) {       // the roots' site tensors of this sweep (transition densities)
          batch_alloc(c, keepC[i], T(i), n, blk);
          b_copy(C1, 0, n, keepC[i], 0);
        }
        // [H_mu^{L} x h x H_0^{R}] C0 for every vector (Eq. sigv2, first line); it enters
        // both the site sigma of the corrections and the reduced matrices below
        SiteBatch dHC0;
        batch_alloc(c, dHC0, T(i), l, blk);
        std::vector<Enl> XE = enlarge_left_batch(i, HL);
        dh_left_batch(i, XE, dHC0);
        // correction vectors (Eqs. sigv1, rnorm, error, param)
        if (first) {
          for (int mu = 0; mu < n; ++mu) start_site(i, mu, C1.v(m + mu));
          b_projC(i, C1, m, n);
        } else {
          SiteBatch sig, t1;
          batch_alloc(c, sig, T(i), n, blk);
          batch_alloc(c, t1, T(i), n, blk);
          h0(i, C1, n, sig);
          b_axpy(1.0, dHC0, 0, sig, 0, n);
          dh_right_batch(i, HRrot, n, t1);
          b_axpy(1.0, t1, 0, sig, 0, n);
          launch_rank1_batch(C1.v(0), C1.stride, d_theta.p, -1.0, n, sig.v(0), sig.stride, T(i), c->st);  // r
          b_projC(i, sig, 0, n);                                                                           // Q^C r
          launch_vdots(sig.v(0), sig.stride, sig.v(0), sig.stride, n, T(i), d_r2.p, true, dwork.p, c->st);
          if (any_gs) {
            // roots with the sweep correction: z_i = -D^-1 Q^C (r_i + [H_z^{L_{i-1}} x h_i x
            // H_0^{R_i}] C0_i), the new vector's own left part (sites < i) entering its
            // site-i equation
            launch_rank1_batch(dHC0.v(m), dHC0.stride, d_gs.p, 1.0, n, sig.v(0), sig.stride, T(i), c->st);
            b_projC(i, sig, 0, n);
          }
          // -D^-1 r (Eq. error; the sign of a new trial vector does not change the subspace)
          launch_precond_batch(sig.v(0), sig.stride, diag[i].p, d_theta.p, n, T(i), C1.v(m), C1.stride, 1.0,
                               c->st);
          b_projC(i, C1, m, n);
        }
        // projected coefficients (Eq. cwfn1st) and reduced matrices (Eqs. hleft2, sleft2)
        SiteBatch Ct, H0Ct;
        batch_alloc(c, Ct, T(i), l, blk);
        batch_alloc(c, H0Ct, T(i), l, blk);
        b_projL(i, C1, l, Ct);
        h0(i, Ct, l, H0Ct);
        double* D1 = d_D.p;
        double* D2 = D1 + (size_t)l * l;
        double* D3 = D2 + (size_t)l * l;
        launch_pair_dots_strided(Ct.v(0), Ct.stride, l, H0Ct.v(0), H0Ct.stride, l, T(i), D1, dwork.p, c->st);
        launch_pair_dots_strided(Ct.v(0), Ct.stride, l, dHC0.v(0), dHC0.stride, l, T(i), D2, dwork.p, c->st);
        launch_pair_dots_strided(Ct.v(0), Ct.stride, l, Ct.v(0), Ct.stride, l, T(i), D3, dwork.p, c->st);
        launch_reduced_acc(D1, D2, D3, l, d_H.p, d_S.p, c->st);
        // Eqs. left1st and lopr1st
        batch_alloc(c, L1[i], T(i), l, blk);
        b_rmul(i, Ct, l, ilam[i + 1], L1[i], false);
        if (i + 1 < k) HL = grow_HL_batch(i, XE, L1[i], l);
        Cprev = std::move(C1);
      }
      HL.clear();
      // ---------------- backward sweep ----------------
      std::vector<SiteBatch> newR1(k);
      std::vector<SetBatch> newHR(k + 1);
      std::vector<FirstOrder> HR(l);
      SiteBatch Cb;
      batch_alloc(c, Cb, T(k - 1), l, blk);
      b_rmul(k - 1, L1[k - 1], l, lam[k], Cb, false);
      for (int i = k - 1; i >= 0; --i) {
        if (i < k - 1) {
          // Eq. gauge_bwd: C1_i = L1_i Lambda_{i+1} + L0_i (C1_{i+1} R0_{i+1}^T)
          BondBatch Y;
          b_rc(i + 1, Cb, l, R0(i + 1), Y);
          SiteBatch nb;
          batch_alloc(c, nb, T(i), l, blk);
          b_rmul(i, L1[i], l, lam[i + 1], nb, false);
          b_rmulb(i, L0(i), Y, l, nb, true);
          Cb = std::move(nb);
        }
        L1[i] = SiteBatch();
        // Eq. right1st
        SiteBatch pr;
        batch_alloc(c, pr, T(i), l, blk);
        b_projR(i, Cb, l, pr);
        batch_alloc(c, newR1[i], T(i), l, blk);
        b_lmul(i, ilam[i], pr, l, newR1[i], false);
        if (i > 0) {
          HR = grow_HR_batch(i, HR, newR1[i], l);
          set_batch(c, newHR[i], *HR[0].f, *HR[0].r, l);
          for (int mu = 0; mu < l; ++mu) {
            if (HR[mu].f->total != HR[0].f->total || HR[mu].r->total != HR[0].r->total)
              throw Error(LRT_EINVAL, "sweep_tda: first-order right sets of different layouts");
            if (HR[mu].f->total > 0)
              CK(cudaMemcpyAsync(newHR[i].fv(mu), HR[mu].f->d, (size_t)HR[mu].f->total * sizeof(double),
                                 cudaMemcpyDeviceToDevice, c->st));
            if (HR[mu].r->total > 0)
              CK(cudaMemcpyAsync(newHR[i].rv(mu), HR[mu].r->d, (size_t)HR[mu].r->total * sizeof(double),
                                 cudaMemcpyDeviceToDevice, c->st));
          }
        }
      }
      HR.clear();
      oldR1 = std::move(newR1);
      oldHR = std::move(newHR);
      lold = l;
      // the sweep's reduced matrices and residual norms: the one synchronization
      Hr.assign((size_t)l * l, 0.0);
      Sr.assign((size_t)l * l, 0.0);
      CK(cudaMemcpyAsync(Hr.data(), d_H.p, Hr.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaMemcpyAsync(Sr.data(), d_S.p, Sr.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaMemcpyAsync(r2.data(), d_r2.p, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      CK(cudaGetLastError());
      c->sweep_log.push_back(
          {std::chrono::duration<double>(std::chrono::steady_clock::now() - t_sweep).count(), sweep_mixed ? 1 : 0});
      if (!first) {
        ++it;
        bool conv = true;
        for (int mu = 0; mu < n; ++mu) conv = conv && (r2[mu] < P.eps);
        if (mixed) {
          // FP64 residual correction: once the tensor-core sweeps have brought every
          // residual below refine_tol, the remaining sweeps (and the results) are FP64
          const double rt = P.refine_tol > 0.0 ? P.refine_tol : 1e-6;
          bool low = true;
          for (int mu = 0; mu < n; ++mu) low = low && (r2[mu] < std::max(rt, P.eps));
          // at the latest after two thirds of the sweeps, so that the last ones are FP64
          if (low || it >= (2 * P.max_iter) / 3) mixed = false;
          conv = false;
        }
        if (conv || it >= P.max_iter) {
          for (int mu = 0; mu < n; ++mu) {
            theta_out[mu] = mu < (int)theta.size() ? theta[mu] : 0.0;
            resid_out[mu] = r2[mu];
          }
          if (iters_out) *iters_out = it;
          if (want_gamma) compute_gamma(n, gamma_out);
          if (!conv) throw Error(LRT_ENOCONV, "sweep_tda: not converged within max_iter");
          return;
        }
      }
      first = false;
      // keep the whole subspace while the next one (at most l + n vectors: the GEP may drop
      // directions of S below the cut, so l need not be a multiple of n) still fits in N;
      // otherwise restart from the lowest Ritz vectors
      m = (l + n <= N) ? l : keep;
    }
  }

  // ---- frequency-dependent linear response at the Tamm-Dancoff level ----
  // (Eqs. realresp, imagresp): the first-order wavefunction X of a one-body perturbation V
  // in the tangent space, from the site equations
  //     Q^C (H_0^[i] - shift) Q^C C1_i = -Q^C (ΔH_i C0 + V_i C0),
  // ΔH_i C0 the products of the first-order left and right sets of the rest of X (as in the
  // TDA's sigma, Eq. sigv2) and V_i C0 the site-i effective V applied to C0 (`vc0`).  Each
  // forward sweep solves every site in turn, the rest of X fixed (site Gauss-Seidel), by
  // preconditioned MINRES (the shifted equations may be indefinite); the backward sweep
  // carries the gauge and builds the first-order right sets as in the TDA.  Returns
  // <V Psi0|X> = sum_i <piece_i, V_i C0> over the centred one-site pieces of X (the
  // decomposition of the transition densities); res2 = the last sweep's sum_i |site
  // residual|^2 before its solve.
  DevBuf rtmp;
  double dotd(const double* a, const double* b, int64_t n) {
    rtmp.ensure(8);
    return dev_dot(a, b, n, rtmp.p, c->st);
  }
  // y = a x + b y
  void axpbyd(double a, const double* x, double b, double* y, int64_t n) {
    rtmp.ensure(8);
    CK(cudaMemcpyAsync(rtmp.p, &a, sizeof(double), cudaMemcpyHostToDevice, c->st));
    launch_lincomb(x, n, 1, rtmp.p, n, y, b, c->st);
    CK(cudaStreamSynchronize(c->st));
  }
  void projCd(int i, double* x) { axpbyd(-dotd(C0(i).d, x, T(i)), C0(i).d, 1.0, x, T(i)); }
  // x = solution of Q (H_0^[i] - shift) Q x = b (b orthogonal to C0_i), x on entry the
  // start; preconditioned MINRES with M = |diag H_0^[i] - shift|, both projected by Q^C
  int site_minres(int i, double shift, const double* b, double* x, int maxit, double rtol) {
    const int64_t n = T(i);
    if (n == 0) return 0;
    std::vector<DevBuf> buf(9);
    for (auto& q : buf) {
      q.ensure((size_t)n);
      CK(cudaMemsetAsync(q.p, 0, (size_t)n * sizeof(double), c->st));
    }
    double *v0 = buf[0].p, *v1 = buf[1].p, *v2 = buf[2].p, *z1 = buf[3].p, *z2 = buf[4].p, *w0 = buf[5].p,
           *w1 = buf[6].p, *w2 = buf[7].p, *az = buf[8].p;
    auto A = [&](const double* in, double* out) {   // out = Q (H_0 - shift) in, in orthogonal to C0
      run_plan(*h0one[i], in, out, 1, false);
      axpbyd(-shift, in, 1.0, out, n);
      projCd(i, out);
    };
    auto Minv = [&](const double* in, double* out) {
      launch_precond_abs(in, diag[i].p, shift, n, out, c->st);
      projCd(i, out);
    };
    projCd(i, x);
    A(x, az);                                       // v1 = b - A x
    CK(cudaMemcpyAsync(v1, b, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    axpbyd(-1.0, az, 1.0, v1, n);
    Minv(v1, z1);
    double g1 = std::sqrt(std::max(0.0, dotd(z1, v1, n)));
    const double g_start = g1;
    if (!(g1 > 0.0)) return 0;
    double g0 = 1.0, eta = g1, s0 = 0.0, s1 = 0.0, c0 = 1.0, c1 = 1.0;
    int it = 0;
    while (it < maxit) {
      ++it;
      axpbyd(0.0, z1, 1.0 / g1, z1, n);             // z1 /= g1
      A(z1, az);
      const double delta = dotd(az, z1, n);
      CK(cudaMemcpyAsync(v2, az, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      axpbyd(-delta / g1, v1, 1.0, v2, n);
      axpbyd(-g1 / g0, v0, 1.0, v2, n);
      Minv(v2, z2);
      const double g2 = std::sqrt(std::max(0.0, dotd(z2, v2, n)));
      const double a0 = c1 * delta - c0 * s1 * g1;
      const double a1 = std::sqrt(a0 * a0 + g2 * g2);
      const double a2 = s1 * delta + c0 * c1 * g1;
      const double a3 = s0 * g1;
      if (!(a1 > 0.0)) break;
      const double c2 = a0 / a1, s2 = g2 / a1;
      // w2 = (z1 - a3 w0 - a2 w1) / a1
      CK(cudaMemcpyAsync(w2, z1, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      axpbyd(-a3, w0, 1.0, w2, n);
      axpbyd(-a2, w1, 1.0, w2, n);
      axpbyd(0.0, w2, 1.0 / a1, w2, n);
      axpbyd(c2 * eta, w2, 1.0, x, n);
      eta = -s2 * eta;
      std::swap(v0, v1);
      std::swap(v1, v2);
      std::swap(z1, z2);
      std::swap(w0, w1);
      std::swap(w1, w2);
      g0 = g1;
      g1 = g2;
      c0 = c1;
      c1 = c2;
      s0 = s1;
      s1 = s2;
      if (std::fabs(eta) <= rtol * g_start || !(g2 > 0.0)) break;
    }
    return it;
  }

  // The same response component in a growing subspace of tangent vectors (the sweep
  // Davidson of the TDA, Fig. alg:dmrgtda, carried to the linear system): every sweep adds
  // the preconditioned residual of the current solution X as a new trial vector, and X is
  // the Galerkin solution of (H - shift) X = -v on the subspace, from the reduced matrices
  // H_R, S_R of the sweep (Eqs. hleft2, sleft2) and b_R = <trial|V Psi0> summed site by site
  // over the same left-gauge pieces.  The reduced system is solved through the S-orthonormal
  // Ritz vectors (c = -sum_k u_k (u_k . b_R) / (w_k - shift)), which takes any shift; with
  // the diagonal preconditioner the subspace converges fast below the first pole and slowly
  // for the indefinite component between poles.  Vector 0 of every sweep is the current X; the others are the Ritz
  // vectors of the last subspace (all but the highest, which X replaces), or the lowest
  // keep of them at a restart.  Returns <V Psi0|X> for the X whose residual is res2.
  double response_krylov(const std::vector<DevBuf>& vc0, double shift, int max_iter, double tol, int max_space,
                         double& res2_out, int& sweeps_out) {
    blk = 1;
    const int N = std::max(4, std::min(max_space > 0 ? max_space : 24, JACOBI_MAXN));
    const int keep = std::max(2, N / 2);
    std::vector<SiteBatch> oldR1(k);
    std::vector<SetBatch> oldHR(k + 1);
    int lold = 0, m = 0, it = 0;
    bool first = true;
    std::vector<double> Hr, Sr, bR, alpha, bsite;
    double r2 = 0.0, a_prev = 0.0;
    DevBuf d_alpha, d_shift, d_H, d_S, d_D, d_r2, d_b;
    d_shift.ensure(1);
    CK(cudaMemcpyAsync(d_shift.p, &shift, sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (;;) {
      if (!first) {
        std::vector<double> w, U;
        solve_gep(Hr, Sr, lold, w, U);
        const int r = (int)w.size();
        if (r < 1) throw Error(LRT_EINVAL, "sweep_response: the trial subspace is empty");
        std::vector<double> cvec(lold, 0.0);
        for (int q = 0; q < r; ++q) {
          double ub = 0.0;
          for (int a = 0; a < lold; ++a) ub += U[(size_t)a * r + q] * bR[a];
          const double den = w[q] - shift;
          const double f = std::fabs(den) > 1e-300 ? -ub / den : 0.0;
          for (int a = 0; a < lold; ++a) cvec[a] += f * U[(size_t)a * r + q];
        }
        a_prev = 0.0;
        for (int a = 0; a < lold; ++a) a_prev += bR[a] * cvec[a];
        const int nritz = (lold + 1 <= N) ? r - 1 : std::min(r, keep) - 1;
        m = 1 + std::max(0, nritz);
        alpha.assign((size_t)lold * m, 0.0);
        for (int a = 0; a < lold; ++a) {
          alpha[(size_t)a * m] = cvec[a];
          for (int j = 1; j < m; ++j) alpha[(size_t)a * m + j] = U[(size_t)a * r + (j - 1)];
        }
        d_alpha.ensure(alpha.size());
        CK(cudaMemcpyAsync(d_alpha.p, alpha.data(), alpha.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
      }
      const int l = m + 1;
      d_H.ensure((size_t)l * l);
      d_S.ensure((size_t)l * l);
      d_D.ensure((size_t)3 * l * l);
      d_r2.ensure(1);
      d_b.ensure((size_t)k * l);
      CK(cudaMemsetAsync(d_H.p, 0, (size_t)l * l * sizeof(double), c->st));
      CK(cudaMemsetAsync(d_S.p, 0, (size_t)l * l * sizeof(double), c->st));
      CK(cudaMemsetAsync(d_r2.p, 0, sizeof(double), c->st));
      CK(cudaMemsetAsync(d_b.p, 0, (size_t)k * l * sizeof(double), c->st));
      dwork.ensure((size_t)dot_work((int64_t)l * l));
      // ---------------- forward sweep ----------------
      SiteBatch Cprev;
      std::vector<FirstOrder> HL(l);
      std::vector<SiteBatch> L1(k);
      for (int i = 0; i < k; ++i) {
        SiteBatch C1;
        batch_alloc(c, C1, T(i), l, 1);
        SetBatch HRrot;
        if (m > 0) {
          SiteBatch R1;
          batch_alloc(c, R1, T(i), m, 1);
          launch_rotate(oldR1[i].buf.p, oldR1[i].stride, lold, d_alpha.p, m, R1.buf.p, R1.stride, T(i), c->st);
          if (i + 1 < k && !oldHR[i + 1].empty()) {
            const SetBatch& O = oldHR[i + 1];
            set_batch(c, HRrot, *O.fp, *O.rp, m);
            launch_rotate(O.f.p, O.fs, lold, d_alpha.p, m, HRrot.f.p, HRrot.fs, O.fp->total, c->st);
            launch_rotate(O.r.p, O.rs, lold, d_alpha.p, m, HRrot.r.p, HRrot.rs, O.rp->total, c->st);
          }
          if (i > 0) {
            BondBatch X;
            b_lc(i - 1, L0(i - 1), Cprev, m, X);
            b_lmulb(i, X, m, R0(i), C1, false);
            b_lmul(i, lam[i], R1, m, C1, true);
          } else {
            b_lmul(i, lam[0], R1, m, C1, false);
          }
        }
        SiteBatch dHC0;
        batch_alloc(c, dHC0, T(i), l, 1);
        std::vector<Enl> XE = enlarge_left_batch(i, HL);
        dh_left_batch(i, XE, dHC0);
        if (T(i) > 0) {
          if (first) {
            // start: the preconditioned drive, -V_i C0 / (diag - shift)
            launch_precond_batch(vc0[i].p, T(i), diag[i].p, d_shift.p, 1, T(i), C1.v(0), C1.stride, 1.0, c->st);
            b_projC(i, C1, 0, 1);
          } else {
            // residual of X (vector 0): H_0 C1 + dH C0 - shift C1 + V_i C0, projected
            SiteBatch sig, t1;
            batch_alloc(c, sig, T(i), 1, 1);
            batch_alloc(c, t1, T(i), 1, 1);
            h0(i, C1, 1, sig);
            b_axpy(1.0, dHC0, 0, sig, 0, 1);
            dh_right_batch(i, HRrot, 1, t1);
            b_axpy(1.0, t1, 0, sig, 0, 1);
            launch_rank1_batch(C1.v(0), C1.stride, d_shift.p, -1.0, 1, sig.v(0), sig.stride, T(i), c->st);
            launch_rank1_batch(vc0[i].p, T(i), nullptr, 1.0, 1, sig.v(0), sig.stride, T(i), c->st);
            b_projC(i, sig, 0, 1);
            launch_vdots(sig.v(0), sig.stride, sig.v(0), sig.stride, 1, T(i), d_r2.p, true, dwork.p, c->st);
            // the correction -D^-1 r as the new trial vector
            launch_precond_batch(sig.v(0), sig.stride, diag[i].p, d_shift.p, 1, T(i), C1.v(m), C1.stride, 1.0, c->st);
            b_projC(i, C1, m, 1);
          }
        }
        // reduced matrices and the drive b_R (Eqs. cwfn1st, hleft2, sleft2)
        SiteBatch Ct, H0Ct;
        batch_alloc(c, Ct, T(i), l, 1);
        batch_alloc(c, H0Ct, T(i), l, 1);
        b_projL(i, C1, l, Ct);
        h0(i, Ct, l, H0Ct);
        if (T(i) > 0) {
          double* D1 = d_D.p;
          double* D2 = D1 + (size_t)l * l;
          double* D3 = D2 + (size_t)l * l;
          launch_pair_dots_strided(Ct.v(0), Ct.stride, l, H0Ct.v(0), H0Ct.stride, l, T(i), D1, dwork.p, c->st);
          launch_pair_dots_strided(Ct.v(0), Ct.stride, l, dHC0.v(0), dHC0.stride, l, T(i), D2, dwork.p, c->st);
          launch_pair_dots_strided(Ct.v(0), Ct.stride, l, Ct.v(0), Ct.stride, l, T(i), D3, dwork.p, c->st);
          launch_reduced_acc(D1, D2, D3, l, d_H.p, d_S.p, c->st);
          launch_pair_dots_strided(Ct.v(0), Ct.stride, l, vc0[i].p, T(i), 1, T(i), d_b.p + (size_t)i * l, dwork.p,
                                   c->st);
        }
        batch_alloc(c, L1[i], T(i), l, 1);
        b_rmul(i, Ct, l, ilam[i + 1], L1[i], false);
        if (i + 1 < k) HL = grow_HL_batch(i, XE, L1[i], l);
        Cprev = std::move(C1);
      }
      HL.clear();
      // ---------------- backward sweep ----------------
      std::vector<SiteBatch> newR1(k);
      std::vector<SetBatch> newHR(k + 1);
      std::vector<FirstOrder> HR(l);
      SiteBatch Cb;
      batch_alloc(c, Cb, T(k - 1), l, 1);
      b_rmul(k - 1, L1[k - 1], l, lam[k], Cb, false);
      for (int i = k - 1; i >= 0; --i) {
        if (i < k - 1) {
          BondBatch Y;
          b_rc(i + 1, Cb, l, R0(i + 1), Y);
          SiteBatch nb;
          batch_alloc(c, nb, T(i), l, 1);
          b_rmul(i, L1[i], l, lam[i + 1], nb, false);
          b_rmulb(i, L0(i), Y, l, nb, true);
          Cb = std::move(nb);
        }
        L1[i] = SiteBatch();
        SiteBatch pr;
        batch_alloc(c, pr, T(i), l, 1);
        b_projR(i, Cb, l, pr);
        batch_alloc(c, newR1[i], T(i), l, 1);
        b_lmul(i, ilam[i], pr, l, newR1[i], false);
        if (i > 0) {
          HR = grow_HR_batch(i, HR, newR1[i], l);
          set_batch(c, newHR[i], *HR[0].f, *HR[0].r, l);
          for (int mu = 0; mu < l; ++mu) {
            if (HR[mu].f->total != HR[0].f->total || HR[mu].r->total != HR[0].r->total)
              throw Error(LRT_EINVAL, "sweep_response: first-order right sets of different layouts");
            if (HR[mu].f->total > 0)
              CK(cudaMemcpyAsync(newHR[i].fv(mu), HR[mu].f->d, (size_t)HR[mu].f->total * sizeof(double),
                                 cudaMemcpyDeviceToDevice, c->st));
            if (HR[mu].r->total > 0)
              CK(cudaMemcpyAsync(newHR[i].rv(mu), HR[mu].r->d, (size_t)HR[mu].r->total * sizeof(double),
                                 cudaMemcpyDeviceToDevice, c->st));
          }
        }
      }
      HR.clear();
      oldR1 = std::move(newR1);
      oldHR = std::move(newHR);
      lold = l;
      Hr.assign((size_t)l * l, 0.0);
      Sr.assign((size_t)l * l, 0.0);
      bsite.assign((size_t)k * l, 0.0);
      CK(cudaMemcpyAsync(Hr.data(), d_H.p, Hr.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaMemcpyAsync(Sr.data(), d_S.p, Sr.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaMemcpyAsync(bsite.data(), d_b.p, bsite.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaMemcpyAsync(&r2, d_r2.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      CK(cudaGetLastError());
      bR.assign(l, 0.0);
      for (int i = 0; i < k; ++i)
        for (int a = 0; a < l; ++a) bR[a] += bsite[(size_t)i * l + a];
      if (!first) {
        ++it;
        if (r2 < tol || it >= max_iter) break;
      }
      first = false;
    }
    res2_out = r2;
    sweeps_out = it;
    return a_prev;
  }

  double response_component(const std::vector<DevBuf>& vc0, double shift, int max_sweeps, double tol, int mr_max,
                             double mr_tol, double& res2_out, int& sweeps_out) {
    blk = 1;
    std::vector<SiteBatch> oldR1(k);
    std::vector<SetBatch> oldHR(k + 1);
    bool have_old = false;
    std::vector<SiteBatch> keep(k);
    double res2 = 0.0;
    int sw = 0;
    while (sw < max_sweeps) {
      ++sw;
      res2 = 0.0;
      // ---------------- forward sweep: solve every site ----------------
      SiteBatch Cprev;
      std::vector<FirstOrder> HL(1);
      std::vector<SiteBatch> L1(k);
      for (int i = 0; i < k; ++i) {
        SiteBatch C1;
        batch_alloc(c, C1, T(i), 1, 1);
        // Eq. gauge_fwd: the left part carried in, the right part of the last backward sweep
        if (i > 0) {
          BondBatch X;
          b_lc(i - 1, L0(i - 1), Cprev, 1, X);
          b_lmulb(i, X, 1, R0(i), C1, false);
          if (have_old) b_lmul(i, lam[i], oldR1[i], 1, C1, true);
        } else if (have_old) {
          b_lmul(i, lam[0], oldR1[i], 1, C1, false);
        }
        // rhs = -Q^C (ΔH_i C0 + V_i C0)
        SiteBatch dl, dr, rhs;
        batch_alloc(c, dl, T(i), 1, 1);
        batch_alloc(c, dr, T(i), 1, 1);
        batch_alloc(c, rhs, T(i), 1, 1);
        std::vector<Enl> XE = enlarge_left_batch(i, HL);
        dh_left_batch(i, XE, dl);
        if (have_old && i + 1 < k && !oldHR[i + 1].empty()) dh_right_batch(i, oldHR[i + 1], 1, dr);
        if (T(i) > 0) {
          double* r = rhs.v(0);
          axpbyd(-1.0, dl.v(0), 0.0, r, T(i));
          axpbyd(-1.0, dr.v(0), 1.0, r, T(i));
          axpbyd(-1.0, vc0[i].p, 1.0, r, T(i));
          projCd(i, r);
          // the residual of the current C1_i, then the solve from it
          DevBuf az;
          az.ensure((size_t)T(i));
          projCd(i, C1.v(0));
          run_plan(*h0one[i], C1.v(0), az.p, 1, false);
          axpbyd(-shift, C1.v(0), 1.0, az.p, T(i));
          projCd(i, az.p);
          axpbyd(-1.0, r, 1.0, az.p, T(i));
          res2 += dotd(az.p, az.p, T(i));
          site_minres(i, shift, r, C1.v(0), mr_max, mr_tol);
        }
        batch_alloc(c, keep[i], T(i), 1, 1);
        b_copy(C1, 0, 1, keep[i], 0);
        // Eqs. left1st and lopr1st
        SiteBatch Ct;
        batch_alloc(c, Ct, T(i), 1, 1);
        b_projL(i, C1, 1, Ct);
        batch_alloc(c, L1[i], T(i), 1, 1);
        b_rmul(i, Ct, 1, ilam[i + 1], L1[i], false);
        if (i + 1 < k) HL = grow_HL_batch(i, XE, L1[i], 1);
        Cprev = std::move(C1);
      }
      HL.clear();
      // ---------------- backward sweep: gauge, R1 and the first-order right sets ----------------
      std::vector<SiteBatch> newR1(k);
      std::vector<SetBatch> newHR(k + 1);
      std::vector<FirstOrder> HR(1);
      SiteBatch Cb;
      batch_alloc(c, Cb, T(k - 1), 1, 1);
      b_rmul(k - 1, L1[k - 1], 1, lam[k], Cb, false);
      for (int i = k - 1; i >= 0; --i) {
        if (i < k - 1) {
          BondBatch Y;
          b_rc(i + 1, Cb, 1, R0(i + 1), Y);
          SiteBatch nb;
          batch_alloc(c, nb, T(i), 1, 1);
          b_rmul(i, L1[i], 1, lam[i + 1], nb, false);
          b_rmulb(i, L0(i), Y, 1, nb, true);
          Cb = std::move(nb);
        }
        L1[i] = SiteBatch();
        SiteBatch pr;
        batch_alloc(c, pr, T(i), 1, 1);
        b_projR(i, Cb, 1, pr);
        batch_alloc(c, newR1[i], T(i), 1, 1);
        b_lmul(i, ilam[i], pr, 1, newR1[i], false);
        if (i > 0) {
          HR = grow_HR_batch(i, HR, newR1[i], 1);
          set_batch(c, newHR[i], *HR[0].f, *HR[0].r, 1);
          if (HR[0].f->total > 0)
            CK(cudaMemcpyAsync(newHR[i].fv(0), HR[0].f->d, (size_t)HR[0].f->total * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->st));
          if (HR[0].r->total > 0)
            CK(cudaMemcpyAsync(newHR[i].rv(0), HR[0].r->d, (size_t)HR[0].r->total * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->st));
        }
      }
      HR.clear();
      oldR1 = std::move(newR1);
      oldHR = std::move(newHR);
      have_old = true;
      CK(cudaStreamSynchronize(c->st));
      if (sw > 1 && res2 < tol) break;
    }
    // <V Psi0|X> over the centred pieces of the last forward sweep
    const int cc = k / 2;
    double a = 0.0;
    for (int i = 0; i < k; ++i) {
      if (T(i) == 0) continue;
      SiteBatch P;
      batch_alloc(c, P, T(i), 1, 1);
      if (i < cc) b_projL(i, keep[i], 1, P);
      else if (i == cc) b_copy(keep[i], 0, 1, P, 0);
      else b_projR(i, keep[i], 1, P);
      a += dotd(P.v(0), vc0[i].p, T(i));
    }
    res2_out = res2;
    sweeps_out = sw;
    return a;
  }
};

// Mixed-canonical gauge of the whole MPS (the form the TDA sweep works in): on every
// bond the Schmidt basis, with C0_i = L0_i Lambda_{i+1} = Lambda_i R0_i.  Input: the
// MPS in c->sites with sites 1..k-1 right-orthonormal and the centre at site 0 (the
// state sweep_gs leaves).  A left-to-right pass, per right sector of every site, takes
// the SVD of the left-fused C_i = Lambda_i V_prev^T R_i = L S Vn^T (cuSOLVER Jacobi SVD,
// FP64 on the GPU): L0_i = L, Lambda_{i+1} = S, R0_i = V_prev^T R_i Vn, C0_i = C_i Vn.
// Bond dimensions are kept: when a sector has fewer fused rows than states, the
// missing singular values are zero and the matching columns of L0 are zero.
static void tda_prepare_impl(lrt_ctx* c, double* norm_out) {
  const int k = c->k;
  cudaStream_t st = c->st;
  SolverHandle sh;
  if (cusolverDnCreate(&sh.h) != CUSOLVER_STATUS_SUCCESS) throw Error(LRT_ECUDA, "cusolverDnCreate failed");
  cusolverDnSetStream(sh.h, st);
  gesvdjInfo_t params = nullptr;
  if (cusolverDnCreateGesvdjInfo(&params) != CUSOLVER_STATUS_SUCCESS) throw Error(LRT_ECUDA, "gesvdj info");
  struct ParamsGuard {
    gesvdjInfo_t p;
    ~ParamsGuard() {
      if (p) cusolverDnDestroyGesvdjInfo(p);
    }
  } pg{params};
  DevBuf tmp, work, A, U, V, S;
  tmp.ensure(4);
  int* dinfo = nullptr;
  if (dev_alloc((void**)&dinfo, sizeof(int)) != cudaSuccess) throw Error(LRT_ENOMEM, "cusolver info");
  struct InfoGuard {
    int* p;
    ~InfoGuard() { dev_free(p); }
  } ig{dinfo};

  // normalize the centre
  SiteTensor& S0 = c->sites[0];
  const double nrm = std::sqrt(std::max(0.0, dev_dot(S0.d, S0.d, S0.total, tmp.p, st)));
  if (!(nrm > 0.0)) throw Error(LRT_EINVAL, "tda_prepare: zero wavefunction");
  t_axpby(c, 1.0 / nrm, S0, 0.0, S0, tmp);
  if (norm_out) *norm_out = nrm;

  auto tda = std::make_unique<TdaState>();
  tda->C0.resize(k);
  tda->lam.resize(k + 1);
  tda->lam[0].assign(1, 1.0);
  std::vector<SiteTensor> L0(k), R0(k);
  // X = Lambda_i V_prev^T and V_prev^T on bond i (identity on bond 0)
  BondMat X, VT;
  bond_layout(c->bonds[0], X, st);
  bond_layout(c->bonds[0], VT, st);
  {
    const double one = 1.0;
    CK(cudaMemcpyAsync(X.buf.p, &one, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(VT.buf.p, &one, sizeof(double), cudaMemcpyHostToDevice, st));
  }
  for (int i = 0; i < k; ++i) {
    const Sectors& Rb = c->bonds[i + 1];
    const SiteTensor& Ri = c->sites[i];
    SiteTensor Ci = new_site(c, i), Rt = new_site(c, i);
    t_lmul(c, i, X, Ri, Ci, false);
    t_lmul(c, i, VT, Ri, Rt, false);
    SiteTensor Li = new_site(c, i);
    BondMat Vn;
    bond_layout(Rb, Vn, st);
    std::vector<double> lam;
    std::vector<GatherTask> tasks;
    std::vector<GatherSrc> srcs;
    // SVD results of all sectors live in U/V buffers until the gathers below
    std::vector<int64_t> uoff(Rb.n(), -1), voff(Rb.n(), -1);
    int64_t ut = 0, vt = 0, at = 0;
    for (int q = 0; q < Rb.n(); ++q) {
      const int D = Rb.d[q], rows = Ci.blk_off[q] >= 0 ? Ci.blk_rows[q] : 0;
      if (rows == 0 || D == 0) continue;
      uoff[q] = ut;
      voff[q] = vt;
      ut += (int64_t)D * D;
      vt += (int64_t)rows * rows;
      at = std::max<int64_t>(at, (int64_t)D * rows);
    }
    U.ensure(std::max<int64_t>(ut, 1));
    V.ensure(std::max<int64_t>(vt, 1));
    A.ensure(std::max<int64_t>(at, 1));
    S.ensure(1);
    std::vector<double> sv;
    for (int q = 0; q < Rb.n(); ++q) {
      const int D = Rb.d[q];
      if (uoff[q] < 0) {
        // no fused rows: Schmidt values zero, rotation the identity
        std::vector<double> I((size_t)D * D, 0.0);
        for (int a = 0; a < D; ++a) I[(size_t)a * D + a] = 1.0;
        if (D > 0)
          CK(cudaMemcpyAsync(Vn.buf.p + Vn.off[q], I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        lam.insert(lam.end(), D, 0.0);
        CK(cudaStreamSynchronize(st));
        continue;
      }
      const int rows = Ci.blk_rows[q];
      const int p = std::min(D, rows);
      // the row-major block (rows x D) is the column-major D x rows matrix A = M^T;
      // A = U_a S V_a^T gives M = V_a S U_a^T
      CK(cudaMemcpyAsync(A.p, Ci.d + Ci.blk_off[q], (size_t)D * rows * sizeof(double), cudaMemcpyDeviceToDevice, st));
      S.ensure(std::max(1, p));
      int lwork = 0;
      if (cusolverDnDgesvdj_bufferSize(sh.h, CUSOLVER_EIG_MODE_VECTOR, 0, D, rows, A.p, D, S.p, U.p + uoff[q], D,
                                       V.p + voff[q], rows, &lwork, params) != CUSOLVER_STATUS_SUCCESS)
        throw Error(LRT_ECUDA, "gesvdj buffer size");
      work.ensure(std::max(lwork, 1));
      if (cusolverDnDgesvdj(sh.h, CUSOLVER_EIG_MODE_VECTOR, 0, D, rows, A.p, D, S.p, U.p + uoff[q], D, V.p + voff[q],
                            rows, work.p, lwork, dinfo, params) != CUSOLVER_STATUS_SUCCESS)
        throw Error(LRT_ECUDA, "gesvdj");
      int info = 0;
      sv.resize(p);
      CK(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(sv.data(), S.p, p * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (info < 0) throw Error(LRT_ECUDA, "gesvdj: invalid argument " + std::to_string(-info));
      for (int a = 0; a < D; ++a) lam.push_back(a < p ? sv[a] : 0.0);
      // L block (rows x D, row-major): columns j < p are V_a's columns (column-major,
      // ld rows); Vn (D x D, row-major) = U_a (column-major, ld D)
      tasks.push_back(GatherTask{Li.d + Li.blk_off[q], D, rows, p, (int)srcs.size(), 1});
      srcs.push_back(GatherSrc{V.p + voff[q], rows, 1, 1.0});
      tasks.push_back(GatherTask{Vn.buf.p + Vn.off[q], D, D, D, (int)srcs.size(), 1});
      srcs.push_back(GatherSrc{U.p + uoff[q], D, 1, 1.0});
    }
    if (!tasks.empty()) {
      GatherPlan gp;
      build_gather(gp, tasks, srcs, st);
      gp.run(st);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(st));
    }
    SiteTensor C0 = new_site(c, i), R0i = new_site(c, i);
    t_rmul(c, i, Ci, Vn, C0, false);
    t_rmul(c, i, Rt, Vn, R0i, false);
    L0[i] = std::move(Li);
    R0[i] = std::move(R0i);
    tda->C0[i] = std::move(C0);
    tda->lam[i + 1] = lam;
    if (i + 1 < k) {
      // next bond: X = Lambda Vn^T, VT = Vn^T
      bond_layout(Rb, X, st);
      bond_layout(Rb, VT, st);
      std::vector<GatherTask> t2;
      std::vector<GatherSrc> s2;
      for (int q = 0; q < Rb.n(); ++q) {
        const int D = Rb.d[q];
        if (D == 0) continue;
        t2.push_back(GatherTask{VT.buf.p + VT.off[q], D, D, D, (int)s2.size(), 1});
        s2.push_back(GatherSrc{Vn.buf.p + Vn.off[q], D, 1, 1.0});
      }
      if (!t2.empty()) {
        GatherPlan gp;
        build_gather(gp, t2, s2, st);
        gp.run(st);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
      }
      // X_q = diag(lambda_q) VT_q
      std::vector<GemmOut> o;
      std::vector<GemmSeg> g;
      BondMat Lm, Lmi;
      lam_mats(c, i + 1, lam, 0.0, Lm, Lmi);
      for (int q = 0; q < Rb.n(); ++q) {
        const int D = Rb.d[q];
        if (D == 0) continue;
        o.push_back(GemmOut{X.buf.p + X.off[q], 0, D, D, D, (int)g.size(), 1, 0, 0});
        g.push_back(GemmSeg{Lm.buf.p + Lm.off[q], VT.buf.p + VT.off[q], 0, 0, D, D, D, 0, 0, 0, 0, 1.0});
      }
      run_gemms(c, o, g);
    }
  }
  c->sites = std::move(L0);
  c->sites_r = std::move(R0);
  tda->loaded = true;
  c->tda = std::move(tda);
  // environments and plans belong to the old gauge
  drop_plans(c);
  for (int b = 0; b < k; ++b) {
    c->XL[b].reset();
    c->YR[b].reset();
  }
  for (int b = 1; b < k; ++b) c->L[b].reset();
  for (int b = 0; b < k; ++b) c->R[b].reset();
}

}  // namespace lrt

// ===========================================================================
// batched sigma: several independent instances (contexts) in one grouped launch per
// phase, replayed from a CUDA graph while the caller's buffers stay the same
// ===========================================================================
namespace lrt {

struct BatchPlan {
  std::vector<uint64_t> ids, serials;   // instances and the plans this batch was built from
  int precision = LRT_FP64;
  double flops = 0.0;
  // FP64: merged task lists, bases (x, y, T) per instance
  GemmPlan p1, p2;
  DevArray<GemmBases> bases;
  std::vector<GemmBases> hbases;
  // split-TF32: merged work streams, y per instance
  DevArray<TcItem> tci1, tci2;
  DevArray<int> tcb1, tcb2;
  int tcn1 = 0, tcn2 = 0, tn1 = 64, tn2 = 64;
  DevArray<double*> ys;
  std::vector<double*> hys;
  // one call captured as a CUDA graph
  cudaGraphExec_t exec = nullptr;
  std::vector<const double*> gx;
  std::vector<double*> gy;
  bool ran = false;
  cudaStream_t cap = nullptr;   // private stream the call is captured on (the caller's may be the legacy one)
  ~BatchPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
  }
};

template <class T>
static std::vector<T> download(const DevArray<T>& a, cudaStream_t st) {
  std::vector<T> h(a.n);
  if (a.n) CK(cudaMemcpyAsync(h.data(), a.p, a.n * sizeof(T), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return h;
}

static void merge_fp64(GemmPlan& out, const std::vector<SigmaPlan*>& plans, bool phase2, cudaStream_t st) {
  std::vector<GemmOut> O;
  std::vector<GemmSeg> S;
  for (size_t j = 0; j < plans.size(); ++j) {
    const GemmPlan& g = phase2 ? plans[j]->p2 : plans[j]->p1;
    std::vector<GemmOut> o = download(g.outs, st);
    o.resize(g.nbase);   // not the K parts of split tiles: the merged plan tiles anew
    std::vector<GemmSeg> sg = download(g.segs, st);
    const int sb = (int)S.size();
    for (GemmOut x : o) {
      x.seg_begin += sb;
      x.inst = (int)j;
      O.push_back(x);
    }
    S.insert(S.end(), sg.begin(), sg.end());
  }
  build_gemm(out, O, S, st);
}

// one batched call (the graph body): no host synchronization inside
static void batch_issue(lrt_ctx* c0, BatchPlan& B, const std::vector<SigmaPlan*>& plans,
                        const std::vector<const double*>& x, int nvec, cudaStream_t st) {
  if (B.precision == LRT_MIXED) {
    for (size_t j = 0; j < plans.size(); ++j) {
      SigmaPlan& p = *plans[j];
      launch_tc_pack(p.xpack.p, (int)p.tc.pack1.size(), x[j], p.nelem, p.pool_hi[1], p.pool_lo[1],
                     p.tc.pool_size[1], nvec, st);
    }
    const TcOut to = tc_out(c0, nullptr, B.ys.p);
    launch_gemm_tf32x3(B.tci1.p, B.tcb1.p, B.tcn1, B.tn1, to, c0->derr, st);
    launch_gemm_tf32x3(B.tci2.p, B.tcb2.p, B.tcn2, B.tn2, to, c0->derr, st);
  } else {
    launch_gemm_fp64_multi(B.p1.outs.p, B.p1.segs.p, B.p1.tiles.p, B.p1.ntiles, B.bases.p, st);
    launch_gemm_fp64_multi(B.p2.outs.p, B.p2.segs.p, B.p2.tiles.p, B.p2.ntiles, B.bases.p, st);
  }
}

static void sigma_batched_impl(lrt_ctx* const* ctxs, int n, const int* sites, int nsite, int nvec,
                               const double* const* x, double* const* y, int precision) {
  lrt_ctx* c0 = ctxs[0];
  std::vector<SigmaPlan*> plans(n);
  std::string key = std::to_string(nsite) + ":" + std::to_string(nvec) + ":" + std::to_string(precision);
  for (int j = 0; j < n; ++j) {
    lrt_ctx* c = ctxs[j];
    if (!c) throw Error(LRT_EINVAL, "sigma_batched: NULL context");
    if (c->dev != c0->dev) throw Error(LRT_EINVAL, "sigma_batched: contexts on different devices");
    if (!c->have_mps || !c->have_ham) throw Error(LRT_ESTATE, "sigma_batched: op_build and mps_load first");
    if (sites[j] < 0 || sites[j] + nsite > c->k || !c->L[sites[j]])
      throw Error(LRT_ESTATE, "sigma_batched: environment of instance " + std::to_string(j) + " missing");
    if (!x[j] || !y[j]) throw Error(LRT_EINVAL, "sigma_batched: NULL vector");
    PoolScope ps(&c->pool);
    plans[j] = &get_plan(c, sites[j], nsite, nvec, precision == LRT_MIXED);
    key += ":" + std::to_string(c->id) + "/" + std::to_string(sites[j]);
  }
  auto& slot = c0->batches[key];
  bool fresh = false;
  if (slot) {
    for (int j = 0; j < n && !fresh; ++j) fresh = slot->serials[j] != plans[j]->serial;
  }
  if (!slot || fresh) {
    auto B = std::make_unique<BatchPlan>();
    B->precision = precision;
    for (int j = 0; j < n; ++j) {
      B->ids.push_back(ctxs[j]->id);
      B->serials.push_back(plans[j]->serial);
      B->flops += plans[j]->flops_alg;
    }
    if (precision == LRT_MIXED) {
      std::vector<TcSource> s1, s2;
      for (int j = 0; j < n; ++j) {
        PoolScope ps(&ctxs[j]->pool);
        prepare_tc(ctxs[j], *plans[j], nvec);
        SigmaPlan& p = *plans[j];
        s1.push_back(TcSource{&p.tc, &p.tc.out1, p.pool_hi, p.pool_lo, p.nelem, j});
        s2.push_back(TcSource{&p.tc, &p.tc.out2, p.pool_hi, p.pool_lo, p.nelem, j});
      }
      // tile widths tuned on the merged streams, outputs into per-instance scratch
      std::vector<DevBuf> scr(n);
      std::vector<double*> sp(n);
      for (int j = 0; j < n; ++j) sp[j] = scr[j].ensure((size_t)std::max<int64_t>(plans[j]->nelem * nvec, 1));
      DevArray<double*> sys;
      sys.upload(sp, c0->st);
      const TcOut scratch = tc_out(c0, nullptr, sys.p);
      B->tn1 = tune_tc_stream(c0, s1, nvec, scratch, B->tci1, B->tcb1, B->tcn1);
      B->tn2 = tune_tc_stream(c0, s2, nvec, scratch, B->tci2, B->tcb2, B->tcn2);
      CK(cudaStreamSynchronize(c0->st));
    } else {
      merge_fp64(B->p1, plans, false, c0->st);
      merge_fp64(B->p2, plans, true, c0->st);
    }
    CK(cudaStreamSynchronize(c0->st));
    slot = std::move(B);
  }
  BatchPlan& B = *slot;
  if (precision == LRT_MIXED && !c0->derr) {
    if (dev_alloc((void**)&c0->derr, sizeof(int)) != cudaSuccess) throw Error(LRT_ENOMEM, "error flag");
    CK(cudaMemsetAsync(c0->derr, 0, sizeof(int), c0->st));
  }
  // per-call buffers: re-upload the base tables when they change (invalidates the graph)
  std::vector<const double*> xv(x, x + n);
  std::vector<double*> yv(y, y + n);
  for (int j = 0; j < n; ++j) {
    const double* lo = x[j];
    const double* hi = x[j] + plans[j]->nelem * nvec;
    for (int q = 0; q < n; ++q)
      if ((const double*)y[q] < hi && lo < (const double*)y[q] + plans[q]->nelem * nvec)
        throw Error(LRT_EINVAL, "sigma_batched: an x overlaps a y");
  }
  const bool same = B.ran && xv == B.gx && yv == B.gy;
  if (!same) {
    if (precision == LRT_MIXED) {
      B.hys = yv;
      B.ys.upload(B.hys, c0->st);
    } else {
      B.hbases.resize(n);
      for (int j = 0; j < n; ++j) B.hbases[j] = GemmBases{x[j], y[j], plans[j]->tbuf};
      B.bases.upload(B.hbases, c0->st);
    }
    if (B.exec) {
      cudaGraphExecDestroy(B.exec);
      B.exec = nullptr;
    }
  }
  if (same && !B.exec) {
    // second call with the same buffers: capture the call once, replay it from now on
    cudaGraph_t g = nullptr;
    if (!B.cap) CK(cudaStreamCreateWithFlags(&B.cap, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeThreadLocal));
    batch_issue(c0, B, plans, xv, nvec, B.cap);
    const cudaError_t ce = cudaStreamEndCapture(B.cap, &g);
    if (ce != cudaSuccess || !g) throw Error(LRT_ECUDA, "sigma_batched: graph capture failed");
    const cudaError_t ie = cudaGraphInstantiate(&B.exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      B.exec = nullptr;
      throw Error(LRT_ECUDA, "sigma_batched: graph instantiation failed");
    }
  }
  if (B.exec) {
    CK(cudaGraphLaunch(B.exec, c0->st));
  } else {
    batch_issue(c0, B, plans, xv, nvec, c0->st);
  }
  CK(cudaGetLastError());
  B.gx = xv;
  B.gy = yv;
  B.ran = true;
  if (precision == LRT_MIXED) {
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, c0->derr, sizeof(int), cudaMemcpyDeviceToHost, c0->st));
    CK(cudaStreamSynchronize(c0->st));
    if (flag) {
      CK(cudaMemsetAsync(c0->derr, 0, sizeof(int), c0->st));
      throw Error(LRT_ETIMEOUT, "sigma_batched: a tensor-core pipeline wait expired; results are invalid");
    }
  }
  c0->last.flops = B.flops;
  c0->last.flops_issued = 0.0;
  c0->last.launches = 2;
  c0->last.n_terms = 0;
  c0->last.n_products = 0;
  c0->last.op_bytes = 0.0;
}

}  // namespace lrt

// ===========================================================================
// C ABI
// ===========================================================================
using namespace lrt;

namespace lrt {

int ctx_device(lrt_ctx* ctx) { return ctx ? ctx->dev : -1; }
void ctx_set_error(lrt_ctx* ctx, const std::string& msg) {
  if (ctx) ctx->err = msg;
}

// Launch an existing sigma plan with a caller-chosen workspace; allocates nothing.
int sigma_launch_existing_plan(lrt_ctx* ctx, int site, int nsite, int nvec, const double* x_dev,
                               double* y_dev, double* workspace, int64_t workspace_doubles) {
  if (!ctx) return LRT_EINVAL;
  try {
    if (nsite < 1 || nsite > 2 || site < 0 || nvec <= 0 || !x_dev || !y_dev || !workspace)
      throw Error(LRT_EINVAL, "sigma_noalloc: bad arguments");
    SigmaPlan* p = find_plan(ctx, site, nsite, nvec);
    if (!p)
      throw Error(LRT_ESTATE, "sigma_noalloc: no prepared plan for this (site, nsite, nvec); call sigma() once "
                              "with the same arguments after the last renormalize()");
    if (p->tsize > workspace_doubles)
      throw Error(LRT_EINVAL, "sigma_noalloc: needs " + std::to_string(p->tsize) +
                                  " doubles of scratch, the static maximum is " + std::to_string(workspace_doubles));
    if ((const double*)y_dev < x_dev + p->nelem * nvec && x_dev < (const double*)y_dev + p->nelem * nvec)
      throw Error(LRT_EINVAL, "sigma_noalloc: x and y overlap");
    p->p1.run(ctx->st, x_dev, y_dev, workspace, &p->ex);
    p->p2.run(ctx->st, x_dev, y_dev, workspace, &p->ex);
    CK(cudaGetLastError());
    ctx->err.clear();
    return LRT_OK;
  } catch (const Error& e) {
    ctx->err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    ctx->err = e.what();
    return LRT_EINVAL;
  }
}

}  // namespace lrt

static thread_local std::string g_create_err;

template <class F>
static int guard(lrt_ctx* c, F&& f) {
  if (!c) return LRT_EINVAL;
  try {
    CK(cudaSetDevice(c->dev));
    PoolScope ps(&c->pool);
    f();
    c->err.clear();
    return LRT_OK;
  } catch (const Error& e) {
    c->err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    return LRT_ENOMEM;
  } catch (const std::exception& e) {
    c->err = e.what();
    return LRT_EINVAL;
  }
}

extern "C" {

int lrt_create(lrt_t* out, int device, void* cuda_stream) {
  if (!out) return LRT_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    g_create_err = "no CUDA device " + std::to_string(device);
    return LRT_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    g_create_err = "cudaSetDevice failed";
    return LRT_ECUDA;
  }
  auto* c = new (std::nothrow) lrt_ctx();
  if (!c) return LRT_ENOMEM;
  static std::atomic<uint64_t> next_id{0};
  c->id = ++next_id;
  c->dev = device;
  c->st = (cudaStream_t)cuda_stream;
  *out = c;
  return LRT_OK;
}

int lrt_destroy(lrt_t ctx) {
  if (!ctx) return LRT_EINVAL;
  cudaSetDevice(ctx->dev);
  cudaStreamSynchronize(ctx->st);
  {
    PoolScope ps(&ctx->pool);
    delete ctx;
  }
  return LRT_OK;
}

const char* lrt_last_error(lrt_t ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int op_build(lrt_t ctx, int k, const double* h, const double* eri, int n_factor, const double* B,
             double e_core) {
  return guard(ctx, [&] {
    // no eri and no factor: a one-body operator
    if (k <= 0 || k > 128 || !h || n_factor < 0 || (!eri && n_factor > 0 && !B))
      throw Error(LRT_EINVAL, "op_build: bad arguments");
    if (ctx->have_mps && ctx->k != k) throw Error(LRT_EINVAL, "op_build: k differs from the loaded MPS");
    build_ints(ctx->I, k, h, eri, n_factor, B, e_core);
    ctx->have_ham = true;
    reset_env(ctx);
  });
}

int mps_load(lrt_t ctx, const lrt_mps_desc* m) {
  return guard(ctx, [&] {
    if (!m || m->k <= 0 || !m->bond_nsect || !m->bond_sectors || !m->site_data)
      throw Error(LRT_EINVAL, "mps_load: bad descriptor");
    if (ctx->have_ham && ctx->I.k != m->k) throw Error(LRT_EINVAL, "mps_load: k differs from op_build");
    std::vector<Sectors> bonds(m->k + 1);
    int pos = 0;
    for (int b = 0; b <= m->k; ++b) {
      if (m->bond_nsect[b] <= 0) throw Error(LRT_EINVAL, "mps_load: empty bond " + std::to_string(b));
      for (int s = 0; s < m->bond_nsect[b]; ++s, ++pos) {
        const int* t = m->bond_sectors + 3 * pos;
        if (t[2] <= 0) throw Error(LRT_EINVAL, "mps_load: non-positive sector dimension");
        if (bonds[b].find(t[0], t[1]) >= 0) throw Error(LRT_EINVAL, "mps_load: duplicate sector");
        bonds[b].add(t[0], t[1], t[2]);
      }
    }
    if (bonds[0].n() != 1 || bonds[0].a[0] != 0 || bonds[0].b[0] != 0 || bonds[0].d[0] != 1)
      throw Error(LRT_EINVAL, "mps_load: bond 0 must be the single sector (0,0,1)");
    if (bonds[m->k].n() != 1 || bonds[m->k].a[0] != m->n_alpha || bonds[m->k].b[0] != m->n_beta ||
        bonds[m->k].d[0] != 1)
      throw Error(LRT_EINVAL, "mps_load: bond k must be the single sector (n_alpha,n_beta,1)");
    auto upload = [&](const double* const* data, std::vector<SiteTensor>& out) {
      out.resize(m->k);
      for (int i = 0; i < m->k; ++i) {
        site_layout(out[i], bonds[i], bonds[i + 1]);
        if (out[i].total > 0) {
          if (!data[i]) throw Error(LRT_EINVAL, "mps_load: missing site data");
          if (dev_alloc((void**)&out[i].d, (size_t)out[i].total * sizeof(double)) != cudaSuccess)
            throw Error(LRT_ENOMEM, "mps_load: device allocation");
          CK(cudaMemcpyAsync(out[i].d, data[i], (size_t)out[i].total * sizeof(double),
                             cudaMemcpyHostToDevice, ctx->st));
        }
      }
    };
    std::vector<SiteTensor> sites, sites_r;
    upload(m->site_data, sites);
    if (m->site_data_right) upload(m->site_data_right, sites_r);
    CK(cudaStreamSynchronize(ctx->st));
    ctx->k = m->k;
    ctx->na = m->n_alpha;
    ctx->nb = m->n_beta;
    ctx->bonds = std::move(bonds);
    ctx->sites = std::move(sites);
    ctx->sites_r = std::move(sites_r);
    ctx->have_mps = true;
    reset_env(ctx);
  });
}

int wfn_layout(lrt_t ctx, int site, int nsite, int64_t* nelem, int* nblocks, int64_t* block_offsets) {
  return guard(ctx, [&] {
    if (!ctx->have_mps) throw Error(LRT_ESTATE, "wfn_layout: no MPS loaded");
    if (nsite < 1 || nsite > 2 || site < 0 || site + nsite > ctx->k) throw Error(LRT_EINVAL, "wfn_layout: bad site");
    auto wb = wfn_blocks(ctx, site, nsite);
    int64_t n = 0;
    for (auto& w : wb) n = std::max(n, w.off + (int64_t)w.rows * w.cols);
    if (nelem) *nelem = n;
    if (nblocks) *nblocks = (int)wb.size();
    if (block_offsets)
      for (size_t i = 0; i < wb.size(); ++i) block_offsets[i] = wb[i].off;
  });
}

int renormalize(lrt_t ctx, int site, int dir, int precision) {
  return guard(ctx, [&] {
    if (!ctx->have_mps || !ctx->have_ham) throw Error(LRT_ESTATE, "renormalize: op_build and mps_load first");
    if (site < 0 || site >= ctx->k || (dir != 1 && dir != -1)) throw Error(LRT_EINVAL, "renormalize: bad site/dir");
    if (precision != LRT_FP64 && precision != LRT_MIXED) throw Error(LRT_EINVAL, "renormalize: bad precision");
    if (dir == 1) {
      if (!ctx->L[site]) throw Error(LRT_ESTATE, "renormalize: left block of bond " + std::to_string(site) + " missing");
      renorm_left(ctx, site, precision);
    } else {
      if (!ctx->R[site + 1]) throw Error(LRT_ESTATE, "renormalize: right block of bond " + std::to_string(site + 1) + " missing");
      renorm_right(ctx, site, precision);
    }
  });
}

int sigma(lrt_t ctx, int site, int nsite, int nvec, const double* x_dev, double* y_dev, int precision) {
  return guard(ctx, [&] {
    if (!ctx->have_mps || !ctx->have_ham) throw Error(LRT_ESTATE, "sigma: op_build and mps_load first");
    if (nsite < 1 || nsite > 2 || site < 0 || site + nsite > ctx->k || nvec <= 0 || !x_dev || !y_dev)
      throw Error(LRT_EINVAL, "sigma: bad arguments");
    if (precision != LRT_FP64 && precision != LRT_MIXED) throw Error(LRT_EINVAL, "sigma: bad precision");
    if (!ctx->L[site]) throw Error(LRT_ESTATE, "sigma: left block of bond " + std::to_string(site) + " missing");
    SigmaPlan& p = get_plan(ctx, site, nsite, nvec, precision == LRT_MIXED);
    if ((const double*)y_dev < x_dev + p.nelem * nvec && x_dev < (const double*)y_dev + p.nelem * nvec)
      throw Error(LRT_EINVAL, "sigma: x and y overlap");
    if (precision == LRT_MIXED) {
      run_tc(ctx, p, x_dev, y_dev, nvec);
    } else {
      p.p1.run(ctx->st, x_dev, y_dev, p.tbuf, &p.ex);
      p.p2.run(ctx->st, x_dev, y_dev, p.tbuf, &p.ex);
    }
    CK(cudaGetLastError());
    ctx->last.flops = p.flops_alg;
    ctx->last.flops_issued = p.p1.flops + p.p2.flops;
    ctx->last.launches = p.p1.launches() + p.p2.launches();
    ctx->last.n_terms = p.n_terms;
    ctx->last.n_products = p.n_products;
    ctx->last.op_bytes = p.op_bytes;
  });
}

int sigma_batched(const lrt_t* ctxs, int n_inst, const int* sites, int nsite, int nvec, const double* const* x_dev,
                  double* const* y_dev, int precision) {
  if (!ctxs || n_inst <= 0 || !ctxs[0]) return LRT_EINVAL;
  return guard(ctxs[0], [&] {
    if (!sites || !x_dev || !y_dev || nsite < 1 || nsite > 2 || nvec <= 0)
      throw Error(LRT_EINVAL, "sigma_batched: bad arguments");
    if (precision != LRT_FP64 && precision != LRT_MIXED) throw Error(LRT_EINVAL, "sigma_batched: bad precision");
    sigma_batched_impl(ctxs, n_inst, sites, nsite, nvec, x_dev, y_dev, precision);
  });
}

int heff_diag(lrt_t ctx, int site, int nsite, double* d_dev) {
  return guard(ctx, [&] {
    if (!ctx->have_mps || !ctx->have_ham) throw Error(LRT_ESTATE, "heff_diag: op_build and mps_load first");
    if (nsite < 1 || nsite > 2 || site < 0 || site + nsite > ctx->k || !d_dev) throw Error(LRT_EINVAL, "heff_diag: bad arguments");
    if (!ctx->L[site]) throw Error(LRT_ESTATE, "heff_diag: left block missing");
    SigmaPlan& p = get_plan(ctx, site, nsite, 1);
    launch_diag(p.douts.p, p.dterms.p, p.ndiag, d_dev, ctx->st);
    CK(cudaGetLastError());
  });
}

int sweep_gs(lrt_t ctx, const lrt_gs_params* p, double* e0) {
  return guard(ctx, [&] {
    if (!ctx->have_mps || !ctx->have_ham) throw Error(LRT_ESTATE, "sweep_gs: op_build and mps_load first");
    if (!p || !p->M_schedule || p->n_schedule <= 0 || p->max_sweeps <= 0 || !e0)
      throw Error(LRT_EINVAL, "sweep_gs: bad parameters");
    int nsw = 0;
    *e0 = sweep_gs_impl(ctx, *p, &nsw);
    if (p->onesite_sweeps > 0) *e0 = sweep_onesite_impl(ctx, *p, p->onesite_sweeps);
    ctx->last_sweeps = nsw;
  });
}

int tda_load(lrt_t ctx, const double* const* C0, const double* const* lam) {
  return guard(ctx, [&] {
    if (!ctx->have_mps || !ctx->have_ham) throw Error(LRT_ESTATE, "tda_load: op_build and mps_load first");
    if (ctx->sites_r.empty()) throw Error(LRT_ESTATE, "tda_load: the MPS must be loaded with its right-orthonormal form");
    if (!C0 || !lam) throw Error(LRT_EINVAL, "tda_load: NULL arrays");
    auto st = std::make_unique<TdaState>();
    for (int i = 0; i < ctx->k; ++i) {
      SiteTensor T;
      site_layout(T, ctx->bonds[i], ctx->bonds[i + 1]);
      if (dev_alloc((void**)&T.d, (size_t)std::max<int64_t>(T.total, 1) * sizeof(double)) != cudaSuccess)
        throw Error(LRT_ENOMEM, "tda_load");
      if (!C0[i]) throw Error(LRT_EINVAL, "tda_load: missing C0");
      CK(cudaMemcpyAsync(T.d, C0[i], (size_t)T.total * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
      st->C0.push_back(std::move(T));
    }
    for (int b = 0; b <= ctx->k; ++b) {
      int64_t n = 0;
      for (int q = 0; q < ctx->bonds[b].n(); ++q) n += ctx->bonds[b].d[q];
      if (!lam[b]) throw Error(LRT_EINVAL, "tda_load: missing Lambda");
      st->lam.emplace_back(lam[b], lam[b] + n);
    }
    CK(cudaStreamSynchronize(ctx->st));
    st->loaded = true;
    ctx->tda = std::move(st);
  });
}

int tda_prepare(lrt_t ctx, double* norm) {
  return guard(ctx, [&] {
    if (!ctx->have_mps || !ctx->have_ham) throw Error(LRT_ESTATE, "tda_prepare: op_build and mps_load first");
    if (ctx->k < 1) throw Error(LRT_EINVAL, "tda_prepare: empty MPS");
    tda_prepare_impl(ctx, norm);
  });
}

int tda_stationarity(lrt_t ctx, double* grad2, double* e0) {
  return guard(ctx, [&] {
    if (!ctx->tda || !ctx->tda->loaded) throw Error(LRT_ESTATE, "tda_stationarity: tda_load first");
    if (!grad2) throw Error(LRT_EINVAL, "tda_stationarity: NULL output");
    lrt_tda_params p{};
    p.precision = LRT_FP64;
    p.pinv_cut = 1e-12;
    TdaRunner R(ctx, p);
    *grad2 = R.stationarity();
    if (e0) *e0 = R.E0;
  });
}

int sweep_tda(lrt_t ctx, int nroots, const lrt_tda_params* p, double* omega, double* resid, double* e0) {
  int rc = LRT_OK;
  std::vector<double> th(std::max(nroots, 1), 0.0), rs(std::max(nroots, 1), 0.0);
  double E0 = 0.0;
  const int r = guard(ctx, [&] {
    if (!ctx->tda || !ctx->tda->loaded) throw Error(LRT_ESTATE, "sweep_tda: tda_load first");
    if (!p || nroots <= 0 || !omega || !resid) throw Error(LRT_EINVAL, "sweep_tda: bad arguments");
    TdaRunner R(ctx, *p);
    int its = 0;
    try {
      R.run(nroots, th.data(), rs.data(), &its);
    } catch (const Error& e) {
      if (e.code != LRT_ENOCONV) throw;
      rc = LRT_ENOCONV;
    }
    E0 = R.E0;
    ctx->last_sweeps = its;
  });
  if (r != LRT_OK) return r;
  for (int mu = 0; mu < nroots; ++mu) {
    omega[mu] = th[mu] - E0;
    resid[mu] = rs[mu];
  }
  if (e0) *e0 = E0;
  if (rc != LRT_OK) ctx->err = "sweep_tda: not converged within max_iter (results written)";
  return rc;
}

int sweep_tda_density(lrt_t ctx, int nroots, const lrt_tda_params* p, double* omega, double* resid, double* e0,
                      double* gamma) {
  int rc = LRT_OK;
  std::vector<double> th(std::max(nroots, 1), 0.0), rs(std::max(nroots, 1), 0.0);
  double E0 = 0.0;
  const int r = guard(ctx, [&] {
    if (!ctx->tda || !ctx->tda->loaded) throw Error(LRT_ESTATE, "sweep_tda_density: tda_load first");
    if (!p || nroots <= 0 || !omega || !resid || !gamma) throw Error(LRT_EINVAL, "sweep_tda_density: bad arguments");
    TdaRunner R(ctx, *p);
    int its = 0;
    try {
      R.run(nroots, th.data(), rs.data(), &its, gamma);
    } catch (const Error& e) {
      if (e.code != LRT_ENOCONV) throw;
      rc = LRT_ENOCONV;
    }
    E0 = R.E0;
    ctx->last_sweeps = its;
  });
  if (r != LRT_OK) return r;
  for (int mu = 0; mu < nroots; ++mu) {
    omega[mu] = th[mu] - E0;
    resid[mu] = rs[mu];
  }
  if (e0) *e0 = E0;
  if (rc != LRT_OK) ctx->err = "sweep_tda_density: not converged within max_iter (results written)";
  return rc;
}

int sweep_response(lrt_t ctx, lrt_t vctx, double omega, const lrt_resp_params* p, double* alpha, double* resid,
                   int* sweeps) {
  return guard(ctx, [&] {
    if (!p || !alpha || !resid || !sweeps || !vctx || vctx == ctx || !(omega >= 0.0))
      throw Error(LRT_EINVAL, "sweep_response: bad arguments");
    if (!ctx->tda || !ctx->tda->loaded) throw Error(LRT_ESTATE, "sweep_response: tda_load or tda_prepare first");
    if (!vctx->tda || !vctx->tda->loaded || !vctx->have_ham)
      throw Error(LRT_ESTATE, "sweep_response: the perturbation's context needs op_build and tda_prepare");
    if (vctx->dev != ctx->dev || vctx->k != ctx->k) throw Error(LRT_EINVAL, "sweep_response: contexts differ in device or k");
    const int k = ctx->k;
    lrt_tda_params tp{};
    tp.precision = LRT_FP64;
    tp.pinv_cut = p->pinv_cut > 0.0 ? p->pinv_cut : 1e-12;
    TdaRunner R(ctx, tp);
    R.setup();
    // V_i C0 at every site from the perturbation's environment, on the same reference
    std::vector<DevBuf> vc0(k);
    for (int i = 0; i < k; ++i) vc0[i].ensure((size_t)std::max<int64_t>(R.T(i), 1));
    CK(cudaStreamSynchronize(ctx->st));
    {
      PoolScope ps(&vctx->pool);
      TdaRunner V(vctx, tp);
      V.setup();
      for (int i = 0; i < k; ++i) {
        if (V.T(i) != R.T(i)) throw Error(LRT_EINVAL, "sweep_response: the two contexts hold different MPS layouts");
        if (R.T(i) == 0) continue;
        // the same reference in both: C0_i bit for bit (tda_prepare is deterministic)
        DevBuf dif;
        dif.ensure((size_t)R.T(i));
        CK(cudaMemcpyAsync(dif.p, R.C0(i).d, (size_t)R.T(i) * sizeof(double), cudaMemcpyDeviceToDevice, vctx->st));
        V.axpbyd(-1.0, V.C0(i).d, 1.0, dif.p, R.T(i));
        if (V.dotd(dif.p, dif.p, R.T(i)) != 0.0)
          throw Error(LRT_EINVAL, "sweep_response: the two contexts hold different references");
        V.run_plan(*V.h0one[i], R.C0(i).d, vc0[i].p, 1, false);
      }
      CK(cudaStreamSynchronize(vctx->st));
    }
    const int ms = p->max_sweeps > 0 ? p->max_sweeps : 40;
    const double tol = p->tol > 0.0 ? p->tol : 1e-16;
    const int mr = p->minres_max > 0 ? p->minres_max : 200;
    const double mrt = p->minres_tol > 0.0 ? p->minres_tol : 1e-12;
    // X: (H - (E0 + omega)) X = -v, Y: (H - (E0 - omega)) Y = -v; alpha = v.(X + Y)
    double r2x = 0.0, r2y = 0.0;
    int swx = 0, swy = 0;
    if (p->method != LRT_RESP_SITE && p->method != LRT_RESP_SUBSPACE)
      throw Error(LRT_EINVAL, "sweep_response: unknown method");
    double ax, ay;
    if (p->method == LRT_RESP_SUBSPACE) {
      ax = R.response_krylov(vc0, R.E0 + omega, ms, tol, p->max_space, r2x, swx);
      ay = R.response_krylov(vc0, R.E0 - omega, ms, tol, p->max_space, r2y, swy);
    } else {
      ax = R.response_component(vc0, R.E0 + omega, ms, tol, mr, mrt, r2x, swx);
      ay = R.response_component(vc0, R.E0 - omega, ms, tol, mr, mrt, r2y, swy);
    }
    *alpha = ax + ay;
    resid[0] = r2x;
    resid[1] = r2y;
    sweeps[0] = swx;
    sweeps[1] = swy;
    ctx->last_sweeps = swx + swy;
  });
}

int lrt_set_wait_limit(lrt_t ctx, double seconds, int stall_next) {
  return guard(ctx, [&] {
    if (!(seconds >= 0.0) || seconds > 60.0) throw Error(LRT_EINVAL, "lrt_set_wait_limit: seconds in [0, 60]");
    ctx->tc_wait_ns = (uint64_t)(seconds * 1e9);
    ctx->tc_stall = stall_next ? 1 : 0;
  });
}

int lrt_sweep_log(lrt_t ctx, int cap, double* seconds, int* mixed, int* n) {
  return guard(ctx, [&] {
    if (!n || cap < 0 || (cap > 0 && (!seconds || !mixed))) throw Error(LRT_EINVAL, "lrt_sweep_log: bad arguments");
    const int m = (int)ctx->sweep_log.size();
    for (int j = 0; j < std::min(cap, m); ++j) {
      seconds[j] = ctx->sweep_log[j].first;
      mixed[j] = ctx->sweep_log[j].second;
    }
    *n = m;
  });
}

int lrt_sweeps(lrt_t ctx, int* sweeps) {
  return guard(ctx, [&] {
    if (!sweeps) throw Error(LRT_EINVAL, "lrt_sweeps: NULL output");
    *sweeps = ctx->last_sweeps;
  });
}

int sweep_tda_batched(const lrt_t* ctxs, int n_inst, int nroots, const lrt_tda_params* p, double* omega,
                      double* resid, double* e0) {
  if (!ctxs || n_inst <= 0 || nroots <= 0 || !p || !omega || !resid) return LRT_EINVAL;
  for (int j = 0; j < n_inst; ++j) {
    if (!ctxs[j]) return LRT_EINVAL;
    for (int q = 0; q < j; ++q)
      if (ctxs[q] == ctxs[j]) {
        ctxs[j]->err = "sweep_tda_batched: an instance appears twice";
        return LRT_EINVAL;
      }
  }
  // lazily initialized device queries, before the threads start
  lrt::gemm_fp64_slots();
  lrt::tc_num_ctas(1);
  std::vector<int> rc(n_inst, LRT_OK);
  std::atomic<int> next{0};
  auto work = [&] {
    for (int j = next++; j < n_inst; j = next++)
      rc[j] = sweep_tda(ctxs[j], nroots, p, omega + (size_t)j * nroots, resid + (size_t)j * nroots,
                        e0 ? e0 + j : nullptr);
  };
  const int nt = std::max(1, std::min(n_inst, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> threads;
  for (int t = 1; t < nt; ++t) threads.emplace_back(work);
  work();
  for (auto& t : threads) t.join();
  int out = LRT_OK;
  for (int j = 0; j < n_inst; ++j) {
    if (rc[j] != LRT_OK && rc[j] != LRT_ENOCONV) return rc[j];
    if (rc[j] == LRT_ENOCONV) out = LRT_ENOCONV;
  }
  return out;
}

int mps_save(lrt_t ctx, lrt_mps_out* out) {
  return guard(ctx, [&] {
    if (!out) throw Error(LRT_EINVAL, "mps_save: NULL descriptor");
    if (!ctx->have_mps) throw Error(LRT_ESTATE, "mps_save: no MPS");
    out->k = ctx->k;
    out->n_alpha = ctx->na;
    out->n_beta = ctx->nb;
    out->has_right = ctx->sites_r.empty() ? 0 : 1;
    int tot = 0;
    for (int b = 0; b <= ctx->k; ++b) {
      if (out->bond_nsect) out->bond_nsect[b] = ctx->bonds[b].n();
      for (int q = 0; q < ctx->bonds[b].n(); ++q, ++tot)
        if (out->bond_sectors) {
          out->bond_sectors[3 * tot] = ctx->bonds[b].a[q];
          out->bond_sectors[3 * tot + 1] = ctx->bonds[b].b[q];
          out->bond_sectors[3 * tot + 2] = ctx->bonds[b].d[q];
        }
    }
    out->total_sectors = tot;
    for (int i = 0; i < ctx->k; ++i) {
      const SiteTensor& T = ctx->sites[i];
      if (out->site_nelem) out->site_nelem[i] = T.total;
      if (out->site_data && out->site_data[i] && T.total > 0)
        CK(cudaMemcpyAsync(out->site_data[i], T.d, (size_t)T.total * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->st));
      if (out->site_data_right && out->site_data_right[i] && !ctx->sites_r.empty() && ctx->sites_r[i].total > 0)
        CK(cudaMemcpyAsync(out->site_data_right[i], ctx->sites_r[i].d, (size_t)ctx->sites_r[i].total * sizeof(double),
                           cudaMemcpyDeviceToHost, ctx->st));
    }
    CK(cudaStreamSynchronize(ctx->st));
  });
}

int mps_get_bonds(lrt_t ctx, int* bond_nsect, int* bond_sectors, int* total_sectors) {
  return guard(ctx, [&] {
    if (!ctx->have_mps) throw Error(LRT_ESTATE, "mps_get_bonds: no MPS");
    int tot = 0;
    for (int b = 0; b <= ctx->k; ++b) {
      if (bond_nsect) bond_nsect[b] = ctx->bonds[b].n();
      for (int s = 0; s < ctx->bonds[b].n(); ++s, ++tot)
        if (bond_sectors) {
          bond_sectors[3 * tot] = ctx->bonds[b].a[s];
          bond_sectors[3 * tot + 1] = ctx->bonds[b].b[s];
          bond_sectors[3 * tot + 2] = ctx->bonds[b].d[s];
        }
    }
    if (total_sectors) *total_sectors = tot;
  });
}

int mps_get_site(lrt_t ctx, int site, double* host_out, int64_t* nelem) {
  return guard(ctx, [&] {
    if (!ctx->have_mps) throw Error(LRT_ESTATE, "mps_get_site: no MPS");
    if (site < 0 || site >= ctx->k) throw Error(LRT_EINVAL, "mps_get_site: bad site");
    const SiteTensor& T = ctx->sites[site];
    if (nelem) *nelem = T.total;
    if (host_out && T.total > 0) {
      CK(cudaMemcpyAsync(host_out, T.d, (size_t)T.total * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
    }
  });
}

int sigma_stats(lrt_t ctx, lrt_sigma_stats* out) {
  return guard(ctx, [&] {
    if (!out) throw Error(LRT_EINVAL, "sigma_stats: NULL");
    *out = ctx->last;
  });
}

}  // extern "C"
