"""Renormalized operator sets, blocking, renormalization and sigma (plain FP64).

This is the "x" of the paper (Sec. "Sweep algorithm for the projected
Hamiltonian", Eqs. hzero_sb, hleft_sb, lopr1st, ropr1st): the summation over
normal and complementary renormalized operators, written out.

Notation (spin orbitals, real integrals, t_pq and v_pqrs = <pq|rs>):
  H = sum t_pq a+_p a_q + 1/2 sum v_pqrs a+_p a+_q a_s a_r.
For a bipartition X | Y (X before Y in Jordan-Wigner order), with operators
written X-part first, every term of H falls into exactly one of

  H = H^X + H^Y
    + sum_{x in X} ( C_x S^Y_x - c_x S^Y_x^T )  + sum_{y in Y} ( S^X_y^T c_y - S^X_y C_y )
    + [X normal] sum_{p<q in X} ( A_pq P^Y_pq + A_pq^T P^Y_pq^T ) + sum_{p,q in X} B_pq Q^Y_pq
    | [Y normal] sum_{r<s in Y} ( P^X_rs^T A_rs^T + P^X_rs A_rs ) + sum_{u,w in Y} Q^X_uw B_uw

with C_p = a+_p, c_p = a_p and, for a block Z and indices outside it,
  S^Z_x  = 1/2 sum_{q in Z} t_xq c_q + sum_{q,r,s in Z} v_xqrs C_q c_s c_r
  A_pq   = C_p C_q,                 B_pq = C_p c_q
  P^Z_pq = sum_{r,s in Z} v_pqrs c_s c_r
  Q^Z_pq = sum_{r,s in Z} (v_prqs - v_prsq) C_r c_s.
The derivation moves fermion operators into X-first order; each exchange of
two odd operators on different modes gives a factor -1.  The test suite
assembles this sum on small Fock spaces and checks it against the directly
built H.

A product X_op Y_op acts on |x>|y> as (-1)^{parity(Y_op) N(x)} X_op|x> Y_op|y>,
where N(x) is the electron count of the ket state of X.

Blocks store H, C_p (p in block), S_x (x outside) and, by mode, the normal
pairs A_pq (p<q), B_pq (p<=q) ("N") or the complementary pairs P_pq (p<q),
Q_pq (p<=q) for p,q outside ("C").  The normal side of a cut is the one with
fewer orbitals (the left side at cut b when 2b <= k).
"""
from __future__ import annotations

import itertools

import numpy as np

from synth import QN_SITE

# ----------------------------------------------------------------------------
# block-sparse operator helpers: an operator is a dict {(bra_label, ket_label): ndarray}
# ----------------------------------------------------------------------------


def op_T(op):
    if op is None:
        return None
    return {(k, b): m.T for (b, k), m in op.items()}


def op_scale(op, c):
    if op is None or c == 0.0:
        return None
    return {kk: c * m for kk, m in op.items()}


def op_axpy(acc, op, c=1.0):
    """acc += c * op (acc may be None); returns acc."""
    if op is None or c == 0.0:
        return acc
    if acc is None:
        acc = {}
    for kk, m in op.items():
        if kk in acc:
            acc[kk] = acc[kk] + c * m
        else:
            acc[kk] = c * m
    return acc


ODD_KINDS = {"C", "c", "S", "St"}


def parity(spec) -> int:
    return 1 if spec[0] in ODD_KINDS else 0


def qn_add(a, b):
    return (a[0] + b[0], a[1] + b[1])


class Block:
    """A block of spin orbitals with a (renormalized) basis and its operator set.

    labels: dict label -> dimension; `nel(label)` gives the electron number of
    the states of that label (used for the fermionic sign).  `transition`
    marks a first-order set <0|O|1>, whose identity is zero (Eq. left-orthoSeb).
    """

    def __init__(self, orbs, mode, labels, nel, ops, v, transition=False, rev=None):
        self.orbs = list(orbs)
        self.orbset = set(orbs)
        self.mode = mode
        self.labels = dict(labels)
        self.nel = nel
        self.ops = ops
        self.v = v
        self.transition = transition
        # A transition set <0|O|1> is not closed under transposition:
        # (<0|O|1>)^T = <1|O^dag|0>.  `rev` holds the reverse set <1|O|0>, so
        # that the adjoint in the forward direction is <0|O^dag|1> = (<1|O|0>)^T.
        self.rev = self if rev is None else rev
        self._cache = {}

    # ---- getters -----------------------------------------------------------
    def get(self, spec):
        """Operator for spec = (kind, *indices); None stands for zero."""
        if spec in self._cache:
            return self._cache[spec]
        r = self._get(spec)
        self._cache[spec] = r
        return r

    def _get(self, spec):
        kind = spec[0]
        if kind == "I":
            # the renormalized identity <l'|l> (a Gram matrix unless the basis
            # is orthonormal; zero for a first-order set, Eq. left-orthoSeb)
            if ("I",) in self.ops:
                return self.ops[("I",)]
            if self.transition:
                return None
            return {(q, q): np.eye(d) for q, d in self.labels.items()}
        if kind == "H":
            return self.ops.get(("H",))
        if kind == "C":
            return self.ops.get(("C", spec[1]))
        if kind == "c":
            return op_T(self.rev.get(("C", spec[1])))
        if kind == "S":
            return self.ops.get(("S", spec[1]))
        if kind == "St":
            return op_T(self.rev.get(("S", spec[1])))
        if kind in ("A", "P"):
            p, q = spec[1], spec[2]
            if p == q:
                return None
            if p > q:
                return op_scale(self.get((kind, q, p)), -1.0)
            if kind == "P" and self.mode == "N":
                return self._p_from_normal(p, q)
            return self.ops.get((kind, p, q))
        if kind in ("B", "Q"):
            p, q = spec[1], spec[2]
            if p > q:
                return op_T(self.rev.get((kind, q, p)))
            if kind == "Q" and self.mode == "N":
                return self._q_from_normal(p, q)
            return self.ops.get((kind, p, q))
        if kind in ("At", "Pt", "Bt", "Qt"):
            return op_T(self.rev.get((kind[0],) + tuple(spec[1:])))
        raise KeyError(spec)

    def _p_from_normal(self, p, q):
        # P_pq = sum_{r<s in Z} (v_pqrs - v_pqsr) A_rs^T   (since c_s c_r = A_rs^T)
        acc = None
        for r, s in itertools.combinations(self.orbs, 2):
            c = self.v[p, q, r, s] - self.v[p, q, s, r]
            if c != 0.0:
                acc = op_axpy(acc, self.get(("At", r, s)), c)
        return acc

    def _q_from_normal(self, p, q):
        # Q_pq = sum_{r,s in Z} (v_prqs - v_prsq) B_rs
        acc = None
        for r in self.orbs:
            for s in self.orbs:
                c = self.v[p, r, q, s] - self.v[p, r, s, q]
                if c != 0.0:
                    acc = op_axpy(acc, self.get(("B", r, s)), c)
        return acc


def kron_term(X: Block, Y: Block, xspec, yspec, coef, acc):
    """acc += coef * (X_op (x) Y_op) on the product basis, with the fermionic sign."""
    xo = X.get(xspec)
    if xo is None:
        return acc
    yo = Y.get(yspec)
    if yo is None:
        return acc
    py = parity(yspec)
    if acc is None:
        acc = {}
    for (xb, xk), mx in xo.items():
        sgn = -1.0 if (py and X.nel(xk) % 2) else 1.0
        for (yb, yk), my in yo.items():
            key = ((xb, yb), (xk, yk))
            val = (coef * sgn) * np.kron(mx, my)
            if key in acc:
                acc[key] = acc[key] + val
            else:
                acc[key] = val
    return acc


# ----------------------------------------------------------------------------
# the decomposition of H across a cut, and the blocking formulas
# ----------------------------------------------------------------------------
def cross_terms(X: Block, Y: Block, normal: str):
    """Terms of H that act on both X and Y, as (coef, X spec, Y spec)."""
    T = []
    for x in X.orbs:
        T += [(1.0, ("C", x), ("S", x)), (-1.0, ("c", x), ("St", x))]
    for y in Y.orbs:
        T += [(1.0, ("St", y), ("c", y)), (-1.0, ("S", y), ("C", y))]
    if normal == "X":
        for p, q in itertools.combinations(X.orbs, 2):
            T += [(1.0, ("A", p, q), ("P", p, q)), (1.0, ("At", p, q), ("Pt", p, q))]
        for p in X.orbs:
            T += [(1.0, ("B", p, p), ("Q", p, p))]
        for p, q in itertools.combinations(X.orbs, 2):
            T += [(1.0, ("B", p, q), ("Q", p, q)), (1.0, ("Bt", p, q), ("Qt", p, q))]
    else:
        for r, s in itertools.combinations(Y.orbs, 2):
            T += [(1.0, ("Pt", r, s), ("At", r, s)), (1.0, ("P", r, s), ("A", r, s))]
        for u in Y.orbs:
            T += [(1.0, ("Q", u, u), ("B", u, u))]
        for u, w in itertools.combinations(Y.orbs, 2):
            T += [(1.0, ("Q", u, w), ("B", u, w)), (1.0, ("Qt", u, w), ("Bt", u, w))]
    return T


def hamiltonian_terms(X: Block, Y: Block, normal: str, e_core: float = 0.0):
    T = [(1.0, ("H",), ("I",)), (1.0, ("I",), ("H",))] + cross_terms(X, Y, normal)
    if e_core != 0.0:
        T.append((e_core, ("I",), ("I",)))
    return T


def blocking_terms(X: Block, Y: Block, mode: str, outside, v):
    """Operator set of the union X (+) Y as sums of products of X and Y operators."""
    orbs = X.orbs + Y.orbs
    normal_xy = "Y" if len(Y.orbs) <= len(X.orbs) else "X"
    terms = {("H",): hamiltonian_terms(X, Y, normal_xy), ("I",): [(1.0, ("I",), ("I",))]}
    for p in X.orbs:
        terms[("C", p)] = [(1.0, ("C", p), ("I",))]
    for p in Y.orbs:
        terms[("C", p)] = [(1.0, ("I",), ("C", p))]
    for z in outside:
        L = [(1.0, ("S", z), ("I",)), (1.0, ("I",), ("S", z))]
        L += [(1.0, ("C", q), ("P", z, q)) for q in X.orbs]
        L += [(1.0, ("P", z, q), ("C", q)) for q in Y.orbs]
        L += [(1.0, ("Q", z, w), ("c", w)) for w in Y.orbs]
        L += [(1.0, ("c", u), ("Q", z, u)) for u in X.orbs]
        terms[("S", z)] = L
    if mode == "N":
        for p, q in itertools.combinations(orbs, 2):
            if p in X.orbset and q in X.orbset:
                terms[("A", p, q)] = [(1.0, ("A", p, q), ("I",))]
            elif p in Y.orbset and q in Y.orbset:
                terms[("A", p, q)] = [(1.0, ("I",), ("A", p, q))]
            else:
                terms[("A", p, q)] = [(1.0, ("C", p), ("C", q))]
        for p in orbs:
            for q in orbs:
                if p > q:
                    continue
                if p in X.orbset and q in X.orbset:
                    terms[("B", p, q)] = [(1.0, ("B", p, q), ("I",))]
                elif p in Y.orbset and q in Y.orbset:
                    terms[("B", p, q)] = [(1.0, ("I",), ("B", p, q))]
                else:
                    terms[("B", p, q)] = [(1.0, ("C", p), ("c", q))]
    else:
        for p, q in itertools.combinations(outside, 2):
            L = [(1.0, ("P", p, q), ("I",)), (1.0, ("I",), ("P", p, q))]
            for x in X.orbs:
                for y in Y.orbs:
                    c = v[p, q, y, x] - v[p, q, x, y]
                    if c != 0.0:
                        L.append((c, ("c", x), ("c", y)))
            terms[("P", p, q)] = L
        for p in outside:
            for q in outside:
                if p > q:
                    continue
                L = [(1.0, ("Q", p, q), ("I",)), (1.0, ("I",), ("Q", p, q))]
                for x in X.orbs:
                    for y in Y.orbs:
                        c1 = v[p, x, q, y] - v[p, x, y, q]
                        if c1 != 0.0:
                            L.append((c1, ("C", x), ("c", y)))
                        c2 = -(v[p, y, q, x] - v[p, y, x, q])
                        if c2 != 0.0:
                            L.append((c2, ("c", x), ("C", y)))
                terms[("Q", p, q)] = L
    return terms


def enlarge(X: Block, Y: Block, mode: str, n_so: int, v, transition_side: str | None = None):
    """The block X (+) Y in the product basis, with its full operator set.

    `transition_side` = "X" or "Y" marks that side as a first-order
    (transition) operator set; the result is then the first-order set of the
    union (Eq. lopr1st / ropr1st, first bracket), with its reverse set built
    from the reverse set of that side.
    """
    if transition_side is not None:
        fwd = _enlarge_one(X, Y, mode, n_so, v, True)
        if transition_side == "X":
            rev = _enlarge_one(X.rev, Y, mode, n_so, v, True)
        else:
            rev = _enlarge_one(X, Y.rev, mode, n_so, v, True)
        fwd.rev, rev.rev = rev, fwd
        return fwd
    return _enlarge_one(X, Y, mode, n_so, v, False)


def _enlarge_one(X: Block, Y: Block, mode: str, n_so: int, v, transition: bool):
    orbs = X.orbs + Y.orbs
    outside = [p for p in range(n_so) if p not in set(orbs)]
    terms = blocking_terms(X, Y, mode, outside, v)
    ops = {}
    for key, L in terms.items():
        acc = None
        for coef, xs, ys in L:
            acc = kron_term(X, Y, xs, ys, coef, acc)
        if acc is not None:
            ops[key] = acc
    labels = {}
    for xl, dx in X.labels.items():
        for yl, dy in Y.labels.items():
            labels[(xl, yl)] = dx * dy
    nel = lambda lab, X=X, Y=Y: X.nel(lab[0]) + Y.nel(lab[1])
    return Block(orbs, mode, labels, nel, ops, v, transition=transition)


# ----------------------------------------------------------------------------
# elementary blocks
# ----------------------------------------------------------------------------
def _nel(q):
    return q[0] + q[1]


def vacuum_block(mode: str, v) -> Block:
    return Block([], mode, {(0, 0): 1}, _nel, {("H",): {((0, 0), (0, 0)): np.zeros((1, 1))}}, v)


def site_block(i: int, n_so: int, t, v) -> Block:
    """Exact operator set of spatial site i (spin orbitals 2i, 2i+1), normal mode.

    The site basis is |0>, |a>, |b>, |ab> = C_2i C_2i+1 |vac>, one state per label.
    """
    pa, pb = 2 * i, 2 * i + 1
    # local annihilators on the 4-state basis (index n)
    ca = np.zeros((4, 4))
    cb = np.zeros((4, 4))
    ca[0, 1] = 1.0            # a_a |a> = |0>
    ca[2, 3] = 1.0            # a_a a+_a a+_b |0> = a+_b |0>
    cb[0, 2] = 1.0            # a_b |b> = |0>
    cb[1, 3] = -1.0           # a_b a+_a a+_b |0> = -a+_a |0>
    ann = {pa: ca, pb: cb}
    cre = {p: m.T for p, m in ann.items()}
    loc = [pa, pb]

    def to_op(m):
        out = {}
        for b in range(4):
            for kk in range(4):
                if m[b, kk] != 0.0:
                    out[(QN_SITE[b], QN_SITE[kk])] = np.array([[m[b, kk]]])
        return out if out else None

    ops = {}
    Hm = np.zeros((4, 4))
    for p in loc:
        for q in loc:
            Hm += t[p, q] * cre[p] @ ann[q]
    for p, q, r, s in itertools.product(loc, repeat=4):
        Hm += 0.5 * v[p, q, r, s] * cre[p] @ cre[q] @ ann[s] @ ann[r]
    ops[("H",)] = to_op(Hm) or {((0, 0), (0, 0)): np.zeros((1, 1))}
    for p in loc:
        ops[("C", p)] = to_op(cre[p])
    for z in range(n_so):
        if z in loc:
            continue
        Sm = np.zeros((4, 4))
        for q in loc:
            Sm += 0.5 * t[z, q] * ann[q]
        for q, r, s in itertools.product(loc, repeat=3):
            Sm += v[z, q, r, s] * cre[q] @ ann[s] @ ann[r]
        o = to_op(Sm)
        if o is not None:
            ops[("S", z)] = o
    ops[("A", pa, pb)] = to_op(cre[pa] @ cre[pb])
    for p in loc:
        for q in loc:
            if p <= q:
                ops[("B", p, q)] = to_op(cre[p] @ ann[q])
    ops = {kk: m for kk, m in ops.items() if m is not None}
    labels = {q: 1 for q in QN_SITE}
    return Block(loc, "N", labels, _nel, ops, v)


# ----------------------------------------------------------------------------
# renormalization (Eqs. gauge-shift, lopr1st, ropr1st)
# ----------------------------------------------------------------------------
def _renorm_op(op, bra_iso, ket_iso):
    """out[(qb, qk)] = sum bra_iso[xb]^T op[(xb, xk)] ket_iso[xk] over product labels.

    iso: dict product_label -> list of (new_label, matrix D_product x D_new).
    """
    out = {}
    for (xb, xk), m in op.items():
        if xb not in bra_iso or xk not in ket_iso:
            continue
        for (qb, Ub) in bra_iso[xb]:
            for (qk, Uk) in ket_iso[xk]:
                val = Ub.T @ m @ Uk
                kk = (qb, qk)
                out[kk] = out[kk] + val if kk in out else val
    return out


def left_iso(site_blocks):
    """Left isometry from a site tensor {(q_l, n, q_r): D_l x D_r}: product label (q_l, s) -> [(q_r, M)]."""
    iso = {}
    for (ql, n, qr), m in site_blocks.items():
        iso.setdefault((ql, QN_SITE[n]), []).append((qr, m))
    return iso


def right_iso(site_blocks, n_alpha, n_beta):
    """Right isometry: product label (s, own(q_r)) -> [(own(q_l), M^T)] with own(q) = N - q."""
    iso = {}
    for (ql, n, qr), m in site_blocks.items():
        own_r = (n_alpha - qr[0], n_beta - qr[1])
        own_l = (n_alpha - ql[0], n_beta - ql[1])
        iso.setdefault((QN_SITE[n], own_r), []).append((own_l, m.T))
    return iso


def renormalize(Xe: Block, bra_iso, ket_iso, new_labels, transition=False, acc=None) -> Block:
    """New block <bra|O|ket> for every operator of the enlarged block Xe.

    With bra = ket this is O' = L^T [O (x) h] L; with `acc` the result is added
    to an existing first-order set (the two terms of Eq. lopr1st / ropr1st).
    """
    ops = {} if acc is None else dict(acc.ops)
    for key, op in Xe.ops.items():
        r = _renorm_op(op, bra_iso, ket_iso)
        if not r:
            continue
        if key in ops:
            ops[key] = op_axpy(dict(ops[key]), r)
        else:
            ops[key] = r
    return Block(Xe.orbs, Xe.mode, new_labels, _nel, ops, Xe.v, transition=transition)


# ----------------------------------------------------------------------------
# environment of an MPS
# ----------------------------------------------------------------------------
def left_mode(b, k):
    """Mode of the left block at cut b: normal when it holds no more orbitals than the right."""
    return "N" if 2 * b <= k else "C"


def right_mode(b, k):
    return "C" if 2 * b <= k else "N"


class Environment:
    """Left blocks L[b] (sites 0..b-1) and right blocks R[b] (sites b..k-1) of an MPS.

    site_blocks[i]: dict (q_l, n, q_r) -> array of site i; left blocks are
    built with the site tensors as left isometries, right blocks with them as
    right isometries (the caller passes left- or right-canonical tensors, or
    any tensors for a non-orthogonal projection).
    """

    def __init__(self, ham, t, v):
        self.k = ham.k
        self.na = ham.n_alpha
        self.nb = ham.n_beta
        self.n_so = 2 * ham.k
        self.t = t
        self.v = v
        self.e_core = ham.e_core
        self.sites = [site_block(i, self.n_so, t, v) for i in range(self.k)]
        self.L = {0: vacuum_block(left_mode(0, self.k), v)}
        self.R = {self.k: vacuum_block(right_mode(self.k, self.k), v)}

    def left_enlarged(self, b):
        """L[b] (+) site b: the left block of cut b+1 before renormalization."""
        return enlarge(self.L[b], self.sites[b], left_mode(b + 1, self.k), self.n_so, self.v)

    def right_enlarged(self, b):
        """site b (+) R[b+1]: the right block of cut b before renormalization."""
        return enlarge(self.sites[b], self.R[b + 1], right_mode(b, self.k), self.n_so, self.v)

    def grow_left(self, b, site_blocks, Xe=None):
        """L[b+1] = renormalized (L[b] (+) site b)."""
        Xe = self.left_enlarged(b) if Xe is None else Xe
        iso = left_iso(site_blocks)
        new = {}
        for (ql, n, qr), m in site_blocks.items():
            new[qr] = m.shape[1]
        self.L[b + 1] = renormalize(Xe, iso, iso, new)
        return self.L[b + 1]

    def grow_right(self, b, site_blocks, Ye=None):
        """R[b] = renormalized (site b (+) R[b+1])."""
        Ye = self.right_enlarged(b) if Ye is None else Ye
        iso = right_iso(site_blocks, self.na, self.nb)
        new = {}
        for (ql, n, qr), m in site_blocks.items():
            new[(self.na - ql[0], self.nb - ql[1])] = m.shape[0]
        self.R[b] = renormalize(Ye, iso, iso, new)
        return self.R[b]


# ----------------------------------------------------------------------------
# sigma = H_eff x (Eq. dmrg) and its diagonal (Eq. error)
# ----------------------------------------------------------------------------
FLOP_COUNTER = [0.0]    # 2mnk of every block product done by apply_terms


def apply_terms(X: Block, Y: Block, terms, psi):
    """y = sum_t coef_t (X_t (x) Y_t) psi, psi: dict (x_label, y_label) -> matrix.

    In matrix form each term is Y[x', y'] += sign * X_t[x', x] @ psi[x, y] @ Y_t[y', y]^T.
    FLOP_COUNTER accumulates the multiply-add count of the block products.
    """
    out = {kk: np.zeros_like(m) for kk, m in psi.items()}
    by_x = {}
    for (xl, yl), m in psi.items():
        by_x.setdefault(xl, []).append((yl, m))
    for coef, xs, ys in terms:
        xo = X.get(xs)
        if xo is None:
            continue
        yo = Y.get(ys)
        if yo is None:
            continue
        py = parity(ys)
        ymap = {}
        for (yb, yk), my in yo.items():
            ymap.setdefault(yk, []).append((yb, my))
        for (xb, xk), mx in xo.items():
            if xk not in by_x:
                continue
            sgn = -1.0 if (py and X.nel(xk) % 2) else 1.0
            for yl, m in by_x[xk]:
                if yl not in ymap:
                    continue
                t1 = mx @ m
                FLOP_COUNTER[0] += 2.0 * mx.shape[0] * mx.shape[1] * m.shape[1]
                for yb, my in ymap[yl]:
                    key = (xb, yb)
                    if key not in out:
                        continue          # outside the target sector: zero by symmetry
                    out[key] = out[key] + (coef * sgn) * (t1 @ my.T)
                    FLOP_COUNTER[0] += 2.0 * t1.shape[0] * t1.shape[1] * my.shape[0]
    return out


def diagonal_terms(X: Block, Y: Block, terms, psi_shape):
    """Diagonal of sum_t coef_t X_t (x) Y_t on the blocks of psi_shape."""
    out = {kk: np.zeros(s) for kk, s in psi_shape.items()}
    for coef, xs, ys in terms:
        xo = X.get(xs)
        if xo is None:
            continue
        yo = Y.get(ys)
        if yo is None:
            continue
        py = parity(ys)
        for (xl, yl) in psi_shape:
            if (xl, xl) in xo and (yl, yl) in yo:
                sgn = -1.0 if (py and X.nel(xl) % 2) else 1.0
                out[(xl, yl)] += (coef * sgn) * np.outer(np.diag(xo[(xl, xl)]), np.diag(yo[(yl, yl)]))
    return out


def onesite_to_psi(wfn, na, nb):
    """One-site blocks (q_l, n, q_r) -> {((q_l, s), own(q_r)): D_l x D_r}."""
    return {((ql, QN_SITE[n]), (na - qr[0], nb - qr[1])): m for (ql, n, qr), m in wfn.items()}


def psi_to_onesite(psi, na, nb):
    return {(xl[0], QN_SITE.index(xl[1]), (na - yl[0], nb - yl[1])): m for (xl, yl), m in psi.items()}


def twosite_to_psi(wfn, na, nb):
    """Two-site blocks (q_l, n1, n2, q_r) -> {((q_l, s1), (s2, own(q_r))): D_l x D_r}."""
    return {((ql, QN_SITE[n1]), (QN_SITE[n2], (na - qr[0], nb - qr[1]))): m
            for (ql, n1, n2, qr), m in wfn.items()}


def psi_to_twosite(psi, na, nb):
    return {(xl[0], QN_SITE.index(xl[1]), QN_SITE.index(yl[0]), (na - yl[1][0], nb - yl[1][1])): m
            for (xl, yl), m in psi.items()}


def sigma_onesite(env: Environment, i: int, wfn, Xe=None, Ye=None, form: str = "left"):
    """H_eff x for a one-site tensor at site i (Eq. dmrg, H_i C_i).

    form "left": X = L[i] (+) site i, Y = R[i+1]; form "right": X = L[i],
    Y = site i (+) R[i+1].  Both give the same H_eff.
    """
    k, na, nb = env.k, env.na, env.nb
    if form == "left":
        X = env.left_enlarged(i) if Xe is None else Xe
        Y = env.R[i + 1]
        normal = "X" if 2 * (i + 1) <= k else "Y"
        psi = onesite_to_psi(wfn, na, nb)
        out = apply_terms(X, Y, hamiltonian_terms(X, Y, normal, env.e_core), psi)
        return psi_to_onesite(out, na, nb)
    X = env.L[i]
    Y = env.right_enlarged(i) if Ye is None else Ye
    normal = "X" if 2 * i <= k else "Y"
    psi = {(ql, (QN_SITE[n], (na - qr[0], nb - qr[1]))): m for (ql, n, qr), m in wfn.items()}
    out = apply_terms(X, Y, hamiltonian_terms(X, Y, normal, env.e_core), psi)
    return {(xl, QN_SITE.index(yl[0]), (na - yl[1][0], nb - yl[1][1])): m for (xl, yl), m in out.items()}


def sigma_twosite(env: Environment, i: int, wfn, Xe=None, Ye=None):
    """H_eff x for a two-site tensor on sites i, i+1 (cut i+1 between them)."""
    k, na, nb = env.k, env.na, env.nb
    X = env.left_enlarged(i) if Xe is None else Xe
    Y = env.right_enlarged(i + 1) if Ye is None else Ye
    normal = "X" if 2 * (i + 1) <= k else "Y"
    psi = twosite_to_psi(wfn, na, nb)
    out = apply_terms(X, Y, hamiltonian_terms(X, Y, normal, env.e_core), psi)
    return psi_to_twosite(out, na, nb)


def diag_onesite(env: Environment, i: int, shapes, Xe=None):
    """diag(H_eff) at site i, one-site (left form); shapes: (q_l, n, q_r) -> (D_l, D_r)."""
    k, na, nb = env.k, env.na, env.nb
    X = env.left_enlarged(i) if Xe is None else Xe
    Y = env.R[i + 1]
    normal = "X" if 2 * (i + 1) <= k else "Y"
    ps = {((ql, QN_SITE[n]), (na - qr[0], nb - qr[1])): s for (ql, n, qr), s in shapes.items()}
    out = diagonal_terms(X, Y, hamiltonian_terms(X, Y, normal, env.e_core), ps)
    return psi_to_onesite(out, na, nb)


def diag_twosite(env: Environment, i: int, shapes, Xe=None, Ye=None):
    k, na, nb = env.k, env.na, env.nb
    X = env.left_enlarged(i) if Xe is None else Xe
    Y = env.right_enlarged(i + 1) if Ye is None else Ye
    normal = "X" if 2 * (i + 1) <= k else "Y"
    ps = {((ql, QN_SITE[n1]), (QN_SITE[n2], (na - qr[0], nb - qr[1]))): s
          for (ql, n1, n2, qr), s in shapes.items()}
    out = diagonal_terms(X, Y, hamiltonian_terms(X, Y, normal, env.e_core), ps)
    return psi_to_twosite(out, na, nb)
