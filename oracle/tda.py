"""DMRG-TDA (Sec. "Tamm-Dancoff Approximation", Fig. alg:dmrgtda).

Two routes:

* `tangent_rr` is the definition: the TDA eigenvalues are the Rayleigh-Ritz
  values of H on the span of the first-order (tangent) spaces
  V_i = span{|l0_{i-1} n_i r0_i>} with the reference Psi_0 removed (the TDA
  eigenproblem H X = omega S X of Eq. dmrgrpa with W = 0 is variational in
  that space).  Brute force in the determinant basis; small k only.

* `sweep_tda` is the paper's sweep algorithm, step by step: the block
  Davidson iteration of Fig. alg:david_gep carried out through forward and
  backward sweeps with the Ritz rotation (Eq. ritzrot2), the first-order gauge
  shifts (Eqs. gauge_fwd, gauge_bwd, left1st, right1st), the site sigma vector
  (Eqs. sigv1, sigv2), residual (Eq. rnorm), diagonal preconditioner
  (Eq. error), projection (Eq. param), projected coefficients (Eq. cwfn1st),
  reduced matrix elements (Eqs. hleft2, sleft2) and first-order renormalized
  operators (Eqs. lopr1st, ropr1st).

Energies are total energies theta; excitation energies are omega = theta - E0.
"""
from __future__ import annotations

import numpy as np

from . import blocks as ob
from . import mps as om
from . import fock
from synth import QN_SITE
import synth


# ----------------------------------------------------------------------------
# site-tensor algebra (dict {(q_l, n, q_r): matrix})
# ----------------------------------------------------------------------------
def t_add(A, B, b=1.0, a=1.0):
    out = {kk: a * m for kk, m in A.items()}
    for kk, m in B.items():
        out[kk] = out[kk] + b * m if kk in out else b * m
    return out


def t_scale(A, c):
    return {kk: c * m for kk, m in A.items()}


def t_dot(A, B):
    return float(sum(np.sum(m * B[kk]) for kk, m in A.items() if kk in B))


def t_zero(shapes):
    return {kk: np.zeros(s) for kk, s in shapes.items()}


def bond_lmul(X, A):
    """(X A)[(ql,n,qr)] = X[ql] @ A[(ql,n,qr)]."""
    return {(ql, n, qr): X[ql] @ m for (ql, n, qr), m in A.items() if ql in X}


def bond_rmul(A, X):
    """(A X)[(ql,n,qr)] = A[(ql,n,qr)] @ X[qr]."""
    return {(ql, n, qr): m @ X[qr] for (ql, n, qr), m in A.items() if qr in X}


def contract_left(A, B):
    """(A^T B) over (q_l, n): bond matrix keyed by q_r."""
    out = {}
    for kk, a in A.items():
        if kk in B:
            v = a.T @ B[kk]
            out[kk[2]] = out[kk[2]] + v if kk[2] in out else v
    return out


def contract_right(A, B):
    """(A B^T) over (n, q_r): bond matrix keyed by q_l."""
    out = {}
    for kk, a in A.items():
        if kk in B:
            v = a @ B[kk].T
            out[kk[0]] = out[kk[0]] + v if kk[0] in out else v
    return out


def diag_mat(lam):
    return {q: np.diag(s) for q, s in lam.items()}


def inv_diag_mat(lam, cut=1e-12):
    smax = max((s.max() for s in lam.values() if len(s)), default=1.0)
    return {q: np.diag(np.where(s > cut * smax, 1.0 / np.where(s > 0, s, 1.0), 0.0)) for q, s in lam.items()}


def proj_C(C, C0):
    """Q^C C = C - C0 (C0 . C)   (Eq. realresp, Q^C = 1 - C0 C0^dag)."""
    return t_add(C, C0, -t_dot(C0, C))


def proj_L(C, L0):
    """Q^L C = C - L0 (L0^T C)   (Eq. cwfn1st)."""
    return t_add(C, bond_rmul(L0, contract_left(L0, C)), -1.0)


def proj_R(C, R0):
    """C Q^R = C - (C R0^T) R0   (Eq. right1st)."""
    return t_add(C, bond_lmul(contract_right(C, R0), R0), -1.0)


def onesite_shapes(left_dims, right_dims):
    shapes = {}
    for ql, dl in left_dims.items():
        for n, s in enumerate(QN_SITE):
            qr = (ql[0] + s[0], ql[1] + s[1])
            if qr in right_dims:
                shapes[(ql, n, qr)] = (dl, right_dims[qr])
    return shapes


# ----------------------------------------------------------------------------
# the definition: Rayleigh-Ritz on the tangent space
# ----------------------------------------------------------------------------
def tangent_space(ham, L0, R0, C0, Lam, cut=1e-10):
    """Orthonormal basis (determinant space, columns) of (sum_i V_i) minus Psi_0, with the
    normalized reference, the sector Hamiltonian and its determinants."""
    k = ham.k
    Hd, dets = fock.fci_hamiltonian(ham.h, ham.eri_full(), ham.e_core, k, ham.n_alpha, ham.n_beta)
    cols = []
    psi0 = None
    for i in range(k):
        left = {q: len(Lam[i][q]) for q in Lam[i]}
        right = {q: len(Lam[i + 1][q]) for q in Lam[i + 1]}
        shapes = onesite_shapes(left, right)
        sites = [L0[j] for j in range(i)] + [t_zero(shapes)] + [R0[j] for j in range(i + 1, k)]
        P, idx = om.product_basis_onesite(sites, i, k, dets)
        cols.append(P)
        if i == 0:
            psi0 = P @ om.blocks_to_vec(C0[0], idx)
    B = np.hstack(cols)
    U, s, _ = np.linalg.svd(B, full_matrices=False)
    U = U[:, s > cut * s[0]]
    psi0 = psi0 / np.linalg.norm(psi0)
    U = U - np.outer(psi0, psi0 @ U)
    U2, s2, _ = np.linalg.svd(U, full_matrices=False)
    return U2[:, s2 > cut], psi0, Hd, dets


def tangent_rr(ham, L0, R0, C0, Lam, nroots, cut=1e-10):
    """TDA total energies by Rayleigh-Ritz of H on (sum_i V_i) minus Psi_0 (determinant space)."""
    U2, psi0, Hd, _ = tangent_space(ham, L0, R0, C0, Lam, cut)
    w = np.linalg.eigvalsh(U2.T @ Hd @ U2)
    E0 = psi0 @ Hd @ psi0
    return w[:nroots], E0, U2.shape[1]


# ----------------------------------------------------------------------------
# the sweep algorithm
# ----------------------------------------------------------------------------
class _Vec:
    """One trial vector: R1[i] site tensors and first-order right blocks HR[b]."""

    def __init__(self):
        self.R1 = {}
        self.HR = {}


def _zero_block(mode, v):
    return ob.Block([], mode, {(0, 0): 1}, lambda q: q[0] + q[1], {}, v, transition=True)


def _combine_one(pairs, template):
    ops = {}
    for c, blk in pairs:
        if blk is None or c == 0.0:
            continue
        for key, op in blk.ops.items():
            ops[key] = ob.op_axpy(dict(ops[key]) if key in ops else None, op, c)
    return ob.Block(template.orbs, template.mode, template.labels, template.nel, ops, template.v,
                    transition=True)


def _combine_blocks(pairs, template):
    """sum_j c_j * block_j over every operator of the sets, both directions (Eq. ritzrot2 on H^R)."""
    fwd = _combine_one(pairs, template)
    rev = _combine_one([(c, b.rev if b is not None else None) for c, b in pairs], template)
    fwd.rev, rev.rev = rev, fwd
    return fwd


def _solve_gep(Hr, Sr, cut=1e-12):
    """H alpha = theta S alpha for symmetric H, S (S semi-definite): ascending theta."""
    Hr = 0.5 * (Hr + Hr.T)
    Sr = 0.5 * (Sr + Sr.T)
    s, U = np.linalg.eigh(Sr)
    keep = s > cut * max(s.max(), 1e-300)
    X = U[:, keep] / np.sqrt(s[keep])
    w, Y = np.linalg.eigh(X.T @ Hr @ X)
    return w, X @ Y


class TDASweeper:
    """State and steps of the DMRG-TDA sweep (Fig. alg:dmrgtda)."""

    def __init__(self, ham, t, v, L0, R0, C0, Lam, pinv_cut=1e-12):
        self.ham = ham
        self.k = k = ham.k
        self.v = v
        self.L0, self.R0, self.C0, self.Lam = L0, R0, C0, Lam
        self.env = env = ob.Environment(ham, t, v)
        for b in range(k - 1):
            env.grow_left(b, L0[b])
        for b in range(k - 1, 0, -1):
            env.grow_right(b, R0[b])
        self.XL = [env.left_enlarged(i) for i in range(k)]      # L0[i] (+) site i
        self.YR = [env.right_enlarged(i) for i in range(k)]     # site i (+) R0[i+1]
        self.lam = [diag_mat(Lam[b]) for b in range(k + 1)]
        self.ilam = [inv_diag_mat(Lam[b], pinv_cut) for b in range(k + 1)]
        self.shapes = [onesite_shapes({q: len(Lam[i][q]) for q in Lam[i]},
                                      {q: len(Lam[i + 1][q]) for q in Lam[i + 1]}) for i in range(k)]
        self.diag = [ob.diag_onesite(env, i, self.shapes[i], Xe=self.XL[i]) for i in range(k)]
        y = ob.sigma_onesite(env, 0, C0[0], Xe=self.XL[0])
        self.E0 = t_dot(C0[0], y)

    # --- sigma pieces -----------------------------------------------------------
    def _normal(self, i):
        return "X" if 2 * (i + 1) <= self.k else "Y"

    def h0(self, i, C):
        """H_0^[i] C  (Eq. hzero_sb)."""
        return ob.sigma_onesite(self.env, i, C, Xe=self.XL[i])

    def dh_left(self, i, HL):
        """[H_mu^{L_{i-1}} x h_i x H_0^{R_i}] C0_i  (Eq. hleft_sb applied to C0)."""
        if HL is None or not (HL.ops or HL.rev.ops):
            return {}
        na, nb = self.ham.n_alpha, self.ham.n_beta
        X = ob.enlarge(HL, self.env.sites[i], ob.left_mode(i + 1, self.k), 2 * self.k, self.v,
                       transition_side="X")
        Y = self.env.R[i + 1]
        out = ob.apply_terms(X, Y, ob.hamiltonian_terms(X, Y, self._normal(i), self.ham.e_core),
                             ob.onesite_to_psi(self._full(i, self.C0[i]), na, nb))
        return ob.psi_to_onesite(out, na, nb)

    def dh_right(self, i, HR):
        """[H_0^{L_{i-1}} x h_i x H_mu^{R_i}] C0_i  (second line of Eq. sigv2)."""
        if HR is None or not (HR.ops or HR.rev.ops):
            return {}
        na, nb = self.ham.n_alpha, self.ham.n_beta
        X = self.XL[i]
        out = ob.apply_terms(X, HR, ob.hamiltonian_terms(X, HR, self._normal(i), self.ham.e_core),
                             ob.onesite_to_psi(self._full(i, self.C0[i]), na, nb))
        return ob.psi_to_onesite(out, na, nb)

    def _full(self, i, C):
        return {kk: C.get(kk, np.zeros(s)) for kk, s in self.shapes[i].items()}

    # --- first-order renormalized operators (Eqs. lopr1st, ropr1st) ---------------
    def grow_HL(self, i, HL, L1):
        """First-order left set at cut i+1 (Eq. lopr1st), both transition directions."""
        L0 = self.L0[i]
        new = {}
        for (ql, n, qr), m in L0.items():
            new[qr] = m.shape[1]
        iso0 = ob.left_iso(L0)
        iso1 = ob.left_iso(L1)
        fwd = rev = None
        if HL is not None and (HL.ops or HL.rev.ops):
            X1 = ob.enlarge(HL, self.env.sites[i], ob.left_mode(i + 1, self.k), 2 * self.k, self.v,
                            transition_side="X")
            fwd = ob.renormalize(X1, iso0, iso0, new, transition=True)
            rev = ob.renormalize(X1.rev, iso0, iso0, new, transition=True)
        fwd = ob.renormalize(self.XL[i], iso0, iso1, new, transition=True, acc=fwd)
        rev = ob.renormalize(self.XL[i], iso1, iso0, new, transition=True, acc=rev)
        fwd.rev, rev.rev = rev, fwd
        return fwd

    def grow_HR(self, i, HR, R1):
        """First-order right set at cut i (Eq. ropr1st), both transition directions."""
        R0 = self.R0[i]
        na, nb = self.ham.n_alpha, self.ham.n_beta
        new = {}
        for (ql, n, qr), m in R0.items():
            new[(na - ql[0], nb - ql[1])] = m.shape[0]
        iso0 = ob.right_iso(R0, na, nb)
        iso1 = ob.right_iso(R1, na, nb)
        fwd = rev = None
        if HR is not None and (HR.ops or HR.rev.ops):
            Y1 = ob.enlarge(self.env.sites[i], HR, ob.right_mode(i, self.k), 2 * self.k, self.v,
                            transition_side="Y")
            fwd = ob.renormalize(Y1, iso0, iso0, new, transition=True)
            rev = ob.renormalize(Y1.rev, iso0, iso0, new, transition=True)
        fwd = ob.renormalize(self.YR[i], iso0, iso1, new, transition=True, acc=fwd)
        rev = ob.renormalize(self.YR[i], iso1, iso0, new, transition=True, acc=rev)
        fwd.rev, rev.rev = rev, fwd
        return fwd


def sweep_tda(ham, t, v, L0, R0, C0, Lam, nroots, N=None, eps=1e-14, max_iter=60,
              seed=12345, pinv_cut=1e-12, verbose=False):
    """DMRG-TDA by the sweep algorithm; returns (theta[:nroots], E0, residual norms^2, iterations)."""
    sw = TDASweeper(ham, t, v, L0, R0, C0, Lam, pinv_cut)
    k = sw.k
    n = nroots
    N = max(4 * n, 16) if N is None else N
    env = sw.env

    def random_site(mu, i):
        sh = sw.shapes[i]
        size = sum(a * b for a, b in sh.values())
        x = synth.random_vector(size, seed * 7919 + 1000 * mu + i)
        out, c0 = {}, 0
        for kk in sorted(sh):
            a, b = sh[kk]
            out[kk] = x[c0:c0 + a * b].reshape(a, b)
            c0 += a * b
        return proj_C(out, C0[i])

    # initial sweep: the n random trial vectors enter as "new" vectors (m = 0)
    old = []              # list of _Vec in the previous numbering
    alpha = np.zeros((0, 0))
    theta = np.zeros(0)
    m = 0
    it = 0
    resid = np.full(n, np.inf)
    first = True
    while True:
        if not first:
            w, U = _solve_gep(Hr, Sr)
            m_keep = min(m, U.shape[1])
            alpha = U[:, :m_keep]
            theta = w[:m_keep]
            m = m_keep
        l = m + n
        Hr = np.zeros((l, l))
        Sr = np.zeros((l, l))
        r2 = np.zeros(n)
        # --- forward sweep -----------------------------------------------------
        Cprev = [None] * l
        HLcur = [_zero_block(ob.left_mode(0, k), v) for _ in range(l)]
        L1 = [[None] * k for _ in range(l)]
        rotR1 = [None] * m
        for i in range(k):
            C1 = [None] * l
            HRrot = [None] * m
            for mu in range(m):
                # Eq. ritzrot2: rotate the right-block objects at this site
                R1 = None
                for j, vec in enumerate(old):
                    R1 = t_add(R1 or {}, vec.R1[i], alpha[j, mu])
                HRrot[mu] = (_combine_blocks([(alpha[j, mu], vec.HR.get(i + 1)) for j, vec in enumerate(old)],
                                             env.R[i + 1]) if i + 1 < k else None)
                # Eq. gauge_fwd
                if i == 0:
                    C1[mu] = bond_lmul(sw.lam[0], R1)
                else:
                    X = contract_left(L0[i - 1], Cprev[mu])
                    C1[mu] = t_add(bond_lmul(X, R0[i]), bond_lmul(sw.lam[i], R1))
                C1[mu] = sw._full(i, C1[mu])
            # correction vectors (Eqs. sigv1, rnorm, error, param)
            for mu in range(n):
                if first:
                    C1[m + mu] = random_site(mu, i)
                    continue
                sig = t_add(sw.h0(i, C1[mu]), sw.dh_left(i, HLcur[mu]))
                sig = t_add(sig, sw.dh_right(i, HRrot[mu]))
                sig = sw._full(i, sig)
                # Eq. rnorm, projected by Q^C: at a stationary reference the C0 component
                # <Psi0|H|Psi_mu> of r is zero; elsewhere the projected sum is the residual of the
                # Rayleigh-Ritz problem on the tangent space minus Psi_0
                r = proj_C(t_add(sig, C1[mu], -theta[mu]), C0[i])
                r2[mu] += t_dot(r, r)
                z = {}
                for kk, rm in r.items():
                    den = sw.diag[i][kk] - theta[mu]
                    den = np.where(np.abs(den) < 1e-4, np.copysign(1e-4, den), den)
                    z[kk] = rm / den
                C1[m + mu] = proj_C(z, C0[i])
            # projected coefficients (Eq. cwfn1st) and reduced matrices (Eqs. hleft2, sleft2)
            Ct = [proj_L(C1[mu], L0[i]) for mu in range(l)]
            H0Ct = [sw.h0(i, Ct[mu]) for mu in range(l)]
            dHC0 = [sw.dh_left(i, HLcur[mu]) for mu in range(l)]
            for a in range(l):
                for b in range(l):
                    Hr[a, b] += t_dot(Ct[a], H0Ct[b]) + t_dot(Ct[a], dHC0[b]) + t_dot(dHC0[a], Ct[b])
                    Sr[a, b] += t_dot(Ct[a], Ct[b])
            # Eqs. left1st and lopr1st
            for mu in range(l):
                L1[mu][i] = bond_rmul(Ct[mu], sw.ilam[i + 1])
                if i + 1 < k:
                    HLcur[mu] = sw.grow_HL(i, HLcur[mu], L1[mu][i])
            Cprev = C1
        # --- backward sweep ----------------------------------------------------------
        new = [_Vec() for _ in range(l)]
        for mu in range(l):
            Cb = bond_rmul(L1[mu][k - 1], sw.lam[k])
            HR = None
            for i in range(k - 1, -1, -1):
                if i < k - 1:
                    # Eq. gauge_bwd: C1_i = L1_i C0_{i+1} R0_{i+1}^T + L0_i C1_{i+1} R0_{i+1}^T,
                    # with C0_{i+1} R0_{i+1}^T = Lambda at bond i+1
                    Y = contract_right(Cb, R0[i + 1])
                    Cb = t_add(bond_rmul(L1[mu][i], sw.lam[i + 1]), bond_rmul(L0[i], Y))
                # Eq. right1st
                R1 = bond_lmul(sw.ilam[i], proj_R(Cb, R0[i]))
                new[mu].R1[i] = sw._full(i, R1)
                if i > 0:
                    HR = sw.grow_HR(i, HR, new[mu].R1[i])
                    new[mu].HR[i] = HR
        old = new
        if not first:
            it += 1
            resid = r2.copy()
            if verbose:
                print(f"iter {it}: theta-E0 = {theta[:n] - sw.E0}, r2 = {r2}")
            if np.all(r2 < eps) or it >= max_iter:
                return theta[:n], sw.E0, resid, it
        first = False
        m = l if l < N else n
