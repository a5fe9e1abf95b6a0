"""DMRG-RPA (Sec. "Tamm-Dancoff Approximation (TDA) and Random Phase Approximation (RPA)",
Eq. dmrgrpa; Sec. "Non-Redundant Parameterizations of the First and Second Order Spaces";
Sec. "Generalization to DMRG-RPA", Eq. bmatrix).  TEST INFRASTRUCTURE ONLY.

The RPA eigenproblem couples the tangent-space Hamiltonian H_ij = <d_i Psi|H - E0|d_j Psi>
with the second-order matrix W_ij = <d_i d_j Psi|H - E0|Psi> through

    [[H, W], [W*, H*]] [X; Y] = omega [[S, 0], [0, -S*]] [X; Y].

Everything here is real and works in an orthonormal basis of the tangent space 𝒯 with
Psi_0 removed (the basis of `tda.tangent_space`), so S = 1.  Tangent vectors are
determinant-space vectors; the site tensors of a tangent vector X follow the
first-order gauge relations of the paper:

    C1_i[X]  the coefficients of X on V_i = span{|l0_{i-1} n_i r0_i>}  (centre at site i),
    L1_i[X] = Q^L_i C1_i[X] Lam_i^-1                                  (Eq. left1st),
    R1_i[X] = Lam_{i-1}^-1 C1_i[X] Q^R_i                              (Eq. right1st),

with Lam the Schmidt values of the bond to the right (left) of site i.  In code, bond b
sits between sites b-1 and b, so L1_i uses Lam[i+1] and R1_i uses Lam[i].

Three constructions of W:

* `w_chart` is the definition through the manifold: in the chart centred at site c,

      Psi_c(X) = prod_{s<c}(L0_s + L1_s[X]) (C0_c + C1_c[X]) prod_{s>c}(R0_s + R1_s[X]),

  whose first-order term is X itself, the energy functional's second-order term along X
  is <X|H-E0|X> + 2<Psi_0|H-E0|Psi_2(X)> with Psi_2 the sum over site pairs of the
  chain with two sites replaced by their first-order tensors.  W is the polarized
  second part.  At a stationary Psi_0 (<𝒯|H-E0|Psi_0> = 0) it does not depend on c.

* `w_paper` follows Eq. bmatrix and the non-redundant second-order projection
  Q^L_i x Q^R_j (i < j): each pair is taken in the gauge whose centre lies between the two
  sites, L1_i on the left and R1_j on the right, joined by Lam (neighbours) or by the
  zeroth-order sites between them (C0 on the first of them).

* `w_sweep` is Eq. bmatrix as the sweep evaluates it, site by site, from the reverse
  first-order left sets; it equals `w_paper` term by term.  `w_action` applies W to one
  vector through the sweep, for the residuals of the RPA Davidson.

Reading: the paper's complex conjugates are trivial here (real MPS); omega are the
positive RPA frequencies, ascending.  Brute force in the determinant basis; small k only.
"""
from __future__ import annotations

import numpy as np

from . import blocks as ob
from . import mps as om
from . import tda as ot


# ----------------------------------------------------------------------------
# first-order site tensors of a tangent vector
# ----------------------------------------------------------------------------
class Tangent:
    """The reference MPS in all gauges with the site product bases V_i on determinants."""

    def __init__(self, ham, L0, R0, C0, Lam, cut=1e-10):
        self.k = ham.k
        self.L0, self.R0, self.C0, self.Lam = L0, R0, C0, Lam
        self.U, self.psi0, self.Hd, self.dets = ot.tangent_space(ham, L0, R0, C0, Lam, cut)
        self.E0 = float(self.psi0 @ self.Hd @ self.psi0)
        # g = (H - E0) Psi_0: every W element is <g| second-order vector>
        self.g = self.Hd @ self.psi0 - self.E0 * self.psi0
        self.shapes, self.P, self.idx = [], [], []
        for i in range(self.k):
            left = {q: len(Lam[i][q]) for q in Lam[i]}
            right = {q: len(Lam[i + 1][q]) for q in Lam[i + 1]}
            shp = ot.onesite_shapes(left, right)
            P, idx = om.product_basis_onesite(self._chain_lr(i, ot.t_zero(shp)), i, self.k, self.dets)
            self.shapes.append(shp)
            self.P.append(P)
            self.idx.append(idx)

    def _chain_lr(self, i, t):
        return [self.L0[s] for s in range(i)] + [t] + [self.R0[s] for s in range(i + 1, self.k)]

    def c1(self, X, i):
        """C1_i[X]: coefficients of X on the orthonormal product basis of V_i."""
        return om.vec_to_blocks(self.P[i].T @ X, self.idx[i])

    def l1(self, X, i):
        """L1_i = Q^L C1_i Lam^-1 (Eq. left1st)."""
        return ot.bond_rmul(ot.proj_L(self.c1(X, i), self.L0[i]), ot.inv_diag_mat(self.Lam[i + 1]))

    def r1(self, X, i):
        """R1_i = Lam^-1 C1_i Q^R (Eq. right1st)."""
        return ot.bond_lmul(ot.inv_diag_mat(self.Lam[i]), ot.proj_R(self.c1(X, i), self.R0[i]))

    # ------------------------------------------------------------------ charts
    def base(self, c, s):
        """Zeroth-order tensor of site s in the gauge centred at site c."""
        return self.L0[s] if s < c else (self.C0[s] if s == c else self.R0[s])

    def comp(self, c, X, s):
        """First-order tensor of site s of X in the gauge centred at site c."""
        return self.l1(X, s) if s < c else (self.c1(X, s) if s == c else self.r1(X, s))

    def chart_state(self, c, X, t):
        """Psi_c(t X) on the determinants: every site tensor base_s + t comp_s."""
        sites = [ot.t_add(self.base(c, s), self.comp(c, X, s), b=t) for s in range(self.k)]
        return om.to_determinants(sites, self.k, self.dets)


# ----------------------------------------------------------------------------
# W as a sum over site pairs of <g| chain with two first-order sites>
# ----------------------------------------------------------------------------
def _units(shapes):
    """Unit site tensors, one per entry, in block order."""
    out = []
    for key in sorted(shapes):
        dl, dr = shapes[key]
        for a in range(dl):
            for b in range(dr):
                t = ot.t_zero(shapes)
                t[key][a, b] = 1.0
                out.append(t)
    return out


def _flat(t, shapes):
    return np.concatenate([t[key].ravel() if key in t else np.zeros(shapes[key][0] * shapes[key][1])
                           for key in sorted(shapes)])


def _pair_form(tg, chain_of, i, j):
    """F[e, e'] = <g| chain with site i = unit e and site j = unit e'> for i < j.

    chain_of(ti) returns the site list with site i set to ti; site j is left free and
    read through its product basis."""
    k = tg.k
    units = _units(tg.shapes[i])
    cols_j = sorted(tg.shapes[j])
    F = np.zeros((len(units), sum(tg.shapes[j][key][0] * tg.shapes[j][key][1] for key in cols_j)))
    for a, e in enumerate(units):
        sites = chain_of(e)
        sites[j] = ot.t_zero(tg.shapes[j])
        P, idx = om.product_basis_onesite(sites, j, k, tg.dets)
        row = tg.g @ P
        F[a] = np.concatenate([row[idx[key][0]:idx[key][0] + idx[key][1] * idx[key][2]]
                               if key in idx else np.zeros(tg.shapes[j][key][0] * tg.shapes[j][key][1])
                               for key in cols_j])
    return F


def _w_from_pairs(tg, pairs):
    """W[a, b] = sum over pairs of F(comp_i(a), comp_j(b)) + F(comp_i(b), comp_j(a)).

    pairs: list of (i, j, chain_of, comp_i, comp_j) with comp_x(X) the first-order tensor
    of X that the chain takes at that site."""
    n = tg.U.shape[1]
    W = np.zeros((n, n))
    for i, j, chain_of, comp_i, comp_j in pairs:
        F = _pair_form(tg, chain_of, i, j)
        Ci = np.stack([_flat(comp_i(tg.U[:, a]), tg.shapes[i]) for a in range(n)])
        Cj = np.stack([_flat(comp_j(tg.U[:, a]), tg.shapes[j]) for a in range(n)])
        G = Ci @ F @ Cj.T
        W += G + G.T
    return W


def w_chart(tg, c):
    """W in the chart centred at site c (the energy functional's second-order term)."""
    k = tg.k
    pairs = []
    for i in range(k):
        for j in range(i + 1, k):
            def chain_of(e, i=i):
                return [e if s == i else tg.base(c, s) for s in range(k)]
            pairs.append((i, j, chain_of,
                          lambda X, i=i: tg.comp(c, X, i), lambda X, j=j: tg.comp(c, X, j)))
    return _w_from_pairs(tg, pairs)


def w_paper(tg):
    """W by Eq. bmatrix: L1_i on the left, R1_j on the right, the reference between.

    Neighbours (j = i + 1): L0_<i, L1_i Lam, R1_j, R0_>j.
    Otherwise:              L0_<i, L1_i, C0_{i+1}, R0_{i+2..j-1}, R1_j, R0_>j."""
    k = tg.k
    pairs = []
    for i in range(k):
        for j in range(i + 1, k):
            if j == i + 1:
                def chain_of(e, i=i):
                    lam = ot.diag_mat(tg.Lam[i + 1])
                    return ([tg.L0[s] for s in range(i)] + [ot.bond_rmul(e, lam)]
                            + [tg.R0[s] for s in range(i + 1, k)])
            else:
                def chain_of(e, i=i):
                    return ([tg.L0[s] for s in range(i)] + [e, tg.C0[i + 1]]
                            + [tg.R0[s] for s in range(i + 2, k)])
            pairs.append((i, j, chain_of, lambda X, i=i: tg.l1(X, i), lambda X, j=j: tg.r1(X, j)))
    return _w_from_pairs(tg, pairs)


# ----------------------------------------------------------------------------
# the RPA eigenproblem
# ----------------------------------------------------------------------------
def h_tangent(tg):
    """H_ij = <d_i Psi|H - E0|d_j Psi> in the orthonormal tangent basis (S = 1)."""
    U = tg.U
    return U.T @ tg.Hd @ U - tg.E0 * np.eye(U.shape[1])


def rpa_omega(H, W):
    """Positive frequencies of [[H, W], [W, H]] [X; Y] = omega [[1, 0], [0, -1]] [X; Y].

    For real H, W with H - W positive definite, omega^2 are the eigenvalues of
    (H - W)^1/2 (H + W) (H - W)^1/2.  Raises when the reference is unstable (a
    non-positive H +- W), where RPA frequencies are not real."""
    H = 0.5 * (H + H.T)
    W = 0.5 * (W + W.T)
    em, Vm = np.linalg.eigh(H - W)
    ep = np.linalg.eigvalsh(H + W)
    if em.min() <= 0.0 or ep.min() <= 0.0:
        raise ValueError("RPA stability matrix is not positive definite")
    sq = (Vm * np.sqrt(em)) @ Vm.T
    w2 = np.linalg.eigvalsh(sq @ (H + W) @ sq)
    return np.sqrt(w2)


def rpa_full(H, W):
    """All eigenvalues of the non-Hermitian RPA matrix [[H, W], [-W, -H]] (Eq. dmrgrpa with
    the metric moved to the left), sorted by real part: they come in +-omega pairs."""
    n = H.shape[0]
    M = np.block([[H, W], [-W, -H]])
    ev = np.linalg.eigvals(M)
    return ev[np.argsort(ev.real)], n


def rpa_roots(ham, L0, R0, C0, Lam, nroots, route="paper", centre=None, cut=1e-10):
    """Lowest `nroots` RPA excitation energies omega (ascending), with the TDA ones
    (eigenvalues of H alone) and E0: (omega_rpa, omega_tda, E0)."""
    tg = Tangent(ham, L0, R0, C0, Lam, cut)
    H = h_tangent(tg)
    W = w_paper(tg) if route == "paper" else w_chart(tg, ham.k - 1 if centre is None else centre)
    return rpa_omega(H, W)[:nroots], np.linalg.eigvalsh(H)[:nroots], tg.E0


# ----------------------------------------------------------------------------
# the reduced RPA problem of the Davidson iteration (Sec. "Generalization to DMRG-RPA")
# ----------------------------------------------------------------------------
def reduced_rpa(H, W, X, Y):
    """Eq. reducedrpa on the trial pairs (X^mu, Y^mu) (columns) and their partners
    (Y^mu, X^mu): the m x m matrices H_R, W_R, S_R, D_R and the positive-norm solutions.

    Returns (omega[m], alpha_X[m, m], alpha_Y[m, m]) for the m roots with positive omega,
    ascending, each normalized to alpha^T [[S, D], [-D, -S]] alpha = 1."""
    HX, HY, WX, WY = H @ X, H @ Y, W @ X, W @ Y
    Hr = X.T @ HX + X.T @ WY + Y.T @ WX + Y.T @ HY
    Wr = X.T @ HY + X.T @ WX + Y.T @ WY + Y.T @ HX
    Sr = X.T @ X - Y.T @ Y
    Dr = X.T @ Y - Y.T @ X
    A = np.block([[Hr, Wr], [Wr, Hr]])
    B = np.block([[Sr, Dr], [-Dr, -Sr]])
    # A is symmetric positive definite for a stable reference: solve B a = (1/omega) A a
    # through the Cholesky factor of A, a symmetric-definite route with real omega
    A = 0.5 * (A + A.T)
    Lc = np.linalg.cholesky(A)
    Li = np.linalg.inv(Lc)
    K = Li @ B @ Li.T                       # antisymmetric part is zero: B is symmetric
    mu, Z = np.linalg.eigh(0.5 * (K + K.T))
    m = X.shape[1]
    keep = np.argsort(-mu)[:m]              # 1/omega > 0, largest first = lowest omega
    omega = 1.0 / mu[keep]
    alpha = Li.T @ Z[:, keep]
    norm = np.einsum("ij,ij->j", alpha, B @ alpha)
    alpha = alpha / np.sqrt(norm)
    return omega, alpha[:m], alpha[m:]


def davidson_rpa(H, W, nroots, tol=1e-10, max_space=None, max_iter=200, seed=0):
    """Block Davidson for the lowest RPA roots on dense H, W (Fig. alg:david_gep carried to
    the paired trial space of Sec. "Generalization to DMRG-RPA").

    Each iteration solves Eq. reducedrpa on the pairs, rotates X and Y together by the Ritz
    vectors (X <- X aX + Y aY, Y <- Y aX + X aY), forms the residuals
    r_X = H X + W Y - omega X and r_Y = W X + H Y + omega Y, preconditions them with the
    diagonal of H (r_X / (h - omega), r_Y / (h + omega)) and appends the corrections
    orthonormalized against the pairs and their partners; past `max_space` pairs it
    restarts from the current Ritz vectors.  Returns (omega[nroots], X, Y, iterations)."""
    n = H.shape[0]
    max_space = max_space or max(4 * nroots, 16)
    rng = np.random.default_rng(seed)
    hd = np.diag(H).copy()
    X = rng.standard_normal((n, nroots))
    Y = np.zeros((n, nroots))
    X, Y = _orth_pairs(X, Y, np.zeros((n, 0)), np.zeros((n, 0)))
    for it in range(1, max_iter + 1):
        omega, aX, aY = reduced_rpa(H, W, X, Y)
        om_ = omega[:nroots]
        Xr = X @ aX[:, :nroots] + Y @ aY[:, :nroots]
        Yr = Y @ aX[:, :nroots] + X @ aY[:, :nroots]
        rX = H @ Xr + W @ Yr - Xr * om_
        rY = W @ Xr + H @ Yr + Yr * om_
        res = np.sqrt(np.sum(rX * rX, axis=0) + np.sum(rY * rY, axis=0))
        if res.max() < tol:
            return om_, Xr, Yr, it
        act = res >= tol
        dX = rX[:, act] / _safe(hd[:, None] - om_[act])
        dY = rY[:, act] / _safe(hd[:, None] + om_[act])
        if X.shape[1] + int(act.sum()) > max_space:
            X, Y = _orth_pairs(Xr, Yr, np.zeros((n, 0)), np.zeros((n, 0)))
        nX, nY = _orth_pairs(dX, dY, X, Y)
        if nX.shape[1] == 0:
            return om_, Xr, Yr, it
        X, Y = np.hstack([X, nX]), np.hstack([Y, nY])
    return om_, Xr, Yr, max_iter


def _safe(d, eps=1e-8):
    return np.where(np.abs(d) < eps, np.copysign(eps, d), d)


def _orth_pairs(dX, dY, X, Y, cut=1e-10):
    """Orthonormalize new pairs (dX, dY) against the span of the pairs (X, Y) and their
    partners (Y, X) in the doubled space, and among themselves with their partners."""
    def both(a, b):
        return np.vstack([np.hstack([a, b]), np.hstack([b, a])])
    basis = both(X, Y)
    outX, outY = [], []
    for j in range(dX.shape[1]):
        v = np.concatenate([dX[:, j], dY[:, j]])
        for _ in range(2):
            if basis.shape[1]:
                v = v - basis @ (basis.T @ v)
        nv = np.linalg.norm(v)
        if nv < cut:
            continue
        v = v / nv
        n = len(v) // 2
        # v is orthogonal to the basis, and then so is its partner p = (y, x); rotate within
        # span{v, p} to w = cos(t) v + sin(t) p with sin(2t) = -<v, p>, which makes w
        # orthogonal to its own partner
        p = np.concatenate([v[n:], v[:n]])
        ov = v @ p
        if abs(ov) > 1.0 - cut:             # v is its own partner up to sign: X = +-Y
            continue
        t = -0.5 * np.arcsin(ov)
        v = np.cos(t) * v + np.sin(t) * p
        v = v / np.linalg.norm(v)
        outX.append(v[:n])
        outY.append(v[n:])
        basis = np.hstack([basis, both(v[:n, None], v[n:, None])])
    if not outX:
        return np.zeros((dX.shape[0], 0)), np.zeros((dX.shape[0], 0))
    return np.stack(outX, axis=1), np.stack(outY, axis=1)


# ----------------------------------------------------------------------------
# W through the sweep (Eq. bmatrix)
# ----------------------------------------------------------------------------
def w_sweep(ham, t, v, L0, R0, C0, Lam, Xs, tg=None):
    """W_mu,nu = sum_i W^[i]_mu,nu for the tangent vectors Xs (determinant-space columns), by
    Eq. bmatrix: W^[i]_mu,nu = (Lam_i R1_i^mu)^T (Delta H_nu^[i])^dag C0_i + (mu <-> nu).

    Lam_i R1_i^mu = C1_i^mu Q^R (Eq. right1st), and (Delta H_nu^[i])^dag C0_i is the site-i
    vector <l1_nu n r0|H|Psi_0>: the effective Hamiltonian of Eq. hleft_sb built on the
    reverse first-order left set <l1|O|l0> of nu (Eq. lopr1st, grown from
    L1_j^nu = Q^L C1_j^nu Lam^-1 for j < i) and applied to C0_i.  Contracted with
    C1_i^mu Q^R it is the overlap of (H - E0) Psi_0 with the second-order chains
    L1_j^nu ... (Lam R1^mu)_i of every j < i."""
    tg = tg or Tangent(ham, L0, R0, C0, Lam)
    sw = ot.TDASweeper(ham, t, v, L0, R0, C0, Lam)
    k = ham.k
    n = Xs.shape[1]
    HL = [ot._zero_block(ob.left_mode(0, k), v) for _ in range(n)]
    W = np.zeros((n, n))
    for i in range(k):
        cr = [ot.proj_R(tg.c1(Xs[:, a], i), R0[i]) for a in range(n)]
        if i > 0:
            dh = [sw.dh_left(i, HL[b].rev) for b in range(n)]
            for a in range(n):
                for b in range(n):
                    W[a, b] += ot.t_dot(cr[a], dh[b])
        if i + 1 < k:
            for b in range(n):
                HL[b] = sw.grow_HL(i, HL[b], tg.l1(Xs[:, b], i))
    return W + W.T


def w_action(ham, t, v, L0, R0, C0, Lam, y, tg=None):
    """The tangent vector W y (determinant space), through the sweep.

    Every pair of W couples the left-gauge tensor of one vector with the right-gauge tensor
    of the other, so W(x, y) = sum_i <C1_i^x, c_i^y> with

        c_i^y = a_i^y Q^R + Q^L b_i^y,
        a_i^y = (Delta H_y^[i])^dag C0_i   from the reverse first-order left set of y
                                            (sites j < i, Eq. lopr1st),
        b_i^y = (Delta H'_y^[i])^dag C0_i  from the reverse first-order right set of y
                                            (sites j > i, Eq. ropr1st),

    and W y = sum_i L0_<i c_i^y R0_>i with Psi_0 projected out."""
    tg = tg or Tangent(ham, L0, R0, C0, Lam)
    sw = ot.TDASweeper(ham, t, v, L0, R0, C0, Lam)
    k = ham.k
    a, b = [{}] * k, [{}] * k
    HL = ot._zero_block(ob.left_mode(0, k), v)
    for i in range(k):
        if i > 0:
            a[i] = sw.dh_left(i, HL.rev)
        if i + 1 < k:
            HL = sw.grow_HL(i, HL, tg.l1(y, i))
    HR = None
    for i in range(k - 1, -1, -1):
        if HR is not None:
            b[i] = sw.dh_right(i, HR.rev)
        if i > 0:
            HR = sw.grow_HR(i, HR, tg.r1(y, i))
    w = np.zeros(len(tg.dets))
    for i in range(k):
        c = ot.t_add(ot.proj_R(sw._full(i, a[i]), R0[i]), ot.proj_L(sw._full(i, b[i]), L0[i]))
        w += tg.P[i] @ om.blocks_to_vec(c, tg.idx[i])
    return w - tg.psi0 * (tg.psi0 @ w)
