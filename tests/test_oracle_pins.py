"""Pins of the CPU oracle against closed forms, brute force and invariants (no GPU)."""
import itertools
import math
import os

import numpy as np
import pytest

import synth
from oracle import blocks as ob
from oracle import dmrg, fock
from oracle import mps as om
from oracle import tda

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ham(k, na, nb, seed=7):
    H = synth.ab_initio(k, na, nb, seed)
    t, v = fock.spin_integrals(H.h, H.eri)
    return H, t, v


def _sites(m):
    return [om.unpack_site(m.sites[i], m.bonds[i], m.bonds[i + 1]) for i in range(m.k)]


# ----------------------------------------------------------------------------
# determinant space: closed forms and two independent constructions of H
# ----------------------------------------------------------------------------
def test_hubbard_dimer_closed_form():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "hubbard_dimer.txt")) if not l.startswith("#")]
    for t_, U, E0 in [(float(a), float(b), float(c)) for a, b, c in rows]:
        h = np.array([[0.0, -t_], [-t_, 0.0]])
        eri = np.zeros((2, 2, 2, 2))
        eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
        e = fock.fci_energies(h, eri, 0.0, 2, 1, 1, 1)[0]
        assert abs(e - E0) < 1e-12


def test_hueckel_limit_of_ppp():
    # PPP with U = 0 (so V = 0): non-interacting, E0 = sum of the lowest orbital energies per spin
    H = synth.ppp_polyene(6, U=0.0)
    e = fock.fci_energies(H.h, H.eri, H.e_core, 6, 3, 3, 1)[0]
    eps = np.linalg.eigvalsh(H.h)
    assert abs(e - 2 * eps[:3].sum()) < 1e-12


def test_single_site_spectrum():
    h = np.array([[-0.7]])
    eri = np.full((1, 1, 1, 1), 0.9)
    for (na, nb), ref in {(0, 0): 0.0, (1, 0): -0.7, (0, 1): -0.7, (1, 1): -1.4 + 0.9}.items():
        assert abs(fock.fci_energies(h, eri, 0.0, 1, na, nb, 1)[0] - ref) < 1e-14


def test_fci_matches_spin_orbital_fock_space():
    # spin-free E_ij construction vs spin-orbital second quantization on the full Fock space
    H, t, v = _ham(3, 2, 1, 5)
    Hf = fock.fock_hamiltonian(t, v, 6)
    qn = fock.fock_qn(6)
    idx = [D for D in range(64) if qn[D, 0] == 2 and qn[D, 1] == 1]
    Hd, dets = fock.fci_hamiltonian(H.h, H.eri, 0.0, 3, 2, 1)
    assert list(dets) == idx
    assert np.abs(Hf[np.ix_(idx, idx)] - Hd).max() < 1e-13


def test_eri_factor_symmetry():
    H = synth.ab_initio(5, 2, 2, 3)
    e = H.eri
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)]:
        assert np.abs(e - e.transpose(perm)).max() < 1e-14
    # positive semidefinite as a k^2 x k^2 matrix
    assert np.linalg.eigvalsh(e.reshape(25, 25)).min() > -1e-12


# ----------------------------------------------------------------------------
# the complementary-operator decomposition ("x", Eqs. hzero_sb, hleft_sb)
# ----------------------------------------------------------------------------
def _assemble(X, Y, terms, nx, ny, xbits, ybits):
    """Dense sum of coef * (X_op (x) Y_op) on the full Fock space of X u Y."""
    dim = 1 << (nx + ny)
    A = np.zeros((dim, dim))
    for coef, xs, ys in terms:
        xo, yo = X.get(xs), Y.get(ys)
        if xo is None or yo is None:
            continue
        py = ob.parity(ys)
        for (xb, xk), mx in xo.items():
            sg = -1.0 if (py and X.nel(xk) % 2) else 1.0
            for (yb, yk), my in yo.items():
                rb = [xbits[xb][i] | (ybits[yb][j] << nx) for i in range(mx.shape[0]) for j in range(my.shape[0])]
                rk = [xbits[xk][i] | (ybits[yk][j] << nx) for i in range(mx.shape[1]) for j in range(my.shape[1])]
                A[np.ix_(rb, rk)] += coef * sg * np.kron(mx, my)
    return A


def _exact_block(k_sites, first_site, n_so, t, v, mode):
    """Exact (untruncated) block over sites first..first+k-1 by repeated enlargement.

    Returns the block (product labels flattened) and a map label -> Fock bit list."""
    blk = ob.site_block(first_site, n_so, t, v)
    bits = {q: [n] for n, q in enumerate(synth.QN_SITE)}
    for s in range(1, k_sites):
        site = ob.site_block(first_site + s, n_so, t, v)
        e = ob.enlarge(blk, site, mode, n_so, v)
        # flatten product labels to (na, nb)
        lab, newbits, ops = {}, {}, {}
        order = {}
        for (xl, yl), d in sorted(e.labels.items(), key=lambda z: (z[0][1], z[0][0])):
            q = (xl[0] + yl[0], xl[1] + yl[1])
            order[(xl, yl)] = (q, lab.get(q, 0))
            lab[q] = lab.get(q, 0) + d
            newbits.setdefault(q, []).extend([b | (synth.QN_SITE.index(yl) << (2 * s)) for b in bits[xl]])
        for key, op in e.ops.items():
            out = {}
            for (pb, pk), m in op.items():
                qb, ob_ = order[pb]
                qk, ok = order[pk]
                M = out.setdefault((qb, qk), np.zeros((lab[qb], lab[qk])))
                M[ob_:ob_ + m.shape[0], ok:ok + m.shape[1]] += m
            ops[key] = out
        blk = ob.Block(e.orbs, mode, lab, lambda q: q[0] + q[1], ops, v)
        bits = newbits
    return blk, bits


@pytest.mark.parametrize("kx,ky", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_cut_decomposition_assembles_H(kx, ky):
    k = kx + ky
    H, t, v = _ham(k, 1, 1, 11)
    n_so = 2 * k
    Hf = fock.fock_hamiltonian(t, v, n_so)
    for xmode, ymode, normal in [("N", "C", "X"), ("C", "N", "Y")]:
        X, xb = _exact_block(kx, 0, n_so, t, v, xmode)
        Y, yb = _exact_block(ky, kx, n_so, t, v, ymode)
        A = _assemble(X, Y, ob.hamiltonian_terms(X, Y, normal), 2 * kx, 2 * ky, xb, yb)
        assert np.abs(A - Hf).max() < 1e-13


def test_renormalized_operators_match_definition():
    # <l'|O|l> with |l> expanded in the Fock space of the block (definition)
    k, na, nb = 4, 2, 2
    H, t, v = _ham(k, na, nb, 3)
    sites = _sites(synth.random_mps(k, na, nb, 12, 3))
    env = ob.Environment(H, t, v)
    b = 2
    for j in range(b):
        env.grow_left(j, sites[j])
    L = env.L[b]
    nso = 2 * b
    a = fock.fock_annihilators(nso)
    c = [x.T for x in a]

    def full(key):
        kind = key[0]
        if kind == "I":
            return np.eye(1 << nso)
        if kind == "H":
            return fock.fock_hamiltonian(t[:nso, :nso], v[:nso, :nso, :nso, :nso], nso)
        if kind == "C":
            return c[key[1]]
        if kind == "A":
            return c[key[1]] @ c[key[2]]
        if kind == "B":
            return c[key[1]] @ a[key[2]]
        if kind == "S":
            z = key[1]
            S = 0.5 * sum(t[z, q] * a[q] for q in range(nso))
            for q, r, s in itertools.product(range(nso), repeat=3):
                S = S + v[z, q, r, s] * c[q] @ a[s] @ a[r]
            return S
        raise KeyError(key)

    EL = om.expand_left(sites, b)
    seen = set()
    for key, op in L.ops.items():
        F = full(key)
        seen.add(key[0])
        for (qb, qk), m in op.items():
            bb, Pb = EL[qb]
            bk, Pk = EL[qk]
            assert np.abs(Pb.T @ F[np.ix_(bb, bk)] @ Pk - m).max() < 1e-13
    assert {"H", "C", "S", "A", "B", "I"} <= seen
    # conservation: the renormalized N_alpha = sum_x B_{x a, x a} (and N_beta) is diagonal
    # with the sector label: every block state is an eigenstate, so <l'|N|l> = N(q) <l'|l>,
    # the label times the renormalized identity (the Gram matrix of this non-orthonormal
    # block) on the (q, q) blocks, and nothing between different sectors
    ident = next(op for key, op in L.ops.items() if key[0] == "I")
    for spin in (0, 1):
        N = {}
        for x in range(spin, nso, 2):
            for blk, m in L.ops[("B", x, x)].items():
                N[blk] = N.get(blk, 0.0) + m
        for (qb, qk), m in N.items():
            want = qb[spin] * ident[(qb, qk)] if qb == qk else np.zeros_like(m)
            assert np.abs(m - want).max() < 1e-13
        assert any(qb[spin] > 0 for qb, _ in N)


def _brute_env(k, na, nb, M, seed):
    H, t, v = _ham(k, na, nb, seed)
    m = synth.random_mps(k, na, nb, M, seed)
    sites = _sites(m)
    Hd, dets = fock.fci_hamiltonian(H.h, H.eri, H.e_core, k, na, nb)
    env = ob.Environment(H, t, v)
    return H, m, sites, Hd, dets, env


@pytest.mark.parametrize("k,na,nb,M", [(3, 1, 2, 8), (4, 2, 2, 10), (5, 3, 2, 12)])
def test_sigma_onesite_equals_projected_H(k, na, nb, M):
    H, m, sites, Hd, dets, env = _brute_env(k, na, nb, M, 1)
    for b in range(k - 1, 0, -1):
        env.grow_right(b, sites[b])
    rng = np.random.default_rng(0)
    for i in range(k):
        P, idx = om.product_basis_onesite(sites, i, k, dets)
        x = rng.standard_normal(P.shape[1])
        y0 = P.T @ (Hd @ (P @ x))
        w = om.vec_to_blocks(x, idx)
        for form in ("left", "right"):
            y = om.blocks_to_vec(ob.sigma_onesite(env, i, w, form=form), idx)
            assert np.abs(y - y0).max() <= 1e-12 * np.abs(y0).max()
        d = om.blocks_to_vec(ob.diag_onesite(env, i, {kk: vv.shape for kk, vv in w.items()}), idx)
        assert np.abs(d - np.einsum("ij,ij->j", P, Hd @ P)).max() < 1e-12 * np.abs(d).max()
        if i + 1 < k:
            env.grow_left(i, sites[i])


@pytest.mark.parametrize("k,na,nb,M", [(4, 2, 2, 10), (5, 3, 2, 12)])
def test_sigma_twosite_equals_projected_H(k, na, nb, M):
    H, m, sites, Hd, dets, env = _brute_env(k, na, nb, M, 2)
    for b in range(k - 1, 1, -1):
        env.grow_right(b, sites[b])
    rng = np.random.default_rng(1)
    for i in range(k - 1):
        P, idx = om.product_basis_twosite(sites, i, k, dets)
        x = rng.standard_normal(P.shape[1])
        y0 = P.T @ (Hd @ (P @ x))
        y = om.blocks_to_vec(ob.sigma_twosite(env, i, om.vec_to_blocks(x, idx)), idx)
        assert np.abs(y - y0).max() <= 1e-12 * np.abs(y0).max()
        env.grow_left(i, sites[i])


def test_sigma_hermitian_and_packing_roundtrip():
    k, na, nb = 6, 3, 3
    H, t, v = _ham(k, na, nb, 4)
    m = synth.random_mps(k, na, nb, 20, 4, )
    sites = _sites(m)
    env = ob.Environment(H, t, v)
    for b in range(k - 1, 3, -1):
        env.grow_right(b, sites[b])
    for b in range(2):
        env.grow_left(b, sites[b])
    i = 2
    lt, rt = m.bonds[i], m.bonds[i + 2]
    n = synth.twosite_size(synth.twosite_layout(lt, rt))
    x = synth.random_vector(n, 1)
    y = synth.random_vector(n, 2)
    assert np.array_equal(om.pack_twosite(om.unpack_twosite(x, lt, rt), lt, rt), x)
    bx = om.unpack_twosite(x, lt, rt)
    by = om.unpack_twosite(y, lt, rt)
    Hx = ob.sigma_twosite(env, i, bx)
    Hy = ob.sigma_twosite(env, i, by)
    a = sum(np.sum(by[kk] * Hx[kk]) for kk in bx)
    b = sum(np.sum(Hy[kk] * bx[kk]) for kk in bx)
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)
    # conservation: every output block is an allowed (q_l, n1, n2, q_r) block
    assert set(Hx) == set(bx)


# ----------------------------------------------------------------------------
# ground state and gauges
# ----------------------------------------------------------------------------
def test_dmrg_exact_bond_dimension_equals_fci():
    k, na, nb = 5, 3, 2
    H, t, v = _ham(k, na, nb, 7)
    ef = fock.fci_energies(H.h, H.eri, H.e_core, k, na, nb, 1)[0]
    E, sites, _ = dmrg.ground_state(H, t, v, [8, 64], synth.random_mps(k, na, nb, 8, 3))
    assert abs(E - ef) < 1e-8
    assert abs(dmrg.energy(H, t, v, sites) - ef) < 1e-8


def test_dmrg_truncated_is_variational_and_gauges_consistent():
    k, na, nb = 5, 3, 2
    H, t, v = _ham(k, na, nb, 8)
    ef = fock.fci_energies(H.h, H.eri, H.e_core, k, na, nb, 1)[0]
    E, sites, _ = dmrg.ground_state(H, t, v, [6], synth.random_mps(k, na, nb, 6, 3))
    assert E >= ef - 1e-10
    L0, R0, C0, Lam, norm = om.mixed_canonical(sites)
    for i in range(k):
        lam_l = tda.diag_mat(Lam[i])
        lam_r = tda.diag_mat(Lam[i + 1])
        a = tda.bond_rmul(L0[i], lam_r)
        b = tda.bond_lmul(lam_l, R0[i])
        assert max(np.abs(a[kk] - C0[i][kk]).max() for kk in C0[i]) < 1e-12
        assert max(np.abs(b[kk] - C0[i][kk]).max() for kk in C0[i]) < 1e-12
        # isometries (Eq. mps_wave): sum L^T L = 1, sum R R^T = 1
        for q, g in tda.contract_left(L0[i], L0[i]).items():
            assert np.abs(g - np.eye(len(g))).max() < 1e-12
        for q, g in tda.contract_right(R0[i], R0[i]).items():
            assert np.abs(g - np.eye(len(g))).max() < 1e-12


# ----------------------------------------------------------------------------
# DMRG-TDA: sweep algorithm against the tangent-space definition
# ----------------------------------------------------------------------------
def _tda_reference(k, na, nb, M, seed=7):
    H, t, v = _ham(k, na, nb, seed)
    E, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(k, na, nb, M, 3))
    E, sites, _ = dmrg.onesite_sweeps(H, t, v, sites)
    return H, t, v, om.mixed_canonical(sites)


def test_tda_exact_space_gives_fci_excited_states():
    k, na, nb = 4, 2, 2
    H, t, v, (L0, R0, C0, Lam, _) = _tda_reference(k, na, nb, 16)
    ef = fock.fci_energies(H.h, H.eri, H.e_core, k, na, nb, 5)
    w, E0, dim = tda.tangent_rr(H, L0, R0, C0, Lam, 4)
    assert abs(E0 - ef[0]) < 1e-9
    assert dim == 35            # the whole 36-dimensional sector minus Psi_0
    assert np.abs(w - ef[1:5]).max() < 1e-9


@pytest.mark.slow
def test_tda_sweep_matches_tangent_space_definition():
    k, na, nb = 4, 2, 2
    H, t, v, (L0, R0, C0, Lam, _) = _tda_reference(k, na, nb, 8)
    ef = fock.fci_energies(H.h, H.eri, H.e_core, k, na, nb, 4)
    w, E0, dim = tda.tangent_rr(H, L0, R0, C0, Lam, 2)
    th, E0s, r2, it = tda.sweep_tda(H, t, v, L0, R0, C0, Lam, 2, eps=1e-16, max_iter=40)
    assert abs(E0s - E0) < 1e-10
    assert np.abs(th - w).max() < 1e-8
    # Rayleigh-Ritz in a subspace: interlacing with the exact spectrum
    assert np.all(th >= ef[1:3] - 1e-10)


def test_tda_first_order_gauge_conditions_and_overlap_structure():
    # Eqs. left-orthoSeb / sleft2: L1^T L0 = 0 and the site terms are mutually orthogonal
    k, na, nb = 4, 2, 2
    H, t, v, (L0, R0, C0, Lam, _) = _tda_reference(k, na, nb, 8)
    Hd, dets = fock.fci_hamiltonian(H.h, H.eri, H.e_core, k, na, nb)
    sw = tda.TDASweeper(H, t, v, L0, R0, C0, Lam)
    rng = np.random.default_rng(5)
    terms = []
    for i in range(k):
        C = {kk: rng.standard_normal(s) for kk, s in sw.shapes[i].items()}
        Ct = tda.proj_L(tda.proj_C(C, C0[i]), L0[i])
        L1 = tda.bond_rmul(Ct, sw.ilam[i + 1])
        for q, g in tda.contract_left(L1, L0[i]).items():
            assert np.abs(g).max() < 1e-12
        sites = [L0[j] for j in range(i)] + [tda.t_zero(sw.shapes[i])] + [R0[j] for j in range(i + 1, k)]
        P, idx = om.product_basis_onesite(sites, i, k, dets)
        terms.append(P @ om.blocks_to_vec(Ct, idx))
    G = np.array(terms) @ np.array(terms).T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-12 * np.abs(G).max()
    # S_ii = Q^dag Q: the rank of the projected site space is the number of non-redundant parameters
    i = 1
    dims = {kk: s for kk, s in sw.shapes[i].items()}
    n_par = sum(a * b for a, b in dims.values())
    basis = []
    for j in range(n_par):
        e = np.zeros(n_par)
        e[j] = 1.0
        blocks, c0 = {}, 0
        for kk in sorted(dims):
            a, b = dims[kk]
            blocks[kk] = e[c0:c0 + a * b].reshape(a, b)
            c0 += a * b
        Ct = tda.proj_L(tda.proj_C(blocks, C0[i]), L0[i])
        basis.append(np.concatenate([Ct[kk].ravel() for kk in sorted(dims)]))
    rank = np.linalg.matrix_rank(np.array(basis), tol=1e-10)
    fused_rows = {}
    for (ql, n, qr), (a, b) in dims.items():
        fused_rows[qr] = fused_rows.get(qr, 0) + a
    expect = sum((fused_rows[qr] - len(Lam[i + 1][qr])) * len(Lam[i + 1][qr]) for qr in fused_rows)
    assert rank == expect


def test_tangent_space_equals_the_mps_tangent_projector(stationary_k5):
    # The MPS tangent-space projector P_T = sum_i P_L<i x 1_i x P_R>i - sum_i P_L<=i x P_R>i
    # (one-site product spaces V_i minus the bond spaces they share) must be the orthogonal
    # projector onto the span the TDA definition builds (its basis plus Psi_0).
    H, (L0, R0, C0, Lam, _) = stationary_k5
    k = H.k
    U, psi0, _, dets = tda.tangent_space(H, L0, R0, C0, Lam)
    P = np.zeros((len(dets), len(dets)))
    for i in range(k):
        left = {q: len(Lam[i][q]) for q in Lam[i]}
        right = {q: len(Lam[i + 1][q]) for q in Lam[i + 1]}
        shapes = tda.onesite_shapes(left, right)
        sites = [L0[j] for j in range(i)] + [tda.t_zero(shapes)] + [R0[j] for j in range(i + 1, k)]
        Pi, idx = om.product_basis_onesite(sites, i, k, dets)
        P += Pi @ Pi.T
        if i == k - 1:
            continue
        # bond space between sites i and i+1: site-i coefficients L0_i G, G a bond matrix
        cols = []
        for qr, dr in right.items():
            for a in range(dr):
                for b in range(dr):
                    C = {kk: np.outer(m[:, a], np.eye(dr)[b]) for kk, m in L0[i].items() if kk[2] == qr}
                    cols.append(Pi @ om.blocks_to_vec(C, idx))
        Bm = np.array(cols).T
        assert np.abs(Bm.T @ Bm - np.eye(Bm.shape[1])).max() < 1e-12
        P -= Bm @ Bm.T
    want = U @ U.T + np.outer(psi0, psi0)
    assert np.abs(P - P.T).max() < 1e-12
    assert np.abs(P @ P - P).max() < 1e-11
    assert np.abs(P - want).max() < 1e-11


def test_tda_roots_interlace_above_the_exact_excited_states(stationary_k5):
    # at a stationary reference (<T|H|Psi_0> = 0) H is block diagonal on span{Psi_0} + T, so
    # Cauchy interlacing on that space gives E0 >= lambda_1 and theta_j >= lambda_{j+1}
    # for every TDA root, within the same (N_alpha, N_beta) sector
    H, (L0, R0, C0, Lam, _) = stationary_k5
    U, psi0, Hd, _ = tda.tangent_space(H, L0, R0, C0, Lam)
    assert np.linalg.norm(U.T @ (Hd @ psi0)) < 1e-6
    theta = np.linalg.eigvalsh(U.T @ Hd @ U)
    lam = np.linalg.eigvalsh(Hd)
    E0 = psi0 @ Hd @ psi0
    assert E0 >= lam[0] - 1e-12 and E0 <= theta[0]
    assert np.all(theta >= lam[1:len(theta) + 1] - 1e-10)
    # and the upper interlacing side: theta_j <= lambda_{j + 1 + (n - dim)}
    n, m = len(lam), len(theta) + 1
    assert np.all(theta <= lam[n - m + 1:] + 1e-10)
