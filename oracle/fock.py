"""Determinant-space and Fock-space reference operators (plain definitions).

Spin orbitals are ordered 0a, 0b, 1a, 1b, ... (index p = 2*i + sigma).  A
determinant is a bit string D (bit p set = spin orbital p occupied) standing
for a+_{p1} a+_{p2} ... |vac> with p1 < p2 < ...; hence
a_p |D> = (-1)^{#occupied q < p} |D - p>.

The Hamiltonian is the one of the paper's ab initio applications:
H = sum_ij h_ij E_ij + 1/2 sum_ijkl (ij|kl) (E_ij E_kl - delta_jk E_il) + e_core,
E_ij = sum_sigma a+_{i sigma} a_{j sigma}  (spin-free form, used for FCI), or in
spin orbitals H = sum_pq t_pq a+_p a_q + 1/2 sum_pqrs v_pqrs a+_p a+_q a_s a_r
with v_pqrs = <pq|rs> = (pr|qs) delta(s_p, s_r) delta(s_q, s_s).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def spin_integrals(h: np.ndarray, eri: np.ndarray):
    """Spin-orbital t_pq and physicist v_pqrs = <pq|rs> = (pr|qs) delta delta."""
    k = h.shape[0]
    n = 2 * k
    t = np.zeros((n, n))
    v = np.zeros((n, n, n, n))
    for s in range(2):
        t[s::2, s::2] = h
    for s1 in range(2):
        for s2 in range(2):
            # v[p, q, r, s] with p,r of spin s1 and q,s of spin s2: (pr|qs)
            v[s1::2, s2::2, s1::2, s2::2] = eri.transpose(0, 2, 1, 3)
    return t, v


def _popcount(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.uint64)
    x = x - ((x >> np.uint64(1)) & np.uint64(0x5555555555555555))
    x = (x & np.uint64(0x3333333333333333)) + ((x >> np.uint64(2)) & np.uint64(0x3333333333333333))
    x = (x + (x >> np.uint64(4))) & np.uint64(0x0F0F0F0F0F0F0F0F)
    return ((x * np.uint64(0x0101010101010101)) >> np.uint64(56)).astype(np.int64)


def sector_dets(k: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """All determinants with n_alpha alpha and n_beta beta electrons, sorted."""
    out = []
    for ao in itertools.combinations(range(k), n_alpha):
        abits = sum(1 << (2 * i) for i in ao)
        for bo in itertools.combinations(range(k), n_beta):
            out.append(abits | sum(1 << (2 * i + 1) for i in bo))
    return np.array(sorted(out), dtype=np.int64)


def excitation(dets: np.ndarray, p: int, q: int) -> sp.csr_matrix:
    """Sparse matrix of a+_p a_q on the span of `dets` (same particle numbers)."""
    n = len(dets)
    d = dets.astype(np.uint64)
    bp, bq = np.uint64(1 << p), np.uint64(1 << q)
    has_q = (d & bq) != 0
    if p == q:
        idx = np.nonzero(has_q)[0]
        return sp.csr_matrix((np.ones(len(idx)), (idx, idx)), shape=(n, n))
    ok = has_q & ((d & bp) == 0)
    src = np.nonzero(ok)[0]
    d1 = d[src] & ~bq
    sgn = _popcount(d[src] & np.uint64((1 << q) - 1)) + _popcount(d1 & np.uint64((1 << p) - 1))
    d2 = (d1 | bp).astype(np.int64)
    dst = np.searchsorted(dets, d2)
    vals = np.where(sgn % 2 == 0, 1.0, -1.0)
    return sp.csr_matrix((vals, (dst, src)), shape=(n, n))


def fci_hamiltonian(h: np.ndarray, eri: np.ndarray, e_core: float, k: int,
                    n_alpha: int, n_beta: int, dense: bool = True):
    """H in the (n_alpha, n_beta) determinant space, spin-free E_ij form."""
    dets = sector_dets(k, n_alpha, n_beta)
    n = len(dets)
    E = [[excitation(dets, 2 * i, 2 * j) + excitation(dets, 2 * i + 1, 2 * j + 1)
          for j in range(k)] for i in range(k)]
    H = sp.csr_matrix((n, n))
    for i in range(k):
        for j in range(k):
            coef = h[i, j] - 0.5 * sum(eri[i, m, m, j] for m in range(k))
            if coef != 0.0:
                H = H + coef * E[i][j]
    for i in range(k):
        for j in range(k):
            F = sp.csr_matrix((n, n))
            for kk in range(k):
                for l in range(k):
                    if eri[i, j, kk, l] != 0.0:
                        F = F + eri[i, j, kk, l] * E[kk][l]
            H = H + 0.5 * (E[i][j] @ F)
    H = H + e_core * sp.identity(n, format="csr")
    return (H.toarray() if dense else H.tocsr()), dets


def fci_energies(h, eri, e_core, k, n_alpha, n_beta, nroots: int = 1) -> np.ndarray:
    """Lowest `nroots` eigenvalues of H in the sector (dense eigh)."""
    H, _ = fci_hamiltonian(h, eri, e_core, k, n_alpha, n_beta, dense=True)
    w = np.linalg.eigvalsh(H)
    return w[:nroots]


# ----------------------------------------------------------------------------
# full Fock space (all particle numbers) over a contiguous set of spin orbitals
# ----------------------------------------------------------------------------
def fock_annihilators(n_so: int) -> list[np.ndarray]:
    """Dense a_p, p = 0..n_so-1, on the 2^n_so Fock space; state index = bit string."""
    dim = 1 << n_so
    out = []
    for p in range(n_so):
        a = np.zeros((dim, dim))
        for D in range(dim):
            if D >> p & 1:
                sgn = -1.0 if bin(D & ((1 << p) - 1)).count("1") % 2 else 1.0
                a[D ^ (1 << p), D] = sgn
        out.append(a)
    return out


def fock_hamiltonian(t: np.ndarray, v: np.ndarray, n_so: int) -> np.ndarray:
    """sum_pq t a+_p a_q + 1/2 sum_pqrs v a+_p a+_q a_s a_r over spin orbitals 0..n_so-1."""
    a = fock_annihilators(n_so)
    c = [x.T for x in a]
    dim = 1 << n_so
    H = np.zeros((dim, dim))
    for p in range(n_so):
        for q in range(n_so):
            if t[p, q] != 0.0:
                H += t[p, q] * (c[p] @ a[q])
    pair_c = {(p, q): c[p] @ c[q] for p in range(n_so) for q in range(n_so)}
    pair_a = {(s, r): a[s] @ a[r] for s in range(n_so) for r in range(n_so)}
    for p, q, r, s in itertools.product(range(n_so), repeat=4):
        if v[p, q, r, s] != 0.0:
            H += 0.5 * v[p, q, r, s] * (pair_c[(p, q)] @ pair_a[(s, r)])
    return H


def fock_qn(n_so: int) -> np.ndarray:
    """(N_alpha, N_beta) of every Fock state (even bits alpha, odd bits beta)."""
    dim = 1 << n_so
    qn = np.zeros((dim, 2), dtype=np.int64)
    for D in range(dim):
        for p in range(n_so):
            if D >> p & 1:
                qn[D, p % 2] += 1
    return qn
