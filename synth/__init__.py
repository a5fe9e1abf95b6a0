"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no arithmetic of the DMRG method.  It draws random numbers
and lays them out: one- and two-electron integrals shaped like the paper's
polyene, water and [2Fe-2S] active spaces, bond sector tables, random MPS
site tensors and random trial wavefunctions.  Both sides read identical
arrays from here; nothing here depends on either side.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of stream s is splitmix64 applied to s + (i+1)*GAMMA.
Normal deviates use the Box-Muller transform.

Site quantum numbers: a spatial orbital holds one of d = 4 states ordered
|0>, |alpha>, |beta>, |alpha beta>, with (N_alpha, N_beta) labels QN_SITE.
Within a site the alpha spin orbital precedes the beta one (Jordan-Wigner
order 0a, 0b, 1a, 1b, ...).

Bond b (0..k) separates sites 0..b-1 from b..k-1.  A bond sector is labelled
by the (N_alpha, N_beta) count of the electrons LEFT of the bond.

Site tensor layout ("left-fused"): for site i, for each sector q_r of bond
i+1 in table order, the rows of the fused block are the sub-blocks
n = 0, 1, 2, 3 (sector q_l = q_r - QN_SITE[n] of bond i, skipped when absent),
each D(q_l) rows; the block has D(q_r) columns and is stored row-major.  The
site tensor is the concatenation of those fused blocks.  One-site
wavefunctions use the same layout.  Two-site wavefunctions on sites (i, i+1):
for each sector q_m of bond i+1 that has both a left fusion (bond i sectors
q_m - QN_SITE[n1]) and a right fusion (bond i+2 sectors q_m + QN_SITE[n2]),
a row-major block whose rows run over (n1, l) and columns over (n2, r).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

QN_SITE = ((0, 0), (1, 0), (0, 1), (1, 1))
BASE_SEED = 13111646
EV_TO_EH = 1.0 / 27.211386


# ----------------------------------------------------------------------------
# counter-based random numbers
# ----------------------------------------------------------------------------
def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Return draws offset..offset+count-1 of the SplitMix64 stream `seed`."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in (0, 1): (top 53 bits + 0.5) * 2^-53."""
    z = splitmix64(seed, count, offset)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal deviates by Box-Muller on consecutive uniform pairs."""
    u = uniform(seed, 2 * count, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


class Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def normal(self, count: int) -> np.ndarray:
        out = normal(self.seed, count, self.pos)
        self.pos += count
        return out

    def uniform(self, count: int) -> np.ndarray:
        out = uniform(self.seed, count, 2 * self.pos)
        self.pos += count
        return out


# ----------------------------------------------------------------------------
# Hamiltonians
# ----------------------------------------------------------------------------
@dataclass
class Hamiltonian:
    """H = sum_ij h_ij E_ij + 1/2 sum_ijkl (ij|kl) (E_ij E_kl - delta_jk E_il) + e_core.

    `eri` is the chemist-notation (ij|kl) array (k^4), or None when only the
    factor `B` (nL x k x k, (ij|kl) = sum_L B[L,i,j] B[L,k,l]) is kept.
    """
    name: str
    k: int
    n_alpha: int
    n_beta: int
    h: np.ndarray
    eri: np.ndarray | None
    e_core: float = 0.0
    B: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    def eri_full(self) -> np.ndarray:
        if self.eri is not None:
            return self.eri
        return np.einsum("Lij,Lkl->ijkl", self.B, self.B, optimize=True)


def _sym_normal(stream: Stream, k: int, sd: float) -> np.ndarray:
    """Symmetric k x k matrix: upper triangle (with diagonal) drawn N(0, sd^2), mirrored."""
    iu = np.triu_indices(k)
    vals = stream.normal(len(iu[0])) * sd
    m = np.zeros((k, k))
    m[iu] = vals
    return m + np.triu(m, 1).T


def _factor(stream: Stream, k: int, nL: int, sd: float, decay: float | None) -> np.ndarray:
    B = np.empty((nL, k, k))
    if decay is not None:
        i = np.arange(k)
        env = np.exp(-np.abs(i[:, None] - i[None, :]) / decay)
    for L in range(nL):
        b = _sym_normal(stream, k, sd)
        B[L] = b * env if decay is not None else b
    return B


def ab_initio(k: int, n_alpha: int, n_beta: int, seed: int, *, nL: int | None = None,
              decay: float | None = None, diag: np.ndarray | None = None,
              replace_diag: bool = False, name: str = "ab_initio",
              keep_eri: bool = True) -> Hamiltonian:
    """Ab initio-form synthetic Hamiltonian.

    h: symmetric N(0, 0.5^2) plus linspace(-2, 0, k) on the diagonal (or `diag`,
    added, or replacing the random diagonal when `replace_diag`).
    (ij|kl) = sum_L B^L_ij B^L_kl with symmetric B^L ~ N(0, 0.3^2), optionally
    multiplied elementwise by exp(-|i-j|/decay); nL defaults to k.
    """
    st = Stream(seed)
    h = _sym_normal(st, k, 0.5)
    if diag is None:
        diag = np.linspace(-2.0, 0.0, k)
    if replace_diag:
        h[np.diag_indices(k)] = diag
    else:
        h[np.diag_indices(k)] += diag
    B = _factor(st, k, k if nL is None else nL, 0.3, decay)
    eri = np.einsum("Lij,Lkl->ijkl", B, B, optimize=True) if keep_eri else None
    return Hamiltonian(name, k, n_alpha, n_beta, h, eri, 0.0, B)


def ppp_polyene(n_sites: int = 12, n_elec: int | None = None, *, t_short: float = -2.4,
                t_long: float = -2.2, U: float = 11.13, r_short: float = 1.35,
                r_long: float = 1.46) -> Hamiltonian:
    """Pariser-Parr-Pople trans-polyene with Ohno interaction (energies in Eh).

    Zigzag chain with 120 degree bond angles, bonds alternating short/long
    starting with a short bond.  H = sum t a+a + U sum n_up n_dn
    + sum_{i<j} V_ij (n_i - 1)(n_j - 1), V_ij = U / sqrt(1 + (U r_ij / 14.397)^2),
    folded into h, (ij|kl) and e_core.
    """
    n_elec = n_sites if n_elec is None else n_elec
    pos = np.zeros((n_sites, 2))
    for b in range(n_sites - 1):
        r = r_short if b % 2 == 0 else r_long
        ang = math.radians(30.0 if b % 2 == 0 else -30.0)
        pos[b + 1] = pos[b] + r * np.array([math.cos(ang), math.sin(ang)])
    h = np.zeros((n_sites, n_sites))
    for b in range(n_sites - 1):
        t = t_short if b % 2 == 0 else t_long
        h[b, b + 1] = h[b + 1, b] = t
    eri = np.zeros((n_sites,) * 4)
    e_core = 0.0
    for i in range(n_sites):
        eri[i, i, i, i] = U
        for j in range(n_sites):
            if i == j:
                continue
            r = float(np.linalg.norm(pos[i] - pos[j]))
            V = U / math.sqrt(1.0 + (U * r / 14.397) ** 2)
            eri[i, i, j, j] = V
            h[i, i] -= V          # -V_ij n_i summed over j != i
            if i < j:
                e_core += V
    na = (n_elec + 1) // 2
    nb = n_elec // 2
    return Hamiltonian("ppp_polyene", n_sites, na, nb, h * EV_TO_EH, eri * EV_TO_EH,
                       e_core * EV_TO_EH, None, {"geometry": pos})


def config(idx: int, batch_index: int = 0, keep_eri: bool = True) -> dict:
    """The five workloads (1-based idx) with their sweep parameters.

    1: k=8, 4a4b, ab initio form, M=64 (M=256 is the exact bond dimension).
    2: PPP polyene, 12 sites, 6a6b, M=256, two-site, 6 roots.
    3: water-shaped, k=24, 5a5b, factor decaying exp(-|i-j|/6), M=500, 6 roots.
    4: batch member `batch_index` of 32: k ~ U{10..16}, N ~ {k-2, k, k+2},
       M ~ 32*U{4..12}, 4 roots.
    5: [2Fe-2S]-shaped, k=36, 15a15b, near-degenerate diagonal, rank-200 factor,
       M=1500, 8 roots.
    """
    seed = BASE_SEED + 100 * idx
    if idx == 1:
        H = ab_initio(8, 4, 4, seed, name="abinitio_k8")
        return dict(ham=H, M=64, nroots=4, nsite=2, precision="fp64")
    if idx == 2:
        H = ppp_polyene(12)
        return dict(ham=H, M=256, nroots=6, nsite=2, precision="fp64")
    if idx == 3:
        H = ab_initio(24, 5, 5, seed, decay=6.0, name="water_k24", keep_eri=keep_eri)
        return dict(ham=H, M=500, nroots=6, nsite=1, precision="mixed")
    if idx == 4:
        s = seed + batch_index
        st = Stream(s ^ 0x5BD1E995)
        u = st.uniform(3)
        k = 10 + min(6, int(u[0] * 7))
        n = k + (-2, 0, 2)[min(2, int(u[1] * 3))]
        nb = n // 2
        na = n - nb
        M = 32 * (4 + min(8, int(u[2] * 9)))
        H = ab_initio(k, na, nb, s, name=f"batch_{batch_index}", keep_eri=keep_eri)
        return dict(ham=H, M=M, nroots=4, nsite=1, precision="mixed")
    if idx == 5:
        k = 36
        d = np.empty(k)
        d[:10] = np.linspace(-2.0, -1.1, 10)
        d[10:26] = -1.0 + 0.1 * Stream(seed ^ 0xA5A5).uniform(16)
        d[26:] = np.linspace(-0.8, 0.0, 10)
        H = ab_initio(k, 15, 15, seed, nL=200, diag=d, replace_diag=True,
                      name="fe2s2_k36", keep_eri=keep_eri)
        return dict(ham=H, M=1500, nroots=8, nsite=1, precision="mixed")
    raise ValueError(f"no workload {idx}")


# ----------------------------------------------------------------------------
# bond sector tables and random MPS
# ----------------------------------------------------------------------------
def _fock_count(n_orb: int, na: int, nb: int) -> int:
    if na < 0 or nb < 0 or na > n_orb or nb > n_orb:
        return 0
    return math.comb(n_orb, na) * math.comb(n_orb, nb)


def bond_tables(k: int, n_alpha: int, n_beta: int, M: int) -> list[list[tuple[int, int, int]]]:
    """Sector tables [(N_alpha_left, N_beta_left, dim)] for bonds 0..k.

    The exact dimension of a sector is min(left Fock count, right Fock count).
    Above M the dimensions are shared out in proportion to the exact ones
    (each populated sector keeps at least 1) and then clipped so that every
    sector is reachable from its neighbours: D_b(q) <= sum_n D_{b-1}(q - n)
    and D_b(q) <= sum_n D_{b+1}(q + n).
    """
    tables: list[dict] = []
    for b in range(k + 1):
        exact = {}
        for na in range(0, min(b, n_alpha) + 1):
            for nb in range(0, min(b, n_beta) + 1):
                d = min(_fock_count(b, na, nb), _fock_count(k - b, n_alpha - na, n_beta - nb))
                if d > 0:
                    exact[(na, nb)] = d
        tot = sum(exact.values())
        if tot <= M:
            dims = dict(exact)
        else:
            dims = {q: max(1, min(e, int(M * e / tot))) for q, e in exact.items()}
            order = sorted(exact, key=lambda q: (-exact[q], q))
            excess = sum(dims.values()) - M
            i = 0
            while excess > 0 and i < 10 * len(order) + 10:
                q = order[-1 - (i % len(order))]
                if dims[q] > 1:
                    dims[q] -= 1
                    excess -= 1
                i += 1
            rest = M - sum(dims.values())
            for q in order:
                if rest <= 0:
                    break
                add = min(rest, exact[q] - dims[q])
                dims[q] += add
                rest -= add
        tables.append(dims)
    for _ in range(2):
        for b in range(1, k + 1):
            for q in list(tables[b]):
                cap = sum(tables[b - 1].get((q[0] - s[0], q[1] - s[1]), 0) for s in QN_SITE)
                tables[b][q] = min(tables[b][q], cap)
        for b in range(k - 1, -1, -1):
            for q in list(tables[b]):
                cap = sum(tables[b + 1].get((q[0] + s[0], q[1] + s[1]), 0) for s in QN_SITE)
                tables[b][q] = min(tables[b][q], cap)
        for b in range(k + 1):
            tables[b] = {q: d for q, d in tables[b].items() if d > 0}
    return [[(q[0], q[1], d) for q, d in sorted(t.items())] for t in tables]


def site_layout(left: list, right: list) -> list[tuple]:
    """Left-fused layout of a site tensor between bond tables `left` and `right`.

    Returns [(q_l, n, q_r, D_l, D_r, offset)] in storage order; the sub-block
    (q_l, n, q_r) is a row-major D_l x D_r matrix starting at `offset`.
    """
    ldim = {(a, b): d for a, b, d in left}
    out = []
    off = 0
    for (ra, rb, dr) in right:
        for n, s in enumerate(QN_SITE):
            ql = (ra - s[0], rb - s[1])
            if ql in ldim:
                dl = ldim[ql]
                out.append((ql, n, (ra, rb), dl, dr, off))
                off += dl * dr
    return out


def layout_size(layout: list[tuple]) -> int:
    return sum(e[3] * e[4] for e in layout)


def twosite_layout(left: list, right: list) -> list[tuple]:
    """Layout of a two-site wavefunction between bond tables `left` (bond i) and `right` (bond i+2).

    The middle label q_m runs over every sector reachable from both sides
    (q_l + n1 = q_m = q_r - n2), in (N_alpha, N_beta) order.  Returns
    [(q_l, n1, n2, q_r, D_l, D_r, offset, row_off, col_off, rows, cols, block_off)]
    in storage order, one entry per sub-block.
    """
    ldim = {(a, b): d for a, b, d in left}
    rdim = {(a, b): d for a, b, d in right}
    mids = set()
    for ql in ldim:
        for s in QN_SITE:
            mids.add((ql[0] + s[0], ql[1] + s[1]))
    out = []
    off = 0
    for (ma, mb) in sorted(mids):
        lsub = []
        for n1, s in enumerate(QN_SITE):
            ql = (ma - s[0], mb - s[1])
            if ql in ldim:
                lsub.append((n1, ql, ldim[ql]))
        rsub = []
        for n2, s in enumerate(QN_SITE):
            qr = (ma + s[0], mb + s[1])
            if qr in rdim:
                rsub.append((n2, qr, rdim[qr]))
        rows = sum(x[2] for x in lsub)
        cols = sum(x[2] for x in rsub)
        if rows == 0 or cols == 0:
            continue
        ro = 0
        for (n1, ql, dl) in lsub:
            co = 0
            for (n2, qr, dr) in rsub:
                out.append((ql, n1, n2, qr, dl, dr, off + ro * cols + co, ro, co, rows, cols, off))
                co += dr
            ro += dl
        off += rows * cols
    return out


def twosite_size(layout: list[tuple]) -> int:
    return max((e[11] + e[9] * e[10] for e in layout), default=0)


@dataclass
class MPS:
    """Matrix product state in the shared packed format (see module docstring)."""
    k: int
    n_alpha: int
    n_beta: int
    bonds: list            # k+1 tables [(na, nb, dim)]
    sites: list            # k float64 arrays, left-fused layout
    center: int = 0        # gauge centre (informational)

    def layout(self, i: int) -> list[tuple]:
        return site_layout(self.bonds[i], self.bonds[i + 1])


def random_mps(k: int, n_alpha: int, n_beta: int, M: int, seed: int, canonical: str | None = None) -> MPS:
    """Random MPS: every sub-block ~ N(0,1) / sqrt(fused rows of its block).

    canonical="left" turns every fused block (rows (n, l), columns r) into a
    random isometry with orthonormal columns, canonical="right" every
    right-fused block (rows l, columns (n, r)) into one with orthonormal rows
    (Householder QR of the Gaussian draw, signs fixed by the diagonal of R).
    """
    bonds = bond_tables(k, n_alpha, n_beta, M)
    sites = []
    for i in range(k):
        lay = site_layout(bonds[i], bonds[i + 1])
        st = Stream(seed * 1000003 + i)
        arr = np.empty(layout_size(lay))
        rows = {}
        for (ql, n, qr, dl, dr, off) in lay:
            rows[qr] = rows.get(qr, 0) + dl
        for (ql, n, qr, dl, dr, off) in lay:
            arr[off:off + dl * dr] = st.normal(dl * dr) / math.sqrt(rows[qr])
        if canonical == "left":
            _isometrize_left(arr, lay)
        elif canonical == "right":
            _isometrize_right(arr, lay)
        sites.append(arr)
    return MPS(k, n_alpha, n_beta, bonds, sites)


def _orthonormal_columns(G: np.ndarray) -> np.ndarray:
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def _isometrize_left(arr, lay):
    by_r = {}
    for e in lay:
        by_r.setdefault(e[2], []).append(e)
    for qr, ents in by_r.items():
        dr = ents[0][4]
        G = np.vstack([arr[e[5]:e[5] + e[3] * dr].reshape(e[3], dr) for e in ents])
        Q = _orthonormal_columns(G)
        r0 = 0
        for e in ents:
            arr[e[5]:e[5] + e[3] * dr] = Q[r0:r0 + e[3]].ravel()
            r0 += e[3]


def _isometrize_right(arr, lay):
    by_l = {}
    for e in lay:
        by_l.setdefault(e[0], []).append(e)
    for ql, ents in by_l.items():
        dl = ents[0][3]
        G = np.hstack([arr[e[5]:e[5] + dl * e[4]].reshape(dl, e[4]) for e in ents])
        Q = _orthonormal_columns(G.T).T
        c0 = 0
        for e in ents:
            arr[e[5]:e[5] + dl * e[4]] = Q[:, c0:c0 + e[4]].ravel()
            c0 += e[4]


def mixed_mps(k: int, n_alpha: int, n_beta: int, M: int, seed: int, center: int) -> MPS:
    """Random MPS in a mixed-canonical gauge: sites < center left-orthonormal,
    sites > center right-orthonormal, the centre site Gaussian."""
    A = random_mps(k, n_alpha, n_beta, M, seed, "left")
    B = random_mps(k, n_alpha, n_beta, M, seed + 7777, "right")
    C = random_mps(k, n_alpha, n_beta, M, seed + 9999)
    sites = [A.sites[i] if i < center else (C.sites[i] if i == center else B.sites[i]) for i in range(k)]
    return MPS(k, n_alpha, n_beta, A.bonds, sites, center)


def random_vector(n: int, seed: int) -> np.ndarray:
    """Random trial vector ~ N(0,1), length n."""
    return normal(seed, n)
