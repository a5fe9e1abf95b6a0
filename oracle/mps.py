"""Block-sparse MPS utilities (Eqs. mps_wave_gen, mps_wave, gauge-shift).

A site tensor is a dict {(q_l, n, q_r): ndarray D(q_l) x D(q_r)} with bond
labels counting the electrons left of the bond; q_r = q_l + QN_SITE[n].
The packed exchange format (left-fused layout) is defined in `synth`.
"""
from __future__ import annotations

import numpy as np

from synth import QN_SITE, site_layout, twosite_layout


def unpack_site(arr, left, right):
    return {(ql, n, qr): arr[off:off + dl * dr].reshape(dl, dr).copy()
            for (ql, n, qr, dl, dr, off) in site_layout(left, right)}


def pack_site(blocks, left, right):
    lay = site_layout(left, right)
    out = np.zeros(sum(e[3] * e[4] for e in lay))
    for (ql, n, qr, dl, dr, off) in lay:
        if (ql, n, qr) in blocks:
            out[off:off + dl * dr] = blocks[(ql, n, qr)].ravel()
    return out


def unpack_twosite(arr, left, right):
    out = {}
    for (ql, n1, n2, qr, dl, dr, off, ro, co, rows, cols, boff) in twosite_layout(left, right):
        blk = arr[boff:boff + rows * cols].reshape(rows, cols)
        out[(ql, n1, n2, qr)] = blk[ro:ro + dl, co:co + dr].copy()
    return out


def pack_twosite(blocks, left, right):
    lay = twosite_layout(left, right)
    size = 0
    for e in lay:
        size = max(size, e[11] + e[9] * e[10])
    out = np.zeros(size)
    for (ql, n1, n2, qr, dl, dr, off, ro, co, rows, cols, boff) in lay:
        if (ql, n1, n2, qr) in blocks:
            blk = out[boff:boff + rows * cols].reshape(rows, cols)
            blk[ro:ro + dl, co:co + dr] = blocks[(ql, n1, n2, qr)]
    return out


def tables_of(sites, k):
    """Bond tables [(na, nb, dim)] implied by a list of site-tensor dicts."""
    dims = [dict() for _ in range(k + 1)]
    for i, s in enumerate(sites):
        for (ql, n, qr), m in s.items():
            dims[i][ql] = m.shape[0]
            dims[i + 1][qr] = m.shape[1]
    return [[(q[0], q[1], d) for q, d in sorted(t.items())] for t in dims]


# ----------------------------------------------------------------------------
# expansion in the determinant basis (brute force, small k)
# ----------------------------------------------------------------------------
def _site_bits(i, n):
    return ((n & 1) << (2 * i)) | (((n >> 1) & 1) << (2 * i + 1))


def expand_left(sites, b):
    """|l_b> in occupation bit strings of sites 0..b-1: dict q -> (bits array, matrix)."""
    cur = {(0, 0): (np.array([0], dtype=np.int64), np.ones((1, 1)))}
    for i in range(b):
        nxt = {}
        for (ql, n, qr), m in sites[i].items():
            if ql not in cur:
                continue
            bits, P = cur[ql]
            nb = bits | _site_bits(i, n)
            nxt.setdefault(qr, []).append((nb, P @ m))
        cur = {q: (np.concatenate([x[0] for x in L]), np.vstack([x[1] for x in L])) for q, L in nxt.items()}
    return cur


def expand_right(sites, b, k):
    """|r_b> (sites b..k-1) keyed by the bond-b label: dict q -> (bits, matrix n_bits x D(q))."""
    if b == k:
        return {q: (np.array([0], dtype=np.int64), np.ones((1, 1))) for q in right_labels(sites[k - 1])}
    cur = None
    for i in range(k - 1, b - 1, -1):
        nxt = {}
        for (ql, n, qr), m in sites[i].items():
            if cur is None:
                bits, P = np.array([0], dtype=np.int64), np.ones((1, 1))
            else:
                if qr not in cur:
                    continue
                bits, P = cur[qr]
            nbits = bits | _site_bits(i, n)
            # |r_i; q_l, a> = sum m[a, c] |n>|r_{i+1}; q_r, c>: the matrix maps c -> a
            nxt.setdefault(ql, []).append((nbits, P @ m.T))
        cur = {q: (np.concatenate([x[0] for x in L]), np.vstack([x[1] for x in L])) for q, L in nxt.items()}
    return cur


def product_basis_onesite(sites, i, k, dets):
    """Columns |l_i n r_{i+1}> expanded on `dets`; returns (P, index) with index[(q_l,n,q_r)] = slice."""
    EL = expand_left(sites, i)
    ER = expand_right(sites, i + 1, k)
    pos = {int(d): j for j, d in enumerate(dets)}
    cols = []
    index = {}
    c0 = 0
    for (ql, n, qr), m in sorted(sites[i].items()):
        if ql not in EL:
            continue
        lb, Lm = EL[ql]
        if qr not in ER:
            continue
        rb, Rm = ER[qr]
        dl, dr = Lm.shape[1], Rm.shape[1]
        block = np.zeros((len(dets), dl * dr))
        sb = _site_bits(i, n)
        for a_i, a in enumerate(lb):
            for b_i, bb in enumerate(rb):
                det = int(a) | sb | int(bb)
                if det in pos:
                    block[pos[det]] += np.kron(Lm[a_i], Rm[b_i])
        cols.append(block)
        index[(ql, n, qr)] = (c0, dl, dr)
        c0 += dl * dr
    return np.hstack(cols), index


def product_basis_twosite(sites, i, k, dets):
    """Columns |l_i n1 n2 r_{i+2}> on `dets`; index[(q_l, n1, n2, q_r)] = (col, D_l, D_r)."""
    EL = expand_left(sites, i)
    ER = expand_right(sites, i + 2, k)
    pos = {int(d): j for j, d in enumerate(dets)}
    cols, index, c0 = [], {}, 0
    for ql in sorted(EL):
        lb, Lm = EL[ql]
        for n1, s1 in enumerate(QN_SITE):
            qm = (ql[0] + s1[0], ql[1] + s1[1])
            for n2, s2 in enumerate(QN_SITE):
                qr = (qm[0] + s2[0], qm[1] + s2[1])
                if qr not in ER:
                    continue
                rb, Rm = ER[qr]
                dl, dr = Lm.shape[1], Rm.shape[1]
                block = np.zeros((len(dets), dl * dr))
                sb = _site_bits(i, n1) | _site_bits(i + 1, n2)
                for a_i, a in enumerate(lb):
                    for b_i, bb in enumerate(rb):
                        det = int(a) | sb | int(bb)
                        if det in pos:
                            block[pos[det]] += np.kron(Lm[a_i], Rm[b_i])
                cols.append(block)
                index[(ql, n1, n2, qr)] = (c0, dl, dr)
                c0 += dl * dr
    return np.hstack(cols), index


def blocks_to_vec(blocks, index):
    n = sum(d[1] * d[2] for d in index.values())
    x = np.zeros(n)
    for key, (c0, dl, dr) in index.items():
        if key in blocks:
            x[c0:c0 + dl * dr] = blocks[key].ravel()
    return x


def vec_to_blocks(x, index):
    return {key: x[c0:c0 + dl * dr].reshape(dl, dr).copy() for key, (c0, dl, dr) in index.items()}


def to_determinants(sites, k, dets):
    """Coefficients of the MPS (Eq. mps_wave_gen) on the determinant list `dets`."""
    E = expand_left(sites, k)
    pos = {int(d): j for j, d in enumerate(dets)}
    out = np.zeros(len(dets))
    for q, (bits, P) in E.items():
        for r, b in enumerate(bits):
            if int(b) in pos:
                out[pos[int(b)]] += P[r, 0]
    return out


# ----------------------------------------------------------------------------
# fused views, canonical forms and decimation (Eq. gauge-shift)
# ----------------------------------------------------------------------------
def fuse_left(site, qr):
    """Rows (n, l) of the blocks with right label qr: matrix and [(q_l, n, row_off, D_l)]."""
    parts = [(n, ql, m) for (ql, n, q), m in site.items() if q == qr]
    parts.sort(key=lambda x: x[0])
    segs, mats, off = [], [], 0
    for n, ql, m in parts:
        segs.append((ql, n, off, m.shape[0]))
        mats.append(m)
        off += m.shape[0]
    return np.vstack(mats), segs


def fuse_right(site, ql):
    """Columns (n, r) of the blocks with left label ql: matrix and [(q_r, n, col_off, D_r)]."""
    parts = [(n, qr, m) for (q, n, qr), m in site.items() if q == ql]
    parts.sort(key=lambda x: x[0])
    segs, mats, off = [], [], 0
    for n, qr, m in parts:
        segs.append((qr, n, off, m.shape[1]))
        mats.append(m)
        off += m.shape[1]
    return np.hstack(mats), segs


def right_labels(site):
    return sorted({qr for (_, _, qr) in site})


def left_labels(site):
    return sorted({ql for (ql, _, _) in site})


def right_canonicalize(sites, tol=1e-14):
    """Right-canonical form R_1..R_{k-1} with the norm kept in site 0 (SVD, zero weights dropped)."""
    sites = [dict(s) for s in sites]
    k = len(sites)
    for i in range(k - 1, 0, -1):
        new_i, carry = {}, {}
        for ql in left_labels(sites[i]):
            M, segs = fuse_right(sites[i], ql)
            U, S, Vt = np.linalg.svd(M, full_matrices=False)
            keep = S > tol * max(1.0, S[0] if len(S) else 1.0)
            if not np.any(keep):
                continue
            U, S, Vt = U[:, keep], S[keep], Vt[keep]
            for (qr, n, c0, dr) in segs:
                new_i[(ql, n, qr)] = Vt[:, c0:c0 + dr]
            carry[ql] = U * S
        sites[i] = new_i
        prev = {}
        for (a, n, b), m in sites[i - 1].items():
            if b in carry:
                prev[(a, n, b)] = m @ carry[b]
        sites[i - 1] = prev
    return sites


def left_canonicalize(sites, tol=1e-14):
    """Left-canonical L_0..L_{k-2} with the norm kept in the last site."""
    sites = [dict(s) for s in sites]
    k = len(sites)
    for i in range(k - 1):
        new_i, carry = {}, {}
        for qr in right_labels(sites[i]):
            M, segs = fuse_left(sites[i], qr)
            U, S, Vt = np.linalg.svd(M, full_matrices=False)
            keep = S > tol * max(1.0, S[0] if len(S) else 1.0)
            if not np.any(keep):
                continue
            U, S, Vt = U[:, keep], S[keep], Vt[keep]
            for (ql, n, r0, dl) in segs:
                new_i[(ql, n, qr)] = U[r0:r0 + dl]
            carry[qr] = S[:, None] * Vt
        sites[i] = new_i
        nxt = {}
        for (a, n, b), m in sites[i + 1].items():
            if a in carry:
                nxt[(a, n, b)] = carry[a] @ m
        sites[i + 1] = nxt
    return sites


def mixed_canonical(sites, tol=1e-12):
    """All gauges at once: L0[i], R0[i], C0[i], Lam[b] with C0_i = L0_i Lam_i = Lam_{i-1} R0_i.

    Starting from the right-canonical form, a left-to-right SVD pass puts every
    bond in its Schmidt basis; Lam[b] (bond b between sites b-1 and b) is a
    dict q -> singular values.  Returns (L0, R0, C0, Lam, norm).
    """
    k = len(sites)
    R = right_canonicalize(sites, tol)
    norm = np.sqrt(sum(np.sum(m * m) for m in R[0].values()))
    R[0] = {kk: m / norm for kk, m in R[0].items()}
    Lam = {0: {(0, 0): np.array([1.0])}}
    L0, R0, C0 = [None] * k, [None] * k, [None] * k
    V_prev = {(0, 0): np.eye(1)}          # rotation of bond i's old basis into its Schmidt basis
    for i in range(k):
        # C_i in (Schmidt at bond i) x (old bond i+1 basis)
        Ci = {}
        for (ql, n, qr), m in R[i].items():
            if ql in V_prev:
                Ci[(ql, n, qr)] = (Lam[i][ql][:, None] * (V_prev[ql].T @ m))
        Li, Vn, Sn = {}, {}, {}
        for qr in right_labels(Ci):
            M, segs = fuse_left(Ci, qr)
            U, S, Vt = np.linalg.svd(M, full_matrices=False)
            keep = S > tol * max(S[0], 1e-300)
            U, S, Vt = U[:, keep], S[keep], Vt[keep]
            if len(S) == 0:
                continue
            for (ql, n, r0, dl) in segs:
                Li[(ql, n, qr)] = U[r0:r0 + dl]
            Vn[qr] = Vt.T
            Sn[qr] = S
        L0[i] = Li
        Lam[i + 1] = Sn
        R0[i] = {}
        C0[i] = {}
        for (ql, n, qr), m in R[i].items():
            if ql in V_prev and qr in Vn:
                R0[i][(ql, n, qr)] = V_prev[ql].T @ m @ Vn[qr]
                C0[i][(ql, n, qr)] = Ci[(ql, n, qr)] @ Vn[qr]
        V_prev = Vn
    return L0, R0, C0, Lam, norm


def decimate_twosite(theta, left_table, right_table, M, na, nb, tol=1e-14, direction=+1):
    """Split a two-site tensor theta (q_l, n1, n2, q_r) by SVD keeping the M largest weights.

    Singular values are ranked over all middle sectors (ties broken by sector
    order); weights below tol * largest are dropped.  direction +1 keeps the
    left factor isometric (L_i, and S V^T moves right), -1 the right one.
    Returns (A_left, A_right, discarded_weight, kept singular values).
    """
    mids = sorted({(ql[0] + QN_SITE[n1][0], ql[1] + QN_SITE[n1][1]) for (ql, n1, n2, qr) in theta})
    svd = {}
    for qm in mids:
        rows, cols = [], []
        for (ql, n1, n2, qr), m in theta.items():
            if (ql[0] + QN_SITE[n1][0], ql[1] + QN_SITE[n1][1]) != qm:
                continue
            if (ql, n1) not in [r[:2] for r in rows]:
                rows.append((ql, n1, m.shape[0]))
            if (n2, qr) not in [c[:2] for c in cols]:
                cols.append((n2, qr, m.shape[1]))
        rows.sort(key=lambda r: (r[1], r[0]))
        cols.sort(key=lambda c: (c[0], c[1]))
        R = sum(r[2] for r in rows)
        Cn = sum(c[2] for c in cols)
        Mx = np.zeros((R, Cn))
        ro = {}
        o = 0
        for r in rows:
            ro[r[:2]] = o
            o += r[2]
        co = {}
        o = 0
        for c in cols:
            co[c[:2]] = o
            o += c[2]
        for (ql, n1, n2, qr), m in theta.items():
            if (ql[0] + QN_SITE[n1][0], ql[1] + QN_SITE[n1][1]) != qm:
                continue
            r0, c0 = ro[(ql, n1)], co[(n2, qr)]
            Mx[r0:r0 + m.shape[0], c0:c0 + m.shape[1]] = m
        U, S, Vt = np.linalg.svd(Mx, full_matrices=False)
        svd[qm] = (U, S, Vt, rows, cols, ro, co)
    allsv = sorted(((s, qm, j) for qm, (U, S, Vt, *_) in svd.items() for j, s in enumerate(S)),
                   key=lambda x: (-x[0], x[1], x[2]))
    smax = allsv[0][0] if allsv else 0.0
    kept = [x for x in allsv[:M] if x[0] > tol * smax]
    keep = {}
    for s, qm, j in kept:
        keep.setdefault(qm, []).append(j)
    disc = sum(s * s for s, *_ in allsv[len(kept):])
    A, B, lam = {}, {}, {}
    for qm, js in keep.items():
        js = sorted(js)
        U, S, Vt, rows, cols, ro, co = svd[qm]
        U, S, Vt = U[:, js], S[js], Vt[js]
        lam[qm] = S
        if direction > 0:
            left, right = U, S[:, None] * Vt
        else:
            left, right = U * S, Vt
        for (ql, n1, dl) in rows:
            r0 = ro[(ql, n1)]
            A[(ql, n1, qm)] = left[r0:r0 + dl]
        for (n2, qr, dr) in cols:
            c0 = co[(n2, qr)]
            B[(qm, n2, qr)] = right[:, c0:c0 + dr]
    return A, B, disc, lam
