"""Ground-state DMRG sweeps (Eq. dmrg with the gauge shift of Eq. gauge-shift).

Two-site sweeps with a bond-dimension ramp, then the mixed-canonical gauge of
the converged state.  The eigenproblem at each position is solved by a plain
Davidson iteration with the diagonal preconditioner (the paper's Eq. error
applied to the ground state, where S_i = 1).
"""
from __future__ import annotations

import numpy as np

from . import blocks as ob
from . import mps as om
from synth import QN_SITE


def _flat_index(blocks):
    idx, c0 = {}, 0
    for key in sorted(blocks):
        m = blocks[key]
        idx[key] = (c0, m.shape[0], m.shape[1])
        c0 += m.size
    return idx


def davidson(apply, diag, x0, tol=1e-8, max_iter=200, max_space=24):
    """Lowest eigenpair of a symmetric operator; residual 2-norm below `tol`."""
    V = []
    AV = []
    x = x0 / np.linalg.norm(x0)
    theta = 0.0
    for it in range(max_iter):
        for v in V:
            x = x - v * (v @ x)
        for v in V:                      # twice is enough
            x = x - v * (v @ x)
        nx = np.linalg.norm(x)
        if nx < 1e-14:
            break
        x = x / nx
        V.append(x)
        AV.append(apply(x))
        Vm = np.array(V)
        Hs = Vm @ np.array(AV).T
        Hs = 0.5 * (Hs + Hs.T)
        w, U = np.linalg.eigh(Hs)
        theta = w[0]
        u = U[:, 0] @ Vm
        r = U[:, 0] @ np.array(AV) - theta * u
        rn = np.linalg.norm(r)
        if rn < tol:
            return theta, u, it + 1
        den = diag - theta
        den = np.where(np.abs(den) < 1e-4, np.copysign(1e-4, den), den)
        x = -r / den
        if len(V) >= max_space:
            V = [u]
            AV = [U[:, 0] @ np.array(AV)]
    return theta, u, max_iter


def _theta(A, B):
    """Two-site tensor theta[(q_l, n1, n2, q_r)] = sum_m A[(q_l, n1, m)] B[(m, n2, q_r)]."""
    out = {}
    byl = {}
    for (qm, n2, qr), m in B.items():
        byl.setdefault(qm, []).append((n2, qr, m))
    for (ql, n1, qm), a in A.items():
        for (n2, qr, b) in byl.get(qm, []):
            key = (ql, n1, n2, qr)
            val = a @ b
            out[key] = out[key] + val if key in out else val
    return out


def _twosite_shapes(env, i, left_dims, right_dims):
    """All allowed (q_l, n1, n2, q_r) blocks of the two-site space on sites i, i+1."""
    na, nb = env.na, env.nb
    shapes = {}
    for ql, dl in left_dims.items():
        for n1, s1 in enumerate(QN_SITE):
            for n2, s2 in enumerate(QN_SITE):
                qr = (ql[0] + s1[0] + s2[0], ql[1] + s1[1] + s2[1])
                if qr in right_dims:
                    shapes[(ql, n1, n2, qr)] = (dl, right_dims[qr])
    return shapes


def ground_state(ham, t, v, M_schedule, mps0, sweeps_per_M=2, e_tol=1e-11,
                 dav_tol=1e-8, max_sweeps=30, verbose=False):
    """Two-site DMRG; returns (E0, sites in right-canonical form with the centre at site 0).

    M_schedule: list of bond dimensions, the last one repeated until the
    energy changes by less than e_tol between sweeps.
    """
    k = ham.k
    sites = om.right_canonicalize([om.unpack_site(mps0.sites[i], mps0.bonds[i], mps0.bonds[i + 1])
                                   for i in range(k)])
    env = ob.Environment(ham, t, v)
    for b in range(k - 1, 0, -1):
        env.grow_right(b, sites[b])
    energies = []
    sweep = 0
    while sweep < max_sweeps:
        M = M_schedule[min(sweep // sweeps_per_M, len(M_schedule) - 1)]
        E = None
        # left -> right
        for i in range(k - 1):
            th = _theta(sites[i], sites[i + 1])
            E, th = _solve_twosite(env, i, th, dav_tol)
            A, B, _, _ = om.decimate_twosite(th, None, None, M, env.na, env.nb, direction=+1)
            sites[i], sites[i + 1] = A, B
            env.grow_left(i, A)
        # right -> left
        for i in range(k - 2, -1, -1):
            th = _theta(sites[i], sites[i + 1])
            E, th = _solve_twosite(env, i, th, dav_tol)
            A, B, _, _ = om.decimate_twosite(th, None, None, M, env.na, env.nb, direction=-1)
            sites[i], sites[i + 1] = A, B
            env.grow_right(i + 1, B)
        energies.append(E)
        if verbose:
            print(f"sweep {sweep} M={M} E={E:.12f}")
        sweep += 1
        if (sweep // sweeps_per_M >= len(M_schedule) - 1 and len(energies) >= 2
                and abs(energies[-1] - energies[-2]) < e_tol):
            break
    return energies[-1], sites, energies


def onesite_sweeps(ham, t, v, sites, n_sweeps=4, e_tol=1e-12, dav_tol=1e-10, verbose=False):
    """One-site sweeps at fixed bond dimension (no truncation beyond zero weights).

    Brings a two-site DMRG state to a stationary point of the one-site
    manifold, H_i C_i = E C_i at every site (Eq. dmrg), which the TDA assumes.
    `sites` must be right-canonical with the centre at site 0.
    """
    k = ham.k
    sites = [dict(s) for s in sites]
    env = ob.Environment(ham, t, v)
    for b in range(k - 1, 0, -1):
        env.grow_right(b, sites[b])
    energies = []
    for sw in range(n_sweeps):
        E = None
        for i in range(k):                       # left -> right
            E, C = _solve_onesite(env, i, sites[i], dav_tol)
            if i == k - 1:
                sites[i] = C
                break
            L, carry = _split_left(C)
            sites[i] = L
            sites[i + 1] = {kk: carry[kk[0]] @ m for kk, m in sites[i + 1].items() if kk[0] in carry}
            env.grow_left(i, L)
        for i in range(k - 1, -1, -1):           # right -> left
            E, C = _solve_onesite(env, i, sites[i], dav_tol)
            if i == 0:
                sites[i] = C
                break
            R, carry = _split_right(C)
            sites[i] = R
            sites[i - 1] = {kk: m @ carry[kk[2]] for kk, m in sites[i - 1].items() if kk[2] in carry}
            env.grow_right(i, R)
        energies.append(E)
        if verbose:
            print(f"one-site sweep {sw} E={E:.13f}")
        if len(energies) >= 2 and abs(energies[-1] - energies[-2]) < e_tol:
            break
    return energies[-1], sites, energies


def _onesite_shapes(env, i, ql_dims, qr_dims):
    shapes = {}
    for ql, dl in ql_dims.items():
        for n, s in enumerate(QN_SITE):
            qr = (ql[0] + s[0], ql[1] + s[1])
            if qr in qr_dims:
                shapes[(ql, n, qr)] = (dl, qr_dims[qr])
    return shapes


def _solve_onesite(env, i, C, tol):
    ql_dims = dict(env.L[i].labels)
    qr_dims = {(env.na - q[0], env.nb - q[1]): d for q, d in env.R[i + 1].labels.items()}
    shapes = _onesite_shapes(env, i, ql_dims, qr_dims)
    full = {kk: C.get(kk, np.zeros(s)) for kk, s in shapes.items()}
    idx = _flat_index(full)
    Xe = env.left_enlarged(i)
    dg = om.blocks_to_vec(ob.diag_onesite(env, i, shapes, Xe), idx)

    def apply(x):
        return om.blocks_to_vec(ob.sigma_onesite(env, i, om.vec_to_blocks(x, idx), Xe), idx)

    x0 = om.blocks_to_vec(full, idx)
    E, x, _ = davidson(apply, dg, x0, tol=tol)
    return E, om.vec_to_blocks(x, idx)


def _split_left(C, tol=1e-14):
    """C = L (S V^T) per right sector; returns (L blocks, carry[q_r] = S V^T)."""
    L, carry = {}, {}
    for qr in om.right_labels(C):
        M, segs = om.fuse_left(C, qr)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        keep = S > tol * max(S[0], 1e-300) if len(S) else S > 0
        U, S, Vt = U[:, keep], S[keep], Vt[keep]
        if len(S) == 0:
            continue
        for (ql, n, r0, dl) in segs:
            L[(ql, n, qr)] = U[r0:r0 + dl]
        carry[qr] = S[:, None] * Vt
    return L, carry


def _split_right(C, tol=1e-14):
    """C = (U S) R per left sector; returns (R blocks, carry[q_l] = U S)."""
    R, carry = {}, {}
    for ql in om.left_labels(C):
        M, segs = om.fuse_right(C, ql)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        keep = S > tol * max(S[0], 1e-300) if len(S) else S > 0
        U, S, Vt = U[:, keep], S[keep], Vt[keep]
        if len(S) == 0:
            continue
        for (qr, n, c0, dr) in segs:
            R[(ql, n, qr)] = Vt[:, c0:c0 + dr]
        carry[ql] = U * S
    return R, carry


def _solve_twosite(env, i, th, tol):
    left_dims = {q: d for q, d in env.L[i].labels.items()}
    right_own = env.R[i + 2].labels
    right_dims = {(env.na - q[0], env.nb - q[1]): d for q, d in right_own.items()}
    shapes = _twosite_shapes(env, i, left_dims, right_dims)
    full = {kk: th.get(kk, np.zeros(s)) for kk, s in shapes.items()}
    idx = _flat_index(full)
    Xe = env.left_enlarged(i)
    Ye = env.right_enlarged(i + 1)
    dg = om.blocks_to_vec(ob.diag_twosite(env, i, shapes, Xe, Ye), idx)

    def apply(x):
        return om.blocks_to_vec(ob.sigma_twosite(env, i, om.vec_to_blocks(x, idx), Xe, Ye), idx)

    x0 = om.blocks_to_vec(full, idx)
    if np.linalg.norm(x0) < 1e-12:
        x0 = np.ones_like(x0)
    E, x, _ = davidson(apply, dg, x0, tol=tol)
    return E, om.vec_to_blocks(x, idx)


def energy(ham, t, v, sites):
    """<Psi|H|Psi>/<Psi|Psi> of an MPS given as site-tensor dicts (renormalized-operator route)."""
    k = ham.k
    env = ob.Environment(ham, t, v)
    for b in range(k - 1, 0, -1):
        env.grow_right(b, sites[b])
    y = ob.sigma_onesite(env, 0, sites[0], form="left")
    num = sum(np.sum(sites[0][kk] * y[kk]) for kk in sites[0])
    den = sum(np.sum(sites[0][kk] * ob.apply_terms(
        env.left_enlarged(0), env.R[1], [(1.0, ("I",), ("I",))],
        ob.onesite_to_psi({kk: sites[0][kk]}, env.na, env.nb)).get(
            ((kk[0], QN_SITE[kk[1]]), (env.na - kk[2][0], env.nb - kk[2][1])), 0))
        for kk in sites[0])
    return num / den
