"""Frequency-dependent DMRG linear response (Sec. "Time-Dependent DMRG Equation and Linear
Response Theory (LRT)", Eqs. pt_ext, realresp, imagresp, psi1st).  TEST INFRASTRUCTURE ONLY.

A one-body perturbation V = sum_pq d_pq E_pq (E_pq summed over spin, d real symmetric)
drives the reference as V e^{-i omega t} + V e^{+i omega t} (Eq. pt_ext).  The
first-order wavefunction lies in the tangent space (Eq. psi1st with the gauge conditions
left-orthoSeb, right-orthoSeb and Q^C); in an orthonormal tangent basis its two Fourier
components X (poles at +omega_n) and Y (poles at -omega_n) solve

    (H - omega) X + W Y = -v,      W X + (H + omega) Y = -v,      v = <T|V|Psi_0>,

with H and W the matrices of Eq. dmrgrpa.  W = 0 is the Tamm-Dancoff level, where the two
equations decouple into site-summed forms of Eqs. realresp and imagresp.  The response
function is alpha(omega) = v.(X + Y), which at omega = 0 is the second derivative of the
variational energy with respect to the strength of V.

Reading: Eq. realresp writes E0 - omega for the +omega component; with the e^{-i omega t}
convention used here the frequency sign of the two components is swapped, and
alpha(omega) is symmetric in the two labels, so nothing else depends on it.

Brute force in the determinant basis; small k only.
"""
from __future__ import annotations

import numpy as np

from . import fock


def one_body(dets, k, d):
    """V = sum_pq d_pq sum_sigma a+_{p sigma} a_{q sigma} on the determinants (dense)."""
    V = np.zeros((len(dets), len(dets)))
    for p in range(k):
        for q in range(k):
            if d[p, q] != 0.0:
                for s in (0, 1):
                    V += d[p, q] * fock.excitation(dets, 2 * p + s, 2 * q + s).toarray()
    return V


def drive(tg, d):
    """v = <T_a|V|Psi_0> over the orthonormal tangent basis of `tg` (an rpa.Tangent)."""
    return tg.U.T @ (one_body(tg.dets, tg.k, d) @ tg.psi0)


def alpha_tda(H, v, omega):
    """Tamm-Dancoff response: X = -(H - omega)^-1 v, Y = -(H + omega)^-1 v."""
    n = H.shape[0]
    out = []
    for w in np.atleast_1d(omega):
        X = -np.linalg.solve(H - w * np.eye(n), v)
        Y = -np.linalg.solve(H + w * np.eye(n), v)
        out.append(v @ (X + Y))
    return np.array(out)


def alpha_rpa(H, W, v, omega):
    """RPA response: the coupled equations for (X, Y) solved as one linear system."""
    n = H.shape[0]
    out = []
    for w in np.atleast_1d(omega):
        M = np.block([[H - w * np.eye(n), W], [W, H + w * np.eye(n)]])
        z = -np.linalg.solve(M, np.concatenate([v, v]))
        out.append(v @ (z[:n] + z[n:]))
    return np.array(out)


def rpa_modes(H, W):
    """RPA frequencies and amplitudes from the symmetric form (H - W)^1/2 (H + W) (H - W)^1/2.

    With P = X + Y, Q = X - Y: (H + W) P = omega Q and (H - W) Q = omega P, so
    P = (H - W)^1/2 t / sqrt(omega) for a unit eigenvector t, normalized to P.Q =
    X.X - Y.Y = 1.  Returns (omega[n] ascending, X, Y)."""
    H = 0.5 * (H + H.T)
    W = 0.5 * (W + W.T)
    em, Vm = np.linalg.eigh(H - W)
    S = (Vm * np.sqrt(em)) @ Vm.T
    w2, T = np.linalg.eigh(S @ (H + W) @ S)
    om = np.sqrt(w2)
    P = S @ T / np.sqrt(om)
    Q = (H + W) @ P / om
    return om, 0.5 * (P + Q), 0.5 * (P - Q)


def alpha_sum_over_states(omega_n, f_n, omega):
    """sum_n f_n [1 / (omega - omega_n) - 1 / (omega + omega_n)]."""
    w = np.atleast_1d(omega)[:, None]
    return np.sum(f_n * (1.0 / (w - omega_n) - 1.0 / (w + omega_n)), axis=1)


def alpha_exact(ham, d, omega):
    """The exact response of the ground state of the (N_alpha, N_beta) sector: the sum over
    its excited states n of |<n|V|0>|^2 [1 / (omega - omega_n) - 1 / (omega + omega_n)]."""
    Hd, dets = fock.fci_hamiltonian(ham.h, ham.eri_full(), ham.e_core, ham.k, ham.n_alpha, ham.n_beta)
    e, U = np.linalg.eigh(Hd)
    V = one_body(dets, ham.k, d)
    f = (U[:, 1:].T @ (V @ U[:, 0])) ** 2
    return alpha_sum_over_states(e[1:] - e[0], f, omega)


def site_sweep(tg, d, omega, sign=+1, sweeps=30, tol=1e-12):
    """The first-order wavefunction by the paper's site equations (Eqs. realresp, imagresp),
    solved site by site in forward and backward sweeps.

    At site i the component C1_i of X on V_i solves

        (H_0^[i] - (E0 - sign*omega)) C1_i = -Q^C (Delta H_i C0 + V_i C0),

    where H_0^[i] = P_i^T H P_i is the site effective Hamiltonian, V_i C0 = P_i^T V Psi_0 and
    Delta H_i C0 = P_i^T H X_i' is the first-order change from the rest of X (X_i', the
    part of X orthogonal to V_i), kept fixed while site i is solved.  The sweep then moves
    to the next site with the updated X.  sign = +1 is the component of Eq. realresp, -1
    that of Eq. imagresp.  Determinant-space brute force; `tg` is an rpa.Tangent.
    Returns (X, sweeps used, |change| of the last sweep)."""
    n = len(tg.dets)
    Hd, psi0, E0 = tg.Hd, tg.psi0, tg.E0
    vpsi = one_body(tg.dets, tg.k, d) @ psi0
    shift = E0 - sign * omega
    X = np.zeros(n)
    order = list(range(tg.k)) + list(range(tg.k - 2, 0, -1))
    change = np.inf
    for sw in range(1, sweeps + 1):
        X_old = X.copy()
        for i in order:
            P = tg.P[i]
            c0 = P.T @ psi0                                  # C0_i in the product basis
            Xp = X - P @ (P.T @ X)                           # the rest of X
            rhs = -(P.T @ (Hd @ Xp) + P.T @ vpsi)
            rhs -= c0 * (c0 @ rhs)                           # Q^C
            Hi = P.T @ Hd @ P - shift * np.eye(P.shape[1])
            Q = np.eye(P.shape[1]) - np.outer(c0, c0)
            # solve on the range of Q^C: (Q Hi Q) c = rhs with c orthogonal to C0_i
            c = np.linalg.lstsq(Q @ Hi @ Q, rhs, rcond=None)[0]
            c -= c0 * (c0 @ c)
            X = Xp + P @ c
        change = np.linalg.norm(X - X_old)
        if change < tol:
            return X, sw, change
    return X, sweeps, change
