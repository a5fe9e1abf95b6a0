"""One-particle transition densities of DMRG-TDA states (TEST INFRASTRUCTURE ONLY).

The paper characterizes each excited state by its one-particle transition density
matrix gamma^nu_pq = <Psi^nu| a+_p a_q |Psi_0> and the square norm
sum_pq (gamma^nu_pq)^2 (Sec. "Results", Table site_excitation): a large norm marks a
single-particle excitation, which the single-site DMRG-TDA describes well.

Reading: p, q are spatial orbitals and a+_p a_q is summed over the two spins
(E_pq = sum_sigma a+_{p sigma} a_{q sigma}), the operator whose square norm reaches 2 for
a singlet single excitation (the paper's values go up to 1.57).  Spin orbitals follow the
Jordan-Wigner order of `fock`: 2p is p alpha, 2p + 1 is p beta.

Brute force in the determinant basis of the (N_alpha, N_beta) sector; small k only.
"""
from __future__ import annotations

import numpy as np

from . import fock
from . import tda


def tda_states(ham, L0, R0, C0, Lam, nroots: int, cut: float = 1e-10):
    """TDA states as determinant-space vectors: the Rayleigh-Ritz eigenvectors of H on the
    tangent space with Psi_0 removed (the definition `tda.tangent_rr` evaluates).
    Returns (theta[nroots], vectors[ndet, nroots], E0, psi0, dets)."""
    U2, psi0, Hd, dets = tda.tangent_space(ham, L0, R0, C0, Lam, cut)
    w, Z = np.linalg.eigh(U2.T @ Hd @ U2)
    E0 = psi0 @ Hd @ psi0
    return w[:nroots], U2 @ Z[:, :nroots], E0, psi0, dets


def transition_density(dets: np.ndarray, k: int, psi_nu: np.ndarray, psi0: np.ndarray) -> np.ndarray:
    """gamma[p, q] = <psi_nu| sum_sigma a+_{p sigma} a_{q sigma} |psi0> over spatial orbitals."""
    g = np.zeros((k, k))
    for p in range(k):
        for q in range(k):
            for s in (0, 1):
                g[p, q] += psi_nu @ (fock.excitation(dets, 2 * p + s, 2 * q + s) @ psi0)
    return g


def square_norm(gamma: np.ndarray) -> float:
    """sum_pq gamma_pq^2 (Table site_excitation)."""
    return float(np.sum(gamma * gamma))
