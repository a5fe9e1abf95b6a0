"""Pins of the oracle's one-particle transition densities (oracle/transition.py).

gamma^nu_pq = <Psi^nu| E_pq |Psi_0>, E_pq = sum_sigma a+_{p sigma} a_{q sigma}, and its
square norm (Sec. "Results", Table site_excitation).  Checked against a single excitation
of a determinant worked out by hand, the adjoint identity, particle-number conservation
and, on the full tangent space, the transition densities of the FCI excited states.
"""
import numpy as np

import synth
from oracle import dmrg, fock, tda, transition
from oracle import mps as om


def test_single_excitation_of_a_determinant_by_hand():
    # k = 3 spatial orbitals, spin orbitals 0a 0b 1a 1b 2a 2b at bits 0..5.
    # |Phi> = |0a 0b 1a> (bits 0, 1, 2); a+_{2a} a_{1a} |Phi>: removing 1a passes the two
    # electrons below bit 2 (+), adding 2a at bit 4 passes bits 0, 1 (+), so
    # |nu> = +|0a 0b 2a> (bits 0, 1, 4) and gamma = e_2 e_1^T, square norm 1.
    dets = fock.sector_dets(3, 2, 1)
    phi = np.zeros(len(dets))
    phi[np.searchsorted(dets, 0b000111)] = 1.0
    nu = np.zeros(len(dets))
    nu[np.searchsorted(dets, 0b010011)] = 1.0
    g = transition.transition_density(dets, 3, nu, phi)
    want = np.zeros((3, 3))
    want[2, 1] = 1.0
    assert np.abs(g - want).max() == 0.0
    assert transition.square_norm(g) == 1.0


def test_singlet_single_excitation_has_square_norm_two():
    # (a+_{1a} a_{0a} + a+_{1b} a_{0b}) |0a 0b> / sqrt(2): gamma_10 = sqrt(2), norm 2
    dets = fock.sector_dets(2, 1, 1)
    phi = np.zeros(len(dets))
    phi[np.searchsorted(dets, 0b0011)] = 1.0
    nu = (fock.excitation(dets, 2, 0) @ phi + fock.excitation(dets, 3, 1) @ phi) / np.sqrt(2.0)
    g = transition.transition_density(dets, 2, nu, phi)
    assert abs(g[1, 0] - np.sqrt(2.0)) < 1e-14
    assert abs(transition.square_norm(g) - 2.0) < 1e-14


def _reference(k, na, nb, M, seed=7):
    H = synth.ab_initio(k, na, nb, seed)
    t, v = fock.spin_integrals(H.h, H.eri)
    E, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(k, na, nb, M, 3))
    E, sites, _ = dmrg.onesite_sweeps(H, t, v, sites)
    return H, om.mixed_canonical(sites)


def test_tda_transition_densities_conserve_particles_and_satisfy_the_adjoint_identity(stationary_k5):
    H, (L0, R0, C0, Lam, _) = stationary_k5
    k = H.k
    theta, X, E0, psi0, dets = transition.tda_states(H, L0, R0, C0, Lam, 3)
    w, E0r, _ = tda.tangent_rr(H, L0, R0, C0, Lam, 3)
    assert np.abs(theta - w).max() < 1e-12 and abs(E0 - E0r) < 1e-12
    for m in range(3):
        g = transition.transition_density(dets, k, X[:, m], psi0)
        # sum_p E_pp = N and <nu|Psi_0> = 0: the trace vanishes
        assert abs(np.trace(g)) < 1e-12
        # E_pq^T = E_qp: <0|E_qp|nu> = <nu|E_pq|0>
        gt = transition.transition_density(dets, k, psi0, X[:, m])
        assert np.abs(gt.T - g).max() < 1e-12


def test_full_tangent_space_gives_the_fci_transition_densities():
    # at the exact bond dimension the TDA states are the FCI excited states
    k, na, nb = 4, 2, 2
    H, (L0, R0, C0, Lam, _) = _reference(k, na, nb, 16)
    theta, X, E0, psi0, dets = transition.tda_states(H, L0, R0, C0, Lam, 4)
    Hd, dets2 = fock.fci_hamiltonian(H.h, H.eri_full(), H.e_core, k, na, nb)
    assert np.array_equal(dets, dets2)
    e, V = np.linalg.eigh(Hd)
    assert np.min(np.diff(e[:6])) > 1e-6          # non-degenerate: eigenvectors fixed up to sign
    v0 = V[:, 0] * np.sign(V[:, 0] @ psi0)
    for m in range(4):
        vf = V[:, m + 1] * np.sign(V[:, m + 1] @ X[:, m])
        gf = transition.transition_density(dets, k, vf, v0)
        g = transition.transition_density(dets, k, X[:, m], psi0)
        assert np.abs(g - gf).max() < 1e-8
        assert abs(transition.square_norm(g) - transition.square_norm(gf)) < 1e-8
