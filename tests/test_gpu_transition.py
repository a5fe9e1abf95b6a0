"""One-particle transition densities of the DMRG-TDA roots on the GPU (GPU).

gamma^mu_pq = <Psi^mu| sum_sigma a+_{p sigma} a_{q sigma} |Psi0> and its square norm
(Sec. "Qualitative understanding of DMRG-LRT excitations", Table site_excitation),
from sweep_tda_density, against the oracle's brute force in the determinant basis on the
same reference (`oracle.transition`: the Rayleigh-Ritz eigenvectors of H on the tangent
space, then E_pq applied determinant by determinant).  An eigenvector's sign is arbitrary,
so each root is compared up to one overall sign.  The vectors carry the error of a
converged Davidson, of the order of the residual norm, so the bar is relative to the
largest |gamma| of the roots.
"""
import numpy as np
import pytest

import synth
from oracle import dmrg, fock, transition
from oracle import mps as om

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_1646_gb300 import build
    build.build()
    import paper_1311_1646_gb300 as p
    p.load()
    return p


def _right_form(k, sites):
    R = om.right_canonicalize(sites)
    tables = []
    for b in range(k + 1):
        secs = {}
        if b < k:
            for (ql, _n, _qr), m in R[b].items():
                secs[ql] = m.shape[0]
        else:
            for (_ql, _n, qr), m in R[k - 1].items():
                secs[qr] = m.shape[1]
        tables.append([(q[0], q[1], secs[q]) for q in sorted(secs)])
    return tables, [om.pack_site(R[i], tables[i], tables[i + 1]) for i in range(k)]


def _compare(gpu, ref, tol):
    # One scale for all roots: a root of another spin (a triplet in the M_S = 0 sector) has
    # gamma = 0 exactly, since E_pq is a spin singlet, and the GPU then returns the vector's
    # error, of the order of the residual norm times |E_pq|, not a relative error.
    scale = np.abs(ref).max()
    for mu in range(len(ref)):
        s = 1.0 if np.sum(gpu[mu] * ref[mu]) >= 0 else -1.0
        assert np.abs(gpu[mu] - s * ref[mu]).max() < tol * scale, (mu, np.abs(gpu[mu] - s * ref[mu]).max(), scale)
        assert abs(transition.square_norm(gpu[mu]) - transition.square_norm(ref[mu])) < 2 * tol * max(
            transition.square_norm(ref[mu]), 1e-3)


@pytest.mark.parametrize("k,na,nb,M,n,eps,tol", [(4, 2, 2, 8, 2, 1e-12, 1e-5), (5, 3, 2, 10, 3, 1e-10, 1e-4),
                                               (6, 3, 3, 12, 3, 1e-10, 1e-4)])
def test_transition_density_matches_the_oracle(pkg, k, na, nb, M, n, eps, tol):
    H = synth.ab_initio(k, na, nb, 7)
    t, v = fock.spin_integrals(H.h, H.eri)
    _, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(k, na, nb, M, 3))
    _, sites, _ = dmrg.onesite_sweeps(H, t, v, sites, n_sweeps=30, dav_tol=1e-13)
    L0, R0, C0, Lam, _ = om.mixed_canonical(sites)
    th, vecs, E0, psi0, dets = transition.tda_states(H, L0, R0, C0, Lam, n)
    ref = np.array([transition.transition_density(dets, k, vecs[:, mu], psi0) for mu in range(n)])
    tables, Rp = _right_form(k, sites)
    ctx = pkg.Context(0)
    ctx.op_build(k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(k, na, nb, tables, Rp, 0)
    ctx.tda_prepare()
    omega, resid, e0, gamma = ctx.sweep_tda_density(n, max_iter=150, eps=eps, keep=2 * n)
    ctx.close()
    assert np.all(resid < eps)
    assert np.abs(omega + e0 - th).max() < 1e-8
    _compare(gamma, ref, tol)


def test_transition_density_on_the_full_space_is_the_fci_one(pkg):
    """At the exact bond dimension the TDA roots are FCI excited states, and their
    transition densities are those of the FCI eigenvectors."""
    k, na, nb, M, n = 4, 2, 2, 16, 2
    H = synth.ab_initio(k, na, nb, 7)
    t, v = fock.spin_integrals(H.h, H.eri)
    _, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(k, na, nb, M, 3))
    Hd, dets = fock.fci_hamiltonian(H.h, H.eri_full(), H.e_core, k, na, nb)
    w, V = np.linalg.eigh(Hd)
    ref = np.array([transition.transition_density(dets, k, V[:, 1 + mu], V[:, 0]) for mu in range(n)])
    tables, Rp = _right_form(k, sites)
    ctx = pkg.Context(0)
    ctx.op_build(k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(k, na, nb, tables, Rp, 0)
    ctx.tda_prepare()
    omega, resid, e0, gamma = ctx.sweep_tda_density(n, max_iter=150, eps=1e-10, keep=2 * n)
    ctx.close()
    assert np.abs(omega - (w[1:n + 1] - w[0])).max() < 1e-8
    _compare(gamma, ref, 1e-4)
