"""Pins of the oracle's DMRG-RPA (oracle/rpa.py; Eq. dmrgrpa, Eq. bmatrix).

* The chart Psi_c(X) built from the first-order gauge relations (Eqs. left1st, right1st)
  reproduces Psi_0 and X as its zeroth- and first-order Taylor terms, from a full MPS
  contraction at several step sizes (independent of the pairwise construction of W).
* H + W is the second derivative of the energy functional along the chart, by finite
  differences of the Rayleigh quotient, and W is the chart's second-order term.
* At a stationary reference, W does not depend on the chart, and the paper's pairwise
  construction (L1_i ... R1_j) gives the same RPA frequencies.
* The RPA frequencies come in +-omega pairs and the lowest lies at or below the lowest
  TDA one (Thouless' minimum principle); the TDA limit is the tangent-space Rayleigh-Ritz.
* At the exact bond dimension Psi_0 is an eigenstate: W = 0 and RPA = TDA = FCI.
* Eq. bmatrix through the sweep (the reverse first-order left sets applied to C0, contracted
  with C1 Q^R site by site) equals the pairwise W on any set of tangent vectors, and the
  action W y built from the reverse left and right sets of y is the dense W applied to y.
"""
import numpy as np
import pytest

import synth
from oracle import dmrg, fock, rpa, tda
from oracle import mps as om


def _reference(k, na, nb, M, seed=7):
    H = synth.ab_initio(k, na, nb, seed)
    t, v = fock.spin_integrals(H.h, H.eri)
    E, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(k, na, nb, M, 3))
    E, sites, _ = dmrg.onesite_sweeps(H, t, v, sites, n_sweeps=30, dav_tol=1e-13)
    return H, om.mixed_canonical(sites)


@pytest.fixture(scope="module")
def truncated(stationary_k5):
    # k = 5 at M = 6 (bond dimensions 4, 6, 6, 4): the middle sites have non-empty Q^L and
    # Q^R spaces, so pairs that are not neighbours (C0 between them) carry weight
    H, (L0, R0, C0, Lam, _) = stationary_k5
    return H, rpa.Tangent(H, L0, R0, C0, Lam), (L0, R0, C0, Lam)


def _taylor(tg, c, X, order):
    ts = np.array([-0.5, -0.25, -0.1, 0.0, 0.1, 0.25, 0.5, 0.75])
    V = np.stack([tg.chart_state(c, X, t) for t in ts])
    A = np.vander(ts, tg.k + 1, increasing=True)       # Psi_c(tX) is a polynomial of degree k
    coef = np.linalg.lstsq(A, V, rcond=None)[0]
    assert np.abs(A @ coef - V).max() < 1e-12
    return coef[:order + 1]


def test_chart_first_order_term_is_the_tangent_vector(truncated):
    _, tg, _ = truncated
    rng = np.random.default_rng(3)
    for c in range(tg.k):
        X = tg.U @ rng.standard_normal(tg.U.shape[1])
        c0, c1 = _taylor(tg, c, X, 1)
        assert np.abs(c0 - tg.psi0).max() < 1e-12
        assert np.abs(c1 - X).max() < 1e-12


def test_w_is_the_second_order_term_and_h_plus_w_the_energy_hessian(truncated):
    _, tg, _ = truncated
    Ht = rpa.h_tangent(tg)
    rng = np.random.default_rng(4)
    for c in (0, 2, 4):
        W = rpa.w_chart(tg, c)
        a = rng.standard_normal(tg.U.shape[1])
        X = tg.U @ a
        _, _, c2 = _taylor(tg, c, X, 2)
        # E(tX) = E0 + t^2 (X^T (H - E0) X + 2 <g|Psi_2>) + O(t^3): W(X, X) = 2 <g|Psi_2>
        assert abs(a @ W @ a - 2 * tg.g @ c2) < 1e-10 * max(1.0, abs(a @ W @ a))

        def energy(t):
            psi = tg.chart_state(c, X, t)
            return (psi @ tg.Hd @ psi) / (psi @ psi)

        # central second differences at h and h/2, Richardson-extrapolated: O(h^4)
        def d2(h):
            return (energy(h) - 2 * energy(0.0) + energy(-h)) / (h * h)
        h = 2e-3
        hess = (4 * d2(h / 2) - d2(h)) / 3
        want = 2 * (a @ Ht @ a + a @ W @ a)
        assert abs(hess - want) < 1e-6 * abs(want)


def test_w_is_chart_independent_at_the_stationary_point(truncated):
    _, tg, _ = truncated
    grad = np.linalg.norm(tg.U.T @ tg.g)          # <T|H - E0|Psi_0> over the tangent space
    assert grad < 1e-6
    Ht = rpa.h_tangent(tg)
    Wp = rpa.w_paper(tg)
    assert np.abs(Wp).max() > 0.1                 # a truncated reference: W does not vanish
    wp = rpa.rpa_omega(Ht, Wp)
    for c in range(tg.k):
        Wc = rpa.w_chart(tg, c)
        assert np.abs(Wc - Wp).max() < 10 * grad
        assert np.abs(rpa.rpa_omega(Ht, Wc) - wp).max() < 10 * grad


def test_rpa_pairs_and_thouless_bound(truncated):
    H, tg, (L0, R0, C0, Lam) = truncated
    Ht = rpa.h_tangent(tg)
    Wp = rpa.w_paper(tg)
    w = rpa.rpa_omega(Ht, Wp)
    ev, n = rpa.rpa_full(Ht, Wp)
    assert np.abs(ev.imag).max() < 1e-10
    assert np.abs(np.sort(ev.real)[n:] - w).max() < 1e-10       # the positive branch
    assert np.abs(np.sort(ev.real)[:n] + w[::-1]).max() < 1e-10   # mirrored by -omega
    # TDA limit (W = 0) is the tangent-space Rayleigh-Ritz
    theta, E0, dim = tda.tangent_rr(H, L0, R0, C0, Lam, tg.U.shape[1])
    assert dim == tg.U.shape[1] and abs(E0 - tg.E0) < 1e-12
    w_tda = np.linalg.eigvalsh(Ht)
    assert np.abs(w_tda - (theta - E0)).max() < 1e-12
    assert w[0] <= w_tda[0] + 1e-12
    assert w_tda[0] - w[0] > 1e-3                 # strictly lower here: the bound is not vacuous


def test_w_by_the_sweep_equals_the_pairwise_form(truncated):
    H, tg, (L0, R0, C0, Lam) = truncated
    t, v = fock.spin_integrals(H.h, H.eri)
    A = np.random.default_rng(2).standard_normal((tg.U.shape[1], 5))
    Ws = rpa.w_sweep(H, t, v, L0, R0, C0, Lam, tg.U @ A, tg)
    want = A.T @ rpa.w_paper(tg) @ A
    assert np.abs(want).max() > 1.0
    assert np.abs(Ws - want).max() < 1e-12 * np.abs(want).max()


def test_w_action_by_the_sweep_is_the_dense_product(truncated):
    H, tg, (L0, R0, C0, Lam) = truncated
    t, v = fock.spin_integrals(H.h, H.eri)
    Wp = rpa.w_paper(tg)
    rng = np.random.default_rng(5)
    for _ in range(2):
        c = rng.standard_normal(tg.U.shape[1])
        w = rpa.w_action(H, t, v, L0, R0, C0, Lam, tg.U @ c, tg)
        assert np.linalg.norm(w - tg.U @ (tg.U.T @ w)) < 1e-12     # W y lies in the tangent space
        assert np.abs(tg.U.T @ w - Wp @ c).max() < 1e-12 * np.abs(Wp @ c).max()


def test_exact_bond_dimension_gives_fci():
    k, na, nb = 4, 2, 2
    H, (L0, R0, C0, Lam, _) = _reference(k, na, nb, 16)
    tg = rpa.Tangent(H, L0, R0, C0, Lam)
    Ht = rpa.h_tangent(tg)
    Wp = rpa.w_paper(tg)
    assert np.abs(Wp).max() < 1e-10               # Psi_0 is an eigenstate: (H - E0) Psi_0 = 0
    w = rpa.rpa_omega(Ht, Wp)
    e = fock.fci_energies(H.h, H.eri, H.e_core, k, na, nb, 6)
    assert abs(tg.E0 - e[0]) < 1e-10
    assert np.abs(w[:5] - (e[1:6] - e[0])).max() < 1e-8
    assert np.abs(w - np.linalg.eigvalsh(Ht)).max() < 1e-9
    # the one-call wrapper, by both routes
    for route in ("paper", "chart"):
        w_r, w_t, e0 = rpa.rpa_roots(H, L0, R0, C0, Lam, 3, route=route)
        assert abs(e0 - e[0]) < 1e-10
        assert np.abs(w_r - (e[1:4] - e[0])).max() < 1e-8 and np.abs(w_t - w_r).max() < 1e-9


def test_reduced_rpa_davidson_reaches_the_dense_roots(truncated):
    # Eq. reducedrpa on paired trial vectors: the iteration converges to the lowest roots of
    # the full problem, with Ritz pairs normalized to X.X - Y.Y = 1 that solve Eq. dmrgrpa
    _, tg, _ = truncated
    Ht = rpa.h_tangent(tg)
    Wp = rpa.w_paper(tg)
    w = rpa.rpa_omega(Ht, Wp)
    om_, X, Y, it = rpa.davidson_rpa(Ht, Wp, 4, tol=1e-10, max_space=12)
    assert it < 200
    assert np.abs(om_ - w[:4]).max() < 1e-10
    assert np.abs(np.einsum("ij,ij->j", X, X) - np.einsum("ij,ij->j", Y, Y) - 1.0).max() < 1e-10
    assert np.abs(Ht @ X + Wp @ Y - X * om_).max() < 1e-9
    assert np.abs(Wp @ X + Ht @ Y + Y * om_).max() < 1e-9
    # the partners (Y, X) are the -omega solutions
    assert np.abs(Ht @ Y + Wp @ X - Y * (-om_)).max() < 1e-9
    # on the trial space of a solution and its partner the reduced problem is exact
    om1, aX, aY = rpa.reduced_rpa(Ht, Wp, X[:, :1], Y[:, :1])
    assert abs(om1[0] - om_[0]) < 1e-10 and abs(abs(aX[0, 0]) - 1.0) < 1e-9 and abs(aY[0, 0]) < 1e-9
