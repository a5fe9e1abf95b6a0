"""Pins of the oracle's frequency-dependent linear response (oracle/response.py; Eqs. pt_ext,
realresp, imagresp, psi1st).

* At the exact bond dimension the TDA and RPA responses are the exact response function of
  the sector's ground state (a sum over its FCI excited states).
* The linear-system responses equal their sum-over-states forms built from the TDA and RPA
  eigenpairs (the amplitudes normalized to X.X - Y.Y = 1 and solving Eq. dmrgrpa).
* The static RPA response is the curvature of the variational energy: one-site DMRG at
  fixed bond dimension with h + lambda d, second differences extrapolated in the step.
* The paper's site equations (Eqs. realresp, imagresp), solved site by site in sweeps,
  reach the dense tangent-space solution.
"""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import dmrg, fock, response, rpa
from oracle import mps as om


def _reference(k, na, nb, M, seed=7):
    H = synth.ab_initio(k, na, nb, seed)
    t, v = fock.spin_integrals(H.h, H.eri)
    E, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(k, na, nb, M, 3))
    E, sites, _ = dmrg.onesite_sweeps(H, t, v, sites, n_sweeps=40, dav_tol=1e-13, e_tol=1e-14)
    return H, om.mixed_canonical(sites)


def _perturbation(k, seed=11):
    d = np.random.default_rng(seed).standard_normal((k, k))
    return 0.5 * (d + d.T)


def test_exact_bond_dimension_response_is_exact():
    H, (L0, R0, C0, Lam, _) = _reference(4, 2, 2, 16)
    tg = rpa.Tangent(H, L0, R0, C0, Lam)
    d = _perturbation(4)
    v = response.drive(tg, d)
    Ht, Wp = rpa.h_tangent(tg), rpa.w_paper(tg)
    w1 = np.linalg.eigvalsh(Ht)[0]
    ws = np.array([0.0, 0.3 * w1, 0.9 * w1, 1.1 * w1])    # below and above the first pole
    exact = response.alpha_exact(H, d, ws)
    assert np.abs(response.alpha_tda(Ht, v, ws) - exact).max() < 1e-8 * np.abs(exact).max()
    assert np.abs(response.alpha_rpa(Ht, Wp, v, ws) - exact).max() < 1e-8 * np.abs(exact).max()


def test_linear_response_equals_its_sum_over_states(stationary_k5):
    H, (L0, R0, C0, Lam, _) = stationary_k5
    tg = rpa.Tangent(H, L0, R0, C0, Lam)
    v = response.drive(tg, _perturbation(H.k))
    Ht, Wp = rpa.h_tangent(tg), rpa.w_paper(tg)
    om_, X, Y = response.rpa_modes(Ht, Wp)
    assert np.abs(om_ - rpa.rpa_omega(Ht, Wp)).max() < 1e-10
    assert np.abs(np.einsum("ij,ij->j", X, X) - np.einsum("ij,ij->j", Y, Y) - 1.0).max() < 1e-10
    assert np.abs(Ht @ X + Wp @ Y - X * om_).max() < 1e-9
    assert np.abs(Wp @ X + Ht @ Y + Y * om_).max() < 1e-9
    # the Davidson's lowest amplitudes are the same modes (up to sign)
    _, Xd, Yd, _ = rpa.davidson_rpa(Ht, Wp, 3, tol=1e-10, max_space=12)
    for j in range(3):
        s = np.sign((X[:, j] + Y[:, j]) @ (Xd[:, j] + Yd[:, j]))
        assert np.abs(s * (Xd[:, j] + Yd[:, j]) - (X[:, j] + Y[:, j])).max() < 1e-7
    ws = np.array([0.0, 0.5 * om_[0], 0.5 * (om_[0] + om_[1]), 1.7 * om_[2]])
    a = response.alpha_rpa(Ht, Wp, v, ws)
    sos = response.alpha_sum_over_states(om_, (v @ (X + Y)) ** 2, ws)
    assert np.abs(a - sos).max() < 1e-10 * np.abs(a).max()
    et, xt = np.linalg.eigh(Ht)
    a_t = response.alpha_tda(Ht, v, ws)
    assert np.abs(a_t - response.alpha_sum_over_states(et, (v @ xt) ** 2, ws)).max() < 1e-10 * np.abs(a_t).max()
    # a truncated reference: the two levels differ
    assert np.abs(a - a_t).max() > 0.1


def test_static_rpa_response_is_the_variational_energy_curvature():
    k, na, nb = 4, 2, 2
    H, (L0, R0, C0, Lam, _) = _reference(k, na, nb, 3)
    tg = rpa.Tangent(H, L0, R0, C0, Lam)
    assert np.linalg.norm(tg.U.T @ tg.g) < 1e-7             # stationary reference
    d = _perturbation(k)
    v = response.drive(tg, d)
    Ht, Wp = rpa.h_tangent(tg), rpa.w_paper(tg)
    a_rpa = response.alpha_rpa(Ht, Wp, v, [0.0])[0]
    a_tda = response.alpha_tda(Ht, v, [0.0])[0]
    start = [C0[0]] + [R0[i] for i in range(1, k)]          # right-canonical, centre at site 0

    def energy(lam):
        Hl = dataclasses.replace(H, h=H.h + lam * d)
        t, vv = fock.spin_integrals(Hl.h, Hl.eri)
        E, _, _ = dmrg.onesite_sweeps(Hl, t, vv, start, n_sweeps=60, dav_tol=1e-13, e_tol=1e-14)
        return E

    e0 = energy(0.0)
    d2 = {h: (energy(h) - 2 * e0 + energy(-h)) / (h * h) for h in (5e-3, 2.5e-3)}
    curv = (4 * d2[2.5e-3] - d2[5e-3]) / 3
    assert abs(curv - a_rpa) < 1e-6 * abs(a_rpa)
    assert abs(curv - a_tda) > 0.1                          # the TDA level misses it here


def test_site_sweep_solves_the_tangent_space_response(stationary_k5):
    # Eqs. realresp / imagresp solved site by site in sweeps reach the dense tangent-space
    # solution of (H -+ omega) X = -v below the first pole
    H, (L0, R0, C0, Lam, _) = stationary_k5
    tg = rpa.Tangent(H, L0, R0, C0, Lam)
    d = _perturbation(H.k)
    v = response.drive(tg, d)
    Ht = rpa.h_tangent(tg)
    w1 = np.linalg.eigvalsh(Ht)[0]
    n = len(v)
    for w in (0.0, 0.5 * w1):
        for sign in (+1, -1):
            X, sweeps, change = response.site_sweep(tg, d, w, sign, sweeps=60, tol=1e-13)
            assert sweeps < 60 and change < 1e-13
            want = -tg.U @ np.linalg.solve(Ht + sign * w * np.eye(n), v)
            assert np.abs(X - want).max() < 1e-10 * np.abs(want).max()
