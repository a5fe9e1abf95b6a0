"""Frequency-dependent linear response at the Tamm-Dancoff level on the GPU (GPU).

sweep_response solves the site equations of Eqs. realresp and imagresp in sweeps and
returns alpha(omega) = <V Psi0|X> + <V Psi0|Y> for a one-body perturbation V = sum d_pq E_pq.
Its definition is the dense solve in the orthonormal tangent basis of the same reference
(`oracle.response.alpha_tda` on `oracle.rpa.h_tangent` and `oracle.response.drive`:
X = -(H - omega)^-1 v, Y = -(H + omega)^-1 v), and at the exact bond dimension the exact
response of the FCI ground state (a sum over its excited states).  Two solvers, the site
iteration and the subspace form, at frequencies below the first pole.  The reference is the
oracle's stationary one-site DMRG state, loaded into both contexts (H and V) with tda_load.

Bar: the site residuals are driven to sum |r|^2 < 1e-22, so the components carry errors
of about 1e-11 / (distance to the pole); 1e-8 of |alpha| covers that with margin.
"""
import numpy as np
import pytest

import synth
from oracle import dmrg, fock, response, rpa
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


def _stationary(H, M):
    t, v = fock.spin_integrals(H.h, H.eri)
    _, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(H.k, H.n_alpha, H.n_beta, M, 3))
    _, sites, _ = dmrg.onesite_sweeps(H, t, v, sites, n_sweeps=40, dav_tol=1e-13, e_tol=1e-14)
    return om.mixed_canonical(sites)


def _perturbation(k, seed=11):
    d = np.random.default_rng(seed).standard_normal((k, k))
    return 0.5 * (d + d.T)


def _context(pkg, H, ref, h, eri, e_core):
    """A context holding the one-body h (and eri, or none) on the reference `ref`."""
    L0, R0, C0, Lam, _ = ref
    k = H.k
    tables = [[(q[0], q[1], len(Lam[b][q])) for q in sorted(Lam[b])] for b in range(k + 1)]
    L = [om.pack_site(L0[i], tables[i], tables[i + 1]) for i in range(k)]
    R = [om.pack_site(R0[i], tables[i], tables[i + 1]) for i in range(k)]
    C = [om.pack_site(C0[i], tables[i], tables[i + 1]) for i in range(k)]
    lam = [np.concatenate([Lam[b][q] for q in sorted(Lam[b])]) for b in range(k + 1)]
    ctx = pkg.Context(0)
    ctx.op_build(k, h, eri, e_core=e_core)
    ctx.mps_load(k, H.n_alpha, H.n_beta, tables, L, 0, sites_right=R)
    ctx.tda_load(C, lam)
    return ctx


@pytest.mark.parametrize("k,na,nb,M", [(5, 3, 2, 10), (6, 3, 3, 12)])
def test_response_matches_the_tangent_space_solve(pkg, k, na, nb, M):
    """Both solvers, below the first pole."""
    H = synth.ab_initio(k, na, nb, 7)
    ref = _stationary(H, M)
    L0, R0, C0, Lam, _ = ref
    tg = rpa.Tangent(H, L0, R0, C0, Lam)
    d = _perturbation(k)
    v = response.drive(tg, d)
    Ht = rpa.h_tangent(tg)
    w1 = np.linalg.eigvalsh(Ht)[0]
    ctx = _context(pkg, H, ref, H.h, H.eri, H.e_core)
    vctx = _context(pkg, H, ref, d, None, 0.0)
    cases = [(pkg.LRT_RESP_SITE, 0.0), (pkg.LRT_RESP_SITE, 0.5 * w1), (pkg.LRT_RESP_SUBSPACE, 0.0),
             (pkg.LRT_RESP_SUBSPACE, 0.5 * w1)]
    for method, w in cases:
        a_ref = response.alpha_tda(Ht, v, [w])[0]
        # the subspace form measures its residual on the sweep's site pieces, which settle at
        # the floor the TDA's do (about 1e-11 to 1e-10 here); alpha, a Galerkin value, is
        # second order in that residual
        tol = 1e-22 if method == pkg.LRT_RESP_SITE else 1e-9
        a, res, sw = ctx.sweep_response(vctx, w, tol=tol, max_sweeps=100, method=method, max_space=48)
        assert np.all(res < tol), (method, w, res, sw)
        assert abs(a - a_ref) < 1e-8 * abs(a_ref), (method, w, a, a_ref)
    ctx.close()
    vctx.close()


def test_response_at_the_exact_bond_dimension_is_the_exact_response(pkg):
    """At the exact bond dimension the tangent space holds every excited state of the sector,
    and alpha(omega) is the exact sum over the FCI excited states."""
    k, na, nb, M = 4, 2, 2, 16
    H = synth.ab_initio(k, na, nb, 7)
    ref = _stationary(H, M)
    L0, R0, C0, Lam, _ = ref
    tg = rpa.Tangent(H, L0, R0, C0, Lam)
    d = _perturbation(k)
    w1 = np.linalg.eigvalsh(rpa.h_tangent(tg))[0]
    ws = np.array([0.0, 0.6 * w1])
    exact = response.alpha_exact(H, d, ws)
    ctx = _context(pkg, H, ref, H.h, H.eri, H.e_core)
    vctx = _context(pkg, H, ref, d, None, 0.0)
    for w, a_ref in zip(ws, exact):
        a, res, _ = ctx.sweep_response(vctx, w, tol=1e-22, max_sweeps=80)
        assert abs(a - a_ref) < 1e-8 * abs(a_ref), (w, a, a_ref)
    ctx.close()
    vctx.close()


def test_response_rejects_different_references(pkg):
    """The perturbation's context must hold the same reference (checked bit for bit)."""
    H = synth.ab_initio(5, 3, 2, 7)
    ref = _stationary(H, 10)
    ref2 = _stationary(synth.ab_initio(5, 3, 2, 8), 10)
    ctx = _context(pkg, H, ref, H.h, H.eri, H.e_core)
    vctx = _context(pkg, H, ref2, _perturbation(5), None, 0.0)
    with pytest.raises(pkg.LrtError):
        ctx.sweep_response(vctx, 0.1)
    ctx.close()
    vctx.close()
