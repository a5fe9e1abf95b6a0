"""DMRG-TDA sweep on the GPU against the tangent-space definition, the oracle's sweep and FCI (GPU).

The zeroth-order reference (two-site then one-site sweeps, mixed-canonical gauge)
is produced by the CPU oracle from seeded inputs and handed to both sides.
"""
import numpy as np
import pytest

import synth
from oracle import dmrg, fock
from oracle import mps as om
from oracle import tda

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


def _reference(k, na, nb, M, seed=7):
    H = synth.ab_initio(k, na, nb, seed)
    t, v = fock.spin_integrals(H.h, H.eri)
    E, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(k, na, nb, M, 3))
    E, sites, _ = dmrg.onesite_sweeps(H, t, v, sites)
    return H, t, v, om.mixed_canonical(sites)


def _gpu_tda(pkg, H, ref, nroots, **kw):
    L0, R0, C0, Lam, _ = ref
    k = H.k
    tables = [[(q[0], q[1], len(Lam[b][q])) for q in sorted(Lam[b])] for b in range(k + 1)]
    L = [om.pack_site(L0[i], tables[i], tables[i + 1]) for i in range(k)]
    R = [om.pack_site(R0[i], tables[i], tables[i + 1]) for i in range(k)]
    C = [om.pack_site(C0[i], tables[i], tables[i + 1]) for i in range(k)]
    lam = [np.concatenate([Lam[b][q] for q in sorted(Lam[b])]) for b in range(k + 1)]
    ctx = pkg.Context(0)
    ctx.op_build(k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(k, H.n_alpha, H.n_beta, tables, L, 0, sites_right=R)
    ctx.tda_load(C, lam)
    out = ctx.sweep_tda(nroots, **kw)
    ctx.close()
    return out


def test_tda_matches_tangent_space_definition_and_oracle_sweep(pkg):
    k, na, nb, M, n = 4, 2, 2, 8, 2
    H, t, v, ref = _reference(k, na, nb, M)
    L0, R0, C0, Lam, _ = ref
    w, E0, dim = tda.tangent_rr(H, L0, R0, C0, Lam, n)
    omega, resid, e0 = _gpu_tda(pkg, H, ref, n, max_iter=40, eps=1e-13, allow_noconv=True)
    assert abs(e0 - E0) < 1e-10
    assert np.abs(omega + e0 - w).max() < 1e-7
    th, E0s, r2, it = tda.sweep_tda(H, t, v, L0, R0, C0, Lam, n, eps=1e-13, max_iter=40)
    assert np.abs(omega + e0 - th).max() < 1e-7
    assert np.all(resid < 1e-6)
    ef = fock.fci_energies(H.h, H.eri, H.e_core, k, na, nb, n + 1)
    assert np.all(omega + e0 >= ef[1:n + 1] - 1e-9)     # Rayleigh-Ritz in a subspace


def test_tda_on_the_full_space_gives_fci_excitations(pkg):
    k, na, nb, M, n = 4, 2, 2, 16, 3
    H, t, v, ref = _reference(k, na, nb, M)
    ef = fock.fci_energies(H.h, H.eri, H.e_core, k, na, nb, n + 1)
    omega, resid, e0 = _gpu_tda(pkg, H, ref, n, max_iter=40, eps=1e-13, allow_noconv=True)
    assert abs(e0 - ef[0]) < 1e-9
    assert np.abs(omega - (ef[1:] - ef[0])).max() < 1e-7


def test_tda_odd_electrons(pkg):
    k, na, nb, M, n = 5, 3, 2, 10, 2
    H, t, v, ref = _reference(k, na, nb, M)
    L0, R0, C0, Lam, _ = ref
    w, E0, dim = tda.tangent_rr(H, L0, R0, C0, Lam, n)
    omega, resid, e0 = _gpu_tda(pkg, H, ref, n, max_iter=40, eps=1e-13, allow_noconv=True)
    assert np.abs(omega + e0 - w).max() < 1e-6


def _right_form(k, sites):
    """The oracle's right-orthonormal form (centre on site 0) with its bond tables, packed."""
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


def _prepared(pkg, H, sites):
    tables, Rp = _right_form(H.k, sites)
    ctx = pkg.Context(0)
    ctx.op_build(H.k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(H.k, H.n_alpha, H.n_beta, tables, Rp, 0)
    ctx.tda_prepare()
    return ctx


def test_tda_prepare_gauge_matches_tangent_space_definition(pkg):
    """Mixed-canonical gauge built on the GPU (tda_prepare) instead of the oracle's."""
    k, na, nb, M, n = 5, 3, 2, 10, 2
    H = synth.ab_initio(k, na, nb, 7)
    t, v = fock.spin_integrals(H.h, H.eri)
    E, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(k, na, nb, M, 3))
    E, sites, _ = dmrg.onesite_sweeps(H, t, v, sites)
    L0, R0, C0, Lam, _ = om.mixed_canonical(sites)
    w, E0, dim = tda.tangent_rr(H, L0, R0, C0, Lam, n)
    ctx = _prepared(pkg, H, sites)
    omega, resid, e0 = ctx.sweep_tda(n, max_iter=40, eps=1e-13, allow_noconv=True)
    ctx.close()
    assert abs(e0 - E0) < 1e-10
    assert np.abs(omega + e0 - w).max() < 1e-6


def test_tda_mixed_precision_matches_fp64(pkg):
    """Split-TF32 site products with the FP64 residual correction: the roots agree with the
    FP64 sweep to 1e-6 Eh."""
    k, na, nb, M, n = 5, 3, 2, 10, 2
    H = synth.ab_initio(k, na, nb, 7)
    t, v = fock.spin_integrals(H.h, H.eri)
    E, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(k, na, nb, M, 3))
    E, sites, _ = dmrg.onesite_sweeps(H, t, v, sites)
    L0, R0, C0, Lam, _ = om.mixed_canonical(sites)
    w, E0, dim = tda.tangent_rr(H, L0, R0, C0, Lam, n)
    out = {}
    for prec in (pkg.LRT_FP64, pkg.LRT_MIXED):
        ctx = _prepared(pkg, H, sites)
        out[prec] = ctx.sweep_tda(n, max_iter=40, eps=1e-13, allow_noconv=True, precision=prec)
        ctx.close()
    (w64, r64, e64), (wmx, rmx, emx) = out[pkg.LRT_FP64], out[pkg.LRT_MIXED]
    assert abs(e64 - emx) < 1e-12          # the reference energy is FP64 in both
    assert np.abs(w64 - wmx).max() < 1e-6
    assert np.abs(wmx + emx - w).max() < 1e-6


def test_gpu_ground_state_then_tda_is_variational(pkg):
    """The whole path on the GPU: sweep_gs, tda_prepare, sweep_tda on the 8-orbital ab
    initio workload (bond dimension 64); the TDA roots lie at or above the FCI roots."""
    cfg = synth.config(1)
    H = cfg["ham"]
    m = synth.random_mps(H.k, H.n_alpha, H.n_beta, 16, 3, "right")
    ctx = pkg.Context(0)
    ctx.op_build(H.k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, 0)
    E = ctx.sweep_gs([32, cfg["M"]], max_sweeps=8)
    ctx.tda_prepare()
    n = cfg["nroots"]
    omega, resid, e0 = ctx.sweep_tda(n, max_iter=30, eps=1e-10, allow_noconv=True)
    ctx.close()
    ef = fock.fci_energies(H.h, H.eri, H.e_core, H.k, H.n_alpha, H.n_beta, n + 1)
    assert abs(e0 - E) < 1e-7
    assert e0 >= ef[0] - 1e-9
    assert np.all(omega + e0 >= ef[1:n + 1] - 1e-8)


def test_tda_batched_matches_each_instance_alone(pkg):
    """sweep_tda_batched runs several independent instances concurrently (host threads,
    one stream per context); each instance's roots equal those of its own sweep_tda."""
    cases = [(5, 3, 2, 10, 11), (6, 3, 3, 12, 12), (5, 2, 2, 8, 13)]
    refs, ctxs, streams = [], [], []
    for k, na, nb, M, seed in cases:
        H = synth.ab_initio(k, na, nb, seed)
        t, v = fock.spin_integrals(H.h, H.eri)
        E, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(k, na, nb, M, 3))
        E, sites, _ = dmrg.onesite_sweeps(H, t, v, sites)
        alone = _prepared(pkg, H, sites)
        refs.append(alone.sweep_tda(2, max_iter=8, eps=1e-13, seed=0, allow_noconv=True))
        alone.close()
        tables, Rp = _right_form(H.k, sites)
        streams.append(torch.cuda.Stream())
        ctx = pkg.Context(0, stream=streams[-1].cuda_stream)
        ctx.op_build(H.k, H.h, H.eri, e_core=H.e_core)
        ctx.mps_load(H.k, H.n_alpha, H.n_beta, tables, Rp, 0)
        ctx.tda_prepare()
        ctxs.append(ctx)
    torch.cuda.synchronize()
    omega, resid, e0 = pkg.sweep_tda_batched(ctxs, 2, max_iter=8, eps=1e-13, seed=0, allow_noconv=True)
    for c in ctxs:
        c.close()
    for j, (w, r, e) in enumerate(refs):
        assert abs(e0[j] - e) < 1e-12
        assert np.abs(omega[j] - w).max() < 1e-10
        assert np.abs(resid[j] - r).max() <= 1e-10 * max(1.0, np.abs(r).max())
