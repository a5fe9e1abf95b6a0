"""Ground-state sweeps on the GPU against FCI and the CPU oracle (GPU)."""
import numpy as np
import pytest

import synth
from oracle import dmrg, fock
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


def _gs(pkg, H, M0, schedule, seed=3, **kw):
    m = synth.random_mps(H.k, H.n_alpha, H.n_beta, M0, seed, "right")
    ctx = pkg.Context(0)
    ctx.op_build(H.k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, 0)
    E = ctx.sweep_gs(schedule, **kw)
    bonds, sites = ctx.mps_get()
    ctx.close()
    return E, m, bonds, sites


def _oracle_energy(H, bonds, sites):
    t, v = fock.spin_integrals(H.h, H.eri_full())
    sb = [om.unpack_site(sites[i], bonds[i], bonds[i + 1]) for i in range(H.k)]
    return dmrg.energy(H, t, v, sb)


@pytest.mark.parametrize("k,na,nb,schedule", [(5, 3, 2, [8, 64]), (6, 3, 3, [16, 64]), (6, 2, 3, [16, 64])])
def test_exact_bond_dimension_reaches_fci(pkg, k, na, nb, schedule):
    H = synth.ab_initio(k, na, nb, 7)
    E, m, bonds, sites = _gs(pkg, H, 8, schedule)
    ef = fock.fci_energies(H.h, H.eri, H.e_core, k, na, nb, 1)[0]
    assert abs(E - ef) < 1e-8
    # the MPS left on the device has that energy (evaluated independently by the oracle)
    assert abs(_oracle_energy(H, bonds, sites) - E) < 1e-9


def test_truncated_matches_oracle_dmrg_and_is_variational(pkg):
    k, na, nb, M = 6, 3, 3, 8
    H = synth.ab_initio(k, na, nb, 7)
    E, m, bonds, sites = _gs(pkg, H, M, [M], max_sweeps=20, e_tol=1e-11)
    t, v = fock.spin_integrals(H.h, H.eri)
    Eo, _, _ = dmrg.ground_state(H, t, v, [M], m, e_tol=1e-11)
    ef = fock.fci_energies(H.h, H.eri, H.e_core, k, na, nb, 1)[0]
    assert E >= ef - 1e-10
    assert abs(E - Eo) < 1e-7
    assert max(sum(d for *_, d in b) for b in bonds) <= M


def test_abinitio_k8_exact_at_M256(pkg):
    """The 8-orbital ab initio workload: bond dimension 256 is exact, so E0 = FCI."""
    cfg = synth.config(1)
    H = cfg["ham"]
    E, m, bonds, sites = _gs(pkg, H, 16, [64, 256], max_sweeps=10)
    ef = fock.fci_energies(H.h, H.eri, H.e_core, H.k, H.n_alpha, H.n_beta, 1)[0]
    assert abs(E - ef) < 1e-8
    assert abs(_oracle_energy(H, bonds, sites) - E) < 1e-8


def test_onesite_sweeps_lower_the_energy_and_keep_the_form(pkg):
    """Two-site sweeps at a truncated bond dimension, then one-site sweeps: the energy does
    not rise, it is the energy of the MPS left on the device (evaluated by the oracle), and
    the sites 1..k-1 stay right-orthonormal."""
    k, na, nb, M = 6, 3, 3, 12
    H = synth.ab_initio(k, na, nb, 7)
    E2, m, _, _ = _gs(pkg, H, 8, [M], max_sweeps=6)
    E1, m1, bonds, sites = _gs(pkg, H, 8, [M], max_sweeps=6, onesite_sweeps=3)
    assert E1 <= E2 + 1e-10
    assert abs(_oracle_energy(H, bonds, sites) - E1) < 1e-9
    for i in range(1, k):
        blocks = om.unpack_site(sites[i], bonds[i], bonds[i + 1])
        acc = {}
        for (ql, _n, _qr), a in blocks.items():
            acc[ql] = acc.get(ql, 0) + a @ a.T
        for g in acc.values():
            # rank-deficient sectors keep zero rows; the others are orthonormal
            d = np.diag(g)
            assert np.all((np.abs(d - 1.0) < 1e-10) | (np.abs(d) < 1e-10))


def test_mps_save_round_trip(pkg):
    """mps_save returns the loaded MPS (both forms) in mps_load's layout, and loading the
    saved copy reproduces sigma exactly."""
    k, na, nb, M, i = 6, 3, 3, 12, 2
    H = synth.ab_initio(k, na, nb, 5)
    left = synth.random_mps(k, na, nb, M, 61, "left")
    right = synth.random_mps(k, na, nb, M, 62, "right")
    ctx = pkg.Context(0)
    ctx.op_build(k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(k, na, nb, left.bonds, left.sites, 0, sites_right=right.sites)
    out = ctx.mps_save()
    assert (out["k"], out["n_alpha"], out["n_beta"]) == (k, na, nb)
    assert [list(map(tuple, b)) for b in out["bonds"]] == [list(map(tuple, b)) for b in left.bonds]
    for j in range(k):
        assert np.array_equal(out["sites"][j], np.asarray(left.sites[j]))
        assert np.array_equal(out["sites_right"][j], np.asarray(right.sites[j]))
    copy = pkg.Context(0)
    copy.op_build(k, H.h, H.eri, e_core=H.e_core)
    copy.mps_load(k, na, nb, out["bonds"], out["sites"], 0, sites_right=out["sites_right"])
    ys = []
    for c in (ctx, copy):
        for b in range(i):
            c.renormalize(b, +1)
        for b in range(k - 1, i, -1):
            c.renormalize(b, -1)
        n, _ = c.wfn_layout(i, 1)
        x = torch.tensor(synth.random_vector(n, 8), dtype=torch.float64, device="cuda:0")
        y = torch.empty_like(x)
        c.sigma(i, 1, x, y)
        torch.cuda.synchronize()
        ys.append(y.cpu().numpy())
        c.close()
    assert np.array_equal(ys[0], ys[1])
