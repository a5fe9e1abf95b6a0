"""Degenerate and extreme shapes of the sigma path (GPU): the whole system as one two-site
tensor, full filling, the vacuum, a single electron, and many right-hand sides at once.
H_eff is assembled column by column through sigma (nvec = dimension), so every case is
pinned by what the method fixes: H_eff symmetric and, where the MPS basis is complete, its
lowest eigenvalue the FCI ground-state energy."""
import numpy as np
import pytest

import synth
from oracle import fock

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


def _context(pkg, H, M, i, nsite):
    m = synth.mixed_mps(H.k, H.n_alpha, H.n_beta, M, 5, center=i)
    ctx = pkg.Context(0)
    ctx.op_build(H.k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, i)
    for b in range(i):
        ctx.renormalize(b, +1)
    for b in range(H.k - 1, i + nsite - 1, -1):
        ctx.renormalize(b, -1)
    return ctx


def _dense(pkg, ctx, i, nsite, precision):
    n, _ = ctx.wfn_layout(i, nsite)
    x = torch.eye(n, dtype=torch.float64, device="cuda:0").reshape(-1).contiguous()
    y = torch.full_like(x, float("nan"))
    ctx.sigma(i, nsite, x, y, nvec=n, precision=precision)
    torch.cuda.synchronize()
    return y.cpu().numpy().reshape(n, n)


# (k, n_alpha, n_beta, M, site, nsite): M at least the exact bond dimension
CASES = [
    (2, 1, 1, 4, 0, 2),     # the whole system is one two-site tensor
    (3, 3, 3, 4, 1, 1),     # full filling: one determinant
    (3, 0, 0, 4, 1, 1),     # the vacuum: H_eff = e_core
    (4, 1, 0, 8, 1, 2),     # one electron: the spectrum of h
    (3, 2, 1, 16, 0, 2),    # odd electron count, whole-space bonds
    (5, 2, 3, 64, 2, 1),    # exact bonds, one-site
]


@pytest.mark.parametrize("k,na,nb,M,i,nsite", CASES)
def test_dense_heff_is_symmetric_and_reaches_fci(pkg, k, na, nb, M, i, nsite):
    H = synth.ab_initio(k, na, nb, 3)
    ctx = _context(pkg, H, M, i, nsite)
    A = _dense(pkg, ctx, i, nsite, pkg.LRT_FP64)
    assert np.all(np.isfinite(A))
    assert np.abs(A - A.T).max() <= 1e-12 * max(1.0, np.abs(A).max())
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    ef = fock.fci_energies(H.h, H.eri, H.e_core, k, na, nb, 1)[0]
    assert abs(ev[0] - ef) < 1e-9
    if na + nb == 0:
        assert np.allclose(A, H.e_core * np.eye(A.shape[0]), atol=1e-12)
    if (na, nb) == (1, 0):
        assert abs(ev[0] - (np.linalg.eigvalsh(H.h)[0] + H.e_core)) < 1e-9
    # the split-TF32 path on the same shapes
    B = _dense(pkg, ctx, i, nsite, pkg.LRT_MIXED)
    assert np.abs(B - A).max() <= 1e-5 * max(1.0, np.abs(A).max())
    ctx.close()


def test_many_right_hand_sides_match_one_at_a_time(pkg):
    H = synth.ab_initio(6, 3, 3, 9)
    i, nsite, nvec = 2, 2, 40
    ctx = _context(pkg, H, 20, i, nsite)
    n, _ = ctx.wfn_layout(i, nsite)
    X = torch.tensor(synth.random_vector(n * nvec, 17), dtype=torch.float64, device="cuda:0")
    Y = torch.empty_like(X)
    ctx.sigma(i, nsite, X, Y, nvec=nvec)
    for v in (0, 17, nvec - 1):
        y1 = torch.empty(n, dtype=torch.float64, device="cuda:0")
        ctx.sigma(i, nsite, X[v * n:(v + 1) * n].contiguous(), y1)
        assert float((Y[v * n:(v + 1) * n] - y1).abs().max() / y1.abs().max()) <= 1e-14
    ctx.close()


def test_sigma_on_a_second_device_matches_the_first(pkg):
    """Kernel attributes (dynamic shared memory above 48 KB) are per device: a context on
    device 1 after one on device 0 runs the same FP64 and mixed sigma, to rounding."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one visible device")
    H = synth.ab_initio(6, 3, 3, 9)
    out = []
    for dev in (0, 1):
        m = synth.mixed_mps(H.k, H.n_alpha, H.n_beta, 16, 5, center=2)
        ctx = pkg.Context(dev)
        ctx.op_build(H.k, H.h, H.eri, e_core=H.e_core)
        ctx.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, 2)
        for b in range(2):
            ctx.renormalize(b, +1)
        for b in range(H.k - 1, 2, -1):
            ctx.renormalize(b, -1)
        n, _ = ctx.wfn_layout(2, 1)
        x = torch.tensor(synth.random_vector(n, 3), dtype=torch.float64, device=f"cuda:{dev}")
        ys = []
        for prec in (pkg.LRT_FP64, pkg.LRT_MIXED):
            y = torch.empty_like(x)
            ctx.sigma(2, 1, x, y, precision=prec)
            torch.cuda.synchronize(dev)
            ys.append(y.cpu().numpy())
        ctx.close()
        out.append(ys)
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-12 * np.abs(out[0][0]).max()
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-5 * np.abs(out[0][1]).max()
