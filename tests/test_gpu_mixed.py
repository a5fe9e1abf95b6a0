"""Split-TF32 tensor-core sigma (LRT_MIXED) against the FP64 sigma (GPU)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# 3xTF32 products of FP32-rounded operands, FP32 accumulation inside one block
# product and compensated FP32 sums across products: observed 3e-7..2e-6 of max|y|.
MIXED_RTOL = 1e-5


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_1646_gb300 import build
    build.build()
    import paper_1311_1646_gb300 as p
    p.load()
    return p


def _ctx(pkg, H, M, i, nsite, seed):
    m = synth.mixed_mps(H.k, H.n_alpha, H.n_beta, M, seed, center=i)
    ctx = pkg.Context(0)
    ctx.op_build(H.k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, i)
    for b in range(i):
        ctx.renormalize(b, +1)
    for b in range(H.k - 1, i + nsite - 1, -1):
        ctx.renormalize(b, -1)
    return ctx


def _both(pkg, ctx, i, nsite, nvec, seed):
    n, _ = ctx.wfn_layout(i, nsite)
    x = torch.tensor(synth.random_vector(nvec * n, seed), dtype=torch.float64, device="cuda:0")
    y64 = torch.full_like(x, np.nan)
    ymx = torch.full_like(x, np.nan)
    ctx.sigma(i, nsite, x, y64, nvec=nvec, precision=pkg.LRT_FP64)
    ctx.sigma(i, nsite, x, ymx, nvec=nvec, precision=pkg.LRT_MIXED)
    torch.cuda.synchronize()
    return y64.cpu().numpy(), ymx.cpu().numpy()


@pytest.mark.parametrize("nsite", [1, 2])
def test_mixed_sigma_small_all_sites(pkg, nsite):
    H = synth.ab_initio(6, 3, 3, 21)
    for i in range(6 - nsite + 1):
        ctx = _ctx(pkg, H, 20, i, nsite, 31 + i)
        a, b = _both(pkg, ctx, i, nsite, 2, 41 + i)
        assert np.all(np.isfinite(b))
        assert np.abs(a - b).max() <= MIXED_RTOL * np.abs(a).max(), (i, np.abs(a - b).max() / np.abs(a).max())
        ctx.close()


@pytest.mark.parametrize("cfg,i,nsite,nvec", [(1, 3, 2, 3), (2, 5, 2, 6), (3, 11, 1, 2)])
def test_mixed_sigma_workloads(pkg, cfg, i, nsite, nvec):
    c = synth.config(cfg)
    ctx = _ctx(pkg, c["ham"], c["M"], i, nsite, 300 + cfg)
    a, b = _both(pkg, ctx, i, nsite, nvec, 7)
    err = np.abs(a - b).max() / np.abs(a).max()
    assert np.all(np.isfinite(b))
    print(f"mixed sigma config {cfg}: max-abs relative error {err:.2e}")
    assert err <= MIXED_RTOL, err
    ctx.close()


@pytest.mark.parametrize("cfg,i,nsite", [(1, 3, 2), (2, 5, 2)])
def test_mixed_renormalize(pkg, cfg, i, nsite):
    """Every block renormalized with split-TF32 products (LRT_MIXED); the FP64 sigma on
    those blocks against the all-FP64 one.  Each renormalization adds its own rounding,
    so the bound is looser than for one sigma call."""
    c = synth.config(cfg)
    H = c["ham"]
    m = synth.mixed_mps(H.k, H.n_alpha, H.n_beta, c["M"], 400 + cfg, center=i)
    out = []
    for prec in (pkg.LRT_FP64, pkg.LRT_MIXED):
        ctx = pkg.Context(0)
        ctx.op_build(H.k, H.h, H.eri, e_core=H.e_core)
        ctx.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, i)
        for b in range(i):
            ctx.renormalize(b, +1, prec)
        for b in range(H.k - 1, i + nsite - 1, -1):
            ctx.renormalize(b, -1, prec)
        n, _ = ctx.wfn_layout(i, nsite)
        x = torch.tensor(synth.random_vector(n, 8), dtype=torch.float64, device="cuda:0")
        y = torch.empty_like(x)
        ctx.sigma(i, nsite, x, y)
        out.append(y.cpu().numpy())
        ctx.close()
    err = np.abs(out[0] - out[1]).max() / np.abs(out[0]).max()
    print(f"mixed renormalize config {cfg}: max-abs relative error of sigma {err:.2e}")
    assert err <= 5e-5, err
