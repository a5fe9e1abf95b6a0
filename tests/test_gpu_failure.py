"""Failure detection of the tensor-core kernels (GPU), without a GPU fault.

Every pipeline wait of the split-TF32 kernels gives up after a time limit: the CTA raises
a flag, lets its copies and products in flight finish, releases its tensor memory and
returns, and the call reports LRT_ETIMEOUT.  A test hook makes one CTA of the next launch
wait on a barrier that nothing completes (a flag nobody sets) under a 20 ms limit; the
test checks the status and that the same context then computes correctly."""
import numpy as np
import pytest

import synth

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


def test_expired_wait_returns_etimeout_and_the_context_stays_usable(pkg):
    cfg = synth.config(1)
    H = cfg["ham"]
    i = 3
    m = synth.mixed_mps(H.k, H.n_alpha, H.n_beta, cfg["M"], 31, center=i)
    ctx = pkg.Context(0)
    ctx.op_build(H.k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, i)
    for b in range(i):
        ctx.renormalize(b, +1)
    for b in range(H.k - 1, i, -1):
        ctx.renormalize(b, -1)
    n, _ = ctx.wfn_layout(i, 1)
    x = torch.tensor(synth.random_vector(2 * n, 41), dtype=torch.float64, device="cuda:0")
    y64 = torch.empty_like(x)
    ymx = torch.empty_like(x)
    ctx.sigma(i, 1, x, y64, nvec=2)
    ctx.sigma(i, 1, x, ymx, nvec=2, precision=pkg.LRT_MIXED)       # plans and tunes the kernels
    torch.cuda.synchronize()
    ref = y64.cpu().numpy()
    err0 = np.abs(ymx.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err0 < 1e-5
    ctx.set_wait_limit(0.02, stall_next=True)
    with pytest.raises(pkg.LrtError, match=r"\(-5\)"):
        ctx.sigma(i, 1, x, ymx, nvec=2, precision=pkg.LRT_MIXED)
    # the hook cleared itself: the next launches run normally, under the short limit too
    ymx.fill_(np.nan)
    ctx.sigma(i, 1, x, ymx, nvec=2, precision=pkg.LRT_MIXED)
    torch.cuda.synchronize()
    err1 = np.abs(ymx.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err1 < 1e-5
    ctx.set_wait_limit(0.0)
    ctx.sigma(i, 1, x, ymx, nvec=2, precision=pkg.LRT_MIXED)
    torch.cuda.synchronize()
    assert np.abs(ymx.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-5
    ctx.close()
