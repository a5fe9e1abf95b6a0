"""sigma_noalloc, the sigma entry point for callers that must not allocate GPU memory.

Who needs it: a program whose own memory pool owns the device and forbids other
cudaMalloc/cudaFree traffic, or a loop that cannot absorb the synchronization an
allocation may cause.  These tests call it through the C ABI and check that it
returns what the regular, allocating sigma() returns, on two calls in a row (the
static scratch array is shared and overwritten by every call), and that it refuses
work it cannot do without allocating.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-12


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_1646_gb300 import build
    build.build()
    import paper_1311_1646_gb300 as p
    p.load()
    return p


def _context(pkg, H, M, i, nsite, seed):
    k, na, nb = H.k, H.n_alpha, H.n_beta
    m = synth.mixed_mps(k, na, nb, M, seed, center=i)
    ctx = pkg.Context(0)
    ctx.op_build(k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(k, na, nb, m.bonds, m.sites, i)
    for b in range(i):
        ctx.renormalize(b, +1)
    for b in range(k - 1, i + nsite - 1, -1):
        ctx.renormalize(b, -1)
    return ctx


def _dev(x):
    return torch.tensor(x, dtype=torch.float64, device="cuda:0")


@pytest.mark.parametrize("nsite,nvec", [(1, 1), (2, 3)])
def test_noalloc_matches_sigma_on_two_calls_in_a_row(pkg, nsite, nvec):
    cfg = synth.config(1)
    ctx = _context(pkg, cfg["ham"], cfg["M"], 3, nsite, 77)
    n, _ = ctx.wfn_layout(3, nsite)
    outs = []
    for call in range(2):
        x = _dev(synth.random_vector(nvec * n, 500 + call))
        y_ref = torch.full_like(x, np.nan)
        y = torch.full_like(x, np.nan)
        ctx.sigma(3, nsite, x, y_ref, nvec=nvec)          # the allocating path (prepares the plan)
        ctx.sigma_noalloc(3, nsite, x, y, nvec=nvec)      # the static-scratch path
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= RTOL * np.abs(b).max()
        outs.append(a)
    assert not np.array_equal(outs[0], outs[1])            # the second call really recomputed
    # once the first call has resolved the static array on this device, further calls take
    # no device memory
    x = _dev(synth.random_vector(nvec * n, 502))
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        ctx.sigma_noalloc(3, nsite, x, y, nvec=nvec)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ctx.close()


def test_noalloc_needs_a_prepared_plan(pkg):
    cfg = synth.config(1)
    ctx = _context(pkg, cfg["ham"], cfg["M"], 2, 1, 78)
    n, _ = ctx.wfn_layout(2, 1)
    x = _dev(synth.random_vector(n, 1))
    y = torch.empty_like(x)
    with pytest.raises(pkg.LrtError, match="-6"):
        ctx.sigma_noalloc(2, 1, x, y)
    ctx.close()


def test_noalloc_rejects_work_beyond_the_static_scratch(pkg):
    # the 12-site PPP chain at M = 256 with 6 vectors needs more intermediates than fit
    cfg = synth.config(2)
    ctx = _context(pkg, cfg["ham"], cfg["M"], 5, 2, 79)
    n, _ = ctx.wfn_layout(5, 2)
    x = _dev(synth.random_vector(6 * n, 2))
    y = torch.empty_like(x)
    ctx.sigma(5, 2, x, y, nvec=6)
    with pytest.raises(pkg.LrtError, match="static maximum"):
        ctx.sigma_noalloc(5, 2, x, y, nvec=6)
    ctx.close()
