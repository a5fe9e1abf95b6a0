"""Batched sigma over independent instances (one grouped launch per phase, CUDA graph
replay) against the per-instance sigma of the same library (GPU)."""
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


SHAPES = [(6, 3, 3, 16), (7, 4, 3, 24), (8, 4, 4, 32), (5, 2, 3, 12), (8, 5, 3, 40)]


def _instances(pkg, nsite):
    out = []
    for j, (k, na, nb, M) in enumerate(SHAPES):
        H = synth.ab_initio(k, na, nb, 500 + j)
        i = k // 2 - 1
        m = synth.mixed_mps(k, na, nb, M, 50 + j, center=i)
        ctx = pkg.Context(0)
        ctx.op_build(k, H.h, H.eri, e_core=H.e_core)
        ctx.mps_load(k, na, nb, m.bonds, m.sites, i)
        for b in range(i):
            ctx.renormalize(b, +1)
        for b in range(k - 1, i + nsite - 1, -1):
            ctx.renormalize(b, -1)
        out.append((ctx, i))
    return out


@pytest.mark.parametrize("nsite", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_batched_sigma_matches_per_instance(pkg, nsite, precision):
    insts = _instances(pkg, nsite)
    nvec = 3
    xs, ref = [], []
    for j, (ctx, i) in enumerate(insts):
        n, _ = ctx.wfn_layout(i, nsite)
        x = torch.tensor(synth.random_vector(n * nvec, 70 + j), dtype=torch.float64, device="cuda:0")
        y = torch.empty_like(x)
        ctx.sigma(i, nsite, x, y, nvec=nvec, precision=precision)
        xs.append(x)
        ref.append(y.clone())
    ys = [torch.full_like(x, float("nan")) for x in xs]
    ctxs = [c for c, _ in insts]
    sites = [i for _, i in insts]
    for rep in range(3):          # eager, then captured, then replayed from the graph
        for y in ys:
            y.fill_(float("nan"))
        pkg.sigma_batched(ctxs, sites, nsite, xs, ys, nvec=nvec, precision=precision)
        torch.cuda.synchronize()
        for y, r in zip(ys, ref):
            assert torch.isfinite(y).all()
            assert float((y - r).abs().max() / r.abs().max()) <= 1e-13
    # new data in the same buffers: the replayed graph reads the current contents
    for j, x in enumerate(xs):
        x.copy_(torch.tensor(synth.random_vector(x.numel(), 170 + j), dtype=torch.float64, device="cuda:0"))
    pkg.sigma_batched(ctxs, sites, nsite, xs, ys, nvec=nvec, precision=precision)
    torch.cuda.synchronize()
    for (ctx, i), x, y in zip(insts, xs, ys):
        r = torch.empty_like(x)
        ctx.sigma(i, nsite, x, r, nvec=nvec, precision=precision)
        assert float((y - r).abs().max() / r.abs().max()) <= 1e-13
    for c in ctxs:
        c.close()
