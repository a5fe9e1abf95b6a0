"""Parity of the CUDA sigma / renormalization / diagonal against the CPU oracle (GPU)."""
import numpy as np
import pytest

import synth
from oracle import blocks as ob
from oracle import fock
from oracle import mps as om

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-12   # relative to max|y|, the FP64 agreement bar for sigma


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_1646_gb300 import build
    build.build()
    import paper_1311_1646_gb300 as p
    p.load()
    return p


class Case:
    def __init__(self, pkg, H, M, i, nsite, seed):
        self.H, self.i, self.nsite = H, i, nsite
        k, na, nb = H.k, H.n_alpha, H.n_beta
        self.m = m = synth.mixed_mps(k, na, nb, M, seed, center=i)
        self.ctx = ctx = pkg.Context(0)
        ctx.op_build(k, H.h, H.eri, e_core=H.e_core)
        ctx.mps_load(k, na, nb, m.bonds, m.sites, i)
        for b in range(i):
            ctx.renormalize(b, +1)
        for b in range(k - 1, i + nsite - 1, -1):
            ctx.renormalize(b, -1)
        self.n, _ = ctx.wfn_layout(i, nsite)
        t, v = fock.spin_integrals(H.h, H.eri)
        self.env = env = ob.Environment(H, t, v)
        sites = [om.unpack_site(m.sites[j], m.bonds[j], m.bonds[j + 1]) for j in range(k)]
        for b in range(i):
            env.grow_left(b, sites[b])
        for b in range(k - 1, i + nsite - 1, -1):
            env.grow_right(b, sites[b])

    def gpu_sigma(self, x, nvec=1):
        xd = torch.tensor(x, dtype=torch.float64, device="cuda:0")
        yd = torch.full_like(xd, np.nan)
        self.ctx.sigma(self.i, self.nsite, xd, yd, nvec=nvec)
        torch.cuda.synchronize()
        return yd.cpu().numpy()

    def gpu_diag(self):
        d = torch.full((self.n,), np.nan, dtype=torch.float64, device="cuda:0")
        self.ctx.heff_diag(self.i, self.nsite, d)
        torch.cuda.synchronize()
        return d.cpu().numpy()

    def unpack(self, x):
        b = self.m.bonds
        if self.nsite == 1:
            return om.unpack_site(x, b[self.i], b[self.i + 1])
        return om.unpack_twosite(x, b[self.i], b[self.i + 2])

    def pack(self, blocks):
        b = self.m.bonds
        if self.nsite == 1:
            return om.pack_site(blocks, b[self.i], b[self.i + 1])
        return om.pack_twosite(blocks, b[self.i], b[self.i + 2])

    def oracle_sigma(self, x):
        w = self.unpack(x)
        f = ob.sigma_onesite if self.nsite == 1 else ob.sigma_twosite
        return self.pack(f(self.env, self.i, w))

    def oracle_diag(self):
        w = self.unpack(np.zeros(self.n))
        shapes = {kk: a.shape for kk, a in w.items()}
        f = ob.diag_onesite if self.nsite == 1 else ob.diag_twosite
        return self.pack(f(self.env, self.i, shapes))


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("nsite", [1, 2])
def test_sigma_all_sites_small(pkg, nsite):
    H = synth.ab_initio(6, 3, 3, 21)
    for i in range(6 - nsite + 1):
        c = Case(pkg, H, 20, i, nsite, 31 + i)
        x = synth.random_vector(2 * c.n, 41 + i)
        y = c.gpu_sigma(x, nvec=2)
        for v in range(2):
            ref = c.oracle_sigma(x[v * c.n:(v + 1) * c.n])
            assert _rel(y[v * c.n:(v + 1) * c.n], ref) < RTOL, (i, v)
        assert _rel(c.gpu_diag(), c.oracle_diag()) < RTOL
        c.ctx.close()


@pytest.mark.parametrize("k,na,nb,M,i,nsite", [(5, 1, 3, 12, 2, 1), (7, 4, 3, 24, 2, 2), (7, 4, 3, 24, 6, 1),
                                               (5, 0, 2, 8, 0, 2)])
def test_sigma_odd_ragged_and_boundaries(pkg, k, na, nb, M, i, nsite):
    H = synth.ab_initio(k, na, nb, 5 + k)
    c = Case(pkg, H, M, i, nsite, 17)
    x = synth.random_vector(c.n, 3)
    assert _rel(c.gpu_sigma(x), c.oracle_sigma(x)) < RTOL
    assert _rel(c.gpu_diag(), c.oracle_diag()) < RTOL
    c.ctx.close()


@pytest.mark.parametrize("nsite", [1, 2])
def test_sigma_abinitio_k8_m64(pkg, nsite):
    cfg = synth.config(1)
    c = Case(pkg, cfg["ham"], cfg["M"], 3, nsite, 101)
    x = synth.random_vector(3 * c.n, 7)
    y = c.gpu_sigma(x, nvec=3)
    for v in range(3):
        assert _rel(y[v * c.n:(v + 1) * c.n], c.oracle_sigma(x[v * c.n:(v + 1) * c.n])) < RTOL
    c.ctx.close()


def test_sigma_ppp_polyene_full_size(pkg):
    """The benchmarked workload: PPP polyene, 12 sites, M = 256, two-site at the middle, 6 vectors."""
    cfg = synth.config(2)
    c = Case(pkg, cfg["ham"], cfg["M"], 5, 2, 202)
    nvec = cfg["nroots"]
    x = synth.random_vector(nvec * c.n, 9)
    y = c.gpu_sigma(x, nvec=nvec)
    for v in (0, nvec - 1):
        assert _rel(y[v * c.n:(v + 1) * c.n], c.oracle_sigma(x[v * c.n:(v + 1) * c.n])) < RTOL
    # the vectors are independent: one batched call equals separate calls bit for bit
    y0 = c.gpu_sigma(x[:c.n])
    assert np.array_equal(y0, y[:c.n])
    # H_eff is symmetric: <u, H w> = <H u, w>
    u, w = x[:c.n], x[c.n:2 * c.n]
    a, b = u @ y[c.n:2 * c.n], y[:c.n] @ w
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)
    assert _rel(c.gpu_diag(), c.oracle_diag()) < RTOL
    st = c.ctx.stats()
    assert st["launches"] == 2 and st["flops"] > 0
    c.ctx.close()


def test_sigma_water_k24_M500_middle_site_both_precisions(pkg):
    """The headline workload of the benchmark at full size: water-shaped k = 24, 5 alpha 5 beta,
    M = 500, one-site sigma at the middle position with 6 vectors.  FP64 against the oracle
    at 1e-12; the split-TF32 path against the oracle at 1e-5 (relative to max|y|)."""
    cfg = synth.config(3)
    H = cfg["ham"]
    c = Case(pkg, H, cfg["M"], H.k // 2 - 1, 1, 303)
    nvec = cfg["nroots"]
    x = synth.random_vector(nvec * c.n, 10)
    y = c.gpu_sigma(x, nvec=nvec)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda:0")
    yd = torch.full_like(xd, np.nan)
    c.ctx.sigma(c.i, 1, xd, yd, nvec=nvec, precision=pkg.LRT_MIXED)
    torch.cuda.synchronize()
    ymx = yd.cpu().numpy()
    for v in (0, nvec - 1):
        yo = c.oracle_sigma(x[v * c.n:(v + 1) * c.n])
        assert _rel(y[v * c.n:(v + 1) * c.n], yo) < RTOL
        assert _rel(ymx[v * c.n:(v + 1) * c.n], yo) < 1e-5
    c.ctx.close()


def test_state_errors_are_reported(pkg):
    H = synth.ab_initio(4, 2, 2, 3)
    m = synth.mixed_mps(4, 2, 2, 8, 3, center=1)
    ctx = pkg.Context(0)
    ctx.op_build(4, H.h, H.eri)
    ctx.mps_load(4, 2, 2, m.bonds, m.sites, 1)
    n, _ = ctx.wfn_layout(1, 1)
    x = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    y = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(pkg.LrtError, match="-6"):
        ctx.sigma(1, 1, x, y)              # left block of bond 1 not built yet
    ctx.renormalize(0, +1)
    with pytest.raises(pkg.LrtError, match="-6"):
        ctx.sigma(1, 1, x, y)              # right block of bond 2 not built yet
    for b in (3, 2):
        ctx.renormalize(b, -1)
    with pytest.raises(pkg.LrtError, match="-1"):
        ctx.sigma(1, 1, x, x)              # x and y overlap
    ctx.sigma(1, 1, x, y)
    ctx.close()


@pytest.mark.parametrize("nsite", [1, 2])
def test_sigma_with_factorized_integrals(pkg, nsite):
    """The two-electron integrals given as the factor B ((ij|kl) = sum_L B_Lij B_Lkl, the form
    the [2Fe-2S]-shaped workload uses: rank-limited factor, near-degenerate replaced diagonal)
    instead of the k^4 tensor: the same sigma as from the tensor, and the oracle's."""
    k = 8
    d = np.concatenate([np.linspace(-2.0, -1.1, 3), -1.0 + 0.1 * np.linspace(0.0, 1.0, 3), np.linspace(-0.8, 0.0, 2)])
    H = synth.ab_initio(k, 3, 3, 41, nL=5, diag=d, replace_diag=True)
    c = Case(pkg, H, 24, 3, nsite, 43)
    x = synth.random_vector(2 * c.n, 5)
    y_eri = c.gpu_sigma(x, nvec=2)
    f = pkg.Context(0)
    f.op_build(k, H.h, None, B=H.B, e_core=H.e_core)
    f.mps_load(k, H.n_alpha, H.n_beta, c.m.bonds, c.m.sites, c.i)
    for b in range(c.i):
        f.renormalize(b, +1)
    for b in range(k - 1, c.i + nsite - 1, -1):
        f.renormalize(b, -1)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda:0")
    yd = torch.full_like(xd, np.nan)
    f.sigma(c.i, nsite, xd, yd, nvec=2)
    torch.cuda.synchronize()
    y_fac = yd.cpu().numpy()
    f.close()
    assert _rel(y_fac, y_eri) < RTOL
    for v in range(2):
        assert _rel(y_fac[v * c.n:(v + 1) * c.n], c.oracle_sigma(x[v * c.n:(v + 1) * c.n])) < RTOL
    c.ctx.close()
