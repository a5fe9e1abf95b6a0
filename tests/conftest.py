import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def stationary_k5():
    """A truncated ab initio reference, k = 5 orbitals, 3 alpha 2 beta electrons, M = 6
    (bond dimensions 4, 6, 6, 4): two-site sweeps, then tight one-site sweeps to a
    stationary point of the fixed-bond-dimension MPS manifold.  Returns
    (ham, (L0, R0, C0, Lam, norm)) in the mixed-canonical gauge."""
    import synth
    from oracle import dmrg, fock
    from oracle import mps as om

    k, na, nb, M = 5, 3, 2, 6
    H = synth.ab_initio(k, na, nb, 7)
    t, v = fock.spin_integrals(H.h, H.eri)
    _, sites, _ = dmrg.ground_state(H, t, v, [M], synth.random_mps(k, na, nb, M, 3))
    _, sites, _ = dmrg.onesite_sweeps(H, t, v, sites, n_sweeps=30, dav_tol=1e-13)
    return H, om.mixed_canonical(sites)
