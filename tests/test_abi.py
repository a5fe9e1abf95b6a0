"""The C-ABI library builds for sm_103a, loads, and exports every function of include/lrt.h (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "lrt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1311_1646_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["lrt_create", "lrt_destroy", "lrt_last_error", "op_build", "mps_load",
                     "wfn_layout", "renormalize", "sigma", "heff_diag", "sigma_stats"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    import paper_1311_1646_gb300 as pkg
    assert set(_declared_functions()) <= set(pkg.EXPORTS)


def test_bad_arguments_are_rejected_without_a_gpu(lib):
    # NULL handles and NULL outputs return LRT_EINVAL before any CUDA call
    lib.lrt_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.lrt_create(None, 0, None) == -1
    lib.sigma.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_int]
    assert lib.sigma(None, 0, 1, 1, None, None, 0) == -1
    lib.lrt_destroy.argtypes = [ctypes.c_void_p]
    assert lib.lrt_destroy(None) == -1
    vp = ctypes.c_void_p
    lib.sigma_batched.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int]
    assert lib.sigma_batched(None, 1, None, 1, 1, None, None, 0) == -1
    one_null = (vp * 1)(None)
    assert lib.sigma_batched(one_null, 1, None, 1, 1, None, None, 0) == -1
    lib.sweep_tda_batched.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
    assert lib.sweep_tda_batched(None, 1, 1, None, None, None, None) == -1
    om = (ctypes.c_double * 1)()
    params = (ctypes.c_char * 64)()
    assert lib.sweep_tda_batched(one_null, 1, 1, params, om, om, None) == -1
    lib.tda_prepare.argtypes = [vp, vp]
    assert lib.tda_prepare(None, None) == -1


def test_product_path_fails_loudly_without_the_library(tmp_path):
    import paper_1311_1646_gb300 as pkg
    saved = pkg._lib
    try:
        pkg._lib = None
        with pytest.raises(pkg.LrtError):
            pkg.load(str(tmp_path / "missing.so"))
    finally:
        pkg._lib = saved


def test_binding_checks_host_array_sizes_before_the_call():
    # the loaders read exactly the documented layout from host memory: the binding rejects
    # arrays of the wrong size or count before anything reaches the library
    import numpy as np
    import synth
    import paper_1311_1646_gb300 as pkg
    for k, na, nb, M in [(4, 2, 2, 8), (6, 3, 2, 20), (5, 1, 3, 12)]:
        m = synth.random_mps(k, na, nb, M, 1)
        for i in range(k):
            assert pkg._site_size(m.bonds[i], m.bonds[i + 1]) == len(m.sites[i])
    ctx = object.__new__(pkg.Context)            # no device: the checks run first
    H = synth.ab_initio(4, 2, 2, 3)
    m = synth.random_mps(4, 2, 2, 8, 1)
    bad = [
        lambda: ctx.op_build(4, H.h[:3, :3], H.eri),
        lambda: ctx.op_build(4, H.h, H.eri.ravel()[:-1]),
        lambda: ctx.op_build(4, H.h, None, B=np.zeros((2, 4, 3))),
        lambda: ctx.mps_load(4, 2, 2, m.bonds[:-1], m.sites, 0),
        lambda: ctx.mps_load(4, 2, 2, m.bonds, m.sites[:-1], 0),
        lambda: ctx.mps_load(4, 2, 2, m.bonds, [m.sites[0][:-1]] + list(m.sites[1:]), 0),
        lambda: ctx.mps_load(4, 2, 2, m.bonds, m.sites, 0, sites_right=list(m.sites[:-1]) + [np.zeros(1)]),
    ]
    for f in bad:
        with pytest.raises(pkg.LrtError):
            f()


def test_new_entries_reject_null_handles_without_a_gpu(lib):
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    out = (ctypes.c_double * 4)()
    ni = (ctypes.c_int * 2)()
    lib.sweep_response.argtypes = [vp, vp, d, vp, vp, vp, vp]
    assert lib.sweep_response(None, None, 0.1, None, out, out, ni) == -1
    lib.sweep_tda_density.argtypes = [vp, i, vp, vp, vp, vp, vp]
    assert lib.sweep_tda_density(None, 1, None, out, out, out, out) == -1
    lib.lrt_sweep_log.argtypes = [vp, i, vp, vp, vp]
    assert lib.lrt_sweep_log(None, 0, None, None, ni) == -1
    lib.lrt_set_wait_limit.argtypes = [vp, d, i]
    assert lib.lrt_set_wait_limit(None, 1.0, 0) == -1
