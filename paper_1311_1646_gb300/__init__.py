"""GB300 DMRG effective-Hamiltonian library: Python binding of the C ABI in include/lrt.h.

Argument marshalling only: every step of sigma, renormalization and the
diagonal runs in the CUDA library liblrt.so (built by `build.build()`).  Device
buffers are torch CUDA tensors (float64, contiguous); host arrays are NumPy.
There is no CPU fallback: without the library every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblrt.so")

LRT_FP64 = 0
LRT_MIXED = 1
LRT_CORR_SITE = 0
LRT_CORR_SWEEP = 1

EXPORTS = ["lrt_create", "lrt_destroy", "lrt_last_error", "op_build", "mps_load", "wfn_layout",
           "renormalize", "sigma", "heff_diag", "sigma_stats", "sigma_noalloc", "sweep_gs",
           "mps_save", "mps_get_bonds", "mps_get_site", "tda_load", "tda_prepare", "tda_stationarity", "sweep_tda", "sweep_tda_density", "sweep_response", "lrt_sweeps", "lrt_sweep_log", "lrt_set_wait_limit", "sigma_batched",
           "sweep_tda_batched"]

_lib = None


class MpsDesc(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n_alpha", ctypes.c_int), ("n_beta", ctypes.c_int),
                ("bond_nsect", ctypes.POINTER(ctypes.c_int)),
                ("bond_sectors", ctypes.POINTER(ctypes.c_int)),
                ("site_data", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
                ("center", ctypes.c_int),
                ("site_data_right", ctypes.POINTER(ctypes.POINTER(ctypes.c_double)))]


class MpsOut(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n_alpha", ctypes.c_int), ("n_beta", ctypes.c_int),
                ("total_sectors", ctypes.c_int), ("has_right", ctypes.c_int),
                ("bond_nsect", ctypes.POINTER(ctypes.c_int)), ("bond_sectors", ctypes.POINTER(ctypes.c_int)),
                ("site_nelem", ctypes.POINTER(ctypes.c_int64)),
                ("site_data", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
                ("site_data_right", ctypes.POINTER(ctypes.POINTER(ctypes.c_double)))]


class SigmaStats(ctypes.Structure):
    _fields_ = [("flops", ctypes.c_double), ("flops_issued", ctypes.c_double), ("op_bytes", ctypes.c_double),
                ("launches", ctypes.c_int),
                ("n_terms", ctypes.c_int), ("n_products", ctypes.c_int)]


class GsParams(ctypes.Structure):
    _fields_ = [("max_sweeps", ctypes.c_int), ("n_schedule", ctypes.c_int),
                ("M_schedule", ctypes.POINTER(ctypes.c_int)), ("sweeps_per_M", ctypes.c_int),
                ("e_tol", ctypes.c_double), ("dav_tol", ctypes.c_double), ("dav_max_iter", ctypes.c_int),
                ("dav_max_space", ctypes.c_int), ("trunc_tol", ctypes.c_double), ("onesite_sweeps", ctypes.c_int)]


class TdaParams(ctypes.Structure):
    _fields_ = [("max_space", ctypes.c_int), ("max_iter", ctypes.c_int), ("eps", ctypes.c_double),
                ("pinv_cut", ctypes.c_double), ("seed", ctypes.c_uint64), ("precision", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("keep", ctypes.c_int), ("correction", ctypes.c_int),
                ("corr_tol", ctypes.c_double), ("start_shift", ctypes.c_double)]


class RespParams(ctypes.Structure):
    _fields_ = [("max_sweeps", ctypes.c_int), ("tol", ctypes.c_double), ("minres_max", ctypes.c_int),
                ("minres_tol", ctypes.c_double), ("pinv_cut", ctypes.c_double), ("method", ctypes.c_int),
                ("max_space", ctypes.c_int)]


LRT_RESP_SITE, LRT_RESP_SUBSPACE = 0, 1


class LrtError(RuntimeError):
    pass


def load(path: str | None = None) -> ctypes.CDLL:
    """Load liblrt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise LrtError(f"CUDA library missing: {path} (run paper_1311_1646_gb300.build.build())")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    lib.lrt_create.argtypes = [ctypes.POINTER(vp), i, vp]
    lib.lrt_destroy.argtypes = [vp]
    lib.lrt_last_error.argtypes = [vp]
    lib.lrt_last_error.restype = ctypes.c_char_p
    lib.op_build.argtypes = [vp, i, dp, dp, i, dp, d]
    lib.mps_load.argtypes = [vp, ctypes.POINTER(MpsDesc)]
    lib.mps_save.argtypes = [vp, ctypes.POINTER(MpsOut)]
    lib.wfn_layout.argtypes = [vp, i, i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int64)]
    lib.renormalize.argtypes = [vp, i, i, i]
    lib.sigma.argtypes = [vp, i, i, i, vp, vp, i]
    lib.heff_diag.argtypes = [vp, i, i, vp]
    lib.sigma_stats.argtypes = [vp, ctypes.POINTER(SigmaStats)]
    lib.sigma_noalloc.argtypes = [vp, i, i, i, vp, vp]
    lib.sweep_gs.argtypes = [vp, ctypes.POINTER(GsParams), ctypes.POINTER(ctypes.c_double)]
    lib.mps_get_bonds.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int)]
    lib.mps_get_site.argtypes = [vp, i, dp, ctypes.POINTER(ctypes.c_int64)]
    ppd = ctypes.POINTER(ctypes.POINTER(ctypes.c_double))
    lib.tda_load.argtypes = [vp, ppd, ppd]
    lib.tda_prepare.argtypes = [vp, dp]
    lib.tda_stationarity.argtypes = [vp, dp, dp]
    lib.lrt_sweeps.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.lrt_sweep_log.argtypes = [vp, i, dp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.sweep_response.argtypes = [vp, vp, d, ctypes.POINTER(RespParams), dp, dp, ctypes.POINTER(ctypes.c_int)]
    lib.lrt_set_wait_limit.argtypes = [vp, d, i]
    lib.sigma_batched.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(ctypes.c_int), i, i,
                                  ctypes.POINTER(vp), ctypes.POINTER(vp), i]
    lib.sweep_tda.argtypes = [vp, i, ctypes.POINTER(TdaParams), dp, dp, dp]
    lib.sweep_tda_density.argtypes = [vp, i, ctypes.POINTER(TdaParams), dp, dp, dp, dp]
    lib.sweep_tda_batched.argtypes = [ctypes.POINTER(vp), i, i, ctypes.POINTER(TdaParams), dp, dp, dp]
    for name in EXPORTS:
        if name != "lrt_last_error":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _site_size(left, right) -> int:
    """Elements of a site tensor in the boundary's left-fused layout: for every right sector
    q_r and site state n whose left sector q_r - n exists, a D(q_l) x D(q_r) block."""
    ldim = {(int(a), int(b)): int(d) for a, b, d in left}
    return sum(ldim.get((int(ra) - sa, int(rb) - sb), 0) * int(dr)
               for ra, rb, dr in right for sa, sb in ((0, 0), (1, 0), (0, 1), (1, 1)))


def _tensor_ptr(t, nelem: int) -> int:
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise LrtError("expected a contiguous float64 CUDA tensor")
    if t.numel() < nelem:
        raise LrtError(f"tensor has {t.numel()} elements, need {nelem}")
    return t.data_ptr()


class Context:
    """One library context on one device and stream."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = 0
        h = ctypes.c_void_p()
        rc = self.lib.lrt_create(ctypes.byref(h), device, ctypes.c_void_p(stream))
        if rc != 0:
            raise LrtError(f"lrt_create failed ({rc}): {self.lib.lrt_last_error(None).decode()}")
        self.h = h
        self.device = device
        self._keep = []
        self._k = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.lrt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, what: str):
        if rc != 0:
            msg = self.lib.lrt_last_error(self.h).decode()
            raise LrtError(f"{what} failed ({rc}): {msg}")

    def op_build(self, k: int, h: np.ndarray, eri: np.ndarray | None = None, B: np.ndarray | None = None,
                 e_core: float = 0.0):
        h = np.ascontiguousarray(h, dtype=np.float64)
        e = np.ascontiguousarray(eri, dtype=np.float64) if eri is not None else None
        b = np.ascontiguousarray(B, dtype=np.float64) if B is not None else None
        if h.shape != (k, k):
            raise LrtError(f"op_build: h has shape {h.shape}, need ({k}, {k})")
        if e is not None and e.size != k ** 4:
            raise LrtError(f"op_build: eri has {e.size} elements, need k^4 = {k ** 4}")
        if b is not None and (b.ndim != 3 or b.shape[1:] != (k, k)):
            raise LrtError(f"op_build: B has shape {b.shape}, need (n_factor, {k}, {k})")
        nL = 0 if b is None else b.shape[0]
        self._check(self.lib.op_build(self.h, k, _dptr(h), _dptr(e) if e is not None else None, nL,
                                      _dptr(b) if b is not None else None, float(e_core)), "op_build")

    def mps_load(self, k: int, n_alpha: int, n_beta: int, bonds: list, sites: list, center: int = 0,
                 sites_right: list | None = None):
        """Load an MPS: `sites` (left-orthonormal form, left-fused layout) and optionally the
        right-orthonormal form `sites_right` of every site (same layout)."""
        if len(bonds) != k + 1 or len(sites) != k or (sites_right is not None and len(sites_right) != k):
            raise LrtError(f"mps_load: need {k + 1} bond tables and {k} sites")
        nsect = np.array([len(t) for t in bonds], dtype=np.int32)
        secs = np.array([x for t in bonds for s in t for x in s], dtype=np.int32)
        if len(secs) != 3 * int(nsect.sum()):
            raise LrtError("mps_load: every bond sector is a triple (n_alpha, n_beta, dim)")

        def fused(arrays, what):
            out = [np.ascontiguousarray(s, dtype=np.float64).ravel() for s in arrays]
            for i, a in enumerate(out):
                want = _site_size(bonds[i], bonds[i + 1])
                if a.size != want:
                    raise LrtError(f"mps_load: {what} {i} has {a.size} elements, its layout has {want}")
            return out

        arrs = fused(sites, "site")
        ptrs = (ctypes.POINTER(ctypes.c_double) * k)(*[_dptr(a) for a in arrs])
        rptrs = None
        if sites_right is not None:
            rarrs = fused(sites_right, "right-orthonormal site")
            rptrs = (ctypes.POINTER(ctypes.c_double) * k)(*[_dptr(a) for a in rarrs])
        desc = MpsDesc(k, n_alpha, n_beta, nsect.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                       secs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ptrs, center, rptrs)
        self._check(self.lib.mps_load(self.h, ctypes.byref(desc)), "mps_load")
        self._k = k

    def wfn_layout(self, site: int, nsite: int):
        n = ctypes.c_int64()
        nb = ctypes.c_int()
        self._check(self.lib.wfn_layout(self.h, site, nsite, ctypes.byref(n), ctypes.byref(nb), None),
                    "wfn_layout")
        offs = (ctypes.c_int64 * max(nb.value, 1))()
        self._check(self.lib.wfn_layout(self.h, site, nsite, ctypes.byref(n), ctypes.byref(nb), offs),
                    "wfn_layout")
        return n.value, list(offs)[:nb.value]

    def renormalize(self, site: int, direction: int, precision: int = LRT_FP64):
        self._check(self.lib.renormalize(self.h, site, direction, precision), "renormalize")

    def sigma(self, site: int, nsite: int, x, y, nvec: int = 1, precision: int = LRT_FP64):
        n, _ = self.wfn_layout(site, nsite)
        self._check(self.lib.sigma(self.h, site, nsite, nvec, ctypes.c_void_p(_tensor_ptr(x, n * nvec)),
                                   ctypes.c_void_p(_tensor_ptr(y, n * nvec)), precision), "sigma")

    def sigma_noalloc(self, site: int, nsite: int, x, y, nvec: int = 1):
        """H_eff x without any GPU allocation, for callers that cannot allocate (a program
        whose own pool owns the device memory, a loop that cannot absorb an allocator
        synchronization).  Needs a plan prepared by an earlier sigma() call with the same
        (site, nsite, nvec); shares one static 32 MiB device array across all calls, so
        calls must not overlap on the GPU."""
        n, _ = self.wfn_layout(site, nsite)
        self._check(self.lib.sigma_noalloc(self.h, site, nsite, nvec, ctypes.c_void_p(_tensor_ptr(x, n * nvec)),
                                           ctypes.c_void_p(_tensor_ptr(y, n * nvec))), "sigma_noalloc")

    def heff_diag(self, site: int, nsite: int, d):
        n, _ = self.wfn_layout(site, nsite)
        self._check(self.lib.heff_diag(self.h, site, nsite, ctypes.c_void_p(_tensor_ptr(d, n))), "heff_diag")

    def sweep_gs(self, M_schedule, max_sweeps: int = 20, sweeps_per_M: int = 2, e_tol: float = 1e-10,
                 dav_tol: float = 1e-8, dav_max_iter: int = 200, dav_max_space: int = 24,
                 trunc_tol: float = 1e-14, onesite_sweeps: int = 0) -> float:
        """Two-site ground-state sweeps on the loaded (right-orthonormal) MPS, then
        `onesite_sweeps` one-site sweeps; returns E0."""
        ms = (ctypes.c_int * len(M_schedule))(*M_schedule)
        p = GsParams(max_sweeps, len(M_schedule), ms, sweeps_per_M, e_tol, dav_tol, dav_max_iter,
                     dav_max_space, trunc_tol, onesite_sweeps)
        e = ctypes.c_double()
        self._check(self.lib.sweep_gs(self.h, ctypes.byref(p), ctypes.byref(e)), "sweep_gs")
        return e.value

    def tda_load(self, C0: list, lam: list):
        """Zeroth-order centre tensors C0_i (left-fused layout) and Schmidt values per bond."""
        bonds = self._bond_tables()
        k = len(bonds) - 1
        if len(C0) != k or len(lam) != k + 1:
            raise LrtError(f"tda_load: need {k} centre tensors and {k + 1} Schmidt-value arrays")
        c0 = [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in C0]
        lm = [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in lam]
        for i, a in enumerate(c0):
            want = _site_size(bonds[i], bonds[i + 1])
            if a.size != want:
                raise LrtError(f"tda_load: C0 {i} has {a.size} elements, its layout has {want}")
        for b, a in enumerate(lm):
            want = sum(int(d) for _, _, d in bonds[b])
            if a.size != want:
                raise LrtError(f"tda_load: Lambda of bond {b} has {a.size} values, the bond has {want} states")
        pc = (ctypes.POINTER(ctypes.c_double) * len(c0))(*[_dptr(a) for a in c0])
        pl = (ctypes.POINTER(ctypes.c_double) * len(lm))(*[_dptr(a) for a in lm])
        self._check(self.lib.tda_load(self.h, pc, pl), "tda_load")

    def tda_prepare(self) -> float:
        """Mixed-canonical gauge of the loaded MPS on the GPU (instead of tda_load); returns its norm."""
        nrm = ctypes.c_double()
        self._check(self.lib.tda_prepare(self.h, ctypes.byref(nrm)), "tda_prepare")
        return nrm.value

    def set_wait_limit(self, seconds: float, stall_next: bool = False):
        """Limit of the tensor-core kernels' pipeline waits (0: the default); stall_next makes
        the next tensor-core launch end through the expired-wait path (test hook)."""
        self._check(self.lib.lrt_set_wait_limit(self.h, float(seconds), 1 if stall_next else 0),
                    "lrt_set_wait_limit")

    def sweeps(self) -> int:
        """Sweeps run by the last sweep_gs or sweep_tda on this context."""
        n = ctypes.c_int()
        self._check(self.lib.lrt_sweeps(self.h, ctypes.byref(n)), "lrt_sweeps")
        return n.value

    def sweep_response(self, vctx: "Context", omega: float, max_sweeps: int = 0, tol: float = 0.0,
                       minres_max: int = 0, minres_tol: float = 0.0, pinv_cut: float = 0.0,
                       method: int = LRT_RESP_SITE, max_space: int = 0):
        """Tamm-Dancoff linear response alpha(omega) to the one-body perturbation held by
        `vctx` (op_build with h = d and no two-electron part, the same MPS, tda_prepare'd).
        Returns (alpha, resid[2], sweeps[2])."""
        a = ctypes.c_double()
        rs = np.zeros(2)
        sw = (ctypes.c_int * 2)()
        p = RespParams(max_sweeps, tol, minres_max, minres_tol, pinv_cut, method, max_space)
        self._check(self.lib.sweep_response(self.h, vctx.h, float(omega), ctypes.byref(p), ctypes.byref(a), _dptr(rs),
                                            sw), "sweep_response")
        return a.value, rs, (sw[0], sw[1])

    def sweep_log(self):
        """[(seconds, mixed)] of every sweep of the last sweep_tda (the start sweep first)."""
        n = ctypes.c_int()
        self._check(self.lib.lrt_sweep_log(self.h, 0, None, None, ctypes.byref(n)), "lrt_sweep_log")
        cap = n.value
        sec = np.zeros(max(cap, 1))
        mx = (ctypes.c_int * max(cap, 1))()
        self._check(self.lib.lrt_sweep_log(self.h, cap, _dptr(sec), mx, ctypes.byref(n)), "lrt_sweep_log")
        return [(float(sec[j]), int(mx[j])) for j in range(min(cap, n.value))]

    def tda_stationarity(self):
        """(sum_i |Q^C (H_0^[i] - E0) C0_i|^2, E0) of the loaded reference."""
        g = ctypes.c_double()
        e = ctypes.c_double()
        self._check(self.lib.tda_stationarity(self.h, ctypes.byref(g), ctypes.byref(e)), "tda_stationarity")
        return g.value, e.value

    def sweep_tda(self, nroots: int, max_space: int = 0, max_iter: int = 60, eps: float = 1e-14,
                  pinv_cut: float = 1e-12, seed: int = 12345, allow_noconv: bool = False,
                  precision: int = LRT_FP64, refine_tol: float = 0.0, keep: int = 0, correction: int = 0,
                  corr_tol: float = 0.0, start_shift: float = 0.0):
        """DMRG-TDA roots: returns (omega, resid, e0); omega are excitation energies.  With
        precision=LRT_MIXED the H_0 site products run on the tensor cores until the residuals
        fall below refine_tol, then the sweeps finish in FP64."""
        om = np.zeros(nroots)
        rs = np.zeros(nroots)
        e0 = ctypes.c_double()
        p = TdaParams(max_space, max_iter, eps, pinv_cut, seed, precision, refine_tol, keep, correction,
                      corr_tol, start_shift)
        rc = self.lib.sweep_tda(self.h, nroots, ctypes.byref(p), _dptr(om), _dptr(rs), ctypes.byref(e0))
        if rc != 0 and not (allow_noconv and rc == -4):
            self._check(rc, "sweep_tda")
        return om, rs, e0.value

    def sweep_tda_density(self, nroots: int, max_space: int = 0, max_iter: int = 60, eps: float = 1e-14,
                          pinv_cut: float = 1e-12, seed: int = 12345, allow_noconv: bool = False,
                          precision: int = LRT_FP64, refine_tol: float = 0.0, keep: int = 0, correction: int = 0,
                          corr_tol: float = 0.0, start_shift: float = 0.0):
        """sweep_tda plus the roots' one-particle transition densities: returns
        (omega, resid, e0, gamma) with gamma of shape (nroots, k, k)."""
        om = np.zeros(nroots)
        rs = np.zeros(nroots)
        e0 = ctypes.c_double()
        g = np.zeros(nroots * self._k * self._k)
        p = TdaParams(max_space, max_iter, eps, pinv_cut, seed, precision, refine_tol, keep, correction,
                      corr_tol, start_shift)
        rc = self.lib.sweep_tda_density(self.h, nroots, ctypes.byref(p), _dptr(om), _dptr(rs), ctypes.byref(e0),
                                        _dptr(g))
        if rc != 0 and not (allow_noconv and rc == -4):
            self._check(rc, "sweep_tda_density")
        return om, rs, e0.value, g.reshape(nroots, self._k, self._k)

    def _bond_tables(self):
        """Bond tables [(na, nb, dim)] of the MPS the context holds now."""
        tot = ctypes.c_int()
        self._check(self.lib.mps_get_bonds(self.h, None, None, ctypes.byref(tot)), "mps_get_bonds")
        k = self._k
        ns = (ctypes.c_int * (k + 1))()
        sec = (ctypes.c_int * (3 * tot.value))()
        self._check(self.lib.mps_get_bonds(self.h, ns, sec, ctypes.byref(tot)), "mps_get_bonds")
        bonds, pos = [], 0
        for b in range(k + 1):
            bonds.append([(sec[3 * (pos + s)], sec[3 * (pos + s) + 1], sec[3 * (pos + s) + 2]) for s in range(ns[b])])
            pos += ns[b]
        return bonds

    def mps_save(self):
        """The MPS the context holds: dict with k, n_alpha, n_beta, bonds (tables of
        (na, nb, dim)), sites (left-fused arrays) and sites_right (or None)."""
        q = MpsOut()
        self._check(self.lib.mps_save(self.h, ctypes.byref(q)), "mps_save")
        k = q.k
        nsect = (ctypes.c_int * (k + 1))()
        secs = (ctypes.c_int * (3 * q.total_sectors))()
        nel = (ctypes.c_int64 * k)()
        q.bond_nsect, q.bond_sectors, q.site_nelem = nsect, secs, nel
        self._check(self.lib.mps_save(self.h, ctypes.byref(q)), "mps_save")
        sites = [np.zeros(nel[i]) for i in range(k)]
        right = [np.zeros(nel[i]) for i in range(k)] if q.has_right else None
        q.site_data = (ctypes.POINTER(ctypes.c_double) * k)(*[_dptr(a) for a in sites])
        if right is not None:
            q.site_data_right = (ctypes.POINTER(ctypes.c_double) * k)(*[_dptr(a) for a in right])
        self._check(self.lib.mps_save(self.h, ctypes.byref(q)), "mps_save")
        bonds, pos = [], 0
        for b in range(k + 1):
            bonds.append([(secs[3 * (pos + j)], secs[3 * (pos + j) + 1], secs[3 * (pos + j) + 2])
                          for j in range(nsect[b])])
            pos += nsect[b]
        return {"k": k, "n_alpha": q.n_alpha, "n_beta": q.n_beta, "bonds": bonds, "sites": sites,
                "sites_right": right}

    def mps_get(self):
        """The loaded MPS as (bonds, sites): bond tables [(na, nb, dim)] and left-fused site arrays."""
        bonds = self._bond_tables()
        k = self._k
        sites = []
        for i in range(k):
            n = ctypes.c_int64()
            self._check(self.lib.mps_get_site(self.h, i, None, ctypes.byref(n)), "mps_get_site")
            a = np.empty(n.value)
            self._check(self.lib.mps_get_site(self.h, i, _dptr(a), ctypes.byref(n)), "mps_get_site")
            sites.append(a)
        return bonds, sites

    def stats(self) -> dict:
        s = SigmaStats()
        self._check(self.lib.sigma_stats(self.h, ctypes.byref(s)), "sigma_stats")
        return {"flops": s.flops, "flops_issued": s.flops_issued, "op_bytes": s.op_bytes, "launches": s.launches,
                "n_terms": s.n_terms, "n_products": s.n_products}


def sigma_batched(ctxs: list, sites: list, nsite: int, xs: list, ys: list, nvec: int = 1,
                  precision: int = LRT_FP64):
    """y_j = H_eff^(j) x_j for several independent instances (one Context each) in one grouped
    launch per phase; the first context's stream runs it."""
    n = len(ctxs)
    if not (len(sites) == len(xs) == len(ys) == n) or n == 0:
        raise LrtError("sigma_batched: ctxs, sites, xs and ys must have the same non-zero length")
    hs = (ctypes.c_void_p * n)(*[c.h.value for c in ctxs])
    st = (ctypes.c_int * n)(*sites)
    px = (ctypes.c_void_p * n)(*[_tensor_ptr(x, ctxs[j].wfn_layout(sites[j], nsite)[0] * nvec)
                                 for j, x in enumerate(xs)])
    py = (ctypes.c_void_p * n)(*[_tensor_ptr(y, ctxs[j].wfn_layout(sites[j], nsite)[0] * nvec)
                                 for j, y in enumerate(ys)])
    ctxs[0]._check(ctxs[0].lib.sigma_batched(hs, n, st, nsite, nvec, px, py, precision), "sigma_batched")


def sweep_tda_batched(ctxs: list, nroots: int, max_space: int = 0, max_iter: int = 60, eps: float = 1e-14,
                      pinv_cut: float = 1e-12, seed: int = 12345, allow_noconv: bool = False,
                      precision: int = LRT_FP64, refine_tol: float = 0.0, keep: int = 0, correction: int = 0,
                      corr_tol: float = 0.0, start_shift: float = 0.0):
    """DMRG-TDA of several independent instances (one prepared Context each), run
    concurrently; returns (omega, resid, e0) with omega and resid of shape (n, nroots)."""
    n = len(ctxs)
    if n == 0:
        raise LrtError("sweep_tda_batched: no instances")
    om = np.zeros(n * nroots)
    rs = np.zeros(n * nroots)
    e0 = np.zeros(n)
    hs = (ctypes.c_void_p * n)(*[c.h.value for c in ctxs])
    p = TdaParams(max_space, max_iter, eps, pinv_cut, seed, precision, refine_tol, keep, correction,
                  corr_tol, start_shift)
    lib = ctxs[0].lib
    rc = lib.sweep_tda_batched(hs, n, nroots, ctypes.byref(p), _dptr(om), _dptr(rs), _dptr(e0))
    if rc != 0 and not (allow_noconv and rc == -4):
        msgs = "; ".join(c.lib.lrt_last_error(c.h).decode() for c in ctxs)
        raise LrtError(f"sweep_tda_batched failed ({rc}): {msgs}")
    return om.reshape(n, nroots), rs.reshape(n, nroots), e0
