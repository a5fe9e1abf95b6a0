"""Benchmark of the DMRG effective-Hamiltonian sigma vector on one GB300.

Workload (the water-shaped ab initio case, the largest of the workloads that fits this
design on one GPU): k = 24 spatial orbitals, 5 alpha + 5 beta electrons, integrals from a
seeded factor with |v_ijkl| decaying as exp(-|i-j|/6), bond dimension M = 500, one-site
sigma with a block of 6 trial vectors (the 6 TDA roots), FP64.  One step = diag(H_eff)
plus H_eff X at every one-site position i = 0..23 of a sweep, on environments
(renormalized left/right blocks) built once before timing from random left- and
right-orthonormal MPS with the workload's sector structure.

Prints one JSON line.  --impl reference times the CPU oracle instead.
"""
import os

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import argparse
import json
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rates

# DRAM bytes (read + write) per launch of the dominant kernel: the FP64 sigma launches of one
# timed step of this workload (48 launches, one ncu capture of dram__bytes_read/write.sum with
# --profile-step), valid only for the kernel source it was taken on (sha256 prefix);
# otherwise, and for the mixed form, the bench reports null.
TRAFFIC = {
    "fp64": {"source": "lrt_kernels.cu", "sha256": "4b10c817f69cb891", "bytes": 1107.18e6},
    "mixed": {"source": "lrt_tc.cu", "sha256": "", "bytes": None},
}


def traffic(precision):
    import hashlib
    t = TRAFFIC[precision]
    path = os.path.join(ROOT, "paper_1311_1646_gb300", "csrc", t["source"])
    try:
        with open(path, "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    return t["bytes"] if t["bytes"] and h == t["sha256"] else None


def tf32_peak():
    """Dense TF32 tensor peak: the measured BF16 GEMM rate x the nominal TF32/BF16 ratio."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)["bf16_tflops"] * TF32_PER_BF16, "of measured (bf16 burst x 1.1/2.25)"
    except (OSError, KeyError, ValueError):
        return 1900.0 * TF32_PER_BF16, "of fallback (1.9 PF bf16 x 1.1/2.25)"
WORKLOAD = "water_k24_e10_M500_onesite_6vec_fp64"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                   help="sigma arithmetic: FP64, or split-TF32 tensor-core products (LRT_MIXED)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the side measurements (mixed sigma, PPP sigma, batching, TDA s/root)")
    p.add_argument("--quick-tda", action="store_true", help="TDA side measurement on the 8-orbital workload only")
    p.add_argument("--tda-water", action="store_true",
                   help="also the TDA to convergence on the k = 24, M = 500 workload (long)")
    p.add_argument("--no-fe2s2", action="store_true",
                   help="skip the side measurement on the k = 36, M = 1500 workload")
    p.add_argument("--profile", choices=["fp64", "mixed", "gather", "tda"],
                   help="profiler run: one sigma (fp64 / mixed) or one enlargement + renormalization "
                        "(gather) at the middle position, or three TDA sweeps on the PPP workload (tda), "
                        "between cudaProfilerStart and Stop")
    p.add_argument("--profile-step", action="store_true",
                   help="bracket the first timed step with cudaProfilerStart and Stop")
    p.add_argument("--profile-M", type=int, default=0, help="bond dimension of the profiler run (0: 500)")
    return p.parse_args()


def replica_throughput(total_ms, steps, flops_step, world, device="cpu"):
    """Replicas (one independent copy of the step per rank): the slowest rank's time over
    the timed steps decides, and the whole job did world x flops_step per step.
    Returns (ms_per_step, TFLOP/s of the whole job)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / steps
    return ms_per_step, world * flops_step / (ms_per_step * 1e-3) / 1e12


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _timed(fn, reps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def build_workload(pkg, device, cfg_idx=3, nsite=1):
    """Environments for every position of a sweep: all left blocks from a random
    left-orthonormal MPS, all right blocks from a random right-orthonormal one."""
    cfg = synth.config(cfg_idx)
    H = cfg["ham"]
    k, na, nb, M, nvec = H.k, H.n_alpha, H.n_beta, cfg["M"], cfg["nroots"]
    left = synth.random_mps(k, na, nb, M, 2024, "left")
    right = synth.random_mps(k, na, nb, M, 2025, "right")
    ctx = pkg.Context(device)
    ctx.op_build(k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(k, na, nb, left.bonds, left.sites, 0, sites_right=right.sites)
    for b in range(k - 1):
        ctx.renormalize(b, +1)
    for b in range(k - 1, nsite - 1, -1):
        ctx.renormalize(b, -1)
    positions = list(range(k - nsite + 1))
    sizes = {i: ctx.wfn_layout(i, nsite)[0] for i in positions}
    return ctx, H, positions, sizes, nvec


def fp64_peak(clocks):
    """FP64 FMA-pipe peak of GB300 at the sampled maximum SM clock: 152 SMs x 2 DFMA/clk x 2."""
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    return 152 * 2 * 2 * mhz * 1e6 / 1e12


class SigmaStep:
    """One step: diag + sigma (nvec vectors) at every position, on the library's stream."""

    def __init__(self, ctx, positions, sizes, nvec, nsite, device, prec):
        import torch
        self.ctx, self.positions, self.nvec, self.nsite, self.prec = ctx, positions, nvec, nsite, prec
        self.xs = {i: torch.tensor(synth.random_vector(nvec * sizes[i], 100 + i), dtype=torch.float64,
                                   device=f"cuda:{device}") for i in positions}
        self.ys = {i: torch.empty_like(self.xs[i]) for i in positions}
        self.ds = {i: torch.empty(sizes[i], dtype=torch.float64, device=f"cuda:{device}") for i in positions}
        # algorithmic flops and launches of one step (plans are built on the first call)
        self.flops, self.launches = 0.0, 0
        for i in positions:
            ctx.heff_diag(i, nsite, self.ds[i])
            ctx.sigma(i, nsite, self.xs[i], self.ys[i], nvec=nvec, precision=prec)
            st = ctx.stats()
            self.flops += st["flops"]
            self.launches += st["launches"] + 1
        torch.cuda.synchronize()

    def run(self, stream, ev=None):
        for n, i in enumerate(self.positions):
            self.ctx.heff_diag(i, self.nsite, self.ds[i])
            if ev is not None:
                ev[n][0].record(stream)
            self.ctx.sigma(i, self.nsite, self.xs[i], self.ys[i], nvec=self.nvec, precision=self.prec)
            if ev is not None:
                ev[n][1].record(stream)

    def timed(self, stream, steps, warmup, flush, sampler=None, profile_first=False):
        """(step ms, sigma ms, clocks) over `steps` timed steps, L2 flushed before each."""
        import torch
        for _ in range(warmup):
            self.run(stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        step_ms, sigma_ms = [], []
        for rep in range(steps):
            if profile_first and rep == 0:
                torch.cuda.profiler.start()
            if profile_first and rep == 1:
                torch.cuda.profiler.stop()
            flush.zero_()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in self.positions]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            self.run(stream, ev)
            e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            sigma_ms.append(sum(a.elapsed_time(b) for a, b in ev))
        if profile_first and steps == 1:
            torch.cuda.profiler.stop()
        clocks = sampler.stop() if sampler else None
        return step_ms, sigma_ms, clocks


def run_ours(args):
    import torch
    import paper_1311_1646_gb300 as pkg

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    device = local
    torch.cuda.set_device(device)
    nsite = 1
    ctx, H, positions, sizes, nvec = build_workload(pkg, device, 3, nsite)
    prec = pkg.LRT_MIXED if args.precision == "mixed" else pkg.LRT_FP64
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=f"cuda:{device}")  # 512 MB > L2
    S = SigmaStep(ctx, positions, sizes, nvec, nsite, device, prec)
    if world > 1:
        torch.distributed.barrier()
    step_ms, sigma_ms, clocks = S.timed(stream, args.steps, args.warmup, flush, ClockSampler(device),
                                        profile_first=args.profile_step)
    ms_per_step, value = replica_throughput(sum(step_ms), args.steps, S.flops, world,
                                            f"cuda:{device}" if world > 1 else "cpu")
    achieved = S.flops / (sum(sigma_ms) / args.steps * 1e-3) / 1e12

    # end to end through the public API: pinned host inputs -> device -> sigma -> host
    hx = {i: S.xs[i].cpu().pin_memory() for i in positions}
    hy = {i: torch.empty(nvec * sizes[i], dtype=torch.float64).pin_memory() for i in positions}
    h2d = sum(hx[i].numel() * 8 for i in positions)
    d2h = h2d
    e2e_ms = []
    for rep in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in positions:
            S.xs[i].copy_(hx[i], non_blocking=True)
            ctx.heff_diag(i, nsite, S.ds[i])
            ctx.sigma(i, nsite, S.xs[i], S.ys[i], nvec=nvec, precision=prec)
            hy[i].copy_(S.ys[i], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = world * S.flops / (statistics.mean(e2e_ms) * 1e-3) / 1e12

    mid = H.k // 2 - 1
    # algorithmic flops of one vector at the middle position (the CPU baseline's unit)
    xd = S.xs[mid][: sizes[mid]].clone()
    yd = torch.empty_like(xd)
    ctx.sigma(mid, nsite, xd, yd, nvec=1)
    flops_vec = ctx.stats()["flops"]
    flops_step, launches_step = S.flops, S.launches
    side = None
    if rank == 0 and world == 1 and not args.no_extras:
        try:
            side = extras(pkg, ctx, device, S, stream, flush, args)
        except Exception as e:   # the side measurements never cost the metric line
            side = {"error": repr(e)}
    del S
    ctx.close()
    if isinstance(side, dict) and not args.no_fe2s2:
        try:
            side["fe2s2_k36_M1500_onesite_8vec"] = fe2s2_sigma(pkg, device, stream)
        except Exception as e:
            side["fe2s2_k36_M1500_onesite_8vec"] = {"error": repr(e)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mid, flops_vec)
    if rank == 0:
        if args.precision == "mixed":
            peak, peak_note = tf32_peak()
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic("mixed"),
                    "kernel": "gemm_tf32x3_kernel (sigma phases 1+2)",
                    "peak_note": peak_note + "; achieved counts each split-TF32 product once "
                                 "(the tensor pipe issues it 3x)"}
            metric, dtype = "H_eff sigma TFLOP/s (algorithmic, split-TF32 mixed)", "tf32x3"
        else:
            peak = fp64_peak(clocks)
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic("fp64"),
                    "kernel": "gemm_fp64_kernel (sigma phases 1+2)",
                    "peak_note": "FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop at the sampled maximum SM "
                                 "clock (sm_103a has no FP64 tensor kind); an FMA probe measured "
                                 "1.20 TFLOP/s"}
            metric, dtype = "H_eff sigma TFLOP/s (algorithmic, FP64)", "f64"
        out = {
            "metric": metric,
            "value": value,
            "unit": "TFLOP/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": dtype,
            "data": "synthetic",
            "config": {"workload": WORKLOAD if args.precision == "fp64" else WORKLOAD.replace("fp64", "mixed"),
                       "k": H.k, "electrons": H.n_alpha + H.n_beta, "M": 500, "nsite": nsite,
                       "nvec": nvec, "positions": len(positions),
                       "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_step * args.steps,
            "flops_per_step": flops_step,
            "sigma_ms_per_step": sum(sigma_ms) / args.steps,
            "extras": side,
        }
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


# settings of the TDA side measurements: a thick restart (2 n Ritz vectors kept, subspace
# 32: on the 8-orbital and PPP workloads the fastest per root of subspaces 24 / 32 / 48 with
# 2n / 3n / 4n kept), the sweep correction, start vectors damped by their diagonal energy
TDA_KW = dict(max_space=32, correction=1, start_shift=0.1)
TDA_KEEP = 2


def _tda_run(pkg, device, H, bonds, sites, nr, prec, eps, max_iter):
    import torch
    t = pkg.Context(device)
    t.op_build(H.k, H.h, H.eri, e_core=H.e_core)
    t.mps_load(H.k, H.n_alpha, H.n_beta, bonds, sites, 0)
    t.tda_prepare()
    g2, _ = t.tda_stationarity()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    om, rs, e0 = t.sweep_tda(nr, max_iter=max_iter, eps=eps, allow_noconv=True, precision=prec,
                             keep=TDA_KEEP * nr, **TDA_KW)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    sweeps = t.sweeps()
    t.close()
    return dt, om, rs, e0, g2, sweeps


def _tda_converged(pkg, device, cfg_idx, schedule, eps, max_iter):
    """Ground state on the GPU (two-site sweeps along `schedule`, then one-site sweeps to a
    stationary point), then sweep_tda to convergence in FP64 and in the mixed form."""
    import torch
    cfg = synth.config(cfg_idx)
    H = cfg["ham"]
    nr = cfg["nroots"]
    g = pkg.Context(device)
    g.op_build(H.k, H.h, H.eri, e_core=H.e_core)
    m = synth.random_mps(H.k, H.n_alpha, H.n_beta, 16, 3, "right")
    g.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_gs = g.sweep_gs(schedule, max_sweeps=14, e_tol=1e-12, dav_tol=1e-10, onesite_sweeps=20)
    torch.cuda.synchronize()
    t_gs = time.perf_counter() - t0
    bonds, sites = g.mps_get()
    g.close()
    r64 = _tda_run(pkg, device, H, bonds, sites, nr, pkg.LRT_FP64, eps, max_iter)
    rmx = _tda_run(pkg, device, H, bonds, sites, nr, pkg.LRT_MIXED, eps, max_iter)
    (s64, w64, q64, e64, g2, n64), (smx, wmx, qmx, emx, _, nmx) = r64, rmx
    return {
        "gs_s": t_gs, "e0": e64, "reference_gradient2": g2, "nroots": nr,
        "fp64_s_per_root": s64 / nr, "mixed_s_per_root": smx / nr, "mixed_speedup": s64 / smx,
        "fp64_sweeps": n64, "mixed_sweeps": nmx,
        "omega_fp64": list(w64), "omega_mixed": list(wmx), "abs_domega_Eh": list(np.abs(w64 - wmx)),
        "resid_fp64": list(q64), "resid_mixed": list(qmx), "eps": eps,
        "converged": bool(np.all(q64 < eps) and np.all(qmx < eps)),
        "note": "ground state on the GPU: two-site sweeps with M = %s, then one-site sweeps "
                "(reference_gradient2 = sum_i |Q^C (H_0^[i] - E0) C0_i|^2); TDA: sweep_tda to sum "
                "|Q^C r|^2 < eps for every root, thick restart (2 n kept, subspace 32), sweep "
                "correction, diagonal-damped random start; mixed: tensor-core H_0 site products "
                "until sum |r|^2 < 1e-6, then FP64 sweeps to eps" % schedule}


def _tda_sweep_times(pkg, device, cfg_idx=3, iters=3):
    """Wall time per TDA sweep on the k = 24, M = 500 water workload (6 roots), FP64
    against the mixed form, on a random right-orthonormal reference of the workload's
    sector structure (the cost of a sweep does not depend on how far the roots have
    converged; a converged run needs the M = 500 ground state first, minutes of GPU time).
    Each form runs the start sweep and `iters` sweeps; the mixed form's last third is FP64
    (its refinement), so sweeps are compared index by index where both forms ran their own
    arithmetic."""
    cfg = synth.config(cfg_idx)
    H = cfg["ham"]
    nr = cfg["nroots"]
    m = synth.random_mps(H.k, H.n_alpha, H.n_beta, cfg["M"], 7, "right")
    out = {}
    for name, prec in (("fp64", pkg.LRT_FP64), ("mixed", pkg.LRT_MIXED)):
        t = pkg.Context(device)
        try:
            t.op_build(H.k, H.h, H.eri, e_core=H.e_core)
            t.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, 0)
            t.tda_prepare()
            t0 = time.perf_counter()
            t.sweep_tda(nr, max_iter=iters, eps=1e-30, allow_noconv=True, precision=prec, keep=TDA_KEEP * nr, **TDA_KW)
            dt = time.perf_counter() - t0
            log = t.sweep_log()
        finally:
            t.close()
        out[name] = {"total_s": dt, "setup_s": dt - sum(x for x, _ in log), "sweep_s": [x for x, _ in log],
                     "tensor_core_sweep": [f for _, f in log]}
    fp, mx = out["fp64"], out["mixed"]
    both = [j for j in range(1, min(len(fp["sweep_s"]), len(mx["sweep_s"]))) if mx["tensor_core_sweep"][j]]
    if both:
        a = sum(fp["sweep_s"][j] for j in both)
        b = sum(mx["sweep_s"][j] for j in both)
        out["compared_sweeps"] = both
        out["fp64_s_per_sweep"] = a / len(both)
        out["mixed_s_per_sweep"] = b / len(both)
        out["mixed_speedup_per_sweep"] = a / b
    out["note"] = ("random right-orthonormal reference with the workload's sectors, M = 500, 6 roots, subspace "
                   "growing by 6 vectors per sweep (restart settings of the converged runs); "
                   "sweep_s[0] is the start sweep")
    return out


def _lr_k8(pkg, device, nroots=4):
    """The 8-orbital workload (M = 64): the TDA roots with their one-particle transition
    densities (sweep_tda_density; square norms as in Table site_excitation) and the
    Tamm-Dancoff response alpha(omega) to a seeded one-body perturbation at omega = 0 and
    at half the lowest TDA root (sweep_response), FP64, on the GPU ground state."""
    import torch
    cfg = synth.config(1)
    H = cfg["ham"]
    g = pkg.Context(device)
    g.op_build(H.k, H.h, H.eri, e_core=H.e_core)
    m = synth.random_mps(H.k, H.n_alpha, H.n_beta, 16, 3, "right")
    g.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, 0)
    g.sweep_gs([32, 64], max_sweeps=14, e_tol=1e-12, dav_tol=1e-10, onesite_sweeps=20)
    bonds, sites = g.mps_get()
    g.close()

    def prepared(h, eri, e_core):
        c = pkg.Context(device)
        c.op_build(H.k, h, eri, e_core=e_core)
        c.mps_load(H.k, H.n_alpha, H.n_beta, bonds, sites, 0)
        c.tda_prepare()
        return c

    out = {}
    c = prepared(H.h, H.eri, H.e_core)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    om, rs, e0, gam = c.sweep_tda_density(nroots, max_iter=200, eps=1e-9, allow_noconv=True,
                                          keep=TDA_KEEP * nroots, **TDA_KW)
    torch.cuda.synchronize()
    out["density_s_per_root"] = (time.perf_counter() - t0) / nroots
    out["omega"] = [float(x) for x in om]
    out["square_norm"] = [float(np.sum(gg * gg)) for gg in gam]
    out["resid"] = [float(x) for x in rs]
    d = np.random.default_rng(11).standard_normal((H.k, H.k))
    d = 0.5 * (d + d.T)
    v = prepared(d, None, 0.0)
    resp = []
    for w in (0.0, 0.5 * float(om[0])):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a, r2, sw = c.sweep_response(v, w, tol=1e-20, max_sweeps=80)
        torch.cuda.synchronize()
        resp.append({"omega": w, "alpha": a, "resid": [float(x) for x in r2], "sweeps": list(sw),
                     "s": time.perf_counter() - t0})
    out["response"] = resp
    c.close()
    v.close()
    out["note"] = ("square_norm = sum_pq gamma_pq^2 with gamma_pq = <Psi^mu| sum_sigma a+_p a_q |Psi0>; "
                   "response: X and Y components, site equations to sum |r|^2 < 1e-20")
    return out


def extras(pkg, ctx, device, S, stream, flush, args):
    """Side measurements, outside the timed steps."""
    import torch
    out = {}
    # (1) the mixed form on the same workload: every position, 6 vectors
    y64 = {i: S.ys[i].clone() for i in S.positions}
    M = SigmaStep(ctx, S.positions, {i: S.ds[i].numel() for i in S.positions}, S.nvec, S.nsite, device,
                  pkg.LRT_MIXED)
    for i in S.positions:
        M.xs[i].copy_(S.xs[i])
    step_ms, sigma_ms, _ = M.timed(stream, 3, 1, flush)
    err = max(float((M.ys[i] - y64[i]).abs().max() / y64[i].abs().max()) for i in S.positions)
    peak, note = tf32_peak()
    mx = M.flops / (statistics.mean(sigma_ms) * 1e-3) / 1e12
    out["mixed_same_workload"] = {
        "tflops": mx, "fp64_tflops_same_run": S.flops / 1e9 / statistics.mean(
            S.timed(stream, 2, 1, flush)[1]),
        "roofline": {"bound": "tensor", "achieved": mx, "peak": peak, "frac": mx / peak, "peak_note": note},
        "max_rel_err_vs_fp64": err, "ms_per_step": statistics.mean(step_ms)}
    del M
    # (2) the PPP polyene workload (12 sites, M = 256, two-site, 6 vectors), both precisions
    pctx, PH, ppos, psz, pnv = build_workload(pkg, device, 2, 2)
    res = {}
    for name, prec in (("fp64", pkg.LRT_FP64), ("mixed", pkg.LRT_MIXED)):
        P = SigmaStep(pctx, ppos, psz, pnv, 2, device, prec)
        st, sg, _ = P.timed(stream, 3, 1, flush)
        res[name] = {"tflops": P.flops / (statistics.mean(sg) * 1e-3) / 1e12, "ms_per_step": statistics.mean(st)}
        del P
    pctx.close()
    res["note"] = "diag + two-site sigma with 6 vectors at all 11 positions"
    out["ppp_k12_M256_twosite"] = res
    # (3) 32 independent instances (config 4 shapes), one-site sigma with 4 vectors at the
    # middle site of each: one grouped launch per phase (sigma_batched, CUDA graph replay)
    # against the same instances called one after another
    insts = []
    for b in range(32):
        cfg = synth.config(4, batch_index=b)
        H = cfg["ham"]
        i = H.k // 2 - 1
        m = synth.mixed_mps(H.k, H.n_alpha, H.n_beta, cfg["M"], 900 + b, center=i)
        c = pkg.Context(device)
        c.op_build(H.k, H.h, H.eri, e_core=H.e_core)
        c.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, i)
        for bb in range(i):
            c.renormalize(bb, +1)
        for bb in range(H.k - 1, i, -1):
            c.renormalize(bb, -1)
        n, _ = c.wfn_layout(i, 1)
        x = torch.tensor(synth.random_vector(n * 4, 3 + b), dtype=torch.float64, device=f"cuda:{device}")
        insts.append((c, i, x, torch.empty_like(x)))
    bctx = [a[0] for a in insts]
    bsite = [a[1] for a in insts]
    bx = [a[2] for a in insts]
    by = [a[3] for a in insts]
    batch = {"instances": 32, "nvec": 4, "nsite": 1}
    for name, prec in (("fp64", pkg.LRT_FP64), ("mixed", pkg.LRT_MIXED)):
        fl = 0.0
        for c, i, x, y in insts:
            c.sigma(i, 1, x, y, nvec=4, precision=prec)
            fl += c.stats()["flops"]
        pkg.sigma_batched(bctx, bsite, 1, bx, by, nvec=4, precision=prec)
        pkg.sigma_batched(bctx, bsite, 1, bx, by, nvec=4, precision=prec)
        seq = _timed(lambda: [c.sigma(i, 1, x, y, nvec=4, precision=prec) for c, i, x, y in insts], 3, stream)
        bat = _timed(lambda: pkg.sigma_batched(bctx, bsite, 1, bx, by, nvec=4, precision=prec), 5, stream)
        batch[name] = {"gflop": fl / 1e9, "sequential_ms": seq, "batched_ms": bat,
                       "sequential_tflops": fl / seq / 1e9, "batched_tflops": fl / bat / 1e9}
    for c in bctx:
        c.close()
    out["batch32_config4_onesite"] = batch
    # (4) TDA s/root at convergence, FP64 against the mixed form: the 8-orbital ab initio
    # workload (M = 64, 4 roots) and the PPP polyene (M = 256, 6 roots)
    out["tda_abinitio_k8_M64_4roots"] = _tda_converged(pkg, device, 1, [32, 64], 1e-9, 200)
    try:
        out["linear_response_k8_M64"] = _lr_k8(pkg, device)
    except Exception as e:
        out["linear_response_k8_M64"] = {"error": repr(e)}
    if not args.quick_tda:
        out["tda_ppp_k12_M256_6roots"] = _tda_converged(pkg, device, 2, [64, 128, 256], 1e-9, 200)
        try:
            out["tda_water_k24_M500_sweep_time"] = _tda_sweep_times(pkg, device)
        except Exception as e:   # a side measurement never costs the metric line
            out["tda_water_k24_M500_sweep_time"] = {"error": repr(e)}

    if args.tda_water:
        out["tda_water_k24_M500_6roots"] = _tda_converged(pkg, device, 3, [128, 256, 500], 1e-8, 200)
    return out


def _device_gb(device):
    import torch
    free, total = torch.cuda.mem_get_info(device)
    return (total - free) / 1e9


def fe2s2_sigma(pkg, device, stream):
    """The [2Fe-2S]-shaped workload (k = 36, 15a + 15b electrons, rank-200 factor, M = 1500):
    environments of the middle one-site position from random left/right-orthonormal MPS,
    then sigma with its 8 roots in FP64 and in the mixed form.  Two-electron integrals stay
    in factor form (the k^4 tensor is never formed)."""
    import torch
    cfg = synth.config(5, keep_eri=False)
    H = cfg["ham"]
    k, na, nb, M, nvec = H.k, H.n_alpha, H.n_beta, cfg["M"], cfg["nroots"]
    i = k // 2 - 1
    left = synth.random_mps(k, na, nb, M, 2024, "left")
    right = synth.random_mps(k, na, nb, M, 2025, "right")
    ctx = pkg.Context(device)
    try:
        ctx.op_build(k, H.h, None, B=H.B, e_core=H.e_core)
        ctx.mps_load(k, na, nb, left.bonds, left.sites, 0, sites_right=right.sites)
        del left, right
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b in range(i):
            ctx.renormalize(b, +1)
        for b in range(k - 1, i, -1):
            ctx.renormalize(b, -1)
        torch.cuda.synchronize()
        t_env = time.perf_counter() - t0
        n, _ = ctx.wfn_layout(i, 1)
        x = torch.tensor(synth.random_vector(n * nvec, 11), dtype=torch.float64, device=f"cuda:{device}")
        y = torch.empty_like(x)
        ym = torch.empty_like(x)
        ctx.sigma(i, 1, x, y, nvec=nvec)
        fl = ctx.stats()["flops"]
        t64 = _timed(lambda: ctx.sigma(i, 1, x, y, nvec=nvec), 3, stream)
        # H_eff is symmetric: <a, H b> = <H a, b> for the first two vectors
        a, b, ha, hb = x[:n], x[n:2 * n], y[:n], y[n:2 * n]
        sym = float((a @ hb - ha @ b).abs() / (a.norm() * hb.norm()))
        ctx.sigma(i, 1, x, ym, nvec=nvec, precision=pkg.LRT_MIXED)
        tmx = _timed(lambda: ctx.sigma(i, 1, x, ym, nvec=nvec, precision=pkg.LRT_MIXED), 3, stream)
        err = float((ym - y).abs().max() / y.abs().max())
        tf64, tfmx = fl / t64 / 1e9, fl / tmx / 1e9
        peak, note = tf32_peak()
        return {"site": i, "wfn_elements": n, "nvec": nvec, "gflop": fl / 1e9, "environment_build_s": t_env,
                "fp64_ms": t64, "fp64_tflops": tf64, "fp64_frac": tf64 / fp64_peak(None),
                "mixed_ms": tmx, "mixed_tflops": tfmx, "mixed_frac": tfmx / peak, "mixed_peak_note": note,
                "mixed_max_rel_err_vs_fp64": err, "symmetry_rel": sym, "device_gb": _device_gb(device)}
    finally:
        ctx.close()


def run_profile(args):
    """A short run for ncu: environments of the k = 24 water workload (bond dimension
    --profile-M) up to the middle one-site position, then one region between
    cudaProfilerStart and cudaProfilerStop: one sigma with the 6 vectors (fp64, mixed), or
    the enlargement and renormalization of the left block into the middle bond (gather)."""
    import torch
    import paper_1311_1646_gb300 as pkg
    device = 0
    torch.cuda.set_device(device)
    if args.profile == "tda":
        return run_profile_tda(pkg, device)
    cfg = synth.config(3)
    H = cfg["ham"]
    k, na, nb, nvec = H.k, H.n_alpha, H.n_beta, cfg["nroots"]
    M = args.profile_M or cfg["M"]
    left = synth.random_mps(k, na, nb, M, 2024, "left")
    right = synth.random_mps(k, na, nb, M, 2025, "right")
    ctx = pkg.Context(device)
    ctx.op_build(k, H.h, H.eri, e_core=H.e_core)
    ctx.mps_load(k, na, nb, left.bonds, left.sites, 0, sites_right=right.sites)
    i = k // 2 - 1
    for b in range(i - 1):
        ctx.renormalize(b, +1)
    for b in range(k - 1, i, -1):
        ctx.renormalize(b, -1)
    prec = pkg.LRT_MIXED if args.profile == "mixed" else pkg.LRT_FP64
    x = y = None
    if args.profile != "gather":
        ctx.renormalize(i - 1, +1)
        n, _ = ctx.wfn_layout(i, 1)
        x = torch.tensor(synth.random_vector(n * nvec, 5), dtype=torch.float64, device=f"cuda:{device}")
        y = torch.empty_like(x)
        ctx.sigma(i, 1, x, y, nvec=nvec, precision=prec)    # plans built outside the region
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    if args.profile == "gather":
        ctx.renormalize(i - 1, +1)
    else:
        ctx.sigma(i, 1, x, y, nvec=nvec, precision=prec)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    st = ctx.stats()
    print(json.dumps({"profile": args.profile, "M": M, "site": i, "device_gb": _device_gb(device),
                      "flops": st["flops"], "launches": st["launches"]}))
    ctx.close()


def run_profile_tda(pkg, device):
    """TDA sweeps of the PPP polyene (12 sites, 6a6b, M = 256, 6 roots) for ncu: the ground
    state on the GPU, two warm-up sweeps (plans and templates built), then three sweeps
    between cudaProfilerStart and cudaProfilerStop."""
    import torch
    cfg = synth.config(2)
    H = cfg["ham"]
    nr = cfg["nroots"]
    g = pkg.Context(device)
    g.op_build(H.k, H.h, H.eri, e_core=H.e_core)
    m = synth.random_mps(H.k, H.n_alpha, H.n_beta, 16, 3, "right")
    g.mps_load(H.k, H.n_alpha, H.n_beta, m.bonds, m.sites, 0)
    g.sweep_gs([64, 128, 256], max_sweeps=14, e_tol=1e-12, dav_tol=1e-10, onesite_sweeps=20)
    bonds, sites = g.mps_get()
    g.close()
    t = pkg.Context(device)
    t.op_build(H.k, H.h, H.eri, e_core=H.e_core)
    t.mps_load(H.k, H.n_alpha, H.n_beta, bonds, sites, 0)
    t.tda_prepare()
    kw = dict(eps=1e-9, allow_noconv=True, keep=TDA_KEEP * nr, **TDA_KW)
    t.sweep_tda(nr, max_iter=2, **kw)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    t.sweep_tda(nr, max_iter=3, **kw)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    torch.cuda.profiler.stop()
    print(json.dumps({"profile": "tda", "workload": "ppp_k12_M256_6roots", "sweeps": t.sweeps(), "wall_s": dt,
                      "device_gb": _device_gb(device)}))
    t.close()


def _oracle_setup(H, left, right, i, nsite):
    from oracle import blocks as ob
    from oracle import fock
    from oracle import mps as om
    t, v = fock.spin_integrals(H.h, H.eri)
    env = ob.Environment(H, t, v)
    k = H.k
    L = [om.unpack_site(left.sites[j], left.bonds[j], left.bonds[j + 1]) for j in range(k)]
    R = [om.unpack_site(right.sites[j], right.bonds[j], right.bonds[j + 1]) for j in range(k)]
    for b in range(i):
        env.grow_left(b, L[b])
    for b in range(k - 1, i + nsite - 1, -1):
        env.grow_right(b, R[b])
    return env


_CHILD = {}


def _child_sigma(seed):
    from oracle import blocks as ob
    from oracle import mps as om
    c = _CHILD
    w = om.unpack_site(synth.random_vector(c["n"], seed), c["lb"], c["rb"])
    ob.sigma_onesite(c["env"], c["i"], w)
    return seed


def cpu_baseline_child(spec):
    """Runs in a fresh process that never touches the GPU: the oracle's one-site sigma at the
    middle position of the workload, one vector per call, single-threaded and then with one
    forked worker per host core (the workers share the environment copy-on-write)."""
    import multiprocessing as mp
    from oracle import blocks as ob
    from oracle import mps as om
    cfg = synth.config(3)
    H = cfg["ham"]
    k, na, nb, M = H.k, H.n_alpha, H.n_beta, cfg["M"]
    left = synth.random_mps(k, na, nb, M, 2024, "left")
    right = synth.random_mps(k, na, nb, M, 2025, "right")
    i = spec["site"]
    t0 = time.perf_counter()
    env = _oracle_setup(H, left, right, i, 1)
    t_env = time.perf_counter() - t0
    n = synth.layout_size(synth.site_layout(left.bonds[i], left.bonds[i + 1]))
    _CHILD.update(env=env, i=i, n=n, lb=left.bonds[i], rb=left.bonds[i + 1])
    w = om.unpack_site(synth.random_vector(n, 7), left.bonds[i], left.bonds[i + 1])
    reps, t0 = 0, time.perf_counter()
    while True:
        ob.sigma_onesite(env, i, w)
        reps += 1
        if time.perf_counter() - t0 > spec["budget_s"] or reps >= 3:
            break
    dt1 = (time.perf_counter() - t0) / reps
    cores = os.cpu_count() or 1
    ctx = mp.get_context("fork")
    with ctx.Pool(cores) as pool:
        pool.map(_child_sigma, range(cores))           # warm the workers
        t0 = time.perf_counter()
        pool.map(_child_sigma, range(100, 100 + 2 * cores))
        dtp = time.perf_counter() - t0
    print(json.dumps({"env_s": t_env, "single_s": dt1, "single_reps": reps, "cores": cores,
                      "parallel_calls": 2 * cores, "parallel_s": dtp}))


def _host_cpu():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def cpu_baseline(site, flops_vec, budget_s=10.0):
    """The oracle timed on the host cores, in a child process (this one has used the GPU)."""
    spec = json.dumps({"site": site, "budget_s": budget_s})
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", spec],
                           capture_output=True, text=True, timeout=900, cwd=ROOT)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError) as e:
        return {"value": None, "unit": "TFLOP/s", "cores": None, "kind": "oracle", "error": repr(e)}
    single = flops_vec / d["single_s"] / 1e12
    allc = d["parallel_calls"] * flops_vec / d["parallel_s"] / 1e12
    return {"value": allc, "unit": "TFLOP/s", "cores": d["cores"], "kind": "oracle",
            "single_thread": {"value": single, "cores": 1, "reps": d["single_reps"]},
            "host_cores": os.cpu_count(), "host_cpu": _host_cpu(),
            "environment_build_s": d["env_s"],
            "sample": f"oracle one-site sigma at the middle position (i={site}) of the workload, one vector "
                      f"per call (the GPU step does 6 vectors at 24 positions): single-threaded "
                      f"{d['single_reps']} calls; all cores: {d['parallel_calls']} calls on {d['cores']} "
                      f"forked workers sharing the environment; environment built outside the timing; "
                      f"FLOPs = the GPU line's algorithmic count for the same call"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from oracle import blocks as ob
    from oracle import mps as om
    cfg = synth.config(3)
    H = cfg["ham"]
    k, na, nb, M, nvec = H.k, H.n_alpha, H.n_beta, cfg["M"], cfg["nroots"]
    left = synth.random_mps(k, na, nb, M, 2024, "left")
    right = synth.random_mps(k, na, nb, M, 2025, "right")
    i = k // 2 - 1
    env = _oracle_setup(H, left, right, i, 1)
    lay = synth.site_layout(left.bonds[i], left.bonds[i + 1])
    x = synth.random_vector(synth.layout_size(lay), 7)
    w = om.unpack_site(x, left.bonds[i], left.bonds[i + 1])
    for _ in range(args.warmup):
        ob.sigma_onesite(env, i, w)
    ob.FLOP_COUNTER[0] = 0.0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ob.sigma_onesite(env, i, w)
    dt = time.perf_counter() - t0
    flops = ob.FLOP_COUNTER[0]
    value = flops / dt / 1e12
    out = {"impl": "reference", "metric": "H_eff sigma TFLOP/s (algorithmic, FP64)", "value": value,
           "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "k": k, "electrons": na + nb, "M": M, "nsite": 1, "nvec": nvec},
           "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                            "sample": f"one step = oracle one-site sigma at the middle position (i={i}) for "
                                      "1 vector, single thread; FLOPs counted from the oracle's own block "
                                      "products; environment built before the timed steps"},
           "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    if len(sys.argv) > 2 and sys.argv[1] == "--oracle-child":
        cpu_baseline_child(json.loads(sys.argv[2]))
        sys.exit(0)
    a = parse()
    if a.profile:
        run_profile(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
