#!/usr/bin/env python
"""Benchmark: solves of the heat-equation KKT system to a 1e-8 relative residual on GB300.

One step = one full solve (x_0 = 0) of the 256 x 256, Nt = 1024, N_D = 64 FP64 problem
(nu = 1, omega = 1e-4, seeded random low-mode sine-series target): flexible GMRES(30) with the
block preconditioner whose Schur block is the two-level time-DD inverse, every step of it in
the library's CUDA kernels. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--omega W]

Multi-GPU: one process per GPU (torchrun); every rank solves its own replica (the path has no
exchange step on one instance here), the timing is the max over ranks, value = solves of all
ranks / time. --impl reference times the FP64 CPU oracle on a bounded sample of the same
workload, on rank 0 only.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "KKT solve time to 1e-8 rel. residual; precond applies/s; HBM GB/s vs peak"
TOL = 1e-8
MAXIT = 420
# Roofline denominators: HBM and BF16 from MEASURED_PEAKS.json (the measured copy and cuBLAS
# BF16 GEMM) when present, else the recipe's fallback; FP64 and FP32 from this run's FMA probe
# (kkt_probe_fma_rate) and TF32 from this run's cuBLAS TF32 GEMM (probe_peaks). Without a probe
# the FP64 peak falls back to the unit count: 2 DFMA per SM per clock x 152 SMs x 2070 MHz.
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12
FALLBACK_HBM_GBS = 6800.0
PROBE: dict = {}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            peaks, kind = json.load(fh), "measured"
    else:
        peaks, kind = {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"
    return dict(peaks, **PROBE), kind


def probe_peaks(kkt_mod) -> dict:
    """Measure the compute peaks of this GPU once per run (outside every timed region): FP64 and
    FP32 FMA loops of the library's probe, and cuBLAS dense GEMMs in TF32 (8192^3, best of 10)
    and FP64 (4096^3, best of 3), CUDA events. Stored in PROBE for measured_peaks()."""
    import torch

    if PROBE:
        return PROBE
    out = {"fp64_fma_tflops": kkt_mod.kkt_probe_fma_rate("fp64") / 1e12,
           "fp32_fma_tflops": kkt_mod.kkt_probe_fma_rate("fp32") / 1e12}
    stream = torch.cuda.current_stream()

    def gemm_rate(dtype, n, reps):
        a = torch.randn(n, n, dtype=dtype, device="cuda")
        b = torch.randn(n, n, dtype=dtype, device="cuda")
        c = torch.empty(n, n, dtype=dtype, device="cuda")
        torch.matmul(a, b, out=c)
        best = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.matmul(a, b, out=c)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b, c
        torch.cuda.empty_cache()
        return 2.0 * n ** 3 / (best / 1e3) / 1e12

    tf32_prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        out["tf32_tflops"] = gemm_rate(torch.float32, 8192, 10)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32_prev
    out["fp64_gemm_tflops"] = gemm_rate(torch.float64, 4096, 3)
    out["probe_how"] = ("FP64/FP32: kkt_probe_fma_rate (8 independent FMA chains per thread, 8 CTAs x 256 "
                        "threads per SM, best of 5); TF32: torch.matmul fp32 8192^3 with TF32 allowed, best of "
                        "10; FP64 GEMM: torch.matmul fp64 4096^3, best of 3")
    PROBE.update(out)
    return PROBE


def workload_for(omega: float) -> workloads.Workload:
    w = workloads.CFG_GPU
    return workloads.Workload(w.name, nx=w.nx, ny=w.ny, Nt=w.Nt, n_sub=w.n_sub, nu=w.nu, omega=omega,
                              target=w.target, seed=w.seed)


ORTH_CODE = {"mgs": 0, "cgs2": 1, "mgs2": 2, "mgs4": 3, "mgs8": 4}   # the library's enum kkt_orth
ORTH_TEXT = {
    0: "modified Gram-Schmidt",
    1: "classical Gram-Schmidt with one conditional repeat",
    2: "modified Gram-Schmidt over pairs of basis vectors",
    3: "modified Gram-Schmidt over blocks of four basis vectors",
    4: "modified Gram-Schmidt over blocks of eight basis vectors",
}


def describe(w: workloads.Workload, orth: int = 2) -> dict:
    return {"workload": f"plain FP64 KKT solve nx=ny={w.nx} Nt={w.Nt} N_D={w.n_sub} nu={w.nu} omega={w.omega:g}",
            "nx": w.nx, "ny": w.ny, "Nt": w.Nt, "n_sub": w.n_sub, "nu": w.nu, "omega": w.omega,
            "unknowns": 3 * w.V, "tol": TOL, "restart": 30, "coarse": "exact two-level, multiplicative",
            "residual_norm": "discrete L2 pair (u, z rows weighted h^-1/2, state rows h^1/2)",
            "orthogonalisation": ORTH_TEXT[orth],
            "l2": "inputs larger than L2 (KKT vector 1.6 GB, Krylov basis ~66 GB)"}


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, device, world: int) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's); x itself at N = 1."""
    if world <= 1:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, solves_per_rank: int, seconds: float) -> float:
    """Whole-job throughput: every rank's solves over the slowest rank's time (replicas)."""
    return world * solves_per_rank / seconds


# ---------------------------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------------------------

def oracle_iteration_sample(w: workloads.Workload, krylov_dim: int) -> tuple[float, str]:
    """Seconds of one FGMRES iteration of the FP64 oracle on the full workload, from a sample.

    Timed pieces, each scaled to the full iteration by the share it processed:
    RASQ sweeps of 4 of the N_D subdomains (x N_D/4), the per-mode coarse solve of the first
    4096 modes (x N/4096), S-hat x and K x on a 64-slice time window of the same grid and dt
    (x Nt/64), and the Gram-Schmidt work (2 passes of dots and updates against krylov_dim
    vectors, timed on the first eighth of each KKT vector (x 8); both vectors of that slice are
    far larger than the host caches, so its time grows in proportion to the length).
    """
    from oracle import problem, schwarz
    from oracle.problem import HeatKKT

    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    pre = schwarz.schur_preconditioner(p, w.n_sub, coarse_solver="per-mode")
    r = workloads.random_vector(p.V, 1)
    t = {}
    subs = pre.subs
    t0 = time.perf_counter()
    pre.subs = subs[:4]
    pre.rasq(r)
    pre.subs = subs
    t["rasq"] = (time.perf_counter() - t0) * (w.n_sub / 4)
    lim = min(4096, p.N)
    t0 = time.perf_counter()
    pre.coarse_per_mode(r, mode_limit=lim)
    t["coarse"] = (time.perf_counter() - t0) * (p.N / lim)
    win = 64
    pw = HeatKKT(nx=w.nx, ny=w.ny, Nt=win, T=p.dt * win, nu=w.nu, omega=w.omega)
    prew = schwarz.schur_preconditioner(pw, 4, variant="one-level")
    rw = workloads.random_vector(pw.V, 2)
    t0 = time.perf_counter()
    prew.schur_apply(rw)
    t["schur"] = (time.perf_counter() - t0) * (w.Nt / win)
    xw = workloads.random_vector(3 * pw.V, 3)
    t0 = time.perf_counter()
    problem.kkt_apply_blockwise(pw, xw)
    t["matvec"] = (time.perf_counter() - t0) * (w.Nt / win)
    frac = 8
    vecs = [workloads.random_vector(3 * p.V // frac, 10 + k) for k in range(2)]
    t0 = time.perf_counter()
    for _ in range(2 * krylov_dim):
        np.dot(vecs[0], vecs[1])
        vecs[1] -= 1e-3 * vecs[0]
    t["orth"] = (time.perf_counter() - t0) * 2 * frac
    sample = (f"one FGMRES iteration of the FP64 oracle at full size, sampled: RASQ on 4/{w.n_sub} subdomains, "
              f"coarse solve on {lim}/{p.N} modes, S-hat and K on a {win}/{w.Nt}-slice window, "
              f"CGS2 against {krylov_dim} vectors on 1/{frac} of each KKT vector; scaled to the whole iteration")
    return sum(t.values()), sample


def cpu_threads() -> int:
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count() or 1


def oracle_sample_one_thread(omega: float, krylov_dim: int) -> tuple[float | None, str]:
    """The same oracle sample in a child process with every BLAS/OpenMP pool at one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, bench; s, _ = bench.oracle_iteration_sample(bench.workload_for(%r), %d); "
            "print(json.dumps(s))" % (omega, krylov_dim))
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600,
                             cwd=os.path.dirname(os.path.abspath(__file__)))
        return float(out.stdout.strip().splitlines()[-1]), ""
    except Exception as e:   # reported, not fatal: the all-core figure stands on its own
        return None, f"{type(e).__name__}: {e}"


def error_vs_exact(w: workloads.Workload, x: np.ndarray, kmax: int = 8) -> dict:
    """Relative error of a solution x of the sine-series workload against the exact solution on
    its active modes k, l <= kmax (the right-hand side's modes; the oracle's per-mode banded
    solve), per block, and the content of x off those modes relative to each block."""
    from oracle import spectral
    from oracle.problem import HeatKKT

    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    ut = workloads.make_target(w)
    fu_hat = spectral.dst2(p.h * ut.reshape(-1), p)
    lam = spectral.mode_eigenvalues(p)
    zeros = np.zeros(w.Nt)
    exact = np.empty((3, w.Nt, kmax, kmax))
    for l in range(kmax):
        for k in range(kmax):
            exact[:, :, l, k] = spectral.kkt_exact_mode_solve(p, lam[l, k], fu_hat[:, l, k], zeros, zeros)
    out = {"modes": f"k, l <= {kmax}"}
    errs = []
    for b, name in enumerate("uzw"):
        xh = spectral.dst2(x[b * p.V:(b + 1) * p.V], p)
        err = float(np.linalg.norm(xh[:, :kmax, :kmax] - exact[b]) / np.linalg.norm(exact[b]))
        xh[:, :kmax, :kmax] = 0.0
        out[name] = {"rel_error": err, "off_mode_rel": float(np.linalg.norm(xh) / np.linalg.norm(exact[b]))}
        errs.append(err)
    out["max_block_rel_error"] = max(errs)
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workload_for(args.omega)
    iters = args.ref_iterations
    kdim = (iters % 30) // 2 + 1 if iters else 15
    per = []
    for step in range(args.warmup + args.steps):
        s, sample = oracle_iteration_sample(w, kdim)
        if step >= args.warmup:
            per.append(s * iters)
    solve_s = statistics.median(per)
    value = 1.0 / solve_s
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": solve_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(w, ORTH_CODE[args.orth or "mgs2"]), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample + f"; x {iters} iterations (the GPU solve's count on this "
                                                f"workload)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------

# DRAM traffic per algorithmic byte for kernels captured with ncu (dram__bytes_read.sum +
# dram__bytes_write.sum over the launch, divided by the launch's algorithmic bytes). The blocked
# (paired) MGS step, the FFT sine transform and the tensor-core transform GEMM come from
# single-pass captures of the benchmark workload itself; one-pass MGS from a capture of the
# 256 x 256, Nt = 96 case, whose traffic grows in proportion to the elements processed. Kernels
# not listed report traffic null.
TRAFFIC_RATIO = {"mgs_step_kernel": 0.952, "mgsb_step_kernel": 0.997, "dst_tile_kernel": 0.947,
                 "oz_gemm_kernel": 0.969}
# FP64 pipe busy fraction (sm__pipe_fp64_cycles_active, of peak sustained, active SMs) from the
# --set full captures of the 256 x 256, Nt = 96 case: context for an "alu" roofline whose
# achieved figure counts algorithmic FLOPs, not issued instructions.
FP64_PIPE_BUSY = {"dst_tile_kernel": [0.78, 0.82], "sweep_kernel": [0.85, 0.85], "matvec_kernel": [0.83, 0.83]}


def roofline(prof: dict, peaks: dict, peak_kind: str, precision: str = "fp64", orth: int = 2,
             dst_method: str = "tiles") -> dict:
    """Roofline of the kernel class with the largest device time in the timed region.

    The library sums, for every timed launch, the algorithmic FLOPs and bytes of that launch
    (what the method must compute and move; formulas at each launch site). The binding roof is
    the larger of FLOPs / compute peak and bytes / HBM peak; achieved = work / measured time.
    Compute peaks: FP64 the probe's measured FMA rate (else 2 DFMA/clk/SM x 152 SMs x 2070 MHz
    from the unit counts); BF16 the measured dense GEMM burst; TF32 the probe's measured cuBLAS
    TF32 GEMM (else the BF16 figure x 1.1/2.25, the nominal dense ratio).
    """
    top = max(prof, key=lambda k: prof[k]["ms"])
    e = prof[top]
    sec = e["ms"] / 1e3
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    if top == "dst" and (precision in ("bf16", "tf32") or dst_method == "tensor"):
        bf = float(peaks.get("bf16_tflops", 1900.0))
        if precision == "fp64":   # FP64 transforms as BF16 digit-plane products on the tensor cores
            alu_peak, alu_src = bf, f"{peak_kind} BF16 dense GEMM (digit-plane products)"
        elif precision == "bf16":
            alu_peak, alu_src = bf, f"{peak_kind} BF16 dense GEMM"
        elif "tf32_tflops" in peaks:
            alu_peak, alu_src = float(peaks["tf32_tflops"]), "measured cuBLAS TF32 dense GEMM (this run's probe)"
        else:
            alu_peak, alu_src = bf * 1.1 / 2.25, f"{peak_kind} BF16 dense GEMM x 1.1/2.25 (TF32)"
        alu_kind = "tensor"
        kname = "oz_gemm_kernel" if precision == "fp64" else "tc_dst_gemm_kernel"
    else:
        if "fp64_fma_tflops" in peaks:
            alu_peak = float(peaks["fp64_fma_tflops"])
            alu_src = "measured FP64 FMA rate (this run's kkt_probe_fma_rate)"
        else:
            alu_peak = FP64_PEAK_TFLOPS
            alu_src = "derived: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (FP64)"
        alu_kind = "alu"
        gs = {0: "mgs_step_kernel", 1: "update_norm_kernel"}.get(orth, "mgsb_step_kernel")
        kname = {"dst": "dst_tile_kernel", "multidot": gs if orth != 1 else "multidot_kernel", "update": gs,
                 "axpy": "axpy_multi_kernel" if precision == "fp64" else "scale2_kernel",
                 "pack": "pack_kernel", "matvec": "matvec_kernel", "sweep": "sweep_kernel",
                 "coarse": "coarse_solve_kernel"}.get(top, top)
    t_alu = e["flops"] / (alu_peak * 1e12)
    t_mem = e["bytes"] / (hbm * 1e9)
    per_launch = e["ms"] / max(e["timed"], 1)
    if t_alu >= t_mem:
        ach = e["flops"] / sec / 1e12
        out = {"kernel": kname, "bound": alu_kind, "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
               "frac": ach / alu_peak, "peak_source": alu_src}
    else:
        ach = e["bytes"] / sec / 1e9
        out = {"kernel": kname, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
               "peak_source": f"{peak_kind} HBM copy"}
    bytes_per_launch = e["bytes"] / max(e["timed"], 1)
    if kname in FP64_PIPE_BUSY and alu_kind == "alu":
        out["fp64_pipe_busy_ncu"] = FP64_PIPE_BUSY[kname]
    ratio = TRAFFIC_RATIO.get(kname)
    out.update({"traffic": bytes_per_launch * ratio if ratio else None,
                "traffic_source": ("ncu dram bytes / algorithmic bytes of the same kernel, times this launch's "
                                   "algorithmic bytes" if ratio else None),
                "per_launch_ms": per_launch, "launches": e["timed"],
                "algorithmic_flops_per_launch": e["flops"] / max(e["timed"], 1),
                "algorithmic_bytes_per_launch": e["bytes"] / max(e["timed"], 1),
                "hbm_gbs_algorithmic": e["bytes"] / sec / 1e9, "share_of_step": e["ms"] / sum(v["ms"] for v in prof.values())})
    return out


def time_applies(kkt_mod, solver, V: int, reps: int, dev) -> dict:
    """Standalone P^-1 applies (kkt_precond_apply on a full KKT vector), CUDA events on the
    launching stream. Algorithmic traffic 48 V bytes per apply (3 blocks in, 3 out)."""
    import torch

    r = torch.randn(3 * V, dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(7))
    y = torch.empty_like(r)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        solver.precond_apply(r, out=y)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        solver.precond_apply(r, out=y)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    peaks, kind = measured_peaks()
    gbs = 48.0 * V / (ms / 1e3) / 1e9
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    del r, y
    return {"ms": ms, "applies_per_s": 1e3 / ms, "algorithmic_bytes": 48 * V, "hbm_gbs": gbs,
            "hbm_frac": gbs / hbm, "peak_gbs": hbm, "peak_source": f"{kind} HBM copy"}


def time_solves(kkt_mod, solver, f, steps: int, warmup: int):
    import torch

    x = torch.zeros_like(f)
    for _ in range(warmup):
        x.zero_()
        solver.solve(f, x, tol=TOL, maxit=MAXIT)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = None
    for _ in range(steps):
        x.zero_()
        res = solver.solve(f, x, tol=TOL, maxit=MAXIT)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, res, x


def measure_forms(kkt_mod, dev, steps: int, warmup: int) -> dict:
    """Time to a 1e-8 (weighted) solve of the 512 x 512, Nt = 512, N_D = 64 mixed workload in
    each arithmetic form on this GPU, plus its standalone preconditioner apply."""
    import torch

    w = workloads.CFG_MIXED
    ut = torch.from_numpy(workloads.make_target(w).ravel()).to(dev)
    out = {"workload": f"nx=ny={w.nx} Nt={w.Nt} N_D={w.n_sub} nu={w.nu} omega={w.omega:g}, sine-series target"}
    ref_x = None
    for form in ("fp64", "bf16", "tf32", "bf16_single", "tf32_single"):
        prec = form.split("_")[0]
        s = kkt_mod.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, precision=prec,
                           tc_split=not form.endswith("_single"))
        f = s.build_rhs(ut)
        ms, res, x = time_solves(kkt_mod, s, f, steps, warmup)
        kkt_mod.kkt_profile_read(reset=True)
        kkt_mod.kkt_profile_enable(True)
        apply_stats = time_applies(kkt_mod, s, s.V, 5, dev)
        kkt_mod.kkt_profile_enable(False)
        prof = kkt_mod.kkt_profile_read(reset=True)
        peaks, kind = measured_peaks()
        apply_stats["dominant_kernel_roofline"] = roofline(prof, peaks, kind, prec)
        apply_stats["kernel_ms_per_apply"] = {k: round(v["ms"] / 8, 4) for k, v in prof.items() if v["ms"] > 0}
        entry = {"solve_ms": ms, "iterations": res.iterations, "rel_residual": res.rel_residual,
                 "converged": res.status == kkt_mod.KKT_OK, "precond_apply": apply_stats}
        if prec == "fp64":
            ref_x = x.clone()
        else:
            entry["solution_rel_diff_vs_fp64"] = float(torch.linalg.vector_norm(x - ref_x) / torch.linalg.vector_norm(ref_x))
            entry["transform_operands"] = "single BF16/TF32" if form.endswith("_single") else "hi + lo split (3 products)"
        out[form] = entry
        del f, x
        s.close()
        torch.cuda.empty_cache()
    out["speedup_vs_fp64"] = {p: out["fp64"]["solve_ms"] / out[p]["solve_ms"]
                              for p in ("bf16", "tf32", "bf16_single", "tf32_single")}
    return out


def measure_variants(kkt_mod, dev, w: workloads.Workload, physical_ms: float, steps: int, warmup: int) -> dict:
    """The headline workload's solve in the other configurations: the spectral basis (f and x
    transformed once, no transforms inside the iteration), one-pass MGS and CGS2 (the paired-MGS
    default's alternatives), RAS local solves (Eq 9, an ablation), and the multilevel
    (cyclic-reduction) coarse solve in place of block Thomas. Same tolerance, x_0 = 0, device
    time per solve."""
    import torch

    ut = torch.from_numpy(workloads.make_target(w).ravel()).to(dev)
    out = {}
    for name, opts in (("spectral_basis", {"basis": "spectral"}), ("mgs", {"orth": "mgs"}), ("cgs2", {"orth": "cgs2"}),
                       ("mgs2", {"orth": "mgs2"}), ("mgs4", {"orth": "mgs4"}), ("mgs8", {"orth": "mgs8"}),
                       ("ras_local_solves", {"local": "ras"}), ("coarse_cyclic", {"coarse_solve": "cyclic"})):
        s = kkt_mod.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, **opts)
        f = s.build_rhs(ut)
        ms, res, x = time_solves(kkt_mod, s, f, steps, warmup)
        out[name] = {"solve_ms": ms, "solves_per_s": 1e3 / ms, "iterations": res.iterations,
                     "rel_residual": res.rel_residual, "converged": res.status == kkt_mod.KKT_OK,
                     "speedup_vs_headline": physical_ms / ms}
        del f, x
        s.close()
        torch.cuda.empty_cache()
    return out


def measure_batched(kkt_mod, dev) -> dict:
    """The 64 uneven instances of the batched workload (sizes 64^2..256^2, Nt 128..1024, N_D
    8..64, spread nu and omega): one batched solve (memory waves, one launch per phase over all
    running instances, graph replay; instances of at least 2^20 unknowns per block, which fill
    the GPU alone, take the single-solve path) against the same instances solved one after
    another with kkt_solve, in the physical basis and in the spectral basis; also every
    instance forced through the batched kernels. All to the same 1e-8 weighted
    tolerance from x_0 = 0; device time of the solve calls only (CUDA events), inputs
    resident; the batched value is the second call (the first also autotunes)."""
    import torch

    ws = workloads.batched_instances(64, seed=3)
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    fs = []
    for w in ws:
        s = kkt_mod.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub)
        fs.append(s.build_rhs(torch.from_numpy(workloads.make_target(w).ravel()).to(dev)))
        s.close()
    out = {"workload": "64 uneven instances: nx=ny in {64,128,256}, Nt in {128..1024}, N_D in {8..64}, "
                       "nu in [0.1,10], omega in [1e-6,1e-2] (log-uniform), seed 3",
           "instances": len(ws), "unknowns_total": sum(3 * w.V for w in ws)}
    for basis in ("physical", "spectral"):
        seq_ms, seq_its = 0.0, []
        for w, f in zip(ws, fs):
            s = kkt_mod.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, basis=basis)
            x = torch.zeros_like(f)
            ms, r = timed(lambda: s.solve(f, x, tol=TOL, maxit=MAXIT))
            seq_ms += ms
            seq_its.append(r.iterations if r.status == kkt_mod.KKT_OK else -1)
            del x
            s.close()
            torch.cuda.empty_cache()
        b = kkt_mod.Batch(ws, basis=basis)
        runs = []
        for _ in range(2):
            xs = [torch.zeros_like(f) for f in fs]
            runs.append(timed(lambda: b.solve(fs, xs, tol=TOL, maxit=MAXIT)))
            del xs
        # every instance through the batched kernels (no single-solve dispatch), for comparison
        b.set_single_threshold(0)
        xs = [torch.zeros_like(f) for f in fs]
        all_ms, all_res = timed(lambda: b.solve(fs, xs, tol=TOL, maxit=MAXIT))
        del xs
        b.close()
        torch.cuda.empty_cache()
        ms, res = runs[1]
        its = res.iterations
        out[basis] = {
            "batched": {"solves_per_s": len(ws) / (ms / 1e3), "time_ms": ms, "first_call_ms": runs[0][0],
                        "solo_instances": res.solo,
                        "all_batched_solves_per_s": len(ws) / (all_ms / 1e3), "all_batched_waves": all_res.waves,
                        "waves": res.waves, "graphs": res.graphs, "graph_launches": res.graph_launches,
                        "tile_lines": res.tile_lines, "sweep_block": res.sweep_block,
                        "tune_ms_dst_tl8_16_32": res.tune_ms_dst, "tune_ms_sweep_tb64_128_256": res.tune_ms_sweep,
                        "iterations_min_median_max": [min(its), int(np.median(its)), max(its)],
                        "all_converged": all(st == kkt_mod.KKT_OK for st in res.statuses)},
            "sequential": {"solves_per_s": len(ws) / (seq_ms / 1e3), "time_ms": seq_ms,
                           "all_converged": all(i >= 0 for i in seq_its)},
            "iteration_count_mismatches_gt1": sum(1 for a, c in zip(its, seq_its) if abs(a - c) > 1),
            "speedup_batched_vs_sequential": seq_ms / ms}
    del fs
    torch.cuda.empty_cache()
    # the batched form's own regime: many small instances, where one instance cannot fill the
    # GPU and one-after-another solves are bound by launches and host round trips
    rng = np.random.Generator(np.random.PCG64(6))
    small = [workloads.Workload(f"small{q}", nx=int(n), ny=int(n), Nt=int(nt), n_sub=int(nt) // 8,
                                nu=float(10 ** rng.uniform(-1, 1)), omega=float(10 ** rng.uniform(-6, -2)),
                                target="sine-series", seed=2000 + q)
             for q, (n, nt) in enumerate(zip(rng.choice([16, 32, 64], 128), rng.choice([32, 64, 128], 128)))]
    fsm = []
    for w in small:
        s = kkt_mod.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub)
        fsm.append(s.build_rhs(torch.from_numpy(workloads.make_target(w).ravel()).to(dev)))
        s.close()
    seq_ms = 0.0
    for w, f in zip(small, fsm):
        s = kkt_mod.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub)
        x = torch.zeros_like(f)
        ms, _ = timed(lambda: s.solve(f, x, tol=TOL, maxit=MAXIT))
        seq_ms += ms
        s.close()
    b = kkt_mod.Batch(small)
    runs = [timed(lambda: b.solve(fsm, [torch.zeros_like(f) for f in fsm], tol=TOL, maxit=MAXIT)) for _ in range(2)]
    b.close()
    ms, res = runs[1]
    out["small_instances"] = {
        "workload": "128 instances: nx=ny in {16,32,64}, Nt in {32,64,128}, N_D = Nt/8, nu, omega log-uniform (seed 6)",
        "batched_solves_per_s": len(small) / (ms / 1e3), "sequential_solves_per_s": len(small) / (seq_ms / 1e3),
        "speedup_batched_vs_sequential": seq_ms / ms, "waves": res.waves, "graphs": res.graphs,
        "all_converged": all(st == kkt_mod.KKT_OK for st in res.statuses)}
    return out


def measure_learned(kkt_mod, dev) -> dict:
    """Learned-vs-plain comparison on the 256 x 256, Nt = 2048, N_D = 256 workload (m = 8): the
    network (in 2 N_D + 2 -> 512 -> 512 -> 2 N_D, ReLU) is trained on the GPU on exact coarse
    solves of modes k, l < 32 with (nu, omega) drawn log-uniform from [0.1, 10] x [1e-6, 1e-2],
    first on the squared error to the unit target and then on the coarse residual after the
    minimal-residual step (the guard's quantity). Every form then solves the same seeded
    right-hand side to 1e-8 from x_0 = 0: one-level RASQ, the exact two-level method, the learned
    coarse correction (guarded, exact fallback), the network alone (no guard, no fallback), the
    ablation (no coarse correction on the learned modes), and TF32 transforms with the exact and
    the learned coarse level. Cases: the workload's own (nu, omega) = (1, 1e-4) and one held-out
    pair (seed 5). A second network trained on the squared error alone (the earlier objective)
    gives the guarded and network-only counts before the residual phase."""
    import torch

    w0 = workloads.CFG_LEARNED
    rng = np.random.Generator(np.random.PCG64(5))
    nu_h, om_h = float(10 ** rng.uniform(-1, 1)), float(10 ** rng.uniform(-6, -2))
    cases = [w0, workloads.Workload("held-out", nx=w0.nx, ny=w0.ny, Nt=w0.Nt, n_sub=w0.n_sub, nu=nu_h, omega=om_h,
                                    target=w0.target, seed=5)]

    def train(**over):
        net = kkt_mod.Mlp(**over)
        t0 = time.perf_counter()
        st = net.train()
        info = {"seconds": time.perf_counter() - t0, "samples": st.samples, "adam_steps": st.steps,
                "epochs_unit_direction": net.cfg.epochs, "epochs_coarse_residual": net.cfg.resid_epochs,
                "final_train_loss": st.final_train_loss, "val_loss": st.val_loss, "val_cosine": st.val_cosine,
                "val_coarse_residual": st.val_resid, "val_within_guard": st.val_within_guard,
                "modes_learned": f"k, l < {net.cfg.modes}", "width": net.cfg.width}
        return net, info

    net, info = train()
    out = {"workload": f"nx=ny={w0.nx} Nt={w0.Nt} N_D={w0.n_sub}, sine-series targets", "training": info}
    forms = [("one_level", "fp64", "none", None), ("exact", "fp64", "exact", None),
             ("learned", "fp64", "learned", "learned"), ("network_only", "fp64", "learned", "network"),
             ("learned_ablation", "fp64", "learned", "none"),
             ("tf32_exact", "tf32", "exact", None), ("tf32_learned", "tf32", "learned", "learned")]
    stream = torch.cuda.current_stream()

    def solve_form(w, ut, network, prec, coarse, mode):
        s = kkt_mod.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, precision=prec)
        if mode is not None:
            s.attach_mlp(network, mode)
        s.set_options(precision=prec, coarse=coarse)
        f = s.build_rhs(ut)
        x = torch.zeros_like(f)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = s.solve(f, x, tol=TOL, maxit=MAXIT)
        e1.record(stream)
        torch.cuda.synchronize()
        entry = {"iterations": r.iterations, "solve_ms": e0.elapsed_time(e1),
                 "converged": r.status == kkt_mod.KKT_OK, "rel_residual": r.rel_residual}
        if mode == "learned":
            kept, fb = s.learned_stats()
            entry["learned_corrections_kept"] = kept
            entry["exact_fallbacks"] = fb
            entry["kept_fraction"] = kept / max(kept + fb, 1)
        elif mode == "network":
            applied, beyond = s.learned_stats()
            entry["network_corrections_applied"] = applied
            entry["beyond_guard"] = beyond
            entry["within_guard_fraction"] = 1.0 - beyond / max(applied, 1)
        del f, x
        s.close()
        torch.cuda.empty_cache()
        return entry

    for w in cases:
        ut = torch.from_numpy(workloads.make_target(w).ravel()).to(dev)
        res_case = {"nu": w.nu, "omega": w.omega}
        for name, prec, coarse, mode in forms:
            res_case[name] = solve_form(w, ut, net, prec, coarse, mode)
        base = res_case["exact"]["solve_ms"]
        res_case["time_vs_exact_fp64"] = {k: res_case[k]["solve_ms"] / base for k, *_ in forms}
        out["case_" + ("workload" if w is w0 else "held_out")] = res_case
    net.close()
    # the same network trained on the unit-direction error alone (no coarse-residual phase)
    net0, info0 = train(resid_epochs=0)
    ut = torch.from_numpy(workloads.make_target(w0).ravel()).to(dev)
    out["unit_direction_only"] = {"training": info0,
                                  "learned": solve_form(w0, ut, net0, "fp64", "learned", "learned"),
                                  "network_only": solve_form(w0, ut, net0, "fp64", "learned", "network")}
    net0.close()
    return out


def run_study(args):
    """Section 4's experiment on this GPU: one-level RASQ against the two-level preconditioner,
    iterations of FGMRES(30) to a 1e-6 relative residual (max 420) on the paper's problem:
    (0,1) x (0,2), 17 x 17 mesh points, T = 1, nu = 1, u_0 = -x y (x-1)(y-2),
    u~ = sin 2 pi t sin 2 pi x sin 2 pi y (Eq 16). Figure 1: Nt = 100 .. 3200 with 80, 20 and 5
    steps per subdomain (N_D = Nt / m rounded, at least 1) and omega in {1e-2, 1e-3, 1e-4};
    Figure 2: omega = 1e-2 .. 1e-6 at Nt = 800 with 40 subdomains; the mesh sweep of the text
    (9, 17, 33 points). At omega = 1e-4 Figure 1's cases are also solved with RAS local solves
    (Eq 9, the explicit local Schur complements) in place of RASQ, one- and two-level. The
    residual is the unweighted Euclidean ||f - K x|| / ||f|| (its rounding floor is far below
    1e-6 at these sizes). One JSON line on stdout."""
    import torch

    import paper_2305_04421_gb300.kkt as kkt

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)

    def iterations(nx, Nt, n_sub, omega, coarse, local="rasq"):
        w = workloads.Workload("paper", nx=nx, ny=nx, Nt=Nt, n_sub=n_sub, Lx=1.0, Ly=2.0, omega=omega,
                               target="paper", u0="paper")
        s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, coarse=coarse, residual_norm="euclidean",
                       local=local, Lx=1.0, Ly=2.0)
        f = s.build_rhs(torch.from_numpy(workloads.make_target(w).ravel()).to(dev),
                        torch.from_numpy(workloads.make_u0(w).ravel()).to(dev))
        r = s.solve(f, tol=1e-6, maxit=420)
        s.close()
        return r.iterations if r.status == kkt.KKT_OK else None   # None: not converged in 420

    t0 = time.perf_counter()
    fig1 = []
    for omega in (1e-2, 1e-3, 1e-4):
        for m in (80, 20, 5):
            for Nt in (100, 200, 400, 800, 1600, 3200):
                nd = max(1, round(Nt / m))
                row = {"omega": omega, "steps_per_subdomain": m, "Nt": Nt, "n_sub": nd,
                       "one_level": iterations(16, Nt, nd, omega, "none"),
                       "two_level": iterations(16, Nt, nd, omega, "exact")}
                if omega == 1e-4:   # the RAS ablation (Eq 9 local solves) on one omega
                    row["ras_one_level"] = iterations(16, Nt, nd, omega, "none", "ras")
                    row["ras_two_level"] = iterations(16, Nt, nd, omega, "exact", "ras")
                fig1.append(row)
    fig2 = [{"omega": om, "Nt": 800, "n_sub": 40, "one_level": iterations(16, 800, 40, om, "none"),
             "two_level": iterations(16, 800, 40, om, "exact")} for om in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6)]
    mesh = [{"mesh_points": nx + 1, "Nt": 400, "n_sub": 20, "omega": 1e-4,
             "one_level": iterations(nx, 400, 20, 1e-4, "none"), "two_level": iterations(nx, 400, 20, 1e-4, "exact")}
            for nx in (8, 16, 32)]
    # the coarse solver on the paper's mesh (225 modes): block Thomas against the multilevel
    # (cyclic-reduction) hierarchy, both exact; wall time per solve after one warm-up solve
    def timed(Nt, n_sub, solver, breakdown=False):
        w = workloads.Workload("paper", nx=16, ny=16, Nt=Nt, n_sub=n_sub, Lx=1.0, Ly=2.0, omega=1e-4,
                               target="paper", u0="paper")
        s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, residual_norm="euclidean", Lx=1.0, Ly=2.0,
                       coarse_solve=solver)
        f = s.build_rhs(torch.from_numpy(workloads.make_target(w).ravel()).to(dev),
                        torch.from_numpy(workloads.make_u0(w).ravel()).to(dev))
        s.solve(f, tol=1e-6, maxit=420)
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = s.solve(f, tol=1e-6, maxit=420)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t) * 1e3
        kern = None
        if breakdown:   # device time per kernel class over one more solve (events around each launch)
            kkt.kkt_profile_read(reset=True)
            kkt.kkt_profile_enable(True)
            s.solve(f, tol=1e-6, maxit=420)
            torch.cuda.synchronize()
            kkt.kkt_profile_enable(False)
            kern = {k: {"ms": round(v["ms"], 3), "launches": v["launches"]}
                    for k, v in kkt.kkt_profile_read(reset=True).items() if v["launches"]}
        s.close()
        return r.iterations, ms, kern

    # wall time per solve on the paper's mesh, m = 5 (N_D = Nt / 5): the time-parallel weak scaling
    # on one GPU, with the sequential (Thomas) and the multilevel (cyclic) coarse solve
    coarse_solvers = []
    for Nt in (100, 200, 400, 800, 1600, 3200):
        nd = Nt // 5
        it_t, ms_t, _ = timed(Nt, nd, "thomas")
        it_c, ms_c, kern = timed(Nt, nd, "cyclic", breakdown=Nt == 3200)
        row = {"Nt": Nt, "n_sub": nd, "iterations": [it_t, it_c], "thomas_ms": ms_t, "cyclic_ms": ms_c,
               "cyclic_ms_per_iteration": ms_c / max(it_c, 1), "speedup": ms_t / ms_c}
        if kern:
            row["cyclic_kernel_ms"] = kern
        coarse_solvers.append(row)
    # every two-level solve of Figures 1 and 2 (59 instances of uneven Nt, N_D and omega) as one
    # batched call, against the same solves one after another; wall time with the device idle
    # before and after, inputs resident
    cases = [(r["Nt"], r["n_sub"], r["omega"]) for r in fig1] + [(r["Nt"], r["n_sub"], r["omega"]) for r in fig2]
    ws = [workloads.Workload("paper", nx=16, ny=16, Nt=Nt, n_sub=nd, Lx=1.0, Ly=2.0, omega=om, target="paper",
                             u0="paper") for Nt, nd, om in cases]
    fs, seq_ms, seq_its = [], 0.0, []
    for w in ws:
        s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, residual_norm="euclidean", Lx=1.0, Ly=2.0)
        f = s.build_rhs(torch.from_numpy(workloads.make_target(w).ravel()).to(dev),
                        torch.from_numpy(workloads.make_u0(w).ravel()).to(dev))
        s.solve(f, tol=1e-6, maxit=420)
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = s.solve(f, tol=1e-6, maxit=420)
        torch.cuda.synchronize()
        seq_ms += (time.perf_counter() - t) * 1e3
        seq_its.append(r.iterations)
        fs.append(f)
        s.close()
    b = kkt.Batch(ws, residual_norm="euclidean", Lx=1.0, Ly=2.0)
    for rep in range(2):   # the first call also autotunes and captures its graphs
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = b.solve(fs, tol=1e-6, maxit=420)
        torch.cuda.synchronize()
        b_ms = (time.perf_counter() - t) * 1e3
    b.close()
    batched = {"instances": len(ws), "sequential_ms": seq_ms, "batched_ms": b_ms, "speedup": seq_ms / b_ms,
               "waves": res.waves, "graphs": res.graphs,
               "iteration_mismatches_gt1": sum(abs(a - c) > 1 for a, c in zip(res.iterations, seq_its)),
               "all_converged": all(st == kkt.KKT_OK for st in res.statuses)}
    two = [r["two_level"] for r in fig1 + fig2 if r["two_level"] is not None]
    print(json.dumps({"study": "Section 4 replication (Eq 16 problem): one-level vs two-level FGMRES iterations",
                      "tol": 1e-6, "maxit": 420, "seconds": time.perf_counter() - t0,
                      "two_level_iterations_min_max": [min(two), max(two)],
                      "fig1": fig1, "fig2": fig2, "mesh": mesh, "coarse_solvers": coarse_solvers,
                      "batched_two_level": batched}))
    return 0


def run_coarse_study(args):
    """kkt_coarse_apply (R_0^T S_0^-1 R_0 r: forward 2D DST, restriction, coarse solve,
    prolongation, inverse DST) with the two coarse solvers, across mode counts and N_D; device
    time per call (CUDA events over 20 calls after 3). One JSON line per case."""
    import torch

    import paper_2305_04421_gb300.kkt as kkt

    torch.cuda.set_device(0)
    for nx, Nt, nd in [(16, 3200, 640), (16, 800, 160), (16, 400, 80), (16, 100, 20), (32, 1024, 64),
                       (64, 1024, 64), (96, 1024, 64), (128, 1024, 64), (160, 1024, 64), (256, 1024, 64),
                       (64, 4096, 820), (128, 2048, 410)]:
        s = kkt.Solver(nx, nx, Nt, 1.0, 1.0, 1e-4, nd, coarse_solve="thomas")
        r = torch.randn(s.V, dtype=torch.float64, device="cuda")
        y = torch.empty_like(r)
        row = {"nx": nx, "Nt": Nt, "n_sub": nd, "modes": (nx - 1) ** 2}
        for solver in ("thomas", "cyclic"):
            s.set_options(coarse_solve=solver)
            for _ in range(3):
                s.coarse_apply(r, out=y)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                s.coarse_apply(r, out=y)
            e1.record()
            torch.cuda.synchronize()
            row[solver + "_us"] = e0.elapsed_time(e1) / 20 * 1e3
        s.close()
        print(json.dumps(row), flush=True)
    return 0


def run_profile_case(args):
    """A small solve for counter captures, two solves; prints the iteration count. 'grid':
    256 x 256, Nt = 96, N_D = 8 (a KKT vector of 150 MB, above the 126 MB L2), FGMRES(10) to
    1e-8. 'paper': Section 4's mesh with Nt = 3200 and 640 subdomains, FGMRES(30) to 1e-6."""
    import torch

    import paper_2305_04421_gb300.kkt as kkt

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    if args.profile_case == "tensor":
        # the tensor-core FP64 transform alone: 256 x 256, Nt = 64 (16,320 lines of 255 points,
        # 50 MB of digit planes), three 2D transforms of a seeded random block
        n, Nt = 256, 64
        s = kkt.Solver(n, n, Nt, 1.0, 1.0, 1e-4, 1)
        s.set_dst_method("tensor")
        x = torch.from_numpy(workloads.random_vector((n - 1) ** 2 * Nt, 1)).to(dev)
        for _ in range(3):
            y = s.dst2d(x)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "tensor-core FP64 2D transform 256x256 Nt=64",
                          "finite": bool(torch.isfinite(y).all())}))
        s.close()
        return 0
    if args.profile_case == "batched":
        # two 128 x 128, Nt = 128, N_D = 16 instances (KKT vectors of 48 MB, a 1.5 GB Krylov basis
        # each) solved one after another and then together through the batched kernels (graphs
        # off, so that every kernel is a launch of its own)
        ws = [workloads.Workload(f"profile-batch{q}", nx=128, ny=128, Nt=128, n_sub=16, nu=1.0 + q,
                                 omega=1e-4, target="sine-series", seed=10 + q) for q in range(2)]
        fs = []
        for w in ws:
            s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub)
            fs.append(s.build_rhs(torch.from_numpy(workloads.make_target(w).ravel()).to(dev)))
            r = s.solve(fs[-1], tol=1e-8, maxit=200)
            s.close()
        b = kkt.Batch(ws)
        b.set_single_threshold(0)
        b.set_graphs(False)
        res = b.solve(fs, [torch.zeros_like(f) for f in fs], tol=1e-8, maxit=200)
        b.close()
        print(json.dumps({"profile_case": "2 instances 128x128 Nt=128 N_D=16, single then batched",
                          "iterations": res.iterations[:2], "status": res.status}))
        return 0 if res.status == kkt.KKT_OK and r.status == kkt.KKT_OK else 1
    if args.profile_case == "paper":
        # the Eq 16 problem on the 17 x 17 mesh, 5 steps per subdomain: 225 modes, so the coarse
        # solve runs the multilevel (cyclic-reduction) kernel
        w = workloads.Workload("profile-paper", nx=16, ny=16, Nt=3200, n_sub=640, Lx=1.0, Ly=2.0, omega=1e-4,
                               target="paper", u0="paper")
        s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, residual_norm="euclidean", Lx=1.0, Ly=2.0)
        # the thread-per-line transform (what the create-time timing picks here without a
        # profiler; under one, every launch is slower and the choice can change)
        s.set_dst_method("lane")
        f = s.build_rhs(torch.from_numpy(workloads.make_target(w).ravel()).to(dev),
                        torch.from_numpy(workloads.make_u0(w).ravel()).to(dev))
        tol, name = 1e-6, "Eq 16 problem 16x16 intervals Nt=3200 N_D=640 restart=30 fp64, thread-per-line DST"
    else:
        w = workloads.Workload("profile", nx=256, ny=256, Nt=96, n_sub=8, target="sine-series", seed=1)
        s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, restart=10, basis=args.basis,
                       precision=args.precision)
        f = s.build_rhs(torch.from_numpy(workloads.make_target(w).ravel()).to(dev))
        tol, name = 1e-8, f"256x256 Nt=96 N_D=8 restart=10 {args.precision} {args.basis}"
    for _ in range(2):
        r = s.solve(f, tol=tol, maxit=200)
    print(json.dumps({"profile_case": name, "iterations": r.iterations, "status": r.status}))
    return 0 if r.status == kkt.KKT_OK else 1


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2305_04421_gb300.kkt as kkt

    w = workload_for(args.omega)
    dev = torch.device("cuda", local)
    probe_peaks(kkt)   # compute peaks of this GPU, before (and outside) every timed region
    solver = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub,
                        **({"orth": args.orth} if args.orth else {}))
    if args.dst_method != "auto":
        solver.set_dst_method(args.dst_method)   # (under a profiler the create-time timing can pick another)
    ut = torch.from_numpy(workloads.make_target(w).ravel()).to(dev)
    f = solver.build_rhs(ut)
    x = torch.zeros_like(f)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        x.zero_()
        solver.solve(f, x, tol=TOL, maxit=MAXIT)
    sampler = ClockSampler(local)
    sampler.start()
    kkt.kkt_profile_read(reset=True)
    kkt.kkt_profile_enable(True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = []
    for _ in range(args.steps):
        x.zero_()
        results.append(solver.solve(f, x, tol=TOL, maxit=MAXIT))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    kkt.kkt_profile_enable(False)
    prof = kkt.kkt_profile_read(reset=True)
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dev, world)
    ok = all(r.status == kkt.KKT_OK and r.rel_residual <= TOL for r in results)
    its = results[-1].iterations
    value = job_value(world, args.steps, ms / 1e3)
    launches = sum(v["launches"] for k, v in prof.items() if k != "graph")   # kernels only
    x_solution = x.cpu().numpy() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    applies = sum(r.iterations for r in results)
    # end to end through the C ABI with host buffers: the solve from x_0 = 0 (kkt_solve_zero_guess)
    # uploads f and downloads x inside the timed region
    f_host = f.cpu().pin_memory()
    x_host = torch.zeros(f.numel(), dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    solver.solve(f_host, x_host, tol=TOL, maxit=MAXIT, zero_guess=True)   # warm-up: stages the host path once

    def e2e_seconds():
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            solver.solve(f_host, x_host, tol=TOL, maxit=MAXIT, zero_guess=True)
        torch.cuda.synchronize()
        return max_over_ranks(time.perf_counter() - t0, dev, world)

    # the pinned buffers move by the library's copy kernel (default staging); for context the
    # same steps with the copy engine (cudaMemcpyAsync)
    e2e_s = e2e_seconds()
    solver.set_staging("copy_engine")
    e2e_ce_s = e2e_seconds()
    solver.set_staging("auto")
    nbytes = f.numel() * 8
    # the host link's own bandwidth on this machine (context for e2e): one pinned H2D and D2H copy
    link = {}
    d_tmp = torch.empty_like(f)
    for name, dst, src in (("h2d_gbs", d_tmp, f_host), ("d2h_gbs", x_host, f)):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        dst.copy_(src, non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        link[name] = nbytes / (ev0.elapsed_time(ev1) / 1e3) / 1e9
    del d_tmp
    peaks, peak_kind = measured_peaks()
    apply_stats = time_applies(kkt, solver, w.V, 10, dev)
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(w, kkt.kkt_get_options(solver.h).orth),
            "iterations": its, "converged": ok, "rel_residual": results[-1].rel_residual,
            "rel_residual_euclid": results[-1].rel_residual_euclid,
            "precond_applies_per_s": apply_stats["applies_per_s"], "precond_apply": apply_stats,
            "e2e": {"value": job_value(world, e2e_steps, e2e_s), "unit": "solves/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "staging": "copy kernel through the pinned buffers' device mapping",
                    "value_copy_engine": job_value(world, e2e_steps, e2e_ce_s), "host_link_gbs": link},
            "gpu_launches": launches, "peaks_probed": dict(PROBE), "dst_method": solver.dst_method(),
            "kernel_ms": {k: round(v["ms"], 3) for k, v in prof.items()},
            "kernel_launches": {k: v["launches"] for k, v in prof.items()},
            "clocks": clocks}
    line["roofline"] = roofline(prof, peaks, peak_kind, orth=kkt.kkt_get_options(solver.h).orth,
                                dst_method=solver.dst_method())
    solver.close()
    del f, x, f_host, x_host
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_forms:
        line["variants"] = measure_variants(kkt, dev, w, ms / args.steps, steps=2, warmup=1)
        line["forms"] = measure_forms(kkt, dev, steps=2, warmup=1)
    if rank == 0 and world == 1 and not args.no_batched:
        line["batched"] = measure_batched(kkt, dev)
    if rank == 0 and world == 1 and not args.no_learned:
        line["learned"] = measure_learned(kkt, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        kdim = min(its, 30) // 2 + 1
        s, sample = oracle_iteration_sample(w, kdim)
        line["cpu_baseline"] = {"value": 1.0 / (s * its), "unit": "solves/s", "cores": cpu_threads(),
                                "kind": "oracle", "sample": sample + f"; x {its} iterations"}
        s1, why = oracle_sample_one_thread(w.omega, kdim)
        line["cpu_baseline"]["one_thread"] = ({"value": 1.0 / (s1 * its), "unit": "solves/s", "cores": 1}
                                              if s1 else {"unavailable": why})
        # the timed solve's answer against the oracle's exact solution on the target's modes
        line["rel_error_vs_exact"] = error_vs_exact(w, x_solution)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0 if ok else 1


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--omega", type=float, default=1e-4)
    ap.add_argument("--ref-iterations", type=int, default=25,
                    help="iterations the reference arm scales its per-iteration sample by")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", nargs="?", const="grid", choices=["grid", "paper", "batched", "tensor"],
                    default=None,
                    help="run only a small solve for counter captures: 'grid' (default) 256 x 256, Nt = 96; "
                         "'paper' the Section 4 mesh (17 x 17 points) with Nt = 3200, 640 subdomains; "
                         "'batched' two 128 x 128, Nt = 128 instances, single solves then the batched kernels; "
                         "'tensor' three tensor-core FP64 2D transforms at 256 x 256, Nt = 64")
    ap.add_argument("--basis", choices=["physical", "spectral"], default="physical",
                    help="FGMRES basis of --profile-case")
    ap.add_argument("--precision", choices=["fp64", "bf16", "tf32"], default="fp64",
                    help="preconditioner arithmetic of --profile-case")
    ap.add_argument("--study", choices=["paper", "coarse"], default=None,
                    help="instead of the benchmark: 'paper' runs Section 4's one- vs two-level iteration "
                         "study, 'coarse' times kkt_coarse_apply with block Thomas and the cyclic reduction")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-vs-plain coarse comparison on the 256 x 256, Nt = 2048 workload")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64-instance batched vs one-after-another comparison")
    ap.add_argument("--orth", choices=["mgs", "cgs2", "mgs2", "mgs4", "mgs8"], default=None,
                    help="orthogonalisation of the timed solve (default: the library's)")
    ap.add_argument("--dst-method", choices=["auto", "tiles", "lane", "tensor"], default="auto",
                    help="FP64 sine transforms of the benchmark solve (default: the create-time timing's choice)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP64/BF16/TF32 time-to-solution comparison on the 512 x 512 workload")
    args = ap.parse_args()
    if args.study == "paper":
        return run_study(args)
    if args.study == "coarse":
        return run_coarse_study(args)
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
