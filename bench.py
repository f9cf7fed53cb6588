#!/usr/bin/env python3
"""SI-CTMRG throughput on GB300: CTMRG moves/s on the 3x3-cell, complex
D = 6, chi = 144 workload (half-system 5184 x 5184), split-precision tensor-core
products, through the C ABI of libctm.

One step = one CTMRG iteration: the four directional moves over the 3x3 cell
(9 cuts each: enlarged corners, one subspace-iteration round with QR, small
SVD, projectors, absorption) plus the corner-spectrum convergence scalar.
Inputs are seeded synthetic tensors (ctm_synth); the working set (four
0.43 GB corners per cut plus their bf16 slices) is far larger than L2, so no
explicit flush is needed between timed steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica of the workload
(the path has no exchange step); value = moves of all ranks / max time.
Prints one JSON line on rank 0.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "cfg3_3x3_D6_chi144_c128"
WARM_ITERS, WARM_ROUNDS = 2, 4
# DRAM bytes (read + write) per launch of split_mma_kernel<FmtBF16> over the
# kernel's algorithmic bytes (all slices of both operands + the fp32 split-K
# partials), from a one-pass ncu capture of a corner x block launch at
# N = 5184, k = 149 (469.2 MB / 501.7 MB); only valid for the bf16 kernel as
# captured, so it is set to None whenever that kernel changes
TRAFFIC_PER_OPERAND_BYTE = 0.935
SLICE_PRODUCTS = 6   # bf16 slice products per algorithmic product
METRIC = "CTMRG moves/s & tensor TFLOP/s at D=6, chi=144"
UNIT = "moves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["split", "tf32", "fp64"], default="split",
                    help="split: bf16 x3 slices; tf32: 3xTF32 slices; fp64: no slicing")
    ap.add_argument("--method", choices=["si", "svd"], default="si",
                    help="projectors: subspace iteration or the standard truncated SVD")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-svd-presolve", action="store_true",
                    help="small SVDs in fp64 sweeps only (no fp32 one-sided Jacobi first)")
    ap.add_argument("--no-fp64-tc", action="store_true",
                    help="split modes: Grams, rho and projectors as fp64 GEMMs on the CUDA cores")
    ap.add_argument("--exact", action="store_true",
                    help="split modes: every product an exact-digit fp64-accurate product on "
                         "the tensor cores from the start (split_refine = +inf)")
    ap.add_argument("--no-comparisons", action="store_true",
                    help="skip the plain-FP64 and standard-SVD comparison timings and the "
                         "split-error measurement")
    ap.add_argument("--serve", action="store_true",
                    help="serving mode: Poisson stream of mixed solves, p50/p99 latency")
    ap.add_argument("--requests", type=int, default=128)
    ap.add_argument("--max-iter", type=int, default=100, help="per solve (serve)")
    ap.add_argument("--rate", type=float, default=1.0, help="arrivals per second (serve)")
    ap.add_argument("--concurrency", type=int, default=8, help="solves in flight (serve)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return pk, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampling (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        out.update(sm_mhz=statistics.median(sm) if sm else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons),
                   samples=len(rows))
        return out


# ------------------------------------------------------------- oracle timing
def oracle_sample_seconds(w):
    """Time one cut of the workload in the CPU oracle: the four enlarged
    corners, one subspace-iteration round (rangefinder updates with QR),
    the small SVD and projectors, and the absorption of one site. A move is
    Lx*Ly such cuts. Returns (seconds per move, seconds measured, sample)."""
    import numpy as np
    import ctm_synth as S
    from oracle import ctmrg

    Lx, Ly, d, D, chi, p = w["Lx"], w["Ly"], w["d"], w["D"], w["chi"], w["p"]
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=w["complex_"], diag_weight=w["diag_weight"])
    Cs, Ts = S.initial_env(Lx, Ly, chi, D, D, complex_=w["complex_"])
    N = chi * D * D
    k = min(chi + p, N)
    X0, W0 = S.initial_rangefinders(1, 1, N, k, complex_=w["complex_"])
    ref = ctmrg.CTM(Lx, Ly, A, [a.conj() for a in A], Cs, Ts, chi, method="si", p=p,
                    si_rounds=w["si_rounds"])
    f = ctmrg.Frame(Lx, Ly, 0)
    t0 = time.perf_counter()
    Q = ref.cut_corners(f, 0, 0)
    X = ctmrg.qr_q(X0[0][0])
    W = ctmrg.qr_q(W0[0][0])
    Pl, Pr, s, Xn, Wn, s_all = ctmrg.projectors_si(*Q, X, W, chi, w["si_rounds"])
    # absorption of one site with this cut's projectors on both sides
    C1, T1, T4 = ref.C[0][0], ref.T[0][0], ref.T[3][0]
    E1 = np.einsum("pm,mnuv->puvn", C1, T1).reshape(-1, chi)
    C1n = Pr @ E1
    Pl4 = Pl.reshape(chi, D, D, chi)
    Pr4 = Pr.reshape(chi, chi, D, D)
    Y = np.einsum("tqlw,quvc->tlwuvc", T4, Pl4, optimize=True)
    Y = np.einsum("tlwuvc,sulde->twvcsde", Y, A[0], optimize=True)
    Y = np.einsum("twvcsde,svwDE->tdDceE", Y, A[0].conj(), optimize=True)
    T4n = np.einsum("atdD,tdDceE->aceE", Pr4, Y, optimize=True)
    dt = time.perf_counter() - t0
    del C1n, T4n
    per_move = dt * Lx * Ly
    sample = (f"one cut of the {Lx}x{Ly} D={D} chi={chi} workload (4 enlarged corners, "
              f"{w['si_rounds']} SI round, small SVD, projectors, absorption of one site) "
              f"x {Lx * Ly} cuts per move")
    return per_move, dt, sample


def cpu_cores():
    threads = os.environ.get("OMP_NUM_THREADS") or os.environ.get("OPENBLAS_NUM_THREADS")
    return int(threads) if threads else os.cpu_count()


# -------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    import ctm_synth as S

    if rank != 0:
        return
    w = S.WORKLOADS[args.workload]
    for _ in range(args.warmup):
        oracle_sample_seconds(w)
    per = []
    for _ in range(args.steps):
        pm, dt, sample = oracle_sample_seconds(w)
        per.append(pm)
    ms_per_move = 1000.0 * sum(per) / len(per)
    value = 1000.0 / ms_per_move
    line = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 4 * ms_per_move, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": args.workload, "cell": "3x3", "D": w["D"], "chi": w["chi"],
                   "p": w["p"], "si_rounds": w["si_rounds"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- rank aggregation
def max_over_ranks(x, dist, device):
    """The largest value of a per-rank float over all ranks (x itself for a
    single process): the slowest rank times the whole job."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job rate: the units all ranks processed (each rank an independent
    replica of the same workload) over the time of the slowest rank."""
    return units_per_rank * world / seconds


# -------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import ctm_synth as S
    import paper_2607_15158_gb300 as pkg

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

    w = S.WORKLOADS[args.workload]
    Lx, Ly, d, D, chi, p = w["Lx"], w["Ly"], w["d"], w["D"], w["chi"], w["p"]
    cplx = w["complex_"]
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=cplx, diag_weight=w["diag_weight"])
    Cs, Ts = S.initial_env(Lx, Ly, chi, D, D, complex_=cplx)
    N = chi * D * D
    k = min(chi + p, N)
    X0, W0 = S.initial_rangefinders(Lx, Ly, N, k, complex_=cplx)
    stream = torch.cuda.current_stream()
    prec = {"split": pkg.CTM_PREC_SPLIT_BF16, "tf32": pkg.CTM_PREC_SPLIT_TF32,
            "fp64": pkg.CTM_PREC_FP64}[args.prec]
    # the algorithm's own warm-up (first WARM_ITERS iterations with
    # WARM_ROUNDS subspace-iteration rounds and the fp64 QR schedule) runs in
    # the untimed warm-up steps; timed steps are steady-state SI moves with
    # one round per move
    method = pkg.CTM_PROJ_SVD if args.method == "svd" else pkg.CTM_PROJ_SI
    opts = pkg.ctm_default_opts(p=p, si_rounds=w["si_rounds"], warmup_iters=WARM_ITERS,
                                warmup_rounds=WARM_ROUNDS, prec=prec, method=method,
                                svd_presolve=0 if args.no_svd_presolve else 1,
                                fp64_tc=0 if args.no_fp64_tc else 1,
                                split_refine=float("inf") if args.exact else 0.0,
                                stream=stream.cuda_stream)
    ctx = pkg.ctm_init(Lx, Ly, A, d, D, chi, cplx=cplx, opts=opts)
    ctx.ctm_set_env(Cs, Ts)
    ctx.ctm_set_rangefinders(X0, W0)

    def step():
        it, delta, _ = ctx.ctm_converge(0.0, 1)
        _, launches = ctx.ctm_last_timing()
        return launches

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    ctx.ctm_profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    # bracket the timed steps for profilers started with --profile-from-start off
    torch.cuda.profiler.start()
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        launches += step()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = ctx.ctm_profile_read() if prec != pkg.CTM_PREC_FP64 else None
    phases = {k_: round(v / args.steps, 2) for k_, v in ctx.ctm_profile_phases().items()}
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(4 * args.steps, world, ms / 1000.0)

    # end to end through the C ABI with host buffers: per step the
    # environment is copied in from pinned host memory, the iteration runs,
    # and all corner spectra (the step's result) are read back
    Ch = torch.from_numpy(np.ascontiguousarray(np.asarray(Cs), dtype=np.complex128 if cplx
                                               else np.float64)).pin_memory().numpy()
    Th = torch.from_numpy(np.ascontiguousarray(np.asarray(Ts), dtype=np.complex128 if cplx
                                               else np.float64)).pin_memory().numpy()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.ctm_set_env(Ch, Th)
        step()
        ctx.ctm_spectra()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e_value = job_throughput(4 * args.steps, world, e2e_s)
    h2d = Ch.nbytes + Th.nbytes
    d2h = 4 * Lx * Ly * chi * 8

    if rank != 0:
        ctx.ctm_free()
        return
    peaks, src = load_peaks()
    roofline = None
    if prof is not None and prof[1] > 0:
        mma_ms, mma_n, mma_flops, mma_bytes = prof
        # algorithmic flops: the complex (or real) product itself, 8 (2) real
        # flops per multiply-add = the tensor-pipe flops of the six bf16 slice
        # products / 6
        pipe = mma_flops / (mma_ms * 1e-3) / 1e12
        nprod = SLICE_PRODUCTS if args.prec == "split" else 3
        achieved = pipe / nprod
        peak = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        if args.prec == "tf32":
            peak = peak / 2.0   # tf32 kind at half the bf16 rate (nominal ratio)
        traffic = (None if TRAFFIC_PER_OPERAND_BYTE is None or args.prec != "split"
                   else round(TRAFFIC_PER_OPERAND_BYTE * mma_bytes / mma_n))
        roofline = {"bound": "tensor",
                    "kernel": "split_mma_kernel (tcgen05 %s, fp32 accum)"
                              % ("kind::f16 bf16" if args.prec == "split" else "kind::tf32"),
                    "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
                    "frac": round(achieved / peak, 4), "traffic": traffic,
                    "traffic_basis": "bytes per launch: ncu dram read + write of one "
                                     "corner x block launch (N = 5184, k = 149) over its "
                                     "algorithmic bytes (0.935) x this run's algorithmic "
                                     "bytes per launch",
                    "achieved_basis": "algorithmic flops (8 per complex multiply-add) per "
                                      "launch / CUDA-event duration on the launching stream",
                    "tensor_pipe_achieved": round(pipe, 2),
                    "tensor_pipe_frac": round(pipe / peak, 4),
                    "tensor_pipe_basis": f"{nprod} {'bf16' if nprod == 6 else 'tf32'} slice "
                                         "products of the real-embedded problem",
                    "peak_source": (f"{src} bf16 sustained (of measured)" if src == "measured"
                                    else "fallback 1.7 PFLOP/s sustained (of fallback)")
                    + (" x 1/2 (nominal tf32 / bf16 ratio)" if args.prec == "tf32" else ""),
                    "launches": mma_n, "launches_covered": "every launch of the timed steps",
                    "kernel_ms": round(mma_ms, 3),
                    "kernel_share_of_step": round(mma_ms / ms, 4),
                    "overlap": "lanes run the cuts of a column concurrently: a launch's event "
                               "interval includes time shared with other lanes' kernels"}
    cpu = None
    if not args.no_cpu_baseline:
        per_move, dt, sample = oracle_sample_seconds(w)
        cpu = {"value": 1.0 / per_move, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": sample, "seconds_measured": round(dt, 2)}
    algo_flops_move = move_flops(w, args.method)
    extra = {}
    if not args.no_comparisons and args.workload == WORKLOAD and args.prec == "split":
        ctx.ctm_free()
        ctx = None
        extra = comparisons(pkg, S, value)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128" if cplx else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "cell": f"{Lx}x{Ly}", "d": d, "D": D, "chi": chi,
                   "p": p, "N": N, "k": k, "si_rounds": w["si_rounds"],
                   "precision": ("exact-digit fp64-accurate products on the tensor cores "
                                 "(8 bf16 digits, 36 digit products), fp64 QR/SVD"
                                 if args.exact and args.prec != "fp64" else
                                 {"split": "split-bf16x3 (6 slice products; s0 t0 and the rest "
                                           "in separate fp32 accumulators), fp64 QR/SVD",
                                  "tf32": "split-3xTF32 (3 slice products), fp64 QR/SVD",
                                  "fp64": "fp64"}[args.prec]),
                   "projectors": "subspace iteration" if args.method == "si"
                   else "standard truncated SVD (dense gesvd)",
                   "small_svd": "fp64 one-sided Jacobi" if args.no_svd_presolve
                   else "fp32 one-sided Jacobi pre-solve, then fp64 sweeps",
                   "fp64_products": "fp64 GEMMs (CUDA cores)" if (args.no_fp64_tc or args.prec == "fp64")
                   else "Grams, rho, projectors: exact 8-digit fixed-point bf16 products on the "
                        "tensor cores (fp64-accurate)",
                   "step": "1 iteration = 4 moves + corner-spectrum scalar",
                   "l2": "working set >> L2 (no flush)", "replicas": world},
        "algorithmic_tflops": round(algo_flops_move * value / 1e12, 3),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "phase_ms_per_step": phases,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                   "reasons": clk["reasons"]},
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.ctm_free()


def _time_moves(pkg, w, prec, method, moves, warm_moves=1):
    """Seconds per move of a fresh context (no warm-up rounds: every move one
    SI round, as in steady state), after warm_moves untimed moves."""
    import torch
    import ctm_synth as S
    Lx, Ly, d, D, chi, p = w["Lx"], w["Ly"], w["d"], w["D"], w["chi"], w["p"]
    cplx = w["complex_"]
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=cplx, diag_weight=w["diag_weight"])
    Cs, Ts = S.initial_env(Lx, Ly, chi, D, D, complex_=cplx)
    N, k = chi * D * D, min(chi + p, chi * D * D)
    X0, W0 = S.initial_rangefinders(Lx, Ly, N, k, complex_=cplx)
    ctx = pkg.ctm_init(Lx, Ly, A, d, D, chi, cplx=cplx, opts=pkg.ctm_default_opts(
        p=p, si_rounds=w["si_rounds"], warmup_iters=0, prec=prec, method=method))
    ctx.ctm_set_env(Cs, Ts)
    ctx.ctm_set_rangefinders(X0, W0)
    for i in range(warm_moves):
        ctx.ctm_move(i % 4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(moves):
        ctx.ctm_move(i % 4)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / moves
    ctx.ctm_free()
    return dt


def comparisons(pkg, S, split_value):
    """The metric's comparison lines on the same GPU, in the same run: plain
    FP64 SI-CTMRG on the bench workload (one timed move), standard truncated-
    SVD CTMRG and FP64 SI-CTMRG on the 3x3 D = 4 chi = 64 workload (two timed
    moves each), and the measured error of split precision."""
    import numpy as np
    out = {}
    w3 = S.WORKLOADS[WORKLOAD]
    w2 = S.WORKLOADS["cfg2_3x3_D4_chi64"]
    t_fp64 = _time_moves(pkg, w3, pkg.CTM_PREC_FP64, pkg.CTM_PROJ_SI, 1)
    t_si2 = _time_moves(pkg, w2, pkg.CTM_PREC_FP64, pkg.CTM_PROJ_SI, 2)
    t_svd2 = _time_moves(pkg, w2, pkg.CTM_PREC_FP64, pkg.CTM_PROJ_SVD, 2)
    out["comparisons"] = {
        "fp64_si_same_workload": {"value": 1.0 / t_fp64, "unit": UNIT, "moves_timed": 1,
                                  "split_over_fp64": split_value * t_fp64},
        "cfg2_3x3_D4_chi64": {"si_fp64": 1.0 / t_si2, "standard_svd_fp64": 1.0 / t_svd2,
                              "unit": UNIT, "moves_timed": 2, "si_over_standard": t_svd2 / t_si2},
        "note": "standard CTMRG on the bench workload (dense 5184 x 5184 complex SVD per cut) "
                "is not timed: at this GPU's fp64 rate one move takes minutes"}
    # split error against the fp64 path: (1) one enlarged corner and one
    # corner x block product at the bench size, (2) a converged D = 6 2x2 cell
    w = w3
    Lx, Ly, d, D, chi, p = w["Lx"], w["Ly"], w["d"], w["D"], w["chi"], w["p"]
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=True, diag_weight=w["diag_weight"])
    Cs, Ts = S.initial_env(Lx, Ly, chi, D, D, complex_=True)

    def ctx_for(prec, A, Cs, Ts, Lx, Ly, D, chi, **kw):
        c = pkg.ctm_init(Lx, Ly, A, 2, D, chi, cplx=True,
                         opts=pkg.ctm_default_opts(p=5, prec=prec, **kw))
        c.ctm_set_env(Cs, Ts)
        return c
    cs = ctx_for(pkg.CTM_PREC_SPLIT_BF16, A, Cs, Ts, Lx, Ly, D, chi)
    cf = ctx_for(pkg.CTM_PREC_FP64, A, Cs, Ts, Lx, Ly, D, chi)
    Qs, Qf = cs.ctm_corner(0, 0, 0, 2), cf.ctm_corner(0, 0, 0, 2)
    e_corner = float(np.abs(Qs - Qf).max() / np.abs(Qf).max())
    rng = np.random.default_rng(1)
    Z = rng.standard_normal((cs.N, cs.k)) + 1j * rng.standard_normal((cs.N, cs.k))
    Y = cs.ctm_corner_apply(0, 0, 0, 2, Z)
    R = Qs @ Z
    e_apply = float(np.abs(Y - R).max() / np.abs(R).max())
    cs.ctm_free()
    cf.ctm_free()
    del Qs, Qf, Y, R
    A6 = S.ipeps_tensors(2, 2, 2, 6, complex_=True, seed=0, bond_decay=0.5)
    C6, T6 = S.initial_env(2, 2, 8, 6, 6, complex_=True, seed=1)
    heis = S.heisenberg_bond()
    res = []
    for prec in (pkg.CTM_PREC_SPLIT_BF16, pkg.CTM_PREC_FP64):
        c = ctx_for(prec, A6, C6, T6, 2, 2, 6, 8)
        c.ctm_converge(1e-11 if prec == pkg.CTM_PREC_FP64 else 1e-9, 150)
        res.append((c.ctm_spectra(), np.array([c.ctm_expect(heis, x, y, dr)
                                               for y in range(2) for x in range(2)
                                               for dr in (0, 1)])))
        c.ctm_free()
    out["split_error"] = {
        "vs": "the fp64 path of this library on the same inputs",
        "corner_full_size": e_corner, "corner_x_block_full_size": e_apply,
        "full_size_basis": "max |split - fp64| / max |fp64| over one enlarged corner and one "
                           "corner x block product of the bench workload",
        "converged_spectra": float(np.abs(res[0][0] - res[1][0]).max()),
        "converged_energies": float(np.abs(res[0][1] - res[1][1]).max()),
        "converged_basis": "2x2 cell, complex D = 6, chi = 8, bond weights decaying as "
                           "0.5^(u+l+d+r), converged; unit-normalised corner spectra and "
                           "Heisenberg bond energies"}
    return out


def move_flops(w, method="si"):
    """Algorithmic real flops of one move (complex MAC = 8 real flops): per
    cut 4 enlarged corners (chi^3 D^2 + chi^3 D^4 + 2 chi^2 d D^6 MAC each)
    and the absorption (chi^3 D^2 + 2 chi^3 D^4 + 2 chi^2 d D^6); SI adds the
    round(s) (16 N^2 k), Z_R and Z_L (4 N^2 k) and rho (N k^2); the standard
    method adds M = H_L H_R (3 N^3), the projectors (2 N^2 chi) and the dense
    SVD (~21 N^3 real flops, x4 complex)."""
    chi, D, d, p = w["chi"], w["D"], w["d"], w["p"]
    N = chi * D * D
    k = min(chi + p, N)
    r = w["si_rounds"]
    per_mac = 8 if w["complex_"] else 2
    mac = 4 * (chi ** 3 * D ** 2 + chi ** 3 * D ** 4 + 2 * chi ** 2 * d * D ** 6)
    mac += chi ** 3 * D ** 2 + 2 * chi ** 3 * D ** 4 + 2 * chi ** 2 * d * D ** 6
    extra = 0.0
    if method == "svd":
        mac += 3 * N ** 3 + 2 * N * N * chi
        extra = 21.0 * N ** 3 * (4 if w["complex_"] else 1)
    else:
        mac += (16 * r + 4) * N * N * k + N * k * k
    return (per_mac * mac + extra) * w["Lx"] * w["Ly"]


# ------------------------------------------------------------------ serving
SERVE_SPLIT_ABOVE_N = 1024   # solves with a larger half-system run in split precision


def serve_mix(n, seed=4):
    """Seeded request stream of the serving workload: each request a random
    unit cell (1x1, 2x2 or 3x3) of real tensors A[2,D,D,D,D] with D uniform in
    {3, ..., 7} and chi uniform in [D^2, 4 D^2], tolerance 1e-8."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        L = int(rng.choice([1, 2, 3]))
        D = int(rng.integers(3, 8))
        chi = int(rng.integers(D * D, 4 * D * D + 1))
        out.append((L, L, D, chi, 1000 + i))
    return out


def run_serve(args):
    import numpy as np
    import torch

    import ctm_synth as S
    import paper_2607_15158_gb300 as pkg

    torch.cuda.set_device(0)
    mix = serve_mix(args.requests)
    rng = np.random.default_rng(5)
    gaps = rng.exponential(1.0 / args.rate, size=len(mix))
    heis = S.heisenberg_bond()
    tensors = [S.ipeps_tensors(Lx, Ly, 2, D, complex_=False, seed=sd) for (Lx, Ly, D, chi, sd) in mix]
    srv = pkg.Server(hbm_budget=0, max_concurrent=args.concurrency)
    t0 = time.perf_counter()
    tickets, precs = [], []
    for (Lx, Ly, D, chi, sd), A, gap in zip(mix, tensors, gaps):
        time.sleep(gap)
        split = chi * D * D > SERVE_SPLIT_ABOVE_N
        o = pkg.ctm_default_opts(prec=pkg.CTM_PREC_SPLIT_BF16 if split else pkg.CTM_PREC_FP64,
                                 recycle_sin2=1e-3, min_si_steps=3)
        precs.append("split" if split else "fp64")
        tickets.append(srv.ctm_server_submit(A, 2, D, chi, 1e-8, args.max_iter, op=heis,
                                             cplx=False, Lx=Lx, Ly=Ly, opts=o))
    res = [srv.ctm_server_result(t) for t in tickets]
    wall = time.perf_counter() - t0
    st = srv.ctm_server_stats()
    srv.ctm_server_free()
    conv = [r["delta"] < 1e-8 for r in res]
    line = {
        "metric": "serve p50/p99 latency", "value": st["p50_ms"], "unit": "ms",
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "solves_per_s": st["solves_per_s"],
        "n_gpus": 1, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "serve: Poisson arrivals of random cells 1x1/2x2/3x3, real "
                               "A[2,D,...] with D in {3..7}, chi in [D^2, 4 D^2], tol 1e-8",
                   "requests": len(mix), "rate_per_s": args.rate,
                   "concurrency": args.concurrency, "max_iter": args.max_iter,
                   "precision": f"fp64 for N = chi D^2 <= {SERVE_SPLIT_ABOVE_N}, split bf16x3 "
                                "above (fp64 solves of the largest requests take tens of "
                                "minutes at this GPU's fp64 rate)",
                   "recycling": "paper step 4 policy: no update round once mean sin^2 < 1e-3 "
                                "after 3 updates"},
        "wall_s": wall,
        "mean_queue_ms": float(np.mean([r["queue_ms"] for r in res])),
        "mean_run_ms": float(np.mean([r["run_ms"] for r in res])),
        "converged_1e-8": {"fp64": int(sum(c for c, p in zip(conv, precs) if p == "fp64")),
                           "split": int(sum(c for c, p in zip(conv, precs) if p == "split")),
                           "fp64_requests": precs.count("fp64"),
                           "split_requests": precs.count("split")},
        "split_final_delta_median": float(np.median([r["delta"] for r, p in zip(res, precs)
                                                     if p == "split"] or [0.0])),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.serve:
        run_serve(args)
        return
    if args.impl == "ours" and args.warmup < WARM_ITERS:
        args.warmup = WARM_ITERS
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
