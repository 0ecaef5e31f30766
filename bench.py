"""Benchmark of the GP hot path on GB300: fused on-the-fly kernel product throughput.

Workload (one "step"): one fused pass Kh V, dKh/df V, dKh/dl V (dKh/ds V = V)
over n = 100,000 points in d = 3 (uniform on [0,1]^3, seeded), Matern-3/2 with
f = 1.5, l = 0.2, s = 0.05, V = [y | 31 Rademacher columns] (w = 32), FP32.
Metric: kernel entries x columns per second, n^2 w / (pass time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gp|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload on
its own GPU (the product does not shard without an exchange step); the value is
the sum over ranks / the slowest rank's time.

`--impl reference` times the FP64 CPU oracle (test infrastructure, never the
product path) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("kernel entries×cols/s and loss+grad ms per Θ on 1 GB300, "
          "mixed vs FP32 at ≤1e-4 rel err")
UNIT = "entries*cols/s"
WORKLOAD = ("fused on-the-fly product Kh.V + dKh/df.V + dKh/dl.V: n=100000 d=3 uniform[0,1]^3, "
            "Matern-3/2 f=1.5 l=0.2 s=0.05, V=[y | 31 Rademacher] w=32, FP32")
N_PTS, D, W = 100_000, 3, 32
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def _refs():
    """FP64 reference values written by tests/golden/make_bench_refs.py (which
    calls only the oracle); the accuracy columns of the extra legs compare
    against them."""
    return np.load(os.path.join(ROOT, "tests", "golden", "bench_refs.npz"))


def _traffic():
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest of the ranks' values (the slowest replica sets the job's time);
    `value` itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world: int, work_per_rank: float, slowest_ms: float) -> float:
    """Whole-job throughput of `world` independent replicas: all ranks' work over
    the slowest rank's time."""
    return world * work_per_rank / (slowest_ms * 1e-3)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_oracle_rate(target_s: float = 12.0) -> dict:
    """FP64 oracle on sampled rows of the same workload: entries*cols/s on the host."""
    import oracle as O
    from paper_2503_02259_gb300 import inputs
    prob = inputs.matvec_problem(seed=0)
    V = inputs.multivector(prob.y, W, seed=0)
    rng = np.random.default_rng(1)
    rows = rng.choice(prob.n, 4000, replace=False)
    t0 = time.perf_counter()
    O.kmv_rows(prob.X, V, prob.kind, prob.theta, rows=rows[:16], block=16)
    per_row = (time.perf_counter() - t0) / 16
    nrows = int(max(16, min(4000, target_s / max(per_row, 1e-9))))
    t0 = time.perf_counter()
    O.kmv_rows(prob.X, V, prob.kind, prob.theta, rows=rows[:nrows], block=64)
    dt = time.perf_counter() - t0
    value = nrows * prob.n * W / dt
    return {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"FP64 NumPy oracle, fused Kh.V + dKh.V on {nrows} sampled rows of the "
                       f"n=100000 w=32 workload ({dt:.1f} s); NumPy elementwise single-threaded, "
                       "BLAS matmul on default threads")}


def run_reference(args) -> int:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    vals = []
    t_all = time.perf_counter()
    budget = max(3.0, 60.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_rate(target_s=min(budget, 8.0))
        if i >= args.warmup:
            vals.append(r)
    value = statistics.median(v["value"] for v in vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": N_PTS * N_PTS * W / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": vals[-1]["sample"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle", "sample": vals[-1]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)
    return 0


PRECS = {"fp32": 0, "tf32": 1, "bf16": 2, "tf32x3": 3, "bf16x3": 4}
NPROD = {1: 1, 2: 2, 3: 3, 4: 3}   # tensor-core products per operand pair (BF16: A B_hi + A B_lo)


def measure_rates(B, api, dev) -> dict:
    """The FP32 FMA-pipe rate (packed FFMA2, TFLOP/s) and the MUFU ex2 rate (1e9/s)
    of this GPU, from the library's microbenchmarks."""
    fma_t, mufu_g = B.c_double(), B.c_double()
    B.check(B.lib().gp_measure_pipe_rates(B.ctypes.byref(fma_t), B.ctypes.byref(mufu_g),
                                          api._stream(dev)), "gp_measure_pipe_rates")
    return {"fp32_ffma2_tflops": fma_t.value, "mufu_ex2_gops": mufu_g.value}


def eval_flops(d: int, matern: bool) -> int:
    """FP32 flops of one kernel entry's evaluation besides MUFU operations: the
    squared distance (3d) and the kernel's own arithmetic."""
    return 3 * d + (6 if matern else 1)


def tc_roofline(n: int, d: int, w_pad: int, matern: bool, grad: bool, prec: int, kms: float,
                rates: dict, peaks: dict) -> dict:
    """Floors of one tensor-core product launch: the tensor pipe (NPROD products of
    2 w_pad flops per entry per accumulator, against the measured cuBLAS BF16 peak,
    x 0.5 for TF32) and the MUFU evaluation (sqrt + ex2 for Matern-3/2, ex2 for the
    Gaussian, per entry, against the measured ex2 rate); the binding one is the
    larger, and frac = that floor / the kernel's time."""
    ratio = 0.5 if prec in (1, 3) else 1.0
    tpeak = peaks.get("bf16_tflops", 1900.0) * ratio
    tflops = n * n * 2 * w_pad * NPROD[prec] * (2 if grad else 1)
    t_tensor = tflops / (tpeak * 1e12) * 1e3
    mufu = n * n * (2 if matern else 1)
    t_mufu = mufu / (rates["mufu_ex2_gops"] * 1e9) * 1e3
    bind = "mufu" if t_mufu >= t_tensor else "tensor"
    return {"tensor_floor_ms": t_tensor, "tensor_frac": t_tensor / kms,
            "tensor_peak_tflops": tpeak, "mufu_floor_ms": t_mufu, "mufu_frac": t_mufu / kms,
            "mufu_peak_gops": rates["mufu_ex2_gops"], "binding": bind,
            "frac": max(t_tensor, t_mufu) / kms}


def lossgrad_roofline(n: int, d: int, matern: bool, p: int, k: int, iters: int, ms: float,
                      rates: dict) -> dict:
    """Algorithmic work of one loss + gradient evaluation: block CG on [y | Z]
    (iters products of n^2 entries x (2 w + eval) flops, w = 1 + p), k Lanczos
    products on the p probes and one fused derivative product (4 w + eval + 1), in
    FP32 flops, against the measured FP32 FMA-pipe rate; and the MUFU count of the
    same entries against the measured ex2 rate."""
    w = 1 + p
    e = eval_flops(d, matern)
    flops = float(n) * n * (iters * (2 * w + e) + k * (2 * p + e) + (4 * w + e + 1))
    mufu = float(n) * n * (iters + k + 1) * (2 if matern else 1)
    achieved = flops / (ms * 1e-3) / 1e12
    return {"algorithmic_flops": flops, "achieved_tflops": achieved,
            "fp32_peak_tflops": rates["fp32_ffma2_tflops"],
            "frac_of_fp32_pipe": achieved / rates["fp32_ffma2_tflops"],
            "mufu_floor_ms": mufu / (rates["mufu_ex2_gops"] * 1e9) * 1e3,
            "frac_of_mufu_floor": mufu / (rates["mufu_ex2_gops"] * 1e9) / (ms * 1e-3),
            "counted": "iters = the largest CG iteration count over the columns (the block "
                       "product runs all columns until the last converges)"}


def precond_lossgrad_roofline(n: int, d: int, matern: bool, p: int, k: int, iters: int, r: int,
                              ms: float, rates: dict) -> dict:
    """Algorithmic work of one preconditioned loss + gradient evaluation: the
    products of lossgrad_roofline, plus the Nystrom work in exact (Dot2) products
    of 10 FP32 flops (11 for Z, whose T carries a low part): the rank-r factor
    with dL/dl (three products per row and earlier column: 1.5 n r^2), the Gram
    matrices L^T L and L^T dL/dl (1.5 n r^2), and n r w per L^T V or Z pass over
    w = 1 + p rounded up to 4 columns: one apply (L^T V and Z) per CG iteration
    and two per Lanczos step (M^-1 and M), one for the probes' M^-1 z, the probes'
    Z, and L^T V and dL/dl^T V for the gradient."""
    base = lossgrad_roofline(n, d, matern, p, k, iters, ms, rates)
    wl = 4 * ((1 + p + 3) // 4)
    factor = 10.0 * 1.5 * n * r * r
    gram = 10.0 * 1.5 * n * r * r
    applies = iters + 2 * k + 1
    apply = float(n) * r * wl * (applies * (10 + 11) + 11 + 2 * 10)
    flops = base["algorithmic_flops"] + factor + gram + apply
    achieved = flops / (ms * 1e-3) / 1e12
    return {"algorithmic_flops": flops, "products_flops": base["algorithmic_flops"],
            "nystrom_flops": factor + gram + apply, "achieved_tflops": achieved,
            "fp32_peak_tflops": rates["fp32_ffma2_tflops"],
            "frac_of_fp32_pipe": achieved / rates["fp32_ffma2_tflops"],
            "counted": base["counted"] + "; Nystrom work in 10-flop exact products"}


def precision_modes(api, B, torch, prob, X, V, dev, rates: dict, steps: int = 5) -> dict:
    """Each tensor-core mode on the bench workload: product-kernel throughput and the
    norm-wise error of K.V and dK/dl.V against FP64 oracle values on 100 sampled rows
    (tests/golden/bench_refs.npz)."""
    refs = _refs()
    rows, rY, rL = refs["matvec_rows"], refs["matvec_Y"], refs["matvec_L"]
    L = B.lib()
    out = {}
    for name, prec in PRECS.items():
        pr, _ = api.problem(X, prob.kind, prob.theta)
        ws = api.workspace(B.OP_GRAD_MATMUL, pr, W, api.solve_opts(prec=prec), dev)
        Y = torch.empty_like(V)
        dYf = torch.empty_like(V)
        dYl = torch.empty_like(V)

        def step():
            B.check(L.gp_kernel_grad_matmul(B.ctypes.byref(pr), api._ptr(V), W, api._ptr(Y),
                                            api._ptr(dYf), api._ptr(dYl), prec, api._ptr(ws),
                                            ws.numel(), api._stream(dev)), "grad_matmul")
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        B.check(L.gp_profile_begin(), "profile")
        for _ in range(steps):
            step()
        torch.cuda.synchronize()
        ms = B.c_double()
        n1 = B.c_int64()
        n2 = B.c_int64()
        B.check(L.gp_profile_end(B.ctypes.byref(ms), B.ctypes.byref(n1), B.ctypes.byref(n2)), "profile")
        kms = ms.value / max(1, n1.value)
        yh = Y.cpu().numpy()[rows].astype(np.float64)
        lh = dYl.cpu().numpy()[rows].astype(np.float64)
        err = float(np.max(np.linalg.norm(yh - rY, axis=0) / np.linalg.norm(rY, axis=0)))
        errl = float(np.max(np.linalg.norm(lh - rL, axis=0) / np.linalg.norm(rL, axis=0)))
        out[name] = {"kernel_ms": kms, "value": N_PTS * N_PTS * W / (kms * 1e-3), "unit": UNIT,
                     "relerr_Y": err, "relerr_dYl": errl,
                     "within_3e-3_tile_bound": bool(max(err, errl) <= 3e-3)}
        if prec != 0:
            out[name]["roofline"] = tc_roofline(N_PTS, D, 32, True, True, prec, kms, rates, _peaks())
    out["modes_claimed_for_the_3e-3_tile_bound"] = ["tf32", "tf32x3", "bf16x3"]
    return out


def precision_config(api, B, torch, dev) -> dict:
    """The precision problem (n = 1e6, d = 2 uniform, Gaussian f = 1, l = 0.05, s = 0.01,
    V of width 64): one K-hat.V product per arithmetic, timed with the library's
    product-kernel events, and its norm-wise error against FP64 oracle values on 200
    sampled rows (tests/golden/bench_refs.npz; the same rows for every arithmetic)."""
    from paper_2503_02259_gb300 import inputs
    prob = inputs.precision_problem(seed=0)
    Vh = inputs.multivector(prob.y, 64, seed=0)
    refs = _refs()
    rows, rY = refs["precision_rows"], refs["precision_Y"]
    X = torch.from_numpy(prob.X).to(dev)
    V = torch.from_numpy(Vh).to(dev)
    L = B.lib()
    out = {"workload": "n=1000000 d=2 uniform[0,1]^2, Gaussian f=1 l=0.05 s=0.01, V=[y | 63 "
                       "Rademacher] w=64, one Kh.V product; error on 200 sampled rows vs FP64"}
    for name, prec in PRECS.items():
        pr, _ = api.problem(X, prob.kind, prob.theta)
        ws = api.workspace(B.OP_MATMUL, pr, 64, api.solve_opts(prec=prec), dev)
        Y = torch.empty_like(V)

        def step():
            B.check(L.gp_kernel_matmul(B.ctypes.byref(pr), api._ptr(V), 64, api._ptr(Y), prec,
                                       api._ptr(ws), ws.numel(), api._stream(dev)), "matmul")
        step()
        torch.cuda.synchronize()
        B.check(L.gp_profile_begin(), "profile")
        step()
        torch.cuda.synchronize()
        ms, n1, n2 = B.c_double(), B.c_int64(), B.c_int64()
        B.check(L.gp_profile_end(B.ctypes.byref(ms), B.ctypes.byref(n1), B.ctypes.byref(n2)), "profile")
        yh = Y.cpu().numpy()[rows].astype(np.float64)
        err = float(np.max(np.linalg.norm(yh - rY, axis=0) / np.linalg.norm(rY, axis=0)))
        out[name] = {"kernel_ms": ms.value, "value": prob.n * prob.n * 64 / (ms.value * 1e-3),
                     "unit": UNIT, "relerr_Y_200_rows": err}
        del ws, Y
    return out


def refinement(api, torch, n: int = 20_000) -> dict:
    """Time to a true residual of 1e-6 on the precision problem's kernel at n = 2e4
    (d = 2, Gaussian f = 1, l = 0.05, s = 0.01; kappa ~ 3e4): plain FP32 CG against
    mixed-precision iterative refinement (split-BF16 or split-TF32 inner CG to 1e-2;
    FP32 inner CG preconditioned by a rank-1000 Nystrom factor), each with the
    compensated FP32-pair outer residual over all rows.  The FP32 solve's true
    residual is the library's FP64 gp_true_residual; a refined solve's is its own
    outer residual."""
    from paper_2503_02259_gb300 import inputs
    prob = inputs.precision_problem(seed=0, n=n)
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    out = {"workload": f"n={n} d=2 uniform, Gaussian f=1 l=0.05 s=0.01, B = y (w = 1); "
                       "target true residual 1e-6"}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x32, it32, rr32, _ = api.gp_pcg_solve(X, y, prob.kind, prob.theta,
                                          api.solve_opts(cg_rtol=1e-10, cg_maxit=4000),
                                          raise_not_converged=False)
    torch.cuda.synchronize()
    t32 = time.perf_counter() - t0
    true32 = api.gp_true_residual(X, y, x32, prob.kind, prob.theta)[0]
    out["fp32_cg"] = {"s": t32, "iterations": it32[0], "recurrence_relres": rr32[0],
                      "true_relres": true32}
    for name, prec in (("bf16x3", 4), ("tf32x3", 3)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, it, rr, st = api.gp_pcg_solve_refined(
            X, y, prob.kind, prob.theta,
            api.solve_opts(cg_rtol=1e-2, prec=prec, refine_rtol=1e-7, refine_maxit=40),
            raise_not_converged=False)
        torch.cuda.synchronize()
        out[f"refined_{name}"] = {"s": time.perf_counter() - t0, "inner_iterations": it[0],
                                  "true_relres": rr[0], "status": st}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, it, rr, st = api.gp_pcg_solve_refined(
        X, y, prob.kind, prob.theta,
        api.solve_opts(cg_rtol=1e-2, refine_rtol=1e-7, refine_maxit=40, precond_rank=1000),
        raise_not_converged=False)
    torch.cuda.synchronize()
    out["refined_fp32_nystrom1000"] = {"s": time.perf_counter() - t0, "inner_iterations": it[0],
                                       "true_relres": rr[0], "status": st}
    return out


def precision_refinement(api, B, torch, rank: int = 1500, cap_plain: int = 20,
                         nsample: int = 1000, n: int = 1_000_000) -> dict:
    """The precision problem itself (n = 1e6, d = 2 uniform, Gaussian f = 1,
    l = 0.05, s = 0.01; kappa ~ 1.6e6) solved to the 1e-6 target:
    mixed-precision iterative refinement (compensated FP32-pair outer residual
    over all rows) whose inner solves are FP32 CG preconditioned by the rank-1500
    Nystrom factor, for two inner tolerances; the preconditioned FP32 solve
    without refinement; and, for contrast, unpreconditioned FP32 CG at a
    cap_plain-iteration cap.  Residuals: the refinement's own pair residual over
    all n rows, and the FP64 residual on nsample sampled rows (gp_residual_rows)
    for every solver; then how far the pair residual rows are from the FP64 ones
    and the time of both arithmetics."""
    from paper_2503_02259_gb300 import inputs
    prob = inputs.precision_problem(seed=0, n=n)
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    rows = np.sort(np.random.default_rng(5).choice(n, nsample, replace=False)).astype(np.int64)
    rows_d = torch.from_numpy(rows).cuda()
    ws = api.workspace(B.OP_RESIDUAL, api.problem(X, prob.kind, prob.theta)[0], 1, None, X.device)
    out = {"workload": f"n={n} d=2 uniform[0,1]^2, Gaussian f=1 l=0.05 s=0.01, B = y (w = 1); "
                       f"Nystrom preconditioner of rank {rank}; residuals on {nsample} sampled rows "
                       "in FP64 (gp_residual_rows)",
           "target_true_relres": 1e-6}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    def fp64_rows(x64):
        return api.gp_residual_rows(X, y, x64, prob.kind, prob.theta, rows=rows_d,
                                    arith=B.RESIDUAL_FP64, ws=ws, want_rows=False)[1][0]

    (_, _, piv, rk), tf = timed(lambda: api.gp_nystrom_apply(X, y, prob.kind, prob.theta, rank))
    out["nystrom_factor"] = {"s_factor_and_one_apply": tf, "rank": rk}
    best = None
    for rtol_in in (1e-2, 1e-5):
        opts = api.solve_opts(cg_rtol=rtol_in, cg_maxit=200, refine_rtol=1e-6, refine_maxit=10,
                              precond_rank=rank)
        (x64, it, rr, st), t = timed(lambda: api.gp_pcg_solve_refined(
            X, y, prob.kind, prob.theta, opts, raise_not_converged=False))
        rec = {"s": t, "inner_iterations": it[0], "status": st, "relres_pair_all_rows": rr[0],
               "relres_fp64_sampled_rows": fp64_rows(x64)}
        out[f"refined_fp32_nystrom_inner{rtol_in:g}"] = rec
        if st == 0 and (best is None or t < best[1]["s"]):
            best = (x64, rec)
    (x32, it32, rr32, st32), t32 = timed(lambda: api.gp_pcg_solve(
        X, y, prob.kind, prob.theta, api.solve_opts(cg_rtol=1e-6, cg_maxit=200, precond_rank=rank),
        raise_not_converged=False))
    out["fp32_pcg_nystrom"] = {"s": t32, "iterations": it32[0], "recurrence_relres": rr32[0],
                               "status": st32, "relres_fp64_sampled_rows": fp64_rows(x32.double())}
    (xc, itc, rrc, _), tc = timed(lambda: api.gp_pcg_solve(
        X, y, prob.kind, prob.theta, api.solve_opts(cg_rtol=1e-12, cg_maxit=cap_plain),
        raise_not_converged=False))
    out["fp32_cg_unpreconditioned"] = {"s": tc, "iterations": itc[0], "recurrence_relres": rrc[0],
                                       "relres_fp64_sampled_rows": fp64_rows(xc.double())}
    if best is not None:
        x64 = best[0]
        (Rf, relf), tfr = timed(lambda: api.gp_residual_rows(X, y, x64, prob.kind, prob.theta,
                                                             rows=rows_d, arith=B.RESIDUAL_FP64,
                                                             ws=ws))
        (Rp, relp), tp = timed(lambda: api.gp_residual_rows(X, y, x64, prob.kind, prob.theta,
                                                            rows=rows_d, arith=B.RESIDUAL_PAIR,
                                                            ws=ws))
        (_, relall), tall = timed(lambda: api.gp_residual_rows(X, y, x64, prob.kind, prob.theta,
                                                               arith=B.RESIDUAL_PAIR, ws=ws,
                                                               want_rows=False))
        bn = float(torch.linalg.vector_norm(y[rows_d].double()))
        out["residual_arithmetics"] = {
            "pair_minus_fp64_rows_over_norm_B_rows": float(torch.linalg.vector_norm(Rp - Rf)) / bn,
            "s_fp64_sampled_rows": tfr, "s_pair_sampled_rows": tp, "fp64_over_pair_time": tfr / tp,
            "s_pair_all_rows": tall, "relres_pair_all_rows_recomputed": relall[0],
            "relres_pair_sampled_rows": relp[0], "relres_fp64_sampled_rows": relf[0],
            "pair_entries_per_s": float(n) * n / tall}
        out["best_s_to_target"] = best[1]["s"]
        out["target_met"] = bool(best[1]["relres_fp64_sampled_rows"] <= 1e-6
                                 and best[1]["relres_pair_all_rows"] <= 1e-6)
    else:
        out["target_met"] = False
    return out


def loss_grad_mixed_vs_fp32(api, torch, rates: dict, full_n: int = 200_000) -> dict:
    """L(Theta) and dL/dTheta on the differentiation problem (d = 8, 0.5 N(0,I), Gaussian
    s = 0.1, f = 1, l = 1.2; 32 probes x 40 Lanczos steps, CG to 1e-6): accuracy of each
    arithmetic (CG products / SLQ products) against the FP64 oracle's same-probe estimator
    on the n = 4000 subsample, and wall time per Theta at the full n."""
    from paper_2503_02259_gb300 import inputs
    same = -1
    arms = {"fp32": (0, 0), "tf32x3": (3, same), "bf16x3": (4, same),
            "bf16x3_slq_tf32x3": (4, 3)}
    # Timed at the full n: FP32 and the fastest mixed form (split TF32 throughout
    # measured 28.9 s, between the two).
    timed = ("fp32", "bf16x3_slq_tf32x3")
    sub = inputs.diff_problem(seed=0, n=4000)
    refs = _refs()
    est = {"loss": float(refs["diff_loss"]), "grad": refs["diff_grad"]}
    gref = np.asarray(est["grad"])
    floor = 1e-3 * np.linalg.norm(gref)
    out = {"workload": "differentiation problem, 32 probes x 40 Lanczos steps, CG rtol 1e-6; "
                       "accuracy on the n=4000 subsample vs the FP64 same-probe oracle; time at "
                       f"n={full_n}; arm = CG arithmetic[_slq_<SLQ arithmetic>], gradient pass FP32"}
    Xs, ys = torch.from_numpy(sub.X).cuda(), torch.from_numpy(sub.y).cuda()
    for name, (prec, slq) in arms.items():
        opts = api.solve_opts(nprobe=32, nlanczos=40, cg_rtol=1e-6, seed=77, prec=prec, slq_prec=slq)
        loss, grad, _ = api.gp_loss_and_grad(Xs, ys, sub.kind, sub.theta, opts)
        rel_l = abs(loss - est["loss"]) / abs(est["loss"])
        rel_g = max(abs(g - r) / max(abs(r), floor) for g, r in zip(grad, gref))
        out[name] = {"relerr_loss_n4000": rel_l, "relerr_grad_n4000": rel_g}
    full = inputs.diff_problem(seed=0, n=full_n)
    Xf, yf = torch.from_numpy(full.X).cuda(), torch.from_numpy(full.y).cuda()
    for name in timed:
        prec, slq = arms[name]
        opts = api.solve_opts(nprobe=32, nlanczos=40, cg_rtol=1e-6, seed=77, prec=prec, slq_prec=slq)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss, grad, info = api.gp_loss_and_grad(Xf, yf, full.kind, full.theta, opts)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        out[name].update({"ms_per_theta": ms, "loss": loss, "grad": grad,
                          "cg_iters": info["cg_iters"],
                          "roofline": lossgrad_roofline(full_n, 8, False, 32, 40, info["cg_iters"],
                                                        ms, rates)})
    for name in timed[1:]:
        out[f"speedup_{name}_vs_fp32"] = out["fp32"]["ms_per_theta"] / out[name]["ms_per_theta"]
    # The fastest timed mixed arithmetic whose loss and gradient stay within 1e-4.
    ok = [k for k in timed[1:] if out[k]["relerr_loss_n4000"] <= 1e-4
          and out[k]["relerr_grad_n4000"] <= 1e-4]
    best = min(ok, key=lambda k: out[k]["ms_per_theta"]) if ok else None
    out["mixed_at_1e-4"] = {"arithmetic": best,
                            "ms_per_theta": out[best]["ms_per_theta"] if best else None,
                            "speedup_vs_fp32": out[f"speedup_{best}_vs_fp32"] if best else None}
    return out


def loss_grad_diff_precond(api, torch, rates: dict, m_identity_ms: float | None = None,
                           full_n: int = 200_000, rank_sub: int = 800, rank_full: int = 2000) -> dict:
    """The differentiation problem's L(Theta) and dL/dTheta (32 probes x 40 Lanczos steps,
    CG to 1e-6) with the Nystrom preconditioner (Eq. 1 / Eq. 2 with M = sI + LL^T,
    probes z ~ N(0, M)).  On the n = 4000 subsample: the error against the exact L and
    dL/dTheta (Cholesky, stored FP64 values) for M = I and for the rank-rank_sub M, and
    the split arithmetic's difference from FP32 on the same probes.  At n = full_n: the
    time per Theta with the rank-rank_full M in FP32 and in the split arithmetic, against
    the unpreconditioned FP32 time (m_identity_ms, from loss_grad_mixed_vs_fp32)."""
    from paper_2503_02259_gb300 import inputs
    refs = _refs()
    lref, gref = float(refs["diffx_loss"]), np.asarray(refs["diffx_grad"])

    def relgrad(grad, ref):
        fl = 1e-3 * np.linalg.norm(ref)
        return max(abs(g - r) / max(abs(r), fl) for g, r in zip(grad, ref))

    out = {"workload": f"differentiation problem (n={full_n}, d=8), 32 probes x 40 Lanczos steps, "
                       f"CG 1e-6; Nystrom rank {rank_full} (rank {rank_sub} on the n=4000 "
                       "subsample, accuracy vs the exact loss); arm = CG arithmetic[_slq_<SLQ>]"}
    arms = (("fp32", 0, 0), ("bf16x3_slq_tf32x3", 4, 3), ("bf16x3", 4, 4))
    sub = inputs.diff_problem(seed=0, n=4000)
    Xs, ys = torch.from_numpy(sub.X).cuda(), torch.from_numpy(sub.y).cuda()
    res = {}
    for name, pr, sp in (("m_identity_fp32", 0, 0),) + arms:
        rank = 0 if name.startswith("m_identity") else rank_sub
        opts = api.solve_opts(nprobe=32, nlanczos=40, cg_rtol=1e-6, seed=77, prec=pr, slq_prec=sp,
                              precond_rank=rank)
        loss, grad, info = api.gp_loss_and_grad(Xs, ys, sub.kind, sub.theta, opts)
        res[name] = (loss, grad)
        key = name if rank == 0 else f"nystrom{rank_sub}_{name}"
        out[key] = {"relerr_loss_vs_exact_n4000": abs(loss - lref) / abs(lref),
                    "relerr_grad_vs_exact_n4000": relgrad(grad, gref),
                    "logdet_stderr": info["logdet_stderr"], "cg_iters": info["cg_iters"]}
        if rank and name != "fp32":
            out[key]["reldiff_loss_vs_fp32_same_probes"] = abs(loss - res["fp32"][0]) / abs(res["fp32"][0])
            out[key]["reldiff_grad_vs_fp32_same_probes"] = relgrad(grad, np.asarray(res["fp32"][1]))
    full = inputs.diff_problem(seed=0, n=full_n)
    Xf, yf = torch.from_numpy(full.X).cuda(), torch.from_numpy(full.y).cuda()
    base = None
    for name, pr, sp in arms:
        opts = api.solve_opts(nprobe=32, nlanczos=40, cg_rtol=1e-6, seed=77, prec=pr, slq_prec=sp,
                              precond_rank=rank_full)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss, grad, info = api.gp_loss_and_grad(Xf, yf, full.kind, full.theta, opts)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        rec = {"ms_per_theta": ms, "loss": loss, "grad": grad, "cg_iters": info["cg_iters"],
               "relres_max": info["relres_max"], "logdet_stderr": info["logdet_stderr"],
               "trace_stderr": info["trace_stderr"],
               "roofline": precond_lossgrad_roofline(full_n, 8, False, 32, 40, info["cg_iters"],
                                                     rank_full, ms, rates)}
        if m_identity_ms:
            rec["speedup_vs_m_identity_fp32"] = m_identity_ms / ms
        if base is None:
            base = (loss, np.asarray(grad), ms)
        else:
            rec["reldiff_loss_vs_fp32_same_probes"] = abs(loss - base[0]) / abs(base[0])
            rec["reldiff_grad_vs_fp32_same_probes"] = relgrad(grad, base[1])
            rec["speedup_vs_nystrom_fp32"] = base[2] / ms
        out[f"nystrom{rank_full}_{name}_n{full_n}"] = rec
    # The fastest split arithmetic whose loss and gradient stay within 1e-4 of
    # FP32 on the same probes (at the full n and on the subsample).
    ok = [nm for nm, _, _ in arms[1:]
          if out[f"nystrom{rank_full}_{nm}_n{full_n}"].get("reldiff_loss_vs_fp32_same_probes", 1.0) <= 1e-4
          and out[f"nystrom{rank_full}_{nm}_n{full_n}"].get("reldiff_grad_vs_fp32_same_probes", 1.0) <= 1e-4
          and out[f"nystrom{rank_sub}_{nm}"]["reldiff_loss_vs_fp32_same_probes"] <= 1e-4
          and out[f"nystrom{rank_sub}_{nm}"]["reldiff_grad_vs_fp32_same_probes"] <= 1e-4]
    best = min(ok, key=lambda nm: out[f"nystrom{rank_full}_{nm}_n{full_n}"]["ms_per_theta"]) if ok else None
    rec = out[f"nystrom{rank_full}_{best}_n{full_n}"] if best else {}
    out["mixed_at_1e-4"] = {"arithmetic": best, "ms_per_theta": rec.get("ms_per_theta"),
                            "speedup_vs_nystrom_fp32": rec.get("speedup_vs_nystrom_fp32"),
                            "speedup_vs_m_identity_fp32": rec.get("speedup_vs_m_identity_fp32")}
    return out


def loss_grad_precond(api, B, torch, rates: dict, full_n: int = 200_000, rank_sub: int = 800,
                      rank_full: int = 1500, p: int = 16, k: int = 30, cap_plain: int = 300) -> dict:
    """Eq. 1 / Eq. 2 with the Nystrom preconditioner on the precision problem's kernel
    (d = 2 uniform, Gaussian f = 1, l = 0.05, s = 0.01).  On the n = 4000 subsample:
    the error of the estimate (p probes x k Lanczos steps, CG to 1e-8) against the
    exact L and dL/dTheta (Cholesky, stored FP64 values) for M = I (Rademacher
    probes) and for the rank-rank_sub Nystrom M (Gaussian probes z ~ N(0, M)), with
    the estimator's standard errors.  At n = full_n: the time per Theta with the
    rank-rank_full preconditioner (CG to 1e-6), its CG iterations and standard
    errors, against M = I with CG capped at cap_plain iterations (which does not
    reach 1e-6 there)."""
    from paper_2503_02259_gb300 import inputs
    sub = inputs.precision_problem(seed=0, n=4000)
    refs = _refs()
    lref, gref = float(refs["preck_loss"]), np.asarray(refs["preck_grad"])
    floor = 1e-3 * np.linalg.norm(gref)
    out = {"workload": f"precision problem's kernel; accuracy vs the exact loss and gradient on the "
                       f"n=4000 subsample ({p} probes x {k} Lanczos steps, CG 1e-8); time at "
                       f"n={full_n} (CG 1e-6; M = I capped at {cap_plain} CG iterations)"}
    Xs, ys = torch.from_numpy(sub.X).cuda(), torch.from_numpy(sub.y).cuda()

    def relgrad(grad, ref, fl):
        return max(abs(g - r) / max(abs(r), fl) for g, r in zip(grad, ref))

    # The split tensor-core arithmetics run on the same probes as FP32 (the
    # generator does not depend on the arithmetic), so their difference from the
    # FP32 arm is the arithmetic's own error.
    arms = (("m_identity", {}), (f"nystrom_rank{rank_sub}", {"precond_rank": rank_sub}))
    arms += tuple((f"nystrom_rank{rank_sub}_{tag}", {"precond_rank": rank_sub, "prec": pc, "slq_prec": sp})
                  for tag, pc, sp in PRECOND_TC_ARMS)
    for name, extra in arms:
        opts = api.solve_opts(nprobe=p, nlanczos=k, cg_rtol=1e-8, cg_maxit=20000, seed=0, **extra)
        loss, grad, info = api.gp_loss_and_grad(Xs, ys, sub.kind, sub.theta, opts)
        out[name] = {"relerr_loss_vs_exact_n4000": abs(loss - lref) / abs(lref),
                     "relerr_grad_vs_exact_n4000": relgrad(grad, gref, floor),
                     "logdet_stderr": info["logdet_stderr"], "trace_stderr": info["trace_stderr"],
                     "cg_iters": info["cg_iters"]}
        if "prec" in extra:
            base = out[f"nystrom_rank{rank_sub}"]
            out[name]["reldiff_loss_vs_fp32_same_probes"] = abs(loss - base["_loss"]) / abs(base["_loss"])
            out[name]["reldiff_grad_vs_fp32_same_probes"] = relgrad(
                grad, base["_grad"], 1e-3 * np.linalg.norm(base["_grad"]))
        elif "precond_rank" in extra:
            out[name]["_loss"], out[name]["_grad"] = loss, np.asarray(grad)
    base = out[f"nystrom_rank{rank_sub}"]
    del base["_loss"], base["_grad"]
    full = inputs.precision_problem(seed=0, n=full_n)
    Xf, yf = torch.from_numpy(full.X).cuda(), torch.from_numpy(full.y).cuda()

    def timed(opts):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            res, st = api.gp_loss_and_grad(Xf, yf, full.kind, full.theta, opts), 0
        except B.GPError as exc:
            res, st = None, exc.status
        torch.cuda.synchronize()
        return res, st, (time.perf_counter() - t0) * 1e3

    res, st, ms = timed(api.solve_opts(nprobe=p, nlanczos=k, cg_rtol=1e-6, cg_maxit=2000, seed=0,
                                       precond_rank=rank_full))
    rec = {"ms_per_theta": ms, "status": st}
    if res is not None:
        loss, grad, info = res
        rec.update({"loss": loss, "grad": grad, "cg_iters": info["cg_iters"],
                    "relres_max": info["relres_max"], "logdet_stderr": info["logdet_stderr"],
                    "trace_stderr": info["trace_stderr"], "logdet_m": info["logdet_m"],
                    "products_roofline": lossgrad_roofline(full_n, 2, False, p, k, info["cg_iters"],
                                                           ms, rates)})
    out[f"nystrom_rank{rank_full}_n{full_n}"] = rec
    for tag, pc, sp in PRECOND_TC_ARMS:
        r2, st2, ms2 = timed(api.solve_opts(nprobe=p, nlanczos=k, cg_rtol=1e-6, cg_maxit=2000, seed=0,
                                            precond_rank=rank_full, prec=pc, slq_prec=sp))
        arm = {"ms_per_theta": ms2, "status": st2}
        if r2 is not None and res is not None:
            l2, g2, i2 = r2
            arm.update({"cg_iters": i2["cg_iters"], "relres_max": i2["relres_max"],
                        "reldiff_loss_vs_fp32_same_probes": abs(l2 - rec["loss"]) / abs(rec["loss"]),
                        "reldiff_grad_vs_fp32_same_probes": relgrad(
                            g2, rec["grad"], 1e-3 * np.linalg.norm(rec["grad"])),
                        "speedup_vs_fp32": ms / ms2})
        out[f"nystrom_rank{rank_full}_n{full_n}_{tag}"] = arm
    _, st0, ms0 = timed(api.solve_opts(nprobe=p, nlanczos=k, cg_rtol=1e-6, cg_maxit=cap_plain, seed=0))
    out[f"m_identity_n{full_n}_capped"] = {"ms_per_theta": ms0, "cg_iters": cap_plain,
                                           "status": st0, "converged_to_1e-6": st0 == 0}
    return out


# (tag, CG arithmetic, Lanczos arithmetic) of the preconditioned loss's tensor-core arms.
PRECOND_TC_ARMS = (("bf16x3_slq_tf32x3", 4, 3), ("tf32x3", 3, 3))


# (name, CG arithmetic, SLQ arithmetic, max_batch): max_batch > 1 runs compatible
# loss + gradient requests as batches with one grouped product launch per step.
SERVING_ARMS = (("fp32", 0, 0, 1), ("bf16x3_slq_tf32x3", 4, 3, 1))
SERVING_ARMS_ALL = SERVING_ARMS + (("fp32_batched", 0, 0, 8), ("tf32x3", 3, 3, 1))


def serving_accuracy(torch, precs=SERVING_ARMS, slots: int = 8, budget_gb: int = 32) -> dict:
    """The served result at convergence: the stream's small requests (the first 24 with
    n <= 3000; tests/golden/bench_refs.npz) solved to cg_rtol 1e-8 (cap 6000
    iterations) in each arithmetic, against FP64 oracle values (the same-probe
    estimator with exact solves for loss+grad, the exact posterior mean at 200 test
    points for predictions).  Errors are reported over the requests that converged
    in every arm, for all of them and for those with kappa(Kh) <= 1e4 (the stored
    condition numbers): a solution's error is about kappa times the product's
    relative error in any arithmetic."""
    from paper_2503_02259_gb300 import inputs, server
    refs = _refs()
    idx = refs["serving_idx"]
    reqs = inputs.serving_stream(seed=0, count=512)
    sel = [reqs[int(i)] for i in idx]
    kappa = refs["serving_kappa"]
    out = {"workload": f"{len(sel)} requests of the serving stream with n <= 3000 (16 probes, "
                       "20 Lanczos steps), CG to rtol 1e-8 (cap 6000), vs FP64 oracle values",
           "kappa_p50": float(np.median(kappa)), "kappa_max": float(kappa.max()),
           "requests_kappa_le_1e4": int((kappa <= 1e4).sum())}
    res = {}
    for name, prec, slq, mb in precs:
        with server.Server(budget_gb << 30, slots, max_batch=mb) as srv:
            tickets = []
            for rq in sel:
                p = rq.problem
                r, keep = server.Server.request(rq.kind, p.X, p.y, p.kind, p.theta, nprobe=rq.nprobe,
                                                Xstar=rq.Xstar, cg_maxit=6000, nlanczos=20,
                                                cg_rtol=1e-8, seed=0, prec=prec, slq_prec=slq)
                tickets.append(srv.submit(r, keep))
            t0 = time.perf_counter()
            srv.drain(600)
            wall = time.perf_counter() - t0
            res[name] = [srv.poll(t) for t in tickets]
        out[name] = {"converged": sum(r["status"] == 0 for r in res[name]), "of": len(sel),
                     "wall_s": wall}
    both = [k for k in range(len(sel)) if all(res[nm][k]["status"] == 0 for nm, _, _, _ in precs)]

    def q(v, pc):
        return float(np.percentile(v, pc)) if v else None

    for name, _, _, _ in precs:
        for tag, keep in (("", both), ("_kappa_le_1e4", [k for k in both if kappa[k] <= 1e4])):
            el, eg, em = [], [], []
            for k in keep:
                r = res[name][k]
                if sel[k].kind == 0:
                    lref = float(refs["serving_loss"][k])
                    gref = np.asarray(refs["serving_grad"][k])
                    floor = 1e-3 * np.linalg.norm(gref)
                    el.append(abs(r["loss"] - lref) / abs(lref))
                    eg.append(float(np.max(np.abs(np.asarray(r["grad"]) - gref) /
                                           np.maximum(np.abs(gref), floor))))
                else:
                    mref = refs["serving_mu"][k]
                    em.append(float(np.linalg.norm(r["mu"][:mref.size] - mref) /
                                    np.linalg.norm(mref)))
            out[name].update({f"requests_compared{tag}": len(keep),
                              f"relerr_loss_p50{tag}": q(el, 50), f"relerr_loss_p90{tag}": q(el, 90),
                              f"relerr_grad_p50{tag}": q(eg, 50), f"relerr_grad_p90{tag}": q(eg, 90),
                              f"relerr_mu_p50{tag}": q(em, 50), f"relerr_mu_p90{tag}": q(em, 90),
                              f"relerr_max{tag}": max(el + eg + em) if keep else None})
    return out


def serving(torch, count: int = 512, precs=SERVING_ARMS, slots: int = 8, budget_gb: int = 96) -> dict:
    """Replay one Poisson stream of mixed loss+grad and prediction requests through the
    server once per arithmetic: throughput, p50/p99 latency, and how far each mixed
    run's losses, gradients and predictions are from the FP32 run's (same probes, same
    fixed CG budget, so the difference is the product arithmetic alone)."""
    from paper_2503_02259_gb300 import inputs, server
    reqs = inputs.serving_stream(seed=0, count=count)
    work = 0.0
    for rq in reqs:   # entries x columns issued (CG budget 20 / 50, SLQ 20 steps, 1 gradient pass)
        n = rq.problem.n
        work += (n * n * (1 + rq.nprobe) * 41 if rq.kind == 0 else n * n * 50 + n * rq.Xstar.shape[0])
    out = {"workload": f"{count} requests of the serving stream (Poisson 50/s, n log-uniform "
                       "[1e3, 3e5], d in {2,3,8}, 70% loss+grad with 16 probes, 30% prediction at "
                       "m=10000); fixed CG budget 20 (training) / 50 (prediction), SLQ 20 steps",
           "slots": slots, "budget_gb": budget_gb}
    results = {}
    for name, prec, slq, mb in precs:
        with server.Server(budget_gb << 30, slots, max_batch=mb) as srv:
            t0 = time.perf_counter()
            res = server.replay(srv, reqs, prec=prec, slq_prec=slq, nlanczos=20, cg_rtol=1e-12)
            wall = time.perf_counter() - t0
            stats = srv.stats()
        results[name] = res
        lat = np.array([r["latency_from_arrival_s"] for r in res])
        small = np.array([r["latency_from_arrival_s"] for r, rq in zip(res, reqs)
                          if rq.problem.n <= 20000])
        out[name] = {"requests_ok": sum(r["status"] in (0, 4) for r in res), "wall_s": wall,
                     "requests_per_s": len(res) / wall, "entries_cols_per_s": work / wall,
                     "latency_p50_s": float(np.percentile(lat, 50)),
                     "latency_p99_s": float(np.percentile(lat, 99)),
                     "latency_from": "scheduled arrival (Poisson stream time) to completion",
                     "latency_p99_s_n_le_2e4": float(np.percentile(small, 99)) if small.size else None,
                     "peak_active": stats["peak_active"], "peak_bytes": stats["peak_bytes"],
                     "max_batch": mb, "batches": stats["batches"],
                     "batched_requests": stats["batched_requests"],
                     "largest_batch": stats["largest_batch"]}
    # Accuracy of a fixed-budget solve is its final CG residual (the budget, not the
    # arithmetic, decides how far from K-hat^-1 y the iterate is): compare each mixed
    # arm's residual with the FP32 arm's, request by request, and report how far the
    # results themselves moved.
    def q(v, p):
        return float(np.percentile(v, p)) if v else None

    ref = results.get("fp32")
    if ref is not None:
        for name, _, _, _ in precs:
            if name == "fp32":
                continue
            ratio, dl, dg, dm = [], [], [], []
            for a, b, rq in zip(results[name], ref, reqs):
                if b["relres"] > 0:
                    ratio.append(a["relres"] / b["relres"])
                if rq.kind == 0:
                    dl.append(abs(a["loss"] - b["loss"]) / abs(b["loss"]))
                    g, gr = np.asarray(a["grad"]), np.asarray(b["grad"])
                    floor = 1e-3 * np.linalg.norm(gr)
                    dg.append(float(np.max(np.abs(g - gr) / np.maximum(np.abs(gr), floor))))
                else:
                    dm.append(float(np.linalg.norm(a["mu"] - b["mu"]) / np.linalg.norm(b["mu"])))
            out[name].update({
                "relres_ratio_vs_fp32_p50": q(ratio, 50), "relres_ratio_vs_fp32_p90": q(ratio, 90),
                "reldiff_loss_vs_fp32_p50": q(dl, 50), "reldiff_loss_vs_fp32_p90": q(dl, 90),
                "reldiff_grad_vs_fp32_p50": q(dg, 50), "reldiff_grad_vs_fp32_p90": q(dg, 90),
                "reldiff_mu_vs_fp32_p50": q(dm, 50), "reldiff_mu_vs_fp32_p90": q(dm, 90),
                "throughput_vs_fp32": out["fp32"]["wall_s"] / out[name]["wall_s"]})
        out["fp32"]["relres_p50"] = q([r["relres"] for r in ref], 50)
    return out


def loss_grad_small(api, torch, rates: dict, reps: int = 3) -> dict:
    """Loss + gradient per Theta on the small configuration (n=2000, d=3, Gaussian)."""
    from paper_2503_02259_gb300 import inputs
    prob = inputs.small_problem(seed=0)
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    opts = api.solve_opts(nprobe=10, nlanczos=30, cg_rtol=1e-8, seed=1234)
    api.gp_loss_and_grad(X, y, prob.kind, prob.theta, opts)
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss, grad, info = api.gp_loss_and_grad(X, y, prob.kind, prob.theta, opts)
        ts.append((time.perf_counter() - t0) * 1e3)
    ms = statistics.median(ts)
    return {"workload": "n=2000 d=3 uniform, Gaussian f=1 l=0.3 s=0.1, block CG on [y|10 probes] "
                        "to rtol 1e-8, SLQ 10x30, Hutchinson, FP32",
            "ms": ms, "loss": loss, "grad": grad, "cg_iters": info["cg_iters"],
            "roofline": lossgrad_roofline(prob.n, 3, False, 10, 30, info["cg_iters"], ms, rates)}


def run_leg(args) -> int:
    """One extra leg alone (the same code the full run calls), for profiling it."""
    import torch
    from paper_2503_02259_gb300 import build
    build.build()
    from paper_2503_02259_gb300 import _binding as B
    from paper_2503_02259_gb300 import api, inputs
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    rates = measure_rates(B, api, dev)
    if args.leg == "loss_grad":
        out = loss_grad_small(api, torch, rates)
    elif args.leg == "precision_modes":
        prob = inputs.matvec_problem(seed=0)
        X = torch.from_numpy(prob.X).to(dev)
        V = torch.from_numpy(inputs.multivector(prob.y, W, seed=0)).to(dev)
        out = precision_modes(api, B, torch, prob, X, V, dev, rates)
    elif args.leg == "precision_config":
        out = precision_config(api, B, torch, dev)
    elif args.leg == "refinement":
        out = refinement(api, torch)
    elif args.leg == "precision_refinement":
        out = precision_refinement(api, B, torch, n=args.precision_n)
    elif args.leg == "loss_grad_mixed_vs_fp32":
        out = loss_grad_mixed_vs_fp32(api, torch, rates)
    elif args.leg == "loss_grad_precond":
        out = loss_grad_precond(api, B, torch, rates)
    elif args.leg == "loss_grad_diff_precond":
        out = loss_grad_diff_precond(api, torch, rates, full_n=args.precond_n)
    elif args.leg == "serving_accuracy":
        out = serving_accuracy(torch)
    else:
        out = serving(torch, count=args.serving_requests,
                      precs=SERVING_ARMS_ALL if args.serving_all_arms else SERVING_ARMS)
    print(json.dumps({"leg": args.leg, **out}), flush=True)
    return 0


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gp", choices=["gp", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--prec", default="fp32", choices=list(PRECS), help="arithmetic of the product")
    ap.add_argument("--serving-requests", type=int, default=512,
                    help="requests replayed by the serving leg (the full stream is 512)")
    ap.add_argument("--serving-all-arms", action="store_true",
                    help="also replay the stream with batched FP32 requests and in split TF32")
    ap.add_argument("--precision-n", type=int, default=1_000_000,
                    help="points of the precision_refinement leg when run alone (smaller n for "
                         "profiling; the full run always uses 1e6)")
    ap.add_argument("--precond-n", type=int, default=200_000,
                    help="points of the loss_grad_diff_precond leg when run alone (smaller n for "
                         "profiling; the full run always uses 2e5)")
    ap.add_argument("--leg", default=None,
                    choices=["loss_grad", "precision_modes", "precision_config", "refinement",
                             "precision_refinement", "loss_grad_precond", "loss_grad_diff_precond",
                             "loss_grad_mixed_vs_fp32", "serving", "serving_accuracy"],
                    help="run one extra leg alone on cuda:0 and print its JSON (for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.leg is not None:
        return run_leg(args)

    import torch
    from paper_2503_02259_gb300 import build
    build.build()
    from paper_2503_02259_gb300 import _binding as B
    from paper_2503_02259_gb300 import api, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    prob = inputs.matvec_problem(seed=0)
    Vh = inputs.multivector(prob.y, W, seed=0)
    X = torch.from_numpy(prob.X).to(dev)
    V = torch.from_numpy(Vh).to(dev)
    Y = torch.empty_like(V)
    dYf = torch.empty_like(V)
    dYl = torch.empty_like(V)
    pr, _ = api.problem(X, prob.kind, prob.theta)
    prec = PRECS[args.prec]
    ws = api.workspace(B.OP_GRAD_MATMUL, pr, W, api.solve_opts(prec=prec), dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    L = B.lib()
    stream = torch.cuda.current_stream(dev)

    def step():
        B.check(L.gp_kernel_grad_matmul(B.ctypes.byref(pr), api._ptr(V), W, api._ptr(Y),
                                        api._ptr(dYf), api._ptr(dYl), prec, api._ptr(ws),
                                        ws.numel(), api._stream(dev)), "gp_kernel_grad_matmul")

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    B.check(L.gp_profile_begin(), "gp_profile_begin")
    for i in range(args.steps):
        flush.zero_()                     # L2 flushed between steps, outside the timed bracket
        starts[i].record(stream)
        step()
        stops[i].record(stream)
    torch.cuda.synchronize()
    prod_ms = B.c_double()
    prod_n = B.c_int64()
    launches = B.c_int64()
    B.check(L.gp_profile_end(B.ctypes.byref(prod_ms), B.ctypes.byref(prod_n),
                             B.ctypes.byref(launches)), "gp_profile_end")
    step_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(starts, stops)), dist, dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None

    # End to end through the public call with host buffers: pinned H2D of X and V,
    # the call, D2H of the three outputs, every step.
    e2e_steps = min(args.steps, 10)
    Xp = torch.from_numpy(prob.X).pin_memory()
    Vp = torch.from_numpy(Vh).pin_memory()
    outs = [torch.empty((N_PTS, W), dtype=torch.float32).pin_memory() for _ in range(3)]
    Xd = torch.empty_like(X)
    Vd = torch.empty_like(V)
    pr2, _ = api.problem(Xd, prob.kind, prob.theta)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        Xd.copy_(Xp, non_blocking=True)
        Vd.copy_(Vp, non_blocking=True)
        B.check(L.gp_kernel_grad_matmul(B.ctypes.byref(pr2), api._ptr(Vd), W, api._ptr(Y),
                                        api._ptr(dYf), api._ptr(dYl), prec, api._ptr(ws),
                                        ws.numel(), api._stream(dev)), "gp_kernel_grad_matmul")
        for o, src in zip(outs, (Y, dYf, dYl)):
            o.copy_(src, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, dist, dev)
    h2d = Xp.numel() * 4 + Vp.numel() * 4
    d2h = 3 * N_PTS * W * 4

    # Measured pipe rates of this GPU (microbenchmarks, after the timed region).
    rates = measure_rates(B, api, dev)
    extras = {}
    if rank == 0 and not args.no_extras:
        # Each extra leg runs after the headline measurement; a leg that fails
        # records its error in the line instead of taking the line with it.
        legs = (("loss_grad", lambda: loss_grad_small(api, torch, rates)),
                ("precision_modes", lambda: precision_modes(api, B, torch, prob, X, V, dev, rates)),
                ("precision_config", lambda: precision_config(api, B, torch, dev)),
                ("refinement", lambda: refinement(api, torch)),
                ("precision_refinement", lambda: precision_refinement(api, B, torch)),
                ("loss_grad_mixed_vs_fp32", lambda: loss_grad_mixed_vs_fp32(api, torch, rates)),
                ("loss_grad_diff_precond", lambda: loss_grad_diff_precond(
                    api, torch, rates, (extras.get("loss_grad_mixed_vs_fp32", {}).get("fp32") or {})
                    .get("ms_per_theta"))),
                ("loss_grad_precond", lambda: loss_grad_precond(api, B, torch, rates)),
                ("serving", lambda: serving(torch, count=args.serving_requests,
                                            precs=SERVING_ARMS_ALL if args.serving_all_arms
                                            else SERVING_ARMS)),
                ("serving_accuracy", lambda: serving_accuracy(torch)))
        for name, leg in legs:
            try:
                extras[name] = leg()
            except Exception as exc:  # noqa: BLE001 - reported in the JSON line
                extras[name] = {"error": f"{type(exc).__name__}: {exc}"[:500]}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    per_step_ms = step_ms / args.steps
    work = N_PTS * N_PTS * W
    value = replica_rate(world, work, per_step_ms)
    peaks = _peaks()
    sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 2070.0
    kern_ms = prod_ms.value / max(1, prod_n.value)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    if prec == 0:
        # FP32 pipe: evaluation (3d + 6 flops per entry, Matern) + contraction (4w per entry).
        flops_per_launch = N_PTS * N_PTS * (4 * W + 3 * D + 6)
        peak = 2 * 128 * nsm * sm_mhz * 1e6 / 1e12
        tr = _traffic().get("kmv_simt_matern_d3_w32_grad")
        kname = "kmv_simt_kernel<MATERN32,grad,D=3,TW=32>"
        bound = "alu"
        psrc = (f"FP32 pipe: {nsm} SMs (cudaDevAttrMultiProcessorCount) x 128 lanes x 2 flop x "
                f"{sm_mhz:.0f} MHz (median sampled SM clock in the timed region)")
    else:
        # Tensor pipe: products per entry = NPROD x 2 (K and D) x 2w flops.
        nprod = {1: 1, 2: 2, 3: 3, 4: 3}[prec]
        flops_per_launch = N_PTS * N_PTS * 2 * W * nprod * 2
        ratio = 0.5 if prec in (1, 3) else 1.0
        peak = peaks.get("bf16_tflops", 1900.0) * ratio
        tr = _traffic().get(f"kmv_tc_matern_d3_w32_grad_{args.prec}")
        kname = f"kmv_tc_kernel<MATERN32,grad,D=3,{args.prec}>"
        bound = "tensor"
        psrc = ("measured cuBLAS bf16 dense peak (MEASURED_PEAKS.json)"
                + (" x 0.5, the nominal tf32:bf16 ratio" if ratio != 1.0 else ""))
    achieved = flops_per_launch / (kern_ms * 1e-3) / 1e12
    roofline = {"bound": bound, "kernel": kname,
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": tr.get("bytes_per_launch") if tr else None,
                "peak_source": psrc,
                "kernel_ms": kern_ms, "algorithmic_flops_per_launch": flops_per_launch,
                "kernel_share_of_step": kern_ms / per_step_ms,
                "pipe_rates_measured": {**rates,
                                        "frac_of_measured_fp32": (achieved / rates["fp32_ffma2_tflops"]
                                                                  if prec == 0 else None)}}
    if prec != 0:
        # The tensor-core product is bound by the kernel evaluation (MUFU) far
        # more than by the tensor pipe at these widths: report against the
        # binding floor, with both fractions alongside.
        tcr = tc_roofline(N_PTS, D, 32, True, True, prec, kern_ms, rates, peaks)
        roofline["evaluation_and_tensor"] = tcr
        if tcr["binding"] == "mufu":
            mufu_ops = N_PTS * N_PTS * 2.0
            roofline.update({"bound": "alu", "achieved": mufu_ops / (kern_ms * 1e-3) / 1e12,
                             "peak": rates["mufu_ex2_gops"] / 1e3, "unit": "Top/s (MUFU)",
                             "frac": tcr["mufu_frac"],
                             "peak_source": "measured MUFU ex2 rate of this GPU "
                                            "(gp_measure_pipe_rates); 2 MUFU (sqrt, ex2) per "
                                            "Matern-3/2 entry"})
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_oracle_rate()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f32", 1: "tf32", 2: "bf16", 3: "tf32x3", 4: "bf16x3"}[prec],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "flushed between steps (256 MiB write outside "
                                                   "the timed bracket)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": replica_rate(world, work, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": int(launches.value), "clocks": clocks}
    line.update(extras)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
