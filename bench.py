#!/usr/bin/env python
"""Benchmark: time to solve the space-time KKT system to 1e-8 on one GB300.

Workload: the 32^3-cell x 64-step inverse source problem (35,937 nodes x 65
levels x 3 unknowns = 7,007,715 unknowns), two moving sources, 125 sensors,
1% noise, a(x) from a seeded smooth field, v = (1,1,0) sin(pi z), Dirichlet on
x = 0; two-level space-time RAS with 4x4x4x4 subdomains, overlap 2, ILU(0)
local solves; coarse mesh 16^3 x 32 with overlap 1 and a 4-step coarse GMRES
at tolerance 0.1; FGMRES(30) to a true relative residual of 1e-8, zero
initial guess.

One step = one full solve from observations to recovered source, i.e. every
step of the hot path: right-hand side from the observations, refactorisation
of the fine and coarse subdomain ILU(0) factors, the preconditioned FGMRES
solve (KKT matvecs, RAS gather/solve/scatter, restriction, coarse GMRES,
interpolation, two-level combination, CGS2 Arnoldi, true residual) and the
extraction of the source.  The headline `value` is the mixed form (FP32
subdomain and coarse factors, FP64 Krylov); the plain FP64 form is timed on
the same GPU and reported beside it.

Multi-GPU: the path does not shard across GPUs here; N ranks run N
independent replicas (weak scaling, no collective on the data path; one
barrier and a max-reduction of the elapsed time only).

--impl reference times the CPU oracle on a bounded sample of the same
workload and extrapolates to one solve (the sample is described in the
output line).
"""

from __future__ import annotations

import argparse
import dataclasses
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "KKT solve s to 1e-8 rel. residual (mixed vs FP64) at 32^3x64; matvec HBM GB/s"
UNIT = "s"
OBS_FILE = os.path.join(ROOT, "tests", "golden", "observations_mid_32x32x32x64.txt")
# the same observations from a forward solve on a 2x finer mesh (the paper's data protocol)
OBS_FILE_REFINED = os.path.join(ROOT, "tests", "golden", "observations_mid_32x32x32x64_refined2.txt")
# observations of the 64^3 x 128 workload (same-mesh forward solve)
OBS_FILE_LARGE = os.path.join(ROOT, "tests", "golden", "observations_large_64x64x64x128.txt")


def obs_file(args) -> str:
    return OBS_FILE_REFINED if getattr(args, "data", "same-mesh") == "refined2" else OBS_FILE
# Two-level FGMRES(30) iterations of this workload to 1e-8, as the GPU solve
# measures them; the oracle runs the same algorithm, so its extrapolated solve
# time uses the same count.
ORACLE_ITERATIONS = 23
FALLBACK_HBM_GBS = 6800.0
SLOTS_PER_POINT = 326   # stored ILU(0) values per space-time point (C, G, f rows: 108 + 56 + 162)


def config_dict(w, extra=None):
    d = {
        "workload": "inverse source KKT, 32^3 cells x 64 steps, 7,007,715 unknowns",
        "grid_cells": list(w.cells), "steps": w.M, "unknowns": w.unknowns, "sensors": len(w.sensor_xyz),
        "subdomains": list(w.nsub), "overlap": w.overlap, "local_solver": "ILU(0)",
        "coarse": list(w.coarse_cells) + [w.coarse_M], "coarse_overlap": w.coarse_overlap,
        "coarse_gmres": {"rtol": w.coarse_rtol, "maxit": w.coarse_maxit},
        "outer": f"FGMRES({w.restart}) rtol {w.rtol}", "factor_precision": "fp32 (mixed form)",
        "l2": "no flush needed: each step streams > 9 GB of factors (L2 129 MB)",
        "parallelism": "replicas",
    }
    if extra:
        d.update(extra)
    return d


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle: bounded sample of the same workload
# ---------------------------------------------------------------------------

def oracle_sample(iterations: int, budget_rows: int = 15000):
    """Time the oracle's pieces on the 32^3 x 64 workload and extrapolate one solve.

    Sample: one level-wise FP64 KKT matvec; the ILU(0) factorisation and the
    triangular solve of the leading `budget_rows` rows of one interior fine
    subdomain and of one coarse subdomain (their per-row costs times the
    rows of all subdomains); the CGS2 vector work from numpy dot products.
    """
    import numpy as np

    from oracle import kkt, schwarz
    from paper_1508_06103_gb300 import workloads as W

    w = W.mid()
    t_all = time.time()
    p = kkt.Problem.from_workload(w)
    x = np.random.default_rng(0).standard_normal(p.n)
    t = time.time()
    kkt.apply(p, x)
    t_mv = time.time() - t
    t = time.time()
    for _ in range(4):
        float(np.add.reduce(x * x))   # numpy's own loop: one thread (a BLAS dot may use several)
    t_dot = (time.time() - t) / 4

    def box_costs(pp, nsub, overlap, rows):
        bxs = schwarz.boxes(pp, nsub, overlap)
        # an interior box (index of part 1 along every axis)
        k = 1 + nsub[0] * (1 + nsub[1] * (1 + nsub[2] * 1))
        b = bxs[min(k, len(bxs) - 1)]
        nodes, levels = schwarz.box_nodes_levels(pp, b)
        t0 = time.time()
        A = schwarz.kkt.assemble_box(pp, nodes, levels)
        idx, _ = schwarz.box_unknowns(pp, b)
        rows = min(rows, A.shape[0])
        pat = schwarz.local_pattern(pp, idx, rows=rows)
        ilu = schwarz.ILU0(A, pat, rows=rows)
        t_fac = time.time() - t0
        t0 = time.time()
        ilu.solve(np.ones(rows))
        t_sol = time.time() - t0
        total_rows = sum(3 * int(np.prod(bb.shape())) for bb in bxs)
        return t_fac / rows * total_rows, t_sol / rows * total_rows, rows

    fac_f, sol_f, rows_f = box_costs(p, w.nsub, w.overlap, budget_rows)
    pc = schwarz.coarse_problem(p, w.coarse_cells, w.coarse_M)
    fac_c, sol_c, rows_c = box_costs(pc, w.coarse_split, w.coarse_overlap, budget_rows // 2)
    t = time.time()
    kkt.apply(pc, np.ones(pc.n))
    t_mv_c = time.time() - t
    per_iter = (sol_f + 2 * t_mv + w.coarse_maxit * (sol_c + t_mv_c + 4 * 3 * t_dot / 14)
                + np.mean([4 * (j + 1) + 2 for j in range(min(iterations, w.restart))]) * t_dot)
    est = fac_f + fac_c + iterations * per_iter
    sample = (f"oracle (numpy/scipy, FP64, single-threaded Python loops) on the 32^3x64 workload: one level-wise "
              f"KKT matvec ({t_mv:.2f} s), ILU(0) factor+solve of the leading {rows_f} rows of an interior fine "
              f"subdomain and {rows_c} rows of a coarse one, single-threaded numpy reductions for CGS2; extrapolated to all subdomain "
              f"rows and {iterations} FGMRES iterations; sample wall {time.time() - t_all:.1f} s")
    measured = {"matvec_levelwise_32x32x32x64_s": t_mv, "config1": oracle_config1()}
    return est, sample, measured


def oracle_config1():
    """The oracle's whole solve of the 8^3 x 16 implicit-Euler workload, timed end to end (measured,
    not extrapolated): assembly of F_h, one-level RAS 2x2x2x2 with exact local LU (SuperLU), GMRES(30)
    to 1e-8, on one core."""
    from oracle import forward, kkt, krylov, schwarz
    from paper_1508_06103_gb300 import workloads as W

    w = W.tiny(theta=1.0)
    p = kkt.Problem.from_workload(w)
    cobs = forward.observations(p, forward.forward_march(p, w.true_source()), w.noise(), w.noise_eps)
    t0 = time.time()
    b = kkt.rhs(p, cobs)
    F = kkt.assemble(p)
    ras = schwarz.RAS(p, F, w.nsub, w.overlap, "lu")
    t1 = time.time()
    sol = krylov.gmres(lambda u: F @ u, b, ras.apply, restart=30, rtol=1e-8, maxit=400)
    t2 = time.time()
    return {"workload": "8^3 x 16 implicit Euler, one-level RAS 2x2x2x2 overlap 1, exact local LU, GMRES(30) to 1e-8",
            "setup_s": t1 - t0, "solve_s": t2 - t1, "total_s": t2 - t0, "iterations": sol.iterations,
            "true_relres": sol.relres}


def gpu_config1(api, W):
    """The same 8^3 x 16 solve on the GPU (set-up of the exact local LU factors + GMRES to 1e-8)."""
    import torch

    from oracle import forward, kkt

    w = W.tiny(theta=1.0)
    p = kkt.Problem.from_workload(w)
    cobs = torch.from_numpy(forward.observations(p, forward.forward_march(p, w.true_source()), w.noise(),
                                                 w.noise_eps)).cuda()
    prob = api.Problem.from_workload(w)
    out = {}
    for rep in range(2):   # the first pass loads the kernels
        torch.cuda.synchronize()
        t0 = time.time()
        ras = api.RAS(prob, w.nsub, w.overlap, 64, local="lu")
        b = prob.rhs(cobs)
        t1 = time.time()
        x, st, its, rel = api.gmres_solve(prob, b, ras=ras, restart=30, rtol=1e-8, maxit=400)
        torch.cuda.synchronize()
        t2 = time.time()
        out = {"setup_s": t1 - t0, "solve_s": t2 - t1, "total_s": t2 - t0, "iterations": its, "true_relres": rel}
        ras.close()
    return out


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1508_06103_gb300 import workloads as W

    w = W.mid()
    vals = []
    sample = ""
    for _ in range(args.warmup):
        pass   # the oracle has no warm-up state; warm-up steps are not repeated
    t0 = time.time()
    measured = {}
    for _ in range(args.steps):
        v, sample, measured = oracle_sample(ORACLE_ITERATIONS, budget_rows=15000)
        vals.append(v)
    wall = time.time() - t0
    value = float(sorted(vals)[len(vals) // 2])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(w, {"factor_precision": "fp64 (oracle)"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "value_is": "extrapolated from the measured parts of the sample",
                         "host_cores": os.cpu_count(), "measured": measured},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "sample_wall_s": wall,
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def timed_cold(fn, reps: int) -> float:
    """Mean ms of `fn` over `reps` launches, each timed alone with CUDA events on the current
    stream after a write of 256 MB (twice the L2) outside the timed window, so no launch finds
    its inputs in L2 (the FP32 KKT vectors, 56 MB, would fit)."""
    import torch

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    total = 0.0
    for _ in range(reps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    del flush
    return total / reps


def max_over_ranks(ms: float, dist=None, device: str = "cuda") -> float:
    """The largest value over the ranks of the process group (the job's time)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gpu_arm(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1508_06103_gb300 import api, build
    from paper_1508_06103_gb300 import workloads as W

    if rank == 0 or world == 1:
        build.build()
    barrier()
    w = W.mid()
    cobs_np = np.loadtxt(obs_file(args), ndmin=2)
    assert cobs_np.shape == (w.M + 1, len(w.sensor_xyz)), cobs_np.shape
    cobs_host = torch.from_numpy(cobs_np).pin_memory()
    cobs = cobs_host.cuda()
    prob = api.Problem.from_workload(w)
    stream = torch.cuda.current_stream()
    b, x = prob.zeros(), prob.zeros()
    f = torch.empty(prob.levels * prob.N, dtype=torch.float64, device="cuda")
    f_host = torch.empty(prob.levels * prob.N, dtype=torch.float64).pin_memory()

    def make(prec):
        ras = api.RAS(prob, w.nsub, w.overlap, prec)
        co = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.coarse_split, w.coarse_overlap, w.coarse_rtol,
                        w.coarse_maxit, prec)
        return ras, co

    last = {}

    def step(ras, co, obs):
        prob.rhs(obs, out=b)
        co.refactor_with(ras)          # fine and coarse factorisations together
        x.zero_()
        _, st, its, rel = api.gmres_solve(prob, b, x, ras=ras, coarse=co, restart=w.restart, rtol=w.rtol,
                                          maxit=3000)
        prob.recover_source(x, out=f)
        last.update(status=st, iters=its, relres=rel)

    def timed(fn, steps):
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / steps, dist, "cuda")

    # ---- mixed form: the headline -----------------------------------------
    ras, co = make(32)
    for _ in range(args.warmup):
        step(ras, co, cobs)
    launches0 = api.launch_count()
    api.timing_reset(prob, ras)
    api.timing_enable(True)
    with ClockSampler(local) as clk:
        ms = timed(lambda: step(ras, co, cobs), args.steps)
    api.timing_enable(False)
    launches = (api.launch_count() - launches0) // args.steps
    ras_ms, ras_n = ras.timing(0)
    fac_ms, fac_n = ras.timing(1)
    mv_ms, mv_n = api.matvec_timing(prob)
    mixed = dict(last)
    info = ras.info()
    # end-to-end through the public API with host buffers: H2D observations, D2H source
    def e2e_step():
        obs = cobs_host.to("cuda", non_blocking=True)
        step(ras, co, obs)
        f_host.copy_(f, non_blocking=True)

    e2e_ms = timed(e2e_step, max(1, args.steps // 2))

    # set-up and solve apart (outside the timed region): refactorisation of the
    # fine and coarse subdomain factors, and the FGMRES solve from a zero guess
    prob.rhs(cobs, out=b)
    phases = {"refactor_fine_ms": timed(lambda: ras.refactor(), 2),
              "refactor_coarse_ms": timed(lambda: co.refactor(), 2),
              "refactor_together_ms": timed(lambda: co.refactor_with(ras), 2)}

    def solve_only():
        x.zero_()
        api.gmres_solve(prob, b, x, ras=ras, coarse=co, restart=w.restart, rtol=w.rtol, maxit=3000)

    phases["fgmres_solve_ms"] = timed(solve_only, 2)

    # ---- plain FP64 form on the same GPU -----------------------------------
    del ras, co
    torch.cuda.synchronize()
    ras64, co64 = make(64)
    step(ras64, co64, cobs)
    fp64_ms = timed(lambda: step(ras64, co64, cobs), args.fp64_steps)
    fp64 = dict(last)
    del ras64, co64

    # ---- mixed form with BF16-stored factors (FP32 factorisation and sweeps) --
    torch.cuda.synchronize()
    ras16, co16 = make(16)
    step(ras16, co16, cobs)
    bf16_ms = timed(lambda: step(ras16, co16, cobs), args.fp64_steps)
    bf16 = dict(last)
    del ras16, co16

    # ---- the KKT matvec on its own (FP64 and FP32) --------------------------
    xm = torch.randn(prob.n, dtype=torch.float64, device="cuda")
    ym = torch.empty_like(xm)
    xs, ys = xm.float(), torch.empty(prob.n, dtype=torch.float32, device="cuda")
    reps = 20
    mv64_ms = timed_cold(lambda: prob.apply(xm, ym), reps)
    mv32_ms = timed_cold(lambda: prob.apply(xs, ys), reps)
    coef_bytes = 4 * 27 * prob.N
    mv64_bytes = prob.n * 16 + coef_bytes * 8
    mv32_bytes = prob.n * 8 + coef_bytes * 4

    # ---- P1 elements on the Kuhn split, same workload: mixed-form solve and matvecs --
    # (the observations enter b only, so the Q1 forward solve's data serve here too)
    prob.set_element("p1")
    ras1, co1 = make(32)
    step(ras1, co1, cobs)
    p1_ms = timed(lambda: step(ras1, co1, cobs), args.fp64_steps)
    p1 = dict(last)
    del ras1, co1
    p1_mv64_ms = timed_cold(lambda: prob.apply(xm, ym), reps)
    p1_mv32_ms = timed_cold(lambda: prob.apply(xs, ys), reps)
    prob.set_element("q1")
    p1_coef = 4 * 15 * prob.N   # the 15 offsets the split couples

    peak, peak_kind = measured_peaks()
    traffic = {k: read_traffic(k) for k in ("ras_solve", "ilu0_factor", "matvec_tiled")}
    # algorithmic bytes per launch (unpadded values: no chunk padding or unit rows counted)
    vb = info["value_bytes"]
    fvals = info["points"] * SLOTS_PER_POINT
    kernels = {
        "ilu0_factor": dict(desc="ILU(0) of all 256 fine subdomains, FP32 (refactorisation in every step)",
                            ms=fac_ms, n=fac_n, bytes=2 * fvals * vb),
        "ras_solve": dict(desc="fine subdomain ILU(0) solve, all 256 boxes, FP32 factors",
                          ms=ras_ms, n=ras_n, bytes=fvals * vb + info["points"] * 3 * 8 + prob.n * 8),
        "matvec_tiled": dict(desc="outer FP64 KKT matvec (bound by the FP64 pipe, not by HBM)",
                             ms=mv_ms, n=mv_n, bytes=mv64_bytes),
    }
    table = {}
    for k, d in kernels.items():
        avg = d["ms"] / max(d["n"], 1)
        ach = d["bytes"] / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
        table[k] = {"kernel": d["desc"], "avg_launch_ms": avg, "launches_per_step": d["n"] / args.steps,
                    "share_of_step": d["ms"] / args.steps / ms, "alg_bytes_per_launch": d["bytes"],
                    "achieved_gbs": ach, "frac": ach / peak, "traffic": traffic[k]}
    dom = max(table, key=lambda k: table[k]["share_of_step"])
    roof = {"kernel": dom + ": " + table[dom]["kernel"], "bound": "hbm", "achieved": table[dom]["achieved_gbs"],
            "peak": peak, "peak_source": peak_kind, "unit": "GB/s", "frac": table[dom]["frac"],
            "traffic": table[dom]["traffic"], "alg_bytes_per_launch": table[dom]["alg_bytes_per_launch"],
            "avg_launch_ms": table[dom]["avg_launch_ms"], "share_of_step": table[dom]["share_of_step"]}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64",
        "data": "synthetic" + ("" if obs_file(args) == OBS_FILE else " (observations from a 2x finer mesh)"),
        "config": config_dict(w),
        "solves_per_s": world * 1e3 / ms,
        "iterations": mixed.get("iters"), "true_relres": mixed.get("relres"), "status": mixed.get("status"),
        "fp64_form": {"s_per_solve": fp64_ms / 1e3, "iterations": fp64.get("iters"),
                      "true_relres": fp64.get("relres"), "steps": args.fp64_steps},
        "mixed_speedup_vs_fp64": fp64_ms / ms,
        "mixed_phases": phases,
        "bf16_factor_form": {"s_per_solve": bf16_ms / 1e3, "iterations": bf16.get("iters"),
                             "true_relres": bf16.get("relres"), "steps": args.fp64_steps},
        "matvec": {"fp64_gbs": mv64_bytes / (mv64_ms * 1e-3) / 1e9, "fp64_us": mv64_ms * 1e3,
                   "fp32_gbs": mv32_bytes / (mv32_ms * 1e-3) / 1e9, "fp32_us": mv32_ms * 1e3,
                   "fp64_frac": mv64_bytes / (mv64_ms * 1e-3) / 1e9 / peak,
                   "fp32_frac": mv32_bytes / (mv32_ms * 1e-3) / 1e9 / peak,
                   "bytes_fp64": mv64_bytes, "bytes_fp32": mv32_bytes},
        "p1_form": {"s_per_solve": p1_ms / 1e3, "iterations": p1.get("iters"), "true_relres": p1.get("relres"),
                    "steps": args.fp64_steps, "matvec_fp64_us": p1_mv64_ms * 1e3,
                    "matvec_fp32_us": p1_mv32_ms * 1e3,
                    "matvec_fp32_frac": (prob.n * 8 + p1_coef * 4) / (p1_mv32_ms * 1e-3) / 1e9 / peak,
                    "element": "P1 on the Kuhn split of every cell, mixed form (FP32 factors)"},
        "roofline": roof,
        "kernels": table,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_ms / 1e3, "unit": UNIT, "h2d_bytes_per_step": cobs_np.size * 8,
                "d2h_bytes_per_step": prob.levels * prob.N * 8},
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        est, sample, measured = oracle_sample(int(mixed.get("iters") or ORACLE_ITERATIONS))
        line["cpu_baseline"] = {"value": est, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                                "value_is": "extrapolated from the measured parts of the sample",
                                "host_cores": os.cpu_count(), "measured": measured,
                                "gpu_same_config1": gpu_config1(api, W)}
    print(json.dumps(line))


def read_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summaries, if any.

    A summary states it on one line as `traffic <kernel>: <bytes per launch>`.
    """
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for name in sorted(os.listdir(pdir)):
        if not name.endswith((".md", ".txt")):
            continue
        for ln in open(os.path.join(pdir, name)):
            if ln.strip().startswith(f"traffic {kernel}:"):
                try:
                    return float(ln.split(":", 1)[1].split()[0])
                except ValueError:
                    return None
    return None


def kernel_arm(args):
    """One kernel on a member of the same problem family (for profiling and sweeps).

    --kernel ras     : fine one-level RAS apply (subdomain solve), FP32 factors
    --kernel matvec  : FP64 and FP32 KKT matvecs
    """
    import torch

    from paper_1508_06103_gb300 import api, build
    from paper_1508_06103_gb300 import workloads as W

    build.build()
    c, M = args.cells, args.levels
    w = W.mid(cells=(c, c, c), M=M, coarse_cells=None, coarse_M=None, overlap=args.overlap)
    prob = api.Problem.from_workload(w)
    x = torch.randn(prob.n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    out = {"kernel": args.kernel, "cells": c, "levels": M, "unknowns": prob.n}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.kernel == "peaks":
        res = {}
        for prec in (64, 32):
            tf = [api.fma_peak(prec)[0] for _ in range(5)]
            res[f"fp{prec}_fma_tflops"] = max(tf)
            res[f"fp{prec}_fma_tflops_runs"] = tf
        tm = [api.mma_peak()[0] for _ in range(5)]
        res["fp64_mma_tflops"] = max(tm)
        res["fp64_mma_tflops_runs"] = tm
        print(json.dumps({"kernel": "peaks", **res}))
        return
    if args.kernel == "ras":
        shape = None if not (args.chunk or args.stages or args.place) else (args.chunk, args.stages, 0, args.place)
        ras = api.RAS(prob, w.nsub, w.overlap, args.prec, shape=shape)
        ras.apply(x, y)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.reps):
            ras.apply(x, y)
        e1.record()
        torch.cuda.synchronize()
        info = ras.info()
        ms = e0.elapsed_time(e1) / args.reps
        # algorithmic bytes: unpadded factor values, gathered residual, owned output
        by = info["points"] * SLOTS_PER_POINT * info["value_bytes"] + info["points"] * 24 + prob.n * 8
        out.update(info, shape=ras.solve_shape(), ms=ms, alg_bytes=by, gbs=by / ms / 1e6)
    else:
        xs, ys = x.float(), torch.empty(prob.n, dtype=torch.float32, device="cuda")
        for name, (a, b_) in (("fp64", (x, y)), ("fp32", (xs, ys))):
            prob.apply(a, b_)
            ms = timed_cold(lambda: prob.apply(a, b_), args.reps)
            by = prob.n * (16 if name == "fp64" else 8) + 4 * 27 * prob.N * (8 if name == "fp64" else 4)
            out[name] = {"ms": ms, "alg_bytes": by, "gbs": by / ms / 1e6}
    print(json.dumps(out))


def sweep_arm(args):
    """Overlap and level sweep of the mixed-form solve at 32^3 x 64 (the trends of the paper's
    Tables 2 and 3: iterations and time against the overlap, one level against two).

    For each preconditioner: fine FP32 factors with overlap delta (the coarse level as in the
    workload), one refactorisation and one solve untimed, then the refactorisation and
    `--reps` solves timed with CUDA events, SM clocks sampled meanwhile.  One JSON line per
    preconditioner, the workload's own (two levels, overlap 2) first.
    """
    import numpy as np
    import torch

    from paper_1508_06103_gb300 import api, build
    from paper_1508_06103_gb300 import workloads as W

    build.build()
    w = W.mid()
    cobs = torch.from_numpy(np.loadtxt(obs_file(args), ndmin=2)).cuda()
    prob = api.Problem.from_workload(w)
    b, x = prob.zeros(), prob.zeros()
    prob.rhs(cobs, out=b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for levels, delta in ((2, 2), (2, 0), (2, 1), (2, 3), (1, 1), (1, 2)):
        ras = api.RAS(prob, w.nsub, delta, 32)
        co = None
        if levels == 2:
            co = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.coarse_split, w.coarse_overlap, w.coarse_rtol,
                            w.coarse_maxit, 32)
        last = {}

        def refactor():
            if co is not None:
                co.refactor_with(ras)
            else:
                ras.refactor()

        def solve():
            x.zero_()
            _, st, its, rel = api.gmres_solve(prob, b, x, ras=ras, coarse=co, restart=w.restart, rtol=w.rtol,
                                              maxit=3000)
            last.update(status=st, iterations=its, relres=rel)

        refactor()
        solve()
        with ClockSampler(torch.cuda.current_device()) as clk:
            out = {"levels": levels, "overlap": delta, "refactor_ms": timed(refactor, 1),
                   "solve_ms": timed(solve, args.reps)}
        out.update(last)
        out["clocks"] = clk.summary()
        out["box_points"] = ras.info()["points"]
        print(json.dumps(out), flush=True)
        if co is not None:
            co.close()
        ras.close()


def large_arm(args):
    """The 64^3 x 128 single solve (106M unknowns): FP32 subdomain and coarse solves, FP64 FGMRES(40).

    One step = right-hand side, refactorisation of the fine and coarse factors, the FGMRES solve
    to a true relative residual of 1e-8 and the source extraction, as in the default benchmark.
    """
    import numpy as np
    import torch

    from paper_1508_06103_gb300 import api, build
    from paper_1508_06103_gb300 import workloads as W

    build.build()
    w = W.large()
    if args.coarse_levels:
        w = dataclasses.replace(w, coarse_M=args.coarse_levels)
    cobs = torch.from_numpy(np.loadtxt(OBS_FILE_LARGE, ndmin=2)).cuda()
    prob = api.Problem.from_workload(w)
    b, x = prob.zeros(), prob.zeros()
    f = torch.empty(prob.levels * prob.N, dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_setup = time.time()
    ras = api.RAS(prob, w.nsub, w.overlap, 32)
    co = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.coarse_split, w.coarse_overlap, w.coarse_rtol,
                    w.coarse_maxit, 32)
    setup_s = time.time() - t_setup
    last = {}

    def step():
        prob.rhs(cobs, out=b)
        co.refactor_with(ras)
        x.zero_()
        _, st, its, rel = api.gmres_solve(prob, b, x, ras=ras, coarse=co, restart=w.restart, rtol=w.rtol,
                                          maxit=args.maxit)
        prob.recover_source(x, out=f)
        last.update(status=st, iterations=its, relres=rel)

    for _ in range(args.warmup):
        step()
    api.timing_reset(prob, ras)
    api.timing_enable(True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms = timed(step, args.steps)
    api.timing_enable(False)
    ras_ms, ras_n = ras.timing(0)
    fac_ms, fac_n = ras.timing(1)
    mv_ms, mv_n = api.matvec_timing(prob)
    free, total = torch.cuda.mem_get_info()
    info = ras.info()
    peak, peak_kind = measured_peaks()
    solve_bytes = info["points"] * SLOTS_PER_POINT * info["value_bytes"] + info["points"] * 24 + prob.n * 8
    avg_solve = ras_ms / max(ras_n, 1)
    out = {
        "metric": "KKT solve s to 1e-8 rel. residual at 64^3x128 (FP32 subdomain solves, FGMRES(40))",
        "value": ms / 1e3, "unit": "s", "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
        "maxit": args.maxit, "ms_per_iteration": ms / max(1, last.get("iterations") or 1),
        "workload": f"{w.name}: {prob.n:,} unknowns, 8^4 subdomains overlap 2, coarse {w.coarse_cells[0]}^3 x "
                    f"{w.coarse_M} (4^4, overlap 1)",
        "status": last.get("status"), "iterations": last.get("iterations"), "true_relres": last.get("relres"),
        "setup_s": setup_s, "box_points": info["points"], "factor_gb": info["factor_values"] * info["value_bytes"] / 1e9,
        "device_memory_used_gb": (total - free) / 1e9, "device_memory_total_gb": total / 1e9,
        "kernels": {
            "ilu0_factor": {"avg_launch_ms": fac_ms / max(fac_n, 1), "launches_per_step": fac_n / args.steps},
            "ras_solve": {"avg_launch_ms": avg_solve, "launches_per_step": ras_n / args.steps,
                          "alg_bytes_per_launch": solve_bytes, "achieved_gbs": solve_bytes / avg_solve / 1e6,
                          "frac": solve_bytes / avg_solve / 1e6 / peak, "peak": peak, "peak_source": peak_kind},
            "matvec_fp64": {"avg_launch_ms": mv_ms / max(mv_n, 1), "launches_per_step": mv_n / args.steps},
        },
        "clocks": clk.summary(),
    }
    print(json.dumps(out), flush=True)


def batch_arm(args):
    """Eight independent inverse problems solved together (the batching form).

    Set-up: the subdomain solve's shape is chosen by the library's autotuner on these problems
    (cached in the temporary directory).  One step = the eight right-hand sides from their
    observations, one factorisation launch for all 512 subdomains, the batched FGMRES(30) (all
    problems in lockstep, one captured graph per restart cycle, each to its own 1e-8 true
    residual) and the eight recovered sources.
    """
    import tempfile

    import numpy as np
    import torch

    from paper_1508_06103_gb300 import api, build
    from paper_1508_06103_gb300 import workloads as W

    build.build()
    ws = W.batch()
    probs = [api.Problem.from_workload(w) for w in ws]
    obs = [torch.from_numpy(np.loadtxt(os.path.join(ROOT, "tests", "golden", f"observations_{w.name}.txt"),
                                       ndmin=2)).cuda() for w in ws]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cache = os.path.join(tempfile.gettempdir(), "stkkt_autotune.txt")
    t0 = time.time()
    shape, tuned_ms = api.autotune(probs, ws[0].nsub, ws[0].overlap, 32, reps=3, cache_path=cache)
    tune_s = time.time() - t0
    bras = api.BatchRAS(probs, ws[0].nsub, ws[0].overlap, 32, shape=shape)
    off = bras.offsets
    b = torch.zeros(bras.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    last = {}

    def step():
        for k, p in enumerate(probs):
            p.rhs(obs[k], out=b[off[k]:off[k + 1]])
        bras.refactor()
        _, st, sts, its, rel = api.gmres_solve_batch(probs, bras, b, x, restart=ws[0].restart, rtol=ws[0].rtol,
                                                     maxit=3000)
        for k, p in enumerate(probs):
            p.recover_source(x[off[k]:off[k + 1]])
        last.update(status=st, statuses=sts, iterations=its, relres=rel)

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for _ in range(args.warmup):
        step()
    launches0 = api.launch_count()
    api.timing_reset(probs[0], bras)
    api.timing_enable(True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms = timed(step, args.steps)
    api.timing_enable(False)
    launches = (api.launch_count() - launches0) // args.steps
    ras_ms, ras_n = bras.timing(0)
    fac_ms, fac_n = bras.timing(1)
    info = bras.info()
    peak, peak_kind = measured_peaks()
    solve_bytes = info["points"] * SLOTS_PER_POINT * info["value_bytes"] + info["points"] * 24 + bras.n * 8
    avg = ras_ms / max(ras_n, 1)
    out = {
        "metric": "independent KKT solves to 1e-8 per second, 8 problems together (FP32 subdomain solves)",
        "value": len(probs) * 1e3 / ms, "unit": "problems/s", "ms_per_step": ms, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True,
        "workload": "; ".join(f"{w.name} ({w.unknowns:,})" for w in ws),
        "unknowns": bras.n, "subdomains": info["nbox"], "box_points": info["points"],
        "shape": {"chunk_points": shape[0], "stages": shape[1], "autotune_s": tune_s, "tuned_ms": tuned_ms},
        "status": last.get("status"), "statuses": last.get("statuses"), "iterations": last.get("iterations"),
        "true_relres": last.get("relres"), "gpu_launches": int(launches),
        "kernels": {
            "ras_solve": {"avg_launch_ms": avg, "launches_per_step": ras_n / args.steps,
                          "alg_bytes_per_launch": solve_bytes, "achieved_gbs": solve_bytes / avg / 1e6,
                          "frac": solve_bytes / avg / 1e6 / peak, "peak": peak, "peak_source": peak_kind},
            "ilu0_factor": {"avg_launch_ms": fac_ms / max(fac_n, 1), "launches_per_step": fac_n / args.steps},
        },
        "clocks": clk.summary(),
    }
    print(json.dumps(out), flush=True)


def examples_arm(args):
    """The paper's Examples 1-3 (Sec. 4.1) at the paper's sizes: one-level space-time RAS with
    4 x 4 x 4 x 4 subdomains (the paper's np = 256), overlap 1, ILU(0) local solves in FP32 inside
    FP64 GMRES(30) (the paper's one-level runs use GMRES(50) to 1e-6; here 1e-8), and the
    two-level form where the steps allow a nested coarse level.  The right-hand sides come from
    seeded standard normal sensor values (the observation data only enter b; the operator and the
    preconditioner are the example's), so no forward solve is needed.  One JSON line per case:
    iterations, solve time (CUDA events) and the set-up time of the factors.
    """
    import numpy as np
    import torch

    from paper_1508_06103_gb300 import api, build
    from paper_1508_06103_gb300 import workloads as W

    build.build()
    cases = [("example1", W.example1()), ("example2-h1h1", W.example2("h1h1")), ("example2-h1l2", W.example2("h1l2")),
             ("example3-s21", W.example3(21)), ("example3-s9", W.example3(9))]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, w in cases:
        prob = api.Problem.from_workload(w)
        rng = np.random.Generator(np.random.PCG64(17))
        cobs = torch.from_numpy(rng.standard_normal((w.M + 1, len(w.sensor_xyz)))).cuda()
        b = prob.rhs(cobs)
        ras = api.RAS(prob, w.nsub, w.overlap, 32)
        for levels in (1, 2):
            co = None
            if levels == 2:
                # coarse level: half the cells; half the steps when the step count is even, a third
                # when it divides by 3, else all of them (47 is prime)
                cM = w.M // 2 if w.M % 2 == 0 else (w.M // 3 if w.M % 3 == 0 else w.M)
                co = api.Coarse(prob, tuple(c // 2 for c in w.cells), cM, w.nsub, 1, 0.1, 4, 32)
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            e0.record()
            _, st, its, rel = api.gmres_solve(prob, b, x, ras=ras, coarse=co, restart=30, rtol=1e-8, maxit=3000,
                                              flexible=True)
            e1.record()
            torch.cuda.synchronize()
            print(json.dumps({"case": name, "levels": levels, "cells": list(w.cells), "steps": w.M,
                              "unknowns": prob.n, "sensors": len(w.sensor_xyz), "status": st, "iterations": its,
                              "true_relres": rel, "solve_ms": e0.elapsed_time(e1)}), flush=True)
            if co is not None:
                co.close()
        ras.close()
        prob.close()


def table1_arm(args):
    """The paper's Table 1 experiment on this workload family: the two-level method with the
    fine subdomains factored by ILU(0), ILU(1) or the 3x3 point-block ILU(0) (coarse level:
    ILU(0)), FP32 factors inside FP64 FGMRES(30) to 1e-8.  One JSON line per local solver:
    iterations, refactorisation and solve times (CUDA events), factor values per point.
    """
    import numpy as np
    import torch

    from paper_1508_06103_gb300 import api, build
    from paper_1508_06103_gb300 import workloads as W

    build.build()
    c, M = args.cells, args.levels
    w = W.mid(cells=(c, c, c), M=M, coarse_cells=(c // 2,) * 3, coarse_M=M // 2)
    prob = api.Problem.from_workload(w)
    rng = np.random.Generator(np.random.PCG64(17))
    cobs = torch.from_numpy(rng.standard_normal((w.M + 1, len(w.sensor_xyz)))).cuda()
    b = prob.rhs(cobs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    for local in args.locals.split(","):
        ras = api.RAS(prob, w.nsub, w.overlap, args.prec, local=local)
        co = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.coarse_split, w.coarse_overlap, w.coarse_rtol,
                        w.coarse_maxit, args.prec)
        fac_ms, _ = timed(lambda: ras.refactor())
        x = torch.zeros_like(b)
        api.gmres_solve(prob, b, x, ras=ras, coarse=co, restart=30, rtol=1e-8, maxit=3000)   # warm-up
        x.zero_()
        sol_ms, res = timed(lambda: api.gmres_solve(prob, b, x, ras=ras, coarse=co, restart=30, rtol=1e-8,
                                                    maxit=3000))
        _, st, its, rel = res
        info = ras.info()
        print(json.dumps({"table": 1, "workload": w.name, "local": local, "factor_prec": args.prec,
                          "iterations": its, "status": st, "true_relres": rel, "refactor_fine_ms": fac_ms,
                          "solve_ms": sol_ms, "factor_values": info.get("factor_values"),
                          "box_points": info.get("points")}), flush=True)
        ras.close()
        co.close()


def reduced_arm(args):
    """The reduced-space ("traditional") method of Sec. 1 on the same GPU and workload as the
    all-at-once benchmark (32^3 x 64 by default): f is the only unknown, each application of the
    reduced operator is a forward and a backward march of 64 spatial solves.  Solved to the same
    true KKT relative residual (1e-8) as the all-at-once form; one JSON line with its time beside
    the all-at-once FP64 and mixed forms' times on the same data.
    """
    import numpy as np
    import torch

    from paper_1508_06103_gb300 import api, build
    from paper_1508_06103_gb300 import workloads as W

    build.build()
    c = args.cells
    w = W.mid() if c == 32 else W.mid(cells=(c, c, c), M=args.levels, coarse_cells=(c // 2,) * 3,
                                      coarse_M=args.levels // 2)
    prob = api.Problem.from_workload(w)
    if w.M == 64 and c == 32:
        cobs = torch.from_numpy(np.loadtxt(obs_file(args), ndmin=2)).cuda()
    else:
        rng = np.random.Generator(np.random.PCG64(17))
        cobs = torch.from_numpy(rng.standard_normal((w.M + 1, len(w.sensor_xyz)))).cuda()
    b = prob.rhs(cobs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": w.name, "unknowns": prob.n, "method": "reduced space (Sec. 1), FP64"}
    # reduced system to 1e-9 relative residual, steps to 1e-12: the KKT residual then meets 1e-8
    torch.cuda.synchronize()
    e0.record()
    U, st, its, rel, stats = api.reduced_solve(prob, cobs, restart=30, rtol=args.reduced_rtol, maxit=2000,
                                               step_rtol=1e-12)
    e1.record()
    torch.cuda.synchronize()
    r = prob.residual(b, U)
    out.update({"s_per_solve": e0.elapsed_time(e1) / 1e3, "status": st, "outer_iterations": its,
                "reduced_relres": rel, "true_kkt_relres": float(r.norm() / b.norm()), **stats,
                "step_iterations_mean": stats["step_iterations"] / max(1, stats["step_solves"])})
    # the all-at-once forms on the same data
    for prec in (64, 32):
        ras = api.RAS(prob, w.nsub, w.overlap, prec)
        co = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.coarse_split, w.coarse_overlap, w.coarse_rtol,
                        w.coarse_maxit, prec)
        x = torch.zeros_like(b)
        api.gmres_solve(prob, b, x, ras=ras, coarse=co, restart=w.restart, rtol=w.rtol, maxit=3000)
        x.zero_()
        torch.cuda.synchronize()
        e0.record()
        co.refactor_with(ras)
        _, st2, its2, rel2 = api.gmres_solve(prob, b, x, ras=ras, coarse=co, restart=w.restart, rtol=w.rtol,
                                             maxit=3000)
        e1.record()
        torch.cuda.synchronize()
        f_a = prob.recover_source(x)
        f_r = prob.recover_source(U)
        out[f"all_at_once_fp{prec}"] = {"s_per_solve": e0.elapsed_time(e1) / 1e3, "iterations": its2,
                                       "true_relres": rel2,
                                       "f_rel_diff_vs_reduced": float((f_a - f_r).norm() / f_r.norm())}
        ras.close()
        co.close()
    out["speedup_mixed_vs_reduced"] = out["s_per_solve"] / out["all_at_once_fp32"]["s_per_solve"]
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", choices=["ras", "matvec", "sweep", "peaks", "table1"], default=None,
                    help="time one kernel on a member of the workload family instead of the full solve; "
                         "sweep: overlap and one/two-level sweep of the mixed-form solve")
    ap.add_argument("--cells", type=int, default=32)
    ap.add_argument("--levels", type=int, default=64)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--prec", type=int, default=32)
    ap.add_argument("--chunk", type=int, default=0, help="--kernel ras: points per chunk (0: the library's choice)")
    ap.add_argument("--stages", type=int, default=0, help="--kernel ras: copy-ring buffers (0: the library's choice)")
    ap.add_argument("--place", type=int, default=0,
                    help="--kernel ras: local vectors 1 in shared, 2 in global memory (0: the library's choice)")
    ap.add_argument("--overlap", type=int, default=2, help="--kernel ras/matvec: subdomain overlap")
    ap.add_argument("--data", choices=["same-mesh", "refined2"], default="same-mesh",
                    help="observations: same-mesh forward solve (default) or one on a 2x finer mesh")
    ap.add_argument("--maxit", type=int, default=400,
                    help="--workload large: FGMRES iteration limit of a step (the solve converges slowly)")
    ap.add_argument("--coarse-levels", type=int, default=0,
                    help="--workload large: time steps of the coarse level (0: the workload's)")
    ap.add_argument("--locals", default="ilu0,ilu1,bilu0",
                    help="--kernel table1: fine local solvers (ilu0, ilu1, bilu0)")
    ap.add_argument("--reduced-rtol", type=float, default=1e-9,
                    help="--workload reduced: relative residual of the reduced system")
    ap.add_argument("--workload", choices=["mid", "large", "batch", "examples", "reduced"], default="mid",
                    help="large: time the 64^3 x 128 single solve; batch: eight independent problems solved "
                         "together; instead of the default benchmark")
    args = ap.parse_args()
    if args.workload == "large":
        large_arm(args)
    elif args.workload == "batch":
        batch_arm(args)
    elif args.workload == "examples":
        examples_arm(args)
    elif args.workload == "reduced":
        reduced_arm(args)
    elif args.kernel == "sweep":
        sweep_arm(args)
    elif args.kernel == "table1":
        table1_arm(args)
    elif args.kernel:
        kernel_arm(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
