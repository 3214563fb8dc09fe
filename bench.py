"""Benchmark: time to a 1e-8 relative residual of the algebraic-DD
preconditioned FGMRES solve on the 256x256 MAC Oseen system (196,096
unknowns, nu = 1e-3, seeded 8-mode Fourier wind, 64 subdomains, MSCE
aggregates of nominal size 2048, FGMRES(50)).

One step = dd_setup (interior LU, Schur blocks, their inverses) + gmres_solve
to 1e-8, through the library's C ABI.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|fp64]
  python bench.py --impl reference ...   # the CPU oracle on the host cores
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 residual & GMRES iters (learned/FP32 vs FP64 plain); apply GB/s"
WORKLOAD = "oseen_mac_256x256_uniform_nu1e-3_fourier8_m64_msce_sz2048_fgmres50_tol1e-8"
TOL, RESTART, MAXIT, SZ = 1e-8, 50, 3000, 2048
# dram__bytes_read.sum + dram__bytes_write.sum of one band_solve_fwd_kernel
# launch on this workload (ncu capture summarised in profiles/); None once the
# kernel has changed since the capture
TRAFFIC = {"fp32": 216824320, "fp64": None}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def make_inputs():
    from paper_1104_3349_gb300 import workload as W
    w = W.fourier256()
    agg = W.aggregates(w.A, w.part, w.perm, SZ)
    return w, agg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                mx = float(f[2].split()[0])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws, device=None):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def apply_bytes(st, elem):
    """Algorithmic bytes of one dd_apply: both interior sweeps read L and U
    (in-band entries), the S_hat^-1 blocks, the couplings E and F
    (12 B per entry), y and x, the interior and interface vectors."""
    n, nI, nG = st["n"], st["n_interior"], st["n_interface"]
    return (2 * (elem * st["factor_nonzeros"] + 4 * nI) + st["schur_bytes"] + 12 * st["coupling_nnz"]
            + 8 * 2 * n + elem * (4 * nI + 4 * nG))


def sweep_bytes(st, elem):
    """Algorithmic bytes of one interior solve (band_solve_fwd_kernel): the
    in-band entries of L and U once, y gathered through perm, z1 written."""
    nI = st["n_interior"]
    return elem * st["factor_nonzeros"] + (8 + 4 + elem) * nI


def run_ours(args):
    import torch
    from paper_1104_3349_gb300 import dd

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    dd.build()
    dd.load()
    w, agg = make_inputs()
    prec = {"fp32": dd.DD_FP32, "fp32_tf32": dd.DD_FP32_TF32}.get(args.prec, dd.DD_FP64)
    b_host = torch.from_numpy(w.b).pin_memory()
    b = b_host.to(dev)
    x = torch.empty_like(b)
    stream = torch.cuda.current_stream()

    def step(precision):
        P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=precision)
        r = P.gmres(b, x, tol=TOL, restart=RESTART, maxit=MAXIT)
        return P, r

    for _ in range(args.warmup):
        P, r = step(prec)
        P.close()
    torch.cuda.synchronize()
    barrier(ws)
    iters, statuses, relres = [], [], []
    launches = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            P, r = step(prec)
            iters.append(r["iters"]); statuses.append(r["status"]); relres.append(r["relres"])
            launches += P.stats()["launches"]
            P.close()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    total_ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
    ms_per_step = total_ms / args.steps
    value = ms_per_step / ws  # whole-job: ms per solved system over all ranks

    # end to end through the public API with host buffers
    x_host = torch.empty_like(b_host).pin_memory()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 3))
    f0.record(stream)
    for _ in range(e2e_steps):
        bd = b_host.to(dev, non_blocking=True)
        P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=prec)
        r2 = P.gmres(bd, x, tol=TOL, restart=RESTART, maxit=MAXIT)
        x_host.copy_(x, non_blocking=True)
        P.close()
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1), ws, dev) / e2e_steps / ws

    # the dominant kernels: dd_apply (two interior sweeps + interface solve)
    P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=prec)
    st = P.stats()
    y = torch.from_numpy(w.b).to(dev)
    xa = torch.empty_like(y)
    for _ in range(5):
        P.apply(y, xa)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 50
    g0.record(stream)
    for _ in range(reps):
        P.apply(y, xa)
    g1.record(stream)
    torch.cuda.synchronize()
    apply_ms = g0.elapsed_time(g1) / reps
    elem = 4 if prec == dd.DD_FP32 else 8
    abytes = apply_bytes(st, elem)
    # the dominant kernel alone: the interior solve z1 = D^-1 y1 (part 0)
    g0.record(stream)
    for _ in range(reps):
        P.apply_part(0, y, xa)
    g1.record(stream)
    torch.cuda.synchronize()
    sweep_ms = g0.elapsed_time(g1) / reps
    sbytes = sweep_bytes(st, elem)
    # the SpMV w = C z alone, L2 flushed before every launch (in the solve the
    # apply streams the factors through L2 between two SpMVs)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    spmv_t = []
    for rep in range(23):
        flush.fill_(float(rep))
        g0.record(stream)
        P.spmv(y, xa)
        g1.record(stream)
        torch.cuda.synchronize()
        if rep >= 3:
            spmv_t.append(g0.elapsed_time(g1))
    del flush
    spmv_ms = statistics.median(spmv_t)
    P.close()
    # the CGS2 kernel inside one solve: events around every launch (a solve of
    # its own, outside the timed steps), against the measured FP64 FMA rate
    Pk = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=prec, time_kernels=True)
    Pk.gmres(b, x, tol=TOL, restart=RESTART, maxit=MAXIT)
    kst = Pk.stats()
    Pk.close()
    fp64_gfma = dd.fp64_peak()
    spmv_bytes = 12 * int(w.A.nnz) + 4 * (int(w.A.n) + 1) + 16 * int(w.A.n)

    # the plain FP64 method on the same input, for comparison
    fp64 = None
    if prec != dd.DD_FP64 and not args.skip_fp64:
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        P, r64 = step(dd.DD_FP64)
        h1.record(stream)
        torch.cuda.synchronize()
        fp64 = {"ms": h0.elapsed_time(h1), "iters": r64["iters"], "setup_ms": r64["setup_ms"],
                "solve_ms": r64["solve_ms"], "status": r64["status"]}
        P.close()

    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    achieved = abytes / (apply_ms * 1e-3) / 1e9
    s_ach = sbytes / (sweep_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": round(s_ach, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(s_ach / hbm, 4), "traffic": TRAFFIC.get(args.prec),
            "kernel": "band_solve_fwd_kernel (interior forward+backward sweeps, all subdomains)",
            "algorithmic_bytes": int(sbytes), "launch_ms": round(sweep_ms, 4),
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}

    # the optional legs never cost the headline line: a failure is recorded in its place
    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        try:
            cpu = cpu_baseline(w, agg)
        except Exception as e:  # noqa: BLE001
            cpu = {"error": f"{type(e).__name__}: {e}"[:300]}
    variants = None
    if rank == 0 and ws == 1 and not args.skip_variants:
        try:
            variants = run_variants(args, dev)
        except Exception as e:  # noqa: BLE001
            variants = {"error": f"{type(e).__name__}: {e}"[:300]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "ms", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == dd.DD_FP32 else "f64",
            "data": "synthetic", "impl": "ours",
            "config": {"workload": WORKLOAD, "n": int(w.A.n), "nnz": int(w.A.nnz), "subdomains": w.m,
                       "interface": int(st["n_interface"]), "aggregates": int(st["n_agg"]),
                       "preconditioner": f"{args.prec} factors, FP64 FGMRES(50)",
                       "l2": "inputs larger than L2 (factors %.0f MB)" % (2 * st["factor_bytes"] / 1e6),
                       "parallelism": f"replicas x{ws}"},
            "gmres_iters": iters[0] if iters else None, "gmres_iters_all": iters,
            "relres_true": max(relres) if relres else None, "status": statuses,
            "apply_ms": round(apply_ms, 4), "apply_gbs": round(achieved, 1),
            "fp64_plain": fp64,
            "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": int(8 * w.A.n),
                    "d2h_bytes_per_step": int(8 * w.A.n),
                    "note": "C, partition and aggregates enter dd_setup as host arrays in both numbers"},
            "roofline": roof, "clocks": clk.summary(), "gpu_launches": int(launches),
            "kernels": {
                "spmv": {"ms": round(spmv_ms, 5), "algorithmic_bytes": spmv_bytes,
                         "gbs": round(spmv_bytes / (spmv_ms * 1e-3) / 1e9, 1),
                         "frac_hbm": round(spmv_bytes / (spmv_ms * 1e-3) / 1e9 / hbm, 4),
                         "ms_in_solve_mean": round(kst["spmv_ms"] / max(kst["krylov_steps"], 1), 5),
                         "note": "L2 flushed before each of 20 timed launches; median"},
                "cgs2": {"ms_mean": round(kst["cgs2_ms"] / max(kst["krylov_steps"], 1), 5),
                         "steps": int(kst["krylov_steps"]),
                         "fp64_gfma": round(kst["cgs2_fma"] / (kst["cgs2_ms"] * 1e-3) / 1e9, 1)
                         if kst["cgs2_ms"] > 0 else None,
                         "fp64_peak_gfma": round(fp64_gfma, 1),
                         "frac_fp64": round(kst["cgs2_fma"] / (kst["cgs2_ms"] * 1e-3) / 1e9 / fp64_gfma, 4)
                         if kst["cgs2_ms"] > 0 else None,
                         "note": "every Arnoldi step of one solve timed with events; useful FMAs "
                                 "(4(j+1)+2) n per step; peak from dd_fp64_peak"}},
            "cpu_baseline": cpu, "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_variants(args, dev):
    """Configs 3 and 4 on the same GPU: the stretched 512x512 grid with 256
    uneven subdomains (persistent task lists, graph-captured FGMRES
    iterations, autotuned sweeps) and the 64-system batch (one handle, lock-step
    FGMRES(30)) against solving its systems one after another."""
    import torch
    from paper_1104_3349_gb300 import dd, workload as W

    def ev():
        return torch.cuda.Event(enable_timing=True)

    out = {}
    # config 3
    w = W.stretched512()
    agg = W.aggregates(w.A, w.part, w.perm, SZ)
    b = torch.from_numpy(w.b).to(dev)
    x = torch.zeros_like(b)
    res = {}
    for g in (False, True):
        for rep in range(2):  # the first run warms up
            e0, e1 = ev(), ev()
            e0.record()
            P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=dd.DD_FP32,
                      use_graph=g, autotune=True)
            r = P.gmres(b, x, tol=TOL, restart=RESTART, maxit=args.c3_maxit)
            e1.record()
            torch.cuda.synchronize()
            st = P.stats()
            P.close()
        res[g] = dict(total_ms=round(e0.elapsed_time(e1), 1), setup_ms=round(r["setup_ms"], 1),
                      solve_ms=round(r["solve_ms"], 1), iters=r["iters"], relres=r["relres"],
                      status=r["status"], ms_per_iter=round(r["solve_ms"] / max(r["iters"], 1), 4),
                      launches=int(st["launches"]), graphs=int(st["graphs"]))
    out["stretched512"] = {
        "workload": "oseen_mac_512x512_stretch1.02_nu1e-3_fourier8_m256_msce_sz2048_fgmres50",
        "n": int(w.A.n), "subdomains": w.m, "interface": int(st["n_interface"]),
        "subdomain_sizes": [int(v) for v in (lambda c: (c.min(), c.max()))(np.bincount(w.part[w.part >= 0]))],
        "sweep_grid": int(st["sweep_grid"]), "sweep_slots": int(st["sweep_slots"]),
        "stage_bytes": int(st["stage_bytes"]), "autotune_candidates": int(st["tuned"]),
        "maxit": args.c3_maxit, "graph": res[True], "plain": res[False],
        "note": "MSCE_INF with consecutive aggregates stalls on this stretched grid (the oracle does too); "
                "the line reports the time per FGMRES iteration at a capped iteration count"}
    # config 4
    ws = W.batch64(sz=SZ)
    systems = [(q.A, q.part, q.m, q.perm, q.agg) for q in ws]
    bs = [torch.from_numpy(q.b).to(dev) for q in ws]
    for rep in range(2):
        xs = [torch.zeros_like(v) for v in bs]
        e0, e1 = ev(), ev()
        e0.record()
        P = dd.DDBatch(systems, "msce_inf", prec=dd.DD_FP32, max_restart=30, use_graph=True, autotune=True)
        rc, res4 = P.gmres(bs, xs, tol=TOL, restart=30, maxit=MAXIT)
        e1.record()
        torch.cuda.synchronize()
        st = P.stats()
        P.close()
    its = [q["iters"] for q in res4]
    batched_ms = e0.elapsed_time(e1)
    # the same systems one handle at a time
    e0, e1 = ev(), ev()
    e0.record()
    seq_its = []
    for q, v in zip(ws, bs):
        xq = torch.zeros_like(v)
        P = dd.DD(q.A, q.part, q.m, "msce_inf", perm=q.perm, agg_offsets=q.agg, prec=dd.DD_FP32, max_restart=30)
        r = P.gmres(v, xq, tol=TOL, restart=30, maxit=MAXIT)
        seq_its.append(r["iters"])
        P.close()
    e1.record()
    torch.cuda.synchronize()
    out["batch64"] = {
        "workload": "64 MAC Oseen systems, sides {64..256}, nu log-uniform [1e-3,1e-2], 16-64 subdomains each, "
                    "msce sz2048, FP32 preconditioner in FP64 FGMRES(30)",
        "n_total": int(sum(q.A.n for q in ws)), "subdomains": int(st["m"]), "status": rc,
        "all_converged": all(q["status"] == 0 for q in res4), "relres_max": max(q["relres"] for q in res4),
        "batched_ms": round(batched_ms, 1), "setup_ms": round(res4[0]["setup_ms"], 1),
        "solve_ms": round(res4[0]["solve_ms"], 1), "iters_max": max(its), "iters_sum": sum(its),
        "iters_match_one_by_one": sum(abs(a - c) <= 1 for a, c in zip(its, seq_its)),
        "one_by_one_ms": round(e0.elapsed_time(e1), 1), "sweep_grid": int(st["sweep_grid"]),
        "stage_bytes": int(st["stage_bytes"]), "autotune_candidates": int(st["tuned"]),
        "graphs": int(st["graphs"]), "launches": int(st["launches"])}
    for name, fn in (("learned", run_learned), ("ilu", run_ilu), ("fp32_tf32", run_tf32)):
        try:  # one variant's failure leaves the others' numbers
            out[name] = fn(args, dev)
        except Exception as e:  # noqa: BLE001
            out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
    return out


def run_ilu(args, dev):
    """The headline workload with inexact interior solves (Section 5's
    incomplete LU, drop tolerance tolA) against the exact factorisation."""
    import torch
    from paper_1104_3349_gb300 import dd, workload as W
    w = W.fourier256()
    agg = W.aggregates(w.A, w.part, w.perm, SZ)
    b = torch.from_numpy(w.b).to(dev)
    res = {}
    for tol in (0.0, 1e-4, 1e-3):
        r, st, ms = None, None, []
        for rep in range(2):  # the first run of each tolerance is a warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=dd.DD_FP32, ilu_tol=tol)
            x = torch.empty_like(b)
            r = P.gmres(b, x, tol=TOL, restart=RESTART, maxit=MAXIT)
            e1.record()
            torch.cuda.synchronize()
            st = P.stats()
            P.close()
            ms.append(e0.elapsed_time(e1))
        res[f"tol_{tol:g}"] = {"ms": round(ms[-1], 2), "iters": r["iters"], "status": r["status"],
                               "relres": r["relres"], "factor_bytes": int(st["factor_bytes"])}
    return {"workload": WORKLOAD, "preconditioner": "fp32 factors, FP64 FGMRES(50)",
            "note": "the packed sweep tiles are dense between their trimmed bounds, so dropped entries inside "
                    "them still stream", **res}


def run_tf32(args, dev):
    """The headline workload with DD_FP32_TF32 (the dense block inverses'
    rank-64 updates on the TF32 tensor cores, three TF32 terms per product)
    against DD_FP32: setup + solve, the second run of each."""
    import torch
    from paper_1104_3349_gb300 import dd, workload as W
    w = W.fourier256()
    agg = W.aggregates(w.A, w.part, w.perm, SZ)
    b = torch.from_numpy(w.b).to(dev)
    res = {}
    for name, prec in (("fp32", dd.DD_FP32), ("fp32_tf32", dd.DD_FP32_TF32)):
        for rep in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=prec)
            x = torch.empty_like(b)
            r = P.gmres(b, x, tol=TOL, restart=RESTART, maxit=MAXIT)
            e1.record()
            torch.cuda.synchronize()
            st = P.stats()
            P.close()
        res[name] = {"ms": round(e0.elapsed_time(e1), 2), "setup_ms": round(st["setup_ms"], 2),
                     "iters": r["iters"], "status": r["status"], "relres": r["relres"]}
    return {"workload": WORKLOAD, **res}


WEIGHTS = os.path.join(ROOT, "paper_1104_3349_gb300", "weights", "schur_mlp.bin")


def run_learned(args, dev):
    """The learned correction (DD_LEARNED) against the method without it (LUM)
    and the MSCE_INF blocks it is trained on.  Two workloads: held-out 64x64
    problems like the training set's (seeds outside it), and the 1024x1024
    stretched grid (aspect 100, 1024 subdomains) at an iteration cap."""
    import torch
    from paper_1104_3349_gb300 import dd, workload as W

    def solve(A, part, m, perm, agg, b, kind, prec, maxit):
        try:
            P = dd.DD(A, part, m, kind, perm=perm, agg_offsets=agg, prec=prec,
                      mlp_weights=WEIGHTS if kind == "learned" else None)
        except dd.DDError as e:
            return {"setup_error": str(e)[:120]}
        bd = torch.from_numpy(b).to(dev)
        x = torch.zeros_like(bd)
        r = P.gmres(bd, x, tol=TOL, restart=RESTART, maxit=maxit)
        st = P.stats()
        P.close()
        return {"iters": r["iters"], "status": r["status"], "relres": r["relres"], "setup_ms": round(r["setup_ms"], 2),
                "solve_ms": round(r["solve_ms"], 2), "fallback": int(st["learned_fallback"])}

    kinds = ("lum", "learned", "msce_inf")
    small = {k: [] for k in kinds}
    for seed in range(9000, 9008):
        h = W.learned64(seed)
        for k in kinds:
            small[k].append(solve(h.A, h.part, h.m, h.perm, h.agg, h.b, k, dd.DD_FP32, MAXIT))
    summ = {k: {"iters": [r.get("iters") for r in v], "setup_ms_mean": round(float(np.mean([r["setup_ms"] for r in v])), 2),
                "all_converged": all(r.get("status") == 0 for r in v)} for k, v in small.items()}
    out = {"heldout64": {"workload": "8 held-out 64x64 MAC Oseen problems (nu log-uniform [1e-3,1e-2], stretch [1,1.03], "
                                     "seeds 9000-9007), 4 subdomains, aggregates sz 64, FP32 preconditioner, FGMRES(50)",
                         **summ}}
    if not args.skip_cfg5:
        # aggregates of nominal size 4096: on this grid (aspect 100, 1024
        # subdomains) MSCE_INF's FP32 blocks fail the pivot test up to sz 2048,
        # and after 300 FGMRES(50) steps FP64 reaches 0.31 / 0.21 / 0.12 at
        # sz 1024 / 2048 / 4096, so the largest size is the one compared
        w = W.stretched1024()
        agg = W.aggregates(w.A, w.part, w.perm, 4096)
        big = {}
        for prec, name in ((dd.DD_FP64, "fp64"), (dd.DD_FP32, "fp32")):
            for k in kinds:
                big[f"{k}_{name}"] = solve(w.A, w.part, w.m, w.perm, agg, w.b, k, prec, args.c5_maxit)
        out["stretched1024"] = {"workload": "oseen_mac_1024x1024_aspect100_nu1e-3_fourier8_m1024_sz4096_fgmres50",
                                "n": int(w.A.n), "maxit": args.c5_maxit, **big}
    return out


def cpu_baseline(w, agg):
    """The FP64 oracle on the host cores: full setup + FGMRES(50) to 1e-8."""
    import oracle as O
    t0 = time.perf_counter()
    R = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=agg)
    t1 = time.perf_counter()
    r = R.fgmres(w.b, tol=TOL, restart=RESTART, maxit=MAXIT)
    t2 = time.perf_counter()
    R.close()
    return {"value": round(1e3 * (t2 - t0), 1), "unit": "ms", "cores": O.num_threads(), "kind": "oracle",
            "sample": "the full workload: one oracle setup + FGMRES(50) solve to 1e-8",
            "setup_ms": round(1e3 * (t1 - t0), 1), "solve_ms": round(1e3 * (t2 - t1), 1),
            "iters": r["iters"], "status": r["status"]}


def run_reference(args):
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    w, agg = make_inputs()
    for _ in range(min(args.warmup, 1)):
        cpu_baseline(w, agg)
    vals, its = [], []
    for _ in range(args.steps):
        c = cpu_baseline(w, agg)
        vals.append(c["value"]); its.append(c["iters"])
    import oracle as O
    v = sum(vals) / len(vals)
    line = {"metric": METRIC, "value": round(v, 1), "unit": "ms", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "n": int(w.A.n), "subdomains": w.m},
            "gmres_iters": its[0],
            "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": O.num_threads(), "kind": "oracle",
                             "sample": "full oracle setup + FGMRES(50) solve per step; warm-up capped at 1"},
            "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def apply_only(args):
    """One dd_setup on the bench workload, then args.apply_only dd_apply calls
    (the command the kernel profiles in profiles/ are captured with)."""
    import torch
    from paper_1104_3349_gb300 import dd
    dd.build()
    w, agg = make_inputs()
    prec = {"fp32": dd.DD_FP32, "fp32_tf32": dd.DD_FP32_TF32}.get(args.prec, dd.DD_FP64)
    P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=prec)
    y = torch.from_numpy(w.b).cuda()
    x = torch.empty_like(y)
    for _ in range(args.apply_only):
        P.apply(y, x)
    torch.cuda.synchronize()
    P.close()


def solve_only(args):
    """One dd_setup on the bench workload, then one FGMRES solve capped at
    args.solve_only iterations, no JSON line (the CGS2 kernel's profiles)."""
    import torch
    from paper_1104_3349_gb300 import dd
    dd.build()
    w, agg = make_inputs()
    prec = {"fp32": dd.DD_FP32, "fp32_tf32": dd.DD_FP32_TF32}.get(args.prec, dd.DD_FP64)
    P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=prec)
    b = torch.from_numpy(w.b).cuda()
    x = torch.empty_like(b)
    P.gmres(b, x, tol=TOL, restart=RESTART, maxit=args.solve_only)
    torch.cuda.synchronize()
    P.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "fp32_tf32"],
                    help="preconditioner precision")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-variants", action="store_true",
                    help="leave out the stretched 512x512 and 64-system batch measurements")
    ap.add_argument("--c3-maxit", type=int, default=300,
                    help="FGMRES iteration cap of the stretched 512x512 measurement")
    ap.add_argument("--c5-maxit", type=int, default=200,
                    help="FGMRES iteration cap of the stretched 1024x1024 learned measurement")
    ap.add_argument("--skip-cfg5", action="store_true", help="leave out the 1024x1024 learned measurement")
    ap.add_argument("--apply-only", type=int, default=0,
                    help="profiling mode: one dd_setup, then this many dd_apply calls, no JSON line")
    ap.add_argument("--solve-only", type=int, default=0,
                    help="profiling mode: one dd_setup, then one solve capped at this many iterations")
    args = ap.parse_args()
    if args.apply_only:
        apply_only(args)
        return
    if args.solve_only:
        solve_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
